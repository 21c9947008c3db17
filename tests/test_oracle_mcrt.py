"""Pins of the MCRT oracle (Sec. 3.5.1, Eq. 3.15) against things other than itself:
published Philox known-answer vectors, hand-computed ray/triangle cases, sampling
moments, textbook closed-form view factors, exact closure of a closed enclosure and
brute force == BVH."""
import math

import numpy as np
import pytest

import synth
from oracle import mcrt
from tests import closed_forms as cf
from tests.conftest import load_matrix


# Known-answer vectors published with Random123 (Salmon et al. 2011) for Philox4x32-10.
KAT = [
    ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
]


@pytest.mark.parametrize("ctr,key,expect", KAT)
def test_philox_known_answers(ctr, key, expect):
    assert tuple(int(x) for x in mcrt.philox4x32_10(ctr, key)) == expect


def _one_triangle():
    verts = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    return verts, np.array([[0, 1, 2]], np.int32), np.array([0], np.int32)


def test_ray_triangle_hand_cases():
    v, t, f = _one_triangle()
    o = np.array([[0.25, 0.25, 1.0],    # straight down through the interior: t = 1
                  [0.25, 0.25, 2.0],    # t = 2
                  [0.6, 0.6, 1.0],      # outside (u+v = 1.2)
                  [0.25, 0.25, 1.0],    # parallel to the plane: no hit
                  [0.25, 0.25, -1.0],   # triangle behind the ray: no hit
                  [0.5, 0.5, 1.0],      # on the hypotenuse edge u+v = 1: hit (edge inclusive)
                  [0.0, 0.0, 1.0]], np.float32)  # on a vertex: hit
    d = np.array([[0, 0, -1], [0, 0, -1], [0, 0, -1], [1, 0, 0], [0, 0, -1], [0, 0, -1], [0, 0, -1]],
                 np.float32)
    hit, tt = mcrt.closest_hits(v, t, f, 1, o, d)
    assert hit.tolist() == [0, 0, -1, -1, -1, 0, 0]
    assert tt[0] == 1.0 and tt[1] == 2.0
    # oblique ray: from (0.1, 0.1, 1) along (1, 1, -4)/|.| hits at t = 1/(4/|d|)
    dd = np.array([[1, 1, -4]], np.float32)
    hit, tt = mcrt.closest_hits(v, t, f, 1, np.array([[0.1, 0.1, 1.0]], np.float32), dd)
    assert hit[0] == 0 and abs(float(tt[0]) - 0.25) < 1e-6


def test_closest_hit_and_tie_rule():
    # two parallel triangles at z=0 and z=0.5 and a duplicate of the first one
    verts = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 0.5], [1, 0, 0.5], [0, 1, 0.5]], np.float32)
    tris = np.array([[0, 1, 2], [3, 4, 5], [0, 1, 2]], np.int32)
    tf = np.array([0, 1, 2], np.int32)
    o = np.array([[0.2, 0.2, 1.0]], np.float32)
    d = np.array([[0, 0, -1]], np.float32)
    hit, tt = mcrt.closest_hits(verts, tris, tf, 3, o, d)
    assert hit[0] == 1 and tt[0] == 0.5
    o2 = np.array([[0.2, 0.2, 0.25]], np.float32)
    hit, tt = mcrt.closest_hits(verts, tris, tf, 3, o2, d)
    assert hit[0] == 0  # triangles 0 and 2 tie at t = 0.25: the smaller index wins
    hit, _ = mcrt.closest_hits(verts, tris, tf, 3, o2, d, src_tri=np.array([0], np.int32))
    assert hit[0] == 2  # the source triangle is skipped


def test_sampling_moments():
    """Uniform origins over the face and cosine-weighted directions (diffuse emission)."""
    m = synth.cube()
    n = 200_000
    o, d, tri, att = mcrt.sample_rays(m.verts, m.tris, m.tri_face, m.n_faces, 4, 0, 0, n)  # z=0, normal +z
    lift = np.float32(1e-6 * math.sqrt(3))
    assert np.all(o[:, 2] == lift)             # origins lifted off the face along its normal
    assert abs(o[:, 0].mean() - 0.5) < 4 * math.sqrt(1 / 12 / n)
    assert abs(o[:, 1].mean() - 0.5) < 4 * math.sqrt(1 / 12 / n)
    cz = d[:, 2].astype(np.float64) / np.linalg.norm(d.astype(np.float64), axis=1)
    assert np.all(cz >= 0)
    # cosine-weighted hemisphere: E[cos] = 2/3, Var[cos] = 1/2 - 4/9
    assert abs(cz.mean() - 2 / 3) < 4 * math.sqrt((0.5 - 4 / 9) / n)
    # azimuth uniform: E[d_x] = E[d_y] = 0
    assert abs(d[:, 0].mean()) < 4 * math.sqrt(0.25 / n)
    # both triangles of the face are chosen in proportion to area (1/2 each)
    frac = np.mean(tri == tri.min())
    assert abs(frac - 0.5) < 4 * math.sqrt(0.25 / n)
    assert np.all(att == 0)                    # one draw per ray: no extra direction draws
    # |d| = 1 up to float rounding
    assert np.abs(np.linalg.norm(d.astype(np.float64), axis=1) - 1).max() < 1e-6
    # azimuth uniform over 16 sectors (chi-square, 15 degrees of freedom, p ~ 1e-6 cut)
    phi = np.arctan2(d[:, 1].astype(np.float64), d[:, 0].astype(np.float64))
    hist = np.bincount(((phi + math.pi) / (2 * math.pi) * 16).astype(int) % 16, minlength=16)
    assert ((hist - n / 16) ** 2 / (n / 16)).sum() < 55.0
    # E[cos^2] = 1/2 for a cosine-weighted hemisphere (the radius is sqrt of a uniform)
    assert abs((cz ** 2).mean() - 0.5) < 4 * math.sqrt((1 / 3 - 1 / 4) / n)
    # the direction uses other bits of the draw than the point: no correlation between
    # the origin and the direction components
    for a_ in (o[:, 0], o[:, 1]):
        for b_ in (d[:, 0], d[:, 1], cz):
            assert abs(np.corrcoef(a_.astype(np.float64), b_.astype(np.float64))[0, 1]) < 4 / math.sqrt(n)


def test_face_geometry():
    m = synth.cube()
    area, frame, thr, lift = mcrt.face_geometry(m.verts, m.tris, m.tri_face, m.n_faces)
    assert np.allclose(area, 1.0)
    n = frame[:, 2, :]
    assert np.allclose(n, [[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]])
    # t, b, n orthonormal
    for f in range(6):
        R = frame[f].astype(np.float64)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-6)
    assert abs(lift - 1e-6 * math.sqrt(3)) < 1e-12


def _stat_ok(F, ref, n_rays, k=5.0):
    sigma = math.sqrt(ref * (1 - ref) / n_rays)
    return abs(F - ref) <= k * sigma


def test_cube_closed_forms_and_closure():
    w = synth.workload("cube")
    m = w["mesh"]
    c = mcrt.trace_counts(m.verts, m.tris, m.tri_face, m.n_faces, w["rays"], w["seed"], use_bvh=False)
    assert np.all(c[:, -1] == 0)                         # closed: nothing escapes
    assert np.all(c.sum(axis=1) == w["rays"])            # every ray is counted once
    assert np.all(np.diag(c[:, :6]) == 0)                # planar faces do not see themselves
    F = c / w["rays"][:, None]
    opp = cf.parallel_opposed(1, 1, 1)
    adj = cf.perpendicular_common_edge(1, 1, 1)
    assert abs(opp - 0.199825) < 1e-6 and abs(adj - 0.200044) < 1e-6
    n = int(w["rays"][0])
    pairs_opp = {(0, 1), (2, 3), (4, 5)}
    for i in range(6):
        for j in range(6):
            if i == j:
                continue
            ref = opp if (min(i, j), max(i, j)) in pairs_opp else adj
            assert _stat_ok(F[i, j], ref, n), (i, j, F[i, j], ref)


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_closed_cube_loses_no_ray(seed):
    # rays born within ~1e-7 of an edge hit the adjacent wall at t ~ 1e-7: they must
    # be counted (Sec. 3.5.4: MCRT accounts for every emitted ray)
    m = synth.cube()
    rays = np.full(6, 100_000, np.int64)
    c = mcrt.trace_counts(m.verts, m.tris, m.tri_face, 6, rays, seed, use_bvh=False)
    assert np.all(c[:, -1] == 0)
    assert np.all(c.sum(axis=1) == rays)


def test_brute_force_equals_bvh_bit_exact():
    for mesh, per in ((synth.cube(), 20000), (synth.plates(16), 400), (synth.perpendicular_squares(4), 5000)):
        rays = np.full(mesh.n_faces, per, np.int64)
        a = mcrt.trace_counts(mesh.verts, mesh.tris, mesh.tri_face, mesh.n_faces, rays, 11, use_bvh=False)
        b = mcrt.trace_counts(mesh.verts, mesh.tris, mesh.tri_face, mesh.n_faces, rays, 11, use_bvh=True)
        assert np.array_equal(a, b), mesh.name


def test_brute_force_equals_bvh_small_sat_rows():
    m = synth.small_sat()
    rays = np.full(m.n_faces, 300, np.int64)
    rows = np.arange(0, m.n_faces, 97)
    a = mcrt.trace_counts(m.verts, m.tris, m.tri_face, m.n_faces, rays, 5, use_bvh=False, faces=rows)
    b = mcrt.trace_counts(m.verts, m.tris, m.tri_face, m.n_faces, rays, 5, use_bvh=True, faces=rows)
    assert np.array_equal(a[rows], b[rows])
    assert a[rows].sum() == 300 * len(rows)


def test_counts_are_additive_over_ray_ranges():
    m = synth.plates(4)
    rays = np.full(m.n_faces, 3000, np.int64)
    full = mcrt.trace_counts(m.verts, m.tris, m.tri_face, m.n_faces, rays, 3, 0)
    half = np.full(m.n_faces, 1500, np.int64)
    a = mcrt.trace_counts(m.verts, m.tris, m.tri_face, m.n_faces, half, 3, 0)
    b = mcrt.trace_counts(m.verts, m.tris, m.tri_face, m.n_faces, half, 3, 1500)
    assert np.array_equal(full, a + b)


def test_plates_against_parallel_rectangle_closed_forms():
    m = synth.plates(4)
    per = 40000
    rays = np.full(m.n_faces, per, np.int64)
    c = mcrt.trace_counts(m.verts, m.tris, m.tri_face, m.n_faces, rays, 0)
    F = c / per
    # sub-face (0,0) of the bottom plate: [0,.25]^2 at z=0, faces of the top plate at z=0.5
    top = synth.plates(4)
    for j in range(16, 32):
        tri = np.where(top.tri_face == j)[0]
        xy = top.verts[top.tris[tri].ravel()][:, :2]
        ref = cf.parallel_rectangles(0, 0.25, 0, 0.25, xy[:, 0].min(), xy[:, 0].max(), xy[:, 1].min(),
                                     xy[:, 1].max(), 0.5)
        assert _stat_ok(F[0, j], ref, per), (j, F[0, j], ref)
    assert abs(F[0, :16].sum()) == 0.0


def test_discs_against_eq_6_1():
    m = synth.discs(segments=512)
    per = 400000
    rays = np.full(4, per, np.int64)
    c = mcrt.trace_counts(m.verts, m.tris, m.tri_face, 4, rays, 2)
    F = c / per
    ref = cf.coaxial_discs(1, 2, 1)
    assert abs(ref - (3 - math.sqrt(5))) < 1e-12
    poly = 2 * (2 * math.pi ** 2 / 3) / 512 ** 2   # bound on the polygon-vs-circle area effect
    sigma = math.sqrt(ref * (1 - ref) / per)
    assert abs(F[0, 1] - ref) <= 5 * sigma + poly
    assert F[2, 4] == 1.0 and F[3, 4] == 1.0        # back faces see only the environment


# ------------------------------------------------------------------ diffuse reflections
def test_reflections_with_black_faces_are_the_view_factor_counts():
    # eps = 1, rho = 0: every path ends at its first hit, so the counts are Eq. 3.15's
    m = synth.plates(4)
    rays = np.full(m.n_faces, 3000, np.int64)
    n = m.n_faces
    c0 = mcrt.trace_counts(m.verts, m.tris, m.tri_face, n, rays, 3)
    c1, st = mcrt.trace_reflect(m.verts, m.tris, m.tri_face, n, rays, np.ones(n), np.zeros(n), 3)
    assert np.array_equal(c0, c1)
    assert st["lost"] == 0 and st["overflow"] == 0 and st["rays"] == rays.sum()


def test_reflections_in_a_closed_cube_conserve_every_ray():
    m = synth.cube()
    rays = np.full(6, 20000, np.int64)
    c, st = mcrt.trace_reflect(m.verts, m.tris, m.tri_face, 6, rays, np.full(6, 0.8), np.full(6, 0.2), 1)
    assert np.array_equal(c.sum(axis=1), rays) and np.all(c[:, 6] == 0)
    assert st["lost"] == 0 and st["overflow"] == 0
    # expected hits per path: 1 / eps
    assert abs(st["hits"] / rays.sum() - 1.25) < 0.01


def _within_sigma(counts, rays, B, k=5.0):
    Bh = counts / rays[:, None]
    sig = np.sqrt(np.maximum(B * (1 - B), 1e-12) / rays[:, None])
    return np.abs(Bh - B) <= k * sig


def test_reflections_estimate_the_gebhart_factors_of_the_cube():
    # closed-form cube view factors -> fp64 REFs (Eq. B.5) -> the random walk's expectation
    from oracle import gebhart as G
    opp, adj = cf.parallel_opposed(1, 1, 1), cf.perpendicular_common_edge(1, 1, 1)
    F = np.full((6, 7), adj)
    F[:, 6] = 0.0
    for i in range(6):
        F[i, i] = 0.0
        F[i, i ^ 1] = opp
    eps = np.array([0.9, 0.3, 0.6, 0.8, 0.5, 0.7])
    B = G.gebhart(F, eps, 1 - eps)
    m = synth.cube()
    rays = np.full(6, 200000, np.int64)
    c, _ = mcrt.trace_reflect(m.verts, m.tris, m.tri_face, 6, rays, eps, 1 - eps, 2)
    assert np.all(_within_sigma(c, rays, B))


def test_reflections_reproduce_the_printed_parallel_plate_refs():
    # Sec. 6.3: eps = 0.5 on every face; the plates are set at the distance whose exact
    # view factor is the printed F_23 = 0.285913 (Eq. 6.10), so the walk's expectation is
    # the printed B (Eq. 6.11) up to its 6 decimals
    from scipy.optimize import brentq
    gap = brentq(lambda h: cf.parallel_opposed(1, 1, h) - 0.285913, 0.2, 5.0)
    m = synth.two_sided_plates(gap=gap)
    rays = np.full(4, 400000, np.int64)
    c, st = mcrt.trace_reflect(m.verts, m.tris, m.tri_face, 4, rays, np.full(4, 0.5), np.full(4, 0.5), 5)
    Bp = load_matrix("plates_B.txt")
    Bh = c / rays[:, None]
    sig = np.sqrt(np.maximum(Bp * (1 - Bp), 1e-12) / rays[:, None])
    assert np.all(np.abs(Bh - Bp) <= 5 * sig + 1e-6)
    assert np.all(c[[0, 3], :4] == 0)           # the outer sides only see the environment


def test_unit_circle_of_the_sampling():
    """The direction's cos and sin of 2 pi t 2^-24 (quadrant, fold to [0, pi/4], Taylor
    polynomials in float) against the fp64 library functions, for every one of the 2^24
    angles: within a few float ulps, on the unit circle, and exact at the quadrant
    boundaries."""
    n = 1 << 24
    c, s = mcrt.unit_circle(0, n)
    phi = 2 * np.pi * np.arange(n, dtype=np.float64) / n
    assert np.abs(c - np.cos(phi)).max() < 3e-7
    assert np.abs(s - np.sin(phi)).max() < 3e-7
    assert np.abs(c.astype(np.float64) ** 2 + s.astype(np.float64) ** 2 - 1).max() < 6e-7
    q = np.arange(4) << 22
    assert c[q].tolist() == [1.0, 0.0, -1.0, 0.0] and s[q].tolist() == [0.0, 1.0, 0.0, -1.0]
    with pytest.raises(ValueError):
        mcrt.unit_circle(n - 1, 2)
