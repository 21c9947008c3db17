"""Pins of the side-resolved MCRT oracle (Sec. 5.2.4-5.2.5: factors F^{X->Y} between the
faces A and B of two-sided surfaces) against things other than itself: the one-sided
definition it reduces to on side A, the geometry of each side's rays, closed-form view
factors between parallel and perpendicular squares, exact zeros where a side cannot see
another, exact closure (Eq. 5.30), reciprocity (Eq. 5.34) and brute force == BVH."""
import math

import numpy as np
import pytest

import synth
from oracle import mcrt
from tests import closed_forms as cf


def stacked_plates(n_sub=1, gap=0.5):
    """Three aligned unit squares at z = 0, gap, 2 gap, all with normal +z (side A up)."""
    patches = [((0, 0, k * gap), (1, 0, 0), (0, 1, 0), n_sub, n_sub) for k in range(3)]
    return synth.patch_mesh("stacked_plates", patches, None)


def _sided(m, per, seed=0, use_bvh=True, rows=None):
    rays = np.full(2 * m.n_faces, per, np.int64)
    return mcrt.trace_sided(m.verts, m.tris, m.tri_face, m.n_faces, rays, seed, use_bvh=use_bvh, rows=rows), rays


def _stat_ok(count, ref, n, k=5.0):
    return abs(count / n - ref) <= k * math.sqrt(ref * (1 - ref) / n)


@pytest.mark.parametrize("mesh", [synth.plates(4), synth.perpendicular_squares(2), synth.cube(), stacked_plates(2)],
                         ids=lambda m: m.name)
def test_side_a_rows_are_the_one_sided_rows(mesh):
    # side A emits face f's rays of the one-sided definition; summing its columns over the
    # target side gives the one-sided row (Eq. 5.9: H_ij is the sum over the side pairs)
    c2, rays2 = _sided(mesh, 3000, seed=4)
    c1 = mcrt.trace_counts(mesh.verts, mesh.tris, mesh.tri_face, mesh.n_faces, rays2[::2], 4)
    N = mesh.n_faces
    assert np.array_equal(c2[0::2, 0:2 * N:2] + c2[0::2, 1:2 * N:2], c1[:, :N])
    assert np.array_equal(c2[0::2, 2 * N], c1[:, N])


def test_each_side_emits_from_its_own_side_of_the_face():
    m = synth.small_sat()
    _, frame, _, lift = mcrt.face_geometry(m.verts, m.tris, m.tri_face, m.n_faces)
    f = 777
    n = frame[f, 2].astype(np.float64)
    t = frame[f, 0].astype(np.float64)
    v0 = m.verts[m.tris[np.where(m.tri_face == f)[0][0], 0]].astype(np.float64)
    oA, dA, triA = mcrt.sample_rays_side(m.verts, m.tris, m.tri_face, m.n_faces, f, 0, 9, 0, 20000)
    o1, d1, tri1, _ = mcrt.sample_rays(m.verts, m.tris, m.tri_face, m.n_faces, f, 9, 0, 20000)
    assert np.array_equal(oA, o1) and np.array_equal(dA, d1) and np.array_equal(triA, tri1)
    oB, dB, triB = mcrt.sample_rays_side(m.verts, m.tris, m.tri_face, m.n_faces, f, 1, 9, 0, 20000)
    assert np.all(np.isin(triB, np.where(m.tri_face == f)[0]))
    hA, hB = (oA - v0) @ n, (oB - v0) @ n
    assert np.all(hA > 0) and np.all(hB < 0)                         # lifted off the own side
    assert np.allclose(hB, -lift, rtol=0.2)
    cB = dB.astype(np.float64) @ n
    assert np.all(cB < 0)                                            # leaving through side B
    # cosine-weighted about -n: E|cos| = 2/3, var = 1/18; tangential mean 0, var 1/4
    k = len(cB)
    assert abs(-cB.mean() - 2 / 3) <= 5 * math.sqrt(1 / 18 / k)
    assert abs((dB.astype(np.float64) @ t).mean()) <= 5 * math.sqrt(0.25 / k)
    assert np.allclose(np.linalg.norm(dB, axis=1), 1, atol=1e-6)


def test_parallel_squares_each_side_sees_what_it_faces():
    m = synth.plates(1)             # face 0: z = 0, normal +z; face 1: z = 0.5, normal -z
    per = 200_000
    c, _ = _sided(m, per, seed=1)
    ref = cf.parallel_opposed(1, 1, 0.5)
    # row 0 = bottom A (up), 1 = bottom B (down), 2 = top A (down), 3 = top B (up)
    assert _stat_ok(c[0, 2], ref, per) and _stat_ok(c[2, 0], ref, per)
    assert c[0, [0, 1, 3]].sum() == 0 and c[2, [1, 2, 3]].sum() == 0
    assert c[1, 4] == per and c[3, 4] == per                        # the outer sides see only space
    assert np.all(c.sum(axis=1) == per)                              # Eq. 5.30 on counts


def test_stacked_plates_side_pairs_and_reciprocity():
    m = stacked_plates(1, 0.5)      # faces 0, 1, 2 at z = 0, 0.5, 1, side A up
    per = 200_000
    c, _ = _sided(m, per, seed=2)
    ref = cf.parallel_opposed(1, 1, 0.5)
    # rows/cols: 2f (A, up) and 2f+1 (B, down)
    for src, dst in ((0, 3), (2, 5), (3, 0), (5, 2)):               # bottom A <-> middle B, middle A <-> top B
        assert _stat_ok(c[src, dst], ref, per), (src, dst)
    assert c[1, 6] == per and c[4, 6] == per                        # bottom B and top A see only space
    live = np.zeros_like(c, bool)
    live[[0, 2, 3, 5], [3, 5, 0, 2]] = True
    live[:, 6] = True
    assert np.all(c[~live] == 0)                                    # the middle plate hides the others
    # Eq. 5.34 with equal areas: F^{X->Y}_ij and F^{Y->X}_ji estimate the same number
    F = c / per
    for a, b in ((0, 3), (2, 5)):
        sig = math.sqrt(2 * ref * (1 - ref) / per)
        assert abs(F[a, b] - F[b, a]) <= 5 * sig


def test_perpendicular_squares_back_sides_see_nothing():
    m = synth.perpendicular_squares(1)   # z = 0 (normal +z) and y = 0 (normal +y), common edge
    per = 200_000
    c, _ = _sided(m, per, seed=3)
    ref = cf.perpendicular_common_edge(1, 1, 1)
    assert _stat_ok(c[0, 2], ref, per) and _stat_ok(c[2, 0], ref, per)
    assert c[1, 4] == per and c[3, 4] == per
    assert c[0, [0, 1, 3]].sum() == 0 and c[2, [1, 2, 3]].sum() == 0


def test_closed_cube_inner_sides_keep_every_ray_outer_sides_lose_all():
    m = synth.cube()                 # normals point inward: side A is the inside
    per = 50_000
    c, _ = _sided(m, per, seed=5, use_bvh=False)
    assert np.all(c[0::2, 12] == 0) and np.all(c[0::2, 1:12:2] == 0)  # inside: only inner sides are hit
    assert np.all(c[1::2, 12] == per)                               # outside: everything escapes
    opp = cf.parallel_opposed(1, 1, 1)
    assert _stat_ok(c[0, 2], opp, per) and _stat_ok(c[0, 4], cf.perpendicular_common_edge(1, 1, 1), per)


def test_brute_force_equals_bvh_sided():
    for mesh, per in ((synth.plates(4), 800), (stacked_plates(3), 800), (synth.cube(), 5000)):
        a, _ = _sided(mesh, per, seed=6, use_bvh=False)
        b, _ = _sided(mesh, per, seed=6, use_bvh=True)
        assert np.array_equal(a, b), mesh.name


def test_row_subset_and_ray_ranges():
    m = stacked_plates(2)
    rays = np.full(2 * m.n_faces, 1000, np.int64)
    full = mcrt.trace_sided(m.verts, m.tris, m.tri_face, m.n_faces, rays, 7)
    half = rays // 2
    a = mcrt.trace_sided(m.verts, m.tris, m.tri_face, m.n_faces, half, 7, 0)
    b = mcrt.trace_sided(m.verts, m.tris, m.tri_face, m.n_faces, half, 7, 500)
    assert np.array_equal(full, a + b)
    rows = [1, 6, 17]
    s = mcrt.trace_sided(m.verts, m.tris, m.tri_face, m.n_faces, rays, 7, rows=rows)
    assert np.array_equal(s[rows], full[rows]) and s.sum() == full[rows].sum()


def test_triangle_wound_against_its_face_is_refused():
    m = synth.plates(1)
    tris = m.tris.copy()
    tris[1] = tris[1][[0, 2, 1]]     # second triangle of face 0 flipped
    with pytest.raises(ValueError):
        mcrt.trace_sided(m.verts, tris, m.tri_face, m.n_faces, np.full(4, 10, np.int64), 0)
