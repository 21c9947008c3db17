"""Two-sided faces on the GPU (Sec. 5.2.4-5.2.5, App. C) against the CPU oracle:
side-resolved MCRT counts bit for bit (both trace schedules, ragged ray budgets, the
full-size two-sided plates workload on sampled rows), node view factors and view
fractions, side-resolved aggregation, node couplings, and the whole side-resolved chain
(counts -> F -> enforcement -> REFs of the sides -> node couplings)."""
import numpy as np
import pytest
import torch

import synth
from oracle import enforce as OE
from oracle import gebhart as G
from oracle import mcrt
from oracle import multinode as MN
from paper_2511_04277_gb300 import api
from paper_2511_04277_gb300._native import RadgebError

pytestmark = pytest.mark.gpu


def _dev(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x)).to(dtype=dtype, device="cuda")


def stacked_plates(n_sub=1, gap=0.5):
    patches = [((0, 0, k * gap), (1, 0, 0), (0, 1, 0), n_sub, n_sub) for k in range(3)]
    return synth.patch_mesh("stacked_plates", patches, None)


def _gpu_sided(ctx, m, rays, seed, use_bvh=-1, fma_free=True, ray_offset=0):
    mesh = api.Mesh.from_synth(ctx, m, use_bvh=use_bvh)
    c = api.trace_sided(ctx, mesh, rays, seed, ray_offset=ray_offset, fma_free=fma_free)
    torch.cuda.synchronize()
    return c.cpu().numpy(), mesh


@pytest.mark.parametrize("schedule", [2, 3], ids=["lockstep", "refill"])
@pytest.mark.parametrize("mesh", [synth.plates(4), stacked_plates(3), synth.perpendicular_squares(2)],
                         ids=lambda m: m.name)
def test_sided_counts_bit_exact(rg_ctx, mesh, schedule):
    rng = np.random.default_rng(7)
    rays = rng.integers(500, 4000, 2 * mesh.n_faces).astype(np.int64)
    rays[1] = 0                          # a side that does not radiate
    rays[2] = 1
    rays[-1] = 65536 + 33                # two work items, ragged tail
    g, mh = _gpu_sided(rg_ctx, mesh, rays, 21, use_bvh=schedule)
    assert mh.info()["refill"] == (schedule == 3)
    o = mcrt.trace_sided(mesh.verts, mesh.tris, mesh.tri_face, mesh.n_faces, rays, 21)
    assert np.array_equal(g, o)
    assert np.array_equal(g.sum(axis=1), rays)


def test_sided_without_bvh_and_ray_offset(rg_ctx):
    m = synth.cube()
    rays = np.full(12, 20000, np.int64)
    g, mh = _gpu_sided(rg_ctx, m, rays, 5, use_bvh=0, ray_offset=12345)
    assert mh.info()["bvh_nodes"] == 0
    o = mcrt.trace_sided(m.verts, m.tris, m.tri_face, 6, rays, 5, ray_offset=12345, use_bvh=False)
    assert np.array_equal(g, o)
    assert np.all(g[1::2, 12] == 20000) and np.all(g[0::2, 12] == 0)


def test_side_a_rows_sum_to_the_one_sided_rows(rg_ctx):
    m = synth.small_sat()
    rays = np.full(2 * m.n_faces, 500, np.int64)
    mesh = api.Mesh.from_synth(rg_ctx, m)
    c2 = api.trace_sided(rg_ctx, mesh, rays, 3).cpu().numpy()
    c1 = api.trace(rg_ctx, mesh, rays[::2], 3).cpu().numpy()
    N = m.n_faces
    assert np.array_equal(c2[0::2, 0:2 * N:2] + c2[0::2, 1:2 * N:2], c1[:, :N])
    assert np.array_equal(c2[0::2, 2 * N], c1[:, N])
    rows = [1, 2 * 700 + 1, 2 * N - 1]           # side-B rows of the box and a panel
    o = mcrt.trace_sided(m.verts, m.tris, m.tri_face, N, rays, 3, rows=rows)
    for r in rows:
        assert np.array_equal(c2[r], o[r]), r


def test_sided_plates_full_size_sampled_rows(rg_ctx):
    """The two-sided plates workload at its full budget (1e6 rays per side, 1.024e9 rays)
    in the launch configuration the bench times; rows sampled and recomputed one by one."""
    w = synth.workload("plates_sided")
    m = w["mesh"]
    g, _ = _gpu_sided(rg_ctx, m, w["rays"], w["seed"])
    assert np.array_equal(g.sum(axis=1), w["rays"])
    rows = [0, 1, 511, 512, 1023]
    o = mcrt.trace_sided(m.verts, m.tris, m.tri_face, m.n_faces, w["rays"], w["seed"], rows=rows)
    for r in rows:
        assert np.array_equal(g[r], o[r]), r
    assert np.all(g[1:512:2, :1024] == 0)        # the bottom plate's lower sides see only space


def test_sided_refuses_a_triangle_wound_against_its_face(rg_ctx):
    m = synth.plates(1)
    tris = m.tris.copy()
    tris[1] = tris[1][[0, 2, 1]]
    mesh = api.Mesh(rg_ctx, m.verts, tris, m.tri_face, m.n_faces)
    with pytest.raises(RadgebError, match="RG_ERR_ARG"):
        api.trace_sided(rg_ctx, mesh, np.full(4, 10, np.int64), 0)
    api.trace(rg_ctx, mesh, np.full(2, 10, np.int64), 0)   # one-sided tracing still works


def _random_sided(rng, n, C):
    F2 = rng.random((2 * n, 2 * n + 1)) * (rng.random((2 * n, 2 * n + 1)) < 0.7)
    F2[1::2][np.asarray(C) == 1] = 0.0
    F2[2 * 3:2 * 3 + 2, 2 * 5:2 * 5 + 2] = 0.0       # a node pair that exchanges nothing
    return F2


@pytest.mark.parametrize("n", [7, 300, 1029])
def test_node_view_factors_and_fractions(rg_ctx, n):
    rng = np.random.default_rng(n)
    C = rng.integers(1, 3, n).astype(np.int32)
    F2 = _random_sided(rng, n, C)
    Fn, fr = api.node_view_factors(rg_ctx, _dev(F2), _dev(C, torch.int32))
    Fs, Fe = MN.split_sides(F2)
    Fo = MN.node_view_factors(Fs, Fe, C)
    fo, feo = MN.view_fractions(Fs, Fe)
    assert np.abs(Fn.cpu().numpy() - Fo).max() <= 4e-16 * np.abs(Fo).max()
    frg = fr.cpu().numpy()
    fgs, fge = MN.split_sides(frg)
    assert np.abs(fgs - fo).max() <= 1e-15 and np.abs(fge - feo).max() <= 1e-15
    assert np.all(fgs[3, :, 5, :] == 0.0)


def test_node_functions_refuse_a_bad_face_count(rg_ctx):
    n = 4
    F2 = _dev(np.ones((2 * n, 2 * n + 1)))
    with pytest.raises(RadgebError, match="RG_ERR_ARG"):
        api.node_view_factors(rg_ctx, F2, _dev([1, 2, 3, 2], torch.int32))
    with pytest.raises(RadgebError, match="RG_ERR_ARG"):
        api.node_couplings(rg_ctx, F2, _dev(np.full(2 * n, 0.5)), _dev(np.ones(n)), _dev([2, 0, 2, 2], torch.int32))


@pytest.mark.parametrize("n", [9, 515])
def test_node_couplings_against_the_oracle(rg_ctx, n):
    rng = np.random.default_rng(100 + n)
    C = rng.integers(1, 3, n).astype(np.int32)
    B2 = _random_sided(rng, n, C)
    eps2 = rng.uniform(0.1, 0.9, 2 * n)
    S = rng.uniform(0.5, 2.0, n)
    GR, Bn, en = api.node_couplings(rg_ctx, _dev(B2), _dev(eps2), _dev(S), _dev(C, torch.int32))
    GRo, Bno, eno = MN.node_couplings(B2, eps2, S, C)
    assert np.abs(GR.cpu().numpy() - GRo).max() <= 1e-15 * np.abs(GRo).max()
    assert np.abs(Bn.cpu().numpy() - Bno).max() <= 1e-15 * np.abs(Bno).max()
    assert np.abs(en.cpu().numpy() - eno).max() <= 1e-15


def test_sided_aggregation_against_the_oracle(rg_ctx):
    rng = np.random.default_rng(12)
    n_sub, n_surf = 300, 17
    F2 = rng.random((2 * n_sub, 2 * n_sub + 1))
    S = rng.uniform(0.2, 1.0, n_sub)
    grp = rng.integers(0, n_surf, n_sub)
    grp[:n_surf] = np.arange(n_surf)
    Fg, Sg = api.aggregate_sided(rg_ctx, _dev(F2), _dev(S), _dev(grp, torch.int32), n_surf)
    Fo, So = MN.surface_view_factors_sided(F2, S, grp, n_surf)
    assert np.abs(Fg.cpu().numpy() - Fo).max() <= 1e-13 * np.abs(Fo).max()
    assert np.allclose(Sg.cpu().numpy(), So, rtol=1e-14)


def test_sided_chain_to_node_couplings(rg_ctx):
    """Two-faced plates at 1/1000 of the full budget: side-resolved counts -> F of the 1,024
    sides -> iterative enforcement (Omega = S per side) -> REFs of the sides (fp16 tensor
    cores + refinement) -> node couplings, against the same chain in the oracle."""
    w = synth.workload("plates_sided", rays_scale=0.001)
    m = w["mesh"]
    N = m.n_faces
    mesh = api.Mesh.from_synth(rg_ctx, m)
    counts = api.trace_sided(rg_ctx, mesh, w["rays"], w["seed"])
    F2 = api.counts_to_F(rg_ctx, counts, _dev(w["rays"], torch.int64))
    S = mesh.face_areas()
    S2 = np.repeat(S, 2)
    api.enforce_iterative(rg_ctx, F2, _dev(S2), tol=1e-12)
    eps2, rho2 = w["eps"][0], w["rho"][0]
    B2, _, res = api.gebhart(rg_ctx, F2, _dev(eps2), _dev(rho2), precision="fp16", tol=1e-12)
    C = w["faces_per_node"]
    GR, Bn, en = api.node_couplings(rg_ctx, B2[0], _dev(eps2), _dev(S), _dev(C, torch.int32))
    Fn, _ = api.node_view_factors(rg_ctx, F2, _dev(C, torch.int32), fractions=False)

    co = mcrt.trace_sided(m.verts, m.tris, m.tri_face, N, w["rays"], w["seed"])
    assert np.array_equal(counts.cpu().numpy(), co)
    Fo = OE.iterative(co / w["rays"][:, None], S2, tol=1e-12)[0]
    assert np.abs(F2.cpu().numpy() - Fo).max() <= 1e-12
    Bo = G.gebhart(Fo, eps2, rho2)
    Bg = B2[0].cpu().numpy()
    assert (np.abs(Bg - Bo).max(axis=1) / np.abs(Bo).max(axis=1)).max() <= 1e-6
    GRo, Bno, eno = MN.node_couplings(Bo, eps2, S, C)
    assert np.abs(GR.cpu().numpy() - GRo).max() <= 1e-6 * np.abs(GRo).max()
    assert np.abs(Bn.cpu().numpy() - Bno).max() <= 1e-6 * np.abs(Bno).max()
    Fno = MN.node_view_factors(*MN.split_sides(Fo), C)
    assert np.abs(Fn.cpu().numpy() - Fno).max() <= 1e-12
    # node-level closure and reciprocity of the couplings (Eq. C.3 with Eq. 4.3-4.4)
    GRh = GR.cpu().numpy()
    assert np.abs(GRh.sum(axis=1) - S * (eps2[0::2] + eps2[1::2])).max() <= 1e-6 * GRh.max()
    assert np.abs(GRh[:, :N] - GRh[:, :N].T).max() <= 1e-6 * GRh.max()
