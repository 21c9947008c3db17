"""GPU enforcement and aggregation (rg_enforce_iterative, rg_aggregate) against the oracle."""
import numpy as np
import pytest
import torch

import synth
from oracle import enforce as E
from oracle import mcrt
from oracle import multinode as MN
from paper_2511_04277_gb300 import api
from tests.conftest import load_matrix

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _dev(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x)).to(dtype=dtype, device="cuda")


def _random_F(N, rng, zeros=0.2):
    F = rng.random((N, N + 1))
    F[rng.random((N, N + 1)) < zeros] = 0.0
    np.fill_diagonal(F[:, :N], 0.0)
    F[:, N] += 0.05
    return F / F.sum(axis=1, keepdims=True)


def test_iterative_disc_example(rg_ctx):
    F1 = load_matrix("disc_F1_mcrt.txt")
    A = np.array([1.0, 4.0, 1.0, 4.0])
    Fd = _dev(F1)
    it = api.enforce_iterative(rg_ctx, Fd, _dev(A), tol=TOL)
    Fo, it_o, _ = E.iterative(F1, A, tol=TOL)
    got = Fd.cpu().numpy()
    assert np.abs(got - Fo).max() <= 1e-14
    assert abs(it - it_o) <= 1
    assert np.abs(got - load_matrix("disc_F6_iterative.txt")).max() <= 1e-6


@pytest.mark.parametrize("N", [1, 63, 64, 65, 200, 2048])
def test_iterative_random_sizes(rg_ctx, N):
    rng = np.random.default_rng(N)
    F = _random_F(N, rng)
    A = rng.uniform(0.5, 2.0, N)
    Fd = _dev(F)
    it = api.enforce_iterative(rg_ctx, Fd, _dev(A), tol=TOL)
    Fo, it_o, ok = E.iterative(F, A, tol=TOL)
    assert ok and abs(it - it_o) <= 1
    got = Fd.cpu().numpy()
    # row-normwise: max_j |F - F_ref| <= 1e-6 max_j |F_ref| (here far tighter)
    assert np.all(np.abs(got - Fo).max(axis=1) <= 1e-10 * np.abs(Fo).max(axis=1))


def test_iterative_not_converged_is_reported(rg_ctx):
    rng = np.random.default_rng(3)
    F = _random_F(50, rng)
    A = rng.uniform(0.5, 2.0, 50)
    Fd = _dev(F)
    with pytest.raises(api.RadgebError) as e:
        api.enforce_iterative(rg_ctx, Fd, _dev(A), tol=0.0, maxit=3)
    assert e.value.code == "RG_ERR_NOT_CONVERGED"
    Fo, _, _ = E.iterative(F, A, tol=0.0, maxit=3)
    assert np.abs(Fd.cpu().numpy() - Fo).max() < 1e-13   # holds the last iterate


def test_iterative_on_plates_mcrt(rg_ctx):
    """Config-sized: 512 sub-faces from GPU counts, enforced on the GPU and by the oracle."""
    m = synth.plates(16)
    rays = np.full(m.n_faces, 20000, np.int64)
    mesh = api.Mesh.from_synth(rg_ctx, m)
    c = api.trace(rg_ctx, mesh, rays, 0)
    F = api.counts_to_F(rg_ctx, c, _dev(rays, torch.int64))
    F0 = F.cpu().numpy()
    A = mesh.face_areas()
    api.enforce_iterative(rg_ctx, F, _dev(A), tol=TOL)
    Fo, _, _ = E.iterative(F0, A, tol=TOL)
    got = F.cpu().numpy()
    assert np.all(np.abs(got - Fo).max(axis=1) <= 1e-10 * np.abs(Fo).max(axis=1))
    assert np.abs(got.sum(axis=1) - 1).max() < 1e-13
    eta = A[:, None] * got[:, :512]
    assert np.abs(eta - eta.T).max() < 1e-11


def test_aggregate_plates(rg_ctx):
    m = synth.plates(16)
    rays = np.full(m.n_faces, 20000, np.int64)
    mesh = api.Mesh.from_synth(rg_ctx, m)
    F = api.counts_to_F(rg_ctx, api.trace(rg_ctx, mesh, rays, 0), _dev(rays, torch.int64))
    A = mesh.face_areas()
    api.enforce_iterative(rg_ctx, F, _dev(A))
    grp = m.patch_of_face.astype(np.int32)
    Fg, Sg = api.aggregate(rg_ctx, F, _dev(A), _dev(grp, torch.int32), 2)
    Fo, So = MN.surface_view_factors(F.cpu().numpy(), A, grp, 2)
    assert np.abs(Fg.cpu().numpy() - Fo).max() <= 1e-13
    assert np.abs(Sg.cpu().numpy() - So).max() <= 1e-13
    # whole plates: closed form 0.415253, within the MCRT error of 5.12e6 rays
    assert abs(Fo[0, 1] - 0.415253) < 1e-3


@pytest.mark.parametrize("N,G", [(37, 5), (300, 300), (1000, 17)])
def test_aggregate_random(rg_ctx, N, G):
    rng = np.random.default_rng(N + G)
    F = _random_F(N, rng)
    S = rng.uniform(0.5, 2.0, N)
    grp = rng.integers(0, G, N).astype(np.int32)
    grp[:G] = np.arange(G)
    Fg, _ = api.aggregate(rg_ctx, _dev(F), _dev(S), _dev(grp, torch.int32), G)
    Fo, _ = MN.surface_view_factors(F, S, grp, G)
    assert np.abs(Fg.cpu().numpy() - Fo).max() <= 1e-13


def test_aggregate_rejects_bad_group(rg_ctx):
    F = _random_F(8, np.random.default_rng(0))
    grp = np.array([0, 1, 2, 3, 0, 1, 2, 9], np.int32)
    with pytest.raises(api.RadgebError):
        api.aggregate(rg_ctx, _dev(F), _dev(np.ones(8)), _dev(grp, torch.int32), 4)
