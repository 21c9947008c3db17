"""Dense solves in a caller-owned workspace (the boundary's ownership rule: the caller owns
every device buffer). On a fresh context, every dense-solve call run with a workspace of
the queried size gives the same bits as the context-workspace call and leaves the context
holding no workspace; a short or misaligned workspace is refused."""
import numpy as np
import pytest
import torch

from paper_2511_04277_gb300 import api
from paper_2511_04277_gb300._native import RadgebError

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _system(N, S, rng):
    F = rng.random((N, N + 1)) * (1.0 / N)
    np.fill_diagonal(F[:, :N], 0.0)
    F[:, N] = 0.0
    F[:, N] = 1.0 - F.sum(axis=1)
    A = rng.uniform(0.5, 2.0, N)
    eps = rng.uniform(0.05, 0.9, (S, N))
    return F, A, eps, 1 - eps


def test_solves_in_a_caller_workspace(rg_ctx):
    rng = np.random.default_rng(9)
    N, S = 700, 2
    F, A, eps, rho = _system(N, S, rng)
    Fd, Ad, ed, rd = _dev(F), _dev(A), _dev(eps), _dev(rho)
    api.enforce_iterative(rg_ctx, Fd, Ad, tol=1e-12)
    Q = _dev(rng.uniform(0, 50, (S, N)))
    wT = _dev(rng.standard_normal((S, N)))
    # references through the shared context's own workspace
    B0, _, _ = api.gebhart(rg_ctx, Fd, ed, rd, tol=1e-12)
    T0 = api.temperatures_sets(rg_ctx, Fd, B0, ed, rd, Ad, Q, 3.0, tol=1e-13)
    (fa0, fb0), de_T0 = api.temperatures_adjoint_sets(rg_ctx, Fd, B0, ed, rd, Ad, 3.0, T0, wT, tol=1e-13,
                                                      factored=True)
    de0, dr0 = api.gebhart_adjoint_factored(rg_ctx, Fd, ed, rd, B0, fa0, fb0, tol=1e-12)
    dB0 = torch.einsum("srn,srm->snm", fa0, fb0).contiguous()
    de1_0, dr1_0 = api.gebhart_adjoint(rg_ctx, Fd, ed, rd, B0, dB0, tol=1e-12)
    T1_0 = api.temperatures(rg_ctx, B0[0], ed[0], Ad, Q[0], 3.0, tol=1e-13)
    Fl0 = Fd.clone()
    api.enforce_lsq(rg_ctx, Fl0, Ad)

    ctx = api.Context(0)
    try:
        def ws(kind, **kw):
            nbytes = api.solver_workspace(kind, N, **kw)
            return torch.empty(nbytes, dtype=torch.uint8, device="cuda")

        gb = api.gebhart_workspace(N, S, "bf16")
        B, _, _ = api.gebhart(ctx, Fd, ed, rd, tol=1e-12, ws=torch.empty(gb, dtype=torch.uint8, device="cuda"))
        assert torch.equal(B, B0)
        T = api.temperatures_sets(ctx, Fd, B, ed, rd, Ad, Q, 3.0, tol=1e-13, ws=ws("temperatures_sets"))
        assert torch.equal(T, T0)
        (fa, fb), de_T = api.temperatures_adjoint_sets(ctx, Fd, B, ed, rd, Ad, 3.0, T, wT, tol=1e-13, factored=True,
                                                       ws=ws("temperatures_sets"))
        assert torch.equal(fa, fa0) and torch.equal(fb, fb0) and torch.equal(de_T, de_T0)
        de, dr = api.gebhart_adjoint_factored(ctx, Fd, ed, rd, B, fa, fb, tol=1e-12,
                                              ws=ws("gebhart_adjoint_factored", rank=2))
        assert torch.equal(de, de0) and torch.equal(dr, dr0)
        de1, dr1 = api.gebhart_adjoint(ctx, Fd, ed, rd, B, dB0, tol=1e-12, ws=ws("gebhart_adjoint"))
        assert torch.equal(de1, de1_0) and torch.equal(dr1, dr1_0)
        T1 = api.temperatures(ctx, B[0], ed[0], Ad, Q[0], 3.0, tol=1e-13, ws=ws("temperatures"))
        assert torch.equal(T1, T1_0)
        Fl = Fd.clone()
        api.enforce_lsq(ctx, Fl, Ad, ws=ws("enforce_lsq"))
        assert torch.equal(Fl, Fl0)
        # nothing above touched the context's own workspace
        assert api.workspace_bytes(ctx) == 0
        # a workspace one byte short, and a misaligned one, are refused
        short = torch.empty(gb - 1, dtype=torch.uint8, device="cuda")
        with pytest.raises(RadgebError) as e:
            api.gebhart(ctx, Fd, ed, rd, tol=1e-12, ws=short)
        assert e.value.code == "RG_ERR_ARG"
        big = torch.empty(gb + 512, dtype=torch.uint8, device="cuda")
        with pytest.raises(RadgebError) as e:
            api.gebhart(ctx, Fd, ed, rd, tol=1e-12, ws=big[16:])
        assert e.value.code == "RG_ERR_ARG"
        assert api.workspace_bytes(ctx) == 0
        # without a caller workspace the context grows its own
        api.gebhart(ctx, Fd, ed, rd, tol=1e-12)
        assert api.workspace_bytes(ctx) >= gb
    finally:
        ctx.close()
