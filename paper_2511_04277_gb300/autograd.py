"""torch.autograd wrappers of the REF solve and the steady radiative balance.

Forward passes call rg_gebhart / rg_temperatures; backward passes call the hand-written
adjoints rg_gebhart_adjoint / rg_temperatures_adjoint, which re-solve the transposed
systems on the tensor cores instead of keeping factors (App. B, Eq. B.11 for the REFs;
Eq. 3.13 in steady state for the temperatures). Gradients flow to the optical
properties (eps, rho) and, for the balance, to B; the view factors F, the areas, the
heat loads and the sink temperature are treated as constants, and asking for their
gradients raises.

Composed, ``steady_temperatures`` gives dT/deps and dT/drho for calibrating optical
properties: eps reaches T both through B and directly through the emitted power
sigma eps_i A_i T_i^4, and autograd adds the two contributions.
"""
from __future__ import annotations

import torch

from . import api

SIGMA = 5.67e-8


def _no_grad_for(fn_ctx, names_by_index):
    for i, name in names_by_index.items():
        if fn_ctx.needs_input_grad[i]:
            raise NotImplementedError(f"no gradient with respect to {name}")


class GebhartFunction(torch.autograd.Function):
    """B = REFs of (F, eps, rho); backward gives dL/deps and dL/drho."""

    @staticmethod
    def forward(fn_ctx, rg, F, eps, rho, precision, tol, max_sweeps):
        B, _, _ = api.gebhart(rg, F.detach(), eps.detach().contiguous(), rho.detach().contiguous(), precision,
                              tol, max_sweeps)
        fn_ctx.rg, fn_ctx.precision, fn_ctx.tol, fn_ctx.max_sweeps = rg, precision, tol, max_sweeps
        fn_ctx.save_for_backward(F, eps, rho, B)
        return B

    @staticmethod
    def backward(fn_ctx, dB):
        _no_grad_for(fn_ctx, {1: "F"})
        F, eps, rho, B = fn_ctx.saved_tensors
        deps, drho = api.gebhart_adjoint(fn_ctx.rg, F.detach(), eps.detach().contiguous(),
                                         rho.detach().contiguous(), B, dB.contiguous(), fn_ctx.precision,
                                         fn_ctx.tol, fn_ctx.max_sweeps)
        return None, None, deps.reshape(eps.shape), drho.reshape(rho.shape), None, None, None


class TemperaturesFunction(torch.autograd.Function):
    """T = steady temperatures of (B, eps); backward gives dL/dB and the direct dL/deps."""

    @staticmethod
    def forward(fn_ctx, rg, B, eps, area, Q, T_sink, sigma, precision, tol):
        T = api.temperatures(rg, B.detach().contiguous(), eps.detach().contiguous(), area, Q, T_sink, sigma,
                             precision, tol)
        fn_ctx.rg, fn_ctx.T_sink, fn_ctx.sigma = rg, T_sink, sigma
        fn_ctx.precision, fn_ctx.tol = precision, tol
        fn_ctx.save_for_backward(B, eps, area, T)
        return T

    @staticmethod
    def backward(fn_ctx, dT):
        _no_grad_for(fn_ctx, {3: "area", 4: "Q"})
        B, eps, area, T = fn_ctx.saved_tensors
        dB, deps = api.temperatures_adjoint(fn_ctx.rg, B.detach().contiguous(), eps.detach().contiguous(), area,
                                            fn_ctx.T_sink, T, dT.contiguous(), fn_ctx.sigma, fn_ctx.precision,
                                            fn_ctx.tol)
        return None, dB.reshape(B.shape), deps.reshape(eps.shape), None, None, None, None, None, None


def gebhart(rg: api.Context, F: torch.Tensor, eps: torch.Tensor, rho: torch.Tensor, precision="bf16",
            tol: float = 1e-12, max_sweeps: int = 12) -> torch.Tensor:
    """Differentiable REFs: B [S, N, N+1] for eps, rho of shape [N] or [S, N]."""
    return GebhartFunction.apply(rg, F, eps, rho, precision, tol, max_sweeps)


def temperatures(rg: api.Context, B: torch.Tensor, eps: torch.Tensor, area: torch.Tensor, Q: torch.Tensor,
                 T_sink: float, sigma: float = SIGMA, precision="bf16", tol: float = 1e-13) -> torch.Tensor:
    """Differentiable steady temperatures T [N] from one REF set B [N, N+1]."""
    return TemperaturesFunction.apply(rg, B, eps, area, Q, T_sink, sigma, precision, tol)


def steady_temperatures(rg: api.Context, F: torch.Tensor, eps: torch.Tensor, rho: torch.Tensor,
                        area: torch.Tensor, Q: torch.Tensor, T_sink: float, sigma: float = SIGMA,
                        precision="bf16", tol: float = 1e-12) -> torch.Tensor:
    """T(eps, rho) through the REFs of one optical set: differentiable in eps and rho."""
    B = gebhart(rg, F, eps, rho, precision, tol)
    return temperatures(rg, B[0], eps.reshape(-1), area, Q, T_sink, sigma, precision, min(tol, 1e-13))
