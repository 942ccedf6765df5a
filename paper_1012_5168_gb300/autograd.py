"""torch.autograd.Function for the local loop L_Gamma(t) = sum_{x in t} eta^dag Gamma M^{-1} eta.

Forward: phi = M^{-1} eta by the CUDA solver, then the loop contraction
(Sec. 3, Eq. 2) for all 16 Gamma.  Backward uses one adjoint solve per
right-hand side, with M^dagger = gamma_5 M gamma_5:

  with g = dloss/dconj(L) (PyTorch's convention for complex outputs),
  chi    = M^{-dagger} sum_{Gamma,t} g_{Gamma,t} Gamma^dagger P_t eta,
  grad_eta   = chi + sum_{Gamma,t} conj(g_{Gamma,t}) Gamma P_t phi,
  grad_kappa = Re sum_j chi_j^dagger (-dM/dkappa) phi_j   (dM^{-1}/dkappa = -M^{-1} (dM/dkappa) M^{-1}),

with -dM/dkappa = D for the Wilson matrix and D + c_sw sum sigma F with the
clover term.

Every arithmetic step runs in the library's kernels (solve, adjoint solve,
Gamma-weighted spin matrices, -dM/dkappa, contraction); this module only
passes tensors between them.
"""

from __future__ import annotations

import numpy as np
import torch

from . import Context, Params, SINK_LOCAL


class LoopTrace(torch.autograd.Function):
    """L = LoopTrace.apply(eta, kappa, ctx, params) -> complex128 [n, 16, T] on eta's device."""

    @staticmethod
    def forward(fctx, eta: torch.Tensor, kappa: torch.Tensor, ctx: Context, params: Params | None = None):
        ctx.set_kappa(float(kappa.detach().cpu()))
        eta = eta.detach().contiguous()
        phi, _ = ctx.solve(eta, params)
        L = ctx.trace_loops(eta, phi, SINK_LOCAL)[:, 0]
        fctx.save_for_backward(eta, phi, kappa)
        fctx.dl = ctx
        fctx.params = params
        return torch.from_numpy(L).to(eta.device)

    @staticmethod
    def backward(fctx, g: torch.Tensor):
        eta, phi, kappa = fctx.saved_tensors
        ctx: Context = fctx.dl
        ctx.set_kappa(float(kappa.detach().cpu()))
        w = np.ascontiguousarray(g.detach().to(torch.complex128).cpu().numpy())
        src = ctx.apply_gamma_weights(eta, w, mode=0)
        chi, _ = ctx.solve_adjoint(src, fctx.params)
        grad_kappa = None
        if fctx.needs_input_grad[1]:
            dphi = ctx.apply_dm_dkappa(phi)
            tr = ctx.trace_loops(chi, dphi, SINK_LOCAL, sum_rhs=True, sum_t=True)  # sum_j chi_j^dag (-dM/dk) phi_j
            grad_kappa = torch.tensor(float(tr[0, 0, 0, 0].real), dtype=kappa.dtype, device=kappa.device)
        grad_eta = None
        if fctx.needs_input_grad[0]:
            grad_eta = ctx.apply_gamma_weights(phi, w, mode=1, out=chi, accumulate=True)
        return grad_eta, grad_kappa, None, None


def loop_trace(eta: torch.Tensor, kappa: torch.Tensor, ctx: Context, params: Params | None = None) -> torch.Tensor:
    return LoopTrace.apply(eta, kappa, ctx, params)
