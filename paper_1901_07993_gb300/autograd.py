"""torch.autograd.Function over the hand-written adjoint of the refinement.

`RefineLoss.apply(S_val, S_row_ptr, S_col_idx, n, bs, F, K, tau, ctx)` returns
L = tr(Z_K^T F Z_K) after K frozen-pattern refinement sweeps (see
inv_factor_refine_adjoint in include/ifac.h) as a 0-d CUDA tensor; backward
gives dL/dS_val.  The C ABI computes L and dL/dS in one call (the recording
run is the forward pass and its tape feeds the reverse pass), so forward
already holds the gradient that backward scales.  Marshalling only: all
arithmetic runs in libifac.so.
"""
from __future__ import annotations

import torch

from . import ifac


class RefineLoss(torch.autograd.Function):
    @staticmethod
    def forward(fctx, S_val, S_row_ptr, S_col_idx, n: int, bs: int, F, K: int, tau: float, lib_ctx):
        S = ifac.BorrowedBSR(n, bs, S_row_ptr, S_col_idx, S_val.contiguous())
        L, Sbar = ifac.inv_factor_refine_adjoint(lib_ctx, S, F, K, tau)
        _, _, g = ifac.device_tensors(Sbar)
        fctx.save_for_backward(g.clone())
        return torch.tensor(L, dtype=torch.float64, device=S_val.device)

    @staticmethod
    def backward(fctx, grad_out):
        (g,) = fctx.saved_tensors
        return grad_out * g, None, None, None, None, None, None, None, None
