"""torch.autograd binding of the library's hand-written adjoint (mg_adjoint).

``gibbs_loss(logP, d, sampler, chain, K, w)`` returns the scalar
L = sum_j w_j |s_hat_K,j|^2 of K fixed-P sweeps (P = exp(logP), the chain's next
K noise draws held fixed, data d), as a torch FP64 tensor whose backward
supplies dL/dlogP and dL/dd from the CUDA adjoint.  The forward call itself runs
the adjoint too (one call computes the loss and both gradients).
"""
from __future__ import annotations

import numpy as np
import torch


class GibbsAdjoint(torch.autograd.Function):
    @staticmethod
    def forward(ctx, logP, d, sampler, chain, K, w, group):
        sampler.set_data(group, d.detach().to("cpu", torch.float64).numpy())
        L, gl, gd = sampler.adjoint(chain, K, logP.detach().to("cpu", torch.float64).numpy(), np.asarray(w))
        ctx.save_for_backward(torch.as_tensor(gl).to(logP.device, logP.dtype),
                              torch.as_tensor(gd).reshape(d.shape).to(d.device, d.dtype))
        return torch.tensor(L, dtype=torch.float64, device=logP.device)

    @staticmethod
    def backward(ctx, gout):
        gl, gd = ctx.saved_tensors
        return gout.to(gl.dtype) * gl, gout.to(gd.dtype) * gd, None, None, None, None, None


def gibbs_loss(logP, d, sampler, chain: int, K: int, w, group: int = 0):
    return GibbsAdjoint.apply(logP, d, sampler, chain, K, w, group)
