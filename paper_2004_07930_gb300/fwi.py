"""Frequency-domain FWI misfit as a differentiable function of the model.

The paper's solver is the forward engine of full-waveform inversion (Sec.
"Introduction"). `Misfit.apply(m, ...)` returns the least-squares receiver
misfit chi(m) for per-element squared slowness m (a torch float64 tensor);
its backward pass returns grad_output * dchi/dm, computed by the library's
adjoint-state kernels (one forward and one adjoint solve per source on the
device, hz_fwi_gradient). Every evaluation factors A(m) afresh (hz_setup).
"""
from __future__ import annotations

import numpy as np
import torch

from . import hz


def misfit_and_gradient(prob, m, src_xyz, rec_xyz, d_obs=None, options=None):
    """(chi, grad [ne], d_syn [ns, nr], stats) for the model m = 1/c^2 on
    the mesh, partition and frequency of `prob` (a workloads problem)."""
    m = np.asarray(m, dtype=np.float64)
    p = dict(prob)
    p["velocity"] = 1.0 / np.sqrt(m)
    with hz.Solver.from_problem(p, options=options) as S:
        return S.fwi_gradient(src_xyz, rec_xyz, d_obs)


def synthetic_data(prob, m, src_xyz, rec_xyz, options=None):
    """Receiver data P u_s [ns, nr] for the model m."""
    return misfit_and_gradient(prob, m, src_xyz, rec_xyz, None, options)[2]


class Misfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, prob, src_xyz, rec_xyz, d_obs, options=None):
        chi, g, _, _ = misfit_and_gradient(prob, m.detach().cpu().numpy(), src_xyz, rec_xyz, d_obs, options)
        ctx.save_for_backward(torch.from_numpy(g).to(m.device))
        return torch.tensor(chi, dtype=torch.float64, device=m.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None, None, None, None, None
