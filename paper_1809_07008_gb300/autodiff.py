"""torch.autograd wrapper of the library's reverse-mode drag gradient (imb_drag_gradient).

``drag_mean(u_in, tau, centres, workload, T)`` builds a lattice from ``workload`` with the given
inlet velocity (x component), relaxation time and disk centres, runs T steps from the workload's
initial state and returns the time-averaged total drag as a 0-d tensor; its backward hands torch
the gradient that the library computed in the same call (adjoint of the pull streaming and of the
collision, checkpointed every ``checkpoint_every`` steps, or by the binomial schedule with
``snapshots`` snapshots when that is given).  Torch only carries the values: every
step, forward and backward, runs in the CUDA library.
"""
from __future__ import annotations

import numpy as np
import torch

from .binding import Lattice


class _DragMean(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u_in, tau, centres, workload, T, checkpoint_every, snapshots):
        w = workload.with_(u_in=(float(u_in), float(workload.u_in[1])), tau=float(tau),
                           x=np.ascontiguousarray(centres.detach().cpu().numpy(), dtype=np.float64))
        lat = Lattice.from_workload(w)
        try:
            J, g_u, g_tau, g_x = lat.drag_gradient(int(T), int(checkpoint_every), snapshots)
        finally:
            lat.close()
        ctx.save_for_backward(torch.tensor(g_u, dtype=torch.float64), torch.tensor(g_tau, dtype=torch.float64),
                              torch.from_numpy(np.array(g_x)))
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        g_u, g_tau, g_x = ctx.saved_tensors
        return gJ * g_u, gJ * g_tau, gJ * g_x, None, None, None, None


def drag_mean(u_in, tau, centres, workload, T, checkpoint_every=100, snapshots=None):
    """Time-averaged drag of ``workload`` over T steps as a differentiable function of the inlet
    velocity, tau and the disk centres (tensors; float64 on the host)."""
    return _DragMean.apply(u_in, tau, centres, workload, T, checkpoint_every, snapshots)
