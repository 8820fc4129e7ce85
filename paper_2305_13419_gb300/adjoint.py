"""PyTorch autograd bridge of the discrete adjoint (the gradient of a probe
objective with respect to the material maps, by the transposed time stepping
of Algorithm 1 run on the GPU through `tf_adjoint_run`)."""
from __future__ import annotations

import copy

import torch

from . import twofluid as tf


class ProbePower(torch.autograd.Function):
    """J = |X_k|^2 of a probe DFT after `nsteps` from rest, as a function of
    the per-cell relative permittivity and London depth ([nz][ny][nx]).

    forward(eps_r, lambda_L, workload, nsteps, probe, freq_index, segment)
    runs the forward and the adjoint at once (the adjoint needs the forward
    trajectory, which it recomputes from checkpoints) and keeps the gradients
    for backward."""

    @staticmethod
    def forward(ctx, eps_r, lambda_L, workload, nsteps, probe=0, freq_index=0, segment=256):
        w = copy.copy(workload)
        w.eps_r = eps_r.detach().to("cpu", torch.float32).numpy()
        w.lambda_L = lambda_L.detach().to("cpu", torch.float32).numpy()
        g = tf.Grid.from_workload(w)
        try:
            J, ge, gl = g.adjoint(int(nsteps), int(probe), int(freq_index), int(segment))
        finally:
            g.close()
        ctx.save_for_backward(ge, gl)
        ctx.dtypes = (eps_r.dtype, lambda_L.dtype, eps_r.device, lambda_L.device)
        return torch.tensor(J, dtype=torch.float64, device=eps_r.device)

    @staticmethod
    def backward(ctx, gJ):
        ge, gl = ctx.saved_tensors
        de, dl, ve, vl = ctx.dtypes
        s = gJ.to(torch.float64)
        return ((s * ge.to(torch.float64)).to(ve, de), (s * gl.to(torch.float64)).to(vl, dl),
                None, None, None, None, None)


def probe_power(eps_r, lambda_L, workload, nsteps, probe=0, freq_index=0, segment=256):
    return ProbePower.apply(eps_r, lambda_L, workload, nsteps, probe, freq_index, segment)
