"""Discrete energy of the FP32 GPU step.  With sigma = 0 the scheme conserves
W^n = 1/2 sum eps_e E^2 + 1/2 sum B^{n-1/2} B^{n+1/2} / mu_f
      + 1/2 sum_{kappa > 0} Js^{n-1/2} Js^{n+1/2} / kappa_e
exactly (Algorithm 1: the Yee curls are mutual transposes); with theta = 1/2
it loses exactly dt sum sigma_e ((E^n + E^{n+1}) / 2)^2 per step.  The GPU
fields are read at integer levels through the C ABI and the energy is formed
with the oracle's edge and face coefficients."""
import numpy as np
import pytest

from oracle import stepper
from paper_2305_13419_gb300 import workloads as W
from test_oracle_pins import _energy

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


class _GpuFields:
    """GPU state seen through the oracle's coefficient getters."""

    def __init__(self, gpu, orc):
        self.gpu, self.orc = gpu, orc
        self.d, self.dt = orc.d, orc.dt

    def field(self, c):
        return self.gpu.field(c).astype(np.float64)

    def coeff(self, kind, c):
        return self.orc.coeff(kind, c)


def _pair(w, seed):
    from paper_2305_13419_gb300 import twofluid as tf
    g = tf.Grid.from_workload(w)
    o = stepper.Grid.from_workload(w)
    assert abs(g.dt / o.dt - 1) < 1e-15
    st = W.random_state(seed, w.storage_dims())
    for c in range(9):
        g.set_field(c, st[c].astype(np.float32))
    return g, o


def test_fp32_step_conserves_the_discrete_energy():
    w = W.random_box(n=(40, 33, 44), seed=21, theta=0.5, sigma_range=(0, 0), mu_range=(1, 2),
                     bc=("periodic",) * 3)
    g, o = _pair(w, 7)
    view = _GpuFields(g, o)
    w0 = _energy(view)
    drift = []
    for _ in range(8):
        g.step(500)
        g.sync()
        drift.append(abs(_energy(view) / w0 - 1))
    assert max(drift) < 1e-5, drift


def test_fp32_step_ohmic_balance_theta_half():
    w = W.random_box(n=(24, 20, 28), seed=22, theta=0.5, sigma_range=(0, 5e5), mu_range=(1, 1.5),
                     bc=("periodic",) * 3)
    g, o = _pair(w, 8)
    view = _GpuFields(g, o)
    sig = [o.coeff(1, c) for c in range(3)]
    w_prev = _energy(view)
    e_prev = [view.field(c) for c in range(3)]
    for _ in range(5):
        g.step(1)
        g.sync()
        w_now = _energy(view)
        e_now = [view.field(c) for c in range(3)]
        loss = g.dt * sum(np.sum(sig[c] * (0.5 * (e_prev[c] + e_now[c])) ** 2) for c in range(3))
        assert loss > 0
        assert abs((w_prev - w_now) / loss - 1) < 1e-3
        w_prev, e_prev = w_now, e_now
