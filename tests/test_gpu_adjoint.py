"""GPU discrete adjoint (FP32, through the C ABI) against the FP64 oracle's
adjoint, which is itself pinned by dot-product tests and central
differences; checkpoint-segment independence; the autograd bridge."""
import numpy as np
import pytest

from oracle import stepper
from paper_2305_13419_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

PROBE = (12, 7, 8)
N0 = 20


def _workload():
    """The scaled CPW-like box of the oracle's finite-difference test: CPML on
    all faces, random substrate eps_r, a superconducting Ohmic film, a soft
    source above it, one probe (FP32-representable maps)."""
    n = (20, 14, 16)
    w = W.random_box(n=n, bc=("cpml", "cpml", "cpml"), seed=77, cpml_cells=3, theta=1.0,
                     sc_fraction=0.0, sigma_range=(0.0, 0.0), eps_range=(1.0, 1.0), mu_range=(1.0, 1.0))
    rng = np.random.default_rng(2305_13419 + 40)
    w.eps_r = np.asarray(w.eps_r, np.float32).copy()
    w.lambda_L = np.asarray(w.lambda_L, np.float32).copy()
    w.sigma = np.asarray(w.sigma, np.float32).copy()
    w.eps_r[:7] = rng.uniform(10.0, 13.0, size=(7, 14, 20))
    w.lambda_L[7:9] = rng.uniform(2.0, 6.0, size=(2, 14, 20)) * 12e-9
    w.sigma[7:9] = np.random.default_rng(2305_13419 + 4).uniform(0.0, 1e6, size=(2, 14, 20))
    f = 6e13
    w.sources = [W.Source(comp=1, lo=(6, 5, 9), hi=(8, 8, 10), amp=1.0e3, kind=W.SRC_GAUSS_SIN, f=f,
                          t0=4 / (2 * f), tw=1 / (2 * f))]
    w.probes = [W.Probe(comp=1, p=PROBE, freqs=np.array([f]), n0=N0)]
    return w, f


def _oracle(w, nsteps, f):
    o = stepper.Grid.from_workload(w, with_probes=False)
    return o.adjoint_run(nsteps, 1, PROBE, f, N0)


def test_gpu_adjoint_matches_oracle_adjoint():
    from paper_2305_13419_gb300 import twofluid as tf
    w, f = _workload()
    nsteps = 160
    Jo, geo, glo = _oracle(w, nsteps, f)
    g = tf.Grid.from_workload(w)
    J, ge, gl = g.adjoint(nsteps, 0, 0, segment=48)
    ge, gl = ge.cpu().numpy().astype(np.float64), gl.cpu().numpy().astype(np.float64)
    assert abs(J / Jo - 1) < 1e-3
    for go, gg in ((geo, ge), (glo, gl)):
        big = np.max(np.abs(go))
        m = np.abs(go) >= 1e-3 * big
        assert m.sum() > 50
        rel = np.abs(gg[m] / go[m] - 1)
        assert np.max(rel) < 1e-3, np.max(rel)
        assert np.max(np.abs(gg[~m] - go[~m])) < 2e-6 * big


def test_segments_do_not_change_the_gradient():
    from paper_2305_13419_gb300 import twofluid as tf
    w, f = _workload()
    a = tf.Grid.from_workload(w).adjoint(90, 0, 0, segment=7)
    b = tf.Grid.from_workload(w).adjoint(90, 0, 0, segment=1000)
    assert a[0] == b[0]
    assert torch.equal(a[1], b[1]) and torch.equal(a[2], b[2])


def test_handle_ends_where_the_forward_run_ends():
    from paper_2305_13419_gb300 import twofluid as tf
    w, f = _workload()
    g = tf.Grid.from_workload(w)
    g.adjoint(70, 0, 0, segment=16)
    h = tf.Grid.from_workload(w)
    h.step(70)
    assert g.level == 70
    for c in range(9):
        assert np.array_equal(g.field(c), h.field(c))
    assert np.array_equal(g.probe_dft(0), h.probe_dft(0))


def test_autograd_bridge():
    from paper_2305_13419_gb300 import adjoint
    from paper_2305_13419_gb300 import twofluid as tf
    w, f = _workload()
    eps = torch.tensor(w.eps_r, dtype=torch.float64, device="cuda", requires_grad=True)
    lam = torch.tensor(w.lambda_L, dtype=torch.float64, device="cuda", requires_grad=True)
    J = adjoint.probe_power(eps, lam, w, 60, segment=32)
    (3.0 * J).backward()
    J2, ge, gl = tf.Grid.from_workload(w).adjoint(60, 0, 0, segment=32)
    assert float(J.detach()) == J2
    assert torch.allclose(eps.grad, 3.0 * ge.to(torch.float64), rtol=0, atol=0)
    assert torch.allclose(lam.grad, 3.0 * gl.to(torch.float64), rtol=0, atol=0)


def test_adjoint_rejects_bad_calls():
    from paper_2305_13419_gb300 import twofluid as tf
    w, f = _workload()
    g = tf.Grid.from_workload(w)
    g.step(1)
    with pytest.raises(tf.TFError) as ex:     # not at rest any more
        g.adjoint(10)
    assert ex.value.status == tf.TF_ESTATE
    with pytest.raises(tf.TFError) as ex:
        tf.Grid.from_workload(w).adjoint(10, probe=3)
    assert ex.value.status == tf.TF_EINVAL
