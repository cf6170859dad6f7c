"""How well-conditioned ePIE is, measured on the FP64 oracle alone (no GPU).

These facts set the parity protocol of tests/test_gpu_parity.py: FP32
rounding perturbs an FP32 engine's state by about 1e-7 relative, so an FP32
engine can match the FP64 oracle to 1e-5 only where the oracle's own response
to a 1e-7 perturbation stays far below 1e-5.

* From the paper's start (object of ones, phase-free apodised aperture) the
  model far field of the first exit wave decays like a Gaussian and falls
  below FP32 resolution at high frequencies where the measured intensity is
  not small: the replaced phase is then set by rounding, and a single step
  responds to a 1e-7 perturbation at the 1e-3 level.
* From a textured state the step is linear and well-conditioned over short
  chains, but perturbations grow by roughly 8% per dependent step (alpha =
  beta = 1), so a 256-position sequential sweep amplifies any rounding
  difference to the 1e-2 level whatever its size.
"""
import numpy as np
import pytest

from paper_2308_10674_gb300 import synth


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.fixture(scope="module")
def cfg0(orc):
    d = synth.config0(seed=0)
    return d, orc.prepare_intensity(d["frames"]), orc.order_sequential(5, 0, len(d["pos"]))


def response(orc, d, I, order, O0, P0, eps, n_steps):
    Z = np.random.default_rng(1).standard_normal(P0.shape) * (1 + 1j) / np.sqrt(2)
    o = order[:n_steps]
    gs = np.arange(n_steps + 1)
    Oa, Pa = O0.copy(), P0.copy()
    Ob, Pb = O0.copy(), P0 * (1 + eps * Z)
    orc.sweep_groups(Oa, Pa, I, d["pos"], o, gs)
    orc.sweep_groups(Ob, Pb, I, d["pos"], o, gs)
    return rel(Ob, Oa)


def textured(d):
    rng = np.random.default_rng(3)
    O = d["O_true"] * (1 + 0.05 * synth.smooth_field(d["O_true"].shape, 2.0, rng))
    P = d["P_true"] * (1 + 0.05 * synth.smooth_field(d["P_true"].shape, 2.0, rng))
    return O, P


def test_flat_start_first_step_is_ill_conditioned(orc, cfg0):
    d, I, order = cfg0
    r = response(orc, d, I, order, d["O0"].copy(), d["P0"].copy(), 1e-7, 1)
    assert r > 1e-3, r


def test_textured_start_short_chain_is_linear_and_small(orc, cfg0):
    d, I, order = cfg0
    O, P = textured(d)
    r7 = response(orc, d, I, order, O, P, 1e-7, 16)
    r9 = response(orc, d, I, order, O, P, 1e-9, 16)
    assert r7 < 1e-6 and 0.5 < (r7 / 1e-7) / (r9 / 1e-9) < 2.0, (r7, r9)


def test_full_sequential_sweep_amplifies_any_rounding(orc, cfg0):
    d, I, order = cfg0
    O, P = textured(d)
    r10 = response(orc, d, I, order, O, P, 1e-10, 256)
    assert r10 > 1e-3, r10
