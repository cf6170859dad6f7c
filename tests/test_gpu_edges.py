"""Degenerate and extreme inputs of the step, through the C ABI, against the
FP64 oracle (paper, Sec. "ePIE Implementation": ePIE's projections; the
readings R2 and R4 of the oracle, oracle/epie_oracle.c):

* a probe of zeros: the exit wave and its far field vanish everywhere, so
  every replaced value is sqrt(I) (u(0) = 1), max|P|^2 = 0 turns the object
  update off, and the probe moves to conj(O) F^-1(sqrt I) / max|O|^2;
* frames of zeros: the modulus replacement zeroes the far field, and the
  sweep error is 0 / 0, taken as 0;
* patches at the object's four corners (top-left at (0, 0) and at
  (H - N, W - N)): the loads, stores and bulk copies at the edges;
* one colour class of 169 disjoint 256^2 frames: five waves of clusters in
  one launch."""
import numpy as np
import pytest

from paper_2308_10674_gb300 import _binding as B
from paper_2308_10674_gb300 import synth
from test_gpu_parity import assert_parity, engine, oracle_run, textured_start

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm((np.asarray(a) - b).ravel()) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("N", [64, 256])
def test_zero_probe_one_class(orc, N):
    """Disjoint patches, one colour class: the object stays bit for bit."""
    d = synth.small_scan(N, 2, 2, N + 2, seed=N + 3)
    O0, _ = textured_start(d)
    st = (O0, np.zeros((N, N), complex))
    O, P, e = oracle_run(orc, d, B.EPIE_COLOURED, 1, st)
    assert np.array_equal(O, O0) and np.abs(P).max() > 0  # the reading's consequence
    with engine(d, B.EPIE_COLOURED, st) as eng:
        eng.append(d["frames"], d["pos"])
        assert eng.n_classes == 1
        e_g = eng.iterate(1)
        assert np.array_equal(eng.object(), O0.astype(np.complex64))
        assert rel(eng.probe(), P) <= 1e-5, rel(eng.probe(), P)
        assert abs(e_g[0] - e[0]) <= 1e-6 * e[0]


@pytest.mark.parametrize("N", [64, 256])
def test_zero_probe_overlapping(orc, N):
    """Overlapping patches: the first class moves only the probe, the later
    ones then update both (the oracle's own spread bounds this chain)."""
    d = synth.small_scan(N, 2, 3, N // 2 + 3, seed=N + 6)
    O0, _ = textured_start(d)
    st = (O0, np.zeros((N, N), complex))
    O, P, e = oracle_run(orc, d, B.EPIE_COLOURED, 1, st)
    with engine(d, B.EPIE_COLOURED, st) as eng:
        eng.append(d["frames"], d["pos"])
        assert eng.n_classes > 1
        e_g = eng.iterate(1)
        assert rel(eng.object(), O) <= 1e-5 and rel(eng.probe(), P) <= 1e-5, \
            (rel(eng.object(), O), rel(eng.probe(), P))
        assert abs(e_g[0] - e[0]) <= 1e-6 * e[0]


@pytest.mark.parametrize("N", [64, 256])
def test_zero_frames(orc, N):
    d = synth.small_scan(N, 2, 3, N // 2 + 2, seed=N + 4)
    d = dict(d, frames=np.zeros_like(d["frames"]))
    st = textured_start(d)
    O, P, e = oracle_run(orc, d, B.EPIE_COLOURED, 1, st)
    assert e[0] == 0.0
    with engine(d, B.EPIE_COLOURED, st) as eng:
        eng.append(d["frames"], d["pos"])
        e_g = eng.iterate(1)
        assert e_g[0] == 0.0
        assert_parity(eng.object(), eng.probe(), np.array([0.0]), O, P, np.array([1.0]),
                      tol_e=np.inf, start=st)


@pytest.mark.parametrize("N", [64, 128, 256, 512])
def test_patches_at_the_object_corners(orc, N):
    d = synth.small_scan(N, 3, 3, N // 2, seed=N + 5, margin=0, jitter=0)
    H, W = d["H"], d["W"]
    pos = np.array([[0, 0], [0, W - N], [H - N, 0], [H - N, W - N]], np.int32)
    lam = synth.far_field_intensity(d["O_true"], d["P_true"], pos)
    frames = synth.poisson_u16(lam, np.random.default_rng(N))[0]
    d = dict(d, pos=pos, frames=frames)
    st = textured_start(d)
    O, P, e = oracle_run(orc, d, B.EPIE_COLOURED, 1, st)
    with engine(d, B.EPIE_COLOURED, st) as eng:
        eng.append(d["frames"], d["pos"])
        e_g = eng.iterate(1)
        assert_parity(eng.object(), eng.probe(), e_g, O, P, e, start=st)


def test_one_class_of_169_frames_at_256(orc):
    """13 x 13 raster with a step of N: all 169 patches disjoint, one colour
    class, one launch of 169 clusters (five waves of about 35)."""
    N = 256
    d = synth.small_scan(N, 13, 13, N, seed=77, jitter=0, margin=2, photons=1e7)
    st = textured_start(d)
    O, P, e = oracle_run(orc, d, B.EPIE_COLOURED, 1, st)
    with engine(d, B.EPIE_COLOURED, st) as eng:
        eng.append(d["frames"], d["pos"])
        assert eng.n_classes == 1
        e_g = eng.iterate(1)
        assert_parity(eng.object(), eng.probe(), e_g, O, P, e, start=st)
