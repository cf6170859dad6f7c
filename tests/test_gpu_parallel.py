"""The paper's parallel scheme (disjoint subsets iterated independently, then
object and illumination averaged) against the oracle's composition of the
same rounds, from a well-conditioned textured start."""
import numpy as np
import pytest

from paper_2308_10674_gb300 import _binding as B
from paper_2308_10674_gb300 import synth
from paper_2308_10674_gb300.parallel import ParallelAveraging

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm((np.asarray(a) - b).ravel()) / np.linalg.norm(np.ravel(b)))


def test_parallel_averaging_matches_oracle(orc):
    d = synth.small_scan(64, 4, 4, 16, seed=51)
    rng = np.random.default_rng(5)
    subsets = np.array_split(rng.permutation(len(d["pos"])), 4)
    O0 = (d["O_true"] * (1 + 0.05 * synth.smooth_field(d["O_true"].shape, 2.0, rng)))
    P0 = (d["P_true"] * (1 + 0.05 * synth.smooth_field(d["P_true"].shape, 2.0, rng)))
    O0 = O0.astype(np.complex64).astype(complex)
    P0 = P0.astype(np.complex64).astype(complex)
    I_all = orc.prepare_intensity(d["frames"])

    def oracle(p0):
        O, P = O0.copy(), p0.copy()
        orc.run_parallel_average(O, P, I_all, d["pos"], subsets, 2, 2, 64, seed=10)
        return O, P

    O, P = oracle(P0)
    Z = np.random.default_rng(9).standard_normal(P0.shape)
    O2, P2 = oracle(P0 * (1 + 1e-7 * Z))
    assert max(rel(O2, O), rel(P2, P)) <= 1e-6  # well-conditioned instance
    with ParallelAveraging(64, d["H"], d["W"], P0, [d["pos"][s] for s in subsets], object0=O0,
                           seed=10) as par:
        for q, s in enumerate(subsets):
            par.append(q, d["frames"][s], d["pos"][s])
        for _ in range(2):
            par.round(2)
        assert rel(par.object(), O) <= 1e-5 and rel(par.probe(), P) <= 1e-5
        for e in par.engines:  # every subset holds the averaged state
            assert np.array_equal(e.object(), par.object())
