"""Live mode with a feeder thread (paper, Sec. "Live ePIE": one thread
appends the frames as they arrive while another keeps iterating on the
frames present).  A feeder thread appends chunks while the main thread runs
epie_iterate(n); each sweep covers the frames present when it started, which
the handle reports per sweep (epie_last_sweep_frames).  Replaying those
counts sweep by sweep - on a second handle without threads, and on the FP64
oracle - gives the threaded run's result."""
import threading
import time

import numpy as np
import pytest

from paper_2308_10674_gb300 import _binding as B
from paper_2308_10674_gb300 import synth

pytestmark = pytest.mark.gpu

CHUNK, N_SWEEPS, EVERY = 4, 160, 8
# relative size of the perturbation that enters the oracle's state after
# every sweep in the spread estimate: the rounding of one FP32 2-D transform
# of K = N^2 points, about u log2(K) with u = 2^-24 (7e-7 at 64^2); a
# perturbation of one FP32 ulp (1e-7) underestimates the engine's per-sweep
# rounding by that factor of log2(K)
SWEEP_ROUNDING = 1e-6


def rel(a, b):
    return float(np.linalg.norm((np.asarray(a) - b).ravel()) / np.linalg.norm(np.ravel(b)))


def c64(a):
    return np.asarray(a).astype(np.complex64).astype(np.complex128)


def test_feeder_thread_appends_while_iterating(orc):
    d = synth.small_scan(64, 4, 4, 33, seed=12)
    n = len(d["pos"])
    rng = np.random.default_rng(3)
    O0 = c64(d["O_true"] * (1 + 0.05 * synth.smooth_field(d["O_true"].shape, 2.0, rng)))
    P0 = c64(d["P_true"] * (1 + 0.05 * synth.smooth_field(d["P_true"].shape, 2.0, rng)))

    def engine(flags=0):
        return B.Engine(64, d["H"], d["W"], P0, O0, capacity=n, mode=B.EPIE_COLOURED, seed=5,
                        device=0, flags=flags)

    errors = []
    # EPIE_CHECKED makes every sweep wait for its own result, so the sweeps of
    # the iterating thread run at the GPU's pace and the feeder (a Python
    # thread polling every few tens of microseconds) always finds boundaries
    # to slip in at; it changes no arithmetic
    with engine(B.EPIE_CHECKED) as eng:
        eng.append(d["frames"][:CHUNK], d["pos"][:CHUNK])

        def feeder():
            try:
                for k in range(1, n // CHUNK):
                    # the next chunk arrives once the iterating thread has queued
                    # k*EVERY sweeps (reading the index takes the handle's mutex
                    # between two sweeps, as the append does)
                    t0 = time.time()
                    while eng.sweep_index < k * EVERY and time.time() - t0 < 30:
                        time.sleep(2e-5)
                    a = k * CHUNK
                    eng.append(d["frames"][a:a + CHUNK], d["pos"][a:a + CHUNK])
            except Exception as ex:  # reported by the main thread
                errors.append(ex)

        # the feeder polls the sweep index before the sweeps start, so its
        # start-up latency does not race them
        th = threading.Thread(target=feeder)
        th.start()
        time.sleep(0.05)
        e_g = eng.iterate(N_SWEEPS)
        th.join()
        assert not errors, errors
        counts = eng.last_sweep_frames()
        O_g, P_g = eng.object(), eng.probe()
    # every sweep saw a whole number of chunks, never fewer than the sweep before
    assert len(counts) == N_SWEEPS and counts[0] == CHUNK
    assert np.all(counts % CHUNK == 0) and np.all(np.diff(counts) >= 0) and counts.max() <= n
    assert len(np.unique(counts)) >= 2, counts  # at least one chunk joined mid-call

    # replay on a second handle without threads: bit for bit
    with engine() as ref:
        have = 0
        e_r = []
        for c in counts:
            if c > have:
                ref.append(d["frames"][have:c], d["pos"][have:c])
                have = c
            e_r += list(ref.iterate(1))
        assert np.array_equal(ref.object(), O_g) and np.array_equal(ref.probe(), P_g)
        assert np.array_equal(np.array(e_r), e_g)

    # replay on the oracle: the colouring of the frames present, the sweep's
    # order, one coloured sweep each.  A chain of 160 sweeps is compared
    # within 3x the oracle's own spread when relative perturbations of the
    # size of the engine's per-sweep rounding (SWEEP_ROUNDING) enter its state
    # after every sweep
    I_all = orc.prepare_intensity(d["frames"])

    def run(start, noise_seed=None):
        O, P = start[0].copy(), start[1].copy()
        rng = None if noise_seed is None else np.random.default_rng(noise_seed)
        es = []
        for s, c in enumerate(counts):
            col, ncls = orc.colour_greedy(d["pos"][:c], 64)
            order, gs = orc.order_coloured(5, s, col, ncls)
            er, ir = orc.sweep_groups(O, P, I_all, d["pos"], order, gs)
            es.append(er / ir)
            if rng is not None:
                O *= 1 + SWEEP_ROUNDING * rng.standard_normal(O.shape)
                P *= 1 + SWEEP_ROUNDING * rng.standard_normal(P.shape)
        return O, P, np.array(es)

    O, P, e = run((O0, P0))
    sp = [0.0, 0.0, 0.0]
    for k in range(2):
        O2, P2, e2 = run((O0, P0), noise_seed=100 + k)
        sp = [max(sp[0], rel(O2, O)), max(sp[1], rel(P2, P)),
              max(sp[2], float(np.max(np.abs(e2 - e) / e)))]
    assert rel(O_g, O) <= 3 * sp[0] + 1e-5, (rel(O_g, O), sp)
    assert rel(P_g, P) <= 3 * sp[1] + 1e-5, (rel(P_g, P), sp)
    assert np.max(np.abs(e_g - e) / e) <= 3 * sp[2] + 1e-6, sp
