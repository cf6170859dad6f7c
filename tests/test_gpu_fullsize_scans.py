"""Parity at the full sizes of the batched multi-scan workload (eight uneven
scans, FP16 intensity storage, noise-free model intensities; the scans of
bench.py's multiscan leg, generated the same way): the 128^2 and 512^2 step
kernels on the full objects of their scans, through the engine (amplitudes
derived at append, the engine's own colouring and order).

* One whole colour class of the 128^2 spiral scan (9,000 positions; the
  1-CTA kernel and the default 4-CTA shape) and of the 512^2 raster scan
  (1,024 positions), against the FP64 oracle from a
  textured start: one dependent step, so the comparison is sharp, on the
  state, the increment and the sweep error.
* Two mini-batches of 8 overlapping positions of the 512^2 spiral scan (8,000
  positions) on its full object (the float-atomic accumulator, the
  footprint-local apply and the probe mean of a batch).
"""
import os
import sys

import numpy as np
import pytest

from paper_2308_10674_gb300 import _binding as B
from paper_2308_10674_gb300 import synth

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402
from test_gpu_fullsize import check_class_result  # noqa: E402

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm((np.asarray(a) - b).ravel()) / np.linalg.norm(np.ravel(b)))


def multiscan(i):
    N, n, pat, mode = bench.MULTISCAN[i]
    d = synth.scan(N, n, pat, seed=100 + i, noise=False, dtype=np.float16, workers=8)
    rng = np.random.default_rng(3)
    O0 = d["O_true"] * (1 + 0.05 * synth.smooth_field(d["O_true"].shape, 2.0, rng))
    P0 = d["P_true"] * (1 + 0.05 * synth.smooth_field(d["P_true"].shape, 2.0, rng))
    return N, d, O0.astype(np.complex64), P0.astype(np.complex64)


@pytest.mark.parametrize("scan,shape", [(2, 1), (2, 0), (5, 0)])
def test_class_on_the_full_object(orc, scan, shape):
    N, d, O0, P0 = multiscan(scan)
    col, ncls = orc.colour_greedy(d["pos"], N)
    order, gs = orc.order_coloured(5, 0, col, ncls)
    g = int(np.argmax(np.diff(gs)))  # the largest class of the sweep
    sel = order[gs[g]:gs[g + 1]]
    frames, pos = d["frames"][sel], np.ascontiguousarray(d["pos"][sel])
    with B.Engine(N, d["H"], d["W"], P0, O0, capacity=len(sel), mode=B.EPIE_COLOURED, seed=5,
                  device=0, intensity_dtype=B.EPIE_F16, ctas_per_frame=shape) as eng:
        eng.append(frames, pos)
        assert eng.n_classes == 1
        e_g = eng.iterate(1)
        O_g, P_g = eng.object(), eng.probe()
        o_eng, gs_eng = eng.order(0)
    O, P = O0.astype(complex), P0.astype(complex)
    I_all = orc.prepare_intensity(frames)
    er, ir = orc.sweep_groups(O, P, I_all, pos, o_eng, gs_eng)
    check_class_result(O_g, P_g, e_g, O, P, np.array([er / ir]), O0, P0, pos, N=N)


def test_minibatches_on_the_full_512_object(orc):
    N, d, O0, P0 = multiscan(7)
    sel = np.arange(16)  # consecutive spiral positions: overlapping patches
    frames, pos = d["frames"][sel], np.ascontiguousarray(d["pos"][sel])
    with B.Engine(N, d["H"], d["W"], P0, O0, capacity=len(sel), mode=B.EPIE_MINIBATCH, batch=8,
                  seed=5, device=0, intensity_dtype=B.EPIE_F16) as eng:
        eng.append(frames, pos)
        e_g = eng.iterate(1)
        O_g, P_g = eng.object(), eng.probe()
        order = eng.order(0)[0]
    assert np.array_equal(order, orc.order_sequential(5, 0, len(sel)))
    O, P = O0.astype(complex), P0.astype(complex)
    I_all = orc.prepare_intensity(frames)
    er, ir = orc.sweep_minibatch(O, P, I_all, pos, order, 8)
    # float atomics add a batch's object updates in any order: 1e-5 on the
    # state as for every FP32 path, the increment within 1e-4
    assert rel(O_g, O) <= 1e-5 and rel(P_g, P) <= 1e-5, (rel(O_g, O), rel(P_g, P))
    assert rel(O_g - O0, O - O0) <= 1e-4 and rel(P_g - P0, P - P0) <= 1e-4
    assert abs(e_g[0] - er / ir) <= 1e-6 * (er / ir)
