"""Graph-replayed sweeps and concurrent multi-scan sweeps (independent scans
of uneven size sharing the GPU): same bits as the plain launch sequence.
Mini-batch sweeps accumulate overlapping object updates with float atomics,
so they reproduce only to rounding (relative 1e-5 here)."""
import numpy as np
import pytest

from paper_2308_10674_gb300 import _binding as B
from paper_2308_10674_gb300 import synth

pytestmark = pytest.mark.gpu


def same(x, y, mode):
    if mode == B.EPIE_MINIBATCH:
        assert np.linalg.norm((x - y).ravel()) <= 1e-5 * np.linalg.norm(y.ravel())
    else:
        assert np.array_equal(x, y)


def run(d, mode, n_sweeps, flags=0, chunks=None, **kw):
    with B.Engine(d["N"], d["H"], d["W"], d["P0"], None, capacity=len(d["pos"]), mode=mode,
                  seed=7, device=0, flags=flags, **kw) as eng:
        errs = []
        if chunks is None:
            eng.append(d["frames"], d["pos"])
            errs = list(eng.iterate(n_sweeps))
        else:
            n = 0
            for c in chunks:
                eng.append(d["frames"][n:n + c], d["pos"][n:n + c])
                n += c
                errs += list(eng.iterate(n_sweeps))
        return eng.object(), eng.probe(), np.array(errs)


@pytest.mark.parametrize("mode,kw", [(B.EPIE_COLOURED, {}), (B.EPIE_MINIBATCH, {"batch": 5}),
                                     (B.EPIE_SEQUENTIAL, {})])
def test_graph_replay_is_bit_identical(mode, kw):
    d = synth.small_scan(64, 5, 6, 20, seed=31)
    a = run(d, mode, 3, chunks=[7, 11, 12], **kw)
    b = run(d, mode, 3, flags=B.EPIE_GRAPH, chunks=[7, 11, 12], **kw)
    for x, y in zip(a, b):
        same(x, y, mode)


def test_graph_replay_with_dark_and_global_max():
    d = synth.small_scan(256, 3, 3, 90, seed=32, dark=True, photons=1e8)
    kw = {"omax_mode": B.EPIE_OMAX_GLOBAL}

    def go(flags):
        with B.Engine(256, d["H"], d["W"], d["P0"], None, capacity=9, mode=B.EPIE_COLOURED,
                      seed=3, device=0, flags=flags, **kw) as eng:
            eng.set_dark(d["dark"])
            eng.append(d["frames"], d["pos"])
            e = eng.iterate(2)
            return eng.object(), eng.probe(), e
    for x, y in zip(go(0), go(B.EPIE_GRAPH)):
        assert np.array_equal(x, y)


def test_iterate_many_matches_separate_runs():
    """Three scans of different frame sizes and modes sweep concurrently."""
    scans = [(synth.small_scan(64, 4, 5, 20, seed=41), B.EPIE_COLOURED, {}),
             (synth.small_scan(128, 3, 4, 40, seed=42), B.EPIE_MINIBATCH, {"batch": 4}),
             (synth.small_scan(256, 3, 3, 90, seed=43), B.EPIE_COLOURED, {})]
    ref = [run(d, m, 2, flags=B.EPIE_GRAPH, **kw) for d, m, kw in scans]
    engs = [B.Engine(d["N"], d["H"], d["W"], d["P0"], None, capacity=len(d["pos"]), mode=m,
                     seed=7, device=0, flags=B.EPIE_GRAPH, **kw) for d, m, kw in scans]
    try:
        for e, (d, _, _) in zip(engs, scans):
            e.append(d["frames"], d["pos"])
        errs = B.epie_iterate_many([e.h for e in engs], 2)
        for i, e in enumerate(engs):
            m = scans[i][1]
            same(e.object(), ref[i][0], m)
            same(e.probe(), ref[i][1], m)
            same(errs[i], ref[i][2], m)
            assert e.sweep_index == 2
    finally:
        for e in engs:
            e.close()
