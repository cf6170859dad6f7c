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


def test_iterate_many_matches_the_oracle(orc):
    """Concurrent sweeps of three scans (64^2 coloured, 128^2 mini-batch,
    256^2 coloured) from textured starts: each scan's result against the
    FP64 oracle's sweep of that scan alone (state and increment), so the
    concurrency changes nothing."""
    from test_gpu_parity import assert_parity, c64, textured_start
    scans = [(synth.small_scan(64, 4, 5, 20, seed=51), B.EPIE_COLOURED, 0),
             (synth.small_scan(128, 3, 4, 40, seed=52), B.EPIE_MINIBATCH, 4),
             (synth.small_scan(256, 3, 3, 90, seed=53), B.EPIE_COLOURED, 0)]
    refs, starts = [], []
    for d, mode, batch in scans:
        st = textured_start(d)
        starts.append(st)
        O, P = st[0].copy(), st[1].copy()
        I_all = orc.prepare_intensity(d["frames"])
        if mode == B.EPIE_COLOURED:
            col, ncls = orc.colour_greedy(d["pos"], d["N"])
            order, gs = orc.order_coloured(7, 0, col, ncls)
            er, ir = orc.sweep_groups(O, P, I_all, d["pos"], order, gs)
        else:
            order = orc.order_sequential(7, 0, len(d["pos"]))
            er, ir = orc.sweep_minibatch(O, P, I_all, d["pos"], order, batch)
        refs.append((O, P, np.array([er / ir])))
    engs = [B.Engine(d["N"], d["H"], d["W"], st[1], st[0], capacity=len(d["pos"]), mode=m,
                     batch=max(batch, 1), seed=7, device=0, flags=B.EPIE_GRAPH)
            for (d, m, batch), st in zip(scans, starts)]
    try:
        for e, (d, _, _) in zip(engs, scans):
            e.append(d["frames"], d["pos"])
        errs = B.epie_iterate_many([e.h for e in engs], 1)
        for i, e in enumerate(engs):
            O, P, er = refs[i]
            assert_parity(e.object(), e.probe(), errs[i], O, P, er, start=starts[i])
    finally:
        for e in engs:
            e.close()


def test_autotuner_picks_the_measured_best_and_reuses_its_cache(tmp_path, monkeypatch):
    """The tuner times every candidate (tile shapes 1, 2, 4 CTAs per frame at
    128^2, batch sizes, graph replay), returns the fastest of its own table,
    and a second call with the same key is answered from the cache file
    without building a single engine."""
    from paper_2308_10674_gb300 import autotune
    d = synth.scan(128, 256, "jittered", seed=71, photons=1e8)
    cache = str(tmp_path / "tune.json")
    best, table = autotune.tune(d, mode=B.EPIE_MINIBATCH, batches=(64, 256), graph=(True,),
                                sweeps=2, cache_path=cache)
    assert len(table) == 3 * 2
    top = max(table, key=table.get)
    assert top == (f"tile={best['ctas_per_frame']},batch={best['batch']},"
                   f"graph={int(best['graph'])}")

    def no_engine(*a, **k):
        raise AssertionError("the cached answer needs no engine")
    monkeypatch.setattr(B, "Engine", no_engine)
    again, table2 = autotune.tune(d, mode=B.EPIE_MINIBATCH, batches=(64, 256), graph=(True,),
                                  sweeps=2, cache_path=cache)
    assert again == best and table2 == table


@pytest.mark.parametrize("tile", [1, 4])
def test_tile_shapes_at_128_match_the_oracle(orc, tile):
    """The 1- and 4-CTA tile shapes of the 128^2 step kernel give the oracle's
    coloured sweep like the default 2-CTA shape does."""
    from test_gpu_parity import assert_parity, textured_start
    d = synth.small_scan(128, 4, 5, 65, seed=128)
    st = textured_start(d)
    O, P = st[0].copy(), st[1].copy()
    I_all = orc.prepare_intensity(d["frames"])
    col, ncls = orc.colour_greedy(d["pos"], 128)
    order, gs = orc.order_coloured(5, 0, col, ncls)
    er, ir = orc.sweep_groups(O, P, I_all, d["pos"], order, gs)
    with B.Engine(128, d["H"], d["W"], st[1], st[0], capacity=len(d["pos"]),
                  mode=B.EPIE_COLOURED, seed=5, device=0, ctas_per_frame=tile) as eng:
        eng.append(d["frames"], d["pos"])
        e_g = eng.iterate(1)
        assert_parity(eng.object(), eng.probe(), e_g, O, P, np.array([er / ir]), start=st)
