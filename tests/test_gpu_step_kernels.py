"""The 1-CTA 128^2 step kernel (a radix-16 and a radix-8 stage per axis,
transposes through one CTA's shared memory) and the 512^2 step kernel
(16-CTA clusters, a radix-32 and a radix-16 stage per axis) against the FP64
oracle through the C ABI, in every branch they have: derived amplitudes and
raw rows of each intensity type with a dark field, the mini-batch
instantiation, a group larger than one wave, graph replay from the device
group table, and the global object maximum (paper, Sec. "ePIE
Implementation"; readings R4, R5, R7 of the oracle, oracle/epie_oracle.c).  Sharp parity:
one sweep from a textured start, on instances whose oracle moves by less
than 1e-6 under a 1e-7 perturbation of its start probe."""
import numpy as np
import pytest

from paper_2308_10674_gb300 import _binding as B
from paper_2308_10674_gb300 import synth
from test_gpu_parity import (WELL_CONDITIONED, assert_parity, engine, oracle_run, sharp, spread,
                             textured_start)

pytestmark = pytest.mark.gpu

# per frame side: (types: raster ny, nx, step, seed), (graph: step, seed),
# (sequential: step, seed), (mini-batch: step, seed), (one large class: side
# of the disjoint raster, its frames exceed one wave)
# the tile shape each test asks for: the 1-CTA kernel at 128^2 (the default
# 128^2 shape is the general kernel's 4-CTA clusters), the default at 512^2
SHAPE = {128: 1, 512: 0}

INSTANCES = {
    128: dict(types=(1, 3, 75, 21), graph=(65, 128), seq=(50, 25), mb=(50, 23), wave=13),
    512: dict(types=(1, 3, 300, 21), graph=(260, 512), seq=(200, 25), mb=(200, 23), wave=4),
}


@pytest.mark.parametrize("N", [128, 512])
@pytest.mark.parametrize("dtype,code", [(np.uint16, B.EPIE_U16), (np.float16, B.EPIE_F16),
                                        (np.float32, B.EPIE_F32)])
@pytest.mark.parametrize("raw", [False, True])
def test_types_dark_and_raw_rows(orc, N, dtype, code, raw):
    """Overlapping 1 x 3 raster (two classes) with a dark field; the raw path
    converts the staged rows in the kernel, the other copies the amplitudes
    derived at append: both against the oracle."""
    ny, nx, step, seed = INSTANCES[N]["types"]
    d = synth.small_scan(N, ny, nx, step, seed=seed, dark=True, photons=1e7, dtype=dtype)
    st = textured_start(d)
    O, P, e = sharp(orc, d, B.EPIE_COLOURED, st)
    with engine(d, B.EPIE_COLOURED, st, ctas_per_frame=SHAPE[N], intensity_dtype=code,
                flags=B.EPIE_RAW_INTENSITY if raw else 0) as eng:
        eng.set_dark(d["dark"])
        eng.append(d["frames"], d["pos"])
        e_g = eng.iterate(1)
        assert_parity(eng.object(), eng.probe(), e_g, O, P, e, start=st)


@pytest.mark.parametrize("N", [128, 512])
def test_group_larger_than_a_wave(orc, N):
    """A raster with a step of N + 2: disjoint patches, one class with more
    frames than one wave holds (128^2: 169 one-CTA frames on 148-152 SMs;
    512^2: 16 clusters of 16 CTAs, one per SM)."""
    s = INSTANCES[N]["wave"]
    d = synth.small_scan(N, s, s, N + 2, seed=22, jitter=0, margin=2, photons=1e7)
    st = textured_start(d)
    O, P, e = oracle_run(orc, d, B.EPIE_COLOURED, 1, st)
    with engine(d, B.EPIE_COLOURED, st, ctas_per_frame=SHAPE[N]) as eng:
        eng.append(d["frames"], d["pos"])
        assert eng.n_classes == 1
        e_g = eng.iterate(1)
        assert_parity(eng.object(), eng.probe(), e_g, O, P, e, start=st)


@pytest.mark.parametrize("N", [128, 512])
@pytest.mark.parametrize("batch", [2, 4])
def test_minibatch(orc, N, batch):
    step, seed = INSTANCES[N]["mb"]
    d = synth.small_scan(N, 2, 3, step, seed=seed)
    st = textured_start(d)
    I_all = orc.prepare_intensity(d["frames"])
    order = orc.order_sequential(5, 0, len(d["pos"]))

    def run(s0):
        O, P = s0[0].copy(), s0[1].copy()
        er, ir = orc.sweep_minibatch(O, P, I_all, d["pos"], order, batch)
        return O, P, np.array([er / ir])

    (O, P, e), sp = spread(run, st)
    assert max(sp[:2]) <= WELL_CONDITIONED, sp
    with engine(d, B.EPIE_MINIBATCH, st, ctas_per_frame=SHAPE[N], batch=batch) as eng:
        eng.append(d["frames"], d["pos"])
        assert np.array_equal(eng.order(0)[0], order)
        e_g = eng.iterate(1)
        assert_parity(eng.object(), eng.probe(), e_g, O, P, e, start=st)


@pytest.mark.parametrize("N", [128, 512])
def test_graph_replay_and_global_object_max(orc, N):
    """Two sweeps replayed from a CUDA graph (groups read from the device
    table, surplus CTAs exit at once), with max|O|^2 over the object."""
    step, seed = INSTANCES[N]["graph"]
    d = synth.small_scan(N, 2, 3, step, seed=seed)
    st = textured_start(d)
    O, P, e = sharp(orc, d, B.EPIE_COLOURED, st, n_sweeps=2, omax_global=True)
    with engine(d, B.EPIE_COLOURED, st, ctas_per_frame=SHAPE[N], flags=B.EPIE_GRAPH,
                omax_mode=B.EPIE_OMAX_GLOBAL) as eng:
        eng.append(d["frames"], d["pos"])
        e_g = eng.iterate(2)
        assert_parity(eng.object(), eng.probe(), e_g, O, P, e, start=st)


@pytest.mark.parametrize("N", [128, 512])
def test_sequential(orc, N):
    step, seed = INSTANCES[N]["seq"]
    d = synth.small_scan(N, 2, 2, step, seed=seed)
    st = textured_start(d)
    O, P, e = sharp(orc, d, B.EPIE_SEQUENTIAL, st)
    with engine(d, B.EPIE_SEQUENTIAL, st, ctas_per_frame=SHAPE[N]) as eng:
        eng.append(d["frames"], d["pos"])
        e_g = eng.iterate(1)
        assert_parity(eng.object(), eng.probe(), e_g, O, P, e, start=st)
