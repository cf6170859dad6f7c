"""CUDA engine vs the FP64 oracle, element by element, through the C ABI.

Two kinds of parity, because ePIE with alpha = beta = 1 amplifies rounding:
a perturbation of relative size 1e-7 grows by about 8% per dependent step and
saturates near 1e-2 after a 256-position sequential sweep, in the FP64
oracle itself (tests/test_conditioning.py pins this).

* Sharp parity: from a textured start state (the true object and probe with
  5% smooth perturbations) over chains of at most ~16 dependent steps, the
  oracle is well-conditioned (checked in each test: a 1e-7 perturbation of
  its start probe moves its result by < 1e-6), and the engine must match it
  to relative L2 <= 1e-5 on object and probe, <= 1e-6 on the sweep error.
* Conditioning-relative parity: from the paper's flat start and over full
  sweeps, the engine must lie within 3x the oracle's own spread under 1e-7
  perturbations (plus 1e-5).

Integer work (colour classes, visiting orders) is compared bit for bit, and
two engine runs on the same inputs are bit-identical (fixed-order reductions).
"""
import os

import numpy as np
import pytest

from paper_2308_10674_gb300 import _binding as B
from paper_2308_10674_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_STATE = 1e-5
TOL_ERR = 1e-6
# increments X - X0 of a sharp test (one sweep, or a few short chained ones,
# from a textured start): the FP32 transforms round at about
# u log2(N^2) |psi| with u = 6e-8, and a sweep moves the state by 1-10% of
# its size, so the increment carries a relative error of up to ~2e-5; 1e-4
# leaves a margin of about 5 (the values the suite reports are in the design
# notes)
TOL_INC = 1e-4
WELL_CONDITIONED = 1e-6


def rel(a, b):
    return float(np.linalg.norm((np.asarray(a) - b).ravel()) / np.linalg.norm(np.ravel(b)))


def c64(a):
    return np.asarray(a).astype(np.complex64).astype(np.complex128)


def flat_start(d):
    """The paper's start: object of ones, phase-free aperture probe."""
    return c64(d["O0"]), c64(d["P0"])


def textured_start(d, seed=3):
    rng = np.random.default_rng(seed)
    O = d["O_true"] * (1 + 0.05 * synth.smooth_field(d["O_true"].shape, 2.0, rng))
    P = d["P_true"] * (1 + 0.05 * synth.smooth_field(d["P_true"].shape, 2.0, rng))
    return c64(O), c64(P)


def engine(d, mode, start, seed=5, cap=None, **kw):
    O0, P0 = start
    return B.Engine(d["N"], d["H"], d["W"], P0, O0, capacity=cap or len(d["pos"]),
                    mode=mode, seed=seed, device=0, **kw)


def oracle_run(orc, d, mode, n_sweeps, start, seed=5, frames=None, pos=None, **kw):
    O, P = start[0].copy(), start[1].copy()
    frames = d["frames"] if frames is None else frames
    pos = d["pos"] if pos is None else pos
    I_all = orc.prepare_intensity(frames, d.get("dark"))
    errs = orc.run_sweeps(O, P, I_all, pos, n_sweeps, d["N"], seed=seed,
                          mode=orc.SEQUENTIAL if mode == B.EPIE_SEQUENTIAL else orc.COLOURED, **kw)
    return O, P, np.array(errs)


def spread(run, start, eps=1e-7, samples=2):
    """The oracle's own sensitivity: max relative change of (O, P, E) when its
    start probe is perturbed by eps (FP32 rounding size)."""
    O, P, e = run(start)
    out = [0.0, 0.0, 0.0]
    for k in range(samples):
        rng = np.random.default_rng(100 + k)
        Z = rng.standard_normal(start[1].shape) + 1j * rng.standard_normal(start[1].shape)
        O2, P2, e2 = run((start[0], start[1] * (1 + eps * Z)))
        out = [max(out[0], rel(O2, O)), max(out[1], rel(P2, P)),
               max(out[2], float(np.max(np.abs(e2 - e) / np.abs(e))))]
    return (O, P, e), out


def increment_errors(O_g, P_g, O, P, start):
    """Relative L2 error of what the run changed: (X_gpu - X0) against
    (X_ref - X0) for X in {O, P}, X0 the start state."""
    O0, P0 = start
    return rel(np.asarray(O_g) - O0, O - O0), rel(np.asarray(P_g) - P0, P - P0)


def assert_parity(O_g, P_g, e_g, O, P, e, tol=TOL_STATE, tol_e=TOL_ERR, start=None,
                  tol_inc=TOL_INC):
    """State parity (relative L2 on O, P and the sweep errors) and, given the
    start state, parity of the increments X - X0 that the sweeps produced."""
    ro, rp = rel(O_g, O), rel(P_g, P)
    re = float(np.max(np.abs(np.asarray(e_g) - e) / np.abs(e)))
    inc = increment_errors(O_g, P_g, O, P, start) if start is not None else (0.0, 0.0)
    if os.environ.get("EPIE_PARITY_REPORT"):
        print(f"parity state O {ro:.2e} P {rp:.2e} E {re:.2e} increment O {inc[0]:.2e} "
              f"P {inc[1]:.2e}")
    assert ro <= tol and rp <= tol and re <= tol_e, (ro, rp, re)
    assert inc[0] <= tol_inc and inc[1] <= tol_inc, ("increment", inc)


def sharp(orc, d, mode, start, n_sweeps=1, seed=5, **kw):
    """Oracle reference plus the well-conditioning guard of a sharp test."""
    (O, P, e), sp = spread(lambda st: oracle_run(orc, d, mode, n_sweeps, st, seed, **kw), start)
    assert max(sp[:2]) <= WELL_CONDITIONED, ("instance not well-conditioned", sp)
    return O, P, e


# --------------------------------------------------------------------------- sequential (config 0)

def test_sequential_short_chain_sharp(orc):
    """Config-0 data (64x64, 1e6 photons, Poisson uint16), the first 16
    positions in sequential order from a textured start: 1e-5."""
    d = synth.config0(seed=0)
    d = dict(d, frames=d["frames"][:16], pos=d["pos"][:16])
    st = textured_start(d)
    O, P, e = sharp(orc, d, B.EPIE_SEQUENTIAL, st)
    with engine(d, B.EPIE_SEQUENTIAL, st) as eng:
        eng.append(d["frames"], d["pos"])
        order, gs = eng.order(0)
        assert np.array_equal(order, orc.order_sequential(5, 0, 16))
        assert np.array_equal(gs, np.arange(17))
        e_g = eng.iterate(1)
        assert_parity(eng.object(), eng.probe(), e_g, O, P, e, start=st)


@pytest.mark.parametrize("n_sweeps", [1, 10])
def test_config0_flat_start_within_conditioning(orc, n_sweeps):
    """Config 0 in full (256 positions, flat start, 1 and 10 sweeps): the
    engine lies within 3x the oracle's own spread under 1e-7 perturbations."""
    d = synth.config0(seed=0)
    st = flat_start(d)
    (O, P, e), sp = spread(lambda s0: oracle_run(orc, d, B.EPIE_SEQUENTIAL, n_sweeps, s0), st)
    with engine(d, B.EPIE_SEQUENTIAL, st) as eng:
        eng.append(d["frames"], d["pos"])
        e_g = eng.iterate(n_sweeps)
        O_g, P_g = eng.object(), eng.probe()
    assert rel(O_g, O) <= 3 * sp[0] + 1e-5, (rel(O_g, O), sp)
    assert rel(P_g, P) <= 3 * sp[1] + 1e-5, (rel(P_g, P), sp)
    assert np.max(np.abs(e_g - e) / e) <= 3 * sp[2] + 1e-6, (e_g, e, sp)
    if n_sweeps > 1:
        assert e_g[-1] < e_g[0]


def test_runs_are_bit_identical():
    """Fixed-order reductions: the same inputs give the same bits."""
    d = synth.small_scan(256, 3, 3, 120, seed=21)
    outs = []
    for _ in range(2):
        with engine(d, B.EPIE_COLOURED, flat_start(d)) as eng:
            eng.append(d["frames"], d["pos"])
            e = eng.iterate(2)
            outs.append((eng.object(), eng.probe(), e))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    assert np.array_equal(outs[0][2], outs[1][2])


# --------------------------------------------------------------------------- coloured, all frame sizes

CASES = [(64, 5, 7, 33), (128, 4, 5, 65), (256, 3, 4, 130), (512, 2, 3, 260)]


@pytest.mark.parametrize("N,ny,nx,step", CASES)
@pytest.mark.parametrize("path", [B.EPIE_PATH_FUSED, B.EPIE_PATH_PLAIN])
def test_coloured_one_sweep(orc, N, ny, nx, step, path):
    """Raster scans with overlapping patches (four colour classes of uneven
    size) at every supported frame size, fused and plain paths."""
    d = synth.small_scan(N, ny, nx, step, seed=N)
    st = textured_start(d)
    O, P, e = sharp(orc, d, B.EPIE_COLOURED, st)
    with engine(d, B.EPIE_COLOURED, st, path=path) as eng:
        eng.append(d["frames"], d["pos"])
        col, ncls = orc.colour_greedy(d["pos"], N)
        assert np.array_equal(eng.colours(), col) and eng.n_classes == ncls
        order, gs = eng.order(0)
        o_ref, gs_ref = orc.order_coloured(5, 0, col, ncls)
        assert np.array_equal(order, o_ref) and np.array_equal(gs, gs_ref)
        assert ncls > 1 and np.diff(gs).max() > 1
        e_g = eng.iterate(1)
        assert_parity(eng.object(), eng.probe(), e_g, O, P, e, start=st)


def test_coloured_with_class_cap(orc):
    """Capped first-fit colouring (at most 3 frames per class): same classes,
    order and result as the oracle's capped colouring."""
    d = synth.small_scan(64, 5, 7, 33, seed=64)
    st = textured_start(d)
    O, P, e = sharp(orc, d, B.EPIE_COLOURED, st, class_cap=3)
    with engine(d, B.EPIE_COLOURED, st, class_cap=3) as eng:
        eng.append(d["frames"], d["pos"])
        col, ncls = orc.colour_greedy(d["pos"], 64, cap=3)
        assert np.array_equal(eng.colours(), col) and eng.n_classes == ncls
        assert np.bincount(col).max() == 3
        e_g = eng.iterate(1)
        assert_parity(eng.object(), eng.probe(), e_g, O, P, e, start=st)


@pytest.mark.parametrize("N", [64, 256])
def test_sequential_plain_path(orc, N):
    d = synth.small_scan(N, 3, 3, N // 3, seed=7)
    st = textured_start(d)
    O, P, e = sharp(orc, d, B.EPIE_SEQUENTIAL, st)
    with engine(d, B.EPIE_SEQUENTIAL, st, path=B.EPIE_PATH_PLAIN) as eng:
        eng.append(d["frames"], d["pos"])
        e_g = eng.iterate(1)
        assert_parity(eng.object(), eng.probe(), e_g, O, P, e, start=st)


# --------------------------------------------------------------------------- intensity types, dark field

@pytest.mark.parametrize("dtype,code", [(np.float16, B.EPIE_F16), (np.float32, B.EPIE_F32)])
def test_intensity_types(orc, dtype, code):
    d = synth.small_scan(128, 3, 4, 65, seed=2, dtype=dtype)
    st = textured_start(d)
    O, P, e = sharp(orc, d, B.EPIE_COLOURED, st)
    with engine(d, B.EPIE_COLOURED, st, intensity_dtype=code) as eng:
        eng.append(d["frames"], d["pos"])
        e_g = eng.iterate(1)
        assert_parity(eng.object(), eng.probe(), e_g, O, P, e, start=st)


@pytest.mark.parametrize("path", [B.EPIE_PATH_FUSED, B.EPIE_PATH_PLAIN])
def test_dark_field(orc, path):
    d = synth.small_scan(256, 2, 3, 130, seed=6, dark=True, photons=1e7)
    st = textured_start(d)
    O, P, e = sharp(orc, d, B.EPIE_COLOURED, st)
    with engine(d, B.EPIE_COLOURED, st, path=path) as eng:
        eng.set_dark(d["dark"])
        eng.append(d["frames"], d["pos"])
        e_g = eng.iterate(1)
        assert_parity(eng.object(), eng.probe(), e_g, O, P, e, start=st)


# --------------------------------------------------------------------------- update variants

def test_global_object_max(orc):
    d = synth.small_scan(64, 4, 4, 33, seed=8)
    st = textured_start(d)
    O, P, e = sharp(orc, d, B.EPIE_COLOURED, st, omax_global=True)
    with engine(d, B.EPIE_COLOURED, st, omax_mode=B.EPIE_OMAX_GLOBAL) as eng:
        eng.append(d["frames"], d["pos"])
        e_g = eng.iterate(1)
        assert_parity(eng.object(), eng.probe(), e_g, O, P, e, start=st)


def test_probe_sum_flag(orc):
    d = synth.small_scan(64, 4, 4, 33, seed=9)
    st = textured_start(d)
    O, P, e = sharp(orc, d, B.EPIE_COLOURED, st, beta=0.25, probe_mean=False)
    with engine(d, B.EPIE_COLOURED, st, flags=B.EPIE_PROBE_SUM, beta=0.25) as eng:
        eng.append(d["frames"], d["pos"])
        e_g = eng.iterate(1)
        assert_parity(eng.object(), eng.probe(), e_g, O, P, e, start=st)


@pytest.mark.parametrize("path", [B.EPIE_PATH_FUSED, B.EPIE_PATH_PLAIN])
@pytest.mark.parametrize("batch", [1, 5, 16])
def test_minibatch(orc, path, batch):
    d = synth.small_scan(64, 3, 4, 10, seed=11)
    st = textured_start(d)
    I_all = orc.prepare_intensity(d["frames"])
    order = orc.order_sequential(5, 0, len(d["pos"]))

    def run(s0):
        O, P = s0[0].copy(), s0[1].copy()
        er, ir = orc.sweep_minibatch(O, P, I_all, d["pos"], order, batch)
        return O, P, np.array([er / ir])

    (O, P, e), sp = spread(run, st)
    assert max(sp[:2]) <= WELL_CONDITIONED, sp
    with engine(d, B.EPIE_MINIBATCH, st, path=path, batch=batch) as eng:
        eng.append(d["frames"], d["pos"])
        assert np.array_equal(eng.order(0)[0], order)
        e_g = eng.iterate(1)
        assert_parity(eng.object(), eng.probe(), e_g, O, P, e, start=st)


# --------------------------------------------------------------------------- live mode

def test_live_append_between_sweeps(orc):
    """Frames arrive in chunks between sweeps (paper, Sec. "Live ePIE"); each
    sweep covers the frames present when it starts."""
    d = synth.small_scan(64, 4, 4, 33, seed=12)
    chunks = [3, 4, 9]  # cumulative counts 3, 7, 16
    st = textured_start(d)
    I_all = orc.prepare_intensity(d["frames"])

    def run(s0):
        O, P = s0[0].copy(), s0[1].copy()
        e, n, s = [], 0, 0
        for c in chunks:
            n += c
            col, ncls = orc.colour_greedy(d["pos"][:n], 64)
            order, gs = orc.order_coloured(5, s, col, ncls)
            er, ir = orc.sweep_groups(O, P, I_all, d["pos"], order, gs)
            e.append(er / ir)
            s += 1
        return O, P, np.array(e)

    (O, P, e), sp = spread(run, st)
    assert max(sp[:2]) <= WELL_CONDITIONED, sp
    with engine(d, B.EPIE_COLOURED, st) as eng:
        e_g, n = [], 0
        for c in chunks:
            eng.append(d["frames"][n:n + c], d["pos"][n:n + c])
            n += c
            e_g += list(eng.iterate(1))
        assert_parity(eng.object(), eng.probe(), e_g, O, P, e, start=st)


def test_truncate_reverts_to_prefix():
    d = synth.small_scan(64, 4, 5, 9, seed=13)
    st = flat_start(d)
    with engine(d, B.EPIE_COLOURED, st) as a, engine(d, B.EPIE_COLOURED, st) as b:
        a.append(d["frames"], d["pos"])
        a.truncate(12)
        b.append(d["frames"][:12], d["pos"][:12])
        assert a.n_frames == 12 and a.n_classes == b.n_classes
        assert np.array_equal(a.colours(), b.colours())
        a.iterate(1)
        b.iterate(1)
        assert np.array_equal(a.object(), b.object()) and np.array_equal(a.probe(), b.probe())


def test_resume_equals_continuous_run():
    """Export, re-import into a new handle with the sweep index, continue:
    identical to an uninterrupted run."""
    d = synth.small_scan(64, 3, 4, 12, seed=14)
    st = flat_start(d)
    with engine(d, B.EPIE_COLOURED, st) as a:
        a.append(d["frames"], d["pos"])
        a.iterate(3)
        Oa, Pa = a.object(), a.probe()
    with engine(d, B.EPIE_COLOURED, st) as b:
        b.append(d["frames"], d["pos"])
        b.iterate(1)
        O1, P1, s1 = b.object(), b.probe(), b.sweep_index
    with engine(d, B.EPIE_COLOURED, st) as c:
        c.append(d["frames"], d["pos"])
        c.set_object(O1)
        c.set_probe(P1)
        c.sweep_index = s1
        c.iterate(2)
        assert np.array_equal(c.object(), Oa) and np.array_equal(c.probe(), Pa)


def test_untouched_pixels_stay_exactly_one():
    """Object pixels no patch covers keep the initial value 1 bit for bit
    (paper, Discussion)."""
    d = synth.small_scan(64, 3, 3, 30, seed=15, margin=20)
    with engine(d, B.EPIE_COLOURED, flat_start(d)) as eng:
        eng.append(d["frames"], d["pos"])
        eng.iterate(3)
        O_g = eng.object()
    cover = np.zeros(O_g.shape, bool)
    for y, x in d["pos"]:
        cover[y:y + 64, x:x + 64] = True
    assert (~cover).sum() > 0 and np.all(O_g[~cover] == 1.0)


def test_empty_sweep_and_errors():
    d = synth.small_scan(64, 2, 2, 16, seed=16)
    st = flat_start(d)
    with engine(d, B.EPIE_COLOURED, st, cap=4) as eng:
        e = eng.iterate(2)
        assert np.all(e == 0.0)
        assert np.array_equal(eng.probe(), d["P0"].astype(np.complex64))
        with pytest.raises(B.EpieError) as ex:
            eng.append(d["frames"][:1], np.array([[d["H"] - 63, 0]], np.int32))
        assert ex.value.code == B.EPIE_ERANGE and eng.n_frames == 0
        eng.append(d["frames"], d["pos"])
        with pytest.raises(B.EpieError) as ex:
            eng.append(d["frames"][:1], d["pos"][:1])
        assert ex.value.code == B.EPIE_ECAPACITY and eng.n_frames == 4
        with pytest.raises(B.EpieError) as ex:
            B.epie_set_object(eng.h, np.ones((3, 3), np.complex64))
        assert ex.value.code == B.EPIE_EINVAL
        with pytest.raises(B.EpieError):
            eng.truncate(5)
        eng.iterate(1)


def test_checked_mode_restores_state_on_nonfinite_error():
    """An infinite intensity makes the sweep error non-finite: EPIE_ENUMERIC, and
    with EPIE_CHECKED the object and probe are back at the sweep's start.
    (A NaN intensity is clamped to 0 like any value below 0.)"""
    d = synth.small_scan(64, 2, 3, 20, seed=17, dtype=np.float32)
    fr = d["frames"].copy()
    fr[3, 10, 10] = np.inf
    with engine(d, B.EPIE_COLOURED, flat_start(d), intensity_dtype=B.EPIE_F32,
                flags=B.EPIE_CHECKED) as eng:
        eng.append(d["frames"][:3], d["pos"][:3])
        eng.iterate(1)
        O1, P1 = eng.object(), eng.probe()
        eng.append(fr[3:], d["pos"][3:])
        with pytest.raises(B.EpieError) as ex:
            eng.iterate(1)
        assert ex.value.code == B.EPIE_ENUMERIC
        assert np.array_equal(eng.object(), O1) and np.array_equal(eng.probe(), P1)
        assert eng.sweep_index == 1


def test_append_from_device_tensor(orc):
    torch = pytest.importorskip("torch")
    d = synth.small_scan(128, 2, 3, 65, seed=18)
    st = textured_start(d)
    O, P, e = sharp(orc, d, B.EPIE_COLOURED, st)
    t = torch.from_numpy(d["frames"].view(np.int16).copy()).cuda()
    torch.cuda.synchronize()
    with engine(d, B.EPIE_COLOURED, st) as eng:
        B.epie_append_frames_device(eng.h, t.data_ptr(), d["pos"], len(d["pos"]))
        e_g = eng.iterate(1)
        assert_parity(eng.object(), eng.probe(), e_g, O, P, e, start=st)


def test_frames_in_fft_order_flag():
    """EPIE_FRAMES_FFT_ORDER: frames and dark field given with the zero
    frequency at [0,0] are stored as given, and the run is bit-identical to
    the DC-centred input re-laid out by the engine."""
    d = synth.small_scan(128, 3, 4, 65, seed=12)
    rng = np.random.default_rng(4)
    dark = (20.0 * rng.random((128, 128))).astype(np.float32)
    fr_fft = np.ascontiguousarray(np.fft.ifftshift(d["frames"], axes=(-2, -1)))
    dark_fft = np.ascontiguousarray(np.fft.ifftshift(dark))
    outs = []
    for frames, dk, flags in [(d["frames"], dark, 0), (fr_fft, dark_fft, B.EPIE_FRAMES_FFT_ORDER)]:
        with engine(d, B.EPIE_COLOURED, flat_start(d), flags=flags) as eng:
            eng.set_dark(dk)
            eng.append(frames[:5], d["pos"][:5])
            eng.append(frames[5:], d["pos"][5:])
            e = eng.iterate(2)
            outs.append((eng.object(), eng.probe(), e))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    assert np.array_equal(outs[0][2], outs[1][2])


def test_dark_field_set_after_append_rederives_amplitudes():
    """The measured amplitudes are derived at append and re-derived when the
    dark field changes: setting (or clearing) the dark field after the frames
    gives the same bits as setting it (or never setting it) before."""
    d = synth.small_scan(256, 3, 3, 120, seed=23)
    rng = np.random.default_rng(8)
    dark = (30.0 * rng.random((256, 256))).astype(np.float32)

    def run(order):
        with engine(d, B.EPIE_COLOURED, flat_start(d)) as eng:
            for op in order:
                if op == "dark":
                    eng.set_dark(dark)
                elif op == "clear":
                    eng.set_dark(None)
                else:
                    eng.append(d["frames"], d["pos"])
            e = eng.iterate(2)
            return eng.object(), eng.probe(), e

    for a, b in [(("dark", "frames"), ("frames", "dark")),
                 (("frames",), ("dark", "frames", "clear"))]:
        ra, rb = run(a), run(b)
        assert all(np.array_equal(x, y) for x, y in zip(ra, rb)), (a, b)


def test_minibatch_256_with_dark_field(orc):
    """Mini-batch sweep at 256^2 on 8-CTA clusters with a dark field: the
    derived-amplitude tiles, the tensor-memory values of the mini-batch
    branch and the count-normalised object apply, against the oracle."""
    d = synth.small_scan(256, 2, 3, 130, seed=6, dark=True, photons=1e7)
    st = textured_start(d)
    I_all = orc.prepare_intensity(d["frames"], d["dark"])
    order = orc.order_sequential(5, 0, len(d["pos"]))

    def run(s0):
        O, P = s0[0].copy(), s0[1].copy()
        er, ir = orc.sweep_minibatch(O, P, I_all, d["pos"], order, 3)
        return O, P, np.array([er / ir])

    (O, P, e), sp = spread(run, st)
    assert max(sp[:2]) <= WELL_CONDITIONED, sp
    with engine(d, B.EPIE_MINIBATCH, st, batch=3) as eng:
        eng.set_dark(d["dark"])
        eng.append(d["frames"], d["pos"])
        e_g = eng.iterate(1)
        assert_parity(eng.object(), eng.probe(), e_g, O, P, e, start=st)


# --------------------------------------------------------------------------- mini-batch at the multi-scan batch sizes

@pytest.mark.parametrize("N,n,batch", [(128, 1024, 1024), (128, 512, 64), (256, 192, 64)])
def test_minibatch_at_multiscan_batch_sizes(orc, N, n, batch):
    """Mini-batch sweeps at the batch sizes the multi-scan workload and its
    autotuner use (64 to 1024 members; 1024 overlapping patches accumulate
    into one batch's object update), jittered-raster scans of the live
    model, against the oracle's mini-batch sweep (reading R7)."""
    d = synth.scan(N, n, "jittered", seed=60 + N + batch, photons=1e8)
    st = textured_start(d)
    I_all = orc.prepare_intensity(d["frames"])
    order = orc.order_sequential(5, 0, n)

    def run(s0):
        O, P = s0[0].copy(), s0[1].copy()
        er, ir = orc.sweep_minibatch(O, P, I_all, d["pos"], order, batch)
        return O, P, np.array([er / ir])

    (O, P, e), sp = spread(run, st, samples=1)
    assert max(sp[:2]) <= WELL_CONDITIONED, sp
    with engine(d, B.EPIE_MINIBATCH, st, batch=batch) as eng:
        eng.append(d["frames"], d["pos"])
        assert np.array_equal(eng.order(0)[0], order)
        e_g = eng.iterate(1)
        assert_parity(eng.object(), eng.probe(), e_g, O, P, e, start=st)


@pytest.mark.parametrize("N,ny,nx,step", [(64, 4, 5, 33), (256, 2, 3, 130)])
def test_raw_intensity_staging(orc, N, ny, nx, step):
    """EPIE_RAW_INTENSITY: the step kernel copies the stored uint16 rows and
    forms sqrt(max(I - dark, 0)) itself.  Against the oracle (sharp, with a
    dark field), and object and probe bit-identical to the derived-amplitude
    path (the same FP32 operations on the same values; only the intensity
    sum of the error metric is added in another order)."""
    d = synth.small_scan(N, ny, nx, step, seed=N + 7, dark=True, photons=1e7)
    st = textured_start(d)
    O, P, e = sharp(orc, d, B.EPIE_COLOURED, st)
    outs = []
    for flags in (0, B.EPIE_RAW_INTENSITY):
        with engine(d, B.EPIE_COLOURED, st, flags=flags) as eng:
            eng.set_dark(d["dark"])
            eng.append(d["frames"], d["pos"])
            e_g = eng.iterate(1)
            assert_parity(eng.object(), eng.probe(), e_g, O, P, e, start=st)
            outs.append((eng.object(), eng.probe(), e_g))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    assert abs(outs[0][2][0] - outs[1][2][0]) <= 1e-12 * outs[0][2][0]


@pytest.mark.parametrize("N,shape,step", [(64, 0, 20), (128, 0, 65), (128, 1, 65), (256, 0, 130),
                                          (512, 0, 300)])
@pytest.mark.parametrize("dtype,code", [(np.uint16, B.EPIE_U16), (np.float16, B.EPIE_F16),
                                        (np.float32, B.EPIE_F32)])
def test_derived_amplitudes_equal_staged_rows(N, shape, step, dtype, code):
    """The amplitudes derived at append (8 intensities per 16-byte load, in
    each step kernel's tile layout) against the step kernel's own conversion
    of the staged rows (EPIE_RAW_INTENSITY): object and probe bit-identical
    after one sweep, for every intensity type and tile shape, with a dark
    field above some intensities and, for the float types, negative and NaN
    intensities (clamped to 0 on both paths).  The sweep error differs only
    in the order of the intensity sum."""
    d = synth.small_scan(N, 1, 3, step, seed=N + 31, dark=True, photons=1e7, dtype=dtype)
    fr = d["frames"].copy()
    if code != B.EPIE_U16:
        fr[0, 3, 5] = np.nan
        fr[1, N // 2, N // 3] = -4.0
        fr[2, N - 1, 0] = np.nan
        fr[2, 7, N - 2] = -0.0
    st = textured_start(d)
    outs = []
    for flags in (0, B.EPIE_RAW_INTENSITY):
        with engine(d, B.EPIE_COLOURED, st, ctas_per_frame=shape, intensity_dtype=code,
                    flags=flags) as eng:
            eng.set_dark(d["dark"])
            eng.append(fr, d["pos"])
            e_g = eng.iterate(1)
            outs.append((eng.object(), eng.probe(), e_g))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    assert np.isfinite(outs[0][2][0])
    assert abs(outs[0][2][0] - outs[1][2][0]) <= 1e-12 * outs[0][2][0]
