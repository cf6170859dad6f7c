"""Parity at the benchmark's full size (256^2 uint16 frames, the live
workload's 2725 x 2728 object and Fermat-spiral geometry, dark field).

* test_engine_classes_of_the_full_live_workload runs through the engine, in
  the branch the benchmark times: the dark field is set before the frames are
  appended, so the step kernel reads the measured amplitudes derived at
  append; the engine colours the appended frames itself; the second class of
  a sweep reads its object patches before its dependency wait (o_early) and
  every launch is chained to the previous one by programmatic dependent
  launch.  The members of one whole colour class of the full scan, and then
  of two consecutive classes, are appended to a handle sized for the full
  object and run through epie_iterate; the FP64 oracle runs the same sweep
  (same colouring of the appended frames, same order) from the same textured
  start.  One or two classes are one or two dependent steps, so the
  comparison is sharp, on the state and on the increment.
* test_static_class_of_the_full_live_workload runs one class through the
  allocation-free entry point, whose step kernel converts the raw uint16
  intensities itself (no derived amplitudes), with the whole frame set
  resident on the device.
"""
import numpy as np
import pytest

from paper_2308_10674_gb300 import _binding as B
from paper_2308_10674_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL_STATE, TOL_ERR, TOL_INC = 1e-5, 1e-6, 1e-4


def rel(a, b):
    return float(np.linalg.norm((np.asarray(a) - b).ravel()) / np.linalg.norm(np.ravel(b)))


@pytest.fixture(scope="module")
def live():
    d = synth.live_scan(N=256, n=10000, geometry="A", seed=0, workers=8)
    rng = np.random.default_rng(3)
    O0 = (d["O_true"] * (1 + 0.05 * synth.smooth_field(d["O_true"].shape, 2.0, rng)))
    P0 = (d["P_true"] * (1 + 0.05 * synth.smooth_field(d["P_true"].shape, 2.0, rng)))
    d["start"] = (O0.astype(np.complex64), P0.astype(np.complex64))
    return d


def full_classes(orc, d):
    col, ncls = orc.colour_greedy(d["pos"], 256)
    order, gs = orc.order_coloured(5, 0, col, ncls)
    return order, gs


def check_class_result(O_g, P_g, e_g, O, P, e, O0, P0, pos, N=256):
    assert rel(O_g, O) <= TOL_STATE and rel(P_g, P) <= TOL_STATE, (rel(O_g, O), rel(P_g, P))
    assert rel(O_g - O0, O - O0) <= TOL_INC and rel(P_g - P0, P - P0) <= TOL_INC, (
        rel(O_g - O0, O - O0), rel(P_g - P0, P - P0))
    assert np.all(np.abs(np.asarray(e_g) - e) <= TOL_ERR * np.abs(e)), (e_g, e)
    # the patches changed (where the probe is not 0) and nothing else did
    changed = np.abs(O_g - O0) > 0
    cover = np.zeros(O0.shape, bool)
    for y, x in pos:
        cover[y:y + N, x:x + N] = True
    assert changed[cover].any() and not changed[~cover].any()


@pytest.mark.parametrize("n_classes", [1, 2])
def test_engine_classes_of_the_full_live_workload(orc, live, n_classes):
    d, N = live, 256
    O0, P0 = d["start"]
    order, gs = full_classes(orc, d)
    sizes = np.diff(gs)
    g = int(np.argmax(sizes >= 40))  # full-size classes of the first sweep
    sel = order[gs[g]:gs[g + n_classes]]
    frames, pos = d["frames"][sel], np.ascontiguousarray(d["pos"][sel])
    eng = B.Engine(N, d["H"], d["W"], P0, O0, capacity=len(sel), mode=B.EPIE_COLOURED, seed=5,
                   device=0)
    try:
        eng.set_dark(d["dark"])          # before the frames: amplitudes derived at append
        eng.append(frames, pos)
        col, ncls = orc.colour_greedy(pos, N)
        assert np.array_equal(eng.colours(), col) and eng.n_classes == ncls
        if n_classes == 2:
            assert ncls >= 2             # the second class runs with o_early
        o_sub, gs_sub = orc.order_coloured(5, 0, col, ncls)
        o_eng, gs_eng = eng.order(0)
        assert np.array_equal(o_eng, o_sub) and np.array_equal(gs_eng, gs_sub)
        e_g = eng.iterate(1)
        O_g, P_g = eng.object(), eng.probe()
    finally:
        eng.close()
    O, P = O0.astype(complex), P0.astype(complex)
    I_all = orc.prepare_intensity(frames, d["dark"])
    er, ir = orc.sweep_groups(O, P, I_all, pos, o_sub, gs_sub)
    check_class_result(O_g, P_g, e_g, O, P, np.array([er / ir]), O0, P0, pos)


def test_static_class_of_the_full_live_workload(orc, live):
    d, N = live, 256
    n = len(d["pos"])
    O0, P0 = d["start"]
    order, gs = full_classes(orc, d)
    sizes = np.diff(gs)
    g = int(np.argmax((sizes <= 64) & (sizes >= 32)))  # a full-size class within the limit
    members = order[gs[g]:gs[g + 1]].astype(np.int32)
    dev = torch.device("cuda", 0)
    raw = torch.from_numpy(d["frames"].view(np.int16)).to(dev)
    fft_frames = torch.empty_like(raw)
    B.epie_frames_to_fft_order(raw.data_ptr(), fft_frames.data_ptr(), n, N, B.EPIE_U16)
    del raw
    dark_fft = torch.from_numpy(np.ascontiguousarray(np.fft.ifftshift(d["dark"]))).to(dev)
    O_t = torch.from_numpy(O0.copy()).to(dev)
    P_t = torch.from_numpy(P0.copy()).to(dev)
    pos_t = torch.from_numpy(d["pos"].astype(np.int32)).to(dev)
    mem_t = torch.from_numpy(members).to(dev)
    torch.cuda.synchronize()
    e, s = B.epie_group_step_static(N, B.EPIE_U16, O_t.data_ptr(), d["H"], d["W"], P_t.data_ptr(),
                                    fft_frames.data_ptr(), n, pos_t.data_ptr(), mem_t.data_ptr(),
                                    len(members), dark_ptr=dark_fft.data_ptr())
    O_g, P_g = O_t.cpu().numpy(), P_t.cpu().numpy()
    del fft_frames
    O, P = O0.astype(complex), P0.astype(complex)
    I_all = np.zeros((n, N, N))
    I_all[members] = orc.prepare_intensity(d["frames"][members], d["dark"])
    er, ir = orc.sweep_groups(O, P, I_all, d["pos"], members, np.array([0, len(members)]))
    assert abs(s - ir) <= 1e-6 * ir
    check_class_result(O_g, P_g, [e / s], O, P, np.array([er / ir]), O0, P0, d["pos"][members])
