"""epie_group_step_static: the group update for callers that cannot allocate
device memory (a framework that owns the GPU's memory and lends out fixed
buffers, or a live loop that must not pay cudaMalloc's device-wide
synchronisation).  The caller brings every device buffer (here from torch);
the entry point's scratch lives in the library's static device array.

Checked through the C ABI against the handle-based entry point
(epie_iterate) on the same inputs and visiting order, sweep after sweep
(several calls in a row), with the parity tolerance of the GPU tests
(relative L2 <= 1e-5 on object and probe, 1e-6 on the sweep error).  Runs in
a fresh process as well as after the rest of the suite.
"""
import numpy as np
import pytest

from paper_2308_10674_gb300 import _binding as B
from paper_2308_10674_gb300 import synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def start_state(d):
    rng = np.random.default_rng(3)
    O = d["O_true"] * (1 + 0.05 * synth.smooth_field(d["O_true"].shape, 2.0, rng))
    P = d["P_true"] * (1 + 0.05 * synth.smooth_field(d["P_true"].shape, 2.0, rng))
    return O.astype(np.complex64), P.astype(np.complex64)


# (N, raster ny x nx, step, dark field, probe moved by the mean): 64^2 with the
# probe sum, 128^2 with a dark field, 256^2, and 512^2 with one class of 16
# disjoint members (the entry point's member limit at that size)
CASES = [(64, 4, 5, 33, False, False), (128, 3, 4, 66, True, True),
         (256, 3, 4, 130, False, True), (512, 4, 4, 520, False, True)]


@pytest.mark.parametrize("N,ny,nx,step,dark,mean", CASES)
def test_static_scratch_step_matches_engine(N, ny, nx, step, dark, mean):
    torch = pytest.importorskip("torch")
    d = synth.small_scan(N, ny, nx, step, seed=N + 1, dark=dark)
    O0, P0 = start_state(d)
    n = len(d["pos"])
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    # caller-owned device buffers; frames in FFT order (zero frequency at [0, 0])
    O_t = torch.from_numpy(O0.copy()).to(dev)
    P_t = torch.from_numpy(P0.copy()).to(dev)
    fft_frames = np.ascontiguousarray(np.fft.ifftshift(d["frames"], axes=(-2, -1)))
    F_t = torch.from_numpy(fft_frames.view(np.int16)).to(dev)
    pos_t = torch.from_numpy(np.ascontiguousarray(d["pos"], np.int32)).to(dev)
    dark_t = None
    if dark:
        dark_t = torch.from_numpy(
            np.ascontiguousarray(np.fft.ifftshift(d["dark"]), np.float32)).to(dev)
    torch.cuda.synchronize(dev)

    eng = B.Engine(N, d["H"], d["W"], P0, O0, capacity=n, mode=B.EPIE_COLOURED, seed=5,
                   device=0, flags=0 if mean else B.EPIE_PROBE_SUM)
    try:
        if dark:
            eng.set_dark(d["dark"])
        eng.append(d["frames"], d["pos"])
        if N == 512:
            assert eng.n_classes == 1  # all 16 members in one group
        for sweep in range(2):
            order, gs = eng.order(sweep)
            mem_t = torch.from_numpy(order.astype(np.int32)).to(dev)
            e_sum = s_sum = 0.0
            for g in range(len(gs) - 1):
                a, b = int(gs[g]), int(gs[g + 1])
                e, s = B.epie_group_step_static(
                    N, B.EPIE_U16, O_t.data_ptr(), d["H"], d["W"], P_t.data_ptr(),
                    F_t.data_ptr(), n, pos_t.data_ptr(), mem_t.data_ptr() + 4 * a, b - a,
                    dark_ptr=None if dark_t is None else dark_t.data_ptr(), probe_mean=mean,
                    stream=stream.cuda_stream)
                e_sum += e
                s_sum += s
            err_engine = eng.iterate(1)[0]
            torch.cuda.synchronize(dev)
            O_s = O_t.cpu().numpy()
            P_s = P_t.cpu().numpy()
            assert rel(O_s, eng.object()) <= 1e-5, (sweep, rel(O_s, eng.object()))
            assert rel(P_s, eng.probe()) <= 1e-5, (sweep, rel(P_s, eng.probe()))
            assert abs(e_sum / s_sum - err_engine) <= 1e-6 * err_engine
    finally:
        eng.close()


def test_static_scratch_limits_are_rejected():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    buf = torch.zeros(1 << 16, dtype=torch.float32, device=dev)
    p = buf.data_ptr()
    with pytest.raises(B.EpieError) as ex:  # 65 members of 256^2 exceed the scratch
        B.epie_group_step_static(256, B.EPIE_U16, p, 512, 512, p, p, 100, p, p, 65)
    assert ex.value.code == B.EPIE_EINVAL and "static scratch limit" in str(ex.value)
    with pytest.raises(B.EpieError) as ex:
        B.epie_group_step_static(64, B.EPIE_U16, p, 128, 128, p, p, 20000, p, p, 1)
    assert ex.value.code == B.EPIE_EINVAL and "16384" in str(ex.value)
    # a member id outside the frame set is caught on the device before the step
    ids = torch.tensor([0, 7], dtype=torch.int32, device=dev)
    pos = torch.zeros(8, dtype=torch.int32, device=dev)
    with pytest.raises(B.EpieError) as ex:
        B.epie_group_step_static(64, B.EPIE_U16, p, 128, 128, p, p, 4, pos.data_ptr(),
                                 ids.data_ptr(), 2)
    assert ex.value.code == B.EPIE_EINVAL and "outside" in str(ex.value)


def test_static_misaligned_pointers_are_rejected():
    """Caller-lent buffers at odd offsets are refused before any launch: the
    step copies frame rows with bulk copies (16-byte aligned source), reads
    the object as float2 and the probe reduction moves the probe as float4."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    buf = torch.zeros(1 << 16, dtype=torch.float32, device=dev)
    p = buf.data_ptr()
    ids = torch.zeros(1, dtype=torch.int32, device=dev)
    pos = torch.zeros(2, dtype=torch.int32, device=dev)
    for obj, prb, frm, why in ((p + 4, p, p, "object"), (p, p + 8, p, "probe"),
                               (p, p, p + 2, "frames")):
        with pytest.raises(B.EpieError) as ex:
            B.epie_group_step_static(64, B.EPIE_U16, obj, 128, 128, prb, frm, 1, pos.data_ptr(),
                                     ids.data_ptr(), 1)
        assert ex.value.code == B.EPIE_EINVAL and why in str(ex.value)
