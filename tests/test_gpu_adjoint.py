"""The hand-written adjoint of the amplitude loss against the FP64 oracle's
gradient (which tests/test_oracle_pins.py pins by central finite
differences), through the C ABI and the autograd Function."""
import numpy as np
import pytest

from paper_2308_10674_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def instance(N, ny, nx, step, seed):
    d = synth.small_scan(N, ny, nx, step, seed=seed)
    rng = np.random.default_rng(seed)
    O = (d["O_true"] * (1 + 0.1 * synth.smooth_field(d["O_true"].shape, 2.0, rng))).astype(np.complex64)
    P = (d["P_true"] * (1 + 0.1 * synth.smooth_field(d["P_true"].shape, 2.0, rng))).astype(np.complex64)
    shift = rng.uniform(-0.5, 0.5, (len(d["pos"]), 2)).astype(np.float32)
    return d, O, P, shift


@pytest.mark.parametrize("N,ny,nx,step", [(64, 3, 4, 20), (128, 3, 3, 40), (256, 2, 2, 90)])
@pytest.mark.parametrize("with_shift", [True, False])
def test_gradient_matches_oracle(orc, N, ny, nx, step, with_shift):
    from paper_2308_10674_gb300.autograd import amplitude_loss, frames_to_fft_order
    d, O, P, shift = instance(N, ny, nx, step, seed=N + 3)
    dev = torch.device("cuda", 0)
    o = torch.from_numpy(O).to(dev).requires_grad_()
    p = torch.from_numpy(P).to(dev).requires_grad_()
    s = torch.from_numpy(shift).to(dev).requires_grad_() if with_shift else None
    fr = frames_to_fft_order(torch.from_numpy(d["frames"].view(np.int16)).to(dev))
    pos = torch.from_numpy(d["pos"].astype(np.int32)).to(dev)
    loss = amplitude_loss(o, p, s, fr, pos)
    loss.backward()
    I_all = orc.prepare_intensity(d["frames"])
    L, gO, gP, gd = orc.amp_loss_grad(O.astype(complex), P.astype(complex), I_all, d["pos"],
                                      shift.astype(float) if with_shift else None)
    assert abs(loss.item() - L) <= 1e-5 * L
    assert rel(o.grad.cpu().numpy(), gO) <= 1e-4
    assert rel(p.grad.cpu().numpy(), gP) <= 1e-4
    if with_shift:
        assert rel(s.grad.cpu().numpy(), gd) <= 1e-4


def test_frames_to_fft_order_is_ifftshift():
    from paper_2308_10674_gb300.autograd import frames_to_fft_order
    x = np.arange(2 * 64 * 64, dtype=np.float32).reshape(2, 64, 64)
    y = frames_to_fft_order(torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.array_equal(y, np.fft.ifftshift(x, axes=(-2, -1)))


def test_adam_reconstruction_reduces_the_loss():
    """200 Adam steps on object, probe and positions together (FP32
    parameters, every learning rate non-zero), a smaller instance shaped like
    the differentiable-reconstruction workload simulated at integer
    positions: the loss falls tenfold and the offsets, whose truth is zero,
    stay within a fraction of a pixel (a joint shift of object and probe is a
    symmetry of the loss, so they are not pinned exactly)."""
    from paper_2308_10674_gb300.autograd import amplitude_loss, frames_to_fft_order
    N = 64
    d = synth.small_scan(N, 6, 6, 12, seed=5, photons=1e6)
    dev = torch.device("cuda", 0)
    fr = frames_to_fft_order(torch.from_numpy(d["frames"].view(np.int16)).to(dev))
    pos = torch.from_numpy(d["pos"].astype(np.int32)).to(dev)
    o = torch.ones(d["H"], d["W"], dtype=torch.complex64, device=dev).requires_grad_()
    p = torch.from_numpy(d["P0"].astype(np.complex64)).to(dev).requires_grad_()
    s = torch.zeros(len(d["pos"]), 2, dtype=torch.float32, device=dev, requires_grad=True)
    opt = torch.optim.Adam([{"params": [o], "lr": 2e-2}, {"params": [p], "lr": 2e-3},
                            {"params": [s], "lr": 1e-3}])
    losses = []
    for it in range(200):
        opt.zero_grad()
        loss = amplitude_loss(o, p, s, fr, pos)
        loss.backward()
        opt.step()
        losses.append(loss.item())
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.2 * losses[0], (losses[0], losses[-1])
    shifts = s.detach().cpu().numpy()
    assert np.all(np.isfinite(shifts)) and np.abs(shifts).max() < 0.5, np.abs(shifts).max()


def fourier_shift(P, dy, dx):
    """S_d P = F^-1[F P exp(-2 pi i (ky dy + kx dx) / N)], frequencies in FFT
    order with k >= N/2 standing for k - N (the adjoint's shift model)."""
    N = P.shape[0]
    k = np.fft.fftfreq(N) * N
    ph = np.exp(-2j * np.pi * (k[:, None] * dy + k[None, :] * dx) / N)
    return np.fft.ifft2(np.fft.fft2(P) * ph)


def test_adam_refines_subpixel_positions():
    """Frames simulated with a known sub-pixel offset per position (the probe
    Fourier-shifted by d_j in [-0.4, 0.4] px); from zero offsets with the true
    object and probe held fixed, 150 Adam steps on the offsets alone bring
    them to the truth: the mean offset error falls below 15% of its start."""
    from paper_2308_10674_gb300.autograd import amplitude_loss
    N = 64
    d = synth.small_scan(N, 5, 5, 12, seed=6, photons=1e6)
    rng = np.random.default_rng(11)
    n = len(d["pos"])
    d_true = rng.uniform(-0.4, 0.4, (n, 2))
    I = np.empty((n, N, N), np.float32)
    for j, (y, x) in enumerate(d["pos"]):
        psi = fourier_shift(d["P_true"], *d_true[j]) * d["O_true"][y:y + N, x:x + N]
        I[j] = np.abs(np.fft.fft2(psi)) ** 2           # FFT order, zero frequency at [0, 0]
    dev = torch.device("cuda", 0)
    fr = torch.from_numpy(I).to(dev)
    pos = torch.from_numpy(d["pos"].astype(np.int32)).to(dev)
    o = torch.from_numpy(d["O_true"].astype(np.complex64)).to(dev)
    p = torch.from_numpy(d["P_true"].astype(np.complex64)).to(dev)
    s = torch.zeros(n, 2, dtype=torch.float32, device=dev, requires_grad=True)
    opt = torch.optim.Adam([s], lr=2e-2)
    err0 = float(np.mean(np.abs(d_true)))
    for _ in range(150):
        opt.zero_grad()
        amplitude_loss(o, p, s, fr, pos).backward()
        opt.step()
    err = float(np.mean(np.abs(s.detach().cpu().numpy() - d_true)))
    assert err < 0.15 * err0, (err, err0)
