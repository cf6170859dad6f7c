"""Seeded synthetic ptychography inputs shaped like the paper's workloads.

This module only generates inputs; it holds no step of the reconstruction.
It is shared by the tests (which hand the same arrays to the FP64 oracle and
to the CUDA library) and by the benchmark.  The diffraction frames are
simulated with numpy's own FFT (a library routine that neither the oracle nor
the CUDA path uses).

Shapes follow the paper's data (Sec. "Simulating live and parallel
processing": 256x256 crops, 21x21 raster; Sec. "Live ePIE": 11,245 frames
256x256 on a meander): every array here is synthetic, because the paper's
datasets are not available offline.

Conventions shared with the engine's C ABI:
  * frames: uint16 [n, N, N], detector layout with the zero frequency at
    index (N//2, N//2) ("DC-centred");
  * positions: int32 [n, 2] = (y, x) of the patch's top-left object pixel;
  * object [H, W] and probe [N, N] complex.
"""
from __future__ import annotations

import math

import numpy as np

MASK64 = (1 << 64) - 1


def substream(seed: int, stream_id: int) -> np.random.Generator:
    """Independent numpy generator for one purpose (object, jitter, noise, ...)."""
    return np.random.default_rng([seed & MASK64, stream_id])


# --------------------------------------------------------------------------- fields

def _gauss_kernel_ft(shape, sigma):
    ky = np.fft.fftfreq(shape[0])[:, None]
    kx = np.fft.fftfreq(shape[1])[None, :]
    return np.exp(-2.0 * (math.pi * sigma) ** 2 * (ky ** 2 + kx ** 2))


def smooth_field(shape, sigma, rng):
    """White noise convolved (periodically) with a Gaussian of width sigma px."""
    w = rng.standard_normal(shape)
    return np.real(np.fft.ifft2(np.fft.fft2(w) * _gauss_kernel_ft(shape, sigma)))


def rescale(a, lo, hi):
    a = np.asarray(a, np.float64)
    mn, mx = a.min(), a.max()
    if mx <= mn:
        return np.full_like(a, 0.5 * (lo + hi))
    return lo + (a - mn) * (hi - lo) / (mx - mn)


def make_object(H, W, sigma_phase, rng, amp_lo=0.8, amp_hi=1.0):
    """Amplitude uniform in [amp_lo, amp_hi]; phase a Gaussian-smoothed random
    field rescaled to [-pi/2, pi/2]."""
    amp = rng.uniform(amp_lo, amp_hi, size=(H, W))
    ph = rescale(smooth_field((H, W), sigma_phase, rng), -math.pi / 2, math.pi / 2)
    return (amp * np.exp(1j * ph)).astype(np.complex128)


def aperture_amplitude(N, radius, sigma):
    """Circular aperture of the given radius centred at (N/2, N/2), convolved
    with a Gaussian of width sigma (apodisation)."""
    y, x = np.mgrid[0:N, 0:N].astype(np.float64)
    r = np.hypot(y - N / 2, x - N / 2)
    disc = (r <= radius).astype(np.float64)
    a = np.real(np.fft.ifft2(np.fft.fft2(np.fft.ifftshift(disc)) * _gauss_kernel_ft((N, N), sigma)))
    return np.clip(np.fft.fftshift(a), 0.0, None)


def make_probe(N, radius, sigma, with_phase=True):
    """Apodised aperture times a quadratic defocus phase of 2 pi at the edge."""
    amp = aperture_amplitude(N, radius, sigma)
    if not with_phase:
        return amp.astype(np.complex128)
    y, x = np.mgrid[0:N, 0:N].astype(np.float64)
    r = np.hypot(y - N / 2, x - N / 2)
    return (amp * np.exp(1j * 2 * math.pi * (r / radius) ** 2)).astype(np.complex128)


def intensity_fwhm(P):
    """FWHM (px) of |P|^2 along the horizontal line through the centre."""
    N = P.shape[0]
    prof = np.abs(P[N // 2]) ** 2
    half = prof.max() / 2
    above = np.nonzero(prof >= half)[0]
    lo, hi = above[0], above[-1]
    # linear interpolation at both edges
    def cross(i0, i1):
        a, b = prof[i0], prof[i1]
        return i0 + (half - a) / (b - a) * (i1 - i0) if b != a else i0
    left = cross(lo - 1, lo) if lo > 0 else lo
    right = cross(hi, hi + 1) if hi < N - 1 else hi
    return float(right - left)


def probe_radius_for_fwhm(N, fwhm, sigma_per_radius=3.0 / 20.0):
    """Bisection on the aperture radius so that |P|^2 has the requested FWHM
    (to within 0.5 px); the apodisation width scales with the radius."""
    lo, hi = 2.0, N / 2.0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        f = intensity_fwhm(aperture_amplitude(N, mid, sigma_per_radius * mid))
        if f < fwhm:
            lo = mid
        else:
            hi = mid
        if hi - lo < 1e-3:
            break
    r = 0.5 * (lo + hi)
    assert abs(intensity_fwhm(aperture_amplitude(N, r, sigma_per_radius * r)) - fwhm) <= 0.5
    return r


# --------------------------------------------------------------------------- scan patterns

def raster_positions(ny, nx, step, offset, jitter, rng):
    """Raster of patch top-left positions (y, x) = offset + step*(i, j) + jitter,
    jitter uniform in {-jitter..jitter} per axis."""
    iy, ix = np.mgrid[0:ny, 0:nx]
    pos = np.stack([offset + step * iy.ravel(), offset + step * ix.ravel()], axis=1)
    if jitter:
        pos = pos + rng.integers(-jitter, jitter + 1, size=pos.shape)
    return pos.astype(np.int32)


def round_half_away(a):
    return np.sign(a) * np.floor(np.abs(a) + 0.5)


def fermat_spiral_centres(n, c):
    """Fermat spiral r_k = c sqrt(k), theta_k = k * 137.508 deg, k = 0..n-1."""
    k = np.arange(n, dtype=np.float64)
    r = c * np.sqrt(k)
    th = np.deg2rad(137.508) * k
    return np.stack([r * np.sin(th), r * np.cos(th)], axis=1)


def median_nn_distance(pts):
    pts = np.asarray(pts, np.float64)
    order = np.argsort(pts[:, 0])
    p = pts[order]
    best = np.full(len(p), np.inf)
    # sweep in y: compare with the next few hundred neighbours in y order
    for s in range(1, min(400, len(p))):
        d = np.hypot(p[s:, 0] - p[:-s, 0], p[s:, 1] - p[:-s, 1])
        best[s:] = np.minimum(best[s:], d)
        best[:-s] = np.minimum(best[:-s], d)
    return float(np.median(best))


def spiral_c_for_step(n, step):
    """Spiral constant c giving a median nearest-neighbour distance of `step`."""
    c0 = 1.0
    d0 = median_nn_distance(fermat_spiral_centres(min(n, 4000), c0))
    return step * c0 / d0


def centres_to_topleft(centres, N, margin):
    """Integer patch top-left positions (round half away from zero) and the
    object size covering every patch plus a margin (the paper pads the scan's
    bounding box by half the illumination size on each side)."""
    c = centres - centres.min(axis=0)
    tl = round_half_away(c).astype(np.int64) + margin
    H = int(tl[:, 0].max()) + N + margin
    W = int(tl[:, 1].max()) + N + margin
    return tl.astype(np.int32), H, W


# --------------------------------------------------------------------------- measurement model

def far_field_intensity(O, P, pos, batch=256, dtype=np.complex128):
    """|F(P . O_patch)|^2 per position, DC-centred (fftshift), float64."""
    N = P.shape[0]
    out = np.empty((len(pos), N, N), np.float64)
    Pc = P.astype(dtype)
    for a in range(0, len(pos), batch):
        b = min(len(pos), a + batch)
        psi = np.stack([Pc * O[y:y + N, x:x + N].astype(dtype) for y, x in pos[a:b]])
        F = np.fft.fft2(psi, axes=(-2, -1))
        out[a:b] = np.fft.fftshift(np.abs(F) ** 2, axes=(-2, -1))
    return out


def scale_probe_to_photons(O, P, pos, photons):
    """Scale P so that the mean over positions of sum_k |F(P O_j)|^2 = photons
    (by Parseval this is N^2 sum_r |P O_j|^2)."""
    N = P.shape[0]
    tot = np.mean([np.sum(np.abs(P * O[y:y + N, x:x + N]) ** 2) for y, x in pos]) * N * N
    return P * math.sqrt(photons / tot)


def poisson_u16(lam, rng):
    """Poisson counts clamped to the uint16 range; returns (counts, clamped fraction)."""
    k = rng.poisson(lam)
    clamped = float(np.mean(k > 65535))
    return np.minimum(k, 65535).astype(np.uint16), clamped


def dark_field(N, photons, rng, frac=0.02, sigma=8.0):
    """Dark-offset field D = frac * (photons/N^2) * (1 + 0.5 g), g a smoothed
    random field rescaled to [-1, 1]; DC-centred layout like the frames."""
    g = rescale(smooth_field((N, N), sigma, rng), -1.0, 1.0)
    return (frac * photons / (N * N) * (1.0 + 0.5 * g)).astype(np.float32)


def initial_probe(N, radius, sigma, photons):
    """Starting probe: the apodised aperture without phase, scaled so that
    N^2 sum |P0|^2 equals the mean photon count per frame (object = 1)."""
    P0 = make_probe(N, radius, sigma, with_phase=False)
    return P0 * math.sqrt(photons / (N * N * np.sum(np.abs(P0) ** 2)))


# --------------------------------------------------------------------------- workloads

def config0(seed=0, photons=1e6, noise=True):
    """Plain sequential workload: 64x64 frames, 16x16 raster, step 8 px with
    +-1 px jitter, object 192x192, probe radius 20 / apodisation 3 / defocus
    2 pi at the edge, 1e6 photons per frame with Poisson noise, uint16."""
    N, H, W = 64, 192, 192
    rng_obj, rng_jit, rng_noise = substream(seed, 1), substream(seed, 2), substream(seed, 3)
    O_true = make_object(H, W, 4.0, rng_obj)
    pos = raster_positions(16, 16, 8, 4, 1, rng_jit)
    P_true = scale_probe_to_photons(O_true, make_probe(N, 20.0, 3.0), pos, photons)
    lam = far_field_intensity(O_true, P_true, pos)
    if noise:
        frames, clamped = poisson_u16(lam, rng_noise)
    else:
        frames, clamped = lam.astype(np.float32), 0.0
    return dict(N=N, H=H, W=W, pos=pos, frames=frames, O_true=O_true, P_true=P_true,
                O0=np.ones((H, W), np.complex128), P0=initial_probe(N, 20.0, 3.0, photons),
                dark=None, clamped=clamped, photons=photons, seed=seed)


_W = {}


def _init_worker(O, P, D):
    _W["O"], _W["P"], _W["D"] = O, P, D


def _frames_chunk(args):
    """Frames [a, b) of a scan; noise drawn from a substream keyed by the chunk
    index, so the result does not depend on how chunks are spread over workers."""
    pos, seed, chunk, noise, dtype = args
    lam = far_field_intensity(_W["O"], _W["P"], pos, dtype=np.complex64)
    if _W["D"] is not None:
        lam = lam + _W["D"][None].astype(np.float64)
    if dtype == np.float16:
        if noise:
            lam = substream(seed, 1000 + chunk).poisson(lam).astype(np.float64)
        return np.minimum(lam, 65504.0).astype(np.float16), float(np.mean(lam > 65504.0))
    if noise:
        return poisson_u16(lam, substream(seed, 1000 + chunk))
    return lam.astype(np.float32), 0.0


LIVE_CHUNK = 250


def scan(N, n, pattern="spiral", seed=0, photons=1e8, fwhm=None, noise=True, dark=False,
         dtype=np.uint16, workers=1):
    """Scan of n positions at frame side N on a "raster", "jittered" raster
    (+-20% of the step, seeded) or Fermat "spiral", step 0.35 x the probe
    FWHM (default FWHM 60 px x N/256), object and probe as in live_scan.
    dtype float16 stores the (noisy or model) intensities as binary16,
    clamped to 65504."""
    fwhm = 60.0 * N / 256.0 if fwhm is None else fwhm
    step = 0.35 * fwhm
    rng_jit = substream(seed, 31)
    if pattern == "spiral":
        cen = fermat_spiral_centres(n, spiral_c_for_step(n, step))
    else:
        side = int(math.ceil(math.sqrt(n)))
        iy, ix = np.divmod(np.arange(n), side)
        cen = np.stack([iy * step, ix * step], axis=1).astype(np.float64)
        if pattern == "jittered":
            cen = cen + rng_jit.uniform(-0.2 * step, 0.2 * step, size=cen.shape)
        elif pattern != "raster":
            raise ValueError("pattern must be raster, jittered or spiral")
    return live_scan(N=N, n=n, seed=seed, photons=photons, fwhm=fwhm, noise=noise, dark=dark,
                     workers=workers, centres=cen, dtype=dtype)


def live_scan(N=256, n=10000, geometry="A", seed=0, photons=1e8, fwhm=60.0, noise=True,
              dark=True, n_frames=None, workers=1, centres=None, dtype=np.uint16):
    """Beamline-like live workload: N x N uint16 frames on a Fermat spiral.

    geometry "A": step = 0.35 x probe FWHM (median nearest-neighbour distance),
    giving an object of about 2730^2 at n = 10,000; geometry "B": object about
    1400^2 (step about 9.7 px).  Probe radius and apodisation are scaled so
    that |P|^2 has the given FWHM; object phase smoothing scales with it.
    `n_frames` simulates only the first n_frames positions (the geometry is
    still that of the full scan).  `workers` > 1 simulates chunks of frames
    in a process pool (spawned, so it is safe after CUDA initialisation);
    the frames are identical for any worker count."""
    rng_obj, rng_dark = substream(seed, 11), substream(seed, 14)
    R = probe_radius_for_fwhm(N, fwhm)
    sig_ap = 3.0 * R / 20.0
    c = None
    if centres is None:
        if geometry == "A":
            c = spiral_c_for_step(n, 0.35 * fwhm)
        elif geometry == "B":
            c = (1400 - N - 8) / 2.0 / math.sqrt(n)
        else:
            raise ValueError("geometry must be 'A' or 'B'")
        centres = fermat_spiral_centres(n, c)
    tl, H, W = centres_to_topleft(centres, N, 4)
    O_true = make_object(H, W, 4.0 * R / 20.0, rng_obj)
    m = n if n_frames is None else min(n, n_frames)
    pos = tl[:m]
    P_true = scale_probe_to_photons(O_true, make_probe(N, R, sig_ap), pos[: min(m, 500)], photons)
    D = dark_field(N, photons, rng_dark) if dark else None
    jobs = [(pos[a:min(m, a + LIVE_CHUNK)], seed, a // LIVE_CHUNK, noise, dtype)
            for a in range(0, m, LIVE_CHUNK)]
    O32, P32 = O_true.astype(np.complex64), P_true.astype(np.complex64)
    if workers > 1 and len(jobs) > 1:
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        with ctx.Pool(min(workers, len(jobs)), initializer=_init_worker,
                      initargs=(O32, P32, D)) as pool:
            parts = pool.map(_frames_chunk, jobs)
    else:
        _init_worker(O32, P32, D)
        parts = [_frames_chunk(j) for j in jobs]
    frames = (np.concatenate([p[0] for p in parts]) if parts else
              np.empty((0, N, N), dtype if dtype == np.float16 else
                       (np.uint16 if noise else np.float32)))
    clamped = sum(p[1] * len(j[0]) for p, j in zip(parts, jobs)) / max(m, 1)
    return dict(N=N, H=H, W=W, pos=pos, frames=frames, O_true=O_true, P_true=P_true,
                O0=np.ones((H, W), np.complex128), P0=initial_probe(N, R, sig_ap, photons),
                dark=D, clamped=clamped, photons=photons, seed=seed,
                geometry=geometry, spiral_c=c, probe_radius=R, n_total=n)


def small_scan(N, ny, nx, step, seed=0, photons=1e6, jitter=1, margin=4, noise=True,
               dark=False, dtype=np.uint16):
    """Small raster workload at any frame size (parity cases): ny x nx positions,
    probe radius N*20/64, apodisation N*3/64, object just large enough."""
    rng_obj, rng_jit, rng_noise, rng_dark = (substream(seed, 21), substream(seed, 22),
                                             substream(seed, 23), substream(seed, 24))
    H = margin * 2 + jitter * 2 + step * (ny - 1) + N
    W = margin * 2 + jitter * 2 + step * (nx - 1) + N
    R, sg = N * 20.0 / 64.0, N * 3.0 / 64.0
    O_true = make_object(H, W, max(1.0, N * 4.0 / 64.0), rng_obj)
    pos = raster_positions(ny, nx, step, margin + jitter, jitter, rng_jit)
    P_true = scale_probe_to_photons(O_true, make_probe(N, R, sg), pos, photons)
    lam = far_field_intensity(O_true, P_true, pos)
    D = dark_field(N, photons, rng_dark) if dark else None
    if D is not None:
        lam = lam + D[None].astype(np.float64)
    clamped = 0.0
    if noise and dtype == np.uint16:
        frames, clamped = poisson_u16(lam, rng_noise)
    elif noise:
        frames = np.minimum(rng_noise.poisson(lam), 65504).astype(dtype)
    else:
        frames = lam.astype(dtype)
    return dict(N=N, H=H, W=W, pos=pos, frames=frames, O_true=O_true, P_true=P_true,
                O0=np.ones((H, W), np.complex128), P0=initial_probe(N, R, sg, photons),
                dark=D, clamped=clamped, photons=photons, seed=seed)
