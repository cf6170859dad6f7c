"""The synthetic input recipe (no GPU): the stand-ins for the paper's data
have the stated shapes and statistics, and they are reproducible.

Scan geometry:
* the Fermat spiral follows r = c sqrt(k), theta = 137.508 deg k;
* geometry A's median nearest-neighbour distance is 0.35 x the probe FWHM;
* patches stay inside the object.

Probe:
* |P|^2 has the requested FWHM;
* the start probe obeys N^2 sum |P0|^2 = photons (Parseval).

Fields:
* the dark field averages 2% of the mean photons per pixel, within 1 +- 0.5.

Reproducibility:
* the frames do not depend on the number of worker processes;
* config 0 is a 16 x 16 raster with step 8 and +-1 jitter."""
import math

import numpy as np

from paper_2308_10674_gb300 import synth


def test_fermat_spiral_angles_and_radii():
    c = 3.0
    z = synth.fermat_spiral_centres(50, c)
    r = np.hypot(z[:, 0], z[:, 1])
    k = np.arange(50)
    assert np.allclose(r, c * np.sqrt(k))
    th = np.arctan2(z[:, 0], z[:, 1])
    d = np.mod(np.diff(th[1:]) - math.radians(137.508), 2 * math.pi)
    assert np.all(np.minimum(d, 2 * math.pi - d) < 1e-9)


def test_probe_fwhm_and_start_probe_scale():
    N, fwhm = 256, 60.0
    R = synth.probe_radius_for_fwhm(N, fwhm)
    P = synth.make_probe(N, R, 3.0 * R / 20.0)
    assert abs(synth.intensity_fwhm(P) - fwhm) <= 1.0
    P0 = synth.initial_probe(N, R, 3.0 * R / 20.0, 1e8)
    assert np.isclose(N * N * np.sum(np.abs(P0) ** 2), 1e8, rtol=1e-9)


def test_geometry_a_step_and_patches_inside():
    d = synth.live_scan(N=128, n=400, geometry="A", seed=1, fwhm=30.0, n_frames=8)
    z = synth.fermat_spiral_centres(400, d["spiral_c"])
    assert abs(synth.median_nn_distance(z) - 0.35 * 30.0) < 0.05 * 0.35 * 30.0
    pos = synth.centres_to_topleft(z, 128, 4)[0]
    assert pos.min() >= 0
    assert pos[:, 0].max() + 128 <= d["H"] and pos[:, 1].max() + 128 <= d["W"]


def test_dark_field_statistics():
    D = synth.dark_field(128, 1e8, synth.substream(0, 14))
    mean_px = 1e8 / (128 * 128)
    assert np.isclose(D.mean(), 0.02 * mean_px, rtol=0.1)
    assert D.min() >= 0.02 * mean_px * 0.5 - 1e-3 and D.max() <= 0.02 * mean_px * 1.5 + 1e-3


def test_frames_do_not_depend_on_the_worker_count():
    a = synth.live_scan(N=128, n=600, geometry="B", seed=3, fwhm=30.0, workers=1)
    b = synth.live_scan(N=128, n=600, geometry="B", seed=3, fwhm=30.0, workers=3)
    assert a["frames"].dtype == np.uint16 and a["frames"].shape == (600, 128, 128)
    assert np.array_equal(a["frames"], b["frames"]) and np.array_equal(a["pos"], b["pos"])


def test_config0_raster():
    d = synth.config0(seed=0)
    pos = d["pos"].astype(int)
    assert pos.shape == (256, 2)
    base = np.stack(np.meshgrid(np.arange(16) * 8, np.arange(16) * 8, indexing="ij"), -1)
    off = pos.reshape(16, 16, 2) - base
    assert off.min() >= off.max() - 2 and off.max() - off.min() <= 2  # one offset, jitter +-1
    assert d["frames"].shape == (256, 64, 64) and d["frames"].dtype == np.uint16
