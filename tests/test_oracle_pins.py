"""Pins of the FP64 oracle against facts fixed by mathematics and by the
method's definition (no GPU).  Each test names the plausible oracle mistake
it would catch.

Method: ePIE (Maiden & Rodenburg 2009) as run by the paper's engine (Sec.
"ePIE Implementation"): exit wave, DFT, modulus replacement, inverse DFT,
simultaneous object and illumination update with alpha = beta = 1.
"""
import math
import os

import numpy as np
import pytest

from paper_2308_10674_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def crandn(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


# --------------------------------------------------------------------------- transforms

@pytest.mark.parametrize("n", [2, 4, 8, 16])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft_equals_brute_dft(orc, n, sign):
    """Own FFT = DFT from its definition (wrong twiddle / bit reversal / scale)."""
    a = crandn(np.random.default_rng(n), (n, n))
    assert rel(orc.fft2(a, sign), orc.dft2_brute(a, sign)) <= 1e-13


@pytest.mark.parametrize("n", [64, 128, 256, 512])
def test_fft_equals_library_fft(orc, n):
    """Own FFT = numpy's pocketfft on the engine's frame sizes."""
    a = crandn(np.random.default_rng(n), (n, n))
    assert rel(orc.fft2(a, -1), np.fft.fft2(a)) <= 1e-13
    assert rel(orc.fft2(a, +1), np.fft.ifft2(a)) <= 1e-13


def test_fft_single_plane_wave(orc):
    """exp(+2 pi i (a y + b x)/N) transforms to N^2 at (ky, kx) = (a, b):
    fixes the sign convention and the row/column order without a library."""
    n, a, b = 32, 3, 7
    y, x = np.mgrid[0:n, 0:n]
    f = np.exp(2j * math.pi * (a * y + b * x) / n)
    F = orc.fft2(f, -1)
    expect = np.zeros((n, n), complex)
    expect[a, b] = n * n
    assert np.abs(F - expect).max() <= 1e-9


def test_parseval_and_roundtrip(orc):
    n = 128
    a = crandn(np.random.default_rng(5), (n, n))
    F = orc.fft2(a, -1)
    assert abs(np.sum(np.abs(a) ** 2) - np.sum(np.abs(F) ** 2) / n ** 2) <= 1e-13 * np.sum(np.abs(a) ** 2)
    assert rel(orc.fft2(F, +1), a) <= 1e-14


# --------------------------------------------------------------------------- intensities

def test_prepare_intensity_shift_dark_and_types(orc):
    """DC-centred pixel (N/2 + dy, N/2 + dx) lands at FFT index (dy, dx) mod N;
    dark is subtracted and negatives clamp to 0; binary16 decodes exactly."""
    N = 8
    fr = np.zeros((1, N, N), np.uint16)
    fr[0, N // 2, N // 2] = 100
    fr[0, N // 2 + 1, N // 2 + 3] = 7
    fr[0, 0, 0] = 9            # most negative frequency (-N/2, -N/2) -> index (N/2, N/2)
    I = orc.prepare_intensity(fr)[0]
    assert I[0, 0] == 100 and I[1, 3] == 7 and I[N // 2, N // 2] == 9 and I.sum() == 116
    dark = np.full((N, N), 8.0, np.float32)
    I2 = orc.prepare_intensity(fr, dark)[0]
    assert I2[0, 0] == 92 and I2[1, 3] == 0 and I2[N // 2, N // 2] == 1 and I2.sum() == 93
    h = np.zeros((1, N, N), np.float16)
    h[0, N // 2, N // 2] = np.float16(65504.0)
    h[0, N // 2, N // 2 + 1] = np.frombuffer(np.uint16(1).tobytes(), np.float16)[0]  # 2^-24
    h[0, N // 2, N // 2 + 2] = np.float16(-2.0)
    h[0, N // 2, N // 2 + 3] = np.float16(2049.0)  # rounds to 2048 in binary16
    Ih = orc.prepare_intensity(h)[0]
    assert Ih[0, 0] == 65504.0 and Ih[0, 1] == 2.0 ** -24 and Ih[0, 2] == 0.0 and Ih[0, 3] == 2048.0
    f = np.arange(N * N, dtype=np.float32).reshape(1, N, N) + 0.25
    fn = f.copy()
    fn[0, N // 2, N // 2] = np.nan
    assert orc.prepare_intensity(fn)[0][0, 0] == 0.0  # NaN clamps to 0 like negatives
    If = orc.prepare_intensity(f)[0]
    assert np.array_equal(If, np.fft.ifftshift(f[0]).astype(np.float64))


def test_modulus_projection(orc):
    """|proj(Psi)| = sqrt(I); idempotent; tie rule u(0) = 1; error terms."""
    rng = np.random.default_rng(3)
    Psi = crandn(rng, (16, 16))
    Psi[2, 5] = 0.0
    I = rng.uniform(0, 10, (16, 16))
    Q, e, s = orc.modulus_project(Psi, I)
    assert np.allclose(np.abs(Q), np.sqrt(I), rtol=1e-14, atol=0)
    assert Q[2, 5] == np.sqrt(I[2, 5])
    Q2, e2, _ = orc.modulus_project(Q, I)
    assert rel(Q2, Q) <= 1e-15 and e2 <= 1e-25 * s
    assert np.allclose(np.angle(Q[np.abs(Psi) > 0]), np.angle(Psi[np.abs(Psi) > 0]), atol=1e-13)
    assert abs(e - np.sum((np.abs(Psi) - np.sqrt(I)) ** 2)) <= 1e-12 * e
    assert abs(s - I.sum()) <= 1e-12 * s


# --------------------------------------------------------------------------- one step

def test_step_closed_form_flat_probe(orc):
    """Flat probe c over a flat patch o: psi = c o, Psi = K c o delta(k).  With
    I = A^2 at DC and B^2 at k0 = (1, 3), the replaced wave is
    psi' = (A u + B exp(+2 pi i k0.r/N)) / K, u = co/|co| (B via u(0) = 1), so
    O' = o + alpha conj(c)/|c|^2 (psi' - co), P' = c + beta conj(o)/|o|^2 (psi' - co).
    Catches: conj on the wrong factor, wrong normaliser, missing 1/K, flipped
    transform sign, transposed frequency or patch index, wrong tie rule."""
    N, H, W, y0, x0 = 16, 40, 48, 5, 19
    rng = np.random.default_rng(11)
    c, o = 0.7 - 0.4j, 0.3 + 0.9j
    A, B, alpha, beta = 3.0, 1.5, 0.8, 0.6
    K = N * N
    O = crandn(rng, (H, W))
    O[y0:y0 + N, x0:x0 + N] = o
    P = np.full((N, N), c, complex)
    I = np.zeros((N, N))
    I[0, 0], I[1, 3] = A * A, B * B
    O1, P1, e, s = orc.epie_step(O, P, I, y0, x0, alpha, beta)
    y, x = np.mgrid[0:N, 0:N]
    u = c * o / abs(c * o)
    psi1 = (A * u + B * np.exp(2j * math.pi * (1 * y + 3 * x) / N)) / K
    d = psi1 - c * o
    O_exp = O.copy()
    O_exp[y0:y0 + N, x0:x0 + N] = o + alpha * np.conj(c) / abs(c) ** 2 * d
    P_exp = c + beta * np.conj(o) / abs(o) ** 2 * d
    assert np.abs(O1 - O_exp).max() <= 1e-13
    assert np.abs(P1 - P_exp).max() <= 1e-13
    assert abs(e - ((K * abs(c * o) - A) ** 2 + B * B)) <= 1e-9 * e
    assert s == A * A + B * B


def test_step_global_object_max(orc):
    """omax_global divides the probe update by the maximum over the whole object."""
    N, H, W = 8, 20, 20
    rng = np.random.default_rng(2)
    c, o, big = 1.0 + 0.5j, 0.5 - 0.2j, 3.0
    O = np.full((H, W), o, complex)
    O[0, 0] = big  # outside the patch at (6, 7)
    P = np.full((N, N), c, complex)
    I = np.zeros((N, N))
    I[0, 0] = 5.0
    _, P1, _, _ = orc.epie_step(O, P, I, 6, 7, 1.0, 1.0, omax_global=True)
    d = 5.0 ** 0.5 * (c * o / abs(c * o)) / (N * N) - c * o
    assert np.abs(P1 - (c + np.conj(o) / big ** 2 * d)).max() <= 1e-14
    assert rng is not None


def _truth_instance(N=32, seed=4):
    rng = np.random.default_rng(seed)
    H, W = 70, 90
    O = synth.make_object(H, W, 2.0, rng) * rng.uniform(0.9, 1.1)
    P = synth.make_probe(N, 9.0, 1.5) * (3.0 + 1.0j)
    pos = np.array([[3, 17], [20, 41], [35, 5], [11, 50], [30, 30]], np.int32)
    lam = synth.far_field_intensity(O, P, pos)          # numpy FFT, DC-centred
    I_all = np.fft.ifftshift(lam, axes=(-2, -1))        # shift pinned above
    return O, P, pos, I_all


def test_truth_is_fixed_point(orc):
    """At the true (O, P) on noiseless data Delta = 0: one step and whole
    sweeps leave the state unchanged and the error is zero.  The data come
    from numpy's FFT, so a sign / transpose / shift mistake in the oracle's
    forward model would break the fixed point."""
    O, P, pos, I_all = _truth_instance()
    for j, (y, x) in enumerate(pos):
        O1, P1, e, s = orc.epie_step(O, P, I_all[j], y, x)
        assert rel(O1, O) <= 1e-12 and rel(P1, P) <= 1e-12
        assert e <= 1e-24 * s
    O2, P2 = O.copy(), P.copy()
    errs = orc.run_sweeps(O2, P2, I_all, pos, 2, 32, seed=9)
    assert rel(O2, O) <= 1e-12 and rel(P2, P) <= 1e-12
    assert max(errs) <= 1e-24


def test_zero_strengths_change_nothing(orc):
    O, P, pos, I_all = _truth_instance()
    O0 = np.ones_like(O)
    O1, P1, e, s = orc.epie_step(O0, P * 0.5, I_all[1], pos[1][0], pos[1][1], 0.0, 0.0)
    assert np.array_equal(O1, O0) and np.array_equal(P1, P * 0.5) and e > 0


def test_zero_probe_turns_object_update_off(orc):
    """max|P|^2 = 0 or max|O_j|^2 = 0: the matching update is taken as zero (R4)."""
    N = 8
    O = np.zeros((12, 12), complex)
    P = np.zeros((N, N), complex)
    I = np.ones((N, N))
    O1, P1, _, _ = orc.epie_step(O, P, I, 2, 3)
    assert np.array_equal(O1, O) and np.array_equal(P1, P)


# --------------------------------------------------------------------------- sweeps

def test_sequential_error_drops_on_simulated_data(orc):
    """Noiseless simulated config-0 data from the flat start: the error metric
    falls at least 10x over 10 sweeps and its 3-sweep running mean falls
    monotonically (ePIE is not a descent method, so single sweeps may not)."""
    d = synth.config0(seed=0)
    I_all = np.fft.ifftshift(synth.far_field_intensity(d["O_true"], d["P_true"], d["pos"]),
                             axes=(-2, -1))
    O, P = d["O0"].copy(), d["P0"].copy()
    errs = orc.run_sweeps(O, P, I_all, d["pos"], 10, d["N"], seed=0)
    run = np.convolve(errs, np.ones(3) / 3, mode="valid")
    assert errs[-1] * 10 <= errs[0], errs
    assert np.all(np.diff(run) < 0), errs


def test_untouched_pixels_stay_initial(orc):
    """Object pixels no patch covers keep their initial value exactly
    (paper, Discussion: regions never illuminated stay at their initial values)."""
    d = synth.config0(seed=1)
    I_all = orc.prepare_intensity(d["frames"])
    O, P = d["O0"].copy(), d["P0"].copy()
    orc.run_sweeps(O, P, I_all, d["pos"], 2, d["N"], seed=1)
    cover = np.zeros(O.shape, bool)
    for y, x in d["pos"]:
        cover[y:y + 64, x:x + 64] = True
    assert (~cover).sum() > 0
    assert np.all(O[~cover] == 1.0)
    assert np.all(O[cover] != 1.0)


def _sparse_instance(N=16, seed=6, step=None):
    rng = np.random.default_rng(seed)
    step = step or N // 2
    pos = synth.raster_positions(4, 5, step, 2, 1, rng)
    H = int(pos[:, 0].max()) + N + 3
    W = int(pos[:, 1].max()) + N + 3
    O_true = synth.make_object(H, W, 2.0, rng)
    P_true = synth.make_probe(N, N * 0.3, 1.0) * 40
    I_all = np.fft.ifftshift(synth.far_field_intensity(O_true, P_true, pos), axes=(-2, -1))
    P0 = np.abs(synth.make_probe(N, N * 0.3, 1.0)).astype(complex) * 40
    return pos, I_all, np.ones((H, W), complex), P0


def test_coloured_equals_sequential_for_object_when_beta_zero(orc):
    """C4(i): with beta = 0 coloured ePIE gives the same object as sequential
    ePIE in the concatenated colouring order."""
    N = 16
    pos, I_all, O0, P0 = _sparse_instance(N)
    col, ncls = orc.colour_greedy(pos, N)
    assert ncls > 1 and np.bincount(col).max() > 1
    order, gs = orc.order_coloured(5, 0, col, ncls)
    Oc, Pc = O0.copy(), P0.copy()
    orc.sweep_groups(Oc, Pc, I_all, pos, order, gs, beta=0.0)
    Os, Ps = O0.copy(), P0.copy()
    orc.sweep_groups(Os, Ps, I_all, pos, order, orc.sequential_groups(order), beta=0.0)
    assert rel(Oc, Os) <= 1e-14 and np.array_equal(Pc, P0)


def test_coloured_equals_sequential_when_classes_are_single(orc):
    """C4(ii): when every colour class has one member (here six positions that
    all overlap pairwise), coloured ePIE equals sequential ePIE for O and P."""
    N = 16
    pos2 = np.stack([np.arange(6) * 3 + 2, np.full(6, 4)], 1).astype(np.int32)
    col2, ncls2 = orc.colour_greedy(pos2, N)
    assert ncls2 == 6
    H, W = int(pos2[:, 0].max()) + N + 2, 30
    rng = np.random.default_rng(1)
    O_true = synth.make_object(H, W, 2.0, rng)
    Pt = synth.make_probe(N, 5.0, 1.0) * 30
    I2 = np.fft.ifftshift(synth.far_field_intensity(O_true, Pt, pos2), axes=(-2, -1))
    order, gs = orc.order_coloured(3, 1, col2, ncls2)
    Oa, Pa = np.ones((H, W), complex), np.abs(Pt).astype(complex)
    Ob, Pb = Oa.copy(), Pa.copy()
    orc.sweep_groups(Oa, Pa, I2, pos2, order, gs)
    orc.sweep_groups(Ob, Pb, I2, pos2, order, orc.sequential_groups(order))
    assert rel(Oa, Ob) <= 1e-14 and rel(Pa, Pb) <= 1e-14


def test_parallel_one_subset_is_the_plain_sweep(orc):
    """The paper's parallel scheme with a single subset: R rounds of k sweeps
    are R*k plain sweeps (catches a sweep counter that restarts every round,
    or a wrong order stream)."""
    N = 16
    pos, I_all, O0, P0 = _sparse_instance(N)
    Oa, Pa = O0.copy(), P0.copy()
    orc.run_parallel_average(Oa, Pa, I_all, pos, [np.arange(len(pos))], 2, 3, N, seed=4)
    Ob, Pb = O0.copy(), P0.copy()
    orc.run_sweeps(Ob, Pb, I_all, pos, 6, N, seed=4)
    assert np.array_equal(Oa, Ob) and np.array_equal(Pa, Pb)


def test_parallel_average_of_disjoint_positions_is_a_half_step(orc):
    """Two subsets of one position each, patches disjoint, beta = 0: each copy
    moves only its own patch, and the object update is linear in alpha, so
    the average equals one sequential sweep over both positions with alpha/2
    (catches copies that share state, a missing or wrong divisor).  Two
    copies of the same position average to that position's single step."""
    N = 16
    pos, I_all, O0, P0 = _sparse_instance(N, step=N + 2)
    a, b = 0, len(pos) - 1
    assert abs(int(pos[a, 0]) - int(pos[b, 0])) >= N or abs(int(pos[a, 1]) - int(pos[b, 1])) >= N
    Op, Pp = O0.copy(), P0.copy()
    orc.run_parallel_average(Op, Pp, I_all, pos, [np.array([a]), np.array([b])], 1, 1, N,
                             seed=2, beta=0.0)
    Oh, Ph = O0.copy(), P0.copy()
    two = np.array([a, b])
    orc.run_sweeps(Oh, Ph, I_all[two], pos[two], 1, N, seed=7, alpha=0.5, beta=0.0)
    assert rel(Op, Oh) <= 1e-14 and np.array_equal(Pp, P0) and not np.array_equal(Op, O0)
    Os, Ps = O0.copy(), P0.copy()
    orc.run_parallel_average(Os, Ps, I_all, pos, [np.array([a]), np.array([a])], 1, 1, N, seed=2)
    O1, P1 = O0.copy(), P0.copy()
    orc.run_sweeps(O1, P1, I_all[[a]], pos[[a]], 1, N, seed=0)
    assert rel(Os, O1) <= 1e-15 and rel(Ps, P1) <= 1e-15


def test_group_members_must_not_overlap(orc):
    N = 16
    pos, I_all, O0, P0 = _sparse_instance(N)
    with pytest.raises(ValueError):
        orc.sweep_groups(O0.copy(), P0.copy(), I_all, pos, np.arange(len(pos)),
                         np.array([0, len(pos)]))


def test_minibatch_reductions(orc):
    """C5: batch 1 = sequential; a batch of mutually disjoint patches =
    coloured ePIE with the mean probe move."""
    N = 16
    pos, I_all, O0, P0 = _sparse_instance(N)
    order = orc.order_sequential(2, 0, len(pos))
    Oa, Pa = O0.copy(), P0.copy()
    orc.sweep_minibatch(Oa, Pa, I_all, pos, order, 1)
    Ob, Pb = O0.copy(), P0.copy()
    orc.sweep_groups(Ob, Pb, I_all, pos, order, orc.sequential_groups(order))
    assert rel(Oa, Ob) <= 1e-14 and rel(Pa, Pb) <= 1e-14
    col, ncls = orc.colour_greedy(pos, N)
    order, gs = orc.order_coloured(2, 0, col, ncls)
    sizes = np.diff(gs)
    k = int(np.argmax(sizes))
    sub = order[gs[k]:gs[k + 1]]
    Oc, Pc = O0.copy(), P0.copy()
    orc.sweep_minibatch(Oc, Pc, I_all, pos, sub, len(sub))
    Od, Pd = O0.copy(), P0.copy()
    orc.sweep_groups(Od, Pd, I_all, pos, sub, np.array([0, len(sub)]))
    assert rel(Oc, Od) <= 1e-14 and rel(Pc, Pd) <= 1e-14


def test_minibatch_overlap_count_normalisation(orc):
    """Two identical positions in one batch: the object moves by the average of
    two identical updates, i.e. once; the probe moves by the mean, i.e. once."""
    N = 16
    pos, I_all, O0, P0 = _sparse_instance(N)
    pos2 = np.array([pos[3], pos[3]], np.int32)
    I2 = np.stack([I_all[3], I_all[3]])
    Oa, Pa = O0.copy(), P0.copy()
    orc.sweep_minibatch(Oa, Pa, I2, pos2, np.array([0, 1]), 2)
    Ob, Pb = O0.copy(), P0.copy()
    orc.sweep_minibatch(Ob, Pb, I2[:1], pos2[:1], np.array([0]), 1)
    assert rel(Oa, Ob) <= 1e-15 and rel(Pa, Pb) <= 1e-15


def _flat_batch_instance(N=16, H=40, W=60):
    """Two disjoint flat patches under a flat probe, with intensities that put
    A_j^2 at DC and B_j^2 at one other frequency k_j per frame.  Returns the
    instance and the closed-form replaced exit waves psi1_j (see
    test_step_closed_form_flat_probe)."""
    rng = np.random.default_rng(17)
    c = 0.7 - 0.4j
    pos = np.array([[3, 2], [5, 2 + N + 9]], np.int32)          # disjoint patches
    o = [0.3 + 0.9j, -0.6 + 0.2j]
    A, B = [3.0, 2.2], [1.5, 0.7]
    k = [(1, 3), (4, 1)]
    K = N * N
    O = crandn(rng, (H, W))
    for (y0, x0), oj in zip(pos, o):
        O[y0:y0 + N, x0:x0 + N] = oj
    P = np.full((N, N), c, complex)
    I_all = np.zeros((2, N, N))
    y, x = np.mgrid[0:N, 0:N]
    psi1 = []
    for j in range(2):
        I_all[j, 0, 0], I_all[j, k[j][0], k[j][1]] = A[j] ** 2, B[j] ** 2
        u = c * o[j] / abs(c * o[j])
        psi1.append((A[j] * u + B[j] * np.exp(2j * math.pi * (k[j][0] * y + k[j][1] * x) / N)) / K)
    return O, P, I_all, pos, c, o, psi1


def test_minibatch_alpha_beta_closed_form(orc):
    """C5 at alpha = 0.5, beta = 0.3 on a batch of two disjoint flat patches
    under a flat probe: every pixel is covered once, so each patch moves by
    alpha conj(c)/|c|^2 d_j and the probe by the mean of beta conj(o_j)/|o_j|^2 d_j.
    Planted mistakes this catches: alpha applied twice (alpha/max|P|^2 in the
    accumulator and alpha again when applying it), beta dropped or applied to
    the object, the probe moved by the sum instead of the mean."""
    N = 16
    O, P, I_all, pos, c, o, psi1 = _flat_batch_instance(N)
    alpha, beta = 0.5, 0.3
    O1, P1 = O.copy(), P.copy()
    orc.sweep_minibatch(O1, P1, I_all, pos, np.array([0, 1]), 2, alpha=alpha, beta=beta)
    O_exp = O.copy()
    dP = np.zeros((N, N), complex)
    for j, (y0, x0) in enumerate(pos):
        d = psi1[j] - c * o[j]
        O_exp[y0:y0 + N, x0:x0 + N] = o[j] + alpha * np.conj(c) / abs(c) ** 2 * d
        dP += beta * np.conj(o[j]) / abs(o[j]) ** 2 * d
    assert np.abs(O1 - O_exp).max() <= 1e-13
    assert np.abs(P1 - (c + dP / 2)).max() <= 1e-13


def test_minibatch_alpha_beta_reductions(orc):
    """C5 at alpha = 0.5, beta = 0.3: (i) a batch of disjoint patches equals the
    coloured group update at the same strengths (mean probe move); (ii) two
    copies of one position in a batch equal that position's single ePIE step
    (count normalisation and probe mean both undo the duplication).  With
    alpha applied twice the first part fails; with the count or the mean
    missing the second does."""
    N = 16
    alpha, beta = 0.5, 0.3
    pos, I_all, O0, P0 = _sparse_instance(N)
    col, ncls = orc.colour_greedy(pos, N)
    order, gs = orc.order_coloured(2, 0, col, ncls)
    kk = int(np.argmax(np.diff(gs)))
    sub = order[gs[kk]:gs[kk + 1]]
    assert len(sub) > 1
    Oa, Pa = O0.copy(), P0.copy()
    orc.sweep_minibatch(Oa, Pa, I_all, pos, sub, len(sub), alpha=alpha, beta=beta)
    Ob, Pb = O0.copy(), P0.copy()
    orc.sweep_groups(Ob, Pb, I_all, pos, sub, np.array([0, len(sub)]), alpha=alpha, beta=beta)
    assert rel(Oa, Ob) <= 1e-14 and rel(Pa, Pb) <= 1e-14 and rel(Oa, O0) > 1e-3
    pos2 = np.array([pos[3], pos[3]], np.int32)
    I2 = np.stack([I_all[3], I_all[3]])
    Oc, Pc = O0.copy(), P0.copy()
    orc.sweep_minibatch(Oc, Pc, I2, pos2, np.array([0, 1]), 2, alpha=alpha, beta=beta)
    O1, P1, _, _ = orc.epie_step(O0, P0, I_all[3], pos[3][0], pos[3][1], alpha, beta)
    assert rel(Oc, O1) <= 1e-14 and rel(Pc, P1) <= 1e-14


def test_probe_sum_closed_form_multi_member(orc):
    """Coloured group update with probe_mean off (the EPIE_PROBE_SUM reading):
    a class of two disjoint flat patches under a flat probe moves the probe by
    the SUM of beta conj(o_j)/|o_j|^2 d_j, and each patch as in the single
    step.  Planted mistake it catches: the mean taken regardless of the flag
    (or the flag inverted)."""
    N = 16
    O, P, I_all, pos, c, o, psi1 = _flat_batch_instance(N)
    alpha, beta = 0.8, 0.6
    O1, P1 = O.copy(), P.copy()
    orc.sweep_groups(O1, P1, I_all, pos, np.array([0, 1]), np.array([0, 2]), alpha=alpha,
                     beta=beta, probe_mean=False)
    O_exp = O.copy()
    dP = np.zeros((N, N), complex)
    for j, (y0, x0) in enumerate(pos):
        d = psi1[j] - c * o[j]
        O_exp[y0:y0 + N, x0:x0 + N] = o[j] + alpha * np.conj(c) / abs(c) ** 2 * d
        dP += beta * np.conj(o[j]) / abs(o[j]) ** 2 * d
    assert np.abs(O1 - O_exp).max() <= 1e-13
    assert np.abs(P1 - (c + dP)).max() <= 1e-13
    P2 = P.copy()
    orc.sweep_groups(O.copy(), P2, I_all, pos, np.array([0, 1]), np.array([0, 2]), alpha=alpha,
                     beta=beta, probe_mean=True)
    assert np.abs(P2 - (c + dP / 2)).max() <= 1e-13


def test_group_global_object_max_single_members(orc):
    """omax_global in a sweep of one-member groups equals the chain of single
    ePIE steps with the global maximum (whose closed form is pinned in
    test_step_global_object_max).  Catches a group-level global maximum read
    from the wrong array (the probe, or the patch)."""
    N = 16
    pos, I_all, O0, P0 = _sparse_instance(N)
    O0 = O0 * np.exp(0.3j) * np.linspace(0.5, 1.5, O0.size).reshape(O0.shape)
    order = orc.order_sequential(3, 0, len(pos))
    Oa, Pa = O0.copy(), P0.copy()
    orc.sweep_groups(Oa, Pa, I_all, pos, order, orc.sequential_groups(order), omax_global=True)
    Ob, Pb = O0.copy(), P0.copy()
    for j in order:
        Ob, Pb, _, _ = orc.epie_step(Ob, Pb, I_all[j], pos[j][0], pos[j][1], omax_global=True)
    assert rel(Oa, Ob) <= 1e-14 and rel(Pa, Pb) <= 1e-14
    Oc, Pc = O0.copy(), P0.copy()
    orc.sweep_groups(Oc, Pc, I_all, pos, order, orc.sequential_groups(order))
    assert rel(Pc, Pa) > 1e-6  # the patch maximum gives another probe


def test_group_global_object_max_taken_at_class_start(orc):
    """omax_global in a class of two disjoint members: the maximum is the
    object's at class start (reading R4), so each member's probe move equals
    a single step from the class-start object with the global maximum, and
    the probe moves by their mean.  The object's largest pixel sits in the
    first member's patch and that member's update shrinks it, so a maximum
    re-read after the first member (from the current object) fails here."""
    N = 16
    O, P, I_all, pos, c, o, psi1 = _flat_batch_instance(N)
    y0, x0 = pos[0]
    O[y0 + 2, x0 + 5] = 4.0 + 3.0j                      # |.|^2 = 25, the global maximum
    O[:, :] = np.where(np.abs(O) > 5.0, O / np.abs(O) * 4.5, O)
    O[y0 + 2, x0 + 5] = 4.0 + 3.0j
    assert np.argmax(np.abs(O)) == (y0 + 2) * O.shape[1] + x0 + 5
    I_all = I_all.copy()
    I_all[0] *= 0.01                                    # the update pulls the patch down
    O1, P1 = O.copy(), P.copy()
    orc.sweep_groups(O1, P1, I_all, pos, np.array([0, 1]), np.array([0, 2]), omax_global=True)
    O_exp, dP = O.copy(), np.zeros_like(P)
    for j, (yy, xx) in enumerate(pos):
        Oj, Pj, _, _ = orc.epie_step(O, P, I_all[j], yy, xx, omax_global=True)
        O_exp[yy:yy + N, xx:xx + N] = Oj[yy:yy + N, xx:xx + N]
        dP += Pj - P
    assert rel(O1, O_exp) <= 1e-14 and rel(P1, P + dP / 2) <= 1e-14
    # the teeth: after the first member the object maximum is smaller
    Oa, _, _, _ = orc.epie_step(O, P, I_all[0], y0, x0, omax_global=True)
    assert np.max(np.abs(Oa) ** 2) < 0.9 * np.max(np.abs(O) ** 2)


# --------------------------------------------------------------------------- order, colouring

def test_splitmix64_golden(orc):
    with open(os.path.join(HERE, "golden", "splitmix64_seed0.txt")) as f:
        want = [int(l, 16) for l in f if l.strip() and not l.startswith("#")]
    assert orc.splitmix64_stream(0, len(want)) == want


def test_orders_are_permutations_and_change_per_sweep(orc):
    n = 257
    o0 = orc.order_sequential(7, 0, n)
    o1 = orc.order_sequential(7, 1, n)
    assert sorted(o0) == list(range(n)) and sorted(o1) == list(range(n))
    assert not np.array_equal(o0, o1)
    assert np.array_equal(o0, orc.order_sequential(7, 0, n))


def test_colouring_valid_and_first_fit(orc):
    """Members of a class never conflict, and each frame's class is the
    smallest one free of earlier conflicting frames (first-fit)."""
    rng = np.random.default_rng(0)
    N = 32
    pos = rng.integers(0, 200, size=(300, 2)).astype(np.int32)
    col, ncls = orc.colour_greedy(pos, N)
    conf = (np.abs(pos[:, None, 0] - pos[None, :, 0]) < N) & (np.abs(pos[:, None, 1] - pos[None, :, 1]) < N)
    np.fill_diagonal(conf, False)
    same = col[:, None] == col[None, :]
    assert not np.any(conf & same)
    for i in range(len(pos)):
        earlier = set(col[:i][conf[i, :i]].tolist())
        assert col[i] == min(set(range(ncls + 1)) - earlier)
    order, gs = orc.order_coloured(1, 3, col, ncls)
    assert sorted(order) == list(range(len(pos)))
    # with a cap: classes stay valid, none exceeds the cap, and first-fit now
    # skips full classes as well as conflicting ones
    capc, ncap = orc.colour_greedy(pos, N, cap=5)
    assert np.bincount(capc).max() <= 5 and ncap >= ncls
    assert not np.any(conf & (capc[:, None] == capc[None, :]))
    for i in range(len(pos)):
        blocked = set(capc[:i][conf[i, :i]].tolist())
        blocked |= {c for c in set(capc[:i].tolist()) if np.sum(capc[:i] == c) >= 5}
        assert capc[i] == min(set(range(ncap + 1)) - blocked)
    for g in range(ncls):
        members = order[gs[g]:gs[g + 1]]
        assert len(set(col[members].tolist())) == 1


# --------------------------------------------------------------------------- amplitude-loss gradient

def test_amp_loss_gradient_matches_finite_differences(orc):
    """Gradient of sum_j || |F(S_dj P . O_j)| - sqrt(I_j) ||^2 wrt O, P and the
    sub-pixel shifts against FP64 central differences (h = 1e-6), on a 32x32,
    16-position instance."""
    rng = np.random.default_rng(8)
    N = 32
    pos = synth.raster_positions(4, 4, 6, 1, 0, rng)
    H = W = int(pos.max()) + N + 2
    O = synth.make_object(H, W, 2.0, rng)
    P = synth.make_probe(N, 9.0, 1.5) / 30.0
    I_all = rng.uniform(0.0, 4.0, (len(pos), N, N)) * np.abs(np.fft.fft2(P)) ** 2 / 8
    shift = rng.uniform(-0.5, 0.5, (len(pos), 2))
    L, gO, gP, gd = orc.amp_loss_grad(O, P, I_all, pos, shift)
    h = 1e-6
    # central differences carry rounding noise of about eps * L / h
    noise = 50 * np.finfo(float).eps * L / h

    def f(O_, P_, s_):
        return orc.amp_loss_grad(O_, P_, I_all, pos, s_)[0]

    for (yy, xx) in [(pos[5][0] + 3, pos[5][1] + 7), (pos[0][0] + 10, pos[0][1] + 2)]:
        for unit, part in ((1.0, np.real), (1j, np.imag)):
            Op, Om = O.copy(), O.copy()
            Op[yy, xx] += unit * h
            Om[yy, xx] -= unit * h
            fd = (f(Op, P, shift) - f(Om, P, shift)) / (2 * h)
            assert abs(fd - part(gO[yy, xx])) <= 1e-6 * abs(fd) + noise, (fd, gO[yy, xx])
    for (yy, xx) in [(16, 16), (12, 20)]:
        for unit, part in ((1.0, np.real), (1j, np.imag)):
            Pp, Pm = P.copy(), P.copy()
            Pp[yy, xx] += unit * h
            Pm[yy, xx] -= unit * h
            fd = (f(O, Pp, shift) - f(O, Pm, shift)) / (2 * h)
            assert abs(fd - part(gP[yy, xx])) <= 1e-6 * abs(fd) + noise, (fd, gP[yy, xx])
    for j in (0, 9):
        for ax in (0, 1):
            sp, sm = shift.copy(), shift.copy()
            sp[j, ax] += h
            sm[j, ax] -= h
            fd = (f(O, P, sp) - f(O, P, sm)) / (2 * h)
            assert abs(fd - gd[j, ax]) <= 1e-6 * abs(fd) + noise, (fd, gd[j, ax])
            assert abs(gd[j, ax]) > 100 * noise
