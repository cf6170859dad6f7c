"""The hand-written tcgen05 GEMM (epie_tc_gemm_bf16, and epie_tc_gemm_tf32 on
fp32 operands read as tf32) against exact FP64 products of the same operand
values, and, used as a row DFT, against numpy's FFT.

D = sum_t A_t B_t^T with fp32 accumulation: every element must lie within
4 K 2^-24 (|A| |B|^T) of the exact product (the fp32 summation bound with
margin); a wrong operand layout, swizzle or descriptor gives O(1) errors.
Sizes cover several 128-row tiles, both column tile widths (256 and 128),
a k-loop longer than the 4-stage ring, a row pitch larger than the width and
the three-term split product."""
import numpy as np
import pytest

from paper_2308_10674_gb300 import _binding as B

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def to_bf16(x):
    """float32 -> bf16 bit patterns, round to nearest even."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return u.astype(np.uint16)


def from_bf16(b):
    return (b.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def split(x):
    hi = to_bf16(x)
    lo = to_bf16((np.asarray(x, np.float64) - from_bf16(hi)).astype(np.float32))
    return hi, lo


def tf32_hi(x):
    """x with its low 13 mantissa bits cleared: tf32-exact."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32) & np.uint32(0xFFFFE000)
    return u.view(np.float32)


def tf32_split(x):
    x = np.ascontiguousarray(x, np.float32)
    hi = tf32_hi(x)
    return hi, (x - hi).astype(np.float32)


def run(A0, A1, B0, B1, M, Nn, K, ldd, terms, tf32=False):
    dev = torch.device("cuda:0")
    if tf32:
        t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    else:
        t = lambda a: None if a is None else torch.from_numpy(a.view(np.int16)).to(dev)
    tA0, tA1, tB0, tB1 = t(A0), t(A1), t(B0), t(B1)
    D = torch.full((M, ldd), float("nan"), dtype=torch.float32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    ptr = lambda x: 0 if x is None else x.data_ptr()
    f = B.epie_tc_gemm_tf32 if tf32 else B.epie_tc_gemm_bf16
    f(ptr(tA0), ptr(tA1), ptr(tB0), ptr(tB1), D.data_ptr(), M, Nn, K, ldd, terms,
      status.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    D = D.cpu().numpy()
    if ldd > Nn:  # the pitch padding is never written
        assert np.isnan(D[:, Nn:]).all()
    return D[:, :Nn].astype(np.float64)


@pytest.mark.parametrize("M,Nn,K,ldd,terms", [
    (256, 256, 128, 256, 1),   # 2 row tiles, one 256-wide column tile
    (384, 512, 512, 512, 3),   # 24 k-blocks through a 4-stage ring, 2 column tiles
    (128, 384, 192, 400, 1),   # 128-wide column tiles, row pitch > width
    (640, 128, 64, 132, 3),    # one k-block per term
])
def test_tc_gemm_matches_exact_product(M, Nn, K, ldd, terms):
    rng = np.random.default_rng(M + Nn + K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    Bm = rng.standard_normal((Nn, K)).astype(np.float32)
    (A0, A1), (B0, B1) = split(A), split(Bm)
    if terms == 1:
        A1 = B1 = None
    D = run(A0, A1, B0, B1, M, Nn, K, ldd, terms)
    a0, b0 = from_bf16(A0), from_bf16(B0)
    ref = a0 @ b0.T
    absref = np.abs(a0) @ np.abs(b0).T
    if terms == 3:
        a1, b1 = from_bf16(A1), from_bf16(B1)
        ref = ref + a0 @ b1.T + a1 @ b0.T
        absref = absref + np.abs(a0) @ np.abs(b1).T + np.abs(a1) @ np.abs(b0).T
    bound = 4 * K * terms * 2.0 ** -24 * absref + 1e-30
    err = np.abs(D - ref)
    assert np.all(err <= bound), (float(err.max()), float((err / bound).max()))
    # and it is a real product, not a copy: the split product is far closer to
    # the fp32 inputs' product than the plain bf16 one
    if terms == 3:
        exact = A.astype(np.float64) @ Bm.astype(np.float64).T
        assert np.linalg.norm(D - exact) / np.linalg.norm(exact) < 1e-4


@pytest.mark.parametrize("N", [64, 128, 256])
def test_tc_gemm_as_row_dft(N):
    """Rows of interleaved complex values times the real 2N x 2N twiddle
    matrix are the rows' DFTs (numpy's FFT), to the split-bf16 accuracy."""
    rows = 256
    rng = np.random.default_rng(N)
    x = (rng.standard_normal((rows, N)) + 1j * rng.standard_normal((rows, N))).astype(np.complex64)
    X = x.view(np.float32).reshape(rows, 2 * N)
    k = np.arange(N)
    F = np.exp(-2j * np.pi * np.outer(k, k) / N)
    T = np.zeros((2 * N, 2 * N))
    T[0::2, 0::2], T[1::2, 0::2] = F.real, -F.imag
    T[0::2, 1::2], T[1::2, 1::2] = F.imag, F.real
    (X0, X1), (T0, T1) = split(X), split(T.T.astype(np.float32))
    D = run(X0, X1, T0, T1, rows, 2 * N, 2 * N, 2 * N, 3)
    got = D.reshape(rows, N, 2) @ np.array([1, 1j])
    ref = np.fft.fft(x.astype(np.complex128), axis=1)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-4


@pytest.mark.parametrize("M,Nn,K,ldd,terms", [
    (256, 256, 128, 256, 1),   # 4 k-blocks of 32
    (384, 512, 256, 512, 3),   # 24 k-blocks through the ring, 2 column tiles
    (128, 384, 96, 400, 1),    # 128-wide column tiles, row pitch > width
])
def test_tc_gemm_tf32_matches_exact_product(M, Nn, K, ldd, terms):
    """kind::tf32 on tf32-exact operands (hi and lo of a split both are): the
    result is the exact product up to fp32 summation."""
    rng = np.random.default_rng(M + Nn + K + 1)
    A = rng.standard_normal((M, K)).astype(np.float32)
    Bm = rng.standard_normal((Nn, K)).astype(np.float32)
    (A0, A1), (B0, B1) = tf32_split(A), tf32_split(Bm)
    A1, B1 = tf32_hi(A1), tf32_hi(B1)  # lo made tf32-exact too
    if terms == 1:
        A1 = B1 = None
    D = run(A0, A1, B0, B1, M, Nn, K, ldd, terms, tf32=True)
    a0, b0 = A0.astype(np.float64), B0.astype(np.float64)
    ref, absref = a0 @ b0.T, np.abs(a0) @ np.abs(b0).T
    if terms == 3:
        a1, b1 = A1.astype(np.float64), B1.astype(np.float64)
        ref = ref + a0 @ b1.T + a1 @ b0.T
        absref = absref + np.abs(a0) @ np.abs(b1).T + np.abs(a1) @ np.abs(b0).T
    bound = 4 * K * terms * 2.0 ** -24 * absref + 1e-30
    err = np.abs(D - ref)
    assert np.all(err <= bound), (float(err.max()), float((err / bound).max()))
    if terms == 3:  # about 21 significant bits of the fp32 inputs' product
        exact = A.astype(np.float64) @ Bm.astype(np.float64).T
        assert np.linalg.norm(D - exact) / np.linalg.norm(exact) < 1e-5


@pytest.mark.parametrize("N", [64, 256])
def test_tc_gemm_tf32_as_row_dft(N):
    """The split-tf32 product as a row DFT matches numpy's FFT to 1e-5."""
    rows = 256
    rng = np.random.default_rng(N + 7)
    x = (rng.standard_normal((rows, N)) + 1j * rng.standard_normal((rows, N))).astype(np.complex64)
    X = x.view(np.float32).reshape(rows, 2 * N)
    k = np.arange(N)
    F = np.exp(-2j * np.pi * np.outer(k, k) / N)
    T = np.zeros((2 * N, 2 * N))
    T[0::2, 0::2], T[1::2, 0::2] = F.real, -F.imag
    T[0::2, 1::2], T[1::2, 1::2] = F.imag, F.real
    (X0, X1), (T0, T1) = tf32_split(X), tf32_split(T.T.astype(np.float32))
    D = run(X0, X1, T0, T1, rows, 2 * N, 2 * N, 2 * N, 3, tf32=True)
    got = D.reshape(rows, N, 2) @ np.array([1, 1j])
    ref = np.fft.fft(x.astype(np.complex128), axis=1)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-5
