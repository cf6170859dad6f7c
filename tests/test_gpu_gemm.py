"""The tensor-core DFT path (EPIE_PATH_GEMM) against the FP64 oracle, one
coloured sweep from a well-conditioned textured start (tests/test_gpu_parity.py
explains why).  Bounds per operand precision, from its unit roundoff u
(bf16 2^-8, tf32 2^-11; the split bf16 product drops the lo*lo term, about
2^-16, the split tf32 product about 2^-21; the fp32 emulation is
fp32-accurate): relative L2 on object and probe
and relative error of the sweep error metric within about 8u.  The TC_*
precisions run the same products on the engine's own tcgen05 kernel; at
N = 64 odd colour classes exercise its padded last row block."""
import numpy as np
import pytest

from paper_2308_10674_gb300 import _binding as B
from paper_2308_10674_gb300 import synth

pytestmark = pytest.mark.gpu

BOUNDS = {B.EPIE_GEMM_FP32EMU: 1e-5, B.EPIE_GEMM_BF16X3: 1e-4, B.EPIE_GEMM_TF32: 3e-3,
          B.EPIE_GEMM_BF16: 3e-2, B.EPIE_GEMM_TC_BF16X3: 1e-4, B.EPIE_GEMM_TC_BF16: 3e-2,
          B.EPIE_GEMM_TC_TF32: 3e-3, B.EPIE_GEMM_TC_TF32X3: 1e-5}


def rel(a, b):
    return float(np.linalg.norm((np.asarray(a) - b).ravel()) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("prec", list(BOUNDS))
@pytest.mark.parametrize("N,ny,nx,step", [(64, 5, 7, 33), (128, 4, 5, 65), (256, 3, 4, 130)])
def test_gemm_path_one_sweep(orc, prec, N, ny, nx, step):
    d = synth.small_scan(N, ny, nx, step, seed=N)
    rng = np.random.default_rng(3)
    O0 = (d["O_true"] * (1 + 0.05 * synth.smooth_field(d["O_true"].shape, 2.0, rng)))
    P0 = (d["P_true"] * (1 + 0.05 * synth.smooth_field(d["P_true"].shape, 2.0, rng)))
    O0 = O0.astype(np.complex64).astype(complex)
    P0 = P0.astype(np.complex64).astype(complex)
    with B.Engine(N, d["H"], d["W"], P0, O0, capacity=len(d["pos"]), mode=B.EPIE_COLOURED,
                  seed=5, device=0, path=B.EPIE_PATH_GEMM, gemm_precision=prec) as eng:
        eng.append(d["frames"], d["pos"])
        e_g = eng.iterate(1)
        O_g, P_g = eng.object(), eng.probe()
    O, P = O0.copy(), P0.copy()
    e = orc.run_sweeps(O, P, orc.prepare_intensity(d["frames"]), d["pos"], 1, N, seed=5,
                       mode=orc.COLOURED)
    tol = BOUNDS[prec]
    errs = (rel(O_g, O), rel(P_g, P), abs(e_g[0] - e[0]) / e[0])
    assert max(errs) <= tol, (prec, errs)
