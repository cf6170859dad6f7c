"""The bounded device waits and their error path, exercised without any GPU
fault: a bulk copy that the host tells the kernel not to issue leaves its
mbarrier incomplete, the wait for it gives up after a short limit (1 ms
here), the kernel records the expiry in its status word, finishes without
anything in flight, frees its tensor memory and returns.

* Step kernel: epie_iterate returns EPIE_ETIMEOUT, every later call on the
  handle returns EPIE_ESTATE, and the device stays usable (a new handle runs
  a normal sweep).
* tcgen05 GEMM: the status word carries bit 2 after the call, and the next
  call (no injection) computes the exact product with a clean status."""
import numpy as np
import pytest

from paper_2308_10674_gb300 import _binding as B
from paper_2308_10674_gb300 import synth

pytestmark = pytest.mark.gpu
WAIT_NS = 1_000_000  # 1 ms


@pytest.mark.parametrize("N,ny,nx,step,shape", [(64, 3, 3, 33, 0), (128, 3, 3, 65, 0),
                                                 (128, 3, 3, 65, 1), (256, 2, 3, 130, 0),
                                                 (512, 2, 2, 260, 0)])
def test_step_kernel_wait_expiry_is_reported(N, ny, nx, step, shape):
    d = synth.small_scan(N, ny, nx, step, seed=31)

    def engine():
        return B.Engine(N, d["H"], d["W"], d["P0"], None, capacity=len(d["pos"]),
                        mode=B.EPIE_COLOURED, seed=5, device=0, ctas_per_frame=shape)

    with engine() as eng:
        eng.append(d["frames"], d["pos"])
        eng.iterate(1)
        B.epie_inject_fault(eng.h, B.EPIE_INJECT_STEP_COPY, 1, WAIT_NS)
        with pytest.raises(B.EpieError) as ex:
            eng.iterate(1)
        assert ex.value.code == B.EPIE_ETIMEOUT, ex.value
        for call in (lambda: eng.iterate(1), eng.object, eng.probe,
                     lambda: eng.append(d["frames"][:1], d["pos"][:1])):
            with pytest.raises(B.EpieError) as ex:
                call()
            assert ex.value.code == B.EPIE_ESTATE
    # the context is intact: a fresh handle runs a normal sweep
    with engine() as eng:
        eng.append(d["frames"], d["pos"])
        e = eng.iterate(2)
        assert np.all(np.isfinite(e)) and e[1] > 0
        assert np.all(np.isfinite(eng.object())) and np.all(np.isfinite(eng.probe()))


def test_injection_arguments_are_checked():
    with pytest.raises(B.EpieError) as ex:
        B.epie_inject_fault(None, B.EPIE_INJECT_TC_COPY, 1, 10)  # below 1 us
    assert ex.value.code == B.EPIE_EINVAL
    with pytest.raises(B.EpieError) as ex:
        B.epie_inject_fault(None, B.EPIE_INJECT_STEP_COPY, 1, WAIT_NS)  # no handle
    assert ex.value.code == B.EPIE_EINVAL


def test_tc_gemm_wait_expiry_sets_status_then_recovers():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(2)
    M, Nn, K = 512, 256, 256
    A = rng.standard_normal((M, K)).astype(np.float32)
    Bm = rng.standard_normal((Nn, K)).astype(np.float32)
    # bf16 operands (round to nearest even) and their exact product
    to16 = lambda x: ((x.view(np.uint32).astype(np.uint64) + 0x7FFF +
                       ((x.view(np.uint32).astype(np.uint64) >> 16) & 1)) >> 16).astype(np.uint16)
    f16 = lambda b: (b.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    A16, B16 = to16(A), to16(Bm)
    exact = f16(A16) @ f16(B16).T
    tA = torch.from_numpy(A16.view(np.int16)).to(dev)
    tB = torch.from_numpy(B16.view(np.int16)).to(dev)
    D = torch.zeros((M, Nn), dtype=torch.float32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    B.epie_inject_fault(None, B.EPIE_INJECT_TC_COPY, 1, WAIT_NS)
    B.epie_tc_gemm_bf16(tA.data_ptr(), 0, tB.data_ptr(), 0, D.data_ptr(), M, Nn, K, Nn, 1,
                        status.data_ptr())
    torch.cuda.synchronize()
    assert int(status.item()) & 2
    status.zero_()
    D.fill_(float("nan"))
    B.epie_tc_gemm_bf16(tA.data_ptr(), 0, tB.data_ptr(), 0, D.data_ptr(), M, Nn, K, Nn, 1,
                        status.data_ptr())
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    bound = 4 * K * 2.0 ** -24 * (np.abs(f16(A16)) @ np.abs(f16(B16)).T)
    assert np.all(np.abs(D.cpu().numpy() - exact) <= bound + 1e-30)
