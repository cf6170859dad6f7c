"""C-ABI checks that need no GPU: the library loads, exports every function
include/epie.h declares, the binding's struct layout matches the C compiler's,
configuration errors are reported before any device is touched, and a host
without a usable device gets EPIE_ECUDA (no CPU fallback)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "epie.h")


@pytest.fixture(scope="module")
def B():
    from paper_2308_10674_gb300 import _binding
    from paper_2308_10674_gb300 import build
    build.build()
    _binding.lib()
    return _binding


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^EPIE_API\s+[\w\s\*]*?\b(epie_\w+)\s*\(", text, re.M)))


def test_every_declared_function_is_exported(B):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(B.lib(), n), n
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r" T (epie_\w+)", out))
    assert exported == set(names)


def test_config_struct_layout_matches_c(B, tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(f"""
#include <stddef.h>
#include <stdio.h>
#include "{HEADER}"
int main(void) {{
  printf("%zu", sizeof(epie_config));
#define F(m) printf(" %zu", offsetof(epie_config, m));
  F(N) F(obj_h) F(obj_w) F(capacity) F(intensity_dtype) F(mode) F(batch) F(omax_mode) F(path)
  F(alpha) F(beta) F(seed) F(device) F(stream) F(flags) F(class_cap) F(gemm_precision)
  F(ctas_per_frame)
  return 0;
}}
""")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-o", str(exe), str(src)])
    vals = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    C = B.epie_config
    py = [ctypes.sizeof(C)] + [getattr(C, f).offset for f, _ in C._fields_]
    assert vals == py


def test_defaults(B):
    c = B.epie_config_default()
    assert (c.N, c.obj_h, c.obj_w, c.mode, c.path) == (256, 1024, 1024, B.EPIE_COLOURED,
                                                      B.EPIE_PATH_FUSED)
    assert c.alpha == 1.0 and c.beta == 1.0 and c.intensity_dtype == B.EPIE_U16


@pytest.mark.parametrize("field,value,msg", [
    ("N", 100, "N must be"), ("N", 1024, "N must be"), ("obj_h", 32, "at least N"),
    ("capacity", -1, "capacity"), ("intensity_dtype", 7, "intensity_dtype"),
    ("mode", 9, "mode"), ("omax_mode", 3, "omax_mode"), ("path", 4, "path"),
    ("flags", 1 << 8, "flags"), ("alpha", float("nan"), "finite"),
    ("class_cap", -1, "class_cap"), ("gemm_precision", 9, "gemm_precision"),
])
def test_bad_configuration_is_rejected_on_the_host(B, field, value, msg):
    c = B.epie_config_default()
    c.N, c.obj_h, c.obj_w = 64, 128, 128
    setattr(c, field, value)
    n = c.N if c.N in (64, 128, 256, 512) else 64
    with pytest.raises(B.EpieError) as ex:
        B.epie_init(c, np.ones((c.N, c.N), np.complex64) if field == "N" else
                    np.ones((n, n), np.complex64))
    assert ex.value.code == B.EPIE_EINVAL and msg in str(ex.value)


def test_minibatch_needs_positive_batch(B):
    c = B.epie_config_default()
    c.N, c.obj_h, c.obj_w, c.mode, c.batch = 64, 128, 128, B.EPIE_MINIBATCH, 0
    with pytest.raises(B.EpieError) as ex:
        B.epie_init(c, np.ones((64, 64), np.complex64))
    assert ex.value.code == B.EPIE_EINVAL


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.mark.skipif(_has_gpu(), reason="checks the no-device error path")
def test_no_device_fails_loudly(B):
    c = B.epie_config_default()
    c.N, c.obj_h, c.obj_w = 64, 128, 128
    with pytest.raises(B.EpieError) as ex:
        B.epie_init(c, np.ones((64, 64), np.complex64))
    assert ex.value.code == B.EPIE_ECUDA and "no CUDA device" in str(ex.value)


def test_null_handle_calls_are_rejected(B):
    L = B.lib()
    assert L.epie_iterate(None, 1, None) == B.EPIE_EINVAL
    assert L.epie_append_frames(None, None, None, 0) == B.EPIE_EINVAL
    assert L.epie_destroy(None) == B.EPIE_OK
    n = ctypes.c_int32()
    assert L.epie_num_frames(None, ctypes.byref(n)) == B.EPIE_EINVAL


@pytest.mark.parametrize("M,Nn,K,ldd,terms", [
    (100, 256, 64, 256, 1), (128, 200, 64, 256, 1), (128, 256, 96, 256, 1),
    (128, 256, 64, 255, 1), (128, 256, 64, 256, 2), (128, 256, 64, 128, 1),
])
def test_tc_gemm_rejects_bad_shapes_on_the_host(B, M, Nn, K, ldd, terms):
    """Shape checks of the tensor-core product run before any device call."""
    fake = 1 << 20  # 16-byte aligned, never dereferenced
    with pytest.raises(B.EpieError) as ex:
        B.epie_tc_gemm_bf16(fake, fake, fake, fake, fake, M, Nn, K, ldd, terms, fake)
    assert ex.value.code == B.EPIE_EINVAL


def test_fma_peak_rejects_bad_arguments(B):
    import ctypes
    t, m = ctypes.c_double(), ctypes.c_double()
    assert B.lib().epie_fp32_fma_peak(0, 0, ctypes.byref(t), ctypes.byref(m)) == B.EPIE_EINVAL
    assert B.lib().epie_fp32_fma_peak(0, 10, None, ctypes.byref(m)) == B.EPIE_EINVAL
