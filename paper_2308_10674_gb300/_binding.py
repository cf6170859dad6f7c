"""ctypes binding of the engine's C ABI (include/epie.h).

Functions keep the C names; arguments are marshalled only.  Every step of
the reconstruction runs in the CUDA library: when libepie.so is missing the
import fails loudly, and there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libepie.so")

EPIE_OK, EPIE_EINVAL, EPIE_ERANGE, EPIE_ECAPACITY = 0, -1, -2, -3
EPIE_ECUDA, EPIE_ETIMEOUT, EPIE_ENUMERIC, EPIE_ESTATE = -4, -5, -6, -7
EPIE_U16, EPIE_F16, EPIE_F32 = 0, 1, 2
EPIE_SEQUENTIAL, EPIE_COLOURED, EPIE_MINIBATCH = 0, 1, 2
EPIE_OMAX_PATCH, EPIE_OMAX_GLOBAL = 0, 1
EPIE_PATH_FUSED, EPIE_PATH_PLAIN, EPIE_PATH_GEMM = 0, 1, 2
EPIE_GEMM_BF16, EPIE_GEMM_TF32, EPIE_GEMM_BF16X3, EPIE_GEMM_FP32EMU = 0, 1, 2, 3
EPIE_GEMM_TC_BF16, EPIE_GEMM_TC_BF16X3, EPIE_GEMM_TC_TF32, EPIE_GEMM_TC_TF32X3 = 4, 5, 6, 7
EPIE_CHECKED, EPIE_PROBE_SUM, EPIE_GRAPH, EPIE_FRAMES_FFT_ORDER = 1, 2, 4, 8
EPIE_RAW_INTENSITY = 16

STATUS = {0: "EPIE_OK", -1: "EPIE_EINVAL", -2: "EPIE_ERANGE", -3: "EPIE_ECAPACITY",
          -4: "EPIE_ECUDA", -5: "EPIE_ETIMEOUT", -6: "EPIE_ENUMERIC", -7: "EPIE_ESTATE"}


class epie_config(C.Structure):
    _fields_ = [("N", C.c_int32), ("obj_h", C.c_int32), ("obj_w", C.c_int32),
                ("capacity", C.c_int32), ("intensity_dtype", C.c_int32), ("mode", C.c_int32),
                ("batch", C.c_int32), ("omax_mode", C.c_int32), ("path", C.c_int32),
                ("alpha", C.c_float), ("beta", C.c_float), ("seed", C.c_uint64),
                ("device", C.c_int32), ("stream", C.c_void_p), ("flags", C.c_uint32),
                ("class_cap", C.c_int32), ("gemm_precision", C.c_int32),
                ("ctas_per_frame", C.c_int32)]


class epie_amp_grad_args(C.Structure):
    _fields_ = [("N", C.c_int32), ("intensity_dtype", C.c_int32), ("obj_h", C.c_int32),
                ("obj_w", C.c_int32), ("n", C.c_int32), ("object", C.c_void_p),
                ("probe", C.c_void_p), ("frames", C.c_void_p), ("pos", C.c_void_p),
                ("shift", C.c_void_p), ("grad_object", C.c_void_p), ("grad_probe", C.c_void_p),
                ("grad_shift", C.c_void_p), ("scratch", C.c_void_p),
                ("scratch_bytes", C.c_size_t), ("stream", C.c_void_p)]


class EpieError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2308_10674_gb300.build` (no CPU fallback exists)")
        L = C.CDLL(LIB_PATH)
        H, vp, i32, i64, sz = C.c_void_p, C.c_void_p, C.c_int32, C.c_int64, C.c_size_t
        L.epie_config_default.argtypes = [C.POINTER(epie_config)]
        L.epie_config_default.restype = None
        L.epie_init.argtypes = [C.POINTER(H), C.POINTER(epie_config), vp, vp]
        L.epie_set_dark.argtypes = [H, vp]
        L.epie_append_frames.argtypes = [H, vp, vp, i32]
        L.epie_append_frames_device.argtypes = [H, vp, vp, i32]
        L.epie_truncate_frames.argtypes = [H, i32]
        L.epie_iterate.argtypes = [H, i32, vp]
        L.epie_iterate_many.argtypes = [vp, i32, i32, vp]
        L.epie_average_state.argtypes = [vp, i32]
        for n in ("epie_get_object", "epie_get_probe", "epie_set_object", "epie_set_probe"):
            getattr(L, n).argtypes = [H, vp, sz]
        L.epie_num_frames.argtypes = [H, C.POINTER(i32)]
        L.epie_num_classes.argtypes = [H, C.POINTER(i32)]
        L.epie_get_colours.argtypes = [H, vp, i32]
        L.epie_get_order.argtypes = [H, i64, vp, vp, C.POINTER(i32)]
        L.epie_get_sweep_index.argtypes = [H, C.POINTER(i64)]
        L.epie_set_sweep_index.argtypes = [H, i64]
        L.epie_last_timing.argtypes = [H, C.POINTER(C.c_double), C.POINTER(i64)]
        L.epie_last_sweep_frames.argtypes = [H, vp, i32, C.POINTER(i32)]
        L.epie_inject_fault.argtypes = [H, i32, i32, i64]
        L.epie_launch_count.argtypes = [H, C.POINTER(i64)]
        L.epie_set_kernel_timing.argtypes = [H, i32]
        L.epie_kernel_timing.argtypes = [H, C.POINTER(i64), C.POINTER(C.c_double),
                                         C.POINTER(i64)]
        L.epie_group_step_static.argtypes = [i32, i32, vp, i32, i32, vp, vp, i32, vp, vp, i32,
                                             vp, C.c_float, C.c_float, i32, vp, vp]
        L.epie_amp_grad_scratch_bytes.argtypes = [i32, i32]
        L.epie_amp_grad_scratch_bytes.restype = C.c_size_t
        L.epie_amp_loss_grad.argtypes = [C.POINTER(epie_amp_grad_args), C.POINTER(C.c_double)]
        L.epie_frames_to_fft_order.argtypes = [vp, vp, i32, i32, i32, vp]
        L.epie_tc_gemm_bf16.argtypes = [vp, vp, vp, vp, vp, C.c_int64, i32, i32, i32, i32, vp, vp]
        L.epie_tc_gemm_tf32.argtypes = [vp, vp, vp, vp, vp, C.c_int64, i32, i32, i32, i32, vp, vp]
        L.epie_fp32_fma_peak.argtypes = [i32, i32, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.epie_error.argtypes = [H]
        L.epie_error.restype = C.c_char_p
        L.epie_destroy.argtypes = [H]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# --------------------------------------------------------------------------- C names

def epie_config_default() -> epie_config:
    c = epie_config()
    lib().epie_config_default(C.byref(c))
    return c


def epie_error(h) -> str:
    m = lib().epie_error(h)
    return m.decode() if m else ""


def _check(h, rc):
    if rc != EPIE_OK:
        raise EpieError(rc, epie_error(h))
    return rc


def epie_init(cfg: epie_config, probe0, object0=None):
    """Returns a handle (c_void_p).  probe0 / object0: complex64-compatible arrays."""
    p = np.ascontiguousarray(probe0, dtype=np.complex64)
    o = None if object0 is None else np.ascontiguousarray(object0, dtype=np.complex64)
    if p.shape != (cfg.N, cfg.N):
        raise ValueError("probe0 must be N x N")
    if o is not None and o.shape != (cfg.obj_h, cfg.obj_w):
        raise ValueError("object0 must be obj_h x obj_w")
    h = C.c_void_p()
    rc = lib().epie_init(C.byref(h), C.byref(cfg), _p(p), _p(o))
    if rc != EPIE_OK:
        raise EpieError(rc, epie_error(None))
    return h


def epie_destroy(h):
    return lib().epie_destroy(h)


def epie_set_dark(h, dark):
    d = None if dark is None else np.ascontiguousarray(dark, dtype=np.float32)
    return _check(h, lib().epie_set_dark(h, _p(d)))


def epie_append_frames(h, frames, pos_yx):
    pos = np.ascontiguousarray(pos_yx, dtype=np.int32).reshape(-1, 2)
    fr = np.ascontiguousarray(frames)
    if fr.dtype == np.float16:
        fr = fr.view(np.uint16)
    return _check(h, lib().epie_append_frames(h, _p(fr), _p(pos), len(pos)))


def epie_append_frames_device(h, frames_dev_ptr: int, pos_yx, n: int):
    pos = np.ascontiguousarray(pos_yx, dtype=np.int32).reshape(-1, 2)
    return _check(h, lib().epie_append_frames_device(h, C.c_void_p(frames_dev_ptr), _p(pos), n))


def epie_truncate_frames(h, n_keep):
    return _check(h, lib().epie_truncate_frames(h, n_keep))


def epie_iterate(h, n_sweeps):
    err = np.zeros(max(n_sweeps, 0), np.float64)
    _check(h, lib().epie_iterate(h, n_sweeps, _p(err) if n_sweeps > 0 else None))
    return err


def epie_iterate_many(handles, n_sweeps):
    """Concurrent sweeps of several handles; returns errors [len(handles), n_sweeps]."""
    k = len(handles)
    arr = (C.c_void_p * k)(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    err = np.zeros((k, max(n_sweeps, 0)), np.float64)
    rc = lib().epie_iterate_many(C.cast(arr, C.c_void_p), k, n_sweeps,
                                 _p(err) if n_sweeps > 0 else None)
    if rc != EPIE_OK:
        msgs = "; ".join(epie_error(h) for h in handles if epie_error(h))
        raise EpieError(rc, msgs or epie_error(None))
    return err


def epie_average_state(handles):
    """Replace every handle's object and probe by their mean (paper's
    parallel scheme)."""
    k = len(handles)
    arr = (C.c_void_p * k)(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    rc = lib().epie_average_state(C.cast(arr, C.c_void_p), k)
    if rc != EPIE_OK:
        raise EpieError(rc, "; ".join(epie_error(h) for h in handles if epie_error(h)))


def _get(h, fn, shape):
    out = np.empty(shape, np.complex64)
    _check(h, fn(h, _p(out), out.size * 2))
    return out


def epie_get_object(h, shape):
    return _get(h, lib().epie_get_object, shape)


def epie_get_probe(h, N):
    return _get(h, lib().epie_get_probe, (N, N))


def epie_set_object(h, obj):
    o = np.ascontiguousarray(obj, dtype=np.complex64)
    return _check(h, lib().epie_set_object(h, _p(o), o.size * 2))


def epie_set_probe(h, probe):
    p = np.ascontiguousarray(probe, dtype=np.complex64)
    return _check(h, lib().epie_set_probe(h, _p(p), p.size * 2))


def epie_num_frames(h):
    n = C.c_int32()
    _check(h, lib().epie_num_frames(h, C.byref(n)))
    return n.value


def epie_num_classes(h):
    n = C.c_int32()
    _check(h, lib().epie_num_classes(h, C.byref(n)))
    return n.value


def epie_get_colours(h, n):
    out = np.empty(n, np.int32)
    _check(h, lib().epie_get_colours(h, _p(out), n))
    return out


def epie_get_order(h, sweep):
    n = epie_num_frames(h)
    order = np.empty(max(n, 1), np.int32)
    gs = np.empty(n + 1, np.int32)
    ng = C.c_int32()
    _check(h, lib().epie_get_order(h, sweep, _p(order), _p(gs), C.byref(ng)))
    return order[:n], gs[:ng.value + 1]


def epie_get_sweep_index(h):
    s = C.c_int64()
    _check(h, lib().epie_get_sweep_index(h, C.byref(s)))
    return s.value


def epie_set_sweep_index(h, sweep):
    return _check(h, lib().epie_set_sweep_index(h, sweep))


def epie_last_timing(h):
    ms, k = C.c_double(), C.c_int64()
    _check(h, lib().epie_last_timing(h, C.byref(ms), C.byref(k)))
    return ms.value, k.value


def epie_last_sweep_frames(h):
    """Frame counts of the sweeps of the most recent epie_iterate call."""
    n = C.c_int32()
    _check(h, lib().epie_last_sweep_frames(h, None, 0, C.byref(n)))
    out = np.zeros(n.value, np.int32)
    _check(h, lib().epie_last_sweep_frames(h, _p(out), n.value, C.byref(n)))
    return out[:n.value]


def epie_launch_count(h):
    n = C.c_int64()
    _check(h, lib().epie_launch_count(h, C.byref(n)))
    return n.value


def epie_set_kernel_timing(h, on):
    return _check(h, lib().epie_set_kernel_timing(h, 1 if on else 0))


def epie_kernel_timing(h):
    """(launches, milliseconds, frames) of the step kernel since the last call."""
    n, ms, f = C.c_int64(), C.c_double(), C.c_int64()
    _check(h, lib().epie_kernel_timing(h, C.byref(n), C.byref(ms), C.byref(f)))
    return n.value, ms.value, f.value


def epie_group_step_static(N, intensity_dtype, object_ptr, obj_h, obj_w, probe_ptr, frames_ptr,
                           n_frames, pos_ptr, members_ptr, n_members, dark_ptr=None, alpha=1.0,
                           beta=1.0, probe_mean=True, want_err=True, stream=None):
    """One group update on caller-owned device buffers (integer device
    addresses), allocating no device memory.  Returns the group's
    (sum (|Psi| - sqrt I)^2, sum I) when want_err."""
    err = np.zeros(2, np.float64)
    rc = lib().epie_group_step_static(
        N, intensity_dtype, C.c_void_p(object_ptr), obj_h, obj_w, C.c_void_p(probe_ptr),
        C.c_void_p(frames_ptr), n_frames, C.c_void_p(pos_ptr), C.c_void_p(members_ptr), n_members,
        C.c_void_p(dark_ptr) if dark_ptr else None, alpha, beta, 1 if probe_mean else 0,
        _p(err) if want_err else None, C.c_void_p(stream) if stream else None)
    if rc != EPIE_OK:
        raise EpieError(rc, epie_error(None))
    return err


def epie_frames_to_fft_order(src_ptr, dst_ptr, n, N, intensity_dtype=EPIE_U16, stream=None):
    """Device re-layout of n DC-centred frames into FFT order (integer device
    addresses)."""
    rc = lib().epie_frames_to_fft_order(C.c_void_p(src_ptr), C.c_void_p(dst_ptr), n, N,
                                        intensity_dtype, C.c_void_p(stream) if stream else None)
    if rc != EPIE_OK:
        raise EpieError(rc, epie_error(None))


def epie_tc_gemm_bf16(A0, A1, B0, B1, D, M, Nn, K, ldd, terms, status, stream=None):
    """D = sum_t A_t B_t^T on the tensor cores (integer device addresses; A1,
    B1 may be 0 for terms = 1; status: address of a device int32)."""
    v = lambda x: C.c_void_p(x) if x else None
    rc = lib().epie_tc_gemm_bf16(v(A0), v(A1), v(B0), v(B1), v(D), M, Nn, K, ldd, terms,
                                 v(status), v(stream))
    if rc != EPIE_OK:
        raise EpieError(rc, epie_error(None))


EPIE_INJECT_STEP_COPY, EPIE_INJECT_TC_COPY = 1, 2


def epie_inject_fault(h, what, count, wait_ns):
    """Failure injection for the timeout tests: the next `count` launches of
    the step kernel (what = EPIE_INJECT_STEP_COPY, handle h) or of the tcgen05
    GEMM (EPIE_INJECT_TC_COPY, h may be None) skip one bulk copy, and their
    waits give up after wait_ns."""
    rc = lib().epie_inject_fault(h, what, count, wait_ns)
    if rc != EPIE_OK:
        raise EpieError(rc, epie_error(h))


def epie_fp32_fma_peak(device=0, iters=4096):
    """(TFLOP/s, SM MHz) of an FP32 FMA-chain kernel on the device."""
    t, m = C.c_double(), C.c_double()
    rc = lib().epie_fp32_fma_peak(device, iters, C.byref(t), C.byref(m))
    if rc != EPIE_OK:
        raise EpieError(rc, epie_error(None))
    return t.value, m.value


def epie_tc_gemm_tf32(A0, A1, B0, B1, D, M, Nn, K, ldd, terms, status, stream=None):
    """D = sum_t A_t B_t^T with fp32 operands read as tf32 (integer device
    addresses, as epie_tc_gemm_bf16)."""
    v = lambda x: C.c_void_p(x) if x else None
    rc = lib().epie_tc_gemm_tf32(v(A0), v(A1), v(B0), v(B1), v(D), M, Nn, K, ldd, terms,
                                 v(status), v(stream))
    if rc != EPIE_OK:
        raise EpieError(rc, epie_error(None))


def epie_amp_grad_scratch_bytes(N, n):
    return int(lib().epie_amp_grad_scratch_bytes(N, n))


def epie_amp_loss_grad(args: epie_amp_grad_args, want_loss=True):
    loss = C.c_double(0.0)
    rc = lib().epie_amp_loss_grad(C.byref(args), C.byref(loss) if want_loss else None)
    if rc != EPIE_OK:
        raise EpieError(rc, epie_error(None))
    return loss.value


# --------------------------------------------------------------------------- convenience

class Engine:
    """Small object wrapper over one handle (same calls, numpy in / out)."""

    def __init__(self, N, obj_h, obj_w, probe0, object0=None, capacity=1024,
                 intensity_dtype=EPIE_U16, mode=EPIE_COLOURED, batch=64,
                 omax_mode=EPIE_OMAX_PATCH, path=EPIE_PATH_FUSED, alpha=1.0, beta=1.0, seed=0,
                 device=0, stream=None, flags=0, class_cap=0, gemm_precision=EPIE_GEMM_BF16X3,
                 ctas_per_frame=0):
        cfg = epie_config_default()
        cfg.N, cfg.obj_h, cfg.obj_w, cfg.capacity = N, obj_h, obj_w, capacity
        cfg.intensity_dtype, cfg.mode, cfg.batch = intensity_dtype, mode, batch
        cfg.omax_mode, cfg.path, cfg.alpha, cfg.beta = omax_mode, path, alpha, beta
        cfg.seed, cfg.device, cfg.stream, cfg.flags = seed, device, stream, flags
        cfg.class_cap = class_cap
        cfg.gemm_precision = gemm_precision
        cfg.ctas_per_frame = ctas_per_frame
        self.cfg = cfg
        self.h = epie_init(cfg, probe0, object0)

    def close(self):
        if self.h is not None:
            epie_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_dark(self, dark):
        epie_set_dark(self.h, dark)

    def append(self, frames, pos):
        epie_append_frames(self.h, frames, pos)

    def truncate(self, n_keep):
        epie_truncate_frames(self.h, n_keep)

    def iterate(self, n_sweeps):
        return epie_iterate(self.h, n_sweeps)

    def object(self):
        return epie_get_object(self.h, (self.cfg.obj_h, self.cfg.obj_w))

    def probe(self):
        return epie_get_probe(self.h, self.cfg.N)

    def set_object(self, o):
        epie_set_object(self.h, o)

    def set_probe(self, p):
        epie_set_probe(self.h, p)

    @property
    def n_frames(self):
        return epie_num_frames(self.h)

    @property
    def n_classes(self):
        return epie_num_classes(self.h)

    def colours(self):
        return epie_get_colours(self.h, self.n_frames)

    def order(self, sweep):
        return epie_get_order(self.h, sweep)

    @property
    def sweep_index(self):
        return epie_get_sweep_index(self.h)

    @sweep_index.setter
    def sweep_index(self, s):
        epie_set_sweep_index(self.h, s)

    def last_timing(self):
        return epie_last_timing(self.h)

    def last_sweep_frames(self):
        return epie_last_sweep_frames(self.h)
