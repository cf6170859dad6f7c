"""ctypes wrapper around the FP64 C oracle (oracle/epie_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the product package.

Every function mirrors one C entry point; arrays are numpy complex128 /
float64 / int32, C-contiguous.  The ePIE steps follow Maiden & Rodenburg
(2009), the algorithm the paper names for its engine (Sec. "ePIE
Implementation"); the readings R1..R9 are listed in the C file's header.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "epie_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

U16, F16, F32 = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math, one thread)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fno-fast-math",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            vp, i32, i64, u64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
            L.orc_fft2.argtypes = [vp, C.c_int, C.c_int]
            L.orc_dft2_brute.argtypes = [vp, vp, C.c_int, C.c_int]
            L.orc_prepare_intensity.argtypes = [vp, C.c_int, C.c_long, C.c_int, vp, vp]
            L.orc_modulus_project.argtypes = [vp, vp, C.c_long, vp, vp]
            L.orc_epie_step.argtypes = [vp, C.c_int, C.c_int, vp, C.c_int, vp, C.c_int, C.c_int,
                                        dbl, dbl, C.c_int, vp, vp]
            L.orc_sweep_groups.argtypes = [vp, C.c_int, C.c_int, vp, C.c_int, vp, vp, vp, vp, i32,
                                           dbl, dbl, C.c_int, C.c_int, vp, vp]
            L.orc_sweep_minibatch.argtypes = [vp, C.c_int, C.c_int, vp, C.c_int, vp, vp, vp, i32,
                                              i32, dbl, dbl, C.c_int, vp, vp]
            L.orc_splitmix64.argtypes = [vp]
            L.orc_splitmix64.restype = u64
            L.orc_order_sequential.argtypes = [u64, i64, i32, vp]
            L.orc_colour_greedy.argtypes = [vp, i32, i32, i32, vp]
            L.orc_colour_greedy.restype = i32
            L.orc_order_coloured.argtypes = [u64, i64, i32, vp, i32, vp, vp]
            L.orc_amp_loss_grad.argtypes = [vp, C.c_int, C.c_int, vp, C.c_int, vp, vp, vp, i32,
                                            vp, vp, vp]
            L.orc_amp_loss_grad.restype = dbl
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


# --------------------------------------------------------------------------- transforms

def fft2(a, sign=-1):
    """Own radix-2 2-D FFT (R1): sign -1 forward unnormalised, +1 inverse with 1/N^2."""
    a = _c128(a).copy()
    if lib().orc_fft2(_p(a), a.shape[0], sign) != 0:
        raise ValueError("fft2: side must be a power of two")
    return a


def dft2_brute(a, sign=-1):
    """O(N^4) DFT straight from its definition (pins only)."""
    a = _c128(a)
    out = np.empty_like(a)
    if lib().orc_dft2_brute(_p(a), _p(out), a.shape[0], sign) != 0:
        raise ValueError("dft2_brute: bad arguments")
    return out


# --------------------------------------------------------------------------- intensities

def prepare_intensity(frames, dark=None):
    """Raw DC-centred frames [n,N,N] (uint16 / float16 / float32) -> FFT-order
    float64 intensities with the dark field subtracted and clamped at 0 (R1, R5)."""
    frames = np.ascontiguousarray(frames)
    if frames.ndim == 2:
        frames = frames[None]
    n, N, _ = frames.shape
    if frames.dtype == np.uint16:
        dt = U16
    elif frames.dtype == np.float16:
        dt, frames = F16, frames.view(np.uint16)
    elif frames.dtype == np.float32:
        dt = F32
    else:
        raise TypeError("frames must be uint16, float16 or float32")
    d = None if dark is None else np.ascontiguousarray(dark, dtype=np.float32)
    out = np.empty((n, N, N), np.float64)
    if lib().orc_prepare_intensity(_p(frames), dt, n, N, _p(d), _p(out)) != 0:
        raise ValueError("prepare_intensity: bad arguments")
    return out


def modulus_project(Psi, I):
    """Modulus replacement (ePIE, R2); returns (Psi', err, isum)."""
    Psi = _c128(Psi).copy()
    I = np.ascontiguousarray(I, dtype=np.float64)
    e, s = C.c_double(0.0), C.c_double(0.0)
    lib().orc_modulus_project(_p(Psi), _p(I), Psi.size, C.byref(e), C.byref(s))
    return Psi, e.value, s.value


# --------------------------------------------------------------------------- ePIE

def epie_step(O, P, I, y0, x0, alpha=1.0, beta=1.0, omax_global=False):
    """One sequential ePIE step (R3, R4) on copies; returns (O', P', err, isum)."""
    O = _c128(O).copy()
    P = _c128(P).copy()
    I = np.ascontiguousarray(I, dtype=np.float64)
    e, s = C.c_double(0.0), C.c_double(0.0)
    rc = lib().orc_epie_step(_p(O), O.shape[0], O.shape[1], _p(P), P.shape[0], _p(I), int(y0),
                             int(x0), alpha, beta, int(omax_global), C.byref(e), C.byref(s))
    if rc != 0:
        raise ValueError(f"epie_step: rc={rc}")
    return O, P, e.value, s.value


def sweep_groups(O, P, I_all, pos, order, group_start, alpha=1.0, beta=1.0, omax_global=False,
                 probe_mean=True):
    """Run groups in order (sequential: groups of one; coloured: classes).
    Works in place on O and P (complex128 arrays); returns (err, isum)."""
    assert O.dtype == np.complex128 and O.flags.c_contiguous
    assert P.dtype == np.complex128 and P.flags.c_contiguous
    I_all = np.ascontiguousarray(I_all, dtype=np.float64)
    pos = np.ascontiguousarray(pos, dtype=np.int32)
    order = np.ascontiguousarray(order, dtype=np.int32)
    gs = np.ascontiguousarray(group_start, dtype=np.int32)
    e, s = C.c_double(0.0), C.c_double(0.0)
    rc = lib().orc_sweep_groups(_p(O), O.shape[0], O.shape[1], _p(P), P.shape[0], _p(I_all),
                                _p(pos), _p(order), _p(gs), len(gs) - 1, alpha, beta,
                                int(omax_global), int(probe_mean), C.byref(e), C.byref(s))
    if rc != 0:
        raise ValueError(f"sweep_groups: rc={rc}")
    return e.value, s.value


def sweep_minibatch(O, P, I_all, pos, order, batch, alpha=1.0, beta=1.0, omax_global=False):
    """Mini-batch sweep (R7), in place on O and P; returns (err, isum)."""
    assert O.dtype == np.complex128 and O.flags.c_contiguous
    assert P.dtype == np.complex128 and P.flags.c_contiguous
    I_all = np.ascontiguousarray(I_all, dtype=np.float64)
    pos = np.ascontiguousarray(pos, dtype=np.int32)
    order = np.ascontiguousarray(order, dtype=np.int32)
    e, s = C.c_double(0.0), C.c_double(0.0)
    rc = lib().orc_sweep_minibatch(_p(O), O.shape[0], O.shape[1], _p(P), P.shape[0], _p(I_all),
                                   _p(pos), _p(order), len(order), int(batch), alpha, beta,
                                   int(omax_global), C.byref(e), C.byref(s))
    if rc != 0:
        raise ValueError(f"sweep_minibatch: rc={rc}")
    return e.value, s.value


# --------------------------------------------------------------------------- order, colouring

def splitmix64_stream(state, count):
    st = C.c_uint64(state)
    return [int(lib().orc_splitmix64(C.byref(st))) for _ in range(count)]


def order_sequential(seed, sweep, n):
    out = np.empty(n, np.int32)
    lib().orc_order_sequential(seed, sweep, n, _p(out))
    return out


def colour_greedy(pos, N, cap=0):
    """Greedy first-fit colour classes (R6), at most `cap` frames per class
    when cap > 0."""
    pos = np.ascontiguousarray(pos, dtype=np.int32)
    col = np.empty(len(pos), np.int32)
    ncls = lib().orc_colour_greedy(_p(pos), len(pos), N, int(cap), _p(col))
    return col, int(ncls)


def order_coloured(seed, sweep, colour, ncls):
    colour = np.ascontiguousarray(colour, dtype=np.int32)
    order = np.empty(len(colour), np.int32)
    gs = np.empty(ncls + 1, np.int32)
    lib().orc_order_coloured(seed, sweep, len(colour), _p(colour), ncls, _p(order), _p(gs))
    return order, gs


def sequential_groups(order):
    return np.arange(len(order) + 1, dtype=np.int32)


# --------------------------------------------------------------------------- whole runs

SEQUENTIAL, COLOURED = 0, 1


def run_sweeps(O, P, I_all, pos, n_sweeps, N, seed, mode=SEQUENTIAL, alpha=1.0, beta=1.0,
               sweep_offset=0, omax_global=False, probe_mean=True, class_cap=0):
    """n_sweeps sweeps over all given frames, in place on O and P.
    Returns the per-sweep error metric E_s (R8)."""
    n = len(pos)
    errs = []
    if mode == COLOURED:
        colour, ncls = colour_greedy(pos, N, class_cap)
    for s in range(sweep_offset, sweep_offset + n_sweeps):
        if mode == SEQUENTIAL:
            order = order_sequential(seed, s, n)
            gs = sequential_groups(order)
        else:
            order, gs = order_coloured(seed, s, colour, ncls)
        e, t = sweep_groups(O, P, I_all, pos, order, gs, alpha, beta, omax_global, probe_mean)
        errs.append(e / t if t > 0 else 0.0)
    return errs


def amp_loss_grad(O, P, I_all, pos, shift=None):
    """Amplitude loss sum_j || |F(S_dj P . O_j)| - sqrt(I_j) ||^2 and its gradients
    (dL/dRe + i dL/dIm for O and P; dL/d(dy), dL/d(dx) per position)."""
    O = _c128(O)
    P = _c128(P)
    I_all = np.ascontiguousarray(I_all, dtype=np.float64)
    pos = np.ascontiguousarray(pos, dtype=np.int32)
    n = len(pos)
    sh = None if shift is None else np.ascontiguousarray(shift, dtype=np.float64)
    gO = np.empty_like(O)
    gP = np.empty_like(P)
    gd = np.empty((n, 2), np.float64)
    L = lib().orc_amp_loss_grad(_p(O), O.shape[0], O.shape[1], _p(P), P.shape[0], _p(I_all),
                                _p(pos), _p(sh), n, _p(gO), _p(gP), _p(gd))
    return L, gO, gP, gd


def run_parallel_average(O, P, I_all, pos, subsets, sweeps_per_round, rounds, N, seed,
                         mode=SEQUENTIAL, **kw):
    """The paper's parallel scheme (Sec. "Simulating live and parallel
    processing"): every round, each disjoint subset q of positions runs
    `sweeps_per_round` sweeps from the common (O, P) on its own copy (order
    stream seed + q, sweep counter continuing across rounds), then O and P
    become the mean of the copies (summed in subset order).  In place on O, P."""
    for r in range(rounds):
        Os, Ps = [], []
        for q, idx in enumerate(subsets):
            Oq, Pq = O.copy(), P.copy()
            run_sweeps(Oq, Pq, I_all[idx], pos[idx], sweeps_per_round, N, seed + q, mode=mode,
                       sweep_offset=r * sweeps_per_round, **kw)
            Os.append(Oq)
            Ps.append(Pq)
        O[...] = sum(Os[1:], Os[0]) / len(Os)
        P[...] = sum(Ps[1:], Ps[0]) / len(Ps)
