"""Phase clocks of the fused 256^2 step kernel: a profiling tool.

Rebuilds the library with -DEPIE_PHASE_CLOCKS (thread 0 of every CTA records
clock64() at the kernel's phase boundaries), runs two coloured sweeps of the
live workload (10,000 frames, geometry A), reads the clocks of the last class
launched and prints the median cycles per phase over its CTAs as JSON.  The
normal build is restored afterwards.  Needs a GPU; takes about a minute.

    python -m paper_2308_10674_gb300.phase_clocks [--frames 10000]
"""
from __future__ import annotations

import argparse
import ctypes
import json

import numpy as np

PHASES = ["prologue, dependency wait, object and probe loads, probe product", "column FFT",
          "patch max + cluster sync 1", "transpose read + remote patch maxima",
          "cluster sync 2 + local write", "TMA wait + intensity tile", "row FFT + modulus + IFFT",
          "error reduce", "cluster sync 3", "read back", "cluster sync 4 + write",
          "column IFFT", "update"]


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--frames", type=int, default=10000)
    ap.add_argument("--workers", type=int, default=16)
    args = ap.parse_args()
    from . import build
    extra = build.EXTRA
    build.EXTRA = extra + ["-DEPIE_PHASE_CLOCKS"]
    try:
        build.build(force=True)
        from . import _binding as B, synth
        d = synth.live_scan(N=256, n=args.frames, geometry="A", seed=0, workers=args.workers)
        eng = B.Engine(256, d["H"], d["W"], d["P0"], None, capacity=len(d["pos"]),
                       mode=B.EPIE_COLOURED, seed=5)
        eng.set_dark(d["dark"])
        eng.append(d["frames"], d["pos"])
        eng.iterate(2)
        _, gs = eng.order(1)
        members = int(gs[-1] - gs[-2])
        n = members * 8  # 8-CTA clusters at 256^2
        L = B.lib()
        L.epie_read_phase_clocks.argtypes = [ctypes.c_void_p, ctypes.c_int]
        clk = np.zeros((n, 16), np.int64)
        rc = L.epie_read_phase_clocks(clk.ctypes.data, n)
        eng.close()
        if rc != 0:
            raise RuntimeError(f"reading the phase clocks failed ({rc})")
        dt = np.median(np.diff(clk[:, :14], axis=1), axis=0)
        print(json.dumps({"members": members, "ctas": n,
                          "median_cycles": {p: float(v) for p, v in zip(PHASES, dt)},
                          "total": float(np.median(clk[:, 13] - clk[:, 0]))}, indent=1))
    finally:
        build.EXTRA = extra
        build.build(force=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
