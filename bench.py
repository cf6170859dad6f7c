"""Benchmark of the live ePIE hot path: ePIE frame-updates/s at 256^2 frames.

Workload (live ePIE at beamline-like size, paper Sec. "Live ePIE"): 256x256
uint16 frames, 10,000 positions on a Fermat spiral with a step of 0.35 x the
probe FWHM (60 px), 1e8 photons per frame, Poisson noise, 2% dark-offset
field, coloured ePIE in FP32 on the device.  The frame set lives in HBM.

One step = the live ingest of the scan's last 500-frame chunk (the set is
truncated back to 9,500 frames first, so every step works on the full set)
followed by one sweep over all 10,000 frames: every row of the hot path.
`value` times steps whose chunk comes from device memory; `e2e` times the same
steps through the public API from pinned host memory (host->device copy of the
chunk and the device->host read of the sweep error inside the timed region).

`--impl reference` times the FP64 CPU oracle on the host cores (bounded
sample of the same workload).  Under torchrun every rank runs an independent
replica (the path does not shard; no collective touches the data).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ePIE frame-updates/s at 256^2 px (fused path), error vs FP64 oracle"


def metric_name(N=256, path="fused"):
    """The live workload's metric at frame side N on the given path (the
    default frame side and path give METRIC)."""
    return f"ePIE frame-updates/s at {N}^2 px ({path} path), error vs FP64 oracle"

UNIT = "frame-updates/s"
CHUNK = 500
SM_COUNT = 152
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--geometry", default="A", choices=["A", "B"])
    ap.add_argument("--frames", type=int, default=10000)
    ap.add_argument("--frame-side", type=int, default=256, choices=[64, 128, 256, 512],
                    help="live workload at another frame side (probe FWHM 60 px x N/256); "
                         "the headline is 256")
    ap.add_argument("--path", default="fused", choices=["fused", "plain"])
    ap.add_argument("--graph", action="store_true",
                    help="replay each sweep's launches from a captured CUDA graph")
    ap.add_argument("--ctas-per-frame", type=int, default=0,
                    help="fused path: the step kernel's tile shape (0: the default for the "
                         "frame side; 1, 2 or 4 at 128^2)")
    ap.add_argument("--class-cap", type=int, default=0,
                    help="at most this many frames per colour class (0: no cap)")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-path comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-geometry-b", action="store_true",
                    help="skip the geometry-B sweeps (object about 1400^2)")
    ap.add_argument("--workers", type=int, default=min(16, os.cpu_count() or 1))
    ap.add_argument("--workload", default="live",
                    choices=["live", "multiscan", "adjoint", "live-schedule", "tc-gemm",
                             "oracle-cores", "parallel", "gemm-path"],
                    help="live: the headline 256^2 live scan; multiscan: eight uneven scans "
                         "sweeping concurrently; adjoint: amplitude-loss gradients at 128^2; "
                         "live-schedule: the whole live run, chunk by chunk; tc-gemm: the "
                         "tcgen05 GEMM of the DFT-as-GEMM path on its shapes; oracle-cores: "
                         "the FP64 oracle on one host core and on all of them (no GPU); "
                         "parallel: the paper's disjoint-subset averaging scheme; gemm-path: "
                         "the DFT-as-GEMM path at every operand precision against the FFT path")
    ap.add_argument("--gemm-variant", default=None,
                    help="gemm-path: run only this variant (e.g. \"tc bf16x3\") at --frame-side")
    ap.add_argument("--sweeps-per-chunk", type=int, default=50,
                    help="live-schedule: sweeps after each chunk (and at the end)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def fft_flops(N):
    """FFT work of one frame-update: two 2-D transforms of 5 K log2 K (K = N^2)."""
    K = N * N
    return 2 * 5.0 * K * math.log2(K)


def source_hash():
    """Hash of the 256^2 step kernel's code: its sources with // comments,
    trailing blanks and empty lines removed, so that a comment edit keeps a
    traffic record taken on the same code."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2308_10674_gb300", "csrc")
    for f in ("epie_fft.cuh", "epie_cluster.cuh", "epie_fused_256.cu"):
        with open(os.path.join(d, f)) as fh:
            for line in fh:
                code = line.split("//", 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def step_kernel_name(N, ctas_per_frame=0):
    """The fused step kernel that runs at frame side N and tile shape
    ctas_per_frame (0: the default shape)."""
    if N == 256:
        return "epie_fused256_kernel"
    if N == 512:
        return "epie_fused512_kernel"
    if N == 128:
        cl = ctas_per_frame or 4
        return "epie_fused128_kernel" if cl == 1 else f"epie_fused_kernel<128,{cl},...>"
    return f"epie_fused_kernel<{N},1,...>"


def measured_traffic():
    """DRAM bytes per frame of the fused 256^2 kernel from the committed ncu
    summary (key: value lines), if it was taken on the current kernel source
    (else None)."""
    p = os.path.join(ROOT, "profiles", "fused_256_traffic.txt")
    rec = {}
    try:
        with open(p) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    rec[k.strip()] = v.strip()
    except OSError:
        return None
    if rec.get("source_hash") != source_hash():
        return None
    try:
        rec["dram_bytes_per_frame"] = float(rec["dram_bytes_per_frame"])
    except (KeyError, ValueError):
        return None
    return rec


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            m = json.load(f)
        return m, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        # raw samples go to $EPIE_CLOCKS_DIR (default: the temp directory)
        self.path = os.path.join(os.environ.get("EPIE_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"epie_clocks_{os.getpid()}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}",
                                          f"--query-gpu={self.Q}", "--format=csv,noheader",
                                          "-lms", "100"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1].split()[0]), float(parts[2].split()[0]), parts))
                except ValueError:
                    continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for _, _, p in rows:
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": rows[0][1],
                "samples": len(rows), "reasons": sorted(reasons)}


def replica_rate(units, seconds, device="cpu"):
    """Whole-job throughput of independent replicas: the units all ranks
    processed divided by the slowest rank's time (max over ranks).  Works on
    any initialised process group (gloo on CPU tensors, NCCL on CUDA ones);
    without one it is units / seconds.  Returns (rate, max_seconds)."""
    try:
        import torch.distributed as dist
        active = dist.is_available() and dist.is_initialized()
    except ImportError:
        active = False
    if not active:
        return units / seconds, seconds
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / float(t.item()), float(t.item())


# --------------------------------------------------------------------------- data

def workload(args):
    from paper_2308_10674_gb300 import synth
    t = time.time()
    N = args.frame_side
    d = synth.live_scan(N=N, n=args.frames, geometry=args.geometry, seed=0,
                        workers=args.workers, fwhm=60.0 * N / 256)
    d["gen_s"] = time.time() - t
    return d


def workload_name(args, d):
    N = d["N"]
    return (f"live ePIE {N}^2 uint16, {args.frames} Fermat-spiral positions (step 0.35 FWHM, "
            f"FWHM {60 * N // 256} px), object {d['H']}x{d['W']} c64, 1e8 photons + Poisson + 2% dark, "
            f"coloured, chunks of {CHUNK}")


# --------------------------------------------------------------------------- CPU oracle

def oracle_sample(d, n_sample, seed=5, eps=0.0):
    """One coloured oracle sweep over the first n_sample frames from the start
    state (its probe optionally perturbed by eps, relative); returns
    (seconds, O, P, E)."""
    from oracle import oracle as orc
    N = d["N"]
    pos = d["pos"][:n_sample]
    I_all = orc.prepare_intensity(d["frames"][:n_sample], d["dark"])
    O = d["O0"].astype(np.complex64).astype(np.complex128)
    P = d["P0"].astype(np.complex64).astype(np.complex128)
    if eps:
        Z = np.random.default_rng(7).standard_normal(P.shape)
        P = P * (1 + eps * Z)
    t = time.perf_counter()
    col, ncls = orc.colour_greedy(pos, N)
    order, gs = orc.order_coloured(seed, 0, col, ncls)
    e, s = orc.sweep_groups(O, P, I_all, pos, order, gs)
    return time.perf_counter() - t, O, P, e / s


def calibrate_sample(d, target_s=15.0, lo=16, hi=1000):
    t, *_ = oracle_sample(d, 8)
    n = int(target_s / max(t / 8, 1e-4))
    return max(lo, min(hi, n))


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    d = workload(args)
    per_step = calibrate_sample(d, target_s=3.0, lo=8, hi=400)
    for _ in range(args.warmup):
        oracle_sample(d, per_step)
    tot = 0.0
    for _ in range(args.steps):
        t, *_ = oracle_sample(d, per_step)
        tot += t
    value = per_step * args.steps / tot
    sample = (f"one coloured FP64 oracle sweep over the first {per_step} frames of the workload "
              "per step, single thread")
    line = {"impl": "reference", "metric": metric_name(args.frame_side, args.path), "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tot / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args, d), "sample_frames": per_step},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- GPU

def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    device = local if ws > 1 else 0
    torch.cuda.set_device(device)
    from paper_2308_10674_gb300 import _binding as B

    d = workload(args)
    N, n = d["N"], len(d["pos"])
    assert n > CHUNK
    frames, pos = d["frames"], d["pos"]
    stream = torch.cuda.current_stream(device)
    path = B.EPIE_PATH_FUSED if args.path == "fused" else B.EPIE_PATH_PLAIN

    def make_engine(p=path, cap=n):
        eng = B.Engine(N, d["H"], d["W"], d["P0"], None, capacity=cap, mode=B.EPIE_COLOURED,
                       path=p, seed=5, device=device, stream=stream.cuda_stream,
                       class_cap=args.class_cap, flags=B.EPIE_GRAPH if args.graph else 0,
                       ctas_per_frame=args.ctas_per_frame if p == B.EPIE_PATH_FUSED else 0)
        eng.set_dark(d["dark"])
        return eng

    eng = make_engine()
    eng.append(frames[: n - CHUNK], pos[: n - CHUNK])
    chunk_pos = np.ascontiguousarray(pos[n - CHUNK:])
    chunk_dev = torch.from_numpy(frames[n - CHUNK:].view(np.int16)).to(f"cuda:{device}")
    chunk_host = torch.from_numpy(frames[n - CHUNK:].view(np.int16)).pin_memory().numpy()
    chunk_host = chunk_host.view(np.uint16)
    B.epie_append_frames_device(eng.h, chunk_dev.data_ptr(), chunk_pos, CHUNK)
    n_classes = eng.n_classes

    def step_device():
        eng.truncate(n - CHUNK)
        B.epie_append_frames_device(eng.h, chunk_dev.data_ptr(), chunk_pos, CHUNK)
        return eng.iterate(1)

    def step_host():
        eng.truncate(n - CHUNK)
        eng.append(chunk_host, chunk_pos)
        return eng.iterate(1)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(device)


    # ---- device-resident steps (value): nothing between the launches, so each
    # step kernel overlaps its prologue with the preceding kernel's tail
    for _ in range(args.warmup):
        step_device()
    launches0 = B.epie_launch_count(eng.h)
    errs = []
    with Clocks(device) as clk:
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        # one event at every step boundary too (each step ends with a host read
        # of its sweep error, so they add no wait between launches)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        ev0.record(stream)
        evs[0].record(stream)
        for k in range(args.steps):
            errs.append(float(step_device()[0]))
            evs[k + 1].record(stream)
        ev1.record(stream)
        barrier()
    step_ms = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)]
    dev_str = f"cuda:{device}"
    value, elapsed_s = replica_rate(n * args.steps, ev0.elapsed_time(ev1) / 1e3, dev_str)
    elapsed_ms = elapsed_s * 1e3
    launches = B.epie_launch_count(eng.h) - launches0
    clocks = clk.summary()

    # ---- per-launch durations of the step kernel: the same steps again with a
    # CUDA event pair around every fused launch on the engine's stream (the
    # events serialise the launches, so each is timed alone)
    B.epie_set_kernel_timing(eng.h, True)
    B.epie_kernel_timing(eng.h)
    ev2, ev3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    ev2.record(stream)
    for _ in range(args.steps):
        step_device()
    ev3.record(stream)
    barrier()
    k_launches, k_ms, k_frames = B.epie_kernel_timing(eng.h)
    B.epie_set_kernel_timing(eng.h, False)
    timed_steps_ms = ev2.elapsed_time(ev3) / args.steps

    # ---- end-to-end through the public API from pinned host memory
    for _ in range(max(1, args.warmup)):
        step_host()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step_host()
    barrier()
    e2e_value, _ = replica_rate(n * args.steps, time.perf_counter() - t0, dev_str)
    h2d = chunk_host.nbytes + chunk_pos.nbytes
    d2h = 8  # the sweep error
    eng.close()

    # ---- roofline of the dominant kernel (the fused step kernel)
    pk, pk_kind = peaks()
    kernel_avg_ms = k_ms / max(k_launches, 1)
    frames_per_launch = k_frames / max(k_launches, 1)
    flops_per_launch = fft_flops(N) * frames_per_launch
    achieved = flops_per_launch / (kernel_avg_ms / 1e3) / 1e12
    sm_mhz = pk.get("sm_max_mhz", 2070.0)
    peak_fp32 = SM_COUNT * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    fused = args.path == "fused"
    tr = measured_traffic() if (N == 256 and fused) else None
    traffic = None if tr is None else tr["dram_bytes_per_frame"] * frames_per_launch
    hbm_bytes_per_frame = N * N * 4  # the frame's fp32 measured-amplitude tile
    hbm_achieved = hbm_bytes_per_frame * frames_per_launch / (kernel_avg_ms / 1e3) / 1e9
    # measured FP32 FMA-chain rate, after the timed regions (its clock beside it)
    try:
        fma_tflops, fma_mhz = B.epie_fp32_fma_peak(0, 4096)
        fma = {"tflops": fma_tflops, "sm_mhz": fma_mhz, "frac": achieved / fma_tflops,
               "note": "FP32 FMA-chain kernel, 8 chains x 256 threads x 8 blocks per SM"}
    except B.EpieError as ex:
        fma = {"unavailable": str(ex)}
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_fp32, "unit": "TFLOP/s",
                "frac": achieved / peak_fp32, "traffic": traffic,
                "kernel": step_kernel_name(N, args.ctas_per_frame) if fused else
                          "plain path group (gather, cuFFT, modulus, cuFFT, update)",
                "flops_per_frame": fft_flops(N), "frames_per_launch": frames_per_launch,
                "avg_launch_ms": kernel_avg_ms, "launches": k_launches,
                "peak_note": (f"FP32 FMA peak = {SM_COUNT} SMs x {FP32_LANES_PER_SM} lanes x 2 "
                              f"x {sm_mhz:.0f} MHz (max clock from MEASURED_PEAKS.json)"),
                "hbm": {"achieved_gbs": hbm_achieved, "peak_gbs": pk["hbm_gbs"],
                        "frac": hbm_achieved / pk["hbm_gbs"], "peak_kind": pk_kind,
                        "bytes_per_frame": hbm_bytes_per_frame},
                "peak_measured_fma": fma,
                "kernel_share_of_step": k_ms / (timed_steps_ms * args.steps),
                "timing_region": (f"{args.steps} further steps with events around each fused "
                                  f"launch ({timed_steps_ms:.2f} ms per step there)")}

    line = {"metric": metric_name(N, args.path), "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
            "ms_per_step_median": statistics.median(step_ms),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": workload_name(args, d), "frames": n, "N": N,
                       "object": [d["H"], d["W"]], "colour_classes": n_classes,
                       "geometry": args.geometry, "path": args.path,
                       "class_cap": args.class_cap, "graph_replay": bool(args.graph),
                       "ctas_per_frame": args.ctas_per_frame,
                       "parallelism": f"replicas{ws}" if ws > 1 else "single GPU",
                       "l2": "inputs larger than L2 (frame set %.2f GB)" % (frames.nbytes / 1e9),
                       "sweep_error_last": errs[-1]},
            "clocks": clocks, "gpu_launches": launches, "roofline": roofline,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h}}

    # ---- geometry B of the live workload (object about 1400^2, step about
    # 9.7 px): the same frames and probe on a denser scan, hence many more and
    # much smaller colour classes
    if rank == 0 and args.geometry == "A" and N == 256 and not args.no_geometry_b:
        line["geometry_b"] = geometry_b(args, stream, device)

    # ---- the step kernel staging the raw uint16 rows (EPIE_RAW_INTENSITY) instead
    # of the amplitudes derived at append: sweeps over the same frames
    if rank == 0 and args.path == "fused" and not args.no_plain:
        re_ = B.Engine(N, d["H"], d["W"], d["P0"], None, capacity=n, mode=B.EPIE_COLOURED,
                       seed=5, device=device, stream=stream.cuda_stream,
                       flags=B.EPIE_RAW_INTENSITY)
        re_.set_dark(d["dark"])
        re_.append(frames, pos)
        re_.iterate(1)
        torch.cuda.synchronize(device)
        ksteps = max(2, args.steps // 2)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        re_.iterate(ksteps)
        e1.record(stream)
        torch.cuda.synchronize(device)
        rms = e0.elapsed_time(e1) / ksteps
        re_.close()
        line["raw_intensity_staging"] = {
            "value": n / (rms / 1e3), "unit": UNIT, "ms_per_sweep": rms,
            "hbm_bytes_per_frame": N * N * frames.itemsize,
            "note": "sweeps only (no ingest); the step kernel copies the uint16 rows by TMA and "
                    "converts them itself (EPIE_RAW_INTENSITY)"}

    # ---- plain unfused path on the same workload (speedup at the same accuracy)
    if rank == 0 and not args.no_plain and args.path == "fused":
        pe = make_engine(B.EPIE_PATH_PLAIN)
        pe.append(frames, pos)
        pe.iterate(1)
        torch.cuda.synchronize(device)
        ksteps = max(2, args.steps // 2)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pe.iterate(ksteps)
        e1.record(stream)
        torch.cuda.synchronize(device)
        pms = e0.elapsed_time(e1) / ksteps
        pe.close()
        line["plain_path"] = {"value": n / (pms / 1e3), "unit": UNIT, "ms_per_sweep": pms,
                              "fused_speedup": (n / (pms / 1e3)) and value / ws / (n / (pms / 1e3)),
                              "note": "sweeps only (no ingest); gather / cuFFT / modulus / cuFFT "
                                      "/ update / probe-reduce kernels"}

    # ---- CPU oracle baseline and GPU-vs-oracle error on the same sample
    if rank == 0 and ws == 1 and not args.no_cpu:
        n_s = calibrate_sample(d, target_s=10.0)
        secs, O_r, P_r, E_r = oracle_sample(d, n_s)
        _, O_p, P_p, E_p = oracle_sample(d, n_s, eps=1e-7)
        ge = make_engine(cap=n_s)
        ge.append(frames[:n_s], pos[:n_s])
        E_g = ge.iterate(1)[0]
        O_g, P_g = ge.object(), ge.probe()
        ge.close()
        rel = lambda a, b: float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))
        line["cpu_baseline"] = {"value": n_s / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"one coloured FP64 oracle sweep over the first {n_s} "
                                          f"frames of the workload ({secs:.1f} s, 1 thread)"}
        line["oracle_timings"] = oracle_timings(d, os.cpu_count() or 1)
        line["error_vs_oracle"] = {
            "sample_frames": n_s, "start": "paper's flat start (O = 1, phase-free aperture)",
            "rel_l2_object": rel(O_g, O_r), "rel_l2_probe": rel(P_g, P_r),
            "rel_sweep_error": abs(E_g - E_r) / E_r,
            "oracle_spread_1e-7": {"object": rel(O_p, O_r), "probe": rel(P_p, P_r),
                                   "sweep_error": abs(E_p - E_r) / E_r},
            "note": "one sweep over a long dependency chain from the flat start: the FP64 oracle "
                    "itself moves by oracle_spread_1e-7 when its start probe is perturbed by "
                    "1e-7; sharp 1e-5 parity is tested on well-conditioned chains"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def geometry_b(args, stream, device):
    """Sweeps of the live workload in geometry B (all frames resident, no
    ingest in the timed region): frame-updates/s, colour classes and the step
    kernel's roofline fraction."""
    import torch
    from paper_2308_10674_gb300 import _binding as B, synth
    N = 256
    d = synth.live_scan(N=N, n=args.frames, geometry="B", seed=0, workers=args.workers)
    n = len(d["pos"])
    eng = B.Engine(N, d["H"], d["W"], d["P0"], None, capacity=n, mode=B.EPIE_COLOURED, seed=5,
                   device=device, stream=stream.cuda_stream)
    eng.set_dark(d["dark"])
    eng.append(d["frames"], d["pos"])
    steps = max(3, args.steps // 2)
    eng.iterate(2)
    torch.cuda.synchronize(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    eng.iterate(steps)
    e1.record(stream)
    torch.cuda.synchronize(device)
    ms = e0.elapsed_time(e1) / steps
    B.epie_set_kernel_timing(eng.h, True)
    B.epie_kernel_timing(eng.h)
    eng.iterate(2)
    k_launches, k_ms, k_frames = B.epie_kernel_timing(eng.h)
    classes = eng.n_classes
    eng.close()
    pk, _ = peaks()
    avg = k_ms / max(k_launches, 1)
    fpl = k_frames / max(k_launches, 1)
    achieved = fft_flops(N) * fpl / (avg / 1e3) / 1e12
    peak = SM_COUNT * FP32_LANES_PER_SM * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    return {"value": n / (ms / 1e3), "unit": UNIT, "ms_per_sweep": ms, "frames": n,
            "object": [d["H"], d["W"]], "colour_classes": classes,
            "frames_per_launch": fpl, "avg_launch_ms": avg,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak},
            "note": "sweeps over all frames, no ingest in the timed region"}


# --------------------------------------------------------------------------- other workloads

MULTISCAN = [(128, 2000, "raster", "coloured"), (128, 4096, "jittered", "minibatch"),
             (128, 9000, "spiral", "coloured"), (256, 3000, "raster", "minibatch"),
             (256, 12000, "spiral", "coloured"), (512, 1024, "raster", "coloured"),
             (512, 4096, "jittered", "minibatch"), (512, 8000, "spiral", "minibatch")]


def run_multiscan(args):
    """Eight independent scans of uneven size (128^2 / 256^2 / 512^2 frames,
    raster / jittered raster / spiral, FP16 intensity storage, noise-free
    model intensities) sweeping concurrently with graph-replayed sweeps;
    mini-batch sizes and the 128^2 tile shapes picked by the autotuner.
    Beside the concurrent rate it times every scan's sweep alone: the longest
    of those is the critical path that no schedule of the eight (streams or
    one persistent launch) can beat, because each scan's groups run one
    after the other."""
    import torch
    from paper_2308_10674_gb300 import _binding as B, autotune, synth
    torch.cuda.set_device(0)
    scans, engines, chosen = [], [], []
    t0 = time.time()
    for i, (N, n, pat, mode) in enumerate(MULTISCAN):
        d = synth.scan(N, n, pat, seed=100 + i, noise=False, dtype=np.float16, workers=args.workers)
        scans.append(d)
    gen_s = time.time() - t0
    for (N, n, pat, mode), d in zip(MULTISCAN, scans):
        m = B.EPIE_MINIBATCH if mode == "minibatch" else B.EPIE_COLOURED
        best, _ = autotune.tune(d, mode=m, intensity_dtype=B.EPIE_F16, graph=(True,))
        batch = best["batch"] if m == B.EPIE_MINIBATCH else 64
        tile = best.get("ctas_per_frame", 0)
        chosen.append({"N": N, "frames": n, "pattern": pat, "mode": mode,
                       "batch": batch if m == B.EPIE_MINIBATCH else None,
                       "ctas_per_frame": tile})
        e = B.Engine(N, d["H"], d["W"], d["P0"], None, capacity=n, mode=m, batch=batch, seed=5,
                     intensity_dtype=B.EPIE_F16, flags=B.EPIE_GRAPH, ctas_per_frame=tile)
        e.append(d["frames"], d["pos"])
        engines.append(e)
    handles = [e.h for e in engines]
    total = sum(len(d["pos"]) for d in scans)
    for _ in range(args.warmup):
        B.epie_iterate_many(handles, 1)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(args.steps):
        B.epie_iterate_many(handles, 1)
    conc = (time.perf_counter() - t) / args.steps
    t = time.perf_counter()
    alone = [0.0] * len(engines)
    for _ in range(args.steps):
        for i, e in enumerate(engines):
            e.iterate(1)
            alone[i] += e.last_timing()[0] / args.steps
    seq = (time.perf_counter() - t) / args.steps
    launches = sum(B.epie_launch_count(h) for h in handles)
    for e in engines:
        e.close()
    line = {"metric": "multi-scan ePIE frame-updates/s (8 uneven scans, concurrent sweeps)",
            "value": total / conc, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": conc * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "8 independent scans, FP16 intensity storage", "scans": chosen,
                       "frames_total": total, "generation_s": gen_s},
            "back_to_back": {"value": total / seq, "ms_per_step": seq * 1e3,
                             "concurrency_speedup": seq / conc},
            "critical_path": {"ms_per_sweep_alone": alone, "longest_ms": max(alone),
                              "concurrent_over_longest": conc * 1e3 / max(alone)},
            "gpu_launches_total": launches}
    print(json.dumps(line), flush=True)
    return 0


def adjoint_roofline(n, ms, N=128):
    """The gradient evaluation runs four 2-D transforms per position (the
    probe's Fourier shift, the far field, the far field's adjoint and the
    shift's adjoint) on the FP32 pipes: 4 x 5 K log2 K FLOP, against the FP32
    FMA peak."""
    pk, _ = peaks()
    flops = 4 * 5 * N * N * math.log2(N * N)
    achieved = n * flops / (ms / 1e3) / 1e12
    peak = SM_COUNT * FP32_LANES_PER_SM * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": None, "flops_per_position": flops,
            "note": "whole gradient call (all its kernels) per position"}


def run_adjoint(args):
    """Amplitude-loss gradients (object, probe, sub-pixel positions) at 128^2:
    4,096 jittered-raster positions, object 642 x 642; gradient evaluations
    per second and a 200-step Adam reconstruction from the flat start."""
    import torch
    from paper_2308_10674_gb300 import synth
    from paper_2308_10674_gb300.autograd import amplitude_loss, frames_to_fft_order
    dev = torch.device("cuda", 0)
    d = synth.small_scan(128, 64, 64, 8, seed=9, photons=1e7)
    fr = frames_to_fft_order(torch.from_numpy(d["frames"].view(np.int16)).to(dev))
    pos = torch.from_numpy(d["pos"].astype(np.int32)).to(dev)
    n = len(d["pos"])
    o = torch.ones(d["H"], d["W"], dtype=torch.complex64, device=dev).requires_grad_()
    p = torch.from_numpy(d["P0"].astype(np.complex64)).to(dev).requires_grad_()
    s = torch.zeros(n, 2, dtype=torch.float32, device=dev, requires_grad=True)
    for _ in range(args.warmup):
        amplitude_loss(o, p, s, fr, pos).backward()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        amplitude_loss(o, p, s, fr, pos).backward()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    opt = torch.optim.Adam([{"params": [o], "lr": 2e-2}, {"params": [p], "lr": 2e-3},
                            {"params": [s], "lr": 1e-3}])
    losses = []
    for it in range(200):
        opt.zero_grad()
        loss = amplitude_loss(o, p, s, fr, pos)
        loss.backward()
        opt.step()
        losses.append(loss.item())
    line = {"metric": "amplitude-loss gradient position-evaluations/s at 128^2",
            "value": n / (ms / 1e3), "unit": "positions/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{n} jittered-raster positions, 128^2 uint16, object "
                                   f"{d['H']}x{d['W']}, gradients for object, probe, shifts"},
            "roofline": adjoint_roofline(n, ms),
            "adam_200": {"loss_first": losses[0], "loss_last": losses[-1],
                         "finite": bool(np.all(np.isfinite(losses)))}}
    print(json.dumps(line), flush=True)
    return 0


def run_live_schedule(args):
    """The paper's live run on the bench workload (Sec. "Live ePIE"; Results,
    "Live processing"): chunks of 500 frames arrive from pinned host memory,
    k sweeps follow each chunk over every frame present, and k final sweeps
    end the run.  Reports the wall clock of the whole run and, per chunk, the
    sweep time and how many sweeps fit between chunks arriving at 10 frames/s
    (the paper's engine managed 50 early on and about 6 at the end)."""
    import torch
    from paper_2308_10674_gb300 import _binding as B
    torch.cuda.set_device(0)
    d = workload(args)
    N, n, k = d["N"], len(d["pos"]), args.sweeps_per_chunk
    stream = torch.cuda.current_stream(0)
    host = torch.from_numpy(d["frames"].view(np.int16)).pin_memory().numpy().view(np.uint16)
    pos = np.ascontiguousarray(d["pos"])

    def run(record):
        eng = B.Engine(N, d["H"], d["W"], d["P0"], None, capacity=n, mode=B.EPIE_COLOURED,
                       seed=5, device=0, stream=stream.cuda_stream)
        eng.set_dark(d["dark"])
        rows, fu = [], 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for c in range(0, n, CHUNK):
            m = min(CHUNK, n - c)
            eng.append(host[c:c + m], pos[c:c + m])
            ta = time.perf_counter()
            errs = eng.iterate(k)
            sweep_s = (time.perf_counter() - ta) / k
            fu += k * (c + m)
            if record:
                rows.append({"frames": c + m, "classes": eng.n_classes,
                             "ms_per_sweep": sweep_s * 1e3, "E_last": float(errs[-1]),
                             "sweeps_between_chunks_at_10fps": (CHUNK / 10.0) / sweep_s})
        errs = eng.iterate(k)
        fu += k * n
        wall = time.perf_counter() - t0
        eng.close()
        return wall, fu, rows, float(errs[-1])

    run(False)  # warm-up: first-use set-up (plans, graphs of the allocator, clocks)
    with Clocks(0) as clk:
        wall, fu, rows, e_final = run(True)
    line = {"metric": "live ePIE run, frame-updates/s over the whole schedule (appends included)",
            "value": fu / wall, "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": wall * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(args, d), "sweeps_per_chunk": k,
                       "final_sweeps": k, "frame_updates": fu},
            "clocks": clk.summary(), "wall_s": wall, "E_final": e_final,
            "per_chunk": rows[::4] + ([rows[-1]] if (len(rows) - 1) % 4 else []),
            "paper_engine_sweeps_between_chunks": "50 early, about 6 at the end"}
    print(json.dumps(line), flush=True)
    return 0


TC_SHAPES = [(262144, 512, 512, "256^2 DFT rows, 1024 frames"),
             (131072, 256, 256, "128^2 DFT rows, 1024 frames"),
             (65536, 1024, 1024, "512^2 DFT rows, 128 frames"),
             (16384, 4096, 4096, "square")]


def run_tc_gemm(args):
    """The engine's tcgen05 GEMM (epie_tc_gemm_bf16, D = sum_t A_t B_t^T, bf16
    operands, fp32 accumulation and output) on the DFT-as-GEMM path's shapes,
    one and three (split bf16) terms, against cuBLAS bf16 (torch.matmul).
    The headline line is the 256^2 DFT shape with three terms."""
    import torch
    from paper_2308_10674_gb300 import _binding as B
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    pk, pk_kind = peaks()
    st = torch.cuda.current_stream().cuda_stream
    rows, launches = [], 0

    def timed(f, reps):
        for _ in range(max(3, args.warmup)):
            f()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            f()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    with Clocks(0) as clk:
        for M, Nn, K, what in TC_SHAPES:
            g = torch.Generator(device=dev).manual_seed(M + Nn)
            A0 = torch.randn(M, K, device=dev, generator=g).to(torch.bfloat16)
            A1 = (torch.randn(M, K, device=dev, generator=g) * 2 ** -8).to(torch.bfloat16)
            B0 = torch.randn(Nn, K, device=dev, generator=g).to(torch.bfloat16)
            B1 = (torch.randn(Nn, K, device=dev, generator=g) * 2 ** -8).to(torch.bfloat16)
            D = torch.empty(M, Nn, device=dev)
            status = torch.zeros(1, dtype=torch.int32, device=dev)
            for terms in (1, 3):
                f = lambda: B.epie_tc_gemm_bf16(A0.data_ptr(), A1.data_ptr(), B0.data_ptr(),
                                                B1.data_ptr(), D.data_ptr(), M, Nn, K, Nn, terms,
                                                status.data_ptr(), st)
                ms = timed(f, args.steps * 2)
                launches += args.steps * 2
                if int(status.item()):
                    raise RuntimeError("tcgen05 GEMM reported a wait time-out")
                nbytes = M * K * 2 * (2 if terms == 3 else 1) + Nn * K * 2 * 2 + M * Nn * 4
                rows.append({"shape": [M, Nn, K], "what": what, "terms": terms, "ms": ms,
                             "tflops": 2.0 * M * Nn * K * terms / ms / 1e9,
                             "hbm_gbs": nbytes / ms / 1e6})
            ms = timed(lambda: torch.matmul(A0, B0.t()), args.steps * 2)
            rows.append({"shape": [M, Nn, K], "what": what, "cublas_bf16_ms": ms,
                         "tflops": 2.0 * M * Nn * K / ms / 1e9})
            del A0, A1, B0, B1
            if what != "square":  # fp32 operands read as tf32 (kind::tf32)
                F = [torch.randn(r, K, device=dev, generator=g) for r in (M, M, Nn, Nn)]
                for terms in (1, 3):
                    f = lambda: B.epie_tc_gemm_tf32(F[0].data_ptr(), F[1].data_ptr(),
                                                    F[2].data_ptr(), F[3].data_ptr(),
                                                    D.data_ptr(), M, Nn, K, Nn, terms,
                                                    status.data_ptr(), st)
                    ms = timed(f, args.steps * 2)
                    launches += args.steps * 2
                    if int(status.item()):
                        raise RuntimeError("tcgen05 GEMM reported a wait time-out")
                    nbytes = M * K * 4 * (2 if terms == 3 else 1) + Nn * K * 4 * 2 + M * Nn * 4
                    rows.append({"shape": [M, Nn, K], "what": what, "operands": "tf32",
                                 "terms": terms, "ms": ms,
                                 "tflops": 2.0 * M * Nn * K * terms / ms / 1e9,
                                 "hbm_gbs": nbytes / ms / 1e6})
                del F
            del D
            torch.cuda.empty_cache()
    head = rows[1]  # 256^2 DFT rows, three terms
    M, Nn, K = head["shape"]
    line = {"metric": "tcgen05 DFT-as-GEMM, 256^2 rows of 1024 frames, split-bf16 (3 products)",
            "value": head["tflops"], "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps * 2,
            "warmup": max(3, args.warmup), "ms_per_step": head["ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "D = A B^T, A 262144x512, B 512x512 bf16, fp32 D",
                       "l2": "inputs larger than L2"},
            "clocks": clk.summary(), "gpu_launches": launches,
            "roofline": {"bound": "hbm", "achieved": head["hbm_gbs"], "peak": pk["hbm_gbs"],
                         "unit": "GB/s", "frac": head["hbm_gbs"] / pk["hbm_gbs"], "traffic": None,
                         "peak_kind": pk_kind,
                         "tensor": {"achieved_tflops": head["tflops"],
                                    "peak_tflops": pk.get("bf16_tflops"),
                                    "frac": head["tflops"] / pk["bf16_tflops"]
                                    if pk.get("bf16_tflops") else None}},
            "shapes": rows}
    print(json.dumps(line), flush=True)
    return 0


def run_parallel(args):
    """The paper's parallel scheme on the live workload: the 10,000 positions
    split round-robin into S disjoint subsets, each subset sweeping on its own
    stream (epie_iterate_many), then object and probe averaged on the device;
    one sweep per round.  S = 1 is the plain coloured sweep."""
    import torch
    from paper_2308_10674_gb300 import _binding as B
    from paper_2308_10674_gb300.parallel import ParallelAveraging
    torch.cuda.set_device(0)
    d = workload(args)
    n = len(d["pos"])
    rows = []
    with Clocks(0) as clk:
        for S in (1, 2, 4, 8):
            idx = [np.arange(q, n, S) for q in range(S)]
            with ParallelAveraging(256, d["H"], d["W"], d["P0"], [d["pos"][i] for i in idx],
                                   mode=B.EPIE_COLOURED, seed=5) as par:
                for q, i in enumerate(idx):
                    par.engines[q].set_dark(d["dark"])
                    par.append(q, d["frames"][i], d["pos"][i])
                for _ in range(args.warmup):
                    par.round(1)
                torch.cuda.synchronize()
                t = time.perf_counter()
                for _ in range(args.steps):
                    errs = par.round(1)
                torch.cuda.synchronize()
                dt = (time.perf_counter() - t) / args.steps
            rows.append({"subsets": S, "ms_per_round": dt * 1e3, "frame_updates_per_s": n / dt,
                         "sweep_error_mean": float(np.mean(errs))})
    best = max(rows, key=lambda r: r["frame_updates_per_s"])
    line = {"metric": "parallel-averaging ePIE frame-updates/s (disjoint subsets, one sweep "
                      "per round, then the average)",
            "value": best["frame_updates_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": best["ms_per_round"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": workload_name(args, d),
                                            "subsets": best["subsets"]},
            "clocks": clk.summary(), "by_subsets": rows}
    print(json.dumps(line), flush=True)
    return 0


def run_gemm_path(args):
    """The step with its 2-D DFT done as dense GEMMs, at every operand
    precision (cuBLAS and the engine's own tcgen05 kernel), against the fused
    FFT path: mini-batch sweeps (B = 1024) over 16,384 Fermat-spiral positions
    of the live model (geometry B) at 128^2 and 256^2."""
    import torch
    from paper_2308_10674_gb300 import _binding as B, synth
    torch.cuda.set_device(0)
    V = [("fused FFT", B.EPIE_PATH_FUSED, 0), ("bf16", B.EPIE_PATH_GEMM, B.EPIE_GEMM_BF16),
         ("tf32", B.EPIE_PATH_GEMM, B.EPIE_GEMM_TF32),
         ("bf16x3", B.EPIE_PATH_GEMM, B.EPIE_GEMM_BF16X3),
         ("fp32 emulation", B.EPIE_PATH_GEMM, B.EPIE_GEMM_FP32EMU),
         ("tc bf16", B.EPIE_PATH_GEMM, B.EPIE_GEMM_TC_BF16),
         ("tc bf16x3", B.EPIE_PATH_GEMM, B.EPIE_GEMM_TC_BF16X3),
         ("tc tf32", B.EPIE_PATH_GEMM, B.EPIE_GEMM_TC_TF32),
         ("tc tf32x3", B.EPIE_PATH_GEMM, B.EPIE_GEMM_TC_TF32X3)]
    sides = (128, 256)
    if args.gemm_variant is not None:
        V = [v for v in V if v[0] == args.gemm_variant]
        if not V:
            raise SystemExit(f"unknown --gemm-variant {args.gemm_variant!r}")
        sides = (args.frame_side,)
    rows = []
    with Clocks(0) as clk:
        for N in sides:
            n = 16384
            d = synth.live_scan(N=N, n=n, geometry="B", seed=0, workers=args.workers,
                                fwhm=60.0 * N / 256)
            for name, path, prec in V:
                eng = B.Engine(N, d["H"], d["W"], d["P0"], None, capacity=n,
                               mode=B.EPIE_MINIBATCH, batch=1024, seed=5, path=path,
                               gemm_precision=prec)
                eng.set_dark(d["dark"])
                eng.append(d["frames"], d["pos"])
                eng.iterate(max(1, args.warmup))
                torch.cuda.synchronize()
                t = time.perf_counter()
                errs = eng.iterate(args.steps)
                dt = (time.perf_counter() - t) / args.steps
                eng.close()
                rows.append({"N": N, "path": name, "frame_updates_per_s": n / dt,
                             "ms_per_sweep": dt * 1e3, "sweep_error": float(errs[-1])})
    ref = ([r for r in rows if r["N"] == 256 and r["path"] == "tc bf16x3"] or rows)[0]
    line = {"metric": "DFT-as-GEMM ePIE frame-updates/s at 256^2 (tcgen05 split bf16), "
                      "mini-batch B = 1024",
            "value": ref["frame_updates_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ref["ms_per_sweep"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3", "data": "synthetic",
            "config": {"workload": "16,384 Fermat-spiral positions, geometry B, mini-batch 1024"},
            "clocks": clk.summary(), "paths": rows}
    print(json.dumps(line), flush=True)
    return 0


def _oracle_window(job):
    """One coloured FP64 oracle sweep over a window of the workload's frames
    from the paper's flat start; returns its compute seconds."""
    frames, pos, dark, P0, H, W, N = job
    from oracle import oracle as orc
    I_all = orc.prepare_intensity(frames, dark)
    O = np.ones((H, W), np.complex128)
    P = P0.astype(np.complex64).astype(np.complex128)
    t = time.perf_counter()
    col, ncls = orc.colour_greedy(pos, N)
    order, gs = orc.order_coloured(5, 0, col, ncls)
    orc.sweep_groups(O, P, I_all, pos, order, gs)
    return time.perf_counter() - t


def _oracle_config0(_):
    """The FP64 oracle on config 0 in full: 256 positions of 64^2, ten
    sequential sweeps from the flat start (one process)."""
    from oracle import oracle as orc
    from paper_2308_10674_gb300 import synth
    d = synth.config0(seed=0)
    I_all = orc.prepare_intensity(d["frames"])
    O, P = d["O0"].astype(np.complex128), d["P0"].astype(np.complex128)
    t = time.perf_counter()
    orc.run_sweeps(O, P, I_all, d["pos"], 10, d["N"], seed=0)
    return time.perf_counter() - t


def oracle_timings(d, cores):
    """The FP64 oracle as it stands, on the host cores of this run: config 0
    in full on one core, and one coloured sweep over 500 and over 2,000
    frames of the live 256^2 workload on one core and on all cores (one
    process per core, each on its own window of the workload)."""
    import multiprocessing as mp
    n = len(d["pos"])
    out = {"cores": cores}
    with mp.get_context("spawn").Pool(1) as pool:
        t0 = pool.map(_oracle_config0, [0])[0]
    out["config0_full"] = {"frame_updates": 2560, "seconds": t0, "value": 2560 / t0, "cores": 1}
    for n_w in (500, 2000):
        jobs = []
        for k in range(cores):
            a = (k * n_w) % max(n - n_w, 1)
            jobs.append((d["frames"][a:a + n_w], d["pos"][a:a + n_w], d["dark"], d["P0"], d["H"],
                         d["W"], d["N"]))
        t1 = _oracle_window(jobs[0])
        with mp.get_context("spawn").Pool(cores) as pool:
            times = pool.map(_oracle_window, jobs)
        out[f"live_{n_w}"] = {"one_core": n_w / t1, "all_cores": sum(n_w / t for t in times),
                              "seconds_one_core": t1, "max_seconds_all_cores": max(times)}
    return out


def run_oracle_cores(args):
    """The FP64 oracle as it stands on the host: one coloured sweep over a
    500-frame window of the live workload on one core, then one window per
    core on all cores at once (disjoint windows, one process each).  No GPU."""
    import multiprocessing as mp
    d = workload(args)
    n_w, cores = 500, os.cpu_count() or 1
    n = len(d["pos"])
    jobs = []
    for k in range(cores):
        a = (k * n_w) % (n - n_w)
        jobs.append((d["frames"][a:a + n_w], d["pos"][a:a + n_w], d["dark"], d["P0"], d["H"],
                     d["W"], d["N"]))
    t1 = _oracle_window(jobs[0])
    with mp.get_context("spawn").Pool(cores) as pool:
        times = pool.map(_oracle_window, jobs)
    one = n_w / t1
    all_cores = sum(n_w / t for t in times)
    line = {"metric": "FP64 oracle frame-updates/s on the host, one core and all cores",
            "value": all_cores, "unit": UNIT, "n_gpus": 0, "steps": 1, "warmup": 0,
            "ms_per_step": max(times) * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args, d), "window_frames": n_w},
            "cpu_baseline": {"value": all_cores, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{cores} disjoint {n_w}-frame windows, one coloured "
                                       f"sweep each, one process per core, concurrently"},
            "one_core": {"value": one, "seconds": t1},
            "per_core_seconds": times}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "multiscan":
        return run_multiscan(args)
    if args.workload == "adjoint":
        return run_adjoint(args)
    if args.workload == "live-schedule":
        return run_live_schedule(args)
    if args.workload == "tc-gemm":
        return run_tc_gemm(args)
    if args.workload == "oracle-cores":
        return run_oracle_cores(args)
    if args.workload == "parallel":
        return run_parallel(args)
    if args.workload == "gemm-path":
        return run_gemm_path(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
