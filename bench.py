"""Benchmark: spectral Ewald Stokeslet apply on one GB300 (or N replicas).

A step is one full apply (bin, P2P, P2G, FFT, CNV, IFFT, G2P, SUM) over the
N = 100,000 uniform workload at tol 1e-6 (M = 128, P = 12), FP32-bulk; the
plain FP64 apply on the same points is timed beside it.  Inputs are resident
in HBM; they are smaller than L2, so a 256 MB buffer is rewritten between
timed steps (outside the per-step events) to flush L2.

Prints one JSON line.  `--impl reference` times the CPU FP64 oracle instead
(the only other place this script runs oracle/ code besides `cpu_baseline`).

Multi-GPU (torchrun, one rank per GPU): independent replicas, one workload
per rank, no collective on the data path ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "uniform_1e5_tol1e-6_M128_P12"
METRIC = "particle-applies/s at tol 1e-6 (FP32-bulk vs FP64 plain); per-stage roofline %; p50/p99"
UNIT = "particle-applies/s"
FP32_FLOPS_PER_INRANGE = 52      # FP32 pair kernel, FMA = 2 flops, MUFU = 1
FLOPS_PER_CANDIDATE = 8          # difference + squared distance per tested pair
N_SM = 152
FP32_LANES = 128


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_traffic(kernel_file: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current source of the kernel (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    src = os.path.join(ROOT, "paper_2606_19059_gb300", "csrc", kernel_file)
    try:
        with open(path) as fh:
            d = json.load(fh)
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()
        e = d.get(kernel_file)
        if e and e.get("sha256") == digest and e.get("workload") == WORKLOAD:
            return float(e["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


def pair_counts(x: np.ndarray, L: float, rc: float, nc: int):
    """Exact in-range pair count (0 < |r| <= rc, periodic) and the number of
    27-cell candidate pairs the P2P kernel tests."""
    from scipy.spatial import cKDTree

    xw = np.mod(x, L)
    xw[xw >= L] = 0.0
    tree = cKDTree(xw, boxsize=L)
    inrange = int(tree.count_neighbors(tree, rc)) - x.shape[0]   # drop self pairs
    c = np.minimum((xw / (L / nc)).astype(np.int64), nc - 1)
    occ = np.zeros((nc, nc, nc), dtype=np.int64)
    np.add.at(occ, (c[:, 2], c[:, 1], c[:, 0]), 1)
    nb = np.zeros_like(occ)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                nb += np.roll(occ, (dz, dy, dx), axis=(0, 1, 2))
    cand = int((occ * nb).sum())
    return inrange, cand


def run_gpu(args, rank, world):
    import torch

    from paper_2606_19059_gb300 import ewald, workloads

    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    kind, N, L, tol, M, P, seed = workloads.WORKLOADS[WORKLOAD]
    x, f = workloads.make(kind, N, seed + rank, L)
    xd = torch.tensor(x, device=dev)
    fd = torch.tensor(f, device=dev)
    ud = torch.empty_like(xd)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream

    def timed(plan, steps, warmup):
        for _ in range(warmup):
            ewald.ewald_apply(plan.handle, xd.data_ptr(), fd.data_ptr(), ud.data_ptr(), sp)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for a, b in evs:
            flush.zero_()                      # L2 flush between timed steps
            a.record(stream)
            ewald.ewald_apply(plan.handle, xd.data_ptr(), fd.data_ptr(), ud.data_ptr(), sp)
            b.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        ms = [a.elapsed_time(b) for a, b in evs]
        return ms, wall

    if args.only_split:  # profiling runs: FP32 bulk at tol 1e-8 on the same points (split near field)
        pds = ewald.Plan(N, L, 1e-8, ewald.EWALD_F32_BULK)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for k in range(args.warmup + args.steps):
            if k == args.warmup:
                torch.cuda.synchronize()
                a.record(stream)
            ewald.ewald_apply(pds.handle, xd.data_ptr(), fd.data_ptr(), ud.data_ptr(), sp)
        b.record(stream)
        torch.cuda.synchronize()
        print(json.dumps({"only_split": True, "M": pds.params.M, "ms_per_step": a.elapsed_time(b) / args.steps}))
        pds.close()
        return None
    plan32 = ewald.Plan(N, L, tol, ewald.EWALD_F32_BULK, M=M, P=P)
    if args.only_double_layer:  # profiling runs: the combined applies alone
        rng = np.random.default_rng(seed + 7 + rank)
        qd = torch.tensor(rng.standard_normal((N, 3)), device=dev)
        nd = torch.tensor(rng.standard_normal((N, 3)), device=dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for k in range(args.warmup + args.steps):
            if k == args.warmup:
                torch.cuda.synchronize()
                a.record(stream)
            ewald.ewald_apply_combined(plan32.handle, xd.data_ptr(), fd.data_ptr(), qd.data_ptr(),
                                       nd.data_ptr(), ud.data_ptr(), sp)
        b.record(stream)
        torch.cuda.synchronize()
        print(json.dumps({"only_double_layer": True, "ms_per_step": a.elapsed_time(b) / args.steps}))
        plan32.close()
        return None
    with ClockSampler(local) as clk:
        ms32, wall32 = timed(plan32, args.steps, args.warmup)
    clocks = clk.summary()
    if plan32.sync_status() != ewald.EWALD_OK:
        raise RuntimeError("device error during the timed applies")
    if args.only_f32:  # profiling runs: the timed FP32 applies alone
        print(json.dumps({"only_f32": True, "ms_per_step": float(np.mean(ms32))}))
        plan32.close()
        return None

    # per-stage device times with serialised stages (CUDA events on the launching stream)
    ewald.ewald_set_timing(plan32.handle, 2)
    stage = []
    for _ in range(max(3, args.steps // 2)):
        flush.zero_()
        ewald.ewald_apply(plan32.handle, xd.data_ptr(), fd.data_ptr(), ud.data_ptr(), sp)
        stage.append(ewald.ewald_stage_times(plan32.handle))
    ewald.ewald_set_timing(plan32.handle, 0)
    stages = {k: statistics.median([s[k] for s in stage]) for k in stage[0]}

    # plain FP64 apply, same points
    plan64 = ewald.Plan(N, L, tol, ewald.EWALD_F64, M=M, P=P)
    ms64, _ = timed(plan64, max(3, args.steps // 4), max(1, args.warmup // 2))

    # end to end through the C ABI with pinned host buffers (copies inside the timing)
    xh = torch.from_numpy(x.copy()).pin_memory()
    fh = torch.from_numpy(f.copy()).pin_memory()
    uh = torch.empty_like(xh).pin_memory()
    for _ in range(3):  # direct, replayed and direct again: the plan keeps the faster
        ewald.ewald_apply_host(plan32.handle, xh.data_ptr(), fh.data_ptr(), uh.data_ptr(), sp)
    e2e = []
    for _ in range(max(3, args.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        ewald.ewald_apply_host(plan32.handle, xh.data_ptr(), fh.data_ptr(), uh.data_ptr(), sp)
        e2e.append(time.perf_counter() - t)

    # combined single and double layer apply (Sec. 2.3) on the same points:
    # synthetic source vectors q, n ~ N(0, 1) per component
    dl = None
    if not args.no_double_layer:
        rng = np.random.default_rng(seed + 7 + rank)
        qd = torch.tensor(rng.standard_normal((N, 3)), device=dev)
        nd = torch.tensor(rng.standard_normal((N, 3)), device=dev)

        def combined():
            ewald.ewald_apply_combined(plan32.handle, xd.data_ptr(), fd.data_ptr(), qd.data_ptr(),
                                       nd.data_ptr(), ud.data_ptr(), sp)

        for _ in range(3):
            combined()
        torch.cuda.synchronize()
        ms_dl = []
        for _ in range(max(3, args.steps // 20)):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            combined()
            b.record(stream)
            b.synchronize()
            ms_dl.append(a.elapsed_time(b))
        ewald.ewald_set_timing(plan32.handle, 2)
        flush.zero_()
        combined()
        st_dl = ewald.ewald_stage_times(plan32.handle)
        ewald.ewald_set_timing(plan32.handle, 0)
        dl = {"ms": ms_dl, "stages": st_dl}

    kern, nfft = ewald.ewald_launch_counts(plan32.handle)
    prm = plan32.params
    res = {
        "ms32": ms32, "wall32": wall32, "ms64": ms64, "stages": stages, "e2e_s": e2e, "dl": dl,
        "clocks": clocks, "kernels_per_step": kern, "ffts_per_step": nfft, "params": prm.as_dict(),
        "N": N, "L": L, "tol": tol, "M": M, "P": P, "x": x if rank == 0 else None,
    }
    plan32.close()
    plan64.close()
    return res


CLUSTERED = "clustered_2e6_tol1e-7_M256_P14"


def run_clustered(args, rank, world):
    """The clustered workload (N = 2e6: 200 Gaussian blobs plus 20 % uniform
    background, tol 1e-7, M = 256, P = 14): FP32-bulk applies (double-single
    near field and grid at this tolerance, FP64 FFT), per-stage times, and the
    plain FP64 apply beside them.  Inputs and plan workspaces (~2.5 GB) exceed
    L2; the flush buffer is rewritten between timed steps all the same."""
    import torch

    from paper_2606_19059_gb300 import ewald, workloads

    local = int(os.environ.get("LOCAL_RANK", 0))
    dev = torch.device("cuda", local)
    kind, N, L, tol, M, P, seed = workloads.WORKLOADS[CLUSTERED]
    x, f = workloads.make(kind, N, seed + rank, L)
    xd, fd = torch.tensor(x, device=dev), torch.tensor(f, device=dev)
    ud = torch.empty_like(xd)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream

    def timed(plan, steps, warmup):
        for _ in range(warmup):
            ewald.ewald_apply(plan.handle, xd.data_ptr(), fd.data_ptr(), ud.data_ptr(), sp)
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ewald.ewald_apply(plan.handle, xd.data_ptr(), fd.data_ptr(), ud.data_ptr(), sp)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        return ms

    p32 = ewald.Plan(N, L, tol, ewald.EWALD_F32_BULK, M=M, P=P)
    ms32 = timed(p32, max(3, min(args.steps, 5)), 2)
    if p32.sync_status() != ewald.EWALD_OK:
        raise RuntimeError("device error during the clustered applies")
    ewald.ewald_set_timing(p32.handle, 2)
    flush.zero_()
    ewald.ewald_apply(p32.handle, xd.data_ptr(), fd.data_ptr(), ud.data_ptr(), sp)
    stages = ewald.ewald_stage_times(p32.handle)
    ewald.ewald_set_timing(p32.handle, 0)
    prm = p32.params.as_dict()
    p32.close()
    p64 = ewald.Plan(N, L, tol, ewald.EWALD_F64, M=M, P=P)
    ms64 = timed(p64, 2, 1)
    p64.close()
    ms, rate = job_time_and_rate(float(np.mean(ms32)), N, world)
    m64, rate64 = job_time_and_rate(float(np.mean(ms64)), N, world)
    return {"ms": ms, "value": rate, "ms64": m64, "value64": rate64, "stages": stages, "params": prm,
            "N": N, "L": L, "tol": tol, "M": M, "P": P, "x": x if rank == 0 else None, "steps": len(ms32)}


def clustered_entry(c, peaks):
    """The bench line's clustered object: rates, stage times, the HBM-bound
    stages' fractions and the near field's in-range pair rate."""
    from scipy.spatial import cKDTree

    N, L, M, prm, st = c["N"], c["L"], c["M"], c["params"], c["stages"]
    # in-range pairs (0 < |r| <= rc, periodic), estimated from 2 % of the
    # targets against all sources (the full count takes minutes on the host)
    xw = np.mod(c["x"], L)
    xw[xw >= L] = 0.0
    tree = cKDTree(xw, boxsize=L)
    sel = np.random.default_rng(5).choice(N, N // 50, replace=False)
    inr = (tree.count_neighbors(cKDTree(xw[sel], boxsize=L), prm["rc"]) - len(sel)) * (N / len(sel))
    b = 8 if prm["fft_f64"] else 4
    ncplx = M * M * (M // 2 + 1)
    fft_bytes = 3 * M ** 3 * b + 3 * ncplx * 2 * b
    scale_bytes = 2 * 3 * ncplx * 2 * b
    hbm = peaks["hbm_gbs"]
    roof = {}
    for k, by in (("fft", fft_bytes), ("ifft", fft_bytes), ("scale", scale_bytes)):
        gbs = by / (st[k + "_ms"] * 1e-3) / 1e9
        roof[k] = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                   "bytes_per_launch": by}
    if M in (64, 128, 256):
        # FP32 spectra: 2-D (y, x) transforms of the 3 M planes around one
        # kernel for the z transforms and the CNV; FP64 spectra: 1-D
        # transforms along x, the y and z transforms in double-single kernels
        if prm["fft_f64"]:
            roof["fft"]["kernel"] = "cuFFT 1-D D2Z along x, then k_fft_y64 (double-single y FFT)"
            roof["scale"]["kernel"] = "k_fgc_z64 (double-single): z FFT, CNV (eq. (sca)) and z IFFT"
            roof["ifft"]["kernel"] = "k_fft_y64 inverse (double-single), then cuFFT 1-D Z2D along x"
        else:
            roof["fft"]["kernel"] = "cuFFT 2-D R2C of the 3 M (y, x) planes"
            roof["scale"]["kernel"] = "k_fgc_z: z FFT, CNV (eq. (sca)) and z IFFT, spectrum read and written once"
            roof["ifft"]["kernel"] = "cuFFT 2-D C2R of the 3 M (y, x) planes"
    near = ("double-single" if prm["near_ds"] else ("FP64" if prm["near_f64"] else "FP32"))
    roof["p2p"] = {"inrange_pairs_est": inr, "pairs_per_s": inr / (st["p2p_ms"] * 1e-3),
                   "arithmetic": near + " pairs"}
    for k in ("p2g", "g2p"):
        roof[k] = {"points_per_s": N / (st[k + "_ms"] * 1e-3), "P": c["P"]}
    return {"workload": CLUSTERED, "N": N, "tol": c["tol"], "M": M, "P": c["P"],
            "xi": prm["xi"], "rc": prm["rc"], "n_c": prm["n_c"], "near": near,
            "fft": "FP64" if prm["fft_f64"] else "FP32", "value": c["value"], "unit": UNIT,
            "ms_per_step": c["ms"], "steps": c["steps"],
            "fp64_plain": {"value": c["value64"], "unit": UNIT, "ms_per_step": c["ms64"]},
            "stages_ms": {k: round(v, 5) for k, v in st.items()}, "stage_roofline": roof,
            "l2": "inputs and workspaces larger than L2; 256 MB buffer rewritten between timed steps"}


def run_batch(args, rank):
    """Many boxes (N = 10^U(3, 5), tol in {1e-4, 1e-6, 1e-8}, uniform points),
    autotuned per box, applied as one captured graph per batch step."""
    import torch

    from paper_2606_19059_gb300 import ewald, workloads

    seed = 1004 + rank
    N, tol = workloads.batch_boxes(args.batch_boxes, seed=seed)
    t0 = time.perf_counter()
    ewald.ewald_autotune_clear()
    b = ewald.Batch(N, 1.0, tol, ewald.EWALD_F32_BULK, tune=ewald.EWALD_TUNE_MEASURE, nstreams=16)
    t_create = time.perf_counter() - t0
    for i, n in enumerate(N):
        x, f = workloads.batch_box(seed, i, int(n))
        bx, bf, _ = b.buffers(i)
        bx.copy_(torch.as_tensor(x, device=bx.device))
        bf.copy_(torch.as_tensor(f, device=bf.device))
    stream = torch.cuda.current_stream()
    for _ in range(3):
        b.apply(stream)
    torch.cuda.synchronize()
    steps = max(3, min(args.steps, 5))
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, e in evs:
        a.record(stream)
        b.apply(stream)
        e.record(stream)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(e) for a, e in evs]
    tuned = {(int(b.params(i).M), int(b.params(i).tile)) for i in range(len(N))}
    kern = b.launch_counts()[0]
    b.close()
    ms_med = float(np.median(ms))
    per_tol = [_batch_class(seed, N, tol, t, stream) for t in sorted(set(tol.tolist()), reverse=True)]
    return {"boxes": int(len(N)), "particles": int(N.sum()), "ms_per_step": ms_med,
            "value": float(N.sum()) / (ms_med * 1e-3), "unit": UNIT,
            "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
            "steps": steps, "tune_and_plan_s": t_create, "distinct_tuned_grids": len(tuned),
            "kernels_per_step": int(kern), "graph_launches_per_step": 1, "per_tol": per_tol,
            "workload": "512 boxes, N = round(10^U(3,5)), tol uniform in {1e-4, 1e-6, 1e-8}, uniform points, "
                        "FP32 bulk, autotuned (measured) per half-octave of N; inputs larger than L2"}


def _batch_class(seed, N, tol, t, stream):
    """The boxes of one tolerance class of the batch: as a batch of their own
    (one graph launch a step) and as one plan per box applied one after the
    other on the same stream (the single-apply form), with the same tuned
    parameters (the autotuner's cache from the full batch)."""
    import torch

    from paper_2606_19059_gb300 import ewald, workloads

    idx = np.flatnonzero(tol == t)
    sb = ewald.Batch(N[idx], 1.0, tol[idx], ewald.EWALD_F32_BULK, tune=ewald.EWALD_TUNE_MEASURE)
    for j, i in enumerate(idx):
        x, f = workloads.batch_box(seed, int(i), int(N[i]))
        bx, bf, _ = sb.buffers(j)
        bx.copy_(torch.as_tensor(x, device=bx.device))
        bf.copy_(torch.as_tensor(f, device=bf.device))

    def timed(run, reps=3):
        for _ in range(3):
            run()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for a, e in evs:
            a.record(stream)
            run()
            e.record(stream)
        torch.cuda.synchronize()
        return float(np.median([a.elapsed_time(e) for a, e in evs]))

    bms = timed(lambda: sb.apply(stream))
    plans, io = [], []
    for j in range(len(idx)):
        q = sb.params(j)
        plans.append(ewald.Plan(int(N[idx[j]]), 1.0, t, ewald.EWALD_F32_BULK, M=q.M, P=q.P, tile=q.tile))
        bx, bf, _ = sb.buffers(j)
        io.append((bx, bf, torch.empty_like(bx)))

    def singles():
        for p, (bx, bf, u) in zip(plans, io):
            p.apply(bx, bf, out=u, stream=stream)

    sms = timed(singles)
    for p in plans:
        p.close()
    sb.close()
    n = float(N[idx].sum())
    return {"tol": t, "boxes": int(len(idx)), "particles": int(n), "batched_ms": bms,
            "batched_value": n / (bms * 1e-3), "single_apply_ms": sms, "single_apply_value": n / (sms * 1e-3),
            "unit": UNIT}


def run_serving(args, rank, rate_hz):
    """Poisson arrivals of mobility requests (N = 10^U(3, log10 4e6), uniform or
    clustered 50/50, tol in {1e-4, 1e-6, 1e-8}), 20 applies each with perturbed
    forces, through the continuous-batching server; host arrays in and out."""
    from paper_2606_19059_gb300 import ewald, workloads

    stream = workloads.serving_stream(args.serve_requests, seed=1005 + rank, rate_hz=rate_hz)
    data = [workloads.served_box(r["kind"], r["N"], r["seed"]) for r in stream]
    srv = ewald.Server(200 << 30, max_active=8)
    t0 = time.perf_counter()
    tickets = []
    for r, (x, f) in zip(stream, data):
        dt = r["t"] - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        tickets.append(srv.submit(x, f, r["tol"], napplies=20, perturb=0.1, seed=r["seed"]))
    for t in tickets:
        srv.result(t)
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    return {"requests": len(stream), "rate_hz": rate_hz, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
            "mean_ms": st["mean_ms"], "value": st["throughput"], "unit": UNIT, "completed": st["completed"],
            "failed": st["failed"], "wall_s": wall, "peak_footprint_gb": st["peak_footprint_bytes"] / 1e9,
            "particle_applies": st["particle_applies"],
            "workload": "Poisson arrivals; N = round(10^U(3, log10 4e6)); uniform or clustered (blobs = N/1e4) "
                        "50/50; tol uniform in {1e-4, 1e-6, 1e-8}; FP32 bulk; 20 applies per request with "
                        "f += 0.1 N(0,1) re-centred (Philox4x32-10); latency from submit to the last "
                        "apply's u on the host; HBM budget 200 GB, 8 slots"}


# One oracle sample, the same for the CPU-baseline leg and every step of the
# reference arm: the direct Ewald sum at this many sampled targets (the
# structure factors over all N sources cost the same whatever the count, so
# a fixed count keeps the two rates comparable).
ORACLE_TARGETS = 1024


def oracle_sample(seed_shift: int, x=None, f=None):
    """One timed oracle sample (direct Ewald, FP64, all host cores) of the
    workload: ORACLE_TARGETS targets drawn with seed 99 + seed_shift."""
    import oracle
    from paper_2606_19059_gb300 import workloads

    kind, N, L, tol, M, P, seed = workloads.WORKLOADS[WORKLOAD]
    if x is None:
        x, f = workloads.make(kind, N, seed, L)
    idx = np.random.default_rng(99 + seed_shift).choice(N, ORACLE_TARGETS, replace=False)
    oracle.build()
    t = time.perf_counter()
    oracle.ewald(x, f, L, targets=idx)
    return time.perf_counter() - t, oracle.num_threads(), N


def cpu_baseline(samples: int):
    """The oracle, as it stands, on a bounded sample of the same workload:
    `samples` oracle samples of ORACLE_TARGETS targets each."""
    from paper_2606_19059_gb300 import workloads

    kind, N, L, tol, M, P, seed = workloads.WORKLOADS[WORKLOAD]
    x, f = workloads.make(kind, N, seed, L)
    dt, cores = 0.0, 0
    for k in range(samples):
        t, cores, _ = oracle_sample(k, x, f)
        dt += t
    return {"value": samples * ORACLE_TARGETS / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"direct Ewald (FP64), {samples} samples of {ORACLE_TARGETS} sampled targets of the "
                      f"N={N} workload, structure factors over all {N} sources", "seconds": dt}


def job_time_and_rate(ms_local: float, units_per_rank: int, world: int):
    """Max over ranks of the per-step time (an all-reduce over the gloo group
    when world > 1) and the whole-job rate: the units all ranks processed per
    second at that time."""
    ms = float(ms_local)
    if world > 1:
        import torch
        import torch.distributed as dist

        t = torch.tensor([ms], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * units_per_rank / (ms * 1e-3)


def main_reference(args, rank, world):
    if rank != 0:
        return
    from paper_2606_19059_gb300 import workloads

    kind, N, L, tol, M, P, seed = workloads.WORKLOADS[WORKLOAD]
    per = ORACLE_TARGETS
    x, f = workloads.make(kind, N, seed, L)
    for w in range(args.warmup):
        oracle_sample(1000 + w, x, f)
    times = []
    for k in range(args.steps):
        t, cores, _ = oracle_sample(k, x, f)
        times.append(t)
    total = sum(times)
    value = per * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "ranks_timed": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N, "tol": tol, "M": M, "P": P,
                   "step": f"oracle direct Ewald at {per} sampled targets"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{per} sampled targets per step of the N={N} workload (rank 0 alone)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-samples", type=int, default=4,
                    help="oracle samples of %d targets in the CPU-baseline leg" % ORACLE_TARGETS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the many-box batched run")
    ap.add_argument("--batch-boxes", type=int, default=512)
    ap.add_argument("--no-serve", action="store_true", help="skip the serving run")
    ap.add_argument("--no-double-layer", action="store_true",
                    help="skip the combined single + double layer measurement")
    ap.add_argument("--no-clustered", action="store_true",
                    help="skip the clustered N = 2e6, tol 1e-7 workload")
    ap.add_argument("--serve-requests", type=int, default=24)
    ap.add_argument("--serve-rates", default="2,8",
                    help="Poisson arrival rates (requests/s), comma-separated: the first is the reported "
                         "serving run, the list the sweep toward saturation")
    ap.add_argument("--only-split", action="store_true",
                    help="time FP32-bulk applies at tol 1e-8 on the same points (the split double-single "
                         "near field) and print a short line (for ncu captures)")
    ap.add_argument("--only-batch", action="store_true",
                    help="run the batched many-box workload alone and print a short line (for ncu captures)")
    ap.add_argument("--only-f32", action="store_true",
                    help="time the FP32-bulk applies only and print a short line (for ncu captures)")
    ap.add_argument("--only-double-layer", action="store_true",
                    help="time the combined single + double layer applies only (for ncu captures)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    try:
        if args.impl == "reference":
            main_reference(args, rank, world)
            return
        if args.only_batch:  # profiling runs: the batched boxes alone
            r = run_batch(args, rank)
            if rank == 0:
                print(json.dumps({"only_batch": True, "ms_per_step": r["ms_per_step"],
                                  "kernels_per_step": r["kernels_per_step"], "per_tol": r["per_tol"]}))
            return
        res = run_gpu(args, rank, world)
        if res is None:
            return
        ms_mean, value = job_time_and_rate(float(np.mean(res["ms32"])), res["N"], world)
        N, L, tol, M, P = res["N"], res["L"], res["tol"], res["M"], res["P"]
        ms64, rate64 = job_time_and_rate(float(np.mean(res["ms64"])), N, world)
        e2e_ms, e2e_rate = job_time_and_rate(1e3 * float(np.median(res["e2e_s"])), N, world)
        dl_ms = dl_rate = None
        if res["dl"] is not None:
            dl_ms, dl_rate = job_time_and_rate(float(np.median(res["dl"]["ms"])), N, world)
        clus = None
        if not args.no_clustered:
            clus = run_clustered(args, rank, world)
        if rank != 0:
            return
        peaks, peak_src = load_peaks()
        st = res["stages"]
        prm = res["params"]
        inr, cand = pair_counts(res["x"], L, prm["rc"], prm["n_c"])
        sm_mhz = peaks.get("sm_max_mhz", 2070.0)
        fp32_peak = N_SM * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12  # TFLOP/s
        p2p_flops = FP32_FLOPS_PER_INRANGE * inr + FLOPS_PER_CANDIDATE * cand
        p2p_tf = p2p_flops / (st["p2p_ms"] * 1e-3) / 1e12
        # HBM-bound stages: algorithmic bytes per launch
        b = 4  # FP32 FFT at tol 1e-6
        ncplx = M * M * (M // 2 + 1)
        scale_bytes = 2 * 3 * ncplx * 2 * b
        fft_bytes = 3 * M ** 3 * b + 3 * ncplx * 2 * b
        hbm = peaks["hbm_gbs"]
        stage_roof = {
            "p2p": {"bound": "alu", "achieved": p2p_tf, "peak": fp32_peak, "unit": "TFLOP/s",
                    "frac": p2p_tf / fp32_peak},
            "scale": {"bound": "hbm", "achieved": scale_bytes / (st["scale_ms"] * 1e-3) / 1e9,
                      "peak": hbm, "unit": "GB/s"},
            "fft": {"bound": "hbm", "achieved": fft_bytes / (st["fft_ms"] * 1e-3) / 1e9, "peak": hbm,
                    "unit": "GB/s"},
            "ifft": {"bound": "hbm", "achieved": fft_bytes / (st["ifft_ms"] * 1e-3) / 1e9, "peak": hbm,
                     "unit": "GB/s"},
        }
        for k in ("scale", "fft", "ifft"):
            stage_roof[k]["frac"] = stage_roof[k]["achieved"] / hbm
        if not prm["fft_f64"] and M in (64, 128, 256):
            # FP32 spectra at these M: 2-D (y, x) transforms of the 3 M planes
            # around one kernel for the z transforms and the CNV
            stage_roof["fft"]["kernel"] = "cuFFT 2-D R2C of the 3 M (y, x) planes"
            stage_roof["scale"]["kernel"] = "k_fgc_z: z FFT, CNV (eq. (sca)) and z IFFT, spectrum read and written once"
            stage_roof["ifft"]["kernel"] = "cuFFT 2-D C2R of the 3 M (y, x) planes"
        else:
            stage_roof["fft"]["kernel"] = "cuFFT 3-D R2C"
            stage_roof["scale"]["kernel"] = "k_scale: CNV (eq. (sca))"
            stage_roof["ifft"]["kernel"] = "cuFFT 3-D C2R"
        # P2G / G2P: intensity far above the HBM ridge, so the binding fraction
        # is the FP32 pipe; the algorithmic HBM rate is reported beside it.
        # P2G per source: 3 P nu Horner FMAs, P^2 + P^3 weight products,
        # 3 P^3 force FMAs; bytes 24 N (FP32 x, f) + 12 M^3 (grid write).
        # G2P per target: P^2 + P^3 products and 3 P^3 FMAs; bytes 12 N + 12 N
        # + 12 M^3.
        nu = prm["poly_deg"]
        p2g_flops = N * (6 * P * nu + P * P + 7 * P ** 3)
        g2p_flops = N * (6 * P * nu + P * P + 7 * P ** 3)
        for k, fl, by in (("p2g", p2g_flops, 24 * N + 12 * M ** 3), ("g2p", g2p_flops, 24 * N + 12 * M ** 3)):
            t = st[k + "_ms"] * 1e-3
            stage_roof[k] = {"bound": "alu", "achieved": fl / t / 1e12, "peak": fp32_peak, "unit": "TFLOP/s",
                             "frac": fl / t / 1e12 / fp32_peak, "hbm_gbs": by / t / 1e9,
                             "hbm_frac": by / t / 1e9 / hbm, "flops_per_launch": fl, "bytes_per_launch": by}
        # dominant kernel: the longest stage
        order = sorted(((st[k + "_ms"], k) for k in ("p2p", "p2g", "fft", "scale", "ifft", "g2p", "bin")),
                       reverse=True)
        roof = dict(stage_roof["p2p"])
        roof["traffic"] = kernel_traffic("k_p2p.cu")
        roof["kernel"] = "k_p2p<float> (P2P near field)"
        roof["peak_source"] = (f"FP32 pipe: {N_SM} SMs x {FP32_LANES} lanes x 2 flop x {sm_mhz:.0f} MHz "
                               f"({peak_src} sm_max_mhz)")
        try:  # measured FMA-pipe peaks, beside the derived one
            from paper_2606_19059_gb300 import ewald

            p32, p64 = ewald.ewald_probe_fma_peaks(0)
            roof["peak_probe"] = {"fp32_tflops": p32, "fp64_tflops": p64,
                                  "frac_of_fp32_probe": p2p_tf / p32,
                                  "method": "8 independent FMA chains per thread, 4 x 256 threads per SM, "
                                            "best of 3 timed launches (ewald_probe_fma_peaks)"}
        except Exception as exc:  # pragma: no cover - reported, not fatal
            roof["peak_probe"] = {"error": str(exc)}
        roof["algorithmic"] = {"inrange_pairs": inr, "candidate_pairs": cand,
                               "candidate_basis": "every target's 27 neighbour cells (the paper's P2P flop model, "
                                                  "Sec. 4); the kernel's sub-cell culling tests about 86 % of them, "
                                                  "which would give about 0.92 of this fraction",
                               "flops_per_inrange": FP32_FLOPS_PER_INRANGE,
                               "flops_per_candidate": FLOPS_PER_CANDIDATE, "flops_per_launch": p2p_flops}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_mean, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": N, "L": L, "tol": tol, "M": M, "P": P,
                       "mode": "f32_bulk", "xi": prm["xi"], "rc": prm["rc"], "n_c": prm["n_c"],
                       "poly_deg": prm["poly_deg"], "l2": "256 MB buffer rewritten between timed steps",
                       "parallelism": f"replicas x{world}"},
            "fp64_plain": {"value": rate64, "unit": UNIT, "ms_per_step": ms64},
            "p50_ms": float(np.percentile(res["ms32"], 50)), "p99_ms": float(np.percentile(res["ms32"], 99)),
            "wall_s_timed": res["wall32"],
            "stages_ms": {k: round(v, 5) for k, v in st.items()},
            "stage_roofline": stage_roof,
            "dominant_stage": order[0][1],
            "roofline": roof,
            "e2e": {"value": e2e_rate, "unit": UNIT, "ms_per_step": e2e_ms,
                    "h2d_bytes_per_step": 2 * N * 3 * 8, "d2h_bytes_per_step": N * 3 * 8},
            "gpu_launches": res["kernels_per_step"] * args.steps,
            "clocks": res["clocks"],
        }
        if res["dl"] is not None:
            sd = res["dl"]["stages"]
            line["double_layer"] = {
                "what": "combined single + double layer apply (Sec. 2.3), same points, q and n ~ N(0, 1)",
                "value": dl_rate, "unit": UNIT, "ms_per_step": dl_ms,
                "stages_ms": {k: round(v, 5) for k, v in sd.items()},
                # the FP32 double-layer pairs run after the Stokeslet P2P (in
                # its stage), the FP64 ones after the sum (in that stage)
                "near_dl_ms": round(sd["p2p_ms"] - st["p2p_ms"] + sd["sum_ms"] - st["sum_ms"], 5),
                "near_dl_kernel": ("k_p2p_dl<double> (FP64 pairs, one warp per 32 targets, queued in-range "
                                   "pairs)" if prm["fft_f64"] or prm["near_f64"]
                                   else "k_p2p_dl32 (FP32 pairs on the Stokeslet P2P machinery: sub-cell "
                                        "culling, FP16x2 phase 1, bit queue, two pairs per iteration)"),
            }
        if clus is not None:
            line["clustered"] = clustered_entry(clus, peaks)
        if not args.no_batch:
            line["batched"] = run_batch(args, rank)
        if not args.no_serve:
            rates = [float(r) for r in args.serve_rates.split(",") if r]
            runs = [run_serving(args, rank, r) for r in rates]
            line["serving"] = dict(runs[0])
            line["serving"]["sweep"] = [{k: r[k] for k in ("rate_hz", "p50_ms", "p99_ms", "value", "wall_s",
                                                         "completed")} for r in runs]
        if not args.no_cpu_baseline:
            cb = cpu_baseline(args.cpu_samples)
            cb.pop("seconds", None)
            line["cpu_baseline"] = cb
        print(json.dumps(line))
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
