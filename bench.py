"""Benchmark: time to the lowest nev BSE eigenpairs on one GB300.

Workload (one "step" = the whole hot path over one input): the
pseudo-Hermitian problem of N = 10000 (H of order 20000), complex128,
lowest 100 positive eigenpairs with the FP64 structure-preserving Lanczos:
ingest (packing of A and B already resident in HBM) + solve (folded
products, CGS2, projected eigenproblem, restart/lock, recovery, FP64
residuals).  The adjoint and the block-product bandwidth are timed as
separate lines of the same JSON object.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs independent replicas (one per GPU; the method has no exchange
step on one problem), launched by torch.distributed.run.
"""
from __future__ import annotations

import argparse
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

METRIC = "time-to-nev BSE eigenpairs (s) & block-product HBM GB/s; mixed vs FP64 at 1e-6"
NEV = 100
TOL = 1e-12
SAMPLE_N = 1500          # CPU-baseline sample: dense oracle on the same recipe at this N


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples during the timed region (clocks and throttle reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
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
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _reduce_max(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------ CPU baseline (oracle)
def cpu_baseline_sample(n_sample=SAMPLE_N):
    """Dense FP64 oracle (zgeev of the full 2N matrix) on the same recipe at a
    smaller N, extrapolated to N = 10000 by the O(N^3) cost of dense eig."""
    import oracle as O
    from synthetic import BSEProblemSpec, CONFIGS, make_problem
    spec = CONFIGS[1]
    s = BSEProblemSpec(n=n_sample, n_g=spec.n_g, seed=spec.seed, form="ph", dtype="c128")
    p = make_problem(s)
    t = time.perf_counter()
    O.ph_lowest(p["A"], p["B"], NEV)
    dt = time.perf_counter() - t
    scaled = dt * (spec.n / n_sample) ** 3
    return scaled, dt


def _cores():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        if info:
            return int(max(i.get("num_threads", 1) for i in info))
    except Exception:
        pass
    return os.cpu_count() or 1


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    vals = []
    for i in range(args.warmup + args.steps):
        v, raw = cpu_baseline_sample()
        if i >= args.warmup:
            vals.append(v)
    value = statistics.mean(vals)
    sample = (f"oracle.ph_lowest (dense zgeev of H, order {2 * SAMPLE_N}) on the config-1 recipe at "
              f"N={SAMPLE_N}, scaled by (10000/{SAMPLE_N})^3")
    line = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": _config(), "cpu_baseline": {"value": value, "unit": "s", "cores": _cores(),
                                                  "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _config():
    return {"workload": "pseudo-Hermitian BSE, N=10000 (H 20000x20000), complex128, lowest 100 positive "
                        "eigenpairs, FP64 structure-preserving thick-restart Lanczos, tol 1e-12",
            "N": 10000, "nev": NEV, "tol": TOL, "storage": "complex128", "seed": 1,
            "l2": "inputs larger than L2 (packed A+B 1.6 GB)", "parallelism": "replicas"}


# ------------------------------------------------------------------ GPU arm
def run_gpu(args):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2504_10096_gb300 import bse
    from synthetic import CONFIGS, make_problem_torch
    spec = CONFIGS[1]
    dev = torch.device("cuda", torch.cuda.current_device())
    prob = make_problem_torch(spec, device=dev)
    A, B = prob["A"], prob["B"]
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    lib = bse.load_library()
    N = spec.n

    def one_step():
        s = bse.Solver(A, B, stream=stream)
        vals, vecs, nconv = s.solve(NEV, tol=TOL)
        st = s.stats()
        s.close()
        return vals, st

    for _ in range(args.warmup):
        vals, st = one_step()
    torch.cuda.synchronize()
    _barrier(ws)
    launches0 = None
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    with ClockSampler(torch.cuda.current_device()) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            vals, st = one_step()
            stats.append(st)
        e1.record(stream)
        torch.cuda.synchronize()
    _barrier(ws)
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = _reduce_max(ms, ws)
    prod_ms = sum(s["ms_product"] for s in stats) / args.steps
    passes = stats[-1]["passes"]
    n_tiles = (spec.n + 127) // 128
    launches = int(sum(s["launches"] for s in stats) / args.steps) + 2 * n_tiles  # + packing of A and B
    # ---- block-product roofline (the dominant kernel): FP64 complex products
    per_launch_flops = 16.0 * N * N                       # A x + B conj(x): 8 flops per complex MAC
    per_launch_bytes = 2 * (N * (N + 1) / 2) * 16 + 3 * N * 16
    t_launch = prod_ms / passes * 1e-3
    peaks, peak_kind = _peaks()
    clocks = clk.summary()
    sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp64_peak = 152 * 2 * 2 * sm_mhz * 1e6 / 1e12        # TFLOP/s: 152 SMs x 2 FP64 FMA/clk x 2 flops
    achieved_tf = per_launch_flops / t_launch / 1e12
    achieved_gbs = per_launch_bytes / t_launch / 1e9
    # ---- adjoint (a10) and e2e through host buffers (rank-local)
    s = bse.Solver(A, B, stream=stream)
    s.solve(NEV, tol=TOL, vectors=False)
    g = np.ones(NEV)
    torch.cuda.synchronize()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    dA, dB = s.backward(g)
    a1.record(stream)
    torch.cuda.synchronize()
    adj_ms = a0.elapsed_time(a1)
    del dA, dB
    s.close()
    Ah = A.cpu().numpy()
    Bh = B.cpu().numpy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = max(1, min(2, args.steps))
    for _ in range(e2e_steps):
        s = bse.Solver(Ah, Bh, stream=stream)                # host buffers: H2D inside
        v2, vec2, _ = s.solve(NEV, tol=TOL)
        vec_host = vec2.cpu()                                # D2H of eigenvectors
        s.close()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_s = _reduce_max(e2e_s, ws)
    # ---- parity against the stored oracle values
    gold_path = os.path.join(ROOT, "tests", "golden", "config1_omega.txt")
    max_rel = None
    if os.path.exists(gold_path):
        gold = np.loadtxt(gold_path)
        max_rel = float(np.max(np.abs(vals - gold) / gold))
    if rank != 0:
        return
    cpu_v, cpu_raw = cpu_baseline_sample()
    value = ms_max / 1e3
    line = {
        "metric": METRIC, "value": value, "unit": "s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": _config(),
        "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": achieved_tf / fp64_peak, "traffic": None,
                     "kernel": "k_prod_tiles + k_prod_reduce (one folded product M+/M- over packed A and B)",
                     "peak_note": "FP64 FMA peak from 152 SMs x 2 FP64 FMA/clk/SM x 2 flops x median SM clock",
                     "achieved_hbm_gbs": achieved_gbs, "hbm_peak_gbs": peaks.get("hbm_gbs"),
                     "hbm_frac": achieved_gbs / peaks.get("hbm_gbs", 6800.0), "hbm_peak_kind": peak_kind},
        "cpu_baseline": {"value": cpu_v, "unit": "s", "cores": _cores(), "kind": "oracle",
                         "sample": f"oracle.ph_lowest (dense zgeev, order {2 * SAMPLE_N}) at N={SAMPLE_N} on the "
                                   f"same recipe, {cpu_raw:.1f} s, scaled by (10000/{SAMPLE_N})^3"},
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(Ah.nbytes + Bh.nbytes),
                "d2h_bytes_per_step": int(vec_host.numel() * 16 + NEV * 8)},
        "gpu_launches": launches,
        "clocks": clocks,
        "solver": {"krylov_steps": stats[-1]["steps"], "passes": passes, "restarts": stats[-1]["restarts"],
                   "max_residual": stats[-1]["max_residual"], "max_rel_err_vs_oracle": max_rel,
                   "product_ms_per_solve": prod_ms, "product_share": prod_ms / ms},
        "adjoint_ms": adj_ms,
    }
    print(json.dumps(line), flush=True)


def run_product(args):
    """The structured product alone (bse_apply, one vector): the streaming
    tile kernel of the Lanczos steps, timed with CUDA events on its stream."""
    import torch
    from paper_2504_10096_gb300 import bse
    from synthetic import BSEProblemSpec, make_problem
    torch.cuda.set_device(0)
    N = args.n
    spec = BSEProblemSpec(n=N, n_g=400, seed=1, form="ph", dtype=args.dtype)
    prob = make_problem(spec)          # host generation: no torch.linalg on the device
    stream = torch.cuda.current_stream()
    s = bse.Solver(torch.from_numpy(prob["A"]).cuda(), torch.from_numpy(prob["B"]).cuda(), stream=stream)
    del prob
    cdt = torch.complex128 if args.dtype == "c128" else torch.complex64
    x = torch.randn(N, dtype=cdt, device="cuda")
    for _ in range(args.warmup):
        s.apply(bse.BSE_OP_MPLUS, x)
    times = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.apply(bse.BSE_OP_MPLUS, x)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = statistics.median(times)
    es = 16 if args.dtype == "c128" else 8
    byts = 2 * (N * (N + 1) / 2) * es + 3 * N * es
    flops = 16.0 * N * N
    peaks, kind = _peaks()
    print(json.dumps({"mode": "product", "N": N, "dtype": args.dtype, "ms": ms, "GB/s": byts / ms / 1e6,
                      "TFLOP/s": flops / ms / 1e9, "hbm_frac": byts / ms / 1e6 / peaks["hbm_gbs"],
                      "hbm_peak_kind": kind}), flush=True)
    s.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--mode", default="solve", choices=["solve", "product"])
    ap.add_argument("--n", type=int, default=8000)
    ap.add_argument("--dtype", default="c128", choices=["c128", "c64"])
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "product":
        run_product(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
