"""Benchmark: time to the lowest nev BSE eigenpairs on one GB300.

Headline workload (one "step" = the whole hot path over one input): the
pseudo-Hermitian problem of N = 10000 (H of order 20000), complex128,
lowest 100 positive eigenpairs with the FP64 structure-preserving Lanczos:
ingest (packing of A and B already resident in HBM) + solve (folded
products, CGS2, projected eigenproblem, restart/lock, recovery, FP64
residuals).  The same JSON line carries, measured in the same run:
  * "config4": the metric's own configuration -- PH N = 50000, complex64 A
    and B, lowest 200, residual <= 1e-6 -- solved once on the mixed path, with
    the mixed product's bandwidth; --config4-fp64 adds the plain FP64 solve of
    the same values and the speed-up (about eleven more minutes, so it is not
    in the default run); --skip-config4 leaves the record out;
  * the block-product roofline against the FP64 FMA peak measured in the run,
    the adjoint, the e2e solve through host buffers, and the double-FP32
    variant of the headline solve.

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
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
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


def _config(ncv=0):
    return {"workload": "pseudo-Hermitian BSE, N=10000 (H 20000x20000), complex128, lowest 100 positive "
                        "eigenpairs, FP64 structure-preserving thick-restart Lanczos, tol 1e-12",
            "N": 10000, "nev": NEV, "tol": TOL, "storage": "complex128", "seed": 1,
            "ncv": ncv or max(2 * NEV, NEV + 32),
            "l2": "inputs larger than L2 (packed A+B 1.6 GB)", "parallelism": "replicas"}


# ------------------------------------------------------------------ GPU arm
# dram__bytes_read.sum + dram__bytes_write.sum of one k_prod_tiles(+_df) launch at N = 8000
# (profiles/k_prod_tiles_*_n8000.md); None until the current kernel has been captured
TRAFFIC_N8000 = {"fp64": 1.057860e9 + 10.361088e6, "df": 1.067138e9 + 22.040064e6}


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

    ingest_ms = []

    def one_step():
        i0, i1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        i0.record(stream)
        s = bse.Solver(A, B, stream=stream, df=args.df)     # ingest: pack A and B into tiles
        i1.record(stream)
        vals, vecs, nconv = s.solve(NEV, tol=TOL, ncv=args.ncv)
        st = s.stats()
        s.close()
        ingest_ms.append(i0.elapsed_time(i1))
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
    # M_s as a real-linear map on R^2N is a dense 2N x 2N real matrix: 4N^2 FMAs = 8N^2 flops
    # (forming A x and B conj(x) as two complex products would be 16N^2)
    per_launch_flops = 8.0 * N * N
    per_launch_bytes = 2 * (N * (N + 1) / 2) * 16 + 3 * N * 16
    t_launch = prod_ms / passes * 1e-3
    peaks, peak_kind = _peaks()
    ingest_bytes = 2 * N * N * 16 + 2 * (N * (N + 1) / 2) * 16
    clocks = clk.summary()
    # FP64 FMA peak measured on this GPU (libbse's dependent-free FMA kernel, CUDA events),
    # sampled clocks beside it
    with ClockSampler(torch.cuda.current_device()) as clk64:
        fp64_peak, fp64_ms = bse.bse_measure_fp64_peak(1 << 18)
    clocks64 = clk64.summary()
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
    Ah = A.cpu().pin_memory().numpy()                        # pinned host buffers (DMA copies)
    Bh = B.cpu().pin_memory().numpy()
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
    gold = None
    if os.path.exists(gold_path):
        gold = np.loadtxt(gold_path)
        max_rel = float(np.max(np.abs(vals - gold) / gold))
    # ---- the same solve with the Lanczos products in double-FP32 (BSE_C128_DF)
    variant = None
    if not args.df:
        s = bse.Solver(A, B, stream=stream, df=True)
        vdf, _, _, t_df = _timed_solve(s, NEV, TOL, stream, vectors=False)
        sd = s.stats()
        s.close()
        variant = {"dtype": "f64 storage/basis, products in double-FP32 (error-free transformations)",
                   "s_per_solve": t_df, "krylov_steps": sd["steps"], "max_residual": sd["max_residual"],
                   "product_GBs": per_launch_bytes / (sd["ms_product"] / sd["passes"] * 1e-3) / 1e9,
                   "max_rel_err_vs_oracle": float(np.max(np.abs(vdf - gold) / gold)) if gold is not None else None}
    # ---- the metric's own configuration: config 4, mixed vs plain FP64 at residual <= 1e-6
    c4 = config4_record(args, stream) if not args.skip_config4 else None
    if rank != 0:
        return
    cpu_v, cpu_raw = cpu_baseline_sample()
    value = ms_max / 1e3
    # DRAM traffic per launch from the ncu captures at N = 8000 (profiles/k_prod_tiles_c128_n8000.md,
    # profiles/k_prod_tiles_df_n8000.md): bytes per stored 128x128 tile pair, scaled by the tile
    # count of this workload (traffic grows with the number of tiles streamed)
    n_tiles_8000 = 63 * 64 // 2
    captured = TRAFFIC_N8000.get("df" if args.df else "fp64")
    traffic = None if captured is None else captured / (2 * n_tiles_8000) * 2 * (n_tiles * (n_tiles + 1) // 2)
    if args.df:
        roof = {"bound": "hbm", "achieved": achieved_gbs, "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                "frac": achieved_gbs / peaks.get("hbm_gbs", 6800.0), "traffic": traffic,
                "kernel": "k_prod_tiles_df + k_prod_reduce (one folded product, double-FP32 arithmetic on "
                          "split complex128 tiles, 16 B per element)",
                "peak_kind": peak_kind, "achieved_fp64_equiv_tflops": achieved_tf}
    else:
        roof = {"bound": "alu", "achieved": achieved_tf, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved_tf / fp64_peak, "traffic": traffic,
                "algorithmic_bytes": per_launch_bytes,
                "kernel": "k_prod_tiles + k_prod_reduce (one folded product M+/M- over packed A and B)",
                "peak_note": "FP64 FMA peak measured in this run (bse_measure_fp64_peak: 8 independent FMA "
                             f"chains per thread on every SM, {fp64_ms:.1f} ms launch, CUDA events)",
                "peak_kind": "measured", "peak_clocks": clocks64,
                "achieved_hbm_gbs": achieved_gbs, "hbm_peak_gbs": peaks.get("hbm_gbs"),
                "hbm_frac": achieved_gbs / peaks.get("hbm_gbs", 6800.0), "hbm_peak_kind": peak_kind}
    line = {
        "metric": METRIC, "value": value, "unit": "s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64 (products in double-FP32)" if args.df else "f64",
        "data": "synthetic", "config": _config(args.ncv),
        "roofline": roof,
        "cpu_baseline": {"value": cpu_v, "unit": "s", "cores": _cores(), "kind": "oracle",
                         "sample": f"oracle.ph_lowest (dense zgeev, order {2 * SAMPLE_N}) at N={SAMPLE_N} on the "
                                   f"same recipe, {cpu_raw:.1f} s, scaled by (10000/{SAMPLE_N})^3"},
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(Ah.nbytes + Bh.nbytes),
                "d2h_bytes_per_step": int(vec_host.numel() * 16 + NEV * 8)},
        "gpu_launches": launches,
        "clocks": clocks,
        "solver": {"krylov_steps": stats[-1]["steps"], "passes": passes, "restarts": stats[-1]["restarts"],
                   "max_residual": stats[-1]["max_residual"], "max_rel_err_vs_oracle": max_rel,
                   "product_ms_per_solve": prod_ms, "product_share": prod_ms / ms,
                   "product_shape": {"ctas_per_sm": stats[-1]["shape_ctas_per_sm"],
                                     "strided": stats[-1]["shape_strided"], "tuned": stats[-1]["tuned"]},
                   "krylov_steps_as": "cuda graphs"},
        "adjoint_ms": adj_ms,
        # a1 ingest (bse_create): read the full row-major A and B (2 N^2 x 16 B) and write the packed
        # tiles of P = A + B and Q = A - B (2 x N(N+1)/2 x 16 B) in one launch; the interval also
        # holds the allocations and host set-up of the call
        "ingest": {"ms": statistics.median(ingest_ms), "algorithmic_bytes": ingest_bytes,
                   "GBs": ingest_bytes / statistics.median(ingest_ms) / 1e6,
                   "hbm_frac": ingest_bytes / statistics.median(ingest_ms) / 1e6 / peaks.get("hbm_gbs", 6800.0)},
        "variant_df_products": variant,
        "config4": c4,
    }
    print(json.dumps(line), flush=True)


def config4_record(args, stream):
    """Config 4 (PH, N = 50000, complex64 A and B, energies U[1, 12] eV, N_G = 2000,
    lowest 200, tol 1e-6): one solve on the mixed path (complex64 storage, FP64 basis,
    exact or grid-accumulated double-FP32 products) and one on the plain FP64 path
    (the same complex64 values promoted to complex128), each timed with CUDA events on
    the library's stream, with steps, passes, max FP64 residual, eigenvalue agreement,
    the speed-up and the mixed product's bandwidth."""
    import torch
    from paper_2504_10096_gb300 import bse
    from synthetic import CONFIGS, make_problem_torch
    spec = CONFIGS[4]
    N, nev, tol = spec.n, spec.nev, 1e-6
    p = make_problem_torch(spec, device="cuda")
    A, B = p["A"], p["B"]
    del p
    torch.cuda.synchronize()
    out = {"workload": f"config 4: PH N={N} (H {2 * N}), complex64 A and B, energies U[1,12] eV, N_G=2000, "
                       f"lowest {nev}, tol {tol:g}", "data": "synthetic (device generator)"}
    peaks, _ = _peaks()
    with ClockSampler(torch.cuda.current_device()) as clk:
        s = bse.Solver(A, B, stream=stream, mixed=True)
        vm, _, nm, tm = _timed_solve(s, nev, tol, stream, vectors=False)
        st = s.stats()
        s.close()
    pass_ms = st["ms_product"] / max(st["passes"], 1)
    pbytes = 2 * (N * (N + 1) / 2) * 8 + 3 * N * 16
    out["mixed"] = {"s": tm, "krylov_steps": st["steps"], "passes": st["passes"], "restarts": st["restarts"],
                    "nconv": int(nm), "max_residual": st["max_residual"], "tiles_fine": st["tiles_fine"],
                    "tiles_coarse": st["tiles_coarse"], "retried_exact": st["retried_exact"],
                    "product_ms_per_pass": pass_ms, "product_share": st["ms_product"] / (tm * 1e3),
                    "product_GBs": pbytes / pass_ms / 1e6,
                    "product_hbm_frac": pbytes / pass_ms / 1e6 / peaks.get("hbm_gbs", 6800.0),
                    "product_shape": {"ctas_per_sm": st["shape_ctas_per_sm"], "strided": st["shape_strided"]},
                    "clocks": clk.summary()}
    if args.config4_fp64:
        A64 = A.to(torch.complex128)
        del A
        B64 = B.to(torch.complex128)
        del B
        torch.cuda.synchronize()
        with ClockSampler(torch.cuda.current_device()) as clk:
            s = bse.Solver(A64, B64, stream=stream)
            del A64, B64
            v64, _, n64, t64 = _timed_solve(s, nev, tol, stream, vectors=False)
            st = s.stats()
            s.close()
        out["fp64"] = {"s": t64, "krylov_steps": st["steps"], "passes": st["passes"], "restarts": st["restarts"],
                       "nconv": int(n64), "max_residual": st["max_residual"],
                       "product_ms_per_pass": st["ms_product"] / max(st["passes"], 1), "clocks": clk.summary()}
        out["max_rel_eig_diff_mixed_vs_fp64"] = float(np.max(np.abs(vm - v64) / v64))
        out["speedup_mixed_over_fp64"] = t64 / tm
    else:
        del A, B
        out["fp64"] = None      # leg not run (--config4-fp64 adds it)
    torch.cuda.empty_cache()
    return out


def run_product(args):
    """The structured product alone (bse_apply, one vector): the streaming
    tile kernel of the Lanczos steps, timed with CUDA events on its stream."""
    import torch
    from paper_2504_10096_gb300 import bse
    from synthetic import BSEProblemSpec, make_problem
    torch.cuda.set_device(0)
    N = args.n or 8000
    spec = BSEProblemSpec(n=N, n_g=400, seed=1, form="ph", dtype=args.dtype)
    prob = make_problem(spec)          # host generation: no torch.linalg on the device
    stream = torch.cuda.current_stream()
    s = bse.Solver(torch.from_numpy(prob["A"]).cuda(), torch.from_numpy(prob["B"]).cuda(), stream=stream,
                   df=args.df, mixed=args.mixed)
    del prob
    cdt = torch.complex128 if (args.dtype == "c128" or args.mixed) else torch.complex64
    x = torch.randn(N, dtype=cdt, device="cuda")
    op = bse.BSE_OP_A if args.op == "a" else bse.BSE_OP_MPLUS
    if args.mixed:
        # the mixed path's own product (complex128 vectors): exact double-FP32 tiles and,
        # with --tau >= 0, coarse tiles on the fixed-point grid (bse_apply_mixed)
        y = torch.empty_like(x)

        def apply():
            rc = bse.bse_apply_mixed(s.h, op, args.tau, x.data_ptr(), y.data_ptr())
            if rc != bse.BSE_OK:
                raise bse.BSEError(rc, "bse_apply_mixed")
    else:
        def apply():
            s.apply(op, x)
    for _ in range(args.warmup):
        apply()
    times = []
    for _ in range(max(args.steps, 10)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        apply()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = statistics.median(times)
    es = 16 if args.dtype == "c128" else 8
    nmat = 1 if args.op == "a" else 2
    byts = nmat * (N * (N + 1) / 2) * es + 3 * N * es
    flops = 8.0 * N * N          # A x (complex) or M_s x (real 2N x 2N form): 4N^2 FMAs
    peaks, kind = _peaks()
    st = s.stats()
    print(json.dumps({"mode": "product", "op": args.op, "N": N, "dtype": args.dtype, "df": args.df,
                      "mixed": args.mixed, "tau": args.tau if args.mixed else None,
                      "tiles_fine": st["tiles_fine"] if args.mixed else None,
                      "tiles_coarse": st["tiles_coarse"] if args.mixed else None, "ms": ms, "GB/s": byts / ms / 1e6,
                      "TFLOP/s": flops / ms / 1e9, "hbm_frac": byts / ms / 1e6 / peaks["hbm_gbs"],
                      "hbm_peak_kind": kind}), flush=True)
    s.close()


def _timed_solve(solver, nev, tol, stream, vectors=True, graphs=True, persistent=True):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    vals, vecs, nconv = solver.solve(nev, tol=tol, vectors=vectors, graphs=graphs, persistent=persistent)
    e1.record(stream)
    torch.cuda.synchronize()
    return vals, vecs, nconv, e0.elapsed_time(e1) / 1e3


def run_workload(args):
    """Measurement lines for the other workloads (one JSON line each):
    tda   -- Tamm-Dancoff, N = 2000, complex128, lowest 20 (FP64)
    batch -- 64 pseudo-Hermitian problems, N_i ~ U{500..6000}, complex64, 16 each
    adjoint -- N = 20000, complex64, lowest 50, solve + Hellmann-Feynman backward
    mixed -- N = 50000, complex64 (mixed path) vs complex128 (FP64 path), lowest 200, tol 1e-6
    haydock -- N = 10000 pseudo-Hermitian, complex128, Lanczos-Haydock spectrum (600 steps)
    variants -- config 1 with each structure-preserving Lanczos variant (Shao, Gruning, projected BSE)"""
    import torch
    from paper_2504_10096_gb300 import bse
    from synthetic import CONFIGS, batched_specs, loss_draws, make_problem, make_problem_torch, random_start
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    out = {"mode": args.mode}
    if args.mode == "tda":
        spec = CONFIGS[0]
        p = make_problem(spec)
        A = torch.from_numpy(p["A"]).cuda()
        for _ in range(args.warmup):
            s = bse.Solver(A, stream=stream); s.solve(spec.nev, tol=1e-12); s.close()
        ts, ts_graphs, ts_stream = [], [], []
        for _ in range(max(args.steps, 5)):
            s = bse.Solver(A, stream=stream)          # persistent steps (one launch per cycle)
            vals, _, nconv, t = _timed_solve(s, spec.nev, 1e-12, stream)
            st = s.stats(); s.close(); ts.append(t)
            s = bse.Solver(A, stream=stream)          # the per-phase kernels replayed as CUDA graphs
            _, _, _, t = _timed_solve(s, spec.nev, 1e-12, stream, persistent=False)
            s.close(); ts_graphs.append(t)
            s = bse.Solver(A, stream=stream)          # the same solve with one launch per kernel
            _, _, _, t = _timed_solve(s, spec.nev, 1e-12, stream, graphs=False)
            s.close(); ts_stream.append(t)
        gold = np.loadtxt(os.path.join(ROOT, "tests", "golden", "config0_lambda.txt"))
        out.update({"workload": "TDA N=2000 complex128 nev=20 FP64", "s_per_solve": statistics.median(ts),
                    "s_per_solve_graphs": statistics.median(ts_graphs),
                    "s_per_solve_stream_launches": statistics.median(ts_stream),
                    "max_rel_err_vs_oracle": float(np.max(np.abs(vals - gold) / np.abs(gold))),
                    "krylov_steps": st["steps"], "max_residual": st["max_residual"], "launches": st["launches"],
                    "product_shape": {"ctas_per_sm": st["shape_ctas_per_sm"], "strided": st["shape_strided"],
                                      "tuned": st["tuned"]}})
    elif args.mode == "variants":
        # config 1 (PH N = 10^4 complex128, lowest 100, FP64, tol 1e-12) with each of the three
        # structure-preserving Lanczos variants on one handle (ingest outside the timed solves)
        spec = CONFIGS[1]
        p = make_problem_torch(spec, device="cuda")
        s = bse.Solver(p["A"], p["B"], stream=stream)
        del p
        gold_path = os.path.join(ROOT, "tests", "golden", "config1_omega.txt")
        gold = np.loadtxt(gold_path) if os.path.exists(gold_path) else None
        names = {"shao": bse.BSE_VARIANT_SHAO, "gruning": bse.BSE_VARIANT_GRUNING,
                 "projected": bse.BSE_VARIANT_PROJECTED}
        res = {}
        for name, v in names.items():
            ts = []
            for it in range(args.warmup + max(1, args.steps)):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize(); e0.record(stream)
                vals, _, nconv = s.solve(spec.nev, tol=1e-12, vectors=True, variant=v)
                e1.record(stream); torch.cuda.synchronize()
                if it >= args.warmup:
                    ts.append(e0.elapsed_time(e1) / 1e3)
            st = s.stats()
            res[name] = {"s_per_solve": statistics.median(ts), "nconv": int(nconv), "steps": st["steps"],
                         "passes": st["passes"], "restarts": st["restarts"], "launches": st["launches"],
                         "ms_product": st["ms_product"], "max_residual": st["max_residual"],
                         "max_rel_err_vs_oracle": (float(np.max(np.abs(vals - gold) / gold))
                                                   if gold is not None else None)}
        s.close()
        out.update({"workload": "config 1: PH N=10000 complex128, nev=100, tol 1e-12, FP64, per variant",
                    "variants": res})
    elif args.mode == "batch":
        specs = batched_specs()
        As, Bs = [], []
        for sp in specs:
            p = make_problem_torch(sp, device="cuda")
            As.append(p["A"]); Bs.append(p["B"])
        nev = specs[0].nev
        ts = []
        for it in range(args.warmup + args.steps):
            bs = bse.BatchedSolver(As, Bs, stream=stream, mixed=True)   # residual <= 1e-6 needs the mixed path
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(); e0.record(stream)
            vals, _, nconv = bs.solve(nev, tol=1e-6)
            e1.record(stream); torch.cuda.synchronize()
            st = bs.stats(); bs.close()
            if it >= args.warmup:
                ts.append(e0.elapsed_time(e1) / 1e3)
        gold_path = os.path.join(ROOT, "tests", "golden", "config2_omega.txt")
        err = None
        if os.path.exists(gold_path):
            gold = np.loadtxt(gold_path).reshape(len(specs), nev)
            err = float(np.max(np.abs(vals - gold) / gold))
        out.update({"workload": "64 PH problems, N_i in [500,6000], complex64 (mixed path), nev=16, tol 1e-6",
                    "s_per_batch": statistics.median(ts), "sizes_sum": int(sum(s.n for s in specs)),
                    "max_rel_err_vs_oracle": err, "krylov_steps_total": st["steps"],
                    "passes_total": st["passes"], "launches": st["launches"], "max_residual": st["max_residual"],
                    "product_shape": {"ctas_per_sm": st["shape_ctas_per_sm"], "strided": st["shape_strided"],
                                      "tuned": st["tuned"]}})
    elif args.mode == "backward":
        # the config-3 backward alone (complex64 solve, then one tensor-core and one CUDA-core
        # adjoint): the command the adjoint's ncu capture runs
        spec = CONFIGS[3]
        p = make_problem_torch(spec, device="cuda")
        n = args.n or spec.n                       # --n: a principal block (small ncu captures)
        s = bse.Solver(p["A"][:n, :n].contiguous(), p["B"][:n, :n].contiguous(), stream=stream, mixed=True)
        del p
        vals, _, _, t_solve = _timed_solve(s, spec.nev, 1e-6, stream, vectors=False)
        g = np.linspace(0.5, 1.5, spec.nev)
        res = {}
        for name, impl in (("tensor_cores", bse.BSE_IMPL_TENSOR_CORES), ("cuda_cores", bse.BSE_IMPL_CUDA_CORES)):
            s.backward(g, impl=impl)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.backward(g, impl=impl)
            e1.record(stream); torch.cuda.synchronize()
            res[f"backward_{name}_s"] = e0.elapsed_time(e1) / 1e3
        s.close()
        out.update({"workload": f"PH N={n} complex64 nev=50: backward (Hellmann-Feynman adjoint) only",
                    "solve_s": t_solve, **res,
                    "write_GBs_tensor_cores": 2 * n ** 2 * 8 / res["backward_tensor_cores_s"] / 1e9})
    elif args.mode == "adjoint":
        spec = CONFIGS[3]
        p = make_problem_torch(spec, device="cuda")
        A, B = p["A"], p["B"]
        nev = spec.nev
        s = bse.Solver(A, B, stream=stream, mixed=True)
        vals, _, _, t_solve = _timed_solve(s, nev, 1e-6, stream, vectors=False)
        # FP64 GPU reference on the same complex64 values (targets and gradient reference)
        s64 = bse.Solver(A.to(torch.complex128), B.to(torch.complex128), stream=stream)
        ref, _, _, t_ref = _timed_solve(s64, nev, 1e-12, stream, vectors=False)
        w, noise = loss_draws(nev)
        targets = ref + noise
        g = w + 2.0 * (vals - targets)
        def timed_bwd(impl):
            s.backward(g, impl=impl)                      # warm-up (allocations, tile lists)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = s.backward(g, impl=impl)
            e1.record(stream); torch.cuda.synchronize()
            return r, e0.elapsed_time(e1) / 1e3
        (dA, dB), t_bwd = timed_bwd(bse.BSE_IMPL_TENSOR_CORES)
        (dAs, dBs), t_simt = timed_bwd(bse.BSE_IMPL_CUDA_CORES)
        tc_vs_simt = float(torch.linalg.norm(dA - dAs) / torch.linalg.norm(dAs))
        del dAs, dBs
        dA64, dB64 = s64.backward(w + 2.0 * (ref - targets))
        ra = float(torch.linalg.norm((dA.to(torch.complex128) - dA64)) / torch.linalg.norm(dA64))
        rb = float(torch.linalg.norm((dB.to(torch.complex128) - dB64)) / torch.linalg.norm(dB64))
        out.update({"workload": "PH N=20000 complex64 (mixed path) nev=50, loss sum w*l + sum (l-t)^2",
                    "solve_s": t_solve, "backward_tc_s": t_bwd, "backward_cuda_cores_s": t_simt,
                    "tc_vs_cuda_cores_rel_diff": tc_vs_simt, "fp64_solve_s": t_ref,
                    "max_rel_eig_err_vs_fp64_gpu": float(np.max(np.abs(vals - ref) / ref)),
                    "grad_rel_err_A_vs_fp64_gpu": ra, "grad_rel_err_B_vs_fp64_gpu": rb,
                    "adjoint_write_GBs": 2 * spec.n ** 2 * 8 / t_bwd / 1e9,
                    "adjoint_write_frac": 2 * spec.n ** 2 * 8 / t_bwd / 1e9 / _peaks()[0]["hbm_gbs"]})
        s.close(); s64.close()
    elif args.mode == "profile":
        # one config-1 solve in a fresh process, nothing else: the command the ncu launch lists run
        spec = CONFIGS[1]
        p = make_problem_torch(spec, device="cuda")
        s = bse.Solver(p["A"], p["B"], stream=stream)
        vals, _, nconv, t = _timed_solve(s, NEV, TOL, stream, vectors=False)
        st = s.stats(); s.close()
        out.update({"workload": "one config-1 solve (PH N=10000 complex128, 100 pairs, FP64)", "s": t,
                    "krylov_steps": st["steps"], "passes": st["passes"], "launches": st["launches"]})
    elif args.mode == "haydock":
        # Lanczos-Haydock spectrum on the config-1 shapes (PH, N = 10000, complex128)
        spec = CONFIGS[1]
        p = make_problem_torch(spec, device="cuda")
        A, B = p["A"], p["B"]
        del p
        m = 600
        omega = np.linspace(0.0, 12.0, 4001)
        d = torch.from_numpy(random_start(spec.n, seed=11)).cuda()
        ts = []
        for it in range(args.warmup + args.steps):
            s = bse.Solver(A, B, stream=stream)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            spec_v, F, coefs, steps = s.haydock(d, m, omega, 0.05)
            e1.record(stream); torch.cuda.synchronize()
            st = s.stats(); s.close()
            if it >= args.warmup:
                ts.append(e0.elapsed_time(e1) / 1e3)
        # oracle recurrence on the host: a bounded sample of steps, scaled to m
        import oracle as O
        Ah, Bh = A.cpu().numpy(), B.cpu().numpy()
        dh = d.cpu().numpy()
        k = 4
        t0 = time.perf_counter()
        O.lanczos_ph(Ah, Bh, dh, k)
        t_cpu = (time.perf_counter() - t0) / k * m
        out.update({"workload": f"PH N={spec.n} complex128, Haydock m={m} steps, 4001 frequencies, eta 0.05 eV",
                    "s_per_spectrum": statistics.median(ts), "steps": steps, "passes": st["passes"],
                    "ms_per_step": statistics.median(ts) * 1e3 / m, "launches": st["launches"],
                    "cpu_oracle_s_extrapolated": t_cpu, "cpu_sample": f"{k} oracle steps scaled to {m}",
                    "cores": os.cpu_count()})
    elif args.mode == "mixed":
        spec = CONFIGS[4]
        p = make_problem_torch(spec, device="cuda")
        A, B = p["A"], p["B"]
        del p
        nev = spec.nev
        n = args.n or spec.n                          # --n shrinks the workload for trial runs
        if n != spec.n:
            A, B = A[:n, :n].contiguous(), B[:n, :n].contiguous()
        out["N"] = n

        def leg(name, solver):
            vals, _, nconv, t = _timed_solve(solver, nev, 1e-6, stream, vectors=False)
            st = solver.stats()
            solver.close()
            out.update({f"{name}_s": t, f"{name}_steps": st["steps"], f"{name}_passes": st["passes"],
                        f"{name}_max_residual": st["max_residual"], f"{name}_nconv": int(nconv),
                        f"{name}_product_ms_per_pass": st["ms_product"] / max(st["passes"], 1),
                        f"{name}_product_shape": [st["shape_ctas_per_sm"], st["shape_strided"]]})
            return vals, t

        # the mixed path: complex64 storage, FP64 basis, double-FP32 products
        vals, t_mixed = leg("mixed", bse.Solver(A, B, stream=stream, mixed=True))
        if args.fp32:    # complex64 with plain FP32 products and basis (residual floor ~eps32 * kappa)
            v32, _ = leg("fp32", bse.Solver(A, B, stream=stream))
            out["max_rel_diff_fp32_vs_mixed"] = float(np.max(np.abs(v32 - vals) / vals))
        if args.fp64 or args.df:
            A64 = A.to(torch.complex128); del A
            B64 = B.to(torch.complex128); del B
            if args.df:
                vdf, tdf = leg("fp64df", bse.Solver(A64, B64, stream=stream, df=True))
                out["speedup_mixed_over_fp64df"] = tdf / t_mixed
            if args.fp64:
                v64, t64 = leg("fp64", bse.Solver(A64, B64, stream=stream))
                out["max_rel_diff_mixed_vs_fp64"] = float(np.max(np.abs(vals - v64) / v64))
                out["speedup_mixed_over_fp64"] = t64 / t_mixed
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--mode", default="solve", choices=["solve", "product", "tda", "batch", "adjoint", "mixed",
                                                        "variants",
                                                              "haydock", "profile", "backward"])
    ap.add_argument("--n", type=int, default=0, help="product mode: N (default 8000); mixed mode: principal "
                                                       "block of the config-4 matrices (default: all of it)")
    ap.add_argument("--dtype", default="c128", choices=["c128", "c64"])
    ap.add_argument("--op", default="mplus", choices=["mplus", "a"])
    ap.add_argument("--fp64", action="store_true", help="mixed mode: also run the FP64 path")
    ap.add_argument("--df", action="store_true",
                    help="complex128 with the Lanczos products in double-FP32 arithmetic (BSE_C128_DF)")
    ap.add_argument("--fp32", action="store_true", help="mixed mode: also run plain FP32 (BSE_C64)")
    ap.add_argument("--mixed", action="store_true",
                    help="product mode: complex64 storage with the mixed path's products (BSE_C64_MIXED)")
    ap.add_argument("--skip-config4", action="store_true",
                    help="solve mode: leave out the config-4 record (mixed vs FP64 at N = 50000)")
    ap.add_argument("--config4-fp64", dest="config4_fp64", action="store_true",
                    help="solve mode: add the plain FP64 solve of config 4 and the mixed-over-FP64 speed-up")
    ap.add_argument("--tau", type=float, default=0.0,
                    help="product mode with --mixed: tile threshold (0: the tol-1e-6 default, <0: every tile exact)")
    ap.add_argument("--ncv", type=int, default=0, help="solve mode: Krylov subspace size (0 = library default)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "product":
        run_product(args)
    elif args.mode == "solve":
        run_gpu(args)
    else:
        run_workload(args)


if __name__ == "__main__":
    main()
