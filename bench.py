#!/usr/bin/env python
"""Benchmark: FE SpMV effective HBM bandwidth (and CG solves) on one GB300.

Workload: P1 linear elasticity on a jittered 64^3-node Kuhn tet grid
(786,432 rows, ~34M nnz after clamping z=0), randomly numbered, seeded
(fegen.cube_elasticity(64, 1502)); x ~ U[-1, 1] (seed 1504).

One step = one FP64 product y' = A' x' by the FE warp-slice kernel in the
handle's permuted numbering (the operator CG applies every iteration).  The
matrix (414 MB) is larger than the 126 MB L2, so every step streams it from
HBM; the steps are enqueued back to back between two CUDA events on the
launching stream (mean time per step).  A second figure times steps one by one
after a 256 MB write (cold L2, launch latency included).  Effective bandwidth
uses the minimum bytes of one product: nnz*(8 B value + 4 B index) + n*(8 B x +
8 B y).

Also reported: the CSR baselines, the product in the input numbering, the end-to-end
call with host buffers (copies inside the timed region), CG solves when
available, the CPU oracle timed on the host cores, and SM clocks sampled during
the run.

--impl reference times the CPU oracle (plain FP64 CSR product) on the same
matrix and prints the same JSON line with "impl": "reference".
N > 1 (torchrun): every rank runs an independent replica (the product does not
shard); value is the sum over ranks of bytes / the slowest rank's time.
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "SpMV effective HBM GB/s (% of ~8 TB/s); CG solves/s and p50/p99 latency at 1e-10"
WORKLOAD = "cube_elasticity_64"
NOMINAL_HBM_GBS = 8000.0
PROFILES = os.path.join(ROOT, "profiles")
KERNEL_SRCS = {k: [os.path.join(ROOT, "paper_1501_00324_gb300", "csrc", f) for f in fs]
               for k, fs in {"sliced": ("spmv_kernels.cu", "spmv_device.cuh"),
                             "tiled": ("tiled.cu", "tiled_device.cuh", "spmv_device.cuh")}.items()}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--sigma", type=int, default=1024)
    ap.add_argument("--vec", type=int, default=1,
                    help="entries per lane per load of the headline handle (1: least padding)")
    ap.add_argument("--extras-vec", type=int, default=4,
                    help="vector width of the handle the low-precision and multi-RHS extras use")
    ap.add_argument("--threshold", type=int, default=0)
    ap.add_argument("--block", type=int, default=256)
    ap.add_argument("--tiles", type=int, choices=[0, -1], default=0,
                    help="0: x staged through shared memory per tile of slices; -1: x gathered from L1/L2")
    ap.add_argument("--kernel", choices=["f64", "df64"], default="f64",
                    help="FP64 product: DFMA (f64) or float pairs on the FP32 pipe (df64)")
    ap.add_argument("--only-spmv", action="store_true",
                    help="time the FE product only (for profiling runs)")
    ap.add_argument("--ablation", type=int, default=1,
                    help="the layout ablation (CSR, slices, sort, Morton order, tiles) on two workloads")
    ap.add_argument("--assembly", type=int, default=1,
                    help="time the assembly of the workload matrix from its element matrices")
    ap.add_argument("--multi-cg", type=int, default=1,
                    help="time cg_solve_multi with 32 right-hand sides on the workload matrix")
    ap.add_argument("--profile-target", choices=["multi", "multi64", "fp32", "cg", "cg_f32", "cg_multi", "nb_cg_multi", "assembly",
                                                 "nb_fp32", "nb_multi", "batch"], default=None,
                    help="run only this piece a few times (for ncu), no JSON line")
    ap.add_argument("--cg-solves", type=int, default=5)
    ap.add_argument("--cpu-seconds", type=float, default=16.0,
                    help="host seconds of the CPU baseline (oracle SpMV and CG, 1 core and all cores)")
    ap.add_argument("--c1", type=int, default=1,
                    help="1: also measure the 20^3 cube Laplacian (us per product, CG to 1e-10)")
    ap.add_argument("--serve-seconds", type=float, default=3.0,
                    help="length of each serving run (per arm and arrival rate); 0 skips")
    ap.add_argument("--serve-small", action="store_true",
                    help="a small serving pool: 12 meshes of 5k..300k rows (default: 48 of 5k..3M)")
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-sweep", type=str, default="0.25,0.5,0.75,1.0,1.25",
                    help="arrival rates as fractions of the grouped server's saturation rate")
    ap.add_argument("--shell", type=int, default=1,
                    help="1: also measure the 24x256x512 shell Laplacian (FP64/BF16 products, refined CG)")
    ap.add_argument("--batch-meshes", type=int, default=256,
                    help="cubes in the batched solve (node counts log-uniform in [1k, 200k]); 0 skips")
    return ap.parse_args()


def min_bytes(n, nnz, val_bytes=8, vec_bytes=8):
    return nnz * (val_bytes + 4) + n * 2 * vec_bytes


def fp64_peak_tflops(torch, dev, peaks):
    """FP64 FMA peak of the device: 2 lanes per SM per clock (GB300's nominal 1.25
    TFLOP/s over 152 SMs at 2.07 GHz), 2 FLOP per FMA, at the maximum SM clock."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = (peaks or {}).get("sm_max_mhz", 2070.0)
    return 2 * 2 * sms * mhz * 1e6 / 1e12


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def kernel_hash(family="sliced"):
    h = hashlib.sha256()
    for f in KERNEL_SRCS[family]:
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def profile_traffic(name):
    """DRAM bytes per launch from the committed ncu summary profiles/<name>_cube_elasticity_64.md
    (name: tiled_f64, sliced_f64, sliced_df64), if it matches this source."""
    try:
        text = open(os.path.join(PROFILES, f"{name}_cube_elasticity_64.md")).read()
    except OSError:
        return None, "no ncu summary committed"
    h = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    b = re.search(r"dram_bytes_per_launch_full_size:\s*([0-9.eE+]+)", text)
    if not h or not b:
        return None, "summary lacks traffic figures"
    if h.group(1) != kernel_hash(name.split("_")[0]):
        return None, "kernel changed since the ncu capture"
    return float(b.group(1)), "ncu dram__bytes_read.sum + dram__bytes_write.sum"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms in the background."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = None

    def __enter__(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.proc or not self.f:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.f.flush()
        rows = [ln.split(",") for ln in open(self.f.name).read().strip().splitlines() if ln.strip()]
        os.unlink(self.f.name)
        mhz, mx, reasons, loaded = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm, smax, pw = float(r[1]), float(r[2]), float(r[3])
            except (ValueError, IndexError):
                continue
            mx = smax
            mhz.append(sm)
            if pw > 250:
                loaded.append(sm)
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        use = loaded or mhz
        return {"sm_mhz": statistics.median(use) if use else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(mhz), "samples_under_load": len(loaded)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(value, world):
    """Max over ranks (NCCL on GPUs; the same call over gloo on CPU processes)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def timed_repeats(fn, seconds, min_reps=1):
    """Call fn until `seconds` have passed (at least min_reps times); (reps, elapsed)."""
    t0 = time.perf_counter()
    k = 0
    while True:
        fn()
        k += 1
        el = time.perf_counter() - t0
        if el >= seconds and k >= min_reps:
            return k, el


def cpu_oracle_spmv(p, x, seconds, threads=1):
    """Time the oracle's FP64 CSR product on `threads` host cores for about `seconds`."""
    import oracle
    oracle.set_threads(threads)
    try:
        oracle.csr_spmv(p.rowptr, p.colind, p.values, x)          # warm
        return timed_repeats(lambda: oracle.csr_spmv(p.rowptr, p.colind, p.values, x), seconds)
    finally:
        oracle.set_threads(1)


def cpu_baseline_leg(p, x, y_gpu, seconds, c1=None, cg_iters=None):
    """The CPU oracle on the host cores, bounded samples of the benchmark's workloads:
    the FP64 CSR product of the 64^3 elasticity matrix on 1 core and on all cores,
    Jacobi-PCG iterations on it (all cores; the per-iteration time times the full
    solve's iteration count), and the 20^3 cube Laplacian (product warm and after a
    256 MB host write; full CG solves to 1e-10, 1 core and all cores).  It also
    checks the GPU's headline product y_gpu (input numbering) against the oracle's
    product of the same x: |y - y_oracle| <= 1e-12 * (|A| |x|) per row."""
    import oracle
    import fegen
    cores = host_cores()
    mb = min_bytes(p.n_rows, p.nnz)
    k1, el1 = cpu_oracle_spmv(p, x, 0.25 * seconds, 1)
    kn, eln = cpu_oracle_spmv(p, x, 0.15 * seconds, cores)
    out = {"value": round(mb * kn / eln / 1e9, 3), "unit": "GB/s", "cores": cores, "kind": "oracle",
           "sample": (f"{kn} FP64 CSR products of the {WORKLOAD} matrix in {eln:.1f} s on {cores} cores "
                      f"(row-parallel, same sums as 1 core); 1 core: {k1} in {el1:.1f} s"),
           "spmv_1core_gbs": round(mb * k1 / el1 / 1e9, 3),
           "spmv_1core_ms": round(el1 / k1 * 1e3, 2), "spmv_allcore_ms": round(eln / kn * 1e3, 2),
           "l2_note": "the 420 MB matrix exceeds every host cache: each product is cold"}
    # the headline product's output against the oracle (sampled from the timed kernel)
    if y_gpu is not None:
        oracle.set_threads(cores)
        try:
            yo = oracle.csr_spmv(p.rowptr, p.colind, p.values, x)
            bound = oracle.csr_spmv(p.rowptr, p.colind, np.abs(p.values), np.abs(x))
        finally:
            oracle.set_threads(1)
        err = np.abs(y_gpu - yo)
        ratio = np.where(bound > 0, err / np.where(bound > 0, bound, 1.0), np.where(err > 0, np.inf, 0.0))
        out["headline_output_check"] = {"rows": int(p.n_rows), "worst_err_over_abs_bound": float(ratio.max()),
                                        "bound": 1e-12, "pass": bool(ratio.max() <= 1e-12)}
    # Jacobi-PCG on the elasticity matrix: a bounded number of iterations on all cores
    b = fegen.random_vector(p.n_rows, 1505)
    oracle.set_threads(cores)
    try:
        kit = 30
        t0 = time.perf_counter()
        _, info = oracle.pcg(p.rowptr, p.colind, p.values, b, tol=1e-30, max_iter=kit, max_restarts=0)
        el = time.perf_counter() - t0
    finally:
        oracle.set_threads(1)
    per_it = el / max(1, info["iters"])
    cg = {"cores": cores, "iters_timed": info["iters"], "ms_per_iteration": round(per_it * 1e3, 2)}
    if cg_iters:
        cg.update({"iters_full_solve": cg_iters, "est_s_per_solve": round(per_it * cg_iters, 2),
                   "est_solves_per_s": round(1.0 / (per_it * cg_iters), 4),
                   "note": "iteration time x the iteration count of the FP64 solve to 1e-10 "
                           "(the GPU's count, held within 2 % + 2 of the oracle's by the tests)"})
    out["cg_cube_elasticity_64"] = cg
    if c1 is not None:
        q = c1
        xq = fegen.random_vector(q.n_rows, 1504)
        flush = np.empty(256 * 1024 * 1024 // 8)
        c1o = {}
        for th in (1, cores):
            oracle.set_threads(th)
            try:
                kw, elw = timed_repeats(lambda: oracle.csr_spmv(q.rowptr, q.colind, q.values, xq), 0.05 * seconds, 3)
                cold = []
                for _ in range(5):
                    flush.fill(1.0)
                    t0 = time.perf_counter()
                    oracle.csr_spmv(q.rowptr, q.colind, q.values, xq)
                    cold.append(time.perf_counter() - t0)
                u = fegen.manufactured_solution(q)
                bq = oracle.csr_spmv(q.rowptr, q.colind, q.values, u)
                lat = []
                t_end = time.perf_counter() + 0.05 * seconds
                while time.perf_counter() < t_end or len(lat) < 3:
                    t0 = time.perf_counter()
                    xs, inf = oracle.pcg(q.rowptr, q.colind, q.values, bq, tol=1e-10)
                    lat.append(time.perf_counter() - t0)
            finally:
                oracle.set_threads(1)
            lat_ms = sorted(1e3 * t for t in lat)
            c1o[f"{th}_cores"] = {"spmv_us_warm": round(elw / kw * 1e6, 2),
                                  "spmv_us_cold": round(float(np.median(cold)) * 1e6, 2),
                                  "cg_solves_per_s": round(len(lat) / sum(lat), 2),
                                  "cg_p50_ms": round(float(np.percentile(lat_ms, 50)), 3),
                                  "cg_p99_ms": round(float(np.percentile(lat_ms, 99)), 3),
                                  "cg_iters": inf["iters"], "cg_status": inf["status"],
                                  "true_relres": inf["true_relres"]}
        out["cube_laplace_20"] = c1o
    return out


def run_reference(args, world, rank):
    """CPU oracle arm: the same matrix and metric, the oracle's FP64 CSR product on the
    host cores (row-parallel; every row one sequential sum, as on one core)."""
    if rank != 0:
        return
    import fegen
    import oracle
    cores = host_cores()
    p = fegen.cube_elasticity(64, 1502)
    x = fegen.random_vector(p.n_rows, 1504)
    oracle.set_threads(cores)
    for _ in range(max(0, args.warmup)):
        oracle.csr_spmv(p.rowptr, p.colind, p.values, x)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.csr_spmv(p.rowptr, p.colind, p.values, x)
    el = time.perf_counter() - t0
    oracle.set_threads(1)
    mb = min_bytes(p.n_rows, p.nnz)
    gbs = mb * args.steps / el / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(gbs, 3), "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(el / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "rows": p.n_rows, "nnz": p.nnz,
                   "kernel": f"oracle_csr_spmv (plain C, FP64, rows in parallel on {cores} host cores, "
                             "each row a sequential sum)"},
        "cpu_baseline": {"value": round(gbs, 3), "unit": "GB/s", "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} full products of the {WORKLOAD} matrix"},
        "e2e": {"value": round(gbs, 3), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    world, rank, local = dist_setup()
    if world > 1:
        import torch
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
            dist.init_process_group("nccl")
        else:   # host-only ranks (the reference arm, or tests of this path on CPU)
            dist.init_process_group("gloo")
    if args.impl == "reference":
        run_reference(args, world, rank)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    import torch
    import fegen
    import paper_1501_00324_gb300 as fs

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()

    p = fegen.cube_elasticity(64, 1502)
    n, nnz = p.n_rows, p.nnz
    x = fegen.random_vector(n, 1504)
    t0 = time.perf_counter()
    A = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 3, sigma=args.sigma, vec=args.vec,
                       threshold=args.threshold, block=args.block, tiles=args.tiles,
                       precisions=(0 if args.only_spmv else fs.FESPMV_PREC_F32 | fs.FESPMV_PREC_BF16)
                       | (fs.FESPMV_PREC_DF64 if args.kernel == "df64" else 0))
    create_s = time.perf_counter() - t0
    info = fs.spmv_get_info(A)

    xd = torch.from_numpy(x).to(dev)
    xp = torch.empty_like(xd)
    fs.spmv_permute(A, xd, xp, 0)
    yp = torch.empty_like(xd)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    mb = min_bytes(n, nnz)

    def timed_steps(fn, k):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(k)]
        for (a, b) in evs:
            flush.zero_()
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for (a, b) in evs]

    fe = lambda: fs.spmv_apply(A, xp, yp, fs.FESPMV_IO_PERMUTED)  # noqa: E731
    if args.profile_target:
        profile_piece(fs, torch, A, p, xp, args)
        return
    for _ in range(args.warmup):
        fe()
    torch.cuda.synchronize()

    def back_to_back(fn, k):
        """k launches enqueued back to back between two events; mean per launch (ms)."""
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / k

    clocks = ClockSampler(local)
    with clocks:
        barrier(world)
        torch.cuda.synchronize()
        wall0 = time.perf_counter()
        t_step = back_to_back(fe, args.steps)
        torch.cuda.synchronize()
        barrier(world)
        wall = time.perf_counter() - wall0
        times_flushed = timed_steps(fe, max(10, args.steps // 4))
        extra = {}
        te = None
        if not args.only_spmv:
            # end to end with host buffers (pinned), copies inside the timed region (every rank)
            xh = torch.from_numpy(x).pin_memory().numpy()
            yh = torch.empty(n, dtype=torch.float64).pin_memory().numpy()
            k_e2e = max(10, args.steps // 4)
            fs.spmv_apply(A, xh, yh)
            torch.cuda.synchronize()
            barrier(world)
            te0 = time.perf_counter()
            for _ in range(k_e2e):
                fs.spmv_apply(A, xh, yh)      # synchronous: H2D, permute, kernel, permute, D2H
            te = (time.perf_counter() - te0) / k_e2e
        # the extras characterise one GPU; with replicas on several GPUs only the timed
        # product steps and the end-to-end calls run, so the GPUs are held no longer than
        # the measurement needs
        if not args.only_spmv and world == 1:
            # product in the input numbering (the permutations folded into the tiled product)
            # (every extra product below is timed back to back, like the headline: each
            # matrix is larger than L2, so it streams from HBM on every launch)
            y_user = torch.empty_like(xd)
            fu = lambda: fs.spmv_apply(A, xd, y_user)  # noqa: E731
            fu()
            extra["fe_input_numbering_gbs"] = round(mb / (back_to_back(fu, args.steps) * 1e-3) / 1e9, 1)
            # low-precision and multi-RHS extras on a handle with wider lane loads (these
            # kernels are not on the FP64 pipe, where the headline's V = 1 saves padding)
            E = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 3, sigma=args.sigma,
                               vec=args.extras_vec, precisions=fs.FESPMV_PREC_F32 | fs.FESPMV_PREC_BF16)
            xe = torch.empty_like(xd)
            fs.spmv_permute(E, xd, xe, 0)
            # low-precision products of B = S A S (the refined CG's inner operator)
            xs = xe.float()
            ys = torch.empty_like(xs)
            for name, prec, vb in (("fp32", fs.FESPMV_PREC_F32, 4), ("bf16", fs.FESPMV_PREC_BF16, 2)):
                f = lambda: fs.spmv_apply_scaled(E, xs, ys, prec, fs.FESPMV_IO_PERMUTED)  # noqa: E731
                f()
                tl = back_to_back(f, args.steps)
                extra[f"{name}_spmv_gbs"] = round((nnz * (vb + 4) + n * 8) / (tl * 1e-3) / 1e9, 1)
            # the same products on 3x3 node blocks (one int32 column per 9 values)
            NB = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 3, sigma=args.sigma,
                                vec=args.extras_vec, node_blocks=3,
                                precisions=fs.FESPMV_PREC_F32 | fs.FESPMV_PREC_BF16)
            nbi = fs.spmv_get_info(NB)
            xnb = torch.empty_like(xd)
            fs.spmv_permute(NB, xd, xnb, 0)
            xnb32, ynb32 = xnb.float(), torch.empty(n, dtype=torch.float32, device=dev)
            nbo = {"blocks": nbi["nb_len"], "padding_pct": round(100.0 * (9 * nbi["nb_len"] - nnz) / nnz, 2)}
            for name, prec, vb in (("fp32", fs.FESPMV_PREC_F32, 4), ("bf16", fs.FESPMV_PREC_BF16, 2)):
                f = lambda: fs.spmv_apply_scaled(NB, xnb32, ynb32, prec, fs.FESPMV_IO_PERMUTED)  # noqa: E731
                f()
                tl = back_to_back(f, args.steps)
                nbo[f"{name}_gbs"] = round((nnz * (vb + 4) + n * 8) / (tl * 1e-3) / 1e9, 1)
                nbo[f"{name}_us"] = round(tl * 1e3, 2)
                nbo[f"{name}_moved_gbs"] = round((nbi["nb_len"] * (9 * vb + 4) + n * 8) / (tl * 1e-3) / 1e9, 1)
            if hasattr(fs, "cg_solve"):
                nbo["cg_f32_reliable"] = bench_cg(fs, torch, NB, p, args.cg_solves, fs.FESPMV_CG_F32_REFINE,
                                                  flags=fs.FESPMV_CG_RELIABLE)
            fs.spmv_destroy(NB)
            extra["node_blocks_3x3"] = nbo
            # 32 right-hand sides in one pass over the FP32 matrix (row-major n x 32)
            X32 = torch.rand((n, 32), dtype=torch.float32, device=dev)
            Y32 = torch.empty_like(X32)
            fm = lambda: fs.spmv_apply_multi(E, X32, Y32, fs.FESPMV_PREC_F32, fs.FESPMV_IO_PERMUTED)  # noqa: E731
            fm()
            tmean = back_to_back(fm, max(10, args.steps // 8)) * 1e-3
            extra["multi32_fp32"] = {"gbs": round((nnz * 8 + n * 32 * 8) / tmean / 1e9, 1),
                                     "us_per_apply": round(tmean * 1e6, 1),
                                     "us_per_rhs": round(tmean * 1e6 / 32, 2)}
            # the same on 3x3 node blocks (one X row gathered per column node serves 3 rows)
            NBm = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 3, sigma=args.sigma,
                                 vec=args.extras_vec, node_blocks=3, precisions=fs.FESPMV_PREC_F32)
            fm = lambda: fs.spmv_apply_multi(NBm, X32, Y32, fs.FESPMV_PREC_F32, fs.FESPMV_IO_PERMUTED)  # noqa: E731
            fm()
            tmean = back_to_back(fm, max(10, args.steps // 8)) * 1e-3
            extra["multi32_fp32_node_blocks"] = {"gbs": round((nnz * 8 + n * 32 * 8) / tmean / 1e9, 1),
                                                 "us_per_apply": round(tmean * 1e6, 1),
                                                 "us_per_rhs": round(tmean * 1e6 / 32, 2)}
            fs.spmv_destroy(NBm)
            del X32, Y32
            # the same with the FP64 matrix and FP64 right-hand sides
            X64 = torch.rand((n, 32), dtype=torch.float64, device=dev)
            Y64 = torch.empty_like(X64)
            fm = lambda: fs.spmv_apply_multi(E, X64, Y64, fs.FESPMV_PREC_F64, fs.FESPMV_IO_PERMUTED)  # noqa: E731
            fm()
            tmean = back_to_back(fm, max(10, args.steps // 8)) * 1e-3
            extra["multi32_fp64"] = {"gbs": round((nnz * 12 + n * 32 * 16) / tmean / 1e9, 1),
                                     "us_per_apply": round(tmean * 1e6, 1),
                                     "us_per_rhs": round(tmean * 1e6 / 32, 2)}
            # the same with float-pair products (a handle holding the pairs)
            Fm = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 3, sigma=args.sigma,
                                vec=args.extras_vec, precisions=fs.FESPMV_PREC_DF64)
            fm = lambda: fs.spmv_apply_multi(Fm, X64, Y64, fs.FESPMV_PREC_F64, fs.FESPMV_IO_PERMUTED)  # noqa: E731
            fm()
            tmean = back_to_back(fm, max(10, args.steps // 8)) * 1e-3
            extra["multi32_fp64_float_pairs"] = {"gbs": round((nnz * 12 + n * 32 * 16) / tmean / 1e9, 1),
                                                 "us_per_apply": round(tmean * 1e6, 1)}
            fs.spmv_destroy(Fm)
            fs.spmv_destroy(E)
            del X64, Y64
            # the same FE product with x gathered from L1/L2 (no tiles), for comparison
            if info["n_tiles"] > 0:
                G = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 3, sigma=args.sigma,
                                   vec=args.vec, threshold=args.threshold, block=args.block, tiles=-1)
                fg = lambda: fs.spmv_apply(G, xp, yp, fs.FESPMV_IO_PERMUTED)  # noqa: E731
                fg()
                extra["fe_global_gather_gbs"] = round(mb / (back_to_back(fg, args.steps) * 1e-3) / 1e9, 1)
                fs.spmv_destroy(G)
            # float-pair products (FP32 pipe, FP64 fallback; within the 1e-12 bound): the
            # same tiled layout off the FP64 pipe -- reported beside the FP64 headline
            if info["n_tiles"] > 0 and args.kernel == "f64":
                Fd = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 3, sigma=args.sigma,
                                    vec=args.vec, threshold=args.threshold, precisions=fs.FESPMV_PREC_DF64)
                ff = lambda: fs.spmv_apply(Fd, xp, yp, fs.FESPMV_IO_PERMUTED)  # noqa: E731
                ff()
                extra["fe_float_pair_gbs"] = round(mb / (back_to_back(ff, args.steps) * 1e-3) / 1e9, 1)
                if hasattr(fs, "cg_solve"):
                    # FP64-accurate Jacobi-PCG whose products run as float pairs on the FP32 pipe
                    extra["cg_float_pair_products"] = bench_cg(fs, torch, Fd, p, args.cg_solves, fs.FESPMV_CG_F64)
                fs.spmv_destroy(Fd)
            # CSR baselines on the input CSR
            for lanes in (1, 4, 8):
                B = fs.spmv_create(p.rowptr, p.colind, p.values, format=fs.FESPMV_FMT_CSR,
                                   csr_lanes=lanes)
                fs.spmv_apply(B, xd, y_user)
                tb = back_to_back(lambda: fs.spmv_apply(B, xd, y_user), args.steps)  # noqa: B023
                extra[f"csr_{'scalar' if lanes == 1 else f'vector{lanes}'}_gbs"] = round(
                    mb / (tb * 1e-3) / 1e9, 1)
                fs.spmv_destroy(B)
            if hasattr(fs, "cg_solve"):
                extra["cg"] = bench_cg(fs, torch, A, p, args.cg_solves, fs.FESPMV_CG_F64)
                extra["cg_single_reduction"] = bench_cg(fs, torch, A, p, args.cg_solves, fs.FESPMV_CG_F64,
                                                        flags=fs.FESPMV_CG_SINGLE_REDUCTION)
                extra["cg_f32_refine"] = bench_cg(fs, torch, A, p, args.cg_solves,
                                                  fs.FESPMV_CG_F32_REFINE)
                extra["cg_f32_reliable"] = bench_cg(fs, torch, A, p, args.cg_solves,
                                                    fs.FESPMV_CG_F32_REFINE, flags=fs.FESPMV_CG_RELIABLE)
                extra["cg_bf16_flexible"] = bench_cg(fs, torch, A, p, args.cg_solves,
                                                     fs.FESPMV_CG_BF16_REFINE, flags=fs.FESPMV_CG_FLEXIBLE)
            if hasattr(fs, "cg_solve_multi") and args.multi_cg:
                extra["cg_multi32"] = bench_cg_multi(fs, torch, p, args)
            if hasattr(fs, "assembly_create") and args.assembly:
                extra["assembly"] = bench_assembly(fs, torch, args, back_to_back)
            if args.ablation:
                extra["ablation"] = bench_ablation(fs, torch, args, back_to_back)
            if args.shell:
                extra["shell_24x256x512"] = bench_shell(fs, torch, args)
            if args.batch_meshes > 0:
                extra["batched"] = bench_batched(fs, torch, args)
            if args.c1:
                extra["cube_laplace_20"] = bench_c1(fs, torch, args)
            if args.serve_seconds > 0 and hasattr(fs, "srv_create"):
                extra["serving"] = bench_serving(fs, torch, args)
    clk = clocks.summary()
    # the headline product's output (the last timed step), in the input numbering
    y_check = torch.empty_like(xd)
    fs.spmv_apply(A, xp, yp, fs.FESPMV_IO_PERMUTED)
    fs.spmv_permute(A, yp, y_check, 1)
    y_check = y_check.cpu().numpy()

    t_mean = t_step * 1e-3
    t_max = reduce_max(t_mean, world)
    te_max = reduce_max(te, world) if te is not None else None
    value = mb * world / t_max / 1e9
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    achieved = mb / t_mean / 1e9
    tiled = info["n_tiles"] > 0 and args.kernel == "f64"
    kname = "tiled_f64" if tiled else f"sliced_{args.kernel}"
    traffic, traffic_src = profile_traffic(kname)
    # bytes the layout actually moves: values + 16-bit indices + tile column lists (+ x, y)
    layout_bytes = (info["packed_len"] * 10 + info["tile_dict_len"] * 4 + n * 16 if tiled
                    else info["packed_len"] * 12 + n * 16)

    if rank == 0:
        cpu = None
        if world == 1 and args.cpu_seconds > 0 and not args.only_spmv:
            import fegen as _fg
            cg_it = extra.get("cg", {}).get("iters")
            cpu = cpu_baseline_leg(p, x, y_check, args.cpu_seconds,
                                   c1=_fg.cube_laplace(20, 1501) if args.c1 else None,
                                   cg_iters=cg_it[0] if cg_it else None)
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_max * 1e3, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.kernel == "f64" else "df64 (float pairs, fp32 FMA)",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "rows": n, "nnz": nnz,
                       "kernel": (f"tiled_f64 (x staged in shared memory, {info['n_tiles']} tiles of <= 8 "
                                  f"slices, 16-bit column indices)" if tiled else f"sliced_{args.kernel}")
                                 + f" V={info['vec']} threshold={args.threshold} sigma={args.sigma}"
                                 + ("" if tiled else f" block={args.block}"),
                       "order": "Morton nodes, windowed length sort, sorted columns",
                       "l2": f"inputs larger than L2: the {layout_bytes / 1e6:.0f} MB layout streams from HBM every "
                             "step (x stays L2-resident, as in CG); steps enqueued back to back",
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                       "create_s": round(create_s, 2),
                       "packed_len": info["packed_len"],
                       "padding_pct": round(100.0 * (info["packed_len"] - nnz) / max(nnz, 1), 2)},
            "pct_of_8tbs": round(100 * value / world / NOMINAL_HBM_GBS, 1),
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                         "unit": "GB/s", "frac": round(achieved / peak, 4),
                         "traffic": traffic, "traffic_source": traffic_src,
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if peaks
                         else "fallback 6.8 TB/s",
                         "bytes_per_launch": mb,
                         "layout_bytes_per_launch": layout_bytes,
                         "note": "achieved = algorithmic bytes (FP64 values, int32 indices, x, y) / time; "
                                 "the tiled layout moves layout_bytes_per_launch; the kernel is FP64-pipe "
                                 "bound (roofline_fp64)"},
            # the same kernel against the FP64 pipe, the roof it actually sits on (one DFMA
            # per stored entry; GB300's nominal 1.25 TFLOP/s FP64 is 2 FMA lanes per SM per
            # clock: peak = 2 FLOP x 2 lanes x SMs x the maximum SM clock)
            "roofline_fp64": None if args.kernel != "f64" else {
                "bound": "alu", "unit": "TFLOP/s",
                "achieved": round(2 * nnz / t_mean / 1e12, 4),
                "peak": round(fp64_peak_tflops(torch, dev, peaks), 4),
                "frac": round(2 * nnz / t_mean / 1e12 / fp64_peak_tflops(torch, dev, peaks), 4),
                "peak_source": "derived: 2 FP64 FMA lanes per SM per clock x SMs x max SM clock"},
            "gpu_launches": args.steps * (2 if args.kernel == "df64" else 1),
            "step_with_l2_flush": {"ms": round(statistics.mean(times_flushed), 4),
                                   "gbs": round(mb / (statistics.mean(times_flushed) * 1e-3) / 1e9, 1),
                                   "note": "each step timed alone after a 256 MB write"},
            "wall_s_timed": round(wall, 4),
            "clocks": clk,
        }
        line["e2e"] = None if te_max is None else {
            "value": round(mb * world / te_max / 1e9, 1), "unit": "GB/s",
            "h2d_bytes_per_step": 8 * n * world, "d2h_bytes_per_step": 8 * n * world}
        line.update(extra)
        if cpu:
            line["cpu_baseline"] = cpu
        # last key: a compact view of every stated workload, so that the end of the
        # line (what a log tail keeps) carries all of them
        line["configs_summary"] = configs_summary(line)
        print(json.dumps(line), flush=True)
    fs.spmv_destroy(A)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def bench_c1(fs, torch, args):
    """The 20^3 cube Laplacian (8,000 rows; ~108k stored entries after the Dirichlet
    face).  Its FP64 FE product (1.4 MB, L2-resident) is launch-bound, so it is
    reported in microseconds: per launch back to back on the stream, per product
    inside a CUDA graph of 100 products (device time without the launch overhead),
    each alone after a 256 MB write (cold L2), and end to end through spmv_apply with
    pinned host buffers.  Then Jacobi-PCG to 1e-10 on b = A u* (manufactured u*):
    FP64, and FP32 values with FP64 reliable updates."""
    import fegen
    p = fegen.cube_laplace(20, 1501)
    n, nnz = p.n_rows, p.nnz
    mb = min_bytes(n, nnz)
    A = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 1, sigma=1024,
                       precisions=fs.FESPMV_PREC_F32)
    x = torch.from_numpy(fegen.random_vector(n, 1504)).cuda()
    xp = torch.empty_like(x)
    fs.spmv_permute(A, x, xp, 0)
    yp = torch.empty_like(x)
    f = lambda: fs.spmv_apply(A, xp, yp, fs.FESPMV_IO_PERMUTED)  # noqa: E731
    for _ in range(20):
        f()
    torch.cuda.synchronize()

    def events():
        return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    K = 2000
    a, b = events()
    a.record()
    for _ in range(K):
        f()
    b.record()
    torch.cuda.synchronize()
    us_b2b = a.elapsed_time(b) / K * 1e3
    us_graph = None
    try:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for _ in range(100):
                f()
        g.replay()
        torch.cuda.synchronize()
        a, b = events()
        a.record()
        for _ in range(20):
            g.replay()
        b.record()
        torch.cuda.synchronize()
        us_graph = a.elapsed_time(b) / 2000 * 1e3
        del g
    except Exception as e:  # graph capture is an extra view; the other figures stand alone
        us_graph = f"capture failed: {type(e).__name__}"
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    evs = [events() for _ in range(50)]
    for (ea, eb) in evs:
        flush.zero_()
        ea.record()
        f()
        eb.record()
    torch.cuda.synchronize()
    us_cold = statistics.median(ea.elapsed_time(eb) for ea, eb in evs) * 1e3
    del flush
    xh = torch.from_numpy(fegen.random_vector(n, 1504)).pin_memory().numpy()
    yh = torch.empty(n, dtype=torch.float64).pin_memory().numpy()
    fs.spmv_apply(A, xh, yh)
    ke = 500
    t0 = time.perf_counter()
    for _ in range(ke):
        fs.spmv_apply(A, xh, yh)
    us_e2e = (time.perf_counter() - t0) / ke * 1e6
    out = {"rows": n, "nnz": nnz,
           "spmv_us_back_to_back": round(us_b2b, 2),
           "spmv_us_in_graph": round(us_graph, 2) if isinstance(us_graph, float) else us_graph,
           "spmv_us_cold_l2": round(us_cold, 2),
           "spmv_us_e2e_host_buffers": round(us_e2e, 2),
           "spmv_gbs_in_graph": round(mb / (us_graph * 1e-6) / 1e9, 1) if isinstance(us_graph, float) else None,
           "cg_f64": bench_cg(fs, torch, A, p, 50, fs.FESPMV_CG_F64),
           "cg_f32_reliable": bench_cg(fs, torch, A, p, 50, fs.FESPMV_CG_F32_REFINE,
                                       flags=fs.FESPMV_CG_RELIABLE)}
    fs.spmv_destroy(A)
    return out


def _pick(d, *keys):
    """Nested lookup that tolerates missing pieces (None)."""
    for k in keys:
        if not isinstance(d, dict) or k not in d:
            return None
        d = d[k]
    return d


def configs_summary(line):
    """One compact object per stated workload (numbers taken from the line)."""
    cg = lambda c: None if not isinstance(c, dict) else {  # noqa: E731
        k: c.get(k) for k in ("solves_per_s", "p50_ms", "p99_ms", "iters", "status", "true_relres_max")
        if c.get(k) is not None}
    c1 = line.get("cube_laplace_20") or {}
    cpu = line.get("cpu_baseline") or {}
    out = {
        "C1_cube_laplace_20": {
            "spmv_us": {k: c1.get(f"spmv_us_{k}") for k in ("back_to_back", "in_graph", "cold_l2",
                                                              "e2e_host_buffers")},
            "cg_f64_1e-10": cg(c1.get("cg_f64")), "cg_f32_reliable_1e-10": cg(c1.get("cg_f32_reliable")),
            "cpu": _pick(cpu, "cube_laplace_20")},
        "C2_cube_elasticity_64": {
            "f64_spmv_gbs": line.get("value"), "frac_of_measured": _pick(line, "roofline", "frac"),
            "e2e_gbs": _pick(line, "e2e", "value"), "fp32_spmv_gbs": line.get("fp32_spmv_gbs"),
            "bf16_spmv_gbs": line.get("bf16_spmv_gbs"), "csr_vector4_gbs": line.get("csr_vector4_gbs"),
            "node_block_fp32_bf16_gbs": [_pick(line, "node_blocks_3x3", "fp32_gbs"),
                                         _pick(line, "node_blocks_3x3", "bf16_gbs")],
            "cg_f32_reliable_node_blocks": cg(_pick(line, "node_blocks_3x3", "cg_f32_reliable")),
            "cg_f64_1e-10": cg(line.get("cg")), "cg_f32_reliable_1e-10": cg(line.get("cg_f32_reliable")),
            "cg_bf16_flexible_1e-10": cg(line.get("cg_bf16_flexible")),
            "output_check": _pick(cpu, "headline_output_check", "worst_err_over_abs_bound"),
            "cpu_spmv_gbs": {"1_core": cpu.get("spmv_1core_gbs"), f"{cpu.get('cores')}_cores": cpu.get("value")},
            "cpu_cg_est_solves_per_s": _pick(cpu, "cg_cube_elasticity_64", "est_solves_per_s")},
        "C3_shell_24x256x512": {k: _pick(line, "shell_24x256x512", k) for k in (
            "f64_spmv_gbs", "f32_spmv_gbs", "bf16_spmv_gbs")},
        "C4_batched": {
            "meshes": _pick(line, "batched", "meshes"), "solves_per_s": _pick(line, "batched", "solves_per_s"),
            "frac_of_measured": _pick(line, "batched", "roofline", "frac"),
            "batch_s": _pick(line, "batched", "batched_reliable_s"),
            "rhs32_solves_per_s": _pick(line, "cg_multi32", "f32_reliable", "solves_per_s"),
            "rhs32_product_gbs": [_pick(line, "multi32_fp32", "gbs"), _pick(line, "multi32_fp32_node_blocks", "gbs")]},
    }
    sh = line.get("shell_24x256x512") or {}
    for k in ("cg_f64", "cg_f32_reliable", "cg_bf16_reliable", "cg_bf16_flexible"):
        if k in sh:
            out["C3_shell_24x256x512"][k] = cg(sh[k])
    sv = line.get("serving")
    if isinstance(sv, dict):
        out["C5_serving"] = {"pool": sv.get("pool"), "saturation_per_s": sv.get("saturation_per_s"),
                             "by_rate": {str(r.get("rate_per_s")): {
                                 a: [_pick(r, a, "solves_per_s"), _pick(r, a, "p50_ms_offered"),
                                     _pick(r, a, "p99_ms_offered")]
                                 for a in ("server", "server_grouped", "one_at_a_time")}
                                 for r in sv.get("sweep", [])},
                             "by_rate_fields": "[solves/s, p50 ms, p99 ms over all offered requests; "
                                               "null: that percentile was not served in the run]"}
    return out


def serving_pool(n_meshes, lo, hi, seed):
    """Meshes with row counts log-uniform in [lo, hi], kinds cycling cube / elasticity / shell."""
    import fegen
    rng = np.random.default_rng(seed)
    rows = np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_meshes))
    pool = []
    for i, N in enumerate(rows):
        kind = i % 3
        if kind == 0:
            p = fegen.valid_seed(lambda sd: fegen.cube_laplace(max(3, round(N ** (1 / 3))), sd),
                                 seed + 1 + i)
        elif kind == 1:
            p = fegen.valid_seed(lambda sd: fegen.cube_elasticity(max(3, round((N / 3) ** (1 / 3))), sd),
                                 seed + 1 + i)
        else:
            s = (N / (24 * 256 * 512)) ** (1 / 3)
            p = fegen.valid_seed(lambda sd: fegen.shell_laplace(max(3, round(24 * s)), max(4, round(256 * s)),
                                                                max(8, round(512 * s)), sd), seed + 1 + i)
        pool.append(p)
    return pool


def bench_serving(fs, torch, args):
    """Poisson arrivals of CG solves over a resident pool of 48 meshes (cube,
    elasticity, shell; 5k to 3M rows): the solve server (continuous batching,
    FP32 values with FP64 reliable updates), the same server with lockstep
    multi-RHS groups, and one-at-a-time FP64 cg_solve, all on the same arrival
    trace.  First an overload run (args.serve_rate) finds the grouped server's
    saturation rate; then a sweep of arrival rates at fractions of it, plus one
    rate at 0.5, 1 and 1.5 times the one-at-a-time capacity.  Arrivals span args.serve_seconds;
    either arm may start queued requests for one more second, then what still waits
    is cancelled and counted as not served."""
    import fegen
    if args.serve_small:
        n_mesh, lo, hi = 12, 5_000, 300_000
    else:
        n_mesh, lo, hi = 48, 5_000, 3_000_000
    t0 = time.perf_counter()
    pool = serving_pool(n_mesh, lo, hi, 1505)
    gen_s = time.perf_counter() - t0
    # elasticity meshes keep their FP32 values as 3x3 node blocks (the refined solves' products)
    mats = [fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, p.dofs_per_node, sigma=1024,
                           node_blocks=3 if p.dofs_per_node == 3 else 0, precisions=fs.FESPMV_PREC_F32)
            for p in pool]
    rhs = [[fegen.random_vector(p.n_rows, 7000 + 10 * i + k) for k in range(2)]
           for i, p in enumerate(pool)]
    setup_s = time.perf_counter() - t0
    pool_info = {"meshes": n_mesh, "rows_min": min(p.n_rows for p in pool),
                 "rows_max": max(p.n_rows for p in pool), "rows_total": sum(p.n_rows for p in pool),
                 "nnz_total": sum(p.nnz for p in pool), "gen_s": round(gen_s, 1), "setup_s": round(setup_s, 1)}
    sizes = [p.n_rows for p in pool]
    T = args.serve_seconds
    DRAIN = 1.0   # seconds after the last arrival in which either arm may still start queued requests

    def make_trace(rate, seed):
        rng = np.random.default_rng(seed)
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=int(rate * T * 1.5) + 10))
        arrivals = arrivals[arrivals < T]
        return [(float(a), int(rng.integers(n_mesh)), [1e-8, 1e-10][int(rng.integers(2))],
                 int(rng.integers(2))) for a in arrivals]

    def summarize(trace, lat, served, elapsed):
        """Latency percentiles over the served requests, and over every offered request
        with the unserved ones counted as slower than any served one (null when the
        percentile falls on an unserved request: the run left it unanswered)."""
        lat = np.array(sorted(lat)) * 1e3
        out = {"offered": len(trace), "served": served,
               "solves_per_s": round(served / elapsed, 2) if elapsed > 0 else 0.0,
               "p50_ms": round(float(np.percentile(lat, 50)), 2) if len(lat) else None,
               "p99_ms": round(float(np.percentile(lat, 99)), 2) if len(lat) else None}
        for q in (50, 99):
            k = int(np.ceil(q / 100 * len(trace))) - 1
            out[f"p{q}_ms_offered"] = round(float(lat[k]), 2) if 0 <= k < len(lat) else None
        return out

    def run_server(trace, group=0):
        S = fs.srv_create(48 << 30, 64)
        if group:
            fs.srv_set_grouping(S, group)
        ids = [fs.srv_register(S, A) for A in mats]
        tickets = []
        start = time.perf_counter()
        for (a, m, tol, k) in trace:
            now = time.perf_counter() - start
            if now < a:
                time.sleep(a - now)
            tickets.append(fs.srv_submit(S, ids[m], rhs[m][k], tol=tol,
                                         precision=fs.FESPMV_CG_F32_REFINE, flags=fs.FESPMV_CG_RELIABLE))
        # a drain window as long as the one-at-a-time arm's, then what still waits is cancelled
        t_end = start + T + DRAIN
        while time.perf_counter() < t_end and fs.srv_get_stats(S)["queued"] > 0:
            time.sleep(0.005)
        fs.srv_cancel_queued(S)
        lat, served = [], 0
        for t in tickets:
            rc, _, res, tm = fs.srv_poll(S, t, 0)
            if rc == 0:
                served += 1
                lat.append(tm["t_total_s"])
        elapsed = time.perf_counter() - start
        st = fs.srv_get_stats(S)
        fs.srv_destroy(S)
        out = summarize(trace, lat, served, elapsed)
        out.update({"peak_active": st["peak_active"],
                    "peak_workspace_gb": round(st["peak_workspace_bytes"] / 2 ** 30, 2)})
        return out

    def run_single(trace):
        """One-at-a-time FP64 cg_solve, FIFO, on the same arrivals (host vectors)."""
        lat, served = [], 0
        start = time.perf_counter()
        for (a, m, tol, k) in trace:
            now = time.perf_counter() - start
            if now >= T + DRAIN:
                break
            if now < a:
                time.sleep(a - now)
            x = np.zeros(sizes[m])
            res = fs.cg_solve(mats[m], rhs[m][k], x, tol=tol)
            if res["status"] == 0:
                served += 1
                lat.append(time.perf_counter() - start - a)
        elapsed = time.perf_counter() - start
        return summarize(trace, lat, served, elapsed)

    def three_arms(rate, seed):
        tr = make_trace(rate, seed)
        return {"rate_per_s": round(rate, 1), "offered": len(tr), "server": run_server(tr),
                "server_grouped": run_server(tr, -1), "one_at_a_time": run_single(tr)}

    # warm: graphs and workspaces of every matrix, one solve each on every path
    run_server([(0.0, m, 1e-8, 0) for m in range(n_mesh)], -1)
    for m in range(n_mesh):
        fs.cg_solve(mats[m], rhs[m][0], np.zeros(sizes[m]), tol=1e-8)
    over = three_arms(args.serve_rate, 1506)
    sat = max(1.0, over["server_grouped"]["solves_per_s"])
    single_cap = max(1.0, over["one_at_a_time"]["solves_per_s"])
    rates = [f * single_cap for f in (0.5, 1.0, 1.5)] + \
        [f * sat for f in (float(v) for v in args.serve_sweep.split(",") if v)]
    sweep = [three_arms(r, 1507 + i) for i, r in enumerate(rates)]
    for A in mats:
        fs.spmv_destroy(A)
    return {"pool": pool_info, "seconds_per_run": T,
            "arms": {"server": "continuous batching, FP32 values + FP64 reliable updates",
                     "server_grouped": "the same with lockstep multi-RHS groups per matrix (srv_set_grouping -1)",
                     "one_at_a_time": "FP64 cg_solve per request, FIFO"},
            "saturation_per_s": round(sat, 1), "one_at_a_time_capacity_per_s": round(single_cap, 1),
            "overload": over, "sweep": sweep}


def bench_shell(fs, torch, args):
    """The heart-like shell Laplacian (24 x 256 x 512 nodes, 3.1M rows, ~15 entries per row,
    fibre-rotated 9:1 conductivity): FP64 and BF16/FP32 products of the tiled layout, and
    CG to 1e-10 in FP64 and with BF16 / FP32 values inside FP64 refinement."""
    import fegen
    t0 = time.perf_counter()
    p = fegen.shell_laplace(24, 256, 512, 1503)
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    A = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 1, sigma=1024,
                       precisions=fs.FESPMV_PREC_F32 | fs.FESPMV_PREC_BF16)
    create_s = time.perf_counter() - t0
    n, nnz = p.n_rows, p.nnz
    x = torch.rand(n, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    xs, ys = x.float(), torch.empty(n, dtype=torch.float32, device="cuda")

    def per_launch(fn, k=20):
        fn()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(k):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / k * 1e-3

    t64 = per_launch(lambda: fs.spmv_apply(A, x, y, fs.FESPMV_IO_PERMUTED))
    t32 = per_launch(lambda: fs.spmv_apply_scaled(A, xs, ys, fs.FESPMV_PREC_F32, fs.FESPMV_IO_PERMUTED))
    t16 = per_launch(lambda: fs.spmv_apply_scaled(A, xs, ys, fs.FESPMV_PREC_BF16, fs.FESPMV_IO_PERMUTED))
    out = {"rows": n, "nnz": nnz, "gen_s": round(gen_s, 1), "create_s": round(create_s, 1),
           "n_tiles": fs.spmv_get_info(A)["n_tiles"],
           "f64_spmv_gbs": round((nnz * 12 + n * 16) / t64 / 1e9, 1),
           "f32_spmv_gbs": round((nnz * 8 + n * 8) / t32 / 1e9, 1),
           "bf16_spmv_gbs": round((nnz * 6 + n * 8) / t16 / 1e9, 1)}
    for name, prec, fl in (("cg_f64", fs.FESPMV_CG_F64, 0), ("cg_f32_refine", fs.FESPMV_CG_F32_REFINE, 0),
                           ("cg_f32_reliable", fs.FESPMV_CG_F32_REFINE, fs.FESPMV_CG_RELIABLE),
                           ("cg_bf16_reliable", fs.FESPMV_CG_BF16_REFINE, fs.FESPMV_CG_RELIABLE),
                           ("cg_bf16_flexible", fs.FESPMV_CG_BF16_REFINE, fs.FESPMV_CG_FLEXIBLE)):
        out[name] = bench_cg(fs, torch, A, p, 2, prec, flags=fl)
    fs.spmv_destroy(A)
    return out


def bench_batched(fs, torch, args):
    """Many independent cube Laplacians (node counts log-uniform in [1k, 200k]) solved
    together by batch_cg_solve (FP32 inner CG, FP64 refinement, tol 1e-10), against
    the same problems solved one after another with cg_solve (FP32-refined, and FP64)."""
    import fegen
    rng = np.random.default_rng(2000)
    sizes = np.exp(rng.uniform(np.log(1e3), np.log(2e5), size=args.batch_meshes))
    t0 = time.perf_counter()
    ps = [fegen.valid_seed(lambda sd: fegen.cube_laplace(max(3, round(N ** (1 / 3))), sd), 2000 + i)
          for i, N in enumerate(sizes)]
    gen_s = time.perf_counter() - t0
    # rows-per-warp (K2 threshold), vector width and block from the autotuner, run with the
    # batch's kernels (x gathered from cache, no tiles; FP32 products, those of the solve) on
    # the block-diagonal matrix of the eight largest meshes: large enough that the
    # candidates differ by more than the launch noise
    tune = fs.spmv_autotune(*block_diagonal(sorted(ps, key=lambda q: -q.n_rows)[:8]), 1, sigma=1024,
                            reps=20, tiles=-1, precisions=fs.FESPMV_PREC_F32)
    t0 = time.perf_counter()
    B = fs.batch_create([(p.rowptr, p.colind, p.values, p.node_xyz, 1) for p in ps], sigma=1024,
                        vec=tune["vec"], threshold=tune["threshold"], block=tune["block"])
    create_s = time.perf_counter() - t0
    bs = [fegen.random_vector(p.n_rows, 5000 + j) for j, p in enumerate(ps)]
    bd = torch.from_numpy(np.concatenate(bs)).cuda()
    xd = torch.zeros_like(bd)
    def batch_time(flags):
        fs.batch_cg_solve(B, bd, xd, tol=1e-10, flags=flags)            # warm: graph capture
        torch.cuda.synchronize()
        times = []
        for _ in range(3):
            xd.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc, res = fs.batch_cg_solve(B, bd, xd, tol=1e-10, flags=flags)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        assert rc == 0
        return min(times), res

    batch_rel_s, res_rel = batch_time(fs.FESPMV_CG_RELIABLE)
    batch_s, res = batch_time(0)
    # the batch's roofline: every problem's inner steps times the algorithmic bytes of one
    # FP32 product of it (values + int32 indices, float x and y), over the batch's time
    alg = sum(r["iters"] * (p.nnz * 8 + p.n_rows * 8) for r, p in zip(res_rel, ps))
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    roof = {"bound": "hbm", "achieved": round(alg / batch_rel_s / 1e9, 1), "peak": peak, "unit": "GB/s",
            "frac": round(alg / batch_rel_s / 1e9 / peak, 4),
            "note": "sum over problems of inner steps x (nnz x 8 + n x 8) bytes / batch time; the FP64 "
                    "residual products of the reliable updates are not counted"}
    info = fs.batch_get_info(B)
    fs.batch_destroy(B)
    seq = {}
    for name, prec, fl in (("f32_reliable", fs.FESPMV_CG_F32_REFINE, fs.FESPMV_CG_RELIABLE),
                           ("f32_refine", fs.FESPMV_CG_F32_REFINE, 0), ("f64", fs.FESPMV_CG_F64, 0)):
        mats = [fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 1, sigma=1024,
                               precisions=fs.FESPMV_PREC_F32) for p in ps]
        bds = [torch.from_numpy(b).cuda() for b in bs]
        xs = [torch.zeros_like(b) for b in bds]
        for A, b, x in zip(mats, bds, xs):              # warm: graphs per handle
            fs.cg_solve(A, b, x, tol=1e-10, precision=prec, flags=fl)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for A, b, x in zip(mats, bds, xs):
            x.zero_()
            fs.cg_solve(A, b, x, tol=1e-10, precision=prec, flags=fl)
        torch.cuda.synchronize()
        seq[name] = round(time.perf_counter() - t0, 4)
        for A in mats:
            fs.spmv_destroy(A)
    return {"meshes": len(ps), "rows_total": info["n_rows"], "padded_rows": info["padded_rows"],
            "autotune": {k: tune[k] for k in ("vec", "threshold", "block", "best_us", "tried")},
            "nnz_total": info["nnz"], "gen_s": round(gen_s, 1), "create_s": round(create_s, 1),
            "batched_reliable_s": round(batch_rel_s, 4),
            "solver": "reliable updates: one launch of thread-block clusters (8 CTAs), each cluster "
                      "solving whole problems largest first; restarted refinement: lockstep graphs",
            "roofline": roof,
            "solves_per_s": round(len(ps) / batch_rel_s, 1),
            "max_updates": max(r["outer"] for r in res_rel), "max_iters": max(r["iters"] for r in res_rel),
            "batched_restarted_s": round(batch_s, 4),
            "restarted_max_outer": max(r["outer"] for r in res),
            "restarted_max_inner_iters": max(r["iters"] for r in res),
            "one_after_another_s": seq,
            "speedup_vs_sequential_f32_reliable": round(seq["f32_reliable"] / batch_rel_s, 2),
            "speedup_vs_sequential_f64": round(seq["f64"] / batch_rel_s, 2)}


def profile_piece(fs, torch, A, p, xp, args):
    """Warm-up then `steps` launches of one piece, for ncu launch lists and captures.
    The multi-RHS and FP32 pieces run on the extras' handle (vector width
    --extras-vec), the CG pieces on the headline handle, as in the timed run."""
    n = p.n_rows
    t = args.profile_target
    if t in ("multi", "multi64", "fp32", "cg_multi", "nb_fp32", "nb_multi", "nb_cg_multi"):
        A = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 3, sigma=args.sigma,
                           vec=args.extras_vec, precisions=fs.FESPMV_PREC_F32,
                           node_blocks=3 if t.startswith("nb_") else 0)
        xp = torch.rand_like(xp)          # any x in this handle's numbering
    if t == "batch":
        # the 256-cube batch of the bench, one reliable-update solve per run
        import fegen
        rng = np.random.default_rng(2000)
        sizes = np.exp(rng.uniform(np.log(1e3), np.log(2e5), size=args.batch_meshes))
        ps = [fegen.valid_seed(lambda sd: fegen.cube_laplace(max(3, round(N ** (1 / 3))), sd), 2000 + i)
              for i, N in enumerate(sizes)]
        Bt = fs.batch_create([(q.rowptr, q.colind, q.values, q.node_xyz, 1) for q in ps], sigma=1024)
        bd = torch.from_numpy(np.concatenate([fegen.random_vector(q.n_rows, 5000 + j)
                                              for j, q in enumerate(ps)])).cuda()
        xb = torch.zeros_like(bd)
        f = lambda: fs.batch_cg_solve(Bt, bd, xb, tol=1e-10, flags=fs.FESPMV_CG_RELIABLE)  # noqa: E731
    elif t == "nb_fp32":
        xs = xp.float()
        ys = torch.empty_like(xs)
        f = lambda: fs.spmv_apply_scaled(A, xs, ys, fs.FESPMV_PREC_F32, fs.FESPMV_IO_PERMUTED)  # noqa: E731
    elif t == "nb_multi":
        X = torch.rand((n, 32), dtype=torch.float32, device="cuda")
        Y = torch.empty_like(X)
        f = lambda: fs.spmv_apply_multi(A, X, Y, fs.FESPMV_PREC_F32, fs.FESPMV_IO_PERMUTED)  # noqa: E731
    elif t == "multi":
        X = torch.rand((n, 32), dtype=torch.float32, device="cuda")
        Y = torch.empty_like(X)
        f = lambda: fs.spmv_apply_multi(A, X, Y, fs.FESPMV_PREC_F32, fs.FESPMV_IO_PERMUTED)  # noqa: E731
    elif t == "multi64":
        X = torch.rand((n, 32), dtype=torch.float64, device="cuda")
        Y = torch.empty_like(X)
        f = lambda: fs.spmv_apply_multi(A, X, Y, fs.FESPMV_PREC_F64, fs.FESPMV_IO_PERMUTED)  # noqa: E731
    elif t == "assembly":
        # the workload's element matrices summed into A's values (assembly as a sparse product)
        import fegen
        q = fegen.cube_elasticity(64, 1502, elements=True)
        P = fs.assembly_create(A, q.rowptr, q.colind, q.elem_nodes, 3, q.dirichlet)
        Ke = torch.from_numpy(q.elem_mats).cuda()
        f = lambda: fs.assembly_matrix(P, Ke)  # noqa: E731
    elif t in ("cg_multi", "nb_cg_multi"):
        B = torch.rand((n, 32), dtype=torch.float64, device="cuda")
        X = torch.zeros_like(B)
        # 48 inner iterations (three graphs of 16) of the 32-RHS FP32 CG with reliable updates
        f = lambda: fs.cg_solve_multi(A, B, X, tol=1e-30, max_iter=48,  # noqa: E731
                                      precision=fs.FESPMV_CG_F32_REFINE, flags=fs.FESPMV_CG_RELIABLE)
    elif t == "fp32":
        xs = xp.float()
        ys = torch.empty_like(xs)
        f = lambda: fs.spmv_apply_scaled(A, xs, ys, fs.FESPMV_PREC_F32, fs.FESPMV_IO_PERMUTED)  # noqa: E731
    else:
        b = torch.rand(n, dtype=torch.float64, device="cuda")
        x = torch.zeros_like(b)
        prec = fs.FESPMV_CG_F64 if t == "cg" else fs.FESPMV_CG_F32_REFINE
        f = lambda: fs.cg_solve(A, b, x, tol=1e-30, max_iter=32, max_restarts=-1, max_outer=1,  # noqa: E731
                                precision=prec)
    for _ in range(args.warmup):
        f()
    torch.cuda.synchronize()
    for _ in range(args.steps):
        f()
    torch.cuda.synchronize()
    print(f"profile target {t}: {args.steps} runs done", flush=True)


def bench_cg(fs, torch, A, p, n_solves, precision, flags=0):
    """CG solves to 1e-10 on the same matrix (b = A u*, u* manufactured)."""
    import fegen
    u = fegen.manufactured_solution(p)
    ud = torch.from_numpy(u).cuda()
    bd = torch.empty_like(ud)
    fs.spmv_apply(A, ud, bd)
    lat, iters, outer, rel = [], [], [], []
    name = {0: "f64", 1: "f32_refine", 2: "bf16_refine"}[precision]
    warm = fs.cg_solve(A, bd, torch.zeros_like(bd), tol=1e-10, precision=precision, flags=flags)  # graphs
    if warm["status"] != 0:   # e.g. BF16 refinement stagnating: cond(B) * 2^-8 >= 1
        return {"precision": name, "tol": 1e-10, "status": fs.status_string(warm["status"]),
                "iters": warm["iters"], "outer": warm["outer"], "true_relres": warm["true_relres"]}
    for _ in range(n_solves):
        xs = torch.zeros_like(bd)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = fs.cg_solve(A, bd, xs, tol=1e-10, precision=precision, flags=flags)
        torch.cuda.synchronize()
        lat.append(time.perf_counter() - t0)
        iters.append(res["iters"])
        outer.append(res["outer"])
        rel.append(res["true_relres"])
        assert res["status"] == 0, res
    lat_ms = sorted(1e3 * t for t in lat)
    return {"precision": name, "tol": 1e-10,
            "variant": ("single_reduction" if flags & fs.FESPMV_CG_SINGLE_REDUCTION else
                        "reliable_updates" if flags & fs.FESPMV_CG_RELIABLE else
                        "flexible_cg_8_inner_steps" if flags & fs.FESPMV_CG_FLEXIBLE else
                        "restarted_refinement" if precision else "textbook"),
            "solves": n_solves, "outer": outer[0], "true_relres_max": max(rel),
            "solves_per_s": round(n_solves / sum(lat), 3),
            "p50_ms": round(float(np.percentile(lat_ms, 50)), 2),
            "p99_ms": round(float(np.percentile(lat_ms, 99)), 2),
            "iters": iters}


def block_diagonal(ps):
    """(rowptr, colind, values, node_xyz) of the block-diagonal matrix of the scalar problems
    ps, each mesh's nodes shifted apart so that a locality order keeps the meshes apart."""
    rps, cis, vas, xyz, r0, c0 = [np.zeros(1, dtype=np.int64)], [], [], [], 0, 0
    for i, q in enumerate(ps):
        rps.append(q.rowptr[1:] + r0)
        cis.append(q.colind + c0)
        vas.append(q.values)
        xyz.append(q.node_xyz + np.array([2.0 * i, 0.0, 0.0]))
        r0 += q.nnz
        c0 += q.n_rows
    return (np.concatenate(rps), np.concatenate(cis).astype(np.int32), np.concatenate(vas),
            np.concatenate(xyz))


def bench_cg_multi(fs, torch, p, args):
    """32 right-hand sides of the same matrix solved to 1e-10 in lockstep
    (cg_solve_multi): FP32 values with FP64 reliable updates, their products on 3x3
    node blocks (timed over a few solves after a warm-up that builds the graphs),
    and FP64 (one solve) -- on a handle that keeps float pairs, so that every FP64
    product of both solves runs on the FP32 pipe (within the FP64 bound)."""
    import fegen
    E = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 3, sigma=args.sigma, vec=args.extras_vec,
                       node_blocks=3, precisions=fs.FESPMV_PREC_F32 | fs.FESPMV_PREC_DF64)
    k = 32
    B = np.stack([fegen.random_vector(p.n_rows, 1700 + j) for j in range(k)], axis=1)
    B[:, 0] = manufactured_rhs(fs, torch, E, p)
    Bd = torch.from_numpy(B).cuda()
    out = {}
    for name, precision, flags, reps in (("f32_reliable", fs.FESPMV_CG_F32_REFINE, fs.FESPMV_CG_RELIABLE,
                                          args.cg_solves), ("f64_float_pair_products", fs.FESPMV_CG_F64, 0, 1)):
        if reps > 1:
            fs.cg_solve_multi(E, Bd, torch.zeros_like(Bd), tol=1e-10, precision=precision, flags=flags)
        lat = []
        for _ in range(reps):
            Xd = torch.zeros_like(Bd)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc, res = fs.cg_solve_multi(E, Bd, Xd, tol=1e-10, precision=precision, flags=flags)
            torch.cuda.synchronize()
            lat.append(time.perf_counter() - t0)
            assert rc == 0, [r for r in res if r["status"] != 0][:2]
        iters = [r["iters"] for r in res]
        t = float(np.median(lat))
        out[name] = {"rhs": k, "tol": 1e-10, "solves_per_s": round(k / t, 2),
                     "ms_per_32_solves": round(t * 1e3, 1),
                     "us_per_iteration_all_rhs": round(t * 1e6 / max(iters), 1),
                     "iters_max": max(iters), "iters_min": min(iters),
                     "true_relres_max": max(r["true_relres"] for r in res),
                     "repeats": reps}
    fs.spmv_destroy(E)
    return out


def bench_assembly(fs, torch, args, back_to_back):
    """Assembly as a sparse product (Sec. 4) of the workload matrix from its 1.5 M
    element matrices (12 x 12) into the headline layout, against refreshing the same
    handle from host-assembled CSR-order values already on the device
    (spmv_update_values: the value map of the reordering) -- both calls also rebuild
    the diagonal, S and the FP32/BF16 copies."""
    import fegen
    t0 = time.perf_counter()
    p = fegen.cube_elasticity(64, 1502, elements=True)
    gen_s = time.perf_counter() - t0
    A = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 3, sigma=args.sigma, vec=args.vec,
                       threshold=args.threshold, block=args.block, tiles=args.tiles,
                       precisions=fs.FESPMV_PREC_F32 | fs.FESPMV_PREC_BF16)
    t0 = time.perf_counter()
    P = fs.assembly_create(A, p.rowptr, p.colind, p.elem_nodes, 3, p.dirichlet)
    plan_s = time.perf_counter() - t0
    info = fs.assembly_get_info(P)
    Ke = torch.from_numpy(p.elem_mats).cuda()
    vals = torch.from_numpy(p.values).cuda()
    fa = lambda: fs.assembly_matrix(P, Ke)  # noqa: E731
    fu = lambda: fs.spmv_update_values(A, vals)  # noqa: E731
    fa()
    fu()
    k = max(10, args.steps // 10)
    ta = back_to_back(fa, k) * 1e-3
    tu = back_to_back(fu, k) * 1e-3
    fa()
    torch.cuda.synchronize()
    ok = np.array_equal(fs.spmv_export(A, fs.FESPMV_EXPORT_VALUES).view(np.uint64),
                        fs.spmv_export(fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 3,
                                                      sigma=args.sigma, vec=args.vec, threshold=args.threshold,
                                                      block=args.block, tiles=args.tiles),
                                       fs.FESPMV_EXPORT_VALUES).view(np.uint64))
    newton = newton_steps(fs, torch, p, A, P, Ke)
    sl = fs.spmv_get_info(A)["packed_len"]
    nc = info["contributions"]
    out = {"elements": p.n_elems, "element_matrix": "12 x 12", "contributions": nc,
           "value_positions": sl, "plan_s": round(plan_s, 2), "gen_s": round(gen_s, 1),
           "assembly_us": round(ta * 1e6, 1),
           "assembly_gbs": round((nc * 12 + sl * 16) / ta / 1e9, 1),
           "update_values_us": round(tu * 1e6, 1),
           "bitwise_equal_to_csr_handle": bool(ok),
           "newton_steps_fe_newton_step": newton,
           "bytes_note": "assembly_gbs counts element-matrix reads and 4-byte indices per contribution, "
                         "offsets and the value write per position"}
    del Ke, vals
    fs.assembly_destroy(P)
    fs.spmv_destroy(A)
    return out


def newton_steps(fs, torch, p, A, P, Ke, steps=4):
    """A Newton-like sequence on a fixed pattern (the loop of Sec. 2) through the
    library's fe_newton_step: every step assembles new values and a new right-hand
    side on the GPU from element quantities (here the element matrices scaled by
    1 + 0.05 k and the element vectors K_e u_k of a slowly varying field u_k), then
    solves K dx = R to 1e-10 (FP32 values with FP64 reliable updates) warm-started
    from the previous step's dx, against the same solve started from zero."""
    import fegen
    dpn = p.dofs_per_node
    idx = torch.from_numpy((dpn * p.elem_nodes[:, :, None] + np.arange(dpn)[None, None, :])
                           .reshape(p.n_elems, -1).astype(np.int64)).cuda()
    u0 = torch.from_numpy(fegen.manufactured_solution(p)).cuda()
    du = torch.from_numpy(fegen.random_vector(p.n_rows, 1790)).cuda() * 1e-3
    mask = torch.from_numpy(p.dirichlet.astype(bool)).cuda()
    R = torch.empty_like(u0)
    dx = torch.zeros_like(u0)
    rows = []
    for k in range(steps):
        Kk = Ke * (1.0 + 0.05 * k)
        uk = (u0 + k * du).masked_fill(mask, 0.0)
        Rk = torch.einsum("eij,ej->ei", Kk, uk[idx]).contiguous()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rw = fs.fe_newton_step(P, Kk, Rk, R, dx, None, tol=1e-10, precision=fs.FESPMV_CG_F32_REFINE,
                               flags=fs.FESPMV_CG_RELIABLE | (fs.FESPMV_CG_X0 if k > 0 else 0))
        torch.cuda.synchronize()
        t_step = time.perf_counter() - t0
        dc = torch.zeros_like(u0)
        rc = fs.fe_newton_step(P, Kk, Rk, R, dc, None, tol=1e-10, precision=fs.FESPMV_CG_F32_REFINE,
                               flags=fs.FESPMV_CG_RELIABLE)
        rows.append({"step": k, "step_ms": round(t_step * 1e3, 2),
                     "iters_warm": rw["last_cg"]["iters"], "iters_cold": rc["last_cg"]["iters"],
                     "true_relres": rw["last_cg"]["true_relres"], "status": rw["status"]})
        del Kk, Rk
    return rows


def bench_ablation(fs, torch, args, back_to_back):
    """What each step of the layout buys (the paper's ablation, Sec. 7), FP64 products
    on the 64^3 elasticity and the shell matrices: CSR baselines, then warp slices in
    the generator's (random) node numbering without and with the paper's global length
    sort, Morton locality order, windowed sort, and x staged per tile with 16-bit
    indices.  Each line: algorithmic GB/s of the product, the host planning time and
    the value refresh (spmv_update_values) in products: the reordering cost alpha of
    Sec. 6."""
    import fegen
    out = {}
    CSR, NONE, MORTON = fs.FESPMV_FMT_CSR, fs.FESPMV_REORDER_NONE, fs.FESPMV_REORDER_MORTON
    for wname, maker in (("cube_elasticity_64", lambda: fegen.cube_elasticity(64, 1502)),
                         ("shell_24x256x512", lambda: fegen.shell_laplace(24, 256, 512, 1503))):
        p = maker()
        n, nnz = p.n_rows, p.nnz
        mb = nnz * 12 + n * 16
        vals = torch.from_numpy(p.values).cuda()
        x = torch.from_numpy(fegen.random_vector(n, 1791)).cuda()
        variants = [
            ("csr_scalar", dict(format=CSR, csr_lanes=1)),
            ("csr_vector4", dict(format=CSR, csr_lanes=4)),
            ("slices, generator numbering, no sort", dict(reorder=NONE, sigma=0, tiles=-1, vec=1)),
            ("slices, generator numbering, global length sort", dict(reorder=NONE, sigma=n, tiles=-1, vec=1)),
            ("slices, Morton order, no sort", dict(reorder=MORTON, sigma=0, tiles=-1, vec=1)),
            ("slices, Morton order, sort windows of 1024", dict(reorder=MORTON, sigma=1024, tiles=-1, vec=1)),
            ("K1: input column numbers (y through P^-1), Morton, windows, x from cache",
             dict(reorder=MORTON, sigma=1024, tiles=-1, vec=1, col_order=fs.FESPMV_COLS_ORIGINAL)),
            ("K1r: renumbered, unsorted columns, Morton, windows, x from cache",
             dict(reorder=MORTON, sigma=1024, tiles=-1, vec=1, col_order=fs.FESPMV_COLS_RENUMBERED)),
            ("K1rs: renumbered, sorted columns, Morton, windows, x from cache (as two lines up)",
             dict(reorder=MORTON, sigma=1024, tiles=-1, vec=1)),
            ("K1r + x staged per tile, 16-bit indices",
             dict(reorder=MORTON, sigma=1024, vec=1, col_order=fs.FESPMV_COLS_RENUMBERED)),
            ("+ x staged per tile, 16-bit indices (K1rs: the headline layout)", dict(reorder=MORTON, sigma=1024, vec=1)),
        ]
        rows = []
        for name, kw in variants:
            t0 = time.perf_counter()
            A = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, p.dofs_per_node, **kw)
            create_s = time.perf_counter() - t0
            sliced = kw.get("format", fs.FESPMV_FMT_SLICED) != CSR
            k1 = kw.get("col_order", 0) == fs.FESPMV_COLS_ORIGINAL
            xp = torch.empty_like(x)
            if sliced and not k1:
                fs.spmv_permute(A, x, xp, 0)
            else:
                xp.copy_(x)
            yp = torch.empty_like(x)
            flags = fs.FESPMV_IO_PERMUTED if sliced and not k1 else 0
            fa = lambda: fs.spmv_apply(A, xp, yp, flags)  # noqa: E731
            fi = lambda: fs.spmv_apply(A, x, yp, 0)  # noqa: E731
            fu = lambda: fs.spmv_update_values(A, vals)  # noqa: E731
            fa()
            fi()
            fu()
            ta = back_to_back(fa, max(20, args.steps // 4))
            ti = back_to_back(fi, max(20, args.steps // 4))
            tu = back_to_back(fu, 10)
            info = fs.spmv_get_info(A)
            rows.append({"variant": name, "gbs": round(mb / (ta * 1e-3) / 1e9, 1), "us": round(ta * 1e3, 1),
                         "gbs_input_numbering": round(mb / (ti * 1e-3) / 1e9, 1),
                         "gbs_includes_y_remap": k1,
                         "padding": round(info["packed_len"] / nnz - 1.0, 4) if sliced else 0.0,
                         "tiles": info["n_tiles"], "plan_s": round(create_s, 2),
                         "refresh_products": round(tu / ta, 2)})
            fs.spmv_destroy(A)
        out[wname] = {"rows": n, "nnz": nnz, "variants": rows}
        del vals
    return out


def manufactured_rhs(fs, torch, A, p):
    """b = A u* for the manufactured u*, computed by the library's own FP64 product."""
    import fegen
    ud = torch.from_numpy(fegen.manufactured_solution(p)).cuda()
    bd = torch.empty_like(ud)
    fs.spmv_apply(A, ud, bd)
    return bd.cpu().numpy()


if __name__ == "__main__":
    main()
