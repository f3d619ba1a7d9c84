#!/usr/bin/env python3
"""Benchmark of the omega-FQ block solve on GB300 (one JSON line on rank 0).

Workload (default "cnt20k"): armchair (10,10) carbon nanotube, 500 unit cells,
N = 20,000 atoms; 64 frequencies evenly over 0.05-2.0 eV x 3 field directions =
192 (omega, direction) solves per step, run as ONE launch of the default solver,
shifted GMRES: one real Arnoldi process per field direction serves all 64
frequencies (double-float D products from the FP32 pair planes, FP64 basis,
per-frequency Givens), every column's FP64 true residual checked to 1e-8, then the
polarizability.  `--solver gmres` runs the block form instead: the 192 columns as
one mixed-precision GMRES(50) (3xBF16 tensor-core D products, complex64 basis) with
FP64 iterative refinement; the JSON line also carries that solver's figure
("other_solvers").

A step = one pass of the whole solve path over the 192 columns (RHS, Krylov
iterations with the operator apply, FP64 residuals, alpha).  The geometry (D as
FP64, bf16 planes and FP32 pair planes, Kbar CSR) is built once before the timed
region for `value`; the `e2e` figure rebuilds it every step from host coordinates
and returns q and alpha to host memory through the C ABI.

Metric: freq-point solves/s -- (omega, direction) solves per second that reach
relative residual <= 1e-8 (FP64, every column) and alpha within 1e-6 of the FP64
oracle (sampled columns, checked by the cpu_baseline leg).

--impl reference times the FP64 CPU oracle (oracle/) on the host cores on a bounded
sample of the same workload (one column per step).
"""
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

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cnt20k")
    ap.add_argument("--solver", default="shifted", choices=["shifted", "gmres", "qmr"])
    ap.add_argument("--no-other-solvers", action="store_true")
    ap.add_argument("--other-solvers", default="gmres",
                    help="comma list of block solvers timed beside the shifted one (gmres, qmr)")
    ap.add_argument("--store", default=None,
                    help="comma list of D storages overriding the workload's (fp64, bf16, f32x2, sym)")
    ap.add_argument("--m", type=int, default=50)
    ap.add_argument("--other-warmup", type=int, default=None,
                    help="untimed solves of each other solver form before its timed one (default: min(2, warmup))")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-other-configs", action="store_true",
                    help="default cnt20k line: skip the other configurations' figures")
    ap.add_argument("--cpu-budget-s", type=float, default=25.0)
    ap.add_argument("--mode", default=None, choices=["solve", "apply", "serve", "spectrum"],
                    help="solve: block solves per second (default); apply: operator applies, "
                         "pair interactions per second (default for disk1m); serve: seeded Poisson "
                         "request stream through the request server (default for workload serve)")
    ap.add_argument("--fmm-order", type=int, default=0,
                    help="D product by the fast multipole method of this order (0: direct): the apply "
                         "mode's product, or the mixed inner products of a matrix-free solve")
    ap.add_argument("--requests", type=int, default=2000, help="serve mode: requests in the stream")
    ap.add_argument("--workers", type=int, default=3, help="serve mode: server worker streams")
    ap.add_argument("--pool", default="small", choices=["small", "full"],
                    help="serve mode: resident structures of 1k-20k atoms, or also the 50k flake, the 80k "
                         "tube and the 100k sphere")
    ap.add_argument("--load", type=float, default=0.8, help="serve mode: arrival rate / measured capacity")
    return ap.parse_args()


# D storage per workload: FP64 + bf16 planes where both fit; bf16 planes only for the 150k
# sphere (FP64 D would be 180 GB); nothing stored for the 1M-atom disk (matrix-free).
def store_for(name, wfq, solver="gmres"):
    if name == "sphere150k" and solver == "shifted":
        return wfq.STORE_F32X2           # the FP32 pair planes alone: 180 GB
    if name == "sphere150k":
        # the symmetric FP32 pair tiles are 90 GB, the bf16 planes 90 GB: both fit
        return wfq.STORE_F32X2_SYM | wfq.STORE_BF16X2
    if name in ("disk1m", "disk100k"):
        return 0
    return wfq.STORE_FP64 | wfq.STORE_BF16X2 | wfq.STORE_F32X2


# DRAM bytes per stored D entry that ncu measured for one k_dgemv_df launch (cnt8k, N = 8200:
# 549.3 MB read + written for 8200 x 8320 stored entries of the FP32 pair planes).
DGEMV_DRAM_BYTES_PER_ENTRY = 549.3e6 / (8200.0 * 8320.0)

# Algorithmic bytes of one block apply of D: the FP32 D (4 bytes per entry) read once.
ALG_BYTES_PER_ENTRY = 4.0

# FP32 lane-instructions per second of the whole GPU: 152 SMs x 128 lanes x 2070 MHz.
FP32_LANE_OPS_PER_S = 152 * 128 * 2.07e9

# Minimum FP32-pipe instructions to generate one D entry as a bf16 hi/lo pair on the
# matrix-free path: 3 coordinate differences, 3 for r^2, 1 for sigma^2, 1 far/near test,
# 1 rsqrt (MUFU), 4 for the split (round, widen, subtract, round).
MF_OPS_PER_PAIR = 13


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return dict(PEAKS_FALLBACK), "fallback"


def workload(name):
    from paper_2103_00438_gb300 import structures as S
    if name == "cnt8k":   # small case for ncu captures: same tube, 205 cells, same block width
        wl = S.workload("cnt20k")
        wl["xyz"] = S.nanotube(10, 10, 205)
        return wl
    if name == "sphere30k":   # the 150k sphere's family and band at 30k atoms (solver comparisons)
        wl = S.workload("sphere150k")
        a = 4.23
        wl["xyz"] = S.fcc_sphere(a, S.fcc_sphere_radius_for(30_000, a), 0.05, seed=20210301)
        return wl
    if name == "disk100k":   # small matrix-free case for ncu captures: same disk family, 18.3 nm
        wl = S.workload("disk1m")
        wl["xyz"] = S.graphene_disk(58.0, vacancy_frac=0.01, seed=20210304)
        return wl
    return S.workload(name)


# ------------------------------------------------------------------ replicas

def max_over_ranks(value, dist):
    """Max of a per-rank float over all ranks (the whole-job time of weak-scaled replicas);
    identity without a process group.  Uses a CUDA tensor under NCCL, a CPU one otherwise."""
    if dist is None:
        return float(value)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle

# Largest N for which the oracle's CPU baseline stores D (8 N^2 bytes of host memory) and
# solves sampled columns outright; above it the baseline is the oracle's row-sampled apply
# throughput, extrapolated to solves/s with the iteration counts of the GPU solve.
ORACLE_STORED_MAX_N = 25000


def oracle_rows_rate(wl, nrows=8):
    """Pair evaluations per second of the oracle's row-sampled apply (one column)."""
    from oracle import oracle as orc
    xyz, p = wl["xyz"], wl["params"]
    n = len(xyz)
    rng = np.random.default_rng(11)
    rows = rng.choice(n, size=nrows, replace=False)
    x = rng.standard_normal(n) + 0j
    t0 = time.perf_counter()
    orc.apply_rows(xyz, p, orc.z_of_omega(wl["omega"][0], p), x, rows)
    secs = time.perf_counter() - t0
    return secs, rows


def oracle_sample(wl, budget_s, cols):
    """Solve sampled columns with the FP64 oracle (stored D, GMRES(50), rel tol 1e-10).
    Returns (solves, seconds, {col: alpha}, cores)."""
    from oracle import oracle as orc
    xyz, p = wl["xyz"], wl["params"]
    ndir = len(wl["dirs"])
    D = orc.d_matrix(xyz, p["eta"])
    csr = orc.kbar_csr(xyz, p)
    op = orc.Operator.stored(D, csr)
    alphas, t_total, solved = {}, 0.0, 0
    for c in cols:
        f, d = divmod(int(c), ndir)
        R = orc.rhs_csr(xyz, csr, wl["dirs"][d]).astype(complex)
        t0 = time.perf_counter()
        q, info = op.gmres(orc.z_of_omega(wl["omega"][f], p), R, restart=50, rel_tol=1e-10, max_iter=20000)
        t_total += time.perf_counter() - t0
        alphas[int(c)] = orc.alpha(xyz, q)
        solved += 1
        if t_total >= budget_s:
            break
    return solved, t_total, alphas, os.cpu_count()


def audit_row_probabilities(R):
    """Row-sampling probabilities of the residual audit: half uniform, half proportional
    to |R_i|^2 (the residual of a Krylov iterate lives where R does -- at edges and
    vacancies -- so sampling there cuts the estimate's variance; the uniform half keeps
    every row reachable, so the estimate stays unbiased whatever the residual's shape)."""
    a2 = np.abs(np.asarray(R)) ** 2
    return 0.5 / len(a2) + 0.5 * a2 / a2.sum()


def sampled_residual_estimate(r_rows, p_rows, r_full_norm, seed=20210308, nboot=2000):
    """||r|| / ||R|| from the residual's rows r_s at rows drawn with replacement with
    probabilities p_s: ||r||^2 ~ mean(|r_s|^2 / p_s) (unbiased), with a 95% bootstrap
    interval (the draws resampled with replacement)."""
    t = np.abs(np.asarray(r_rows)) ** 2 / np.asarray(p_rows)
    est = float(np.sqrt(t.mean()) / r_full_norm)
    rng = np.random.default_rng(seed)
    boot = np.sqrt(t[rng.integers(0, len(t), size=(nboot, len(t)))].mean(axis=1)) / r_full_norm
    lo, hi = np.percentile(boot, [2.5, 97.5])
    return est, float(lo), float(hi)


def is_bem(wl):
    return "surface" in wl


def make_geometry(wfq, ctx, wl, store, xyz=None):
    """The workload's geometry: an omega-FQ structure, or a BEM surface (whose FP64 operator
    is always stored)."""
    if is_bem(wl):
        s = wl["surface"]
        return wfq.BemGeometry(ctx, s["xyz"] if xyz is None else xyz, s["normal"], s["area"], s["curvature"],
                               wl["bem"], store=store | wfq.STORE_FP64)
    return wfq.Geometry(ctx, wl["xyz"] if xyz is None else xyz, wl["params"], store=store)


def oracle_sample_bem(wl, budget_s, cols, A=None):
    """BEM workloads: solve sampled columns with the oracle's FP64 GMRES(50) on its dense
    operator (oracle/bem.py; assembly not timed) to rel. residual 1e-10.
    Returns (solves, seconds, {col: alpha}, cores, A)."""
    from oracle import bem as ob
    from oracle import oracle as orc
    s = wl["surface"]
    ndir = len(wl["dirs"])
    if A is None:
        A = ob.a_matrix(s["xyz"], s["normal"], s["area"], s["curvature"])
    op = orc.Operator.dense(A)
    alphas, t_total, solved = {}, 0.0, 0
    for c in cols:
        f, d = divmod(int(c), ndir)
        R = ob.rhs(s["normal"], s["area"], wl["dirs"][d]).astype(complex)
        t0 = time.perf_counter()
        q, info = op.gmres(ob.z_of_omega(wl["omega"][f], wl["bem"]), R, restart=50, rel_tol=1e-10, max_iter=20000)
        t_total += time.perf_counter() - t0
        alphas[int(c)] = ob.alpha(s["xyz"], q)
        solved += 1
        if t_total >= budget_s:
            break
    return solved, t_total, alphas, os.cpu_count(), A


def run_reference(args, rank, world):
    if rank != 0:
        return
    os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count()))
    from oracle import build as ob
    ob.build()
    wl = workload(args.workload)
    ncols = len(wl["omega"]) * len(wl["dirs"])
    rng = np.random.default_rng(20210302)
    order = rng.permutation(ncols)
    per_step = []
    k = 0
    A = None
    for i in range(args.warmup + args.steps):
        if is_bem(wl):
            solved, secs, _, cores, A = oracle_sample_bem(wl, args.cpu_budget_s, [order[k % ncols]], A)
        else:
            solved, secs, _, cores = oracle_sample(wl, args.cpu_budget_s, [order[k % ncols]])
        k += 1
        if i >= args.warmup:
            per_step.append(secs / max(solved, 1))
    t = float(np.mean(per_step))
    val = 1.0 / t
    out = {"impl": "reference", "metric": "freq-point solves/s", "value": val, "unit": "solves/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": args.workload, "n_atoms": len(wl["xyz"]),
                                             "columns": ncols},
           "cpu_baseline": {"value": val, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
                            "sample": "one (omega, direction) column per step, FP64 GMRES(50) on the stored "
                                      "%s to rel. residual 1e-10" % ("dense BEM operator" if is_bem(wl) else "D")},
           "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ GPU arm

def run_ours(args, rank, world, dist):
    import torch
    from paper_2103_00438_gb300 import wfq

    if args.mode == "serve" or args.workload == "serve":
        return run_serve(args, rank, world, dist)
    if args.mode == "spectrum":
        return run_spectrum(args, rank, world, dist)
    if args.workload.startswith("bem_"):
        return run_bem(args, rank, world, dist)
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    wl = workload(args.workload)
    xyz, p, om, dirs = wl["xyz"], wl["params"], wl["omega"], wl["dirs"]
    n, nf, nd = len(xyz), len(om), len(dirs)
    ncols = nf * nd
    ctx = wfq.Context(local)
    store = store_for(args.workload, wfq, args.solver)
    if args.store:
        flags = {"fp64": wfq.STORE_FP64, "bf16": wfq.STORE_BF16X2, "f32x2": wfq.STORE_F32X2,
                 "sym": wfq.STORE_F32X2_SYM}
        store = 0
        for f in args.store.split(","):
            store |= flags[f.strip()]
    g = wfq.Geometry(ctx, xyz, p, store=store)
    mode = args.mode or ("apply" if args.workload in ("disk1m", "disk100k") else "solve")
    if args.fmm_order and mode == "solve":
        g.fmm_build(args.fmm_order)     # the mixed inner products of a matrix-free geometry
    if mode == "apply":
        return run_apply(args, rank, world, dist, ctx, g, wl, store)
    stream = torch.cuda.current_stream()
    q = torch.empty((n, ncols), dtype=torch.complex128, device="cuda")

    def solve(out=None):
        out = q if out is None else out
        if args.solver == "gmres":
            return g.solve_gmres(om, dirs, m=args.m, rel_tol=1e-8, max_iter=4000, prec=wfq.PREC_MIXED, out=out,
                                 stream=stream)
        if args.solver == "shifted":
            return g.solve_gmres_shifted(om, dirs, m_max=0, rel_tol=1e-8, max_iter=4000, prec=wfq.PREC_MIXED,
                                         out=out, stream=stream)
        return g.solve_qmr(om, dirs, rel_tol=1e-8, max_iter=4000, prec=wfq.PREC_MIXED, out=out, stream=stream)

    def step():
        _, st, status = solve()
        alpha = g.polarizability(q, stream=stream)
        return st, status, alpha

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ctx.profile(True)
    launches0 = wfq.kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    stats_all, alpha = [], None
    for _ in range(args.steps):
        st, status, alpha = step()
        stats_all.append((st, status))
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    launches = wfq.kernel_launches() - launches0
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    gemm_n, gemm_ms, gemm_flops = ctx.profile_read(wfq.KT_GEMM_MIXED)
    f64_n, f64_ms, _ = ctx.profile_read(wfq.KT_DAPPLY_FP64)
    sp_n, sp_ms, _ = ctx.profile_read(wfq.KT_SPARSE)
    or_n, or_ms, _ = ctx.profile_read(wfq.KT_ORTHO)
    rs_n, rs_ms, _ = ctx.profile_read(wfq.KT_RESIDUAL)
    gv_n, gv_ms, gv_bytes = ctx.profile_read(wfq.KT_DGEMV_DF)
    ctx.profile(False)
    ms = max_over_ranks(ms, dist)

    st_last, status_last = stats_all[-1]
    max_res = max(s["rel_residual"] for st, _ in stats_all for s in st)
    good_cols = sum(1 for s in st_last if s["rel_residual"] <= 1e-8)
    iters = [s["iters"] for s in st_last]
    solves = good_cols * args.steps * world
    value = solves / (ms / 1e3)

    # dominant kernel roofline: the 3xBF16 tensor-core GEMM.  Work per launch is counted by
    # the library from the columns that launch actually carried (the block narrows as
    # columns converge): 6 N^2 C tensor flops (three bf16 products of 2 N^2 C each).
    peaks, peak_src = load_peaks()
    roof = None
    if gv_n and gv_ms >= gemm_ms and store & wfq.STORE_F32X2_SYM and not store & wfq.STORE_F32X2:
        # shifted solver on the symmetric tiles: half of D streamed, each tile used for two
        # products, so the double-float arithmetic bounds it: 12 FP32-pipe instructions per
        # (entry, vector) product, N^2 x ndir products per launch
        avg_s = gv_ms / gv_n * 1e-3
        achieved = 12.0 * n * n * nd / avg_s / 1e12
        peak = FP32_LANE_OPS_PER_S / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "FP32 Tinst/s",
                "frac": achieved / peak, "traffic": None,
                "kernel": "k_dsymv_df + k_dsymv_finish (symmetric double-float D product)", "launches": gv_n,
                "avg_ms": gv_ms / gv_n, "bytes_per_launch": gv_bytes / gv_n,
                "hbm_achieved_gbs": gv_bytes / gv_n / avg_s / 1e9,
                "hbm_frac": gv_bytes / gv_n / avg_s / 1e9 / peaks["hbm_gbs"],
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2070 MHz (one FP32 instruction per lane "
                               "per clock); work: 12 instructions per double-float multiply-add"}
    elif gv_n and gv_ms >= gemm_ms:
        # shifted solver: the dominant kernel is the D product of the Arnoldi vectors.
        # Algorithmic bytes per launch: 4 bytes per D entry (the FP32 D read once per block
        # apply), N^2 entries.  The kernel itself stores D as FP32 pairs (8 bytes per entry
        # for ~2^-48 products); its utilisation of HBM on those stored bytes is reported
        # beside the fraction, under its own name.
        avg_s = gv_ms / gv_n * 1e-3
        alg_bytes = ALG_BYTES_PER_ENTRY * float(n) * float(n)
        achieved_gbs = alg_bytes / avg_s / 1e9
        peak = peaks["hbm_gbs"]
        stored = gv_bytes / gv_n
        roof = {"bound": "hbm", "achieved": achieved_gbs, "peak": peak, "unit": "GB/s",
                "frac": achieved_gbs / peak,
                "traffic": DGEMV_DRAM_BYTES_PER_ENTRY * n * (-(-n // 128) * 128),
                "traffic_source": "ncu dram__bytes_read+write of k_dgemv_df at N = 8200 "
                                  "(the committed profile summary of that kernel), scaled per D entry to this N",
                "kernel": "k_dgemv_df (double-float D product of the real Arnoldi vectors)", "launches": gv_n,
                "avg_ms": gv_ms / gv_n, "algorithmic_bytes_per_launch": alg_bytes,
                "algorithmic_bytes_rule": "4 bytes per D entry x N^2 entries (FP32 D streamed once per block apply)",
                "stored_bytes_per_launch": stored,
                "hbm_util_of_stored_bytes": stored / avg_s / 1e9 / peak,
                "peak_source": peak_src + " hbm_gbs (STREAM-style copy)"}
    elif gemm_n:
        gemm_avg_ms = gemm_ms / gemm_n
        achieved_tflops = gemm_flops / (gemm_ms * 1e-3) / 1e12
        peak = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
        np_ = -(-n // 128) * 128
        roof = {"bound": "tensor", "achieved": achieved_tflops, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved_tflops / peak, "traffic": None,
                "kernel": "gemm_3xbf16 (k_gemm3_tc)", "launches": gemm_n, "avg_ms": gemm_avg_ms,
                "flops_per_launch_mean": gemm_flops / gemm_n,
                "algorithmic_flops_per_launch_mean": gemm_flops / gemm_n / 3.0,
                "hbm_achieved_gbs": 4.0 * np_ * np_ / (gemm_avg_ms * 1e-3) / 1e9,
                "peak_source": peak_src + " bf16_tflops_sustained (kernel timed inside a long step)"}

    out = {"metric": "freq-point solves/s", "value": value, "unit": "solves/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32x2(double-float)+f64" if args.solver == "shifted" else "bf16x3+f32+f64",
           "data": "synthetic",
           "config": {"workload": args.workload, "n_atoms": n, "nfreq": nf, "ndir": nd, "columns": ncols,
                      "solver": {"gmres": f"gmres({args.m})", "qmr": "qmr",
                                 "shifted": "shifted gmres (one real Arnoldi per direction, all frequencies)"}[args.solver],
                      "precision": ("double-float D products (FP32 pair planes), FP64 Arnoldi basis and "
                                    "per-frequency Givens, FP64-accuracy true residual"
                                    if args.solver == "shifted" else
                                    "mixed: 3xBF16 D products, complex64 basis, FP64 refinement"),
                      "rel_tol": 1e-8, "parallelism": f"replicas{world}",
                      "l2": "inputs larger than L2 (%s %.2f GB)" % (
                          ("FP32 pair D planes", 8.0 * n * n / 1e9)
                          if args.solver == "shifted" and store & wfq.STORE_F32X2 else
                          ("symmetric FP32 pair D tiles", 4.0 * n * n / 1e9) if args.solver == "shifted"
                          else ("bf16 D planes", 4.0 * n * n / 1e9))},
           "accuracy": {"max_rel_residual": max_res, "columns_converged": good_cols,
                        "iters_min_mean_max": [min(iters), float(np.mean(iters)), max(iters)],
                        "status": status_last},
           "kernel_ms_per_step": {"gemm_3xbf16": gemm_ms / args.steps, "dapply_fp64": f64_ms / args.steps,
                                  "dgemv_df": gv_ms / args.steps,
                                  "sparse": sp_ms / args.steps, "ortho_phase": or_ms / args.steps,
                                  "residual_phase": rs_ms / args.steps},
           "kernel_launches_per_step": {"gemm_3xbf16": gemm_n / args.steps, "dapply_fp64": f64_n / args.steps,
                                        "dgemv_df": gv_n / args.steps, "sparse": sp_n / args.steps},
           "roofline": roof, "clocks": clk, "gpu_launches": int(launches)}

    # the other solver form on the same workload (same device, not part of `value`)
    if not args.no_other_solvers:
        others = {}
        q_other = torch.empty_like(q)   # q keeps the timed solver's result for the audit below
        names = [x.strip() for x in args.other_solvers.split(",") if x.strip()] + ["shifted"]
        for name in names:
            if name == args.solver:
                continue
            saved = args.solver
            args.solver = name
            ow = min(2, args.warmup) if args.other_warmup is None else args.other_warmup
            for _ in range(max(0, ow)):
                solve(q_other)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, st_o, status_o = solve(q_other)
            e1.record(stream)
            torch.cuda.synchronize()
            args.solver = saved
            t_o = e0.elapsed_time(e1)
            ok_o = sum(1 for x in st_o if x["rel_residual"] <= 1e-8)
            others[{"gmres": f"gmres({args.m}) mixed 3xBF16 + FP64 refinement",
                    "qmr": "J-symmetric qmr mixed 3xBF16 + FP64 refinement",
                    "shifted": "shifted gmres"}[name]] = {
                "value": ok_o / (t_o / 1e3), "unit": "solves/s", "ms_per_step": t_o, "status": status_o,
                "max_rel_residual": max(x["rel_residual"] for x in st_o), "columns_converged": ok_o,
                "iters_mean_max": [float(np.mean([x["iters"] for x in st_o])), max(x["iters"] for x in st_o)]}
        out["other_solvers"] = others

    # end to end through the C ABI with host buffers: geometry from host coordinates,
    # q and alpha back to pinned host memory, every step
    if not args.no_e2e:
        xyz_pin = torch.from_numpy(np.ascontiguousarray(xyz)).pin_memory().numpy()
        q_host = torch.empty((n, ncols), dtype=torch.complex128).pin_memory()
        # the e2e geometry stores only what the timed solver uses (the shifted solver: the FP32
        # pair planes; the block solvers: bf16 planes for the iterations, FP64 D for residuals)
        store_e2e = wfq.STORE_F32X2 if args.solver == "shifted" else store
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ge = wfq.Geometry(ctx, xyz_pin, p, store=store_e2e)
            if args.solver == "shifted":
                ge.solve_gmres_shifted(om, dirs, m_max=0, rel_tol=1e-8, max_iter=4000, prec=wfq.PREC_MIXED,
                                       out=q_host.numpy())
            else:
                ge.solve_gmres(om, dirs, m=args.m, rel_tol=1e-8, max_iter=4000, prec=wfq.PREC_MIXED,
                               out=q_host.numpy())
            ge.polarizability(q_host.numpy())
            ge.close()
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        te = max_over_ranks(te, dist)
        out["e2e"] = {"value": good_cols * args.steps * world / te, "unit": "solves/s",
                      "h2d_bytes_per_step": int(xyz.nbytes + om.nbytes + dirs.nbytes),
                      "d2h_bytes_per_step": int(n * ncols * 16 + ncols * 3 * 16),
                      "includes": "geometry build (Kbar CSR and the D storage the solver uses) from host "
                                  "coordinates, solve, alpha"}

    # CPU baseline (oracle, rank 0, N = 1 only) and accuracy audit of sampled columns
    if rank == 0 and world == 1 and not args.no_cpu_baseline and n > ORACLE_STORED_MAX_N:
        os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count()))
        from oracle import build as ob
        ob.build()
        secs, rows = oracle_rows_rate(wl)
        nbr = g.info()["nnz"] / n
        pairs_per_s = len(rows) * (2.0 + nbr) * n / secs
        mean_it = float(np.mean(iters))
        # residual audit by the oracle on sampled rows: r_i = R_i - ((A - zI) q)_i, each
        # row's neighbours and D entries recomputed by brute force (Eq. 13, Eq. 3, Eq. 17)
        from oracle import oracle as orc
        qh = q.cpu().numpy()
        rng_a = np.random.default_rng(20210307)
        audits = []
        for c in sorted({0, ncols - 1}):
            f, d = divmod(c, nd)
            Rfull = g.rhs(dirs[d:d + 1])[:, 0]
            # 48 rows drawn with replacement, half uniformly, half where R is large; the
            # oracle recomputes each distinct row once
            pr = audit_row_probabilities(Rfull)
            draws = rng_a.choice(n, size=48, replace=True, p=pr)
            audit_rows, inv = np.unique(draws, return_inverse=True)
            Rr = orc.rhs_rows(xyz, p, dirs[d], audit_rows)
            yr, _ = orc.apply_rows(xyz, p, orc.z_of_omega(om[f], p), qh[:, c], audit_rows)
            # ||r|| estimated from the drawn rows over the exact ||R|| (the library's R,
            # which the oracle's R rows confirm)
            r_est, r_lo, r_hi = sampled_residual_estimate((Rr - yr)[inv], pr[draws], np.linalg.norm(Rfull))
            audits.append({"column": int(c), "sampled_rows": len(audit_rows), "draws": len(draws),
                           "rel_residual_estimate_from_sampled_rows": r_est,
                           "estimate_bootstrap_95": [r_lo, r_hi],
                           "R_rows_vs_library": float(np.abs(Rr - Rfull[audit_rows]).max() / np.abs(Rfull).max()),
                           "library_rel_residual": float(st_last[c]["rel_residual"])})
        out["accuracy"]["oracle_residual_audit"] = audits
        out["cpu_baseline"] = {"value": pairs_per_s / (float(n) * n * mean_it), "unit": "solves/s",
                               "cores": os.cpu_count(), "kind": "oracle",
                               "sample": f"extrapolated: oracle row-sampled apply ({len(rows)} rows, D recomputed "
                                         f"from Eq. 3) at {pairs_per_s / 1e9:.3f} Gpairs/s, N^2 pairs per apply, "
                                         f"{mean_it:.1f} applies per solve (mean iterations of this GPU solve)"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline and n <= ORACLE_STORED_MAX_N:
        os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count()))
        from oracle import build as ob
        ob.build()
        rng = np.random.default_rng(20210302)
        cols = rng.permutation(ncols)[:4]
        solved, secs, alphas, cores = oracle_sample(wl, args.cpu_budget_s, cols)
        al_gpu = g.polarizability(q)
        errs = [float(np.abs(al_gpu[c] - a).max() / np.abs(a).max()) for c, a in alphas.items()]
        out["cpu_baseline"] = {"value": solved / secs, "unit": "solves/s", "cores": cores, "kind": "oracle",
                               "sample": f"{solved} sampled (omega, direction) columns of the same workload, "
                                         "FP64 GMRES(50) on stored FP64 D to rel. residual 1e-10 "
                                         "(D assembly not timed)"}
        out["accuracy"]["alpha_rel_err_vs_oracle_sampled"] = max(errs) if errs else None
        out["accuracy"]["alpha_columns_checked"] = sorted(alphas)
    g.close()
    ctx.close()
    if (mode == "solve" and args.workload == "cnt20k" and world == 1 and rank == 0
            and not args.no_other_configs):
        del q
        torch.cuda.empty_cache()
        out["other_configs"] = run_other_configs(args)
    return out


def _summary(o):
    """The figures of a sub-run's JSON line that the default line carries."""
    keep = {"metric", "value", "unit", "ms_per_step", "steps", "warmup", "dtype", "accuracy", "latency",
            "cpu_baseline", "gpu_launches", "other_solvers"}
    out = {k: v for k, v in o.items() if k in keep}
    cfg = o.get("config", {})
    out["config"] = {k: cfg[k] for k in ("workload", "n_atoms", "columns", "requests", "solver", "path",
                                         "arrival_rate_req_per_s") if k in cfg}
    if o.get("roofline"):
        out["roofline"] = {k: v for k, v in o["roofline"].items()
                           if k in ("bound", "achieved", "peak", "unit", "frac", "kernel", "avg_ms",
                                    "hbm_util_of_stored_bytes", "peak_source")}
    if "plain_fp64_gmres_same_gpu" in o:
        pl = o["plain_fp64_gmres_same_gpu"]
        out["plain_fp64_gmres_same_gpu"] = {"value": pl["value"], "unit": pl["unit"],
                                            "served_over_plain": pl["served_over_plain"]}
    if o.get("clocks"):
        out["clocks"] = {k: o["clocks"].get(k) for k in ("sm_mhz", "sm_max_mhz", "reasons")}
    return out


def run_other_configs(args):
    """The other configurations' figures, carried by the default cnt20k line: the 1M-atom
    disk's matrix-free mixed apply (Gint/s against the derived ALU roof, sampled oracle
    rows) and its fast-multipole apply (order 6), a shortened serving stream (p50/p99 latency;
    served over plain per-column FP64 GMRES on the same GPU) and the 150k-atom sphere's
    solver comparison at equal accuracy (96 columns to 1e-8: one shifted-GMRES step from the
    symmetric FP32 pair tiles, then mixed QMR and mixed GMRES(30) on the bf16 planes beside
    them, each timed once).  Each runs in its own context after the cnt20k geometry is
    freed."""
    import torch
    plans = [
        ("disk1m_apply", dict(workload="disk1m", mode="apply", steps=2, warmup=1, no_e2e=True)),
        ("disk1m_fmm_apply", dict(workload="disk1m", mode="apply", fmm_order=6, steps=3, warmup=1, no_e2e=True)),
        ("serve_240_requests", dict(workload="serve", mode="serve", requests=240, warmup=1)),
        ("sphere150k_solvers", dict(workload="sphere150k", mode="solve", solver="shifted", steps=1, warmup=1,
                                    store="sym,bf16", other_solvers="qmr,gmres", m=30, other_warmup=0,
                                    no_e2e=True, no_other_configs=True)),
    ]
    res = {}
    for key, kw in plans:
        sub = argparse.Namespace(**vars(args))
        sub.__dict__.update(kw)
        t0 = time.perf_counter()
        try:
            res[key] = _summary(run_ours(sub, 0, 1, None))
        except Exception as e:     # one failing configuration does not lose the headline line
            res[key] = {"error": repr(e)[:400]}
        res[key]["wall_s"] = time.perf_counter() - t0
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    return res


def run_bem(args, rank, world, dist):
    """The continuum BEM operator of Section 2.3 (Eq. 21-22) through the same shifted
    solver: every (omega, direction) column of the workload in one shifted GMRES solve,
    the operator streamed from its FP32 pair planes (the FP64 copy serves the residuals)."""
    import torch
    from paper_2103_00438_gb300 import wfq

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    wl = workload(args.workload)
    xyz, om, dirs = wl["xyz"], wl["omega"], wl["dirs"]
    n, nf, nd = len(xyz), len(om), len(dirs)
    ncols = nf * nd
    ctx = wfq.Context(local)
    store = wfq.STORE_FP64 | wfq.STORE_F32X2
    g = make_geometry(wfq, ctx, wl, store)
    stream = torch.cuda.current_stream()
    q = torch.empty((n, ncols), dtype=torch.complex128, device="cuda")

    def step():
        _, st, status = g.solve_gmres_shifted(om, dirs, rel_tol=1e-8, max_iter=4000, prec=wfq.PREC_FP64, out=q,
                                              stream=stream)
        return st, status, g.polarizability(q, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ctx.profile(True)
    launches0 = wfq.kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    res = []
    for _ in range(args.steps):
        res.append(step())
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    launches = wfq.kernel_launches() - launches0
    clk = clocks.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1), dist)
    gv_n, gv_ms, gv_bytes = ctx.profile_read(wfq.KT_DGEMV_DF)
    sp_n, sp_ms, _ = ctx.profile_read(wfq.KT_SPARSE)
    or_n, or_ms, _ = ctx.profile_read(wfq.KT_ORTHO)
    ctx.profile(False)
    st, status, alpha = res[-1]
    good = sum(1 for x in st if x["rel_residual"] <= 1e-8)
    iters = [x["iters"] for x in st]
    peaks, peak_src = load_peaks()
    roof = None
    if gv_n:
        achieved = gv_bytes / (gv_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"],
                "traffic": DGEMV_DRAM_BYTES_PER_ENTRY * n * (-(-n // 128) * 128),
                "traffic_source": "ncu dram__bytes_read+write of k_dgemv_df at N = 8200 (same kernel, same "
                                  "plane layout), scaled per stored entry to this N",
                "kernel": "k_dgemv_df (double-float product of the BEM operator's FP32 pair planes)",
                "launches": gv_n, "avg_ms": gv_ms / gv_n, "bytes_per_launch": gv_bytes / gv_n,
                "peak_source": peak_src + " hbm_gbs (STREAM-style copy)"}
    out = {"metric": "freq-point solves/s", "value": good * args.steps * world / (ms / 1e3), "unit": "solves/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32x2(double-float)+f64", "data": "synthetic",
           "config": {"workload": args.workload, "operator": "continuum BEM (Eq. 21-22), charge form, collocation",
                      "n_elements": n, "nfreq": nf, "ndir": nd, "columns": ncols, "rel_tol": 1e-8,
                      "solver": "shifted gmres (one real Arnoldi per direction, all frequencies)",
                      "parallelism": f"replicas{world}",
                      "l2": "inputs larger than L2 (FP32 pair planes of the operator, %.2f GB)" % (8.0 * n * n / 1e9)},
           "accuracy": {"max_rel_residual": max(x["rel_residual"] for r in res for x in r[0]),
                        "columns_converged": good, "iters_min_mean_max": [min(iters), float(np.mean(iters)),
                                                                          max(iters)], "status": status},
           "kernel_ms_per_step": {"dgemv_df": gv_ms / args.steps, "shift_copy": sp_ms / args.steps,
                                  "ortho_phase": or_ms / args.steps},
           "roofline": roof, "clocks": clk, "gpu_launches": int(launches)}
    if not args.no_e2e:
        s = wl["surface"]
        pins = {k: torch.from_numpy(np.ascontiguousarray(s[k])).pin_memory().numpy()
                for k in ("xyz", "normal", "area", "curvature")}
        q_host = torch.empty((n, ncols), dtype=torch.complex128).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ge = wfq.BemGeometry(ctx, pins["xyz"], pins["normal"], pins["area"], pins["curvature"], wl["bem"],
                                 store=store)
            ge.solve_gmres_shifted(om, dirs, rel_tol=1e-8, max_iter=4000, prec=wfq.PREC_FP64, out=q_host.numpy())
            ge.polarizability(q_host.numpy())
            ge.close()
        torch.cuda.synchronize()
        te = max_over_ranks(time.perf_counter() - t0, dist)
        out["e2e"] = {"value": good * args.steps * world / te, "unit": "solves/s",
                      "h2d_bytes_per_step": int(sum(v.nbytes for v in pins.values()) + om.nbytes + dirs.nbytes),
                      "d2h_bytes_per_step": int(n * ncols * 16 + ncols * 3 * 16),
                      "includes": "operator build (FP64 and FP32 pair planes) from host surface arrays, solve, "
                                  "alpha"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count()))
        from oracle import build as obuild
        obuild.build()
        rng = np.random.default_rng(20210302)
        cols = rng.permutation(ncols)[:4]
        solved, secs, alphas, cores, _ = oracle_sample_bem(wl, args.cpu_budget_s, cols)
        errs = [float(np.abs(alpha[c] - a).max() / np.abs(a).max()) for c, a in alphas.items()]
        out["cpu_baseline"] = {"value": solved / secs, "unit": "solves/s", "cores": cores, "kind": "oracle",
                               "sample": f"{solved} sampled (omega, direction) columns of the same workload, "
                                         "FP64 GMRES(50) on the oracle's dense BEM operator to rel. residual "
                                         "1e-10 (assembly not timed)"}
        out["accuracy"]["alpha_rel_err_vs_oracle_sampled"] = max(errs) if errs else None
        out["accuracy"]["alpha_columns_checked"] = sorted(alphas)
    g.close()
    ctx.close()
    return out


def run_apply(args, rank, world, dist, ctx, g, wl, store):
    """Operator applies y = (A - z I) x on all columns of the workload at once (mixed
    precision), timed on device-resident inputs; metric = pair interactions per second
    (N^2 per apply; one pass over the pairs serves every column)."""
    import torch
    from paper_2103_00438_gb300 import wfq
    xyz, p, om, dirs = wl["xyz"], wl["params"], wl["omega"], wl["dirs"]
    n = len(xyz)
    ncplx = len(om) * len(dirs)
    omc = np.repeat(om, len(dirs))
    rng = np.random.default_rng(20210303)
    xh = ((rng.standard_normal((n, ncplx)) + 1j * rng.standard_normal((n, ncplx))) / np.sqrt(2)).astype(np.complex64)
    x = torch.from_numpy(xh).cuda()
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    prec = wfq.PREC_MIXED
    fmm_build_s = None
    if args.fmm_order:
        t0 = time.perf_counter()
        g.fmm_build(args.fmm_order)
        fmm_build_s = time.perf_counter() - t0
        prec = wfq.PREC_FMM
    for _ in range(args.warmup):
        g.apply(omc, x, y, prec=prec, stream=stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    ctx.profile(True)
    l0 = wfq.kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        g.apply(omc, x, y, prec=prec, stream=stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    launches = wfq.kernel_launches() - l0
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    gemm_n, gemm_ms, gemm_flops = ctx.profile_read(wfq.KT_GEMM_MIXED)
    fmm_n, fmm_ms, _ = ctx.profile_read(wfq.KT_FMM)
    ctx.profile(False)
    ms = max_over_ranks(ms, dist)
    pairs = float(n) * float(n)
    value = pairs * args.steps * world / (ms * 1e-3) / 1e9
    peaks, peak_src = load_peaks()
    gemm_avg = gemm_ms / max(gemm_n, 1)
    if args.fmm_order:
        roof = {"bound": "fmm", "achieved": None, "peak": None, "unit": None, "frac": None, "traffic": None,
                "kernel": "fmm passes (p2m, m2m, m2l, l2l, l2p + near field)", "avg_ms": fmm_ms / max(fmm_n, 1),
                "tree": g.fmm_info(), "build_s": fmm_build_s}
    elif store & wfq.STORE_BF16X2:
        ach = gemm_flops / (gemm_ms * 1e-3) / 1e12
        peak = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
        roof = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": None, "kernel": "gemm_3xbf16 (k_gemm3_tc)", "avg_ms": gemm_avg,
                "peak_source": peak_src + " bf16_tflops_sustained"}
    else:
        props = torch.cuda.get_device_properties(0)
        sm_mhz = peaks.get("sm_max_mhz", 2070.0)
        peak_gpairs = props.multi_processor_count * 128 * sm_mhz * 1e6 / MF_OPS_PER_PAIR / 1e9
        ach = pairs / (gemm_avg * 1e-3) / 1e9
        roof = {"bound": "alu", "achieved": ach, "peak": peak_gpairs, "unit": "Gpairs/s", "frac": ach / peak_gpairs,
                "traffic": None, "kernel": "gemm_3xbf16 matrix-free (k_gemm3_mf)", "avg_ms": gemm_avg,
                "peak_source": f"derived: {props.multi_processor_count} SMs x 128 FP32 lanes x {sm_mhz:.0f} MHz / "
                               f"{MF_OPS_PER_PAIR} instructions per generated D entry",
                "tensor_tflops": gemm_flops / (gemm_ms * 1e-3) / 1e12}
    out = {"metric": "T-pair Gint/s", "value": value, "unit": "Gint/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32 (fmm)" if args.fmm_order else "bf16x3+f32", "data": "synthetic",
           "config": {"workload": args.workload, "n_atoms": n, "columns": 2 * ncplx,
                      "path": (f"fast multipole, order {args.fmm_order}" if args.fmm_order else
                               "stored bf16 D" if store & wfq.STORE_BF16X2 else "matrix-free"),
                      "precision": "mixed: 3xBF16 D products, FP32 accumulation",
                      "parallelism": f"replicas{world}",
                      "l2": "inputs larger than L2" if n * n * 4 > 129e6 or n * 64 > 129e6 else "small"},
           "roofline": roof, "clocks": clk, "gpu_launches": int(launches)}
    # accuracy on sampled rows against the oracle (rows recomputed from Eq. 3 one by one)
    if rank == 0 and not args.no_cpu_baseline:
        os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count()))
        from oracle import build as ob
        from oracle import oracle as orc
        ob.build()
        if True:
            yh = y.cpu().numpy()
            rows = rng.choice(n, size=16, replace=False)
            t0 = time.perf_counter()
            yo, bnd = orc.apply_rows(xyz, p, orc.z_of_omega(omc[0], p), xh[:, 0].astype(complex), rows)
            secs = time.perf_counter() - t0
            ratio = float(np.max(np.abs(yh[rows, 0] - yo) / bnd))
            # pair evaluations the oracle made: a neighbour scan per row plus one N-term row
            # of D for the row and for each neighbour (~49 neighbours in graphene)
            g_info = g.info()
            nbr = g_info["nnz"] / n
            row_pairs = float(len(rows)) * (2.0 + nbr) * n
            out["accuracy"] = {"sampled_rows": len(rows), "max_err_over_bound": ratio,
                               "bound_tolerance": 1e-6 if args.fmm_order else 4e-5}
            out["cpu_baseline"] = {"value": row_pairs / secs / 1e9, "unit": "Gint/s", "cores": os.cpu_count(),
                                   "kind": "oracle",
                                   "sample": f"{len(rows)} rows of (A - zI)x with D recomputed from Eq. 3 for each "
                                             "row and its neighbours (one column)"}
    if not args.no_e2e:
        yh2 = np.empty_like(xh)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            g.apply(omc, xh, yh2, prec=prec)
        te = time.perf_counter() - t0
        out["e2e"] = {"value": pairs * args.steps * world / te / 1e9, "unit": "Gint/s",
                      "h2d_bytes_per_step": int(xh.nbytes), "d2h_bytes_per_step": int(xh.nbytes)}
    g.close()
    ctx.close()
    return out


# ------------------------------------------------------------------ serving

def run_serve(args, rank, world, dist):
    """Seeded Poisson stream of (structure, frequencies, directions) requests through the
    request server (continuous batching, memory admission, worker streams), every request
    through the public API with host buffers.  The arrival rate is `--load` times the
    capacity measured on a closed-loop batch of the same stream just before.  Reported:
    solves/s over the stream, p50/p99 request latency (submit to result in host memory),
    and the same columns solved one (omega, direction) at a time by plain FP64 GMRES(50)
    on the same GPU (sampled per structure, extrapolated over the stream's mix)."""
    import torch
    from paper_2103_00438_gb300 import structures as S
    from paper_2103_00438_gb300 import wfq

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    mix = S.serving_mix(args.requests, pool_size=args.pool)
    pool, reqs, gaps = mix["pool"], mix["requests"], mix["gaps"]
    ctx = wfq.Context(local)
    # structures up to 20k atoms keep every D storage; the larger ones the FP64 D alone (the
    # shifted solver splits it into float pairs as it streams it; plain FP64 GMRES reads it)
    store = lambda p: (wfq.STORE_FP64 | wfq.STORE_BF16X2 | wfq.STORE_F32X2) if len(p["xyz"]) <= 20040 \
        else wfq.STORE_FP64
    geoms = [wfq.Geometry(ctx, p["xyz"], p["params"], store=store(p)) for p in pool]
    m, tol, max_iter = args.m, 1e-8, 4000
    resident = sum(gm.info()["device_bytes"] for gm in geoms)
    sv = wfq.Server(ctx, nworkers=args.workers, budget_bytes=resident + (64 << 30), max_columns=384)
    ncol = lambda r: len(r[1]) * len(r[2])

    def closed_loop(batch):
        t0 = time.perf_counter()
        ids = [sv.submit(geoms[si], om, d, m=m, rel_tol=tol, max_iter=max_iter) for si, om, d in batch]
        res = [sv.poll(i, wait=True) for i in ids]
        return res, time.perf_counter() - t0

    # warm-up and capacity: two closed-loop batches drawn from the same seeded stream
    nwarm = max(args.warmup, 1) * 8
    rng = np.random.default_rng(20210306)
    closed_loop([reqs[int(i)] for i in rng.integers(0, len(reqs), size=nwarm)])
    cal = [reqs[int(i)] for i in rng.integers(0, len(reqs), size=max(len(reqs) // 10, 24))]
    res_cal, t_cal = closed_loop(cal)
    capacity = sum(ncol(r) for r in cal) / t_cal                 # solves/s, closed loop
    mean_cols = float(np.mean([ncol(r) for r in reqs]))
    rate = args.load * capacity / mean_cols                      # requests/s
    arrivals = np.cumsum(gaps) / rate

    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ctx.profile(True)
    launches0 = wfq.kernel_launches()
    ids = [None] * len(reqs)
    submit_err = []

    def submitter():
        t0 = time.perf_counter()
        try:
            for k, (si, om, d) in enumerate(reqs):
                dt = arrivals[k] - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
                ids[k] = sv.submit(geoms[si], om, d, m=m, rel_tol=tol, max_iter=max_iter)
        except Exception as e:    # reported below; the poll loop stops at the first missing id
            submit_err.append(repr(e))

    t_start = time.perf_counter()
    th = threading.Thread(target=submitter)
    th.start()
    results = []
    for k in range(len(reqs)):
        while ids[k] is None and th.is_alive():
            time.sleep(1e-4)
        if ids[k] is None:
            break
        results.append(sv.poll(ids[k], wait=True))
    th.join()
    t_stream = time.perf_counter() - t_start
    launches = wfq.kernel_launches() - launches0
    clk = clocks.stop()
    gemm_n, gemm_ms, gemm_flops = ctx.profile_read(wfq.KT_GEMM_MIXED)
    gv_n, gv_ms, gv_bytes = ctx.profile_read(wfq.KT_DGEMV_DF)
    ctx.profile(False)
    sv.close()
    if submit_err:
        raise RuntimeError("submit failed: " + submit_err[0])

    ok = [r for r in results if r["status"] == "WFQ_OK"]
    solves = sum(len(r["stats"]) for r in ok)
    lat = np.array([r["latency_s"] for r in results])
    qwait = np.array([r["queue_s"] for r in results])
    max_res = max(s["rel_residual"] for r in results for s in r["stats"])
    merged = sum(1 for r, q in zip(results, reqs) if r["batch_columns"] > ncol(q))
    by_status = {}
    for r, q in zip(results, reqs):
        key = "%s/%s" % (pool[q[0]]["name"], r["status"])
        by_status[key] = by_status.get(key, 0) + 1
    value = solves / t_stream

    # plain FP64 GMRES(50), one (omega, direction) column at a time, on the same GPU:
    # two sampled columns per structure, extrapolated over the stream's columns
    t_plain = {}
    for si, gm in enumerate(geoms):
        own = [r for r in reqs if r[0] == si][:2]
        ts = []
        for _, om, d in own:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, st, status = gm.solve_gmres(om[:1], d[:1], m=50, rel_tol=tol, max_iter=max_iter, prec=wfq.PREC_FP64)
            ts.append(time.perf_counter() - t0)
            if status != "WFQ_OK":
                raise RuntimeError(f"plain FP64 GMRES did not converge on {pool[si]['name']}")
        t_plain[si] = float(np.mean(ts))
    plain_time = sum(ncol(r) * t_plain[r[0]] for r in reqs)
    plain_value = sum(ncol(r) for r in reqs) / plain_time

    # accuracy audit against the FP64 oracle: the first request on each structure of at most
    # 2,000 atoms, its first column
    audit = []
    if not args.no_cpu_baseline:
        from oracle import build as ob
        from oracle import oracle as orc
        ob.build()
        for si, pdesc in enumerate(pool):
            if len(pdesc["xyz"]) > 2000:
                continue
            k = next(i for i, r in enumerate(reqs) if r[0] == si)
            xyz, p = pdesc["xyz"], pdesc["params"]
            csr = orc.kbar_csr(xyz, p)
            op = orc.Operator.stored(orc.d_matrix(xyz, p["eta"]), csr)
            R = orc.rhs_csr(xyz, csr, reqs[k][2][0]).astype(complex)
            q, _ = op.gmres(orc.z_of_omega(reqs[k][1][0], p), R, restart=50, rel_tol=1e-10, max_iter=20000)
            a_ref = orc.alpha(xyz, q)
            a_gpu = geoms[si].polarizability(results[k]["q"][:, :1])[0]
            audit.append(float(np.abs(a_gpu - a_ref).max() / np.abs(a_ref).max()))

    peaks, peak_src = load_peaks()
    roof = None
    if gv_n and gv_ms >= gemm_ms:
        # concurrent batches overlap on the device, so the per-launch times include sharing
        achieved = gv_bytes / (gv_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                "kernel": "k_dgemv_df (double-float D product of the real Arnoldi vectors)", "launches": gv_n,
                "avg_ms": gv_ms / gv_n, "peak_source": peak_src + " hbm_gbs (STREAM-style copy)",
                "note": "launch times measured while batches on other worker streams share the GPU"}
    elif gemm_n:
        achieved = gemm_flops / (gemm_ms * 1e-3) / 1e12
        peak = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": "gemm_3xbf16 (k_gemm3_tc)", "launches": gemm_n,
                "avg_ms": gemm_ms / gemm_n,
                "peak_source": peak_src + " bf16_tflops_sustained (kernel timed inside a long step)"}
    h2d = sum(r[1].nbytes + r[2].nbytes for r in reqs)
    d2h = sum(len(pool[r[0]]["xyz"]) * ncol(r) * 16 for r in reqs)
    out = {"metric": "freq-point solves/s (serving mix)", "value": value, "unit": "solves/s", "n_gpus": world,
           "steps": 1, "warmup": nwarm, "ms_per_step": t_stream * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3+f32+f64", "data": "synthetic",
           "config": {"workload": "serve: seeded Poisson stream (seed 20210305) of %d requests over %d resident "
                                  "structures (%s), 1-64 frequencies x 1-3 directions each" %
                                  (len(reqs), len(pool), ", ".join("%s N=%d" % (p["name"], len(p["xyz"]))
                                                                   for p in pool)),
                      "requests": len(reqs), "mean_columns_per_request": mean_cols,
                      "arrival_rate_req_per_s": rate, "load": args.load,
                      "capacity_closed_loop_solves_per_s": capacity, "workers": args.workers,
                      "solver": "shifted gmres per batch (stored D), continuations gmres(50)",
                      "rel_tol": tol, "parallelism": f"replicas{world}",
                      "resident_bytes": resident, "budget_bytes": resident + (64 << 30),
                      "l2": "resident D planes of all structures (%.1f GB) larger than L2" %
                            (sum(4.0 * len(p["xyz"]) ** 2 for p in pool) / 1e9)},
           "latency": {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                       "mean_s": float(lat.mean()), "max_s": float(lat.max()),
                       "queue_p50_s": float(np.percentile(qwait, 50)),
                       "queue_p99_s": float(np.percentile(qwait, 99))},
           "accuracy": {"requests_ok": len(ok), "requests": len(results), "max_rel_residual": max_res,
                        "alpha_rel_err_vs_oracle_sampled": max(audit) if audit else None,
                        "requests_merged_into_larger_blocks": merged, "by_structure_status": by_status},
           "plain_fp64_gmres_same_gpu": {"value": plain_value, "unit": "solves/s",
                                         "sample": "2 columns per structure, one (omega, direction) per "
                                                   "wfq_solve_gmres call, FP64, GMRES(50), rel. tol 1e-8; "
                                                   "extrapolated over the stream's columns",
                                         "seconds_per_column": {pool[s]["name"]: t for s, t in t_plain.items()},
                                         "served_over_plain": value / plain_value},
           "roofline": roof, "clocks": clk, "gpu_launches": int(launches),
           "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                   "includes": "every request through wfq_server_submit/poll with host buffers: the value itself "
                               "is end to end (structures resident, built before the stream)"}}
    for gm in geoms:
        gm.close()
    ctx.close()
    return out


# ------------------------------------------------------------------ spectrum

def run_spectrum(args, rank, world, dist):
    """A whole absorption spectrum in one shifted solve: the workload's structure on a
    0.01 eV grid over its band (x, y, z), sigma_k(omega) = (4 pi omega / c) Im alpha_kk
    (Eq. 28) and the isotropic mean (Eq. 29), with the Krylov iterations each frequency
    needed (its column's Arnoldi steps) -- the iterations-versus-frequency scan."""
    import torch
    from paper_2103_00438_gb300 import structures as S
    from paper_2103_00438_gb300 import wfq

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    wl = workload(args.workload)
    xyz, dirs = wl["xyz"], np.eye(3)
    lo, hi = float(wl["omega"][0]), float(wl["omega"][-1])
    ev_lo, ev_hi = lo * S.HARTREE_EV, hi * S.HARTREE_EV
    grid_ev = np.round(np.arange(ev_lo, ev_hi + 1e-9, 0.01), 6)
    om = S.ev(grid_ev)
    n, nf = len(xyz), len(om)
    ctx = wfq.Context(local)
    g = make_geometry(wfq, ctx, wl, wfq.STORE_F32X2)
    # precision of any continuation: FP64 for a BEM surface (no bf16 planes stored)
    prec = wfq.PREC_FP64 if is_bem(wl) else wfq.PREC_MIXED
    stream = torch.cuda.current_stream()
    q = torch.empty((n, nf * 3), dtype=torch.complex128, device="cuda")
    for _ in range(max(args.warmup, 1)):
        g.solve_gmres_shifted(om, dirs, rel_tol=1e-8, max_iter=4000, prec=prec, out=q, stream=stream)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        _, st, status = g.solve_gmres_shifted(om, dirs, rel_tol=1e-8, max_iter=4000, prec=prec, out=q,
                                              stream=stream)
        sig, sig_iso = g.cross_section(om, dirs, q, stream=stream)    # Eq. 28 per column, Eq. 29
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), dist)
    ni = np.array([s["iters"] for s in st]).reshape(nf, 3)
    good = sum(1 for s in st if s["rel_residual"] <= 1e-8)
    ipk = int(np.argmax(sig_iso))
    out = {"metric": "freq-point solves/s (spectrum)", "value": good * args.steps * world / (ms / 1e3),
           "unit": "solves/s", "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 1),
           "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32x2(double-float)+f64", "data": "synthetic",
           "config": {"workload": f"{args.workload} spectrum: {nf} frequencies on a 0.01 eV grid over "
                                  f"{grid_ev[0]:.2f}-{grid_ev[-1]:.2f} eV x 3 directions, one shifted GMRES solve",
                      "n_atoms": n, "columns": nf * 3, "rel_tol": 1e-8, "parallelism": f"replicas{world}"},
           "accuracy": {"max_rel_residual": max(s["rel_residual"] for s in st), "columns_converged": good,
                        "status": status},
           "spectrum": {"omega_ev": grid_ev.tolist()[::10], "sigma_iso_au": sig_iso.tolist()[::10],
                        "peak_ev": float(grid_ev[ipk]), "peak_sigma_iso_au": float(sig_iso[ipk]),
                        "sampling": "every 10th grid point"},
           "iterations_vs_omega": {"omega_ev": grid_ev.tolist()[::10],
                                   "iters_max_over_directions": ni.max(axis=1).tolist()[::10],
                                   "min": int(ni.min()), "mean": float(ni.mean()), "max": int(ni.max())},
           "clocks": clk}
    g.close()
    ctx.close()
    return out


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        backend = "nccl" if args.impl == "ours" else "gloo"
        if args.impl == "ours":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group(backend=backend)
        dist = tdist
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        else:
            out = run_ours(args, rank, world, dist)
            if rank == 0 and out is not None:
                print(json.dumps(out), flush=True)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
