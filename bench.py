#!/usr/bin/env python3
"""Benchmark of the complex Helmholtz Krylov path on GB300.

One step = one full FP64 BiCGStab solve (Section 7 of the paper: CSR SpMV +
fused zdot/zaxpy/norm kernels, device-side loop in a CUDA graph) of the C2
workload: the jittered P1-FEM cylinder (nr=40, ntheta=96, nz=160, k=20,
impedance ends; 618,401 unknowns, 9.18M nonzeros), from x0 = 0 with
tol 1e-10 and a fixed iteration cap (the cap is reached: preconditioner-free
BiCGStab does not converge on this indefinite k=20 operator, so every step
performs the same work).

value  = algorithmic bytes moved by the solve / device time of the step
         (40*nnz + 312*n bytes per iteration + setup and exit passes), GB/s.
e2e    = the same bytes over the wall time of the public-API call sequence
         with host buffers: pinned H2D of the CSR arrays and b, matrix
         handle creation, solve, D2H of x.
roofline = the dominant kernel (the CSR SpMV core) timed alone with CUDA
         events on its stream, L2 flushed between launches.
cpu_baseline / --impl reference = the C oracle (single thread) on a bounded
         number of BiCGStab iterations of the same system.

Multi-GPU (torchrun, N > 1): replicas -- every rank solves its own copy of
the system on its own GPU (weak scaling, no collective on the data path);
value sums the ranks' bytes over the slowest rank's time.
"""

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "zSpMV GB/s (% HBM peak); BiCGStab s to rel.res 1e-10, mixed/batched vs FP64"
L2_BYTES = 129 * 1024 * 1024
FALLBACK_HBM_GBS = 6800.0


def spmv_flops(A):
    """binary64 flops of one product y = A x with complex x: a complex
    multiply-add (8 flops, four FMAs) per entry, two FMAs (4 flops) for an
    entry whose imaginary part is zero"""
    nreal = int(np.count_nonzero(A.val.imag == 0))
    return 8 * (A.nnz - nreal) + 4 * nreal


def spmv_bytes(n, nnz):
    """Algorithmic bytes of one CSR SpMV: values and columns once, row
    pointers once, x read once, y written once."""
    return 20 * nnz + 36 * n + 4


def iter_bytes(n, nnz):
    """Algorithmic bytes of one fused BiCGStab iteration (two SpMVs plus the
    vector passes F1..F5)."""
    return 40 * nnz + 312 * n


def solve_bytes(n, nnz, iters):
    # start (x0 copy 32n, r = b - A x: SpMV + b 16n + writes r, rh, p, v 64n)
    # + iterations + exit (true residual SpMV + b 16n, copy-out 32n)
    start = 32 * n + spmv_bytes(n, nnz) + 16 * n + 64 * n
    finish = spmv_bytes(n, nnz) + 16 * n + 32 * n
    return start + iters * iter_bytes(n, nnz) + finish


def job_totals(elapsed, nbytes, world, device):
    """Whole-job totals over replicas: the slowest rank's time and the sum of
    every rank's bytes (each rank solves its own system: weak scaling)."""
    if world <= 1:
        return elapsed, nbytes
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(elapsed)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    b = torch.tensor([float(nbytes)], dtype=torch.float64, device=device)
    dist.all_reduce(b, op=dist.ReduceOp.SUM)
    return float(t.item()), float(b.item())


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_sha():
    h = hashlib.sha256()
    for f in ("spmv.cuh", "hz_internal.cuh", "arith.cuh", "spmv.cu"):
        with open(os.path.join(ROOT, "paper_2112_06465_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(name):
    """DRAM bytes per SpMV launch from the committed ncu summary
    profiles/<name>, if it was taken on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", name)
    try:
        kv = {}
        with open(p) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel_source_sha") != kernel_source_sha():
            return None
        return float(kv["dram_bytes_per_launch"])
    except Exception:
        return None


TRAFFIC_FILES = {4: "spmv_ffb_c2_traffic.txt", 6: "spmv_d64b_c2_traffic.txt", 7: "spmv_d64p_c2_traffic.txt"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.out = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                self.out = ""

    def summary(self):
        if not self.out:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out.strip().splitlines():
            f = [c.strip() for c in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def build_workload():
    import workloads as W
    A, b = W.c2_cylinder()
    return A, b


def cpu_oracle_rate(A, b, iters, threads=None):
    """The oracle's BiCGStab for a fixed number of iterations; returns (GB/s,
    seconds, iterations).  threads=None: the plain single-thread build;
    threads=k: the OpenMP build on k threads."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    if threads is None:
        x, info = oracle.bicgstab(A, b, tol=1e-300, maxit=iters, history=False)
    else:
        x, info = oracle.bicgstab_omp(A, b, tol=1e-300, maxit=iters, threads=threads)
    dt = time.perf_counter() - t0
    return solve_bytes(A.n, A.nnz, info.iters) / dt / 1e9, dt, info.iters


def run_reference(args):
    """--impl reference: the CPU oracle timed on the host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    A, b = build_workload()
    iters = args.ref_iters
    for _ in range(args.warmup):
        cpu_oracle_rate(A, b, 2)
    rates, times = [], []
    for _ in range(args.steps):
        r, dt, it = cpu_oracle_rate(A, b, iters)
        rates.append(r)
        times.append(dt)
    value = statistics.median(rates)
    sample = f"{iters} BiCGStab iterations of C2 per step (n={A.n}, nnz={A.nnz}), single-thread build"
    cores = len(os.sched_getaffinity(0))
    try:
        rN, dtN, itN = cpu_oracle_rate(A, b, iters, threads=cores)
        all_cores = {"value": rN, "unit": "GB/s", "cores": cores, "kind": "oracle (OpenMP build)",
                     "sample": f"{itN} BiCGStab iterations of C2 ({dtN:.1f} s)"}
    except Exception as e:   # no OpenMP runtime on this host
        all_cores = {"unavailable": str(e)[:200]}
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(A, iters),
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": sample,
                         "all_cores": all_cores},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


DTYPES = {"fp64": "f64", "ff": "f32x2 (double-float complex128: hi+lo binary32 pairs)"}
SPMV_KINDS = {0: "binary64 CSR-vector (k_spmv)", 1: "binary64 SELL-C-sigma (k_spmv<0>)",
              2: "double-float CSR-vector (k_spmv_ff)", 3: "double-float SELL-C-sigma (k_spmv_ff<0>)",
              4: "double-float block-flat (k_spmv_ffb)",
              5: "double-float block-flat, bulk-copy staged (k_spmv_fft)",
              6: "binary64 block-flat, contiguous lane runs (k_spmv_d64b)",
              7: "binary64 block-flat on the packed stream (k_spmv_d64b<packed>)"}
BINARY64_KINDS = (0, 1, 6, 7)
# binary64 roof of GB300: the nominal FP64 rate of the profiling recipe's
# table (1.25 TFLOP/s); an own FMA-throughput probe measured 1.05 TFLOP/s
FP64_NOMINAL_TFLOPS = 1.25
FP64_PROBE_TFLOPS = 1.052


def run_spmv_only(args):
    """Three launches of the C2 SpMV (the roofline kernel), for ncu captures."""
    import torch
    import paper_2112_06465_gb300 as hz
    A, _ = build_workload()
    M = hz.Matrix.from_csr(A, ff=args.arith == "ff")
    if args.spmv:
        M.set_spmv(args.spmv, args.group)
    x = torch.randn(A.n, dtype=torch.complex128, device="cuda")
    y = torch.empty_like(x)
    for _ in range(3):
        hz.zspmv(M, x, y)
    torch.cuda.synchronize()
    print(json.dumps({"spmv_only": True, "arith": args.arith, "kind": M.props()["spmv_kind"], "group": args.group,
                      "n": A.n, "nnz": A.nnz}))


def run_kernel_case(args):
    """Profiling aid: one small case per kernel family, for ncu captures
    (nothing is timed).  spmv / cspmv: three C2 products (--arith picks
    binary64 or double-float); blas: zdotc, zaxpy, zscal, dznrm2 at 1e8
    elements, twice; outer: the adjoint outer product on C5 64^3, three
    times; batched: a four-box binary64 sweep, 100 iterations, twice; solve:
    two C2 solves of HZ_PROFILE_UNROLL iterations (set HZ_PROFILE_UNROLL=k so
    the iteration kernels are plain graph nodes) with --solve-method,
    --solve-mode and --precond."""
    import numpy as np
    import torch
    import paper_2112_06465_gb300 as hz
    import workloads as W
    dev = torch.device("cuda")
    case = args.kernel_case
    if case in ("spmv", "cspmv", "solve"):
        A, b = build_workload()
        M = hz.Matrix.from_csr(A, ff=args.arith == "ff", c64=case == "cspmv" or args.solve_mode == "mixed",
                               sell=args.spmv in ("sell", "sellff"))
        if args.spmv:
            M.set_spmv(args.spmv, args.group)
        if case == "cspmv":
            x = torch.randn(A.n, dtype=torch.complex64, device=dev)
            for _ in range(3):
                hz.cspmv(M, x)
        elif case == "spmv":
            x = torch.randn(A.n, dtype=torch.complex128, device=dev)
            for _ in range(3):
                hz.zspmv(M, x)
        else:
            bd = torch.as_tensor(b).to(dev)
            k = int(os.environ.get("HZ_PROFILE_UNROLL", "3"))
            kw = dict(method=args.solve_method, mode=args.solve_mode, precond=args.precond)
            it = k
            if args.solve_method == "bicgstabl":   # maxit counts BiCG steps, l = 4 per iteration
                kw["ell"] = 4
                it = 4 * k
            for _ in range(2):
                hz.zsolve(M, bd, tol=1e-10, maxit=it, **kw)
    elif case == "blas":
        n = 100_000_000
        x = torch.randn(n, dtype=torch.complex128, device=dev)
        y = torch.randn(n, dtype=torch.complex128, device=dev)
        a = torch.tensor([0.5 - 0.25j], dtype=torch.complex128, device=dev)
        for _ in range(2):
            hz.zdotc(x, y)
            hz.zaxpy(a, x, y)
            hz.zscal(a, x)
            hz.dznrm2(x)
    elif case == "outer":
        A = W.c5_inverse_problem()["A"]
        M = hz.Matrix.from_csr(A)
        mu = torch.randn(A.n, dtype=torch.complex128, device=dev)
        x = torch.randn(A.n, dtype=torch.complex128, device=dev)
        for _ in range(3):
            hz.outer_on_pattern(M, mu, x)
    elif case == "batched":
        systems = [W.fd_helmholtz_box(m, kh=0.3, damping=0.05) for m in (24, 32, 40, 48)]
        mats = [hz.Matrix.from_csr(A) for A in systems]
        bs = [torch.ones(A.n, dtype=torch.complex128, device=dev) for A in systems]
        for _ in range(2):
            hz.zsolve_batched(mats, bs, tol=1e-10, maxit=100)
    torch.cuda.synchronize()
    print(json.dumps({"kernel_case": case, "arith": args.arith}))


def compare_modes(hz, torch, full_c4, maxit, all_variants=False):
    """Mixed precision and the batched sweep against the plain complex128
    solver on the C4 frequency-sweep systems, each to relative residual 1e-10.

    Every system is solved (x0 = 0) by the binary64 BiCGStab solver, the
    mixed solver (complex64 inner BiCGStab, binary64 outer refinement) and
    binary64 TFQMR, and all systems at once by the persistent batched solver
    in binary64 and in mixed precision.  all_variants adds binary64
    BiCGStab(4) and the double-float variants (BiCGStab, mixed, Jacobi,
    BiCGStab(4), TFQMR, batched).  full_c4: all 64 systems (else the boxes
    and the smallest cylinder, 32 systems).  Times are CUDA events around
    each call, after one untimed call of each kind with a two-iteration cap
    (graph capture, module loading).  Speedups are over the systems every
    variant solved."""
    import workloads as W
    from workloads import configs as WC
    cyl = WC.C4_CYLINDERS if full_c4 else WC.C4_CYLINDERS[:1]
    systems = W.c4_sweep_systems(cylinders=cyl)
    stream = torch.cuda.current_stream()
    mats, bs = [], []
    for name, A, b in systems:
        # autotune: times the SpMV kinds and CSR-vector groups on this matrix;
        # the batched solver's row tile (complex64 / double-float products)
        # per geometry is the group it keeps
        M = hz.Matrix.from_csr(A, ff=True, c64=True, autotune=True)
        mats.append(M)
        bs.append(torch.as_tensor(b).to("cuda"))

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        return out, e0.elapsed_time(e1)

    variants = {
        "fp64_binary64": ("flat64p", dict(mode="fp64")),
        "mixed": ("flat64p", dict(mode="mixed")),
        "tfqmr_binary64": ("flat64p", dict(method="tfqmr")),
    }
    if all_variants:
        variants.update({
            "bicgstab4_binary64": ("flat64p", dict(method="bicgstabl", ell=4)),
            "fp64_double_float": ("ffflat", dict(mode="fp64")),
            "mixed_double_float": ("ffflat", dict(mode="mixed")),
            "fp64_double_float_jacobi": ("ffflat", dict(mode="fp64", precond="jacobi")),
            "bicgstab4_double_float": ("ffflat", dict(method="bicgstabl", ell=4)),
            "tfqmr_double_float": ("ffflat", dict(method="tfqmr")),
        })
    batched_variants = [("batched_fp64", "flat64p", "fp64"), ("batched_mixed", "flat64p", "mixed")]
    if all_variants:
        batched_variants.append(("batched_double_float", "ffflat", "fp64"))
    res = {k: [] for k in variants}
    groups = [M.props()["group"] for M in mats]
    for M, b, g in zip(mats, bs, groups):
        for key, (kind, kw) in variants.items():
            M.set_spmv(kind, g)
            hz.zsolve(M, b, tol=1e-10, maxit=2, **kw)          # graph capture
            (_, info), ms = timed(lambda: hz.zsolve(M, b, tol=1e-10, maxit=maxit, **kw))
            res[key].append((ms, info))
    batched = {}
    for key, kind, mode in batched_variants:
        for M, g in zip(mats, groups):   # the batch runs double-float when every handle's kind is;
            M.set_spmv(kind, g)          # its row tile is each handle's autotuned group
        hz.zsolve_batched(mats, bs, tol=1e-10, maxit=2, mode=mode)
        batched[key] = timed(lambda: hz.zsolve_batched(mats, bs, tol=1e-10, maxit=maxit, mode=mode))
    binfos = batched["batched_fp64"][0][1]
    ok_all = [all(res[k][i][1].converged for k in variants) and binfos[i].converged
              for i in range(len(mats))]

    def summary(rows):
        t_ok = sum(ms for (ms, _), ok in zip(rows, ok_all) if ok)
        return {"s_total": sum(ms for ms, _ in rows) / 1e3, "s_on_common": t_ok / 1e3,
                "converged": sum(1 for _, i in rows if i.converged),
                "iters": sum(i.iters for _, i in rows),
                "max_relres_true": max(i.relres_true for _, i in rows)}

    out = {"systems": len(mats), "solved_by_all": sum(ok_all), "tol": 1e-10, "maxit": maxit,
           "batch_row_tile_groups": groups,
           "workload": "C4 frequency sweep: FD boxes %s x 8 kh in [0.2, 0.8] + jittered P1 cylinders %s x 8 kh, "
                       "shift 0.05i" % (list(WC.C4_BOXES), [list(c) for c in cyl])}
    for key in variants:
        out[key] = summary(res[key])
    out["mixed"]["outer"] = sum(i.outer for _, i in res["mixed"])
    for key, ((_, infs), ms) in batched.items():
        out[key] = {"s_total": ms / 1e3, "converged": sum(1 for i in infs if i.converged),
                    "iters": sum(i.iters for i in infs), "max_relres_true": max(i.relres_true for i in infs)}
    base = out["fp64_binary64"]["s_on_common"]
    out["speedup_vs_fp64_binary64_on_common"] = {
        k: base / max(out[k]["s_on_common"], 1e-12) for k in variants if k != "fp64_binary64"}
    out["speedup_vs_fp64_binary64_all_systems"] = {
        k: out["fp64_binary64"]["s_total"] / out[k]["s_total"]
        for k in list(variants)[1:] + [b[0] for b in batched_variants]}
    # the systems that the binary64 solver and the mixed and batched solvers
    # all solve: time to rel.res 1e-10 on exactly those
    ok_mb = [res["fp64_binary64"][i][1].converged and res["mixed"][i][1].converged
             and batched["batched_fp64"][0][1][i].converged and batched["batched_mixed"][0][1][i].converged
             for i in range(len(mats))]
    out["mixed_batched_vs_binary64_on_common"] = {
        "systems": sum(ok_mb),
        "s_binary64": sum(ms for (ms, _), ok in zip(res["fp64_binary64"], ok_mb) if ok) / 1e3,
        "s_mixed": sum(ms for (ms, _), ok in zip(res["mixed"], ok_mb) if ok) / 1e3,
        "note": "batched solvers run every system in one launch; their time is over all systems"}
    for M in mats:
        M.close()
    return out


def time_spmv(hz, torch, M, n, stream, reps=20, c64=False):
    """Average device time (ms) of one hz_zspmv launch (hz_cspmv with c64).
    Every launch is preceded by a 1 GiB write (flushes the 129 MB L2 and
    keeps the GPU busy while the host enqueues the next launch, so host
    launch latency never lands between the events); all launches are
    enqueued before the one synchronisation."""
    x = torch.randn(n, dtype=torch.complex64 if c64 else torch.complex128, device="cuda")
    y = torch.empty_like(x)
    spmv = hz.cspmv if c64 else hz.zspmv
    flush = torch.empty(8 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(3):
        spmv(M, x, y)
    ev = []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        spmv(M, x, y)
        e1.record(stream)
        ev.append((e0, e1))
    torch.cuda.synchronize()
    return sum(e0.elapsed_time(e1) for e0, e1 in ev) / reps


def blas_sweep(hz, torch, stream, reps=10):
    """The complex128 BLAS-1 sweep of the C2 configuration: zdotc, zaxpy,
    zscal and dznrm2 over lengths 1e3 .. 1e8 in half decades.  Each call is
    preceded by a 1 GiB write (cold L2, GPU busy while the host enqueues),
    timed with CUDA events; median of `reps`.  Bytes: zdotc 32n, zaxpy 48n,
    zscal 32n, dznrm2 16n.  Working sets under the 129 MB L2 are marked."""
    import workloads as W
    import statistics as st_
    flush = torch.empty(8 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    alpha = torch.tensor([0.5 - 0.25j], dtype=torch.complex128, device="cuda")
    out = {"sizes": [], "zdotc": [], "zaxpy": [], "zscal": [], "dznrm2": []}
    nbytes = {"zdotc": 32, "zaxpy": 48, "zscal": 32, "dznrm2": 16}
    for n in W.blas_sweep_sizes():
        x = torch.randn(n, dtype=torch.complex128, device="cuda")
        y = torch.randn(n, dtype=torch.complex128, device="cuda")
        d = torch.empty(1, dtype=torch.complex128, device="cuda")
        r = torch.empty(1, dtype=torch.float64, device="cuda")
        calls = {"zdotc": lambda: hz.zdotc(x, y, out=d), "zaxpy": lambda: hz.zaxpy(alpha, x, y),
                 "zscal": lambda: hz.zscal(alpha, x), "dznrm2": lambda: hz.dznrm2(x, out=r)}
        out["sizes"].append(n)
        for op, fn in calls.items():
            fn()
            ev = []
            for _ in range(reps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                ev.append((e0, e1))
            torch.cuda.synchronize()
            us = 1e3 * st_.median(a.elapsed_time(b) for a, b in ev)
            gbs = nbytes[op] * n / (us * 1e-6) / 1e9
            out[op].append({"us": round(us, 2), "gbs": round(gbs, 1),
                            "l2_resident": nbytes[op] * n < L2_BYTES})
        del x, y
    return out


def spmv_h1(hz, torch, stream):
    """The SpMV on the H1 car-cabin stand-in (Q1 hexahedra, 27-entry rows),
    double-float block-flat and binary64 CSR-vector, L2 flushed."""
    import workloads as W
    A, _ = W.h1_hexcar()
    peak, _ = peaks()
    out = {"workload": "H1 Q1 hexahedral car cabin nx=192 kh=0.5 (27-entry rows)", "n": A.n, "nnz": A.nnz,
           "algorithmic_bytes_per_launch": spmv_bytes(A.n, A.nnz)}
    for key, ff, kind in (("double_float", True, None), ("binary64", False, None)):
        M = hz.Matrix.from_csr(A, ff=ff)
        ms = time_spmv(hz, torch, M, A.n, stream)
        gbs = spmv_bytes(A.n, A.nnz) / (ms / 1e3) / 1e9
        out[key] = {"launch_ms": ms, "achieved_gbs": gbs, "frac": gbs / peak,
                    "kind": M.props()["spmv_kind"], "group": M.props()["group"]}
        M.close()
    return out


def spmv_c64_c2(hz, torch, A, stream):
    """The complex64 SpMV of the mixed solver's inner iteration (block-flat
    complex64 kernel on a double-float handle) on C2, L2 flushed; algorithmic
    bytes 12 nnz + 20 n (8-byte values, 4-byte columns, x read once and y
    written once in complex64, row pointers)."""
    peak, _ = peaks()
    rp = torch.as_tensor(A.rowptr).cuda()
    cl = torch.as_tensor(A.col).cuda()
    vl = torch.as_tensor(A.val).cuda()
    M = hz.Matrix(rp, cl, vl, ff=True, c64=True)
    ms = time_spmv(hz, torch, M, A.n, stream, c64=True)
    nbytes = 12 * A.nnz + 20 * A.n + 4
    gbs = nbytes / (ms / 1e3) / 1e9
    M.close()
    return {"kernel": "complex64 block-flat SpMV through hz_cspmv, L2 flushed", "launch_ms": ms,
            "algorithmic_bytes_per_launch": nbytes, "achieved_gbs": gbs, "frac": gbs / peak}


def adjoint_c5(hz, torch, stream, reps=10):
    """The C5 inverse problem (A(theta) = L - kappa^2 diag(theta), kh = 0.5).

    converged: the adjoint step on the largest grid where a Krylov forward
    solve reaches 1e-12 (32^3, n = 32,768; TFQMR in binary64 for the forward
    and the adjoint solve, through solve_diag_param and loss.backward()),
    with the time of the forward and of the backward pass.
    grid_64: the configured 64^3 grid (n = 262,144), where no method here
    reaches 1e-12 (the forward solve stagnates): 300 binary64 TFQMR
    iterations of the forward solve (time per iteration), then the two
    gradient kernels, each timed alone with the L2 flushed (median of
    `reps`): the outer product on A's pattern (16 nnz bytes written;
    4 nnz + 4 (n + 1) of pattern and 32 n of mu and x read) and the diagonal
    gradient (48 n)."""
    import numpy as np
    import statistics as st_
    import workloads as W

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        return out, e0.elapsed_time(e1)

    # the converged adjoint step at 32^3
    p32 = W.c5_inverse_problem(m=32, nsample=512)
    M32 = hz.Matrix.from_csr(p32["A"])
    base32 = torch.as_tensor(p32["L"].to_scipy().diagonal().astype(np.complex128)).cuda()
    b32 = torch.as_tensor(p32["b"]).cuda()
    idx32 = torch.as_tensor(p32["sample_idx"]).cuda()
    d32 = torch.as_tensor(p32["data"]).cuda()

    def step():
        th = torch.as_tensor(p32["theta"].astype(np.complex128)).cuda().requires_grad_(True)
        x = hz.solve_diag_param(th, b32, M32, base32, -p32["kappa2"], tol=1e-12, maxit=8000, method="tfqmr")
        loss = torch.sum(torch.abs(x[idx32] - d32) ** 2)
        return th, x, loss

    th, x, loss = step()
    loss.backward()                                           # graph capture
    (th, x, loss), ms_fwd = timed(step)
    _, ms_bwd = timed(lambda: loss.backward())
    fwd_info = x.grad_fn.fwd_info if hasattr(x.grad_fn, "fwd_info") else None
    conv = {"workload": "C5 inverse problem at 32^3 (n = 32,768), TFQMR binary64 to 1e-12",
            "forward_ms": ms_fwd, "backward_ms": ms_bwd, "loss": float(loss.detach()),
            "forward_iters": fwd_info.iters if fwd_info else None}
    M32.close()

    prob = W.c5_inverse_problem()
    A = prob["A"]
    n, nnz = A.n, A.nnz
    M = hz.Matrix.from_csr(A)
    base = torch.as_tensor(prob["L"].to_scipy().diagonal().astype(np.complex128)).cuda()
    theta = torch.as_tensor(prob["theta"].astype(np.complex128)).cuda()
    b = torch.as_tensor(prob["b"]).cuda()
    idx = torch.as_tensor(prob["sample_idx"]).cuda()
    d = torch.as_tensor(prob["data"]).cuda()
    scale = -prob["kappa2"]
    flush = torch.empty(8 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    def cold(fn):
        fn()
        ev = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            ev.append((e0, e1))
        torch.cuda.synchronize()
        return st_.median(a.elapsed_time(z) for a, z in ev)

    iters = 300
    hz.mat_set_diag(M, base, scale, theta)
    hz.zsolve(M, b, tol=1e-12, maxit=iters, method="tfqmr")       # graph capture
    (x, inf_f), ms_f = timed(lambda: hz.zsolve(M, b, tol=1e-12, maxit=iters, method="tfqmr"))
    g = torch.zeros_like(x)
    g[idx] = x[idx] - d
    mu = hz.zconj(g)
    gval = torch.empty(nnz, dtype=torch.complex128, device="cuda")
    gth = torch.empty_like(x)
    ms_outer = cold(lambda: hz.outer_on_pattern(M, mu, x, out=gval))
    ms_diag = cold(lambda: hz.diag_grad(M, mu, x, scale, out=gth))
    peak, _ = peaks()
    ob = 20 * nnz + 36 * n + 4
    M.close()
    return {"converged": conv,
            "grid_64": {"workload": "C5 64^3 FD inverse problem, A(theta) = L - kappa^2 diag(theta), kh = 0.5",
                        "n": n, "nnz": nnz,
                        "forward": {"ms": ms_f, "iters": inf_f.iters, "status": inf_f.status_name,
                                    "relres_true": inf_f.relres_true,
                                    "iter_us": 1e3 * ms_f / max(inf_f.iters, 1)},
                        "outer_on_pattern": {"us": 1e3 * ms_outer, "algorithmic_bytes": ob,
                                             "gbs": ob / (ms_outer / 1e3) / 1e9,
                                             "frac": ob / (ms_outer / 1e3) / 1e9 / peak,
                                             # one complex product per entry: 4 binary64
                                             # pipe operations, the kernel's real limit
                                             "fp64_lane_ops": 4 * nnz,
                                             "frac_of_fp64_probe_rate":
                                                 4 * nnz / (ms_outer / 1e3) / (FP64_PROBE_TFLOPS / 2 * 1e12),
                                             "note": "L2 flushed before each launch; the 29 MB it writes fits in L2"},
                        "diag_grad": {"us": 1e3 * ms_diag, "gbs": 48 * n / (ms_diag / 1e3) / 1e9,
                                      "l2_resident": True}}}


def workload_config(A, maxit, arith="fp64", iters=None, status=None):
    return {"workload": "C2 jittered P1-FEM cylinder nr=40 ntheta=96 nz=160 k=20 impedance ends, "
                        f"complex128 BiCGStab x0=0 tol=1e-10 maxit={maxit}",
            "arith": arith, "n": A.n, "nnz": A.nnz, "maxit": maxit,
            "solve_iters": iters, "solve_status": status,
            "l2": "inputs larger than L2 (CSR matrix %.0f MB > 129 MB L2); the SpMV roofline "
                  "launches flush L2 between launches" % (A.nnz * 20 / 1e6)}


def spmv_roofline(hz, torch, M, A, stream, kind):
    """Roofline object of the SpMV core of the handle's kind, timed alone.

    A binary64 kind is bound by GB300's binary64 pipe, so its roofline is
    "alu": the multiply-adds the product needs (8 flops per complex entry,
    4 per entry whose imaginary part is zero, which takes two FMAs against
    a complex x) over the launch time, against the nominal FP64 rate; the
    HBM fraction is given beside it.  A double-float kind is HBM-bound."""
    sp_avg = time_spmv(hz, torch, M, A.n, stream)
    peak, peak_src = peaks()
    gbs = spmv_bytes(A.n, A.nnz) / (sp_avg / 1e3) / 1e9
    traffic = recorded_traffic(TRAFFIC_FILES[kind]) if kind in TRAFFIC_FILES else None
    hbm = {"achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
           "frac_of_nominal_8000": gbs / 8000.0, "peak_source": f"{peak_src} (burst copy)"}
    desc = "%s SpMV through hz_zspmv alone, L2 flushed" % SPMV_KINDS.get(kind, kind)
    if kind in BINARY64_KINDS:
        flops = spmv_flops(A)
        tf = flops / (sp_avg / 1e3) / 1e12
        return {"bound": "alu", "achieved": tf, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                "frac": tf / FP64_NOMINAL_TFLOPS, "traffic": traffic,
                "alu": "binary64 FMA pipe; peak = nominal FP64 rate (1.25 TFLOP/s); own FMA probe: "
                       f"{FP64_PROBE_TFLOPS} TFLOP/s", "frac_of_probe": tf / FP64_PROBE_TFLOPS,
                "kernel": desc, "algorithmic_flops_per_launch": flops,
                "flops_if_every_entry_complex": 8 * A.nnz,
                "algorithmic_bytes_per_launch": spmv_bytes(A.n, A.nnz), "launch_ms": sp_avg, "hbm": hbm}
    return {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
            "traffic": traffic, "frac_of_nominal_8000": gbs / 8000.0,
            "kernel": desc + "; peak %s (burst copy)" % peak_src,
            "algorithmic_bytes_per_launch": spmv_bytes(A.n, A.nnz), "launch_ms": sp_avg}


def double_float_entry(hz, torch, A, rp, cl, vl, bd, args, stream, steps=3):
    """The double-float fast path (48-bit hi+lo binary32 values, binary32
    exponent range), measured the same way as the headline for comparison:
    the same solve from x0 = 0 and its SpMV roofline.  Not the paper's
    arithmetic; reported beside the binary64 line, labelled."""
    M = hz.Matrix(rp, cl, vl, ff=True)
    x = torch.zeros_like(bd)
    hz.zsolve(M, bd, x=x, tol=1e-10, maxit=args.maxit, x0_zero=True)
    ms, its, sts = [], [], []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, info = hz.zsolve(M, bd, x=x, tol=1e-10, maxit=args.maxit, x0_zero=True)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        its.append(info.iters)
        sts.append(info.status_name)
    nbytes = sum(solve_bytes(A.n, A.nnz, it) for it in its)
    out = {"dtype": DTYPES["ff"], "value": nbytes / (sum(ms) / 1e3) / 1e9, "unit": "GB/s",
           "ms_per_step": sum(ms) / steps, "iters_per_step": its, "status": sts,
           "iter_us": 1e3 * sum(ms) / max(sum(its), 1),
           "roofline": spmv_roofline(hz, torch, M, A, stream, M.props()["spmv_kind"])}
    M.close()
    return out


def c3_precision(hz, torch, stream, iters=1000):
    """C3 (the precision configuration): the mixed solver against the plain
    binary64 solver on the same 2M-unknown cylinder.  Neither reaches 1e-10
    on this operator (the method stagnates), so both run the same budget of
    BiCGStab iterations from x0 = 0 (the mixed solver's inner iterations in
    total) and report time, time per iteration and the true relative
    residual reached."""
    import workloads as W
    A, b = W.c3_cylinder_large()
    M = hz.Matrix.from_csr(A, c64=True)
    bd = torch.as_tensor(b).to("cuda")
    out = {"workload": "C3 jittered P1-FEM cylinder nr=60 ntheta=128 nz=256 k=20 (%d unknowns, %d nonzeros)"
                       % (A.n, A.nnz), "iteration_budget": iters}
    for key, kw in (("binary64", dict(mode="fp64")), ("mixed", dict(mode="mixed"))):
        hz.zsolve(M, bd, tol=1e-10, maxit=2, **kw)          # graph capture
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, info = hz.zsolve(M, bd, tol=1e-10, maxit=iters, **kw)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        out[key] = {"s": ms / 1e3, "iters": info.iters, "iter_us": 1e3 * ms / max(info.iters, 1),
                    "status": info.status_name, "relres_true": info.relres_true,
                    "outer": getattr(info, "outer", None)}
    M.close()
    return out


def cpu_baseline_entry(A, b, iters):
    """The oracle's BiCGStab on the host cores: the plain single-thread
    build and the OpenMP build (fixed-order chunk sums) on every core this
    process may run on."""
    import oracle
    r1, dt1, it1 = cpu_oracle_rate(A, b, iters)
    cores = len(os.sched_getaffinity(0))
    out = {"value": r1, "unit": "GB/s", "cores": 1, "kind": "oracle",
           "sample": f"{it1} BiCGStab iterations of C2 ({dt1:.1f} s), single-thread build"}
    try:
        rN, dtN, itN = cpu_oracle_rate(A, b, iters, threads=cores)
        out["all_cores"] = {"value": rN, "unit": "GB/s", "cores": cores, "kind": "oracle (OpenMP build)",
                            "sample": f"{itN} BiCGStab iterations of C2 ({dtN:.1f} s)"}
    except Exception as e:   # no OpenMP runtime on this host
        out["all_cores"] = {"unavailable": str(e)[:200]}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hz", choices=["hz", "reference"])
    ap.add_argument("--maxit", type=int, default=1000)
    ap.add_argument("--arith", default="fp64", choices=["ff", "fp64"],
                    help="fp64: binary64 arithmetic (the paper's); ff: the double-float path")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the labelled double-float entry beside a binary64 line")
    # the oracle runs ~30 ms per C2 iteration on one Grace core: 500
    # iterations are ~15 s of CPU work, 200 per reference step ~6 s
    ap.add_argument("--ref-iters", type=int, default=200)
    ap.add_argument("--cpu-iters", type=int, default=500)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the mixed / batched / double-float comparison on the C4 sweep")
    ap.add_argument("--c4-subset", action="store_true",
                    help="compare on 32 C4 systems (the boxes and the smallest cylinder; default: all 64)")
    ap.add_argument("--compare-all", action="store_true",
                    help="compare also binary64 BiCGStab(4) and the double-float variants")
    ap.add_argument("--compare-maxit", type=int, default=3000)
    ap.add_argument("--c3", action="store_true",
                    help="also run the C3 precision configuration (mixed vs binary64 on 2M unknowns)")
    ap.add_argument("--spmv-only", action="store_true",
                    help="profiling aid: build C2, run three SpMV launches of the chosen "
                         "arithmetic (--arith, --group) and exit without timing")
    ap.add_argument("--kernel-case", default=None, choices=["spmv", "cspmv", "blas", "outer", "batched", "solve"],
                    help="profiling aid: run one small case of a kernel family and exit (see run_kernel_case)")
    ap.add_argument("--solve-method", default="bicgstab", choices=["bicgstab", "tfqmr", "bicgstabl"],
                    help="--kernel-case solve: the Krylov method (bicgstabl with l = 4)")
    ap.add_argument("--solve-mode", default="fp64", choices=["fp64", "mixed"],
                    help="--kernel-case solve: plain binary64 or mixed precision")
    ap.add_argument("--precond", default="none", choices=["none", "jacobi"],
                    help="--kernel-case solve: right preconditioner")
    ap.add_argument("--group", type=int, default=4, help="lanes per row of the CSR-vector kinds")
    ap.add_argument("--spmv", default=None, choices=["csr", "sell", "ff", "sellff", "ffflat", "fftma", "flat64", "flat64p"],
                    help="force an SpMV variant (default: the handle's own choice)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.spmv_only:
        return run_spmv_only(args)
    if args.kernel_case:
        return run_kernel_case(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import paper_2112_06465_gb300 as hz
    from paper_2112_06465_gb300 import hz as hzmod

    A, b = build_workload()
    rp = torch.as_tensor(A.rowptr).to(dev)
    cl = torch.as_tensor(A.col).to(dev)
    vl = torch.as_tensor(A.val).to(dev)
    bd = torch.as_tensor(b).to(dev)
    ff = args.arith == "ff"
    M = hz.Matrix(rp, cl, vl, ff=ff)
    if args.spmv:
        M.set_spmv(args.spmv, args.group)
    xd = torch.zeros_like(bd)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---------------- device-resident solve steps: every step is the whole
    # solve from x0 = 0 (x0_zero: xd only receives the result)
    for _ in range(args.warmup):
        hz.zsolve(M, bd, x=xd, tol=1e-10, maxit=args.maxit, x0_zero=True)
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    infos = []
    barrier()
    with ClockSampler(local) as clk:
        for e0, e1 in ev:
            e0.record(stream)
            _, info = hz.zsolve(M, bd, x=xd, tol=1e-10, maxit=args.maxit, x0_zero=True)
            e1.record(stream)
            infos.append(info)
        barrier()
    step_ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    total_ms = sum(step_ms)
    iters = [i.iters for i in infos]
    my_bytes = sum(solve_bytes(A.n, A.nnz, it) for it in iters)
    t_max, all_bytes = job_totals(total_ms, my_bytes, world, dev)
    value = all_bytes / (t_max / 1e3) / 1e9

    # ---------------- end to end through the public API with host buffers
    h_rp = torch.as_tensor(A.rowptr).pin_memory()
    h_cl = torch.as_tensor(A.col).pin_memory()
    h_vl = torch.as_tensor(A.val).pin_memory()
    h_b = torch.as_tensor(b).pin_memory()
    h_x = torch.empty_like(h_b).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in (h_rp, h_cl, h_vl, h_b))
    d2h = h_x.numel() * h_x.element_size()
    e2e_times, e2e_bytes = [], 0
    for k in range(args.warmup + args.steps):
        barrier()
        t0 = time.perf_counter()
        d_rp = h_rp.to(dev, non_blocking=True)
        d_cl = h_cl.to(dev, non_blocking=True)
        d_vl = h_vl.to(dev, non_blocking=True)
        d_b = h_b.to(dev, non_blocking=True)
        M2 = hz.Matrix(d_rp, d_cl, d_vl, ff=ff)
        if args.spmv:
            M2.set_spmv(args.spmv, args.group)
        x2, inf2 = hz.zsolve(M2, d_b, tol=1e-10, maxit=args.maxit)
        h_x.copy_(x2, non_blocking=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        M2.close()
        if k >= args.warmup:
            e2e_times.append(dt)
            e2e_bytes += solve_bytes(A.n, A.nnz, inf2.iters)
    e2e_t, e2e_bytes = job_totals(sum(e2e_times), e2e_bytes, world, dev)
    e2e_value = e2e_bytes / e2e_t / 1e9

    # ---------------- roofline of the dominant kernel: the SpMV core
    # Every launch is preceded by a 1 GiB write (flushes the 129 MB L2 and
    # keeps the GPU busy while the host enqueues the next launch, so host
    # launch latency never lands between the events); all launches are
    # enqueued before the one synchronisation.
    props = M.props()
    line_roof = spmv_roofline(hz, torch, M, A, stream, props["spmv_kind"])

    launches = sum(4 + 6 * it for it in iters)   # start: x0, r = b - A x; per iteration F1..F5 and the loop guard; exit: true residual, copy-out
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[args.arith], "data": "synthetic",
        "config": workload_config(A, args.maxit, args.arith, iters[0], infos[-1].status_name),
        "solve": {"iters_per_step": iters, "status": [i.status_name for i in infos],
                  "relres_true": infos[-1].relres_true, "s_per_solve": t_max / args.steps / 1e3,
                  "iter_us": 1e3 * t_max / args.steps / max(iters[0], 1),
                  "spmv_variant": {"kind": props["spmv_kind"], "group": props["group"],
                                   "name": SPMV_KINDS.get(props["spmv_kind"])}},
        "e2e": {"value": e2e_value, "unit": "GB/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "roofline": line_roof,
        "clocks": clk.summary(),
        "gpu_launches": launches,
    }
    if rank == 0 and not ff and not args.no_secondary:
        line["double_float"] = double_float_entry(hz, torch, A, rp, cl, vl, bd, args, stream)
    if rank == 0 and not args.no_compare:
        line["compare"] = compare_modes(hz, torch, not args.c4_subset, args.compare_maxit, args.compare_all)
        line["spmv_h1"] = spmv_h1(hz, torch, stream)
        line["spmv_c64_c2"] = spmv_c64_c2(hz, torch, A, stream)
        line["adjoint_c5"] = adjoint_c5(hz, torch, stream)
        line["blas_sweep"] = blas_sweep(hz, torch, stream)
    if rank == 0 and args.c3:
        line["c3_precision"] = c3_precision(hz, torch, stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_entry(A, b, args.cpu_iters)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
