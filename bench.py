#!/usr/bin/env python3
"""Headline benchmark: factorization seconds and solve RHS/s of lambda I + K~
at N = 2^20 (the scale workload: d = 28 points on a 6-D linear manifold, h = 1,
lambda = 1, m = 1024, s_max = 256, tau = 1e-4, one right-hand side), mixed
precision against the plain FP64 GPU path.

One step = the whole hot path on the mixed path: ball tree, skeletonization
(sampling, FP64 ID), factorization (leaf Cholesky, V blocks, reduced systems,
telescoping) and the solve of the right-hand side with its residual check.
``value`` is the factorization time per step (tree + skeletons + Algorithm 2)
in seconds, max over ranks; ``solve_rhs_per_s`` and the FP64 comparison are
reported beside it.  Inputs (points, right-hand side) are resident in HBM when
the timed region starts; the factors are several GB, far larger than L2.

``--impl reference`` times the CPU oracle on a bounded sample of the same
workload instead (see ``cpu_baseline``).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "factorize sec & solve RHS/s at N=1M, rel err≤1e-5; mixed vs FP64 GPU path"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FP64_PEAK_TFLOPS = 1.25          # recipe's nominal FP64 rate (152 SMs, 2.07 GHz)
# DRAM bytes (read + write) of the leaf-level k_pivoted_qr launch at N = 2^20:
# ncu's dram__bytes_read.sum + dram__bytes_write.sum of that launch captured on
# the same recipe at N = 2^17 (128 leaves, 176 GB), scaled by the 8x leaf count
# (every leaf streams the same bytes); None while the kernel differs from the
# captured one.
QR_TRAFFIC_PER_LAUNCH = 1.41e12
QR_TRAFFIC_SRC = "ncu DRAM read+write of this launch at N=2^17 (128 leaves) x8"
ORACLE_SAMPLE_N = 8192           # points per oracle sample step


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return {"hbm_gbs": float(p["hbm_gbs"]), "bf16_tflops": float(p["bf16_tflops"]), "src": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "src": "fallback"}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self):
        self.rows, self.proc = [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self, gpu_index=0):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        return summarize_clocks(self.rows, gpu_index)


def summarize_clocks(rows, gpu_index=0):
    """Median SM clock, maximum SM clock and the throttle reasons seen in
    nvidia-smi samples (index, clocks.sm, clocks.max.sm, power.draw,
    clocks_event_reasons.active, then hw_slowdown, hw_thermal_slowdown,
    sw_thermal_slowdown, sw_power_cap as Active / Not Active) of one GPU."""
    rows = [r for r in rows if len(r) >= 9 and r[0] == str(gpu_index)]
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
            "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- algorithmic work
def qr_flops(ns, c, s):
    """FP64 flops the truncated pivoted Householder QR + P of one node
    executes: the initial column norms; per step k the Householder vector
    (2 (ns - k)), the reflector's dot products and update of the trailing
    columns (4 (ns - k)(c - k - 1)) and one downdate per trailing norm
    (2 (c - k - 1)); then T = R11^-1 R12 (s^2 (c - s)).  The kernel downdates
    the norms and evaluates one again only after it has fallen 16x (a few
    times per column over the whole QR), which this count leaves out."""
    f = 2.0 * ns * c
    for k in range(s):
        rows, cols = ns - k, c - k - 1
        f += 2.0 * rows + 4.0 * rows * cols + 2.0 * cols
    f += float(s) * s * (c - s)
    return f


def qr_flops_bound(ns, c, s):
    """The coarser work bound 4 |S'| c s of one node's ID (every step charged
    the full block)."""
    return 4.0 * ns * c * s


def level_qr_flops(sizes, ranks, N, D, n_samp, s_max, lo, hi, model=None):
    """QR flops per tree level (dict level -> flops), from realized ranks,
    with the executed-flop model (default) or another per-node model."""
    model = model or qr_flops
    out = {}
    for l in range(1, D + 1):
        tot = 0.0
        for a in range(1 << l, 1 << (l + 1)):
            n = hi[a] - lo[a]
            ns = min(n_samp, N - n)
            c = n if l == D else ranks[2 * a] + ranks[2 * a + 1]
            tot += model(ns, c, ranks[a])
        out[l] = tot
    return out


FP32_PEAK_TFLOPS = 80.5          # nominal: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz
FP32_INSTR_PEAK = 40.3e12         # FP32 lane instructions per second at the same clock
TF32_OVER_BF16 = 0.49             # recipe's nominal dense ratio (1.1 / 2.25 PFLOP/s)


def max_over_ranks(values, device=None):
    """Element-wise maximum of a list of numbers over all ranks of the default
    process group (the replicas' timings: the job ends with its slowest
    replica); the values themselves on a single process."""
    import torch
    import torch.distributed as td
    if not (td.is_available() and td.is_initialized()) or td.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return t.tolist()


def phase_work(p, D, lo, hi, ranks, n_samp):
    """Algorithmic work of one factorization (per phase) and of one solve
    sweep / one operator product, from the realized ranks.  Returns
    {phase: (kind, amount, per)} with kind in fp64 / fp32 / fp32i (FP32
    lane instructions, an estimate) / tf32 (tensor flops of 3xTF32) / hbm
    (bytes) and per in {"step", "sweep", "matvec"}."""
    N, d, s_max = p.N, p.d, p.s_max
    r = ranks
    per_level = level_qr_flops(None, ranks, N, D, n_samp, s_max, lo, hi)
    clus = [l for l in range(1, D) if (1 << l) <= 8]   # levels whose QR runs on thread-block clusters
    w = {"qr_leaf": ("fp64", per_level[D], "step"),
         "qr": ("fp64", sum(per_level[l] for l in range(1, D) if l not in clus), "step"),
         "qr_cluster": ("fp64", sum(per_level[l] for l in clus), "step")}
    ent = ventries = 0.0
    zoff = tel = zlu = zinv = 0.0
    chol = phat = 0.0
    b_leaf = b_cs = b_ru = b_z = 0.0
    m_leaf = m_cs = m_ru = 0.0
    for l in range(1, D + 1):
        for a in range(1 << l, 1 << (l + 1)):
            n = hi[a] - lo[a]
            ns = min(n_samp, N - n)
            c = n if l == D else r[2 * a] + r[2 * a + 1]
            ent += ns * c
            ventries += n * r[a ^ 1]
            b_cs += 4.0 * n * r[a ^ 1]
            b_ru += 4.0 * n * r[a]
            m_cs += 8.0 * n * r[a ^ 1]
            if l == D:
                chol += n ** 3 / 3.0
                phat += 2.0 * n * n * r[a]
                b_leaf += 4.0 * n * (n + 1)
                m_leaf += 8.0 * n * n
                m_ru += 8.0 * n * r[a]
    for a in range(1, 1 << D):
        cl, cr = 2 * a, 2 * a + 1
        nl, nr = hi[cl] - lo[cl], hi[cr] - lo[cr]
        z = r[cl] + r[cr]
        zoff += 3 * 2.0 * r[cl] * r[cr] * (nl + nr)
        zlu += 2.0 / 3.0 * z ** 3 + (2.0 * z * z * r[a] if a >= 2 else 0.0)
        if a < 128:  # levels with at most 64 nodes keep Z^-1 (the library's default)
            zinv += 2.0 * z ** 3
        if a >= 2:
            tel += 3 * 2.0 * (nl * r[cl] + nr * r[cr]) * r[a]
        b_z += 8.0 * z * z
    w.update({"eval_A": ("fp64", 3.0 * d * ent, "step"),
              "leaf_cholesky": ("fp32", chol, "step"), "leaf_phat": ("fp32", phat, "step"),
              "eval_V": ("fp32i", ventries * (21.0 * d + 70.0), "step"),
              "zoff": ("tf32", zoff, "step"), "telescope": ("tf32", tel, "step"), "z_lu": ("fp64", zlu, "step"),
              "z_inv": ("fp64", zinv, "step"),
              "solve_leaf": ("hbm", b_leaf, "sweep"), "solve_colsum": ("hbm", b_cs, "sweep"),
              "solve_rowupd": ("hbm", b_ru, "sweep"), "solve_zsolve": ("hbm", b_z, "sweep"),
              "matvec_leaf": ("hbm", m_leaf, "matvec"), "matvec_colsum": ("hbm", m_cs, "matvec"),
              "matvec_rowupd": ("hbm", m_ru, "matvec")})
    return w


def phase_rooflines(work, phase_ms, phase_launches, steps, peaks):
    """Achieved rate and fraction of the roofline per phase; the phase time is
    the sum of its launches' CUDA-event durations, which on the factorization's
    overlapped streams includes time spent sharing the SMs (a lower bound on
    each kernel's own fraction)."""
    sweeps = phase_launches.get("solve_leaf", 0) / max(steps, 1)
    mvs = phase_launches.get("matvec_leaf", 0) / max(steps, 1)
    peak = {"fp64": (FP64_PEAK_TFLOPS * 1e12, "TFLOP/s", 1e12, "nominal"),
            "fp32": (FP32_PEAK_TFLOPS * 1e12, "TFLOP/s", 1e12, "nominal"),
            "fp32i": (FP32_INSTR_PEAK, "Tinstr/s", 1e12, "nominal"),
            "tf32": (peaks["bf16_tflops"] * TF32_OVER_BF16 * 1e12, "TFLOP/s", 1e12,
                     "measured bf16 x nominal tf32/bf16"),
            "hbm": (peaks["hbm_gbs"] * 1e9, "GB/s", 1e9, "measured")}
    out = {}
    for ph, (kind, amount, per) in work.items():
        ms = phase_ms.get(ph, 0.0)
        if ms <= 0 or amount <= 0:
            continue
        count = steps * (1 if per == "step" else (sweeps if per == "sweep" else mvs))
        rate = amount * count / (ms * 1e-3)
        pk, unit, scale, src = peak[kind]
        out[ph] = {"bound": {"fp64": "alu", "fp32": "alu", "fp32i": "alu", "tf32": "tensor", "hbm": "hbm"}[kind],
                   "achieved": round(rate / scale, 3), "unit": unit, "peak": round(pk / scale, 2),
                   "frac": round(rate / pk, 4), "peak_src": src, "per_step": round(count / steps, 2)}
    return out


def tree_ranges(N, m):
    D = 0
    while (m << D) < N:
        D += 1
    lo = [0] * (2 << D)
    hi = [0] * (2 << D)
    lo[1], hi[1] = 0, N
    for a in range(1, 1 << D):
        n = hi[a] - lo[a]
        mid = lo[a] + n // 2
        lo[2 * a], hi[2 * a], lo[2 * a + 1], hi[2 * a + 1] = lo[a], mid, mid, hi[a]
    return D, lo, hi


def solve_bytes(N, D, ranks, lo, hi, tsize):
    """Algorithmic bytes of one solve sweep: the lower triangles of the leaf
    factors (read by the forward and the backward substitution), the V rows
    K(x_i, sib~) and the P^ rows of every level, and the FP64 LU of every Z."""
    b = 0.0
    for a in range(1 << D, 2 << D):
        n = hi[a] - lo[a]
        b += tsize * n * (n + 1)              # two triangular passes over n(n+1)/2 entries
    for l in range(1, D + 1):
        for a in range(1 << l, 1 << (l + 1)):
            n = hi[a] - lo[a]
            b += tsize * n * (ranks[a ^ 1] + ranks[a])
    for a in range(1, 1 << D):
        z = ranks[2 * a] + ranks[2 * a + 1]
        b += 8.0 * z * z
    return b


# ---------------------------------------------------------------- oracle (CPU) leg
def run_oracle_sample(n_points):
    import oracle
    from paper_1701_02324_gb300 import inputs
    oracle.build()
    X = inputs.linear_manifold(n_points, 28, 6, 0.01, 1701003)
    b = np.random.default_rng(1701003 + 17).standard_normal(n_points)
    t0 = time.perf_counter()
    o = oracle.Oracle(X, 1024)
    o.skeletonize(1.0, 1e-4, 256)
    o.factorize(1.0)
    tf = time.perf_counter() - t0
    t0 = time.perf_counter()
    o.solve(b)
    ts = time.perf_counter() - t0
    return tf, ts, o.D


def oracle_scale(n_sample, N=1 << 20, m=1024):
    """Work model of the method (Sec. III: T_f = O(s^2 N log N)): per level
    the work is proportional to N, so time scales with N * (levels + 1)."""
    Ds, _, _ = tree_ranges(n_sample, m)
    Df, _, _ = tree_ranges(N, m)
    return (N * (Df + 1)) / (n_sample * (Ds + 1))


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def oracle_scaling_check(sizes):
    """Times the oracle (tree + skeletonize + factorize, as it stands) once
    at each size of the scale recipe and compares the measured time ratios
    with the work model N * (levels + 1) that extrapolates the CPU baseline
    to N = 2^20."""
    rows = []
    for n in sizes:
        tf, ts, D = run_oracle_sample(n)
        rows.append({"N": n, "levels": D, "factorize_s": round(tf, 3), "solve_s": round(ts, 4)})
    base = rows[0]
    for r in rows:
        r["model_ratio"] = round(oracle_scale(base["N"], r["N"]), 3)
        r["measured_ratio"] = round(r["factorize_s"] / base["factorize_s"], 3)
    return {"oracle_scaling": rows, "cores": int(os.environ.get("OMP_NUM_THREADS", cpu_cores())),
            "model": "factorize time proportional to N * (levels + 1)"}


def reference_main(args, rank, world):
    if rank != 0:
        return
    if args.oracle_sizes:
        print(json.dumps(oracle_scaling_check([int(v) for v in args.oracle_sizes.split(",")])), flush=True)
        return
    scale = oracle_scale(ORACLE_SAMPLE_N)
    for _ in range(args.warmup):
        run_oracle_sample(ORACLE_SAMPLE_N)
    tfs, tss = [], []
    for _ in range(args.steps):
        tf, ts, _ = run_oracle_sample(ORACLE_SAMPLE_N)
        tfs.append(tf)
        tss.append(ts)
    tf = statistics.mean(tfs) * scale
    ts = statistics.mean(tss) * scale
    cores = int(os.environ.get("OMP_NUM_THREADS", cpu_cores()))
    sample = (f"oracle tree+skeletonize+factorize of N={ORACLE_SAMPLE_N} points of the same recipe "
              f"(h=1, lambda=1, m=1024, s_max=256, tau=1e-4), scaled by N*(levels+1) x{scale:.1f} to N=2^20 "
              f"(an extrapolation; the model is within 10% of measured oracle runs at N=2^17, and a whole "
              f"oracle run at N=2^20 on 16 Arm host cores measured 1309 s, 1.9x below the model)")
    line = {
        "impl": "reference", "metric": METRIC, "value": round(tf, 4), "unit": "s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * statistics.mean(tfs), 2),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "scale_N1048576_d28", "N": 1 << 20, "d": 28, "h": 1.0, "lambda": 1.0, "m": 1024,
                   "s_max": 256, "tau": 1e-4, "nrhs": 1, "precision": "fp64-cpu-oracle"},
        "solve_rhs_per_s": round(1.0 / ts, 4),
        "cpu_baseline": {"value": round(tf, 4), "unit": "s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(tf, 4), "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU leg
def gpu_main(args, rank, world):
    import torch

    import paper_1701_02324_gb300 as kf
    from paper_1701_02324_gb300 import _abi, inputs

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    lib = _abi.load()
    p = inputs.scale()
    X_host = np.ascontiguousarray(p.X)
    b_host = np.ascontiguousarray(p.B[:, 0])
    X = torch.from_numpy(X_host).to(dev)
    b = torch.from_numpy(b_host).to(dev)
    torch.cuda.synchronize()
    dist = world > 1

    def barrier():
        if dist:
            torch.distributed.barrier()

    gmres_iters = []
    # kernel variants picked by the library's autotuner on this workload
    # (untimed; the timed steps then use them, as a user would)
    tuned = {}
    if not args.no_autotune:
        tree_t = kf.Tree(X, p.m)
        for prec in (kf.KF_PREC_MIXED, kf.KF_PREC_FP64):
            if prec == kf.KF_PREC_FP64 and args.no_fp64:
                continue
            ch, ms = kf.autotune(tree_t, p.h, p.lam, p.tau, p.s_max, precision=prec,
                                 fp64_operator=(prec == kf.KF_PREC_MIXED))
            tuned[prec] = (ch, ms)
        del tree_t
    opt = lambda prec: tuned[prec][0] if prec in tuned else {}

    def step(prec, refined=None):
        """tree + factorize + solve.  Mixed path: FP64 operator kept and the
        solve refined by GMRES(--gmres-m) to eps_r <= --mixed-tol (at least the
        accuracy of the FP64 path's direct solve); FP64 path: direct solve.
        refined=False: mixed path without the FP64 operator and without
        refinement."""
        tree = kf.Tree(X, p.m)
        if prec == kf.KF_PREC_MIXED and refined is not False:
            F = kf.Factor(tree, p.h, p.lam, p.tau, p.s_max, precision=prec, fp64_operator=True,
                          refine_tol=args.mixed_tol, refine_max_iter=400, gmres_restart=args.gmres_m, sync_errors=False,
                          **opt(prec))
            ev = torch.cuda.Event(enable_timing=True)
            ev.record()
            x, inf = F.solve(b, info=True)
            gmres_iters.append(inf["iters"])
            return tree, F, ev, x
        F = kf.Factor(tree, p.h, p.lam, p.tau, p.s_max, precision=prec, fp64_operator=False, refine_max_iter=-1,
                      sync_errors=False, **opt(prec))
        ev = torch.cuda.Event(enable_timing=True)
        ev.record()
        x = F.solve(b)
        return tree, F, ev, x

    # warm-up (also loads and builds everything)
    for _ in range(args.warmup):
        tree, F, _, _ = step(kf.KF_PREC_MIXED)
        del F, tree
    torch.cuda.synchronize()

    # ---- timed region: mixed path -------------------------------------------
    clocks = ClockSampler()
    clocks.start()
    lib.kf_profile_enable(1)
    nph = len(_abi.PHASES)
    ms_ph = np.zeros(nph)
    ln_ph = np.zeros(nph, dtype=np.int64)
    lib.kf_profile_read(ms_ph.ctypes.data_as(ctypes_p()), ln_ph.ctypes.data_as(ctypes_p()), nph)
    barrier()
    torch.cuda.synchronize()
    launches0 = lib.kf_launch_count()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    fact_ms, solve_ms = [], []
    t_start.record()
    x_mixed = None
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e0.record()
        tree, F, e1, x = step(kf.KF_PREC_MIXED)
        e2 = torch.cuda.Event(enable_timing=True)
        e2.record()
        torch.cuda.synchronize()
        fact_ms.append(e0.elapsed_time(e1))
        solve_ms.append(e1.elapsed_time(e2))
        x_mixed = x
        ranks = F.ranks()
        del F, tree
    t_end.record()
    torch.cuda.synchronize()
    barrier()
    total_ms = t_start.elapsed_time(t_end)
    launches = lib.kf_launch_count() - launches0
    lib.kf_profile_read(ms_ph.ctypes.data_as(ctypes_p()), ln_ph.ctypes.data_as(ctypes_p()), nph)
    lib.kf_profile_enable(0)
    clk = clocks.stop(dev.index)

    # max over ranks
    fact_s = statistics.mean(fact_ms) / 1e3
    solve_s = statistics.mean(solve_ms) / 1e3
    ms_per_step = total_ms / args.steps
    fact_s, solve_s, ms_per_step = max_over_ranks([fact_s, solve_s, ms_per_step], dev)

    # ---- FP64 comparison leg (same workload, same skeletons) ---------------------
    fp64, unref, at_bar, vs_oracle = None, None, None, None
    if not args.no_fp64:
        def timed(prec, refined, nsteps):
            ff, fs, x = [], [], None
            for _ in range(nsteps):
                e0 = torch.cuda.Event(enable_timing=True)
                e0.record()
                tree, F, e1, x = step(prec, refined)
                e2 = torch.cuda.Event(enable_timing=True)
                e2.record()
                torch.cuda.synchronize()
                ff.append(e0.elapsed_time(e1))
                fs.append(e1.elapsed_time(e2))
                del F, tree
            return statistics.mean(ff) / 1e3, statistics.mean(fs) / 1e3, x
        timed(kf.KF_PREC_FP64, None, 1)  # warm
        f64_f, f64_s, x64 = timed(kf.KF_PREC_FP64, None, max(1, args.fp64_steps))
        un_f, un_s, xun = timed(kf.KF_PREC_MIXED, False, max(1, args.fp64_steps))
        # accuracy reference: the FP64 factorization refined by GMRES against the FP64 operator
        tree = kf.Tree(X, p.m)
        Fr = kf.Factor(tree, p.h, p.lam, p.tau, p.s_max, precision=kf.KF_PREC_FP64, fp64_operator=True,
                       refine_max_iter=20, refine_tol=1e-11, gmres_restart=20)
        xref, iref = Fr.solve(b, info=True)
        F64 = kf.Factor(tree, p.h, p.lam, p.tau, p.s_max, precision=kf.KF_PREC_FP64, fp64_operator=True,
                        refine_max_iter=-1)
        _, i64 = F64.solve(b, info=True)
        del Fr, F64, tree
        relf = lambda a: float(torch.linalg.norm(a - xref) / torch.linalg.norm(xref))
        fp64 = {"factorize_s": round(f64_f, 4), "solve_rhs_per_s": round(1.0 / f64_s, 2), "eps_r": i64["eps_r"],
                "rel_err_vs_reference": relf(x64)}
        unref = {"factorize_s": round(un_f, 4), "solve_rhs_per_s": round(1.0 / un_s, 2),
                 "rel_err_vs_reference": relf(xun),
                 "note": "mixed factors without the FP64 operator and without refinement"}
        mixed_rel = relf(x_mixed)
        # errors against the whole oracle run of this workload (a golden written by the oracle alone:
        # its refined solution at 2,000 seeded indices)
        gpath = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden", "scale_oracle.json")
        if os.path.exists(gpath):
            gold = json.load(open(gpath))
            if gold["N"] == p.N and gold["seed"] == p.seed and gold["s_max"] == p.s_max:
                gidx = torch.tensor(gold["index"], device=dev)
                gx = torch.tensor([float(v) for v in gold["x_refined"]], dtype=torch.float64, device=dev)
                relo = lambda a: float(torch.linalg.norm(a[gidx] - gx) / torch.linalg.norm(gx))
                vs_oracle = {"fp64_direct": relo(x64), "mixed_timed_solve": relo(x_mixed),
                             "fp64_refined_reference": relo(xref),
                             "what": "relative error at the 2,000 indices of the whole oracle run's refined "
                                     "solution (eps_r %.1e)" % gold["eps_r_refined"]}
        reference = {"what": "FP64 factorization + GMRES against the FP64 operator", "eps_r": iref["eps_r"],
                     "iters": iref["iters"]}
        # the mixed solve stopped at the metric's own bar instead (relative error <= 1e-5 against the
        # reference): GMRES to eps_r <= 1e-6, same factorization recipe
        tree = kf.Tree(X, p.m)
        Fb = kf.Factor(tree, p.h, p.lam, p.tau, p.s_max, precision=kf.KF_PREC_MIXED, fp64_operator=True,
                       refine_tol=1e-6, refine_max_iter=400, gmres_restart=args.gmres_m, sync_errors=False,
                       **opt(kf.KF_PREC_MIXED))
        Fb.solve(b)  # warm
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        xb_, ib = Fb.solve(b, info=True)
        e1.record()
        torch.cuda.synchronize()
        at_bar = {"refine_tol": 1e-6, "gmres_iters": ib["iters"], "eps_r": ib["eps_r"],
                  "solve_rhs_per_s": round(1e3 / e0.elapsed_time(e1), 2), "rel_err_vs_reference": relf(xb_)}
        if vs_oracle is not None:
            vs_oracle["mixed_at_1e-5"] = relo(xb_)
        del Fb, tree, xb_

    # ---- near-field sampling of S' (knn_kappa = 16): the same workload and metric ------
    # (factorization including the neighbour search; the mixed solve to the metric's
    # bar and to the timed solve's eps_r; the FP64 direct solve; errors against the
    # FP64 factorization of the same K~ refined by GMRES)
    near = None
    if not args.no_near:
        tree = kf.Tree(X, p.m)
        kn = dict(knn_kappa=args.knn_kappa)
        def fact_time(prec, **kw):
            ts = []
            for _ in range(2):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                F = kf.Factor(tree, p.h, p.lam, p.tau, p.s_max, precision=prec, sync_errors=False, **kn, **kw)
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            return F, min(ts) / 1e3
        def solve_time(F):
            # timed without the info record (which adds a residual evaluation); info from a second solve
            F.solve(b)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            x = F.solve(b)
            e1.record()
            torch.cuda.synchronize()
            _, inf = F.solve(b, info=True)
            return x, inf, e0.elapsed_time(e1) / 1e3
        Fr = kf.Factor(tree, p.h, p.lam, p.tau, p.s_max, precision=kf.KF_PREC_FP64, fp64_operator=True,
                       refine_max_iter=30, refine_tol=1e-12, gmres_restart=30, sync_errors=False, **kn)
        xr, ir = Fr.solve(b, info=True)
        del Fr
        relr = lambda a: float(torch.linalg.norm(a - xr) / torch.linalg.norm(xr))
        # a block of 16 right-hand sides: the FP32 sweep reads its factors once for all of them, the FP64
        # sweep is bound by its FP64 arithmetic, which grows with the block
        B16 = torch.from_numpy(inputs.rhs(p.N, 16, 1701003 + 33)).to(dev)

        def block_time(F, B=B16):
            F.solve(B)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            XB = F.solve(B)
            e1.record()
            torch.cuda.synchronize()
            return XB, e0.elapsed_time(e1) / 1e3
        # a block of 64: the FP64 direct sweep against the Richardson solve on factors whose
        # FP64-accurate operator runs on the tensor cores (tc_operator)
        B64 = torch.from_numpy(inputs.rhs(p.N, 64, 1701003 + 65)).to(dev)
        Fr16 = kf.Factor(tree, p.h, p.lam, p.tau, p.s_max, precision=kf.KF_PREC_FP64, fp64_operator=True,
                         refine_max_iter=30, refine_tol=1e-12, gmres_restart=30, sync_errors=False, **kn)
        Xr16 = Fr16.solve(B16)
        del Fr16
        rel16 = lambda A: float(torch.linalg.norm(A - Xr16) / torch.linalg.norm(Xr16))
        F64, f64_s = fact_time(kf.KF_PREC_FP64, fp64_operator=False, refine_max_iter=-1, **opt(kf.KF_PREC_FP64))
        x64, _, s64 = solve_time(F64)
        X64_16, s64_16 = block_time(F64)
        X64_64, s64_64 = block_time(F64, B64)
        ranks_n = F64.ranks()
        del F64
        Fm, fm_s = fact_time(kf.KF_PREC_MIXED, fp64_operator=True, refine_tol=1e-6, refine_max_iter=400,
                             gmres_restart=args.gmres_m, **opt(kf.KF_PREC_MIXED))
        xm, im, sm = solve_time(Fm)
        del Fm
        # x += M^-1 r steps against the FP64-accurate operator until the residual is at the bar
        Fs, _ = fact_time(kf.KF_PREC_MIXED, fp64_operator=True, refine_tol=args.near_rich_tol, refine_max_iter=20,
                          gmres_restart=-1, **opt(kf.KF_PREC_MIXED))
        xs_, is_, ss = solve_time(Fs)
        Xs16, ss16 = block_time(Fs)
        del Fs
        # the factors keep the BF16 digits of V and of the leaf blocks as well (one factorization:
        # two of these at once would hold some 260 GB)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        Ft = kf.Factor(tree, p.h, p.lam, p.tau, p.s_max, precision=kf.KF_PREC_MIXED, sync_errors=False,
                       fp64_operator=True, refine_tol=args.near_rich_tol, refine_max_iter=20, gmres_restart=-1,
                       tc_operator=True, **kn, **opt(kf.KF_PREC_MIXED))
        e1.record()
        torch.cuda.synchronize()
        ft_s = e0.elapsed_time(e1) / 1e3
        Xt16, st16 = block_time(Ft)
        Xt64, st64 = block_time(Ft, B64)
        del Ft
        Fu, _ = fact_time(kf.KF_PREC_MIXED, fp64_operator=False, refine_max_iter=-1, **opt(kf.KF_PREC_MIXED))
        xu, _, su = solve_time(Fu)
        del Fu, tree
        near = {"knn_kappa": args.knn_kappa, "knn_trees": 4, "knn_leaf": 512,
                "reference_eps_r": ir["eps_r"], "ranks_mean": float(np.mean(ranks_n[2:])),
                "fp64": {"factorize_s": round(f64_s, 4), "solve_rhs_per_s": round(1 / s64, 2),
                         "rel_err_vs_reference": relr(x64)},
                "mixed_at_1e-5": {"factorize_s": round(fm_s, 4), "solve_rhs_per_s": round(1 / sm, 2),
                                  "gmres_iters": im["iters"], "eps_r": im["eps_r"], "rel_err_vs_reference": relr(xm)},
                "mixed_richardson": {"refine_tol": args.near_rich_tol, "solve_rhs_per_s": round(1 / ss, 2),
                                     "steps": is_["iters"], "eps_r": is_["eps_r"], "rel_err_vs_reference": relr(xs_)},
                "mixed_unrefined": {"solve_rhs_per_s": round(1 / su, 2), "rel_err_vs_reference": relr(xu)},
                "block16": {"fp64_direct": {"solve_rhs_per_s": round(16 / s64_16, 2), "rel_err_vs_reference":
                                            rel16(X64_16)},
                            "mixed_richardson": {"solve_rhs_per_s": round(16 / ss16, 2), "rel_err_vs_reference":
                                                 rel16(Xs16)},
                            "mixed_richardson_tc_operator": {"solve_rhs_per_s": round(16 / st16, 2),
                                                             "rel_err_vs_reference": rel16(Xt16)},
                            "note": "16 seeded right-hand sides solved together"},
                "block64": {"fp64_direct": {"solve_rhs_per_s": round(64 / s64_64, 2)},
                            "mixed_richardson_tc_operator": {
                                "factorize_s": round(ft_s, 4), "solve_rhs_per_s": round(64 / st64, 2),
                                "rel_err_vs_fp64_direct": float(torch.linalg.norm(Xt64 - X64_64) /
                                                                torch.linalg.norm(X64_64))},
                            "note": "64 seeded right-hand sides; the FP64 direct solution is within ~1e-15 of "
                                    "the reference at this sampling"},
                "note": "S' half from the nodes' near-field lists (kappa nearest neighbours by randomized "
                        "projection trees), half uniform; factorization times include the neighbour search"}

    # ---- memory-lean W (row f2): P^ of the leaves only, T = Z^-1 P_c of every node ----------
    # (factor memory as the device bytes the factorization keeps; the solve is the mixed
    # sweep refined to the timed solve's eps_r; errors against the GMRES-refined FP64 reference)
    lean = None
    if not args.no_lean and not args.no_fp64:
        tree = kf.Tree(X, p.m)
        def lean_run(w):
            torch.cuda.synchronize()
            m0 = torch.cuda.memory_allocated()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            F = kf.Factor(tree, p.h, p.lam, p.tau, p.s_max, precision=kf.KF_PREC_MIXED, fp64_operator=True,
                          refine_tol=args.mixed_tol, refine_max_iter=400, gmres_restart=args.gmres_m,
                          sync_errors=False, w_recompute=w, **opt(kf.KF_PREC_MIXED))
            e1.record()
            torch.cuda.synchronize()
            gb = (torch.cuda.memory_allocated() - m0) / 1e9
            F.solve(b)
            e2 = torch.cuda.Event(enable_timing=True)
            e3 = torch.cuda.Event(enable_timing=True)
            e2.record()
            x = F.solve(b)
            e3.record()
            torch.cuda.synchronize()
            del F
            return {"factor_gb": round(gb, 2), "factorize_s": round(e0.elapsed_time(e1) / 1e3, 4),
                    "solve_rhs_per_s": round(1e3 / e2.elapsed_time(e3), 2), "rel_err_vs_reference": relf(x)}
        lean = {"standard": lean_run(False), "w_recompute": lean_run(True),
                "note": "mixed factors with the FP64 operator copy; GMRES(%d) to eps_r <= %g" % (args.gmres_m,
                                                                                                 args.mixed_tol)}
        del tree

    # ---- GMRES iterations of the mixed solve at other sampler seeds ------------------
    # (the default seed's K~ is the most ill-conditioned of those tried: its
    # iteration count moves with rounding-level changes of the FP32 factors)
    seed_study = None
    if not args.no_seed_study:
        tree = kf.Tree(X, p.m)
        rows = []
        for sd in (1, 2, 3):
            F = kf.Factor(tree, p.h, p.lam, p.tau, p.s_max, precision=kf.KF_PREC_MIXED, fp64_operator=True,
                          refine_tol=args.mixed_tol, refine_max_iter=400, gmres_restart=args.gmres_m,
                          sync_errors=False, seed=sd, **opt(kf.KF_PREC_MIXED))
            F.solve(b)  # warm
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            _, inf = F.solve(b, info=True)
            e1.record()
            torch.cuda.synchronize()
            rows.append({"seed": sd, "gmres_iters": inf["iters"], "eps_r": inf["eps_r"],
                         "solve_rhs_per_s": round(1e3 / e0.elapsed_time(e1), 2)})
            del F
        del tree
        seed_study = {"what": "mixed solve (GMRES to the same eps_r) at sampler seeds other than the default",
                      "runs": rows}

    # ---- end to end through the C ABI with host buffers ----------------------------
    e2e = None
    if not args.no_e2e:
        xh = np.empty_like(b_host)
        lib_t = []
        for _ in range(max(1, args.e2e_steps)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            tree = kf.Tree(torch.from_numpy(X_host), p.m)                  # host X: H2D inside
            F = kf.Factor(tree, p.h, p.lam, p.tau, p.s_max, precision=kf.KF_PREC_MIXED, fp64_operator=True,
                          refine_tol=args.mixed_tol, refine_max_iter=400, gmres_restart=args.gmres_m, sync_errors=False,
                          **opt(kf.KF_PREC_MIXED))
            xt = F.solve(torch.from_numpy(b_host))                         # host b -> host x
            xh[:] = xt.numpy()
            lib_t.append(time.perf_counter() - t0)
            del F, tree
        e2e = {"value": round(statistics.mean(lib_t), 4), "unit": "s",
               "h2d_bytes_per_step": int(X_host.nbytes + b_host.nbytes), "d2h_bytes_per_step": int(xh.nbytes),
               "note": "tree + factorize + solve, host X, b, x"}

    # ---- batched workload: 256 uneven problems, 64 RHS each, one graph launch each ----
    batched = None
    if not args.no_batched:
        probs = inputs.batched(args.batched_n, 64)
        trees_b = [kf.Tree(torch.from_numpy(q.X).to(dev), q.m) for q in probs]
        Bb = [torch.from_numpy(q.B).to(dev) for q in probs]
        hs, lams, taus = [q.h for q in probs], [q.lam for q in probs], [q.tau for q in probs]
        # kernel variants of the batch picked by the autotuner on its median-size problem (untimed)
        im = int(np.argsort([q.X.shape[0] for q in probs])[len(probs) // 2])
        tuned_b, tune_ms = kf.autotune(trees_b[im], hs[im], lams[im], taus[im], probs[im].s_max,
                                       precision=kf.KF_PREC_MIXED)
        tuned_b64, tune_ms64 = kf.autotune(trees_b[im], hs[im], lams[im], taus[im], probs[im].s_max,
                                           precision=kf.KF_PREC_FP64)
        def run_batched(prec):
            fb_ms, sb_ms = [], []
            for it in range(3):  # one warm-up pass, two timed
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e2 = torch.cuda.Event(enable_timing=True)
                e0.record()
                # mixed: solves refined as a batch to eps_r <= 1e-9 (the batched workload's bar is 1e-5 on the error)
                facs = kf.factorize_batched(trees_b, hs, lams, taus, probs[0].s_max, precision=prec,
                                            refine_tol=1e-9 if prec == kf.KF_PREC_MIXED else 0.0,
                                            tc_operator=prec == kf.KF_PREC_MIXED,
                                            **(tuned_b if prec == kf.KF_PREC_MIXED else tuned_b64))
                e1.record()
                xs, binf = kf.solve_batched(facs, Bb, info=True)
                e2.record()
                torch.cuda.synchronize()
                if it > 0:
                    fb_ms.append(e0.elapsed_time(e1))
                    sb_ms.append(e1.elapsed_time(e2))
                del facs
            return statistics.mean(fb_ms) / 1e3, statistics.mean(sb_ms) / 1e3, xs, binf

        fb, sb, xs, binf = run_batched(kf.KF_PREC_MIXED)
        fb64, sb64, xs64, _ = run_batched(kf.KF_PREC_FP64)
        beps = [r["eps_r"] for r in binf]
        biters = [r["iters"] for r in binf]
        errs = [float(torch.linalg.norm(a - c) / torch.linalg.norm(c)) for a, c in zip(xs, xs64)]
        npts = sum(q.X.shape[0] for q in probs)
        nr = len(probs) * 64
        batched = {"workload": f"batched_{len(probs)}_problems", "problems": len(probs), "points": int(npts),
                   "nrhs_each": 64,
                   "mixed": {"factorize_s": round(fb, 4), "solve_s": round(sb, 4), "rhs_per_s": round(nr / sb, 1),
                             "rel_err_vs_fp64": {"median": float(np.median(errs)), "max": float(np.max(errs)),
                                                 "problems_above_1e-5": int(sum(e > 1e-5 for e in errs))},
                             "eps_r": {"median": float(np.median(beps)), "max": float(np.max(beps)),
                                       "problems_above_1e-9": int(sum(e > 1e-9 for e in beps))},
                             "refine_iters": {"median": float(np.median(biters)), "max": int(np.max(biters))}},
                   "fp64": {"factorize_s": round(fb64, 4), "solve_s": round(sb64, 4), "rhs_per_s": round(nr / sb64, 1)},
                   "autotuned": {"chosen": tuned_b, "candidate_ms": [round(t, 3) for t in tune_ms],
                                 "fp64_chosen": tuned_b64, "fp64_candidate_ms": [round(t, 3) for t in tune_ms64],
                                 "candidates": "clusters x (tcgen05 256, tcgen05 128, CUDA cores), then one CTA "
                                               "per node x the same"},
                   "note": "factorize_batched (one CUDA-graph launch) and solve_batched: FP64 direct sweeps (one "
                           "graph launch); mixed sweeps refined as a batch to eps_r <= 1e-9 (two graph launches per "
                           "step, GMRES for problems that stall) against the FP64-accurate operator on the tensor "
                           "cores (tc_operator); the mixed error is per problem against the FP64 path's solution"}
        del xs, xs64, trees_b, Bb

    # ---- differentiation workload (N=2^18, d=54): factorize, solve, gradient ----------
    diff = None
    if not args.no_grad:
        pd = inputs.differentiation()
        Xd = torch.from_numpy(pd.X).to(dev)
        bd = torch.from_numpy(pd.B[:, 0]).to(dev)
        yd = torch.from_numpy(pd.extra["y"]).to(dev)
        treed = kf.Tree(Xd, pd.m)
        for it in range(2):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e2 = torch.cuda.Event(enable_timing=True)
            e3 = torch.cuda.Event(enable_timing=True)
            e0.record()
            Fd = kf.Factor(treed, pd.h, pd.lam, pd.tau, pd.s_max, precision=kf.KF_PREC_MIXED, fp64_operator=True,
                           refine_tol=args.mixed_tol, refine_max_iter=400, gmres_restart=args.gmres_m, sync_errors=False)
            e1.record()
            xd = Fd.solve(bd)
            e2.record()
            db, dl, dh = Fd.grad(xd, 2 * (xd - yd))
            e3.record()
            torch.cuda.synchronize()
            ranks_d = Fd.ranks()
            del Fd
        # accuracy (untimed): the FP64 factorization refined the same way
        Fr = kf.Factor(treed, pd.h, pd.lam, pd.tau, pd.s_max, precision=kf.KF_PREC_FP64, fp64_operator=True,
                       refine_tol=args.mixed_tol, refine_max_iter=400, gmres_restart=args.gmres_m, sync_errors=False)
        xr = Fr.solve(bd)
        dbr, dlr, dhr = Fr.grad(xr, 2 * (xr - yd))
        del Fr
        diff = {"workload": "differentiation_N262144_d54", "factorize_s": round(e0.elapsed_time(e1) / 1e3, 4),
                "solve_s": round(e1.elapsed_time(e2) / 1e3, 4), "grad_s": round(e2.elapsed_time(e3) / 1e3, 4),
                "dL_dlambda": dl, "dL_dh": dh, "rank_mean": float(np.mean(ranks_d[2:])),
                "rel_err_vs_fp64_refined": {
                    "x": float(torch.linalg.norm(xd - xr) / torch.linalg.norm(xr)),
                    "dL_db": float(torch.linalg.norm(db - dbr) / torch.linalg.norm(dbr)),
                    "dL_dlambda": abs(dl - dlr) / abs(dlr), "dL_dh": abs(dh - dhr) / abs(dhr)},
                "note": "mixed path; forward solve and adjoint refined by GMRES against the FP64-accurate operator "
                        "and its transpose, dK~/dh from FP64 coordinates; loss ||x - y||^2"}
        del xr, dbr
        del treed, Xd

    # ---- roofline of the dominant kernel ----------------------------------------
    peaks = load_peaks()
    D, lo, hi = tree_ranges(p.N, p.m)
    phase_ms = {n: float(ms_ph[i]) for i, n in enumerate(_abi.PHASES)}
    phase_launches = {n: int(ln_ph[i]) for i, n in enumerate(_abi.PHASES)}
    qr_total = phase_ms["qr"] + phase_ms["qr_leaf"] + phase_ms["qr_cluster"]
    dominant = "qr" if qr_total >= max(phase_ms.values()) else max(phase_ms, key=phase_ms.get)
    roof = None
    if dominant in ("qr", "qr_leaf") and phase_launches["qr_leaf"] > 0:
        # the leaf level's k_pivoted_qr launch (one CTA per leaf), the largest
        # single launch of the step; the other levels are phases qr and qr_cluster
        per_level = level_qr_flops(None, ranks, p.N, D, 2 * p.s_max, p.s_max, lo, hi)
        bound_level = level_qr_flops(None, ranks, p.N, D, 2 * p.s_max, p.s_max, lo, hi, model=qr_flops_bound)
        avg_ms = phase_ms["qr_leaf"] / phase_launches["qr_leaf"]
        per_launch = per_level[D] * args.steps / phase_launches["qr_leaf"]
        achieved = per_launch / (avg_ms * 1e-3) / 1e12
        achieved_bound = bound_level[D] * args.steps / phase_launches["qr_leaf"] / (avg_ms * 1e-3) / 1e12
        roof = {"kernel": "k_pivoted_qr, leaf level", "bound": "alu",
                "achieved": round(achieved, 4), "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": round(achieved / FP64_PEAK_TFLOPS, 4),
                "traffic": QR_TRAFFIC_PER_LAUNCH, "traffic_src": QR_TRAFFIC_SRC,
                "peak_src": "nominal FP64 (an FMA loop measured 1.20)",
                "work_model": "executed Householder flops, realized ranks",
                "work_per_launch": per_launch, "avg_launch_ms": round(avg_ms, 3),
                "frac_of_bound_model": round(achieved_bound / FP64_PEAK_TFLOPS, 4),
                "bound_model": "4 |S'| c s per node"}
    else:
        sb = solve_bytes(p.N, D, ranks, lo, hi, 4) * args.steps
        sweep_ms = sum(phase_ms[k] for k in ("solve_leaf", "solve_colsum", "solve_zsolve", "solve_rowupd"))
        achieved = sb / (sweep_ms * 1e-3) / 1e9 if sweep_ms > 0 else 0.0
        roof = {"kernel": f"dominant phase {dominant}", "bound": "hbm", "achieved": round(achieved, 1),
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4),
                "traffic": None}
    phase_ms_per_step = {k: round(v / args.steps, 3) for k, v in phase_ms.items() if v > 0}
    phase_roofs = phase_rooflines(phase_work(p, D, lo, hi, ranks, 2 * p.s_max), phase_ms, phase_launches,
                                  args.steps, peaks)

    # ---- CPU baseline (oracle, bounded sample) ------------------------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        tf_o, ts_o, _ = run_oracle_sample(ORACLE_SAMPLE_N)
        sc = oracle_scale(ORACLE_SAMPLE_N)
        cpu = {"value": round(tf_o * sc, 3), "unit": "s", "cores": int(os.environ.get("OMP_NUM_THREADS", cpu_cores())),
               "kind": "oracle",
               "sample": f"oracle tree+skeletons+factorization of N={ORACLE_SAMPLE_N}, {tf_o:.2f} s, x{sc:.0f} "
                         f"by N(levels+1) to 2^20 (extrapolated; a whole 2^20 run took 1309 s); "
                         f"solve {ts_o * sc:.2f} s/RHS",
               "solve_rhs_per_s": round(1.0 / (ts_o * sc), 4)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(fact_s, 4), "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_per_step, 2), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "scale_N1048576_d28", "N": p.N, "d": p.d, "h": p.h, "lambda": p.lam, "m": p.m,
                       "s_max": p.s_max, "tau": p.tau, "n_samp": 2 * p.s_max, "nrhs": 1,
                       "precision": "mixed: FP32 factors, tcgen05 3xTF32 products; FP64 ID, Z, T, operator, GMRES",
                       "parallelism": f"replicas x{world}", "l2": "working set > L2, no flush"},
            # the metric's comparison, as top-level scalars
            "solve_rhs_per_s": round(1.0 / solve_s, 2),
            "solve_note": f"FP32 sweep + GMRES({args.gmres_m}), FP64 operator, eps_r {args.mixed_tol:g}",
            "gmres_iters": float(np.mean(gmres_iters[-args.steps:])) if gmres_iters else None,
            "mixed_rel_err_vs_reference": mixed_rel if fp64 else None,
            "mixed_rel_err_vs_oracle": vs_oracle["mixed_timed_solve"] if vs_oracle else None,
            "fp64_rel_err_vs_oracle": vs_oracle["fp64_direct"] if vs_oracle else None,
            "mixed_solve_rhs_per_s_at_1e-5": at_bar["solve_rhs_per_s"] if at_bar else None,
            "mixed_rel_err_at_1e-5": at_bar["rel_err_vs_reference"] if at_bar else None,
            "fp64_factorize_s": fp64["factorize_s"] if fp64 else None,
            "fp64_solve_rhs_per_s": fp64["solve_rhs_per_s"] if fp64 else None,
            "fp64_rel_err_vs_reference": fp64["rel_err_vs_reference"] if fp64 else None,
            "mixed_unrefined_rel_err": unref["rel_err_vs_reference"] if unref else None,
            "reference": "FP64 factors + GMRES, eps_r %.1e" % reference["eps_r"]
                         if fp64 else None,
            "near_field": {  # near-field sampling (kappa neighbours per point), same points and right-hand side
                "factorize_s": [near["mixed_at_1e-5"]["factorize_s"], near["fp64"]["factorize_s"]],  # mixed, FP64
                "mixed_rhs_per_s_at_1e-5": near["mixed_at_1e-5"]["solve_rhs_per_s"],
                "mixed_rel_err_at_1e-5": near["mixed_at_1e-5"]["rel_err_vs_reference"],
                "richardson_rhs_per_s": near["mixed_richardson"]["solve_rhs_per_s"],
                "richardson_rel_err": near["mixed_richardson"]["rel_err_vs_reference"],
                "fp64_rhs_per_s": near["fp64"]["solve_rhs_per_s"],
                "unrefined_rel_err": near["mixed_unrefined"]["rel_err_vs_reference"],
                "block16_rhs_per_s": {"fp64": near["block16"]["fp64_direct"]["solve_rhs_per_s"],
                                      "mixed": near["block16"]["mixed_richardson"]["solve_rhs_per_s"],
                                      "mixed_tc": near["block16"]["mixed_richardson_tc_operator"]["solve_rhs_per_s"]},
                "block16_mixed_rel_err": near["block16"]["mixed_richardson"]["rel_err_vs_reference"],
                "block64_rhs_per_s": {"fp64": near["block64"]["fp64_direct"]["solve_rhs_per_s"],
                                      "mixed_tc": near["block64"]["mixed_richardson_tc_operator"]["solve_rhs_per_s"]},
                "block64_mixed_tc_rel_err": near["block64"]["mixed_richardson_tc_operator"]["rel_err_vs_fp64_direct"],
            } if near else None,
            "lean": {"factor_gb": [lean["standard"]["factor_gb"], lean["w_recompute"]["factor_gb"]],
                     "mixed_rhs_per_s": lean["w_recompute"]["solve_rhs_per_s"]} if lean else None,
            "batched": {"mixed_rhs_per_s": batched["mixed"]["rhs_per_s"], "fp64_rhs_per_s": batched["fp64"]["rhs_per_s"],
                        "mixed_max_rel_err_vs_fp64": batched["mixed"]["rel_err_vs_fp64"]["max"]} if batched else None,
            "ranks": {"mean": round(float(np.mean(ranks[2:])), 1), "max": int(np.max(ranks))},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clk,
            "peaks_src": peaks["src"],
        }
        detail = {
            "detail_of": METRIC, "workload": "scale_N1048576_d28",
            "phase_ms_per_step": phase_ms_per_step, "phase_rooflines": phase_roofs,
            "autotuned": {("mixed" if k == kf.KF_PREC_MIXED else "fp64"): {"chosen": v[0],
                          "candidate_ms": [round(t, 2) for t in v[1]]} for k, v in tuned.items()} or None,
            "fp64_path": fp64, "mixed_unrefined": unref, "mixed_solve_at_metric_bar": at_bar,
            "solve_seed_study": seed_study, "accuracy_reference": reference if fp64 else None,
            "vs_whole_oracle": vs_oracle,
            "near_field_sampling": near,
            "memory_lean_w": lean,
            "differentiation": diff, "batched": batched,
        }
        print(json.dumps(round_errors(line)), flush=True)
        # the per-phase and per-workload figures: one JSON line on stderr (and a file on request)
        print(json.dumps(detail), file=sys.stderr, flush=True)
        if args.detail_out:
            with open(args.detail_out, "w") as fh:
                json.dump(detail, fh, indent=1)


def round_errors(obj, key=""):
    """Relative errors to three significant figures in the one-line summary
    (nested groups included); everything else as it is."""
    if isinstance(obj, dict):
        return {k: round_errors(v, k) for k, v in obj.items()}
    if isinstance(obj, float) and "rel_err" in key:
        return float(f"{obj:.3g}")
    return obj


def once(args):
    """A single pass of the path at a chosen size, no timing: the command that
    profiler captures run."""
    import torch

    import paper_1701_02324_gb300 as kf
    from paper_1701_02324_gb300 import inputs
    p = inputs.scale(args.n)
    prec = kf.KF_PREC_MIXED if args.precision == "mixed" else kf.KF_PREC_FP64
    tree = kf.Tree(torch.from_numpy(p.X).cuda(), p.m)
    if prec == kf.KF_PREC_MIXED and not args.unrefined:  # the timed step's configuration
        F = kf.Factor(tree, p.h, p.lam, p.tau, p.s_max, precision=prec, fp64_operator=True, refine_tol=args.mixed_tol,
                      refine_max_iter=400, gmres_restart=args.gmres_m, sync_errors=False)
    else:
        F = kf.Factor(tree, p.h, p.lam, p.tau, p.s_max, precision=prec, refine_max_iter=-1, fp64_operator=False)
    x = F.solve(torch.from_numpy(p.B[:, 0]).cuda())
    torch.cuda.synchronize()
    print(f"once: N={p.N} precision={args.precision} |x|={float(torch.linalg.norm(x)):.6e}")


def ctypes_p():
    import ctypes
    return ctypes.c_void_p


def multi_rhs_case(tc_operator=False):
    """The scale recipe at N = 2^17 with near-field sampling, mixed factors with
    the FP64 operator copy and Z^-1 on the levels of at most 8 nodes (so that
    levels 4-6 solve their reduced systems by LU): one operator product and one
    direct sweep of 16 right-hand sides, twice (the case the profiles of the
    several-right-hand-side kernels are taken on).  tc_operator: the factors
    also keep the BF16 digits of V, and the product's V pass runs on the
    tensor cores."""
    import torch
    import paper_1701_02324_gb300 as kf
    from paper_1701_02324_gb300 import inputs
    p = inputs.scale(1 << 17)
    tree = kf.Tree(torch.from_numpy(p.X).cuda(), p.m)
    F = kf.Factor(tree, p.h, p.lam, p.tau, p.s_max, precision=kf.KF_PREC_MIXED, fp64_operator=True,
                  refine_max_iter=-1, knn_kappa=16, sync_errors=False, zinv_max_nodes=8, tc_operator=tc_operator)
    B = torch.from_numpy(inputs.rhs(p.N, 16, 5)).cuda()
    for _ in range(2):
        Y = F.matvec(B)
        X = F.solve(B)
    torch.cuda.synchronize()
    print(json.dumps({"multi_rhs_case": "done", "norm_Y": float(Y.norm()), "norm_X": float(X.norm())}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="kf", choices=["kf", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-grad", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-seed-study", action="store_true", help="skip the mixed solve at other sampler seeds")
    ap.add_argument("--no-near", action="store_true", help="skip the near-field sampling variant of the workload")
    ap.add_argument("--no-lean", action="store_true", help="skip the memory-lean W variant of the workload")
    ap.add_argument("--knn-kappa", type=int, default=16, help="neighbours per point of the near-field variant")
    ap.add_argument("--near-rich-tol", type=float, default=2e-6,
                    help="residual target of the near-field variant's x += M^-1 r solve")
    ap.add_argument("--no-autotune", action="store_true", help="default kernel variants instead of kf_autotune's")
    ap.add_argument("--batched-n", type=int, default=256, help="problems of the batched workload")
    ap.add_argument("--once", action="store_true",
                    help="one tree + factorize + solve of the scale recipe and exit (for profilers)")
    ap.add_argument("--n", type=int, default=1 << 20, help="number of points of the scale recipe")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--gmres-m", type=int, default=50, help="GMRES restart length of the mixed solve")
    ap.add_argument("--mixed-tol", type=float, default=1e-9,
                    help="GMRES target eps_r of the mixed solve (the FP64 direct solve reaches about 1e-8)")
    ap.add_argument("--unrefined", action="store_true", help="--once: mixed factors without the FP64 operator or GMRES")
    ap.add_argument("--oracle-sizes", default=None,
                    help="--impl reference: time the oracle once at each of these comma-separated sizes of the "
                         "scale recipe and compare with the extrapolation model")
    ap.add_argument("--detail-out", default=None, help="also write the per-phase / per-workload details to this file")
    ap.add_argument("--multi-rhs-case", action="store_true",
                    help="run the small case the several-right-hand-side kernels are profiled on and exit")
    ap.add_argument("--tc-operator", action="store_true",
                    help="--multi-rhs-case: factors with the BF16 digits of V (tensor-core V pass)")
    args = ap.parse_args()
    if args.once:
        once(args)
        return
    if args.multi_rhs_case:
        multi_rhs_case(args.tc_operator)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        reference_main(args, rank, world)
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    gpu_main(args, rank, world)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
