#!/usr/bin/env python
"""Benchmark: fast SVT (Alg. 6) iterations/s on a 138,000 x 27,000 rating
matrix with 2e7 entries (1.8e7 observed, 10% held out), plus rSVD-BKI ms at
2e7 nnz (k = 50, s = 10, p = 3).

A step is one outer SVT iteration (rSVD-BKI or a recycled SVD of the sparse
iterate, rank decision, shrink, fused evaluation on Phi and update of Y).
Inputs are synthetic, generated by ``mc_synth.ratings`` (Zipf(1.1) rows and
columns, half-star values of a rank-20 model plus noise), and stay resident in
HBM across steps; they exceed L2 (CSR + CSC + values ~ 0.37 GB), so no flush
is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The timed steps run with CUDA events around the sparse products only (the
roofline's kernel); the per-class breakdown (``timing_ms``) comes from as
many further steps, since events around every launch would slow the step.
Prints one JSON line (rank 0).  ``--impl reference`` times the float64 CPU
oracle (the only other implementation of this method here) on the same
workload on the host cores.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import mc_synth  # noqa: E402

M_ROWS, N_COLS, N_PAIRS, HOLDOUT, SEED = 138_000, 27_000, 20_000_000, 0.1, 0
# Step size: 1.2/rho (the usual SVT choice) makes the iteration diverge on this
# Zipf pattern, whose heaviest rows and columns are fully observed; a constant
# delta below 2 (the bound under which SVT's fixed-point map contracts) is used.
DELTA = 1.9
# Threshold tau = 5n with n the column count (Sec. II.C); Omega of every
# rSVD-BKI starts with the previous right singular block (recycle = 3).
TAU = 5.0 * N_COLS
RECYCLE = 3
# The timed window starts after PREP_ITERS iterations from Y^0, when the rank
# has grown to about 47 (the regime of a long solve); the iterations before it
# prepare the state and are not timed.
PREP_ITERS = 400
K_BKI, S_OVER, P_BKI = 50, 10, 3
HBM_FALLBACK_GBS = 6800.0
# Serving: a bounded sample of the Poisson job stream (m, n log-uniform in
# [256, 8192], 5-50% observed, rank 5-50), submitted at its arrival times.
SERVE_JOBS, SERVE_RATE, SERVE_SLOTS, SERVE_IMAX = 32, 16.0, 8, 300


def workload_config():
    return {"workload": f"rating-svt {M_ROWS}x{N_COLS} {N_PAIRS:.0e} pairs (10% held out), iterations after "
                        f"{PREP_ITERS}",
            "m": M_ROWS, "n": N_COLS, "nnz_observed": int(N_PAIRS * (1 - HOLDOUT)), "nnz_total": N_PAIRS,
            "tau": "5n", "delta": DELTA, "recycle": "Omega warm-started with the previous V (every SVD a fresh rSVD-BKI)",
            "p0": 3, "s": S_OVER, "eps": 1e-4, "prep_iterations": PREP_ITERS,
            "rsvd_bki": {"k": K_BKI, "s": S_OVER, "p": P_BKI},
            "l2": "inputs exceed L2 (no flush)", "seed": SEED}


def load_workload():
    """The rating workload, cached under the temp dir (generation takes ~25 s)."""
    key = hashlib.sha1(f"{M_ROWS},{N_COLS},{N_PAIRS},{HOLDOUT},{SEED},v1".encode()).hexdigest()[:12]
    path = os.path.join(tempfile.gettempdir(), f"mc_bench_{key}.npz")
    if os.path.exists(path):
        z = np.load(path)
        o = mc_synth.Observed(M_ROWS, N_COLS, z["row_ptr"], z["col"], z["val"], z["test_rows"], z["test_cols"],
                              z["test_val"])
        return o
    o = mc_synth.ratings(M_ROWS, N_COLS, N_PAIRS, holdout=HOLDOUT, seed=SEED)
    tmp = path + f".{os.getpid()}.npz"
    np.savez(tmp, row_ptr=o.row_ptr, col=o.col, val=o.val, test_rows=o.test_rows, test_cols=o.test_cols,
             test_val=o.test_val)
    os.replace(tmp, path)
    return o


def full_matrix(o):
    """All 2e7 pairs (observed + held out) as CSR: the standalone rSVD input."""
    rows = np.concatenate([o.rows, o.test_rows])
    cols = np.concatenate([o.col.astype(np.int64), o.test_cols])
    vals = np.concatenate([o.val, o.test_val])
    return mc_synth.to_csr(o.m, o.n, rows, cols, vals)


class Clocks:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"mc_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sms.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sms) if sms else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sms)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return HBM_FALLBACK_GBS, "fallback"


def committed_traffic(kernel_file: str):
    """DRAM traffic of the SpMM from the committed ncu summary, if the kernel's
    source region is unchanged since it was taken."""
    path = os.path.join(ROOT, "profiles", "spmm_dram_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        src = open(os.path.join(ROOT, "paper_1810_06860_gb300", "csrc", kernel_file)).read()
        a = src.index("// --------------------------------------------------------------- products ---")
        b = src.index("// Same work split with a BF16 panel")
        if d.get("source_sha1") != hashlib.sha1(src[a:b].encode()).hexdigest():
            return None
        return d
    except (OSError, ValueError, KeyError):
        return None


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(t_ms: float, world: int, device: str = "cuda") -> float:
    """The slowest rank's time (the job's time): replicas run independently and
    meet only here, after the timed region."""
    if world <= 1:
        return t_ms
    import torch
    import torch.distributed as dist

    tt = torch.tensor([t_ms], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_rate(units_per_rank: int, world: int, t_ms: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / (t_ms / 1e3)


def svt_params(mc, o, precision: int = 0):
    return mc.params(tau=TAU, delta=DELTA, eps=1e-4, recycle=RECYCLE, seed=SEED, precision=precision)


def early_params(mc, o):
    """The first iterations of a solve with tau = 5 sqrt(mn) and the paper's
    strategy 1 (rank 2-3): the low-rank regime, reported beside the window."""
    return mc.params(tau=5.0 * math.sqrt(o.m * o.n), delta=DELTA, eps=1e-4, recycle=1, i_reuse=50, q_reuse=10,
                     seed=SEED)


def oracle_window_shape():
    """(k, p) of the oracle's iterations in the timed window, from its stored
    trajectory (tests/golden/rating_svt_oracle.json); None if absent."""
    path = os.path.join(ROOT, "tests", "golden", "rating_svt_oracle.json")
    try:
        with open(path) as f:
            h = json.load(f)["history"]
    except (OSError, ValueError, KeyError):
        return None
    win = [x for x in h if x["i"] > PREP_ITERS]
    if not win:
        return None
    return int(round(statistics.median(x["k"] for x in win))), int(round(statistics.median(x["p"] for x in win)))


def oracle_iteration_seconds(o, k: int, p: int, rows_frac: float = 1.0, reps: int = 1):
    """Seconds of one float64 oracle Alg. 6 iteration of the window's shape:
    one rSVD-BKI (Alg. 5) at rank k with p Krylov steps and a warm-started
    Omega, the shrink, the evaluation on Phi, the error and the update of Y,
    on the oracle's own Y^0 (the cost of an iteration does not depend on the
    values of Y).  rows_frac < 1 runs it on the leading rows only (a bounded
    sample: row ids are a random permutation of the Zipf ranks)."""
    from oracle import rsvd as orsvd
    from oracle import svt as osvt
    from oracle.philox import omega

    m = int(round(o.m * rows_frac))
    rp = o.row_ptr[:m + 1]
    nnz = int(rp[-1])
    A = orsvd.as_csr64(m, o.n, rp, o.col[:nnz], o.val[:nnz])
    Mv = A.data.copy()
    rows = np.repeat(np.arange(m), np.diff(rp))
    cols = o.col[:nnz].astype(np.int64)
    Y = A.copy()
    Y.data = 3.0 * DELTA * Mv
    times = []
    for rep in range(reps):
        Om = omega(o.n, k + S_OVER, SEED, 1 + rep)
        t0 = time.perf_counter()
        U, S, V, Q = orsvd.rsvd_bki(Y, k, p, S_OVER, Om=Om)
        r = max(1, min(k - 1, S.size))  # the window's rank: r_{i-1} = k - 1
        Us = U[:, :r] * (S[:r] - TAU)
        x = osvt.sample_lowrank(rows, cols, Us, V[:, :r])
        _err = float(np.linalg.norm(x - Mv)) / float(np.linalg.norm(Mv))
        Y.data = Y.data + DELTA * (Mv - x)
        times.append(time.perf_counter() - t0)
    return float(np.median(times)), m, nnz


def run_ours(args, rank, world, local):
    import torch

    import paper_1810_06860_gb300 as mc

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    mc.load()
    o = load_workload()
    stream = torch.cuda.Stream()
    # ---- rSVD-BKI at 2e7 nnz ------------------------------------------------
    rp, ci, va = full_matrix(o)
    hb = mc.Handle(o.m, o.n, rp, ci, va, stream=stream)
    for i in range(3):
        hb.rsvd_bki(K_BKI, S_OVER, P_BKI, seed=SEED, call_id=i, device=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nb = 20
    e0.record(stream)
    for i in range(nb):
        hb.rsvd_bki(K_BKI, S_OVER, P_BKI, seed=SEED, call_id=100 + i, device=True)
    e1.record(stream)
    torch.cuda.synchronize()
    bki_ms = e0.elapsed_time(e1) / nb
    hb.timing_enable(True)
    hb.rsvd_bki(K_BKI, S_OVER, P_BKI, seed=SEED, call_id=200, device=True)
    bki_tm = {k: round(v["ms"], 3) for k, v in hb.timing_read().items()}
    hb.timing_enable(False)
    # the other randomized SVDs on the same matrix (Sec. V.A, Table I): rSVD-PI
    # (Alg. 4) and basic rSVD (Alg. 1, orthonormalised after every product),
    # each at p = 0 and at the same p as rSVD-BKI
    other_ms = {}
    for name, fn, pp in (("rsvd_pi_ms", hb.rsvd_pi, P_BKI), ("rsvd_basic_ms", hb.rsvd_basic, P_BKI),
                         ("rsvd_pi_p0_ms", hb.rsvd_pi, 0), ("rsvd_basic_p0_ms", hb.rsvd_basic, 0)):
        for i in range(3):
            fn(K_BKI, S_OVER, pp, seed=SEED, call_id=300 + i, device=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for i in range(nb):
            fn(K_BKI, S_OVER, pp, seed=SEED, call_id=400 + i, device=True)
        e1.record(stream)
        torch.cuda.synchronize()
        other_ms[name] = round(e0.elapsed_time(e1) / nb, 3)
    hb.close()
    del rp, ci, va
    # ---- SVT iterations in the converged-rank window --------------------------
    h = mc.Handle(o.m, o.n, o.row_ptr, o.col, o.val, stream=stream)
    prm = svt_params(mc, o)
    infos = []
    t_prep = time.perf_counter()
    for _ in range(PREP_ITERS):
        infos.append(h.svt_step(prm))
    t_prep = time.perf_counter() - t_prep
    for _ in range(args.warmup):
        infos.append(h.svt_step(prm))
    torch.cuda.synchronize()
    # the timed region records events around the sparse products only (the
    # roofline's kernel); the per-class breakdown comes from a second pass
    h.timing_enable(2)
    lib = mc.load()
    l0 = lib.mc_launch_count()
    barrier(world)
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            infos.append(h.svt_step(prm))
        h.join()  # the last step's copy of Y into CSC order runs on the handle's second stream
        e1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    launches = lib.mc_launch_count() - l0
    t_ms = e0.elapsed_time(e1)
    tm = h.timing_read()
    h.timing_enable(False)
    t_ms = max_over_ranks(t_ms, world)
    value = job_rate(args.steps, world, t_ms)
    window = infos[-args.steps:]
    # held-out RMSE of X^i at the first iteration from the last timed one on
    # that is a multiple of 5 (the oracle's stored trajectory records the
    # RMSE every 5 iterations); the steps in between are not timed
    while infos[-1]["i"] % 5:
        infos.append(h.svt_step(prm))
    rmse_i = infos[-1]["i"]
    pred = h.sample(o.test_rows, o.test_cols)
    rmse = float(np.sqrt(np.mean((pred.astype(np.float64) - o.test_val) ** 2)))
    # per-class CUDA-event breakdown over the next iterations (not timed: the
    # events around every launch cost about 5 % of the step)
    h.timing_enable(True)
    for _ in range(args.steps):
        h.svt_step(prm)
    tm_all = h.timing_read()
    h.timing_enable(False)
    # the ceiling of the products' gathers: the same panel rows in the same
    # order with no arithmetic (mc_gather_rate), at the window's panel width
    kb_w = 4 * ((window[-1]["k"] + S_OVER + 3) // 4)
    gather_probe = {"csr": round(h.gather_rate(kb_w, trans=False), 1), "csc": round(h.gather_rate(kb_w, trans=True), 1)}
    h.close()
    oracle_rmse = None
    try:
        with open(os.path.join(ROOT, "tests", "golden", "rating_svt_oracle.json")) as f:
            oracle_rmse = json.load(f)["heldout_rmse"].get(str(rmse_i))
    except (OSError, ValueError, KeyError):
        pass
    # ---- the same workload's first iterations (rank 2-3), for contrast --------
    he = mc.Handle(o.m, o.n, o.row_ptr, o.col, o.val, stream=stream)
    pe = early_params(mc, o)
    for _ in range(args.warmup):
        he.svt_step(pe)
    torch.cuda.synchronize()
    e0.record(stream)
    early = [he.svt_step(pe) for _ in range(args.steps)]
    he.join()
    e1.record(stream)
    torch.cuda.synchronize()
    t_early = e0.elapsed_time(e1)
    he.close()
    early_line = {"value": round(args.steps * world / (t_early / 1e3), 3), "unit": "iters/s",
                  "iterations": f"{args.warmup + 1}..{args.warmup + args.steps}", "tau": "5*sqrt(m*n)",
                  "recycle": "Q (strategy 1), i_reuse=50, q_reuse=10", "k_last": early[-1]["k"],
                  "r_last": early[-1]["r"], "err_last": round(early[-1]["err"], 6)}
    # ---- roofline of the dominant kernel class (SpMM over CSR + CSC) --------
    sp_ms = tm["spmm"]["ms"] + tm["spmm_t"]["ms"]
    sp_bytes = tm["spmm"]["bytes"] + tm["spmm_t"]["bytes"]
    sp_launch = tm["spmm"]["launches"] + tm["spmm_t"]["launches"]
    peak, peak_kind = measured_peaks()
    achieved = (sp_bytes / 1e9) / (sp_ms / 1e3) if sp_ms > 0 else 0.0
    tr = committed_traffic("k_sparse.cu")
    roofline = {"bound": "hbm", "kernel": "spmm (Y X over CSR and Y^T X over CSC)", "achieved": round(achieved, 1),
                "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": round(tr["traffic_over_algorithmic"] * sp_bytes / max(sp_launch, 1)) if tr else None,
                "traffic_source": ("ncu DRAM bytes of the SpMM on a 1.6e7-pair case, scaled to this launch by "
                                   "algorithmic bytes" if tr else None),
                "algorithmic_bytes_per_launch": sp_bytes / max(sp_launch, 1),
                "lts_pct_of_peak": tr.get("l2_throughput_pct_of_peak") if tr else None,
                "l1_pct_of_peak": tr.get("l1_throughput_pct_of_peak") if tr else None,
                "share_of_step": round(sp_ms / t_ms, 3) if t_ms > 0 else None}
    gathered = {}
    for cls, key in (("spmm", "csr"), ("spmm_t", "csc")):
        c = tm[cls]
        if c["ms"] > 0:
            gathered[key] = round(c["launches"] * o.nnz * kb_w * 4 / 1e9 / (c["ms"] / 1e3), 1)
    roofline["gather"] = {"panel_width": kb_w, "probe_gbs": gather_probe, "spmm_gathered_gbs": gathered,
                          "frac_of_probe": {k: round(gathered[k] / gather_probe[k], 3) for k in gathered
                                            if gather_probe.get(k)},
                          "note": "gathered panel-row bytes per second of the products against the same gathers "
                                  "alone (mc_gather_rate)"}
    # the fused update's fraction of HBM, from the per-class pass
    sd = tm_all["sddmm"]
    if sd["ms"] > 0 and sd["launches"] > 0:
        sd_gbs = (sd["bytes"] / 1e9) / (sd["ms"] / 1e3)
        roofline["sddmm"] = {"achieved": round(sd_gbs, 1), "unit": "GB/s", "frac": round(sd_gbs / peak, 4),
                             "bytes_per_launch": round(sd["bytes"] / sd["launches"]),
                             "bytes_model": "20 per observed entry (column, row, M, Y read and write) + the "
                                            "factor panels; per-class pass after the timed steps"}
    # ---- mixed-precision form: same workload, bf16 Krylov panels ---------------
    hm = mc.Handle(o.m, o.n, o.row_ptr, o.col, o.val, stream=stream)
    prm_m = svt_params(mc, o, precision=1)
    for _ in range(PREP_ITERS + args.warmup):
        hm.svt_step(prm_m)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        hm.svt_step(prm_m)
    hm.join()
    e1.record(stream)
    torch.cuda.synchronize()
    t_mixed = e0.elapsed_time(e1)
    for _ in range(rmse_i - PREP_ITERS - args.warmup - args.steps):
        hm.svt_step(prm_m)  # to the iteration of the plain form's RMSE
    pred_m = hm.sample(o.test_rows, o.test_cols)
    rmse_m = float(np.sqrt(np.mean((pred_m.astype(np.float64) - o.test_val) ** 2)))
    hm.timing_enable(True)  # per-class breakdown over the following steps
    for _ in range(args.steps):
        hm.svt_step(prm_m)
    tm_mixed = {k: round(v["ms"], 3) for k, v in hm.timing_read().items()}
    hm.timing_enable(False)
    hm.close()
    rp, ci, va = full_matrix(o)
    hbm = mc.Handle(o.m, o.n, rp, ci, va, stream=stream)
    hbm.set_precision(1)
    for i in range(3):
        hbm.rsvd_bki(K_BKI, S_OVER, P_BKI, seed=SEED, call_id=i, device=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(nb):
        hbm.rsvd_bki(K_BKI, S_OVER, P_BKI, seed=SEED, call_id=100 + i, device=True)
    e1.record(stream)
    torch.cuda.synchronize()
    bki_mixed_ms = e0.elapsed_time(e1) / nb
    hbm.close()
    del rp, ci, va
    mixed = {"value": round(args.steps * world / (t_mixed / 1e3), 3), "unit": "iters/s",
             "rsvd_bki_ms": round(bki_mixed_ms, 3), "heldout_rmse": round(rmse_m, 5),
             "heldout_rmse_minus_plain": round(rmse_m - rmse, 6),
             "heldout_rmse_minus_oracle": round(rmse_m - oracle_rmse, 6) if oracle_rmse is not None else None,
             "form": "bf16 panels in the Krylov products, float32 orthonormalisation and final projection",
             "timing_ms": tm_mixed}
    # ---- end to end through the C ABI with host buffers -----------------------
    # Ingest from pinned host CSR (mc_create: copy in, validation, CSC build,
    # segment plans) and the window's steps, each followed by the step's
    # result (the factors of X^i) copied to pinned host memory; the
    # iterations that prepare the window's state run in between, untimed.
    h2d = (o.m + 1) * 8 + o.nnz * 8
    rp_h = torch.from_numpy(np.ascontiguousarray(o.row_ptr, np.int64)).pin_memory()
    ci_h = torch.from_numpy(np.ascontiguousarray(o.col, np.int32)).pin_memory()
    va_h = torch.from_numpy(np.ascontiguousarray(o.val, np.float32)).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hx = mc.Handle(o.m, o.n, rp_h, ci_h, va_h, stream=stream)
    torch.cuda.synchronize()
    t_ingest = time.perf_counter() - t0
    for _ in range(PREP_ITERS + args.warmup):
        hx.svt_step(prm)
    hx.join()
    torch.cuda.synchronize()
    cap = max(x["r"] for x in window) + 16
    us_h = torch.empty((o.m, cap), dtype=torch.float32).pin_memory()
    v_h = torch.empty((o.n, cap), dtype=torch.float32).pin_memory()
    s_h = torch.empty((cap,), dtype=torch.float32).pin_memory()
    d2h = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        hx.svt_step(prm)
        r_i = hx.factors_into(us_h, v_h, s_h)
        d2h += 4 * r_i * (o.m + o.n + 1)
    torch.cuda.synchronize()
    t_e2e = t_ingest + (time.perf_counter() - t0)
    hx.close()
    e2e = {"value": round(args.steps * world / t_e2e, 3), "unit": "iters/s",
           "h2d_bytes_per_step": int(h2d / args.steps), "d2h_bytes_per_step": int(d2h / args.steps),
           "ingest_s": round(t_ingest, 4),
           "note": "mc_create from pinned host CSR + the window's K steps with the factors of each X^i to pinned "
                   "host; the state-preparing iterations between them are not timed"}
    # ---- CPU oracle baseline (rank 0, N = 1 only) -----------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        kk, pp = window[-1]["k"], window[-1]["p"]
        secs, _m, _nnz = oracle_iteration_seconds(o, kk, pp)
        cpu = {"value": round(1.0 / secs, 4), "unit": "iters/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"one float64 oracle Alg. 6 iteration of the window's shape (fresh rSVD-BKI at k = {kk}, "
                         f"p = {pp}, warm-started Omega; shrink, evaluation on Phi, update) on the full workload"}
    # ---- image inpainting solve, plain and mixed --------------------------------
    image = run_image(mc, stream) if world == 1 else None
    table_i = run_table_i(mc, stream) if world == 1 else None
    # ---- serving form (last: it loads the GPU for minutes) ----------------------
    serving = run_serving(mc, SERVE_JOBS) if not args.no_serving and world == 1 else None
    last = window[-1]
    line = {"metric": "SVT iterations/s at 2e7 nnz (rating matrix 138,000 x 27,000)", "value": round(value, 3),
            "unit": "iters/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(t_ms / args.steps, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(workload_config(), parallelism=f"replicas x{world}",
                           timed_iterations=f"{window[0]['i']}..{window[-1]['i']}",
                           k_last=last["k"], r_last=last["r"], p_last=last["p"], err_last=round(last["err"], 6),
                           r_range=[min(x["r"] for x in window), max(x["r"] for x in window)],
                           heldout_rmse=round(rmse, 5), heldout_rmse_iteration=rmse_i,
                           heldout_rmse_oracle=round(oracle_rmse, 5) if oracle_rmse is not None else None,
                           prep_s=round(t_prep, 2)),
            "early_iterations": early_line, "image_inpainting": image, "rsvd_table_i": table_i,
            "rsvd_bki_ms": round(bki_ms, 3), "rsvd_bki_timing_ms": bki_tm, **other_ms, "mixed_precision": mixed, "serving": serving,
            "roofline": roofline, "e2e": e2e, "cpu_baseline": cpu,
            "clocks": clk.summary(), "gpu_launches": int(launches),
            "timing_ms": {k: round(v["ms"], 3) for k, v in tm_all.items()},
            "kernel_ms_per_step": round(sum(v["ms"] for v in tm_all.values()) / args.steps, 3),
            "timing_note": "per-class CUDA-event ms over the steps after the timed ones (same count); "
                           "kernel_ms_per_step is their sum per step, beside ms_per_step: events around every "
                           "launch serialise the classes and add their own cost, so it bounds the kernel time "
                           "from above"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def run_table_i(mc, stream):
    """Sec. V.A / Table I on a synthetic stand-in: basic rSVD (Alg. 1, an
    orthonormalisation after every product) against rSVD-PI (Alg. 4) at k =
    100, s = 10, p = 0 and 4, on a 45,115 x 45,115 Zipf rating matrix with 97
    entries per row and on two sparser copies (24 and 9 per row, entries
    dropped at random): CUDA-event ms per call and the approximation error
    ||A - A_k||_F / ||A||_F = sqrt(1 - sum sigma^2 / ||A||_F^2)."""
    import torch

    n0 = 45_115
    base = mc_synth.ratings(n0, n0, 97 * n0, seed=1)
    rng = np.random.default_rng(1)
    out = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name, per_row in (("matrix1", 97), ("matrix2", 24), ("matrix3", 9)):
        keep = np.ones(base.nnz, bool) if per_row == 97 else rng.random(base.nnz) < per_row / 97.0
        rows = np.repeat(np.arange(n0), np.diff(base.row_ptr))[keep]
        rp, ci, va = mc_synth.to_csr(n0, n0, rows, base.col[keep], base.val[keep])
        fro2 = float(np.sum(va.astype(np.float64) ** 2))
        res = {"nnz_per_row": round(len(va) / n0, 1)}
        with mc.Handle(n0, n0, rp, ci, va, stream=stream) as h:
            for p in (0, 4):
                for label, fn in (("basic", h.rsvd_basic), ("pi", h.rsvd_pi)):
                    for i in range(2):
                        fn(100, 10, p, seed=SEED, call_id=i, device=True)
                    torch.cuda.synchronize()
                    e0.record(stream)
                    for i in range(5):
                        _, S, _ = fn(100, 10, p, seed=SEED, call_id=10 + i, device=True)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    s2 = float(torch.sum(S.double() ** 2))
                    res[f"{label}_p{p}_ms"] = round(e0.elapsed_time(e1) / 5, 3)
                    res[f"{label}_p{p}_err"] = round(math.sqrt(max(0.0, 1.0 - s2 / fro2)), 4)
                res[f"speedup_p{p}"] = round(res[f"basic_p{p}_ms"] / res[f"pi_p{p}_ms"], 2)
        out[name] = res
    out["workload"] = "45,115 x 45,115 Zipf(1.1) rating matrix, k = 100, s = 10 (Sec. V.A, Table I stand-in)"
    return out


def run_image(mc, stream):
    """The image-inpainting solve (1024 x 1024 rank-40 image, half of the
    pixels observed; Alg. 6 with recycled left singular vectors from
    iteration 100) to its stopping tolerance, plain and mixed: solve time
    (CUDA events around all steps, including step 1's set-up), iterations,
    and the errors against the full image beside the oracle's stored solve."""
    import torch

    path = os.path.join(ROOT, "tests", "golden", "image_svt_oracle.json")
    with open(path) as f:
        ref = json.load(f)
    w = ref["workload"]
    o = mc_synth.smooth_image(w["size"], w["size"], w["rank"], sigma_px=w["sigma_px"], frac=w["frac"], seed=w["seed"])
    M = o.dense.astype(np.float64)
    observed = np.zeros(M.shape, bool)
    observed[np.repeat(np.arange(o.m), np.diff(o.row_ptr)), o.col] = True
    kw = dict(ref["params"])
    i_max = kw.pop("i_max")
    out = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name, precision in (("plain", 0), ("mixed", 1)):
        prm = mc.params(**kw, i_max=i_max, precision=precision)
        times = []
        for rep in range(3):  # the first solve warms up (autotuning, allocations)
            with mc.Handle.from_observed(o, stream=stream) as h:
                torch.cuda.synchronize()
                e0.record(stream)
                for _ in range(i_max):
                    info = h.svt_step(prm)
                    if info["converged"]:
                        break
                h.join()
                e1.record(stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
                Us, V, _ = h.factors()
        X = Us.astype(np.float64) @ V.astype(np.float64).T
        ms = statistics.median(times[1:])
        out[name] = {"iterations": info["i"], "converged": bool(info["converged"]), "solve_ms": round(ms, 3),
                     "iters_per_s": round(info["i"] / (ms / 1e3), 1), "rank": int(V.shape[1]),
                     "recovery_rel_err": round(float(np.linalg.norm(X - M) / np.linalg.norm(M)), 7),
                     "unobserved_rmse": round(float(np.sqrt(np.mean((X - M)[~observed] ** 2))), 5)}
    out["oracle"] = {"iterations": ref["iterations"], "recovery_rel_err": round(ref["recovery_rel_err"], 7),
                     "unobserved_rmse": round(ref["unobserved_rmse"], 5)}
    out["workload"] = (f"image {w['size']}x{w['size']} rank {w['rank']} (smooth factors, {w['sigma_px']} px), "
                       f"{w['frac']:.0%} observed; tau {kw['tau']:.0f}, delta {kw['delta']}, eps {kw['eps']}, "
                       f"recycled U from iteration {kw['i_reuse']} (q_reuse {kw['q_reuse']})")
    return out


def serving_sample(num_jobs: int):
    """The first num_jobs jobs of the 2,000-job Poisson stream (seed 0)."""
    spec = mc_synth.serving_jobs(2000, rate=SERVE_RATE, seed=SEED)[:num_jobs]
    obs = [mc_synth.lowrank_uniform(j["m"], j["n"], j["rank"], nobs=j["nobs"], seed=j["seed"]) for j in spec]
    return spec, obs


def run_serving(mc, num_jobs: int):
    """Solves/s and p50/p99 latency of the serving form on a sample of the
    job stream: each job is a whole SVT solve (tau = 5 sqrt(mn), delta =
    1.2/frac, eps = 1e-4, warm-started Omega, i_max = SERVE_IMAX), submitted
    at its arrival time."""
    spec, obs = serving_sample(num_jobs)
    prms = [mc.params(tau=5.0 * math.sqrt(o.m * o.n), delta=1.2 / j["frac"], eps=1e-4, i_max=SERVE_IMAX,
                      seed=j["seed"], recycle=3) for j, o in zip(spec, obs)]
    nnz = [int(o.row_ptr[-1]) for o in obs]
    l0 = mc.load().mc_launch_count()
    with mc.Server(max_active=SERVE_SLOTS) as srv:
        t0 = time.perf_counter()
        ids = []
        for j, o, p in zip(spec, obs, prms):
            dt = j["arrival"] - spec[0]["arrival"] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            ids.append(srv.submit_observed(o, p))
        res = [srv.wait(i, 3600) for i in ids]
        wall = time.perf_counter() - t0
        st = srv.stats()
    lat = np.array([r["latency_s"] for r in res])
    # jobs that do not reach eps (too few samples for their rank) run to i_max
    # and set the tail; converged and unconverged jobs are reported apart
    rec = np.array([bool(r["converged"]) for r in res])
    dof = np.array([j["rank"] * (j["m"] + j["n"] - j["rank"]) for j in spec])
    def pct(x, q):
        return round(float(np.percentile(x, q)), 4) if len(x) else None
    held = []
    for o, r in zip(obs, res):
        if r.get("Us") is None:
            continue
        # relative RMSE on a fixed sample of unobserved entries (true low-rank M)
        rng = np.random.default_rng(0)
        ii = rng.integers(0, o.m, 4096)
        jj = rng.integers(0, o.n, 4096)
        pred = np.einsum("ij,ij->i", r["Us"][ii].astype(np.float64), r["V"][jj].astype(np.float64))
        truth = o.dense[ii, jj].astype(np.float64)
        held.append(float(np.sqrt(np.mean((pred - truth) ** 2)) / np.sqrt(np.mean(truth ** 2))))
    return {"solves_per_s": round(len(res) / wall, 3), "p50_latency_s": round(float(np.percentile(lat, 50)), 4),
            "p99_latency_s": round(float(np.percentile(lat, 99)), 4),
            "p50_queue_s": round(float(np.percentile([r["queue_s"] for r in res], 50)), 4),
            "converged_jobs": {"jobs": int(rec.sum()), "p50_latency_s": pct(lat[rec], 50),
                               "p99_latency_s": pct(lat[rec], 99),
                               "median_samples_per_dof": pct((np.array(nnz) / dof)[rec], 50)},
            "unconverged_jobs": {"jobs": int((~rec).sum()), "p50_latency_s": pct(lat[~rec], 50),
                                 "p99_latency_s": pct(lat[~rec], 99),
                                 "median_samples_per_dof": pct((np.array(nnz) / dof)[~rec], 50)},
            "jobs": len(res), "converged": int(sum(r["converged"] for r in res)),
            "iters_total": int(sum(r["iters"] for r in res)), "nnz_total": int(sum(nnz)),
            "median_rel_rmse_unobserved": round(float(np.median(held)), 5) if held else None,
            "wall_s": round(wall, 3), "slots": SERVE_SLOTS, "peak_active": st["peak_active"],
            "peak_in_use_gb": round(st["peak_in_use_bytes"] / 1e9, 3),
            "gpu_launches": int(mc.load().mc_launch_count() - l0),
            "workload": f"first {len(res)} jobs of a 2,000-job Poisson stream at {SERVE_RATE} jobs/s: m, n "
                        f"log-uniform [256, 8192], 5-50% observed, rank 5-50; i_max {SERVE_IMAX}"}


def run_case(args):
    """A small fixed case of one kernel class, for profiler captures: inputs
    larger than L2 but a few hundred MB on the device, a handful of launches."""
    import torch

    import paper_1810_06860_gb300 as mc

    mc.load()
    if args.case in ("spmm", "sddmm"):
        o = mc_synth.ratings(120_000, 24_000, 16_000_000, seed=3)
        with mc.Handle.from_observed(o) as h:
            if args.case == "spmm":
                for K in (12, 60, 240):
                    for trans in (False, True):
                        X = torch.randn((o.m if trans else o.n), K, device="cuda")
                        h.spmm(X, trans=trans, device=True)
            else:
                prm = mc.params(tau=5.0 * math.sqrt(o.m * o.n), delta=DELTA, eps=1e-4, recycle=1, seed=SEED)
                for _ in range(3):
                    h.svt_step(prm)
    elif args.case == "svt":
        # the timed window alone: the rating workload, the state-preparing
        # iterations, then warm-up and window iterations; prints the library's
        # launch count when the window starts (a profiler's launch skip)
        o = load_workload()
        with mc.Handle(o.m, o.n, o.row_ptr, o.col, o.val) as h:
            prm = svt_params(mc, o)
            for _ in range(PREP_ITERS + args.warmup):
                h.svt_step(prm)
            torch.cuda.synchronize()
            print(json.dumps({"window_start_launches": int(mc.load().mc_launch_count())}), flush=True)
            for _ in range(args.steps):
                h.svt_step(prm)
    elif args.case == "serve":
        print(json.dumps(run_serving(mc, args.steps)), flush=True)
    elif args.case == "panel":
        # the tensor-core panel kernels on panels larger than L2: Z = X W
        # (600,000 x 60 times 60 x 60, and 240 x 52) and the Gram X^T X
        rng = np.random.default_rng(SEED)
        X = rng.standard_normal((600_000, 60)).astype(np.float32)
        mc.panel_gemm(X, rng.standard_normal((60, 60)).astype(np.float32), tensor_cores=True)
        mc.panel_gram(X, X, tensor_cores=True)
        X = rng.standard_normal((300_000, 240)).astype(np.float32)
        mc.panel_gemm(X, rng.standard_normal((240, 52)).astype(np.float32), tensor_cores=True)
    elif args.case == "gram":
        X = torch.randn(138_000, 240, device="cuda")
        for _ in range(3):
            mc.gram(X, tensor_cores=True)
    elif args.case == "orth":
        # the Krylov blocks of the SVT step (m = 138,000, k + s = 12, p = 3)
        # and of rSVD-BKI at k = 50 (60 columns): CUDA-event time per call
        R, res = 138_000, {}
        for K, cols in ((12, 0), (12, 12), (12, 24), (12, 36), (60, 0), (60, 180)):
            Qp = mc.orth_block(torch.randn(R, cols, device="cuda")) if cols else None
            X0 = torch.randn(R, K, device="cuda")
            Xs = [X0.clone() for _ in range(max(args.steps, 1) + 3)]
            for X in Xs[:3]:
                mc.orth_block(X, Qp)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for X in Xs[3:]:
                mc.orth_block(X, Qp)
            e1.record()
            torch.cuda.synchronize()
            res[f"K{K}_cols{cols}_us"] = round(1e3 * e0.elapsed_time(e1) / max(args.steps, 1), 1)
        print(json.dumps(res), flush=True)
    torch.cuda.synchronize()
    print(json.dumps({"case": args.case, "status": "ok"}), flush=True)


def run_reference(args, rank, world, local):
    """The float64 oracle on the host cores, on the window's workload: each
    step is one oracle Alg. 6 iteration of the window's shape (k, p from the
    oracle's own stored trajectory) on the leading eighth of the rows, a
    bounded sample; the rate is scaled to the full workload by that
    fraction (an iteration's work grows in proportion to the rows and
    entries it covers)."""
    if rank != 0:
        return
    o = load_workload()
    shape = oracle_window_shape()
    kk, pp = shape if shape else (48, 3)
    frac = 0.125
    t_start = time.perf_counter()
    secs = []
    for step in range(args.warmup + args.steps):
        t, msub, nnz = oracle_iteration_seconds(o, kk, pp, rows_frac=frac)
        if step >= args.warmup:
            secs.append(t)
    per_iter = float(np.sum(secs)) / len(secs) / frac
    value = 1.0 / per_iter
    sample = (f"float64 oracle Alg. 6 iteration of the window's shape (fresh rSVD-BKI at k = {kk}, p = {pp}, "
              f"warm-started Omega; shrink, evaluation on Phi, update) on the leading {msub} rows ({nnz} observed "
              f"entries, {frac:.3f} of the rows), scaled to the full workload by that fraction")
    line = {"impl": "reference", "metric": "SVT iterations/s at 2e7 nnz (rating matrix 138,000 x 27,000)",
            "value": round(value, 5), "unit": "iters/s", "n_gpus": world, "steps": len(secs), "warmup": args.warmup,
            "ms_per_step": round(1e3 * per_iter, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(),
            "cpu_baseline": {"value": round(value, 5), "unit": "iters/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 5), "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": round(time.perf_counter() - t_start, 1)}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--case", choices=["spmm", "sddmm", "gram", "serve", "orth", "svt", "panel"], default=None,
                    help="run one small kernel case for a profiler capture instead of the benchmark")
    args = ap.parse_args()
    if args.warmup < 3 or args.steps < 1:
        ap.error("--steps must be >= 1 and --warmup >= 3")
    rank, world, local = dist_init()
    if args.case:
        run_case(args)
    elif args.impl == "reference":
        run_reference(args, rank, world, local)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
