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
K_BKI, S_OVER, P_BKI = 50, 10, 3
HBM_FALLBACK_GBS = 6800.0
# Serving: a bounded sample of the Poisson job stream (m, n log-uniform in
# [256, 8192], 5-50% observed, rank 5-50), submitted at its arrival times.
SERVE_JOBS, SERVE_RATE, SERVE_SLOTS, SERVE_IMAX = 32, 16.0, 8, 300


def workload_config():
    return {"workload": f"rating-svt {M_ROWS}x{N_COLS} {N_PAIRS:.0e} pairs (10% held out)",
            "m": M_ROWS, "n": N_COLS, "nnz_observed": int(N_PAIRS * (1 - HOLDOUT)), "nnz_total": N_PAIRS,
            "tau": "5*sqrt(m*n)", "delta": DELTA, "recycle": "Q (strategy 1), i_reuse=50, q_reuse=10",
            "p0": 3, "s": S_OVER, "eps": 1e-4, "rsvd_bki": {"k": K_BKI, "s": S_OVER, "p": P_BKI},
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


def svt_params(mc, o):
    return mc.params(tau=5.0 * math.sqrt(o.m * o.n), delta=DELTA, eps=1e-4, recycle=1, i_reuse=50, q_reuse=10,
                     seed=SEED)


def cpu_oracle_iterations(o, iters: int):
    """Seconds per SVT iteration of the float64 oracle on the same workload:
    iterations 2..iters+1 after its own initialisation (callback timestamps)."""
    from oracle import svt as osvt

    ts = []
    osvt.svt_fast(o.m, o.n, o.row_ptr, o.col, o.val, tau=5.0 * math.sqrt(o.m * o.n), delta=DELTA, eps=1e-4,
                  recycle=1, i_reuse=50, q_reuse=10, i_max=iters + 1, seed=SEED,
                  callback=lambda r: ts.append(time.perf_counter()))
    d = np.diff(ts)
    return float(np.sum(d)), len(d)


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
    # the other two randomized SVDs on the same matrix: rSVD-PI (Alg. 4) with
    # the same p, and basic rSVD (Alg. 1 = Alg. 4 with p = 0)
    other_ms = {}
    for name, pp in (("rsvd_pi_ms", P_BKI), ("rsvd_basic_ms", 0)):
        for i in range(3):
            hb.rsvd_pi(K_BKI, S_OVER, pp, seed=SEED, call_id=300 + i, device=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for i in range(nb):
            hb.rsvd_pi(K_BKI, S_OVER, pp, seed=SEED, call_id=400 + i, device=True)
        e1.record(stream)
        torch.cuda.synchronize()
        other_ms[name] = round(e0.elapsed_time(e1) / nb, 3)
    hb.close()
    del rp, ci, va
    # ---- SVT iterations -----------------------------------------------------
    h = mc.Handle(o.m, o.n, o.row_ptr, o.col, o.val, stream=stream)
    prm = svt_params(mc, o)
    infos = []
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
    # held-out RMSE of the estimate after the timed iterations
    pred = h.sample(o.test_rows, o.test_cols)
    rmse = float(np.sqrt(np.mean((pred.astype(np.float64) - o.test_val) ** 2)))
    # per-class CUDA-event breakdown over the next iterations (not timed: the
    # events around every launch cost about 5 % of the step)
    h.timing_enable(True)
    for _ in range(args.steps):
        h.svt_step(prm)
    tm_all = h.timing_read()
    h.timing_enable(False)
    h.close()
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
    prm_m = svt_params(mc, o)
    prm_m.precision = 1
    for _ in range(args.warmup):
        hm.svt_step(prm_m)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        hm.svt_step(prm_m)
    hm.join()
    e1.record(stream)
    torch.cuda.synchronize()
    t_mixed = e0.elapsed_time(e1)
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
             "form": "bf16 panels in the Krylov products, float32 orthonormalisation and final projection",
             "timing_ms": tm_mixed}
    # ---- end to end through the C ABI with host buffers -----------------------
    h2d = (o.m + 1) * 8 + o.nnz * 8
    # the inputs sit in pinned host memory, as a serving host would stage them
    rp_h = torch.from_numpy(np.ascontiguousarray(o.row_ptr, np.int64)).pin_memory()
    ci_h = torch.from_numpy(np.ascontiguousarray(o.col, np.int32)).pin_memory()
    va_h = torch.from_numpy(np.ascontiguousarray(o.val, np.float32)).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    he = mc.Handle(o.m, o.n, rp_h, ci_h, va_h, stream=stream)
    for _ in range(args.steps):
        he.svt_step(prm)
    Us, V, sg = he.factors()
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    d2h = Us.nbytes + V.nbytes + sg.nbytes
    he.close()
    e2e = {"value": round(args.steps * world / t_e2e, 3), "unit": "iters/s",
           "h2d_bytes_per_step": int(h2d / args.steps), "d2h_bytes_per_step": int(d2h / args.steps),
           "note": "mc_create from pinned host CSR (ingest, CSC build, ||P_Phi M||_2) + K iterations from the start + factors to host"}
    # ---- CPU oracle baseline (rank 0, N = 1 only) -----------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        secs, its = cpu_oracle_iterations(o, 2)
        cpu = {"value": round(its / secs, 4), "unit": "iters/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"float64 oracle (NumPy/SciPy), SVT iterations 2-{its + 1} of the same workload after its own initialisation"}
    # ---- serving form (last: it loads the GPU for minutes) ----------------------
    serving = run_serving(mc, SERVE_JOBS) if not args.no_serving and world == 1 else None
    last = infos[-1]
    line = {"metric": "SVT iterations/s at 2e7 nnz (rating matrix 138,000 x 27,000)", "value": round(value, 3),
            "unit": "iters/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(t_ms / args.steps, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(workload_config(), parallelism=f"replicas x{world}",
                           timed_iterations=f"{args.warmup + 1}..{args.warmup + args.steps}",
                           k_last=last["k"], r_last=last["r"], p_last=last["p"], err_last=round(last["err"], 6),
                           heldout_rmse=round(rmse, 5)),
            "rsvd_bki_ms": round(bki_ms, 3), "rsvd_bki_timing_ms": bki_tm, **other_ms, "mixed_precision": mixed, "serving": serving,
            "roofline": roofline, "e2e": e2e, "cpu_baseline": cpu,
            "clocks": clk.summary(), "gpu_launches": int(launches),
            "timing_ms": {k: round(v["ms"], 3) for k, v in tm_all.items()},
            "timing_note": "per-class CUDA-event ms over the steps after the timed ones (same count)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


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
        # the timed step alone: the rating workload, warm-up then timed SVT iterations
        o = load_workload()
        with mc.Handle(o.m, o.n, o.row_ptr, o.col, o.val) as h:
            prm = svt_params(mc, o)
            for _ in range(args.warmup + args.steps):
                h.svt_step(prm)
    elif args.case == "serve":
        print(json.dumps(run_serving(mc, args.steps)), flush=True)
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
    if rank != 0:
        return
    o = load_workload()
    from oracle import svt as osvt

    ts = []
    n_total = args.warmup + args.steps
    t_start = time.perf_counter()
    osvt.svt_fast(o.m, o.n, o.row_ptr, o.col, o.val, tau=5.0 * math.sqrt(o.m * o.n), delta=DELTA, eps=1e-4,
                  recycle=1, i_reuse=50, q_reuse=10, i_max=n_total + 1, seed=SEED,
                  callback=lambda r: ts.append(time.perf_counter()))
    d = np.diff(ts)[args.warmup:args.warmup + args.steps]
    secs = float(np.sum(d))
    value = len(d) / secs if secs > 0 else 0.0
    sample = (f"float64 oracle SVT iterations {args.warmup + 2}..{args.warmup + 1 + len(d)} of the same "
              f"workload on the host cores (first iteration and initialisation untimed)")
    line = {"impl": "reference", "metric": "SVT iterations/s at 2e7 nnz (rating matrix 138,000 x 27,000)",
            "value": round(value, 4), "unit": "iters/s", "n_gpus": world, "steps": len(d), "warmup": args.warmup,
            "ms_per_step": round(1e3 * secs / max(len(d), 1), 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(),
            "cpu_baseline": {"value": round(value, 4), "unit": "iters/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 4), "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
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
    ap.add_argument("--case", choices=["spmm", "sddmm", "gram", "serve", "orth", "svt"], default=None,
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
