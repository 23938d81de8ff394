"""Benchmark: setup + solve time to a 1e-8 relative residual for root-node AMG.

Workload (one step): the rotated anisotropic diffusion system, Q1 bilinear
elements on a 1024 x 1024 element mesh of the unit square (n = 1,046,529,
nnz = 9,406,489), eps = 1e-3, psi = pi/8, homogeneous Dirichlet, B = 1,
right-hand side uniform in [-1, 1] (seed 2).  A step is the whole hot path:
rn_setup (strength, aggregation, pattern, energy-minimised P with pre- and
post-filter, R, Galerkin RAP, coarsest LU) followed by rn_solve (CG with
the V(1,1) weighted-Jacobi cycle) from x0 = 0 to ||b - A x|| < 1e-8 ||b||.

  value      seconds per step with A, B, b resident in HBM (CUDA events);
             the default form is the mixed-precision one (FP32 cycle inside
             FP64 flexible CG); the plain FP64 form is reported beside it.
  e2e        the same through the C ABI with host buffers (pinned), the
             host->device copies of A, B, b, x0 and the device->host copy
             of x inside the timed region.
  roofline   the dominant kernel of the step (by device time), achieved
             algorithmic bytes / measured duration against the measured HBM
             copy bandwidth.
  cpu_baseline  the FP64 CPU oracle on this machine's host: one full step
             (setup + CG solve to 1e-8) on all host threads, and one on a
             single thread.

--impl reference times the oracle alone on the same workload: every step a
full setup + solve to 1e-8 on all host threads.  With --gpus N under torchrun every rank solves its own
replica (no data-path collective; "replicas only").
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

from paper_1610_03154_gb300 import problems as PR  # noqa: E402

METRIC = "setup+solve s to 1e-8 rel. residual (FP64 vs mixed/batched); HBM GB/s % roofline"
WORKLOAD_NE = 1024


def load_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu capture
    (profiles/roofline_traffic.txt, JSON), or None when there is none or when a
    source file it was captured from has changed since."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "roofline_traffic.txt")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None, None
    ent = rec.get(kernel)
    if not ent:
        return None, None
    for f, md5 in ent.get("sources_md5", {}).items():
        try:
            if hashlib.md5(open(os.path.join(ROOT, f), "rb").read()).hexdigest() != md5:
                return None, "stale: " + f + " changed since the capture"
        except OSError:
            return None, "missing " + f
    return float(ent["dram_bytes_per_launch"]), ent.get("profile")


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d["hbm_gbs"], "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # nvidia-smi's start-up competes with the host thread that drives the
            # GPU: let it print its first sample before the timed region opens
            t0 = time.time()
            while not self.lines and time.time() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.02)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = max(mx, float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def job_step_seconds(step_s: float, device=None) -> float:
    """Replicas run independently; the job's step time is the slowest rank's
    (max over ranks).  No-op without an initialised process group."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return step_s
    t = torch.tensor([step_s], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_oracle_step(pr, threads: int):
    """One full oracle step on the host: setup, then CG with the V(1,1) cycle
    from x0 = 0 to ||b - A x|| < 1e-8 ||b||, on `threads` OpenMP threads.
    Returns (seconds, setup seconds, iterations, relative residual)."""
    from oracle import oracle as O

    O.set_threads(threads)
    t0 = time.perf_counter()
    h = O.Hierarchy(pr.A.to_scipy(), pr.B, **pr.params)
    t_setup = time.perf_counter() - t0
    _, info = h.solve(pr.b, tol=1e-8, maxit=5000, outer=1)
    total = time.perf_counter() - t0
    del h
    return total, t_setup, info["iters"], info["rel_res"]


def host_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def reference_arm(args):
    """The oracle, as it stands, timed on this machine's host cores: every
    warm-up and timed step is a full setup + CG solve to 1e-8 of the workload
    on all host threads (results do not depend on the thread count)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    pr = PR.aniso_problem(args.ne)
    nth = host_threads()
    for _ in range(args.warmup):
        run_oracle_step(pr, nth)
    vals, setups = [], []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        v, ts, iters, rr = run_oracle_step(pr, nth)
        vals.append(v)
        setups.append(ts)
    wall = time.perf_counter() - t_all
    value = float(np.mean(vals))
    sample = (f"every step a full oracle setup + FP64 CG solve to 1e-8 ({iters} iterations) on {nth} threads; "
              f"{args.steps} timed steps in {wall:.1f} s")
    line = {
        "metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": pr.description, "solver": "oracle FP64 CG + V(1,1) Jacobi", "l2": "n/a (CPU)",
                   "setup": pr.params},
        "cpu_baseline": {"value": value, "unit": "s", "cores": nth, "kind": "oracle", "sample": sample,
                         "setup_s": float(np.mean(setups)), "iters": iters, "rel_res": rr,
                         "timed_wall_s": wall},
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def profile_step(args):
    """A bounded run of the same workload for profilers: setup, then a fixed
    number of outer iterations (the solve stops at --profile-iters)."""
    import torch

    from paper_1610_03154_gb300 import rn

    dev = torch.device("cuda", 0)
    pr = PR.aniso_problem(args.ne)
    A = pr.A
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    rp, ci, va, Bd, bd = t(A.rowptr), t(A.col), t(A.val), t(pr.B.reshape(-1)), t(pr.b)
    p = rn.params_from_config(pr.params, precision=rn.RN_MIXED if args.precision == "mixed" else rn.RN_FP64,
                              outer=rn.RN_OUTER_CG, use_graphs=0)
    h = rn.Hierarchy(rp, ci, va, Bd, params=p)
    x = torch.zeros_like(bd)
    info = h.solve(bd, x, rtol=1e-8, maxit=args.profile_iters, raise_on_notconv=False)
    h.close()
    torch.cuda.synchronize()
    print(json.dumps({"profile_step": True, "iters": info["iters"], "rel_res": info["rel_res"]}))
    return 0


def profile_setup_op(args):
    """Build the workload's hierarchy (keep_aux), then run one level-0 setup
    operation (rn_time_setup_op, one run, no flush) between cudaProfilerStart
    and cudaProfilerStop, so that `ncu --profile-from-start off` captures that
    operation's launches and nothing else."""
    import torch

    from paper_1610_03154_gb300 import rn

    dev = torch.device("cuda", 0)
    pr = PR.aniso_problem(args.ne)
    A = pr.A
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    p = rn.params_from_config(pr.params, precision=rn.RN_MIXED if args.precision == "mixed" else rn.RN_FP64,
                              outer=rn.RN_OUTER_CG, keep_aux=1)
    h = rn.Hierarchy(t(A.rowptr), t(A.col), t(A.val), t(pr.B.reshape(-1)), params=p)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    name, us, by = h.time_setup_op(args.profile_setup_op, reps=1, flush_bytes=0)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    h.close()
    print(json.dumps({"profile_setup_op": name, "us": us, "bytes": by}))
    return 0


def grid_rows(rn, torch, dev, stream, flush, peak):
    """Setup + solve to 1e-8 on the other grids of the workload list, each in
    FP64 and mixed precision (one warm-up and one timed step, inputs resident,
    CUDA events, L2 flushed): upwind convection-diffusion on 2048^2 (FGMRES(30)),
    variable-coefficient FV on 512^2 (CG) and the 64^2 Poisson problem with one
    right-hand side (stationary V-cycles).  Each record carries the dominant
    level-0 launch of its solve timed alone (roofline) and the oracle's
    iteration count for the same settings on all host threads."""
    from oracle import oracle as O

    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    out = {}
    for key, pr, latency in (("convdiff_2048", PR.convdiff_problem(2048), False),
                             ("varcoef_512", PR.varcoef_problem(512), False),
                             ("poisson_64", PR.poisson_problem(64), True)):
        A = pr.A
        dA = (t(A.rowptr), t(A.col), t(A.val), t(pr.B.reshape(-1)))
        Bh = None if pr.Bhat is None else t(pr.Bhat.reshape(-1))
        b = t(pr.b)
        x = torch.zeros_like(b)
        outer = pr.params.get("outer", 1)
        rec = {"problem": pr.description, "n": A.n_rows, "nnz": A.nnz,
               "outer": {0: "stationary", 1: "CG", 2: "FGMRES(30)"}[outer],
               "setup": {k: pr.params[k] for k in ("soc_kind", "soc_theta", "degree", "n_sweeps", "method",
                                                    "prefilter", "postfilter") if k in pr.params}}

        def step(prec):
            x.zero_()
            h = rn.Hierarchy(*dA, Bh, params=rn.params_from_config(pr.params, precision=prec, use_graphs=1),
                             stream=stream.cuda_stream)
            info = h.solve(b, x, rtol=1e-8, maxit=5000)
            h.close()
            return info

        for name, prec in (("mixed", rn.RN_MIXED), ("fp64", rn.RN_FP64)):
            step(prec)
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = step(prec)
            e1.record(stream)
            torch.cuda.synchronize()
            res = float(np.linalg.norm(pr.b - A.to_scipy() @ x.cpu().numpy()) / np.linalg.norm(pr.b))
            rec[name] = {"step_s": e0.elapsed_time(e1) / 1e3, "iters": info["iters"], "rel_res": res}
        # the solve's level-0 launches timed alone; the longest is the roofline
        h = rn.Hierarchy(*dA, Bh, params=rn.params_from_config(pr.params, precision=rn.RN_MIXED, use_graphs=1),
                         stream=stream.cuda_stream)
        x.zero_()
        h.solve(b, x, rtol=1e-8, maxit=5000)
        ops = {}
        cg_only = (rn.RN_OP_CG_XR, rn.RN_OP_CG_RZ, rn.RN_OP_CG_P)
        for op in range(rn.RN_OP_COUNT):
            if outer != 1 and op in cg_only:  # launches of the CG iteration only
                continue
            if outer == 1 and op == rn.RN_OP_CG_RZ:  # not issued: the last level-0 sweep carries it
                continue
            r = h.time_op(op, reps=20)
            if r is not None and r[2] > 0:
                ops[r[0]] = r
        h.close()
        nm, us, by = max(ops.values(), key=lambda r: r[1])
        ach = by / (us * 1e-6) / 1e9
        rec["roofline"] = {"bound": "hbm", "kernel": nm, "achieved": ach, "peak": peak, "unit": "GB/s",
                           "frac": ach / peak, "avg_launch_us": us, "algorithmic_bytes": by,
                           "note": ("latency-bound: the operator (0.3 MB) is L2-resident" if latency else
                                    "latency-bound: each level-0 launch moves at most ~20 MB" if A.nnz < 2e6 else None)}
        rec["level0_launches"] = {k: {"us": round(v[1], 2), "GBps": round(v[2] / (v[1] * 1e-6) / 1e9, 1)}
                                  for k, v in sorted(ops.items(), key=lambda kv: -kv[1][1])}
        O.set_threads(host_threads())
        oh = O.Hierarchy(A.to_scipy(), pr.B, Bhat=pr.Bhat, **pr.params)
        _, oinfo = oh.solve(pr.b, tol=1e-8, maxit=5000, outer=outer, restart=pr.params.get("restart", 30))
        del oh
        rec["oracle_iters"] = oinfo["iters"]
        out[key] = rec
        del dA, Bh, b, x
    return out


def profile_op(args):
    """Build the workload's hierarchy and solve once, then run one level-0
    launch of the solve (rn_time_op index, one run, no flush) between
    cudaProfilerStart and cudaProfilerStop, for `ncu --profile-from-start
    off`."""
    import torch

    from paper_1610_03154_gb300 import rn

    dev = torch.device("cuda", 0)
    pr = PR.aniso_problem(args.ne)
    A = pr.A
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    p = rn.params_from_config(pr.params, precision=rn.RN_MIXED if args.precision == "mixed" else rn.RN_FP64,
                              outer=rn.RN_OUTER_CG)
    h = rn.Hierarchy(t(A.rowptr), t(A.col), t(A.val), t(pr.B.reshape(-1)), params=p)
    b = t(pr.b)
    x = torch.zeros_like(b)
    h.solve(b, x, rtol=1e-8, maxit=5000)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    r = h.time_op(args.profile_op, reps=1, flush_bytes=0)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    h.close()
    print(json.dumps({"profile_op": r[0] if r else None, "us": r[1] if r else None, "bytes": r[2] if r else None}))
    return 0


def next_rows(rn, torch, dev, stream, flush, prec):
    """Records for the batched and differentiable forms, each one warm-up
    and one timed pass with device-resident inputs (CUDA events, L2 flushed):
    256 right-hand sides on the 64^2 Poisson operator (setup + rn_solve_multi),
    64 uneven rotated-anisotropy problems (rn_setup_merged + rn_batch_merge +
    rn_batch_solve, beside the per-problem setups and solves)
    and a gradient through the solve on 512^2 variable-coefficient cells
    (forward setup + solve, adjoint solve, dL/dA scatter, chain to theta)."""
    from paper_1610_03154_gb300 import adjoint

    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    precision = rn.RN_MIXED if prec == "mixed" else rn.RN_FP64

    def clock(fn):
        out = []
        for _ in range(2):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            out.append((e0.elapsed_time(e1) / 1e3, r))
        return out[-1]

    # many right-hand sides
    pp = PR.poisson_problem(64)
    s_rhs = 256
    Bm = t(np.random.default_rng(4).uniform(-1.0, 1.0, (pp.A.n_rows, s_rhs)))
    Xm = torch.zeros_like(Bm)
    pd = (t(pp.A.rowptr), t(pp.A.col), t(pp.A.val), t(pp.B.reshape(-1)))

    def multi():
        Xm.zero_()
        h = rn.Hierarchy(*pd, params=rn.params_from_config(pp.params, precision=precision), stream=stream.cuda_stream)
        info = h.solve_multi(Bm, Xm, rtol=1e-8, maxit=500)
        h.close()
        return info

    tm, im = clock(multi)
    # the solve's launches one by one, each bracketed by CUDA events (the
    # library's profiler): algorithmic bytes / time, L2 + HBM (the 4 MB
    # multivectors and the operators stay in L2)
    hm = rn.Hierarchy(*pd, params=rn.params_from_config(pp.params, precision=precision), stream=stream.cuda_stream)
    Xm.zero_()
    torch.cuda.synchronize()
    rn.profile_reset()
    rn.profile_enable(True)
    hm.solve_multi(Bm, Xm, rtol=1e-8, maxit=500)
    rn.profile_enable(False)
    prof = rn.profile_read()
    rn.profile_reset()
    hm.close()
    mk = {k: v for k, v in prof.items() if k.startswith("multi_")}
    m_bytes = sum(v["bytes"] for v in mk.values())
    m_ms = sum(v["ms"] for v in mk.values())
    top = max(mk.items(), key=lambda kv: kv[1]["ms"]) if mk else ("", {"bytes": 0.0, "ms": 0.0, "launches": 0})
    Bh, Xh = Bm.cpu().numpy(), Xm.cpu().numpy()  # FP64 residual of every column, on the host
    res_m = float(np.max(np.linalg.norm(Bh - pp.A.to_scipy() @ Xh, axis=0) / np.linalg.norm(Bh, axis=0)))

    # many problems
    probs = PR.batch_aniso_problems()
    dp = [(t(p.A.rowptr), t(p.A.col), t(p.A.val), t(p.B.reshape(-1))) for p in probs]
    bs = [t(p.b) for p in probs]
    xs = [torch.zeros_like(b) for b in bs]
    bparams = rn.params_from_config(PR.PARAMS_ANISO, precision=precision)

    def batched_streams():
        for x in xs:
            x.zero_()
        hs = rn.setup_batched(dp, params=bparams)
        infos = rn.solve_batched(hs, bs, xs, rtol=1e-8, maxit=2000)
        for h in hs:
            h.close()
        return infos

    phases = {}

    def batched_merged(setup=rn.setup_merged):
        for x in xs:
            x.zero_()
        t0 = time.perf_counter()
        hs = setup(dp, params=bparams)
        t1 = time.perf_counter()
        batch = rn.Batch(hs)
        for h in hs:
            h.close()
        t2 = time.perf_counter()
        infos = batch.solve(bs, xs, rtol=1e-8, maxit=2000)
        t3 = time.perf_counter()
        batch.close()
        phases.update(setup_s=t1 - t0, merge_s=t2 - t1, solve_s=t3 - t2)
        return infos

    tbs, ibs = clock(batched_streams)
    tbt, ibt = clock(lambda: batched_merged(rn.setup_batched))
    phases_st = dict(phases)
    tb, ib = clock(batched_merged)
    phases_thr = dict(phases)
    bparams_thr = bparams
    bparams = rn.params_from_config(PR.PARAMS_ANISO, precision=precision, autotune=1)
    tba, iba = clock(batched_merged)
    phases_at = dict(phases)
    bparams = bparams_thr
    n_b = sum(p.A.n_rows for p in probs)
    nnz_b = sum(p.A.nnz for p in probs)
    del dp, bs, xs

    # gradient through the solve (512^2 cells); the observation comes from a
    # GPU solve with another coefficient field
    m = 512
    op = adjoint.VarCoefFV(m, dev)
    vparams = rn.params_from_config(PR.PARAMS_VARCOEF)
    f = torch.full((m * m,), 1.0 / (m * m), dtype=torch.float64, device=dev)
    with torch.no_grad():
        u_obs = adjoint.solve(op.values(t(PR.gaussian_field(m, 22))), f, op.rowptr, op.col, params=vparams,
                              rtol=1e-10)
    th0 = t(PR.gaussian_field(m, 21))

    def grad():
        th = th0.clone().requires_grad_(True)
        u = adjoint.solve(op.values(th), f, op.rowptr, op.col, params=vparams, rtol=1e-10)
        L = 0.5 * torch.sum((u - u_obs) ** 2)
        L.backward()
        return float(L.detach()), float(torch.linalg.norm(th.grad))

    ta, (La, ga) = clock(grad)
    return {
        "multi_rhs": {"step_s": tm, "columns": s_rhs, "iters": im["iters"], "max_rel_res": res_m,
                      "problem": pp.name, "what": "setup + rn_solve_multi (stationary V(1,1), per-column stop)",
                      "solve_gbs_l2_hbm": (m_bytes / (m_ms * 1e-3) / 1e9) if m_ms > 0 else None,
                      "top_kernel": {"name": top[0], "launches": top[1]["launches"],
                                     "gbs_l2_hbm": (top[1]["bytes"] / (top[1]["ms"] * 1e-3) / 1e9)
                                     if top[1]["ms"] > 0 else None},
                      "gbs_rule": "algorithmic bytes of every solve launch / its CUDA-event time, launches timed "
                                  "one by one (warm L2)",
                      "precision": prec},
        "batched_problems": {"step_s": tb, "problems": len(probs), "n_total": n_b, "nnz_total": nnz_b,
                             "max_iters": max(i["iters"] for i in ib),
                             "max_rel_res": max(i["rel_res"] for i in ib),
                             "phases_s": phases_thr,
                             "autotuned": {"step_s": tba, "max_iters": max(i["iters"] for i in iba), "phases_s": phases_at,
                                           "what": "the same with the merged hierarchy's SpMV schedules picked by "
                                                   "timed trials (params.autotune)"},
                             "what": "rn_setup_merged (one setup pass over the block-diagonal union, per-problem "
                                     "aggregation keys, energy-CG scalars and coarsening stops) + rn_batch_merge + "
                                     "rn_batch_solve (CG per problem, one launch per step for all problems), sides "
                                     "U{32..512}, eps 10^U[-4,-1], psi U[0,pi)",
                             "setup_per_problem": {"step_s": tbt, "max_iters": max(i["iters"] for i in ibt),
                                                   "phases_s": phases_st,
                                                   "what": "the same with rn_setup_batched (a setup per problem on "
                                                           "its own stream, host threads)"},
                             "streams_step_s": tbs, "streams_max_iters": max(i["iters"] for i in ibs),
                             "streams_what": "rn_setup_batched + rn_solve_batched (a stream and host thread per "
                                             "problem)", "precision": prec},
        "adjoint_grad": {"step_s": ta, "cells": m * m, "rtol": 1e-10, "loss": La, "grad_norm": ga,
                         "what": "forward setup + CG solve, adjoint CG solve, dL/dA on A's pattern, chain to theta",
                         "precision": "fp64"},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--ne", type=int, default=WORKLOAD_NE, help="elements per side (default: the 1024^2 workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-step", action="store_true",
                    help="one setup + --profile-iters outer iterations and nothing else (for ncu captures)")
    ap.add_argument("--profile-iters", type=int, default=10)
    ap.add_argument("--profile-op", type=int, default=-1,
                    help="run one level-0 solve launch (rn_time_op index) inside a profiler range")
    ap.add_argument("--profile-setup-op", type=int, default=-1,
                    help="run one level-0 setup operation (rn_time_setup_op index) inside a profiler range")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    if args.profile_step:
        return profile_step(args)
    if args.profile_setup_op >= 0:
        return profile_setup_op(args)
    if args.profile_op >= 0:
        return profile_op(args)

    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1610_03154_gb300 import rn

    pr = PR.aniso_problem(args.ne)
    A = pr.A
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    rp, ci, va, Bd, bd = t(A.rowptr), t(A.col), t(A.val), t(pr.B.reshape(-1)), t(pr.b)
    xd = torch.zeros_like(bd)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > 129 MB L2

    def params(prec, **over):
        return rn.params_from_config(pr.params, precision=rn.RN_MIXED if prec == "mixed" else rn.RN_FP64,
                                     outer=rn.RN_OUTER_CG, use_graphs=1, **over)

    # candidates 1, x, y of the interior grid (the several-candidate setup, k = 3)
    m_int = int(round(math.sqrt(A.n_rows)))
    ii = np.arange(A.n_rows)
    B3 = t(np.column_stack([np.ones(A.n_rows), (ii % m_int + 1) / (m_int + 1), (ii // m_int + 1) / (m_int + 1)]))

    def step(prec, B=None, **over):
        xd.zero_()
        h = rn.Hierarchy(rp, ci, va, Bd if B is None else B, params=params(prec, **over), stream=sptr)
        info = h.solve(bd, xd, rtol=1e-8, maxit=5000)
        h.close()
        return info

    def timed(prec, k, B=None, **over):
        times, infos = [], []
        for _ in range(k):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            infos.append(step(prec, B, **over))
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        return times, infos

    prec = args.precision
    other = "fp64" if prec == "mixed" else "mixed"
    for _ in range(max(3, args.warmup)):
        step(prec)
        step(other)
    # check the solution once against the FP64 residual bar (host, scipy)
    xs = xd.cpu().numpy()
    res_check = float(np.linalg.norm(pr.b - A.to_scipy() @ xs) / np.linalg.norm(pr.b))

    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        # the host-side residual check above leaves the GPU idle long enough for
        # its clocks to drop: one more untimed step brings them back up
        step(prec)
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        l0 = int(rn.rn_kernel_launches())
        times, infos = timed(prec, args.steps)
        launches = int(rn.rn_kernel_launches()) - l0
    torch.cuda.synchronize()
    step_s = job_step_seconds(float(np.mean(times)), dev)
    times_other, infos_other = timed(other, args.steps)
    # the same step with W(1,1) cycles (Sec. 5.2), one warm-up and one timed step
    step(prec, gamma=2)
    times_w, infos_w = timed(prec, 1, gamma=2)
    # the same step with SpMV schedules picked by timed trials (params.autotune;
    # the first setup tunes, later ones take the cached choices)
    step(prec, autotune=1)
    times_at, infos_at = timed(prec, 3, autotune=1)
    # the same step with the symmetric strength measure (the setting measured
    # first), one warm-up and one timed step
    step(prec, soc_kind=0)
    times_sym, infos_sym = timed(prec, 1, soc_kind=0)
    # the same step with three candidates (1, x, y), Sec. 3.6
    step(prec, B3)
    times_k3, infos_k3 = timed(prec, 1, B3)
    # a block system of the same size class (Sec. 3.2, Sec. 5.4): plane-strain
    # elasticity, 2 unknowns per node, 3 rigid-body modes; one warm-up and one
    # timed step (setup + CG solve), inputs resident
    prs = PR.elasticity_problem(args.ne // 4)
    es = dict(rp=t(prs.A.rowptr), ci=t(prs.A.col), va=t(prs.A.val), B=t(prs.B), b=t(prs.b))
    xs_d = torch.zeros_like(es["b"])
    es_times, es_infos = [], []
    for rep in range(2):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        xs_d.zero_()
        hs = rn.Hierarchy(es["rp"], es["ci"], es["va"], es["B"],
                          params=rn.params_from_config(prs.params, precision=rn.RN_MIXED if prec == "mixed"
                                                       else rn.RN_FP64, outer=rn.RN_OUTER_CG, use_graphs=1),
                          stream=sptr)
        es_infos.append(hs.solve(es["b"], xs_d, rtol=1e-8, maxit=5000))
        e1.record(stream)
        torch.cuda.synchronize()
        es_times.append(e0.elapsed_time(e1) / 1e3)
        es_levels = hs.stats()["levels"]
        es_setup_ms = hs.stats().get("setup_ms")
        hs.close()
    del es, xs_d
    nexts = next_rows(rn, torch, dev, stream, flush, prec)
    grids = grid_rows(rn, torch, dev, stream, flush, load_peaks()[0])

    # per-launch device times of the solve's level-0 operations, each timed in
    # isolation with CUDA events on the hierarchy's stream, a 256 MB read before
    # every launch (cold L2 without dirty lines; the GPU stays busy while the
    # launch is enqueued).
    # Each runs once per outer iteration.
    h = rn.Hierarchy(rp, ci, va, Bd, params=params(prec), stream=sptr)
    xd.zero_()
    h.solve(bd, xd, rtol=1e-8, maxit=5000)
    ops = {}
    for op in range(rn.RN_OP_COUNT):
        if op == rn.RN_OP_CG_RZ:  # not issued: the cycle's last level-0 sweep carries these reductions
            continue
        r = h.time_op(op, reps=20)
        if r is not None:
            ops[r[0]] = {"us": r[1], "bytes": r[2]}
    h.close()
    # the setup's level-0 operations, each timed alone the same way
    # (rn_time_setup_op): one energy-minimisation CG sweep and its three
    # launches, the Galerkin products A P and R (A P), and P^T
    peak, peak_kind = load_peaks()
    ha = rn.Hierarchy(rp, ci, va, Bd, params=params(prec, keep_aux=1), stream=sptr)
    sops = {}
    for op in range(rn.RN_SOP_COUNT):
        nm, us, by = ha.time_setup_op(op, reps=10)
        sops[nm] = {"us": round(us, 2), "bytes": by, "GBps": round(by / (us * 1e-6) / 1e9, 1),
                    "frac": round(by / (us * 1e-6) / 1e9 / peak, 4)}
    n_sweeps_l0 = pr.params.get("n_sweeps", 4) + (1 if pr.params.get("postfilter", 0.0) > 0 else 0)
    ha.close()

    def setup_record(key, rule):
        v = sops[key]
        ach = v["bytes"] / (v["us"] * 1e-6) / 1e9
        return {"bound": "hbm", "kernel": key, "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "peak_kind": peak_kind, "avg_launch_us": v["us"], "algorithmic_bytes": v["bytes"], "rule": rule}

    energy_rec = setup_record("energy_sweep_L0", "one level-0 CG energy-minimisation sweep (direction, masked "
                              "product with <D,W>, update with rho) in the setup's precision, timed alone with CUDA "
                              "events after a 256 MB L2 read flush; bytes = 12 nnzA + 4 nnzN + 64 nnzN + 8 n + 8 n_c "
                              "(FP64) or 8 nnzA + 4 nnzN + 32 nnzN + 4 n + 4 n_c (FP32 sweeps)")
    energy_rec["sweeps_per_setup_level0"] = n_sweeps_l0
    energy_rec["launches"] = {k: sops[k] for k in ("energy_direction_L0", "energy_product_L0", "energy_update_L0")}
    rap_rec = setup_record("galerkin_RAP_L0", "R_0 (A_0 P_0) as the setup forms it (symbolic and numeric passes with "
                           "their host synchronisations), timed alone after a 256 MB L2 read flush; bytes = "
                           "12 (nnzR + nnzAP) + 12 nnzA1")
    rap_rec["launches"] = {k: sops[k] for k in ("galerkin_AP_L0", "transpose_P_L0")}
    iters = infos[0]["iters"]
    bw = {k: v for k, v in ops.items() if v["bytes"] > 0}
    name = max(bw, key=lambda k: bw[k]["us"])
    st = bw[name]
    achieved = st["bytes"] / (st["us"] * 1e-6) / 1e9
    traffic, traffic_src = load_traffic(name)
    roofline = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic, "traffic_source": traffic_src,
                "avg_launch_us": st["us"], "algorithmic_bytes": st["bytes"], "launches_per_step": iters,
                "share_of_step": st["us"] * 1e-6 * iters / step_s,
                "rule": "longest level-0 launch of the outer iteration (each runs once per iteration), timed "
                        "alone with CUDA events after a 256 MB L2 read flush (cold, no dirty lines)"}
    kernels = {k: {"us": round(v["us"], 2), "launches_per_step": iters,
                   "GBps": round(v["bytes"] / (v["us"] * 1e-6) / 1e9, 1) if v["bytes"] > 0 else None}
               for k, v in sorted(ops.items(), key=lambda kv: -kv[1]["us"])}

    # end to end through the C ABI with host buffers
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    hrp, hci, hva, hB, hb = pin(A.rowptr), pin(A.col), pin(A.val), pin(pr.B.reshape(-1)), pin(pr.b)
    hx = pin(np.zeros(A.n_rows))
    e2e_times = []
    for rep in range(args.steps + 1):  # the first pass untimed (warm-up: pool growth, first touches)
        hx[:] = 0.0
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = rn.Hierarchy(hrp, hci, hva, hB, params=params(prec), stream=sptr)
        h.solve(hb, hx, rtol=1e-8, maxit=5000)
        h.close()
        torch.cuda.synchronize()
        if rep > 0:
            e2e_times.append(time.perf_counter() - t0)
    h2d = hrp.nbytes + hci.nbytes + hva.nbytes + hB.nbytes + hb.nbytes + hx.nbytes
    d2h = hx.nbytes

    stats_h = rn.Hierarchy(rp, ci, va, Bd, params=params(prec), stream=sptr)
    hs = stats_h.stats()
    # the mixed setup's error against the FP64 setup (which matches the FP64
    # oracle to 1e-12): level-0 P after the FP32 energy-minimisation sweeps
    setup_err = None
    if prec == "mixed":
        ref_h = rn.Hierarchy(rp, ci, va, Bd, params=params("fp64"), stream=sptr)
        Pm, Pf = stats_h.export_csr(0, 4), ref_h.export_csr(0, 4)
        same = np.array_equal(Pm[0], Pf[0]) and np.array_equal(Pm[1], Pf[1])
        setup_err = {"level0_P_pattern_equal": bool(same),
                     "level0_P_max_rel_err": float(np.max(np.abs(Pm[2] - Pf[2])) / np.max(np.abs(Pf[2])))
                     if same else None,
                     "levels": [hs["n"], ref_h.stats()["n"]]}
        ref_h.close()
    stats_h.close()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        # one full step of the oracle (setup + CG to 1e-8) on all host threads,
        # and one on a single thread
        nth = host_threads()
        v, ts, it_o, rr_o = run_oracle_step(pr, nth)
        v1, ts1, _, _ = run_oracle_step(pr, 1)
        cpu = {"value": v, "unit": "s", "cores": nth, "kind": "oracle",
               "sample": f"one full oracle step (setup {ts:.2f} s + FP64 CG to 1e-8, {it_o} iterations) on {nth} "
                         f"threads",
               "one_thread": {"value": v1, "unit": "s", "cores": 1, "setup_s": ts1}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": step_s, "unit": "s", "n_gpus": ws, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": step_s * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32" if prec == "mixed" else "f64",
            "data": "synthetic",
            "config": {"workload": pr.description, "precision": prec, "outer": "flexible CG" if prec == "mixed"
                       else "CG", "cycle": "V(1,1) weighted Jacobi omega=2/3, dense coarsest solve",
                       "setup": "theta=0.25 classical strength, seeded MIS-2 aggregation, d=4, 6 CG energy-min "
                                "sweeps, pre/post filter 0.1", "l2": "256 MB torch fill (write) before every timed step; per-launch timings after a 256 MB read",
                       "setup_roofline": "energy_min and rap records",
                       "parallelism": f"replicas x{ws}"},
            "iters": infos[0]["iters"], "rel_res": infos[0]["rel_res"], "rel_res_host_check": res_check,
            "step_s_all": times,
            f"{other}": {"value": float(np.mean(times_other)), "iters": infos_other[0]["iters"],
                         "rel_res": infos_other[0]["rel_res"]},
            "hierarchy": {"levels": hs["levels"], "n": hs["n"], "nnz_A": hs["nnz_A"], "nnz_P": hs["nnz_P"],
                          "oc": hs["oc"], "cc": hs["cc"], "setup_ms_last": hs["setup_ms"]},
            "e2e": {"value": float(np.mean(e2e_times)), "unit": "s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "mixed_setup_vs_fp64": setup_err,
            "autotuned": {"step_s": float(np.mean(times_at)), "iters": infos_at[0]["iters"],
                          "what": "SpMV schedules (lanes per row / tile height, or the unstaged kernel) per matrix "
                                  "picked by timed trials, cached per shape; threshold schedule = value"},
            "symmetric_soc": {"step_s": times_sym[0], "iters": infos_sym[0]["iters"],
                              "rel_res": infos_sym[0]["rel_res"], "strength": "symmetric, theta 0.25",
                              "precision": prec},
            "w_cycle": {"step_s": times_w[0], "iters": infos_w[0]["iters"], "rel_res": infos_w[0]["rel_res"],
                        "cycle": "W(1,1)", "precision": prec},
            "candidates_3": {"step_s": times_k3[0], "iters": infos_k3[0]["iters"], "rel_res": infos_k3[0]["rel_res"],
                             "B": "1, x, y", "precision": prec},
            **nexts,
            "grids": grids,
            "block_system": {"step_s": es_times[1], "iters": es_infos[1]["iters"], "rel_res": es_infos[1]["rel_res"],
                             "levels": es_levels, "setup_ms": es_setup_ms, "problem": prs.name, "n": prs.A.n_rows, "nnz": prs.A.nnz,
                             "block_size": 2, "B": "3 rigid-body modes", "strength": "classical, theta 0.5",
                             "precision": prec},
            "roofline": roofline,
            "level0_launches": kernels,
            "energy_min": energy_rec,
            "rap": rap_rec,
            "gpu_launches": launches // max(args.steps, 1),
            "gpu_launches_timed_region": launches,
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
