#!/usr/bin/env python
"""SGN steps/sec on GB300: assemble + factor + solve (+ FP64 refinement).

A step is one pass of the SGN hot path at an equilibrium state: element
evaluation and no-atomic assembly of the saddle-point matrix of
Eq. sparseSystemGN, its multifrontal LDL^T, and the solves for (dx, dp,
dlambda) with FP64 iterative refinement.  The default workload is the 3D
Kuhn-tet cube with 40^3 nodes (355,914 tets, 730,314 saddle-point unknowns);
the headline precision is the mixed path (FP32 fronts, FP64 pivots,
residuals and refinement), checked against the plain FP64 GPU path.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun (N > 1) every rank solves its own replica of the workload
(the factorization of one mesh is not sharded); value = all ranks' steps /
max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SGN steps/sec (assemble+factor+solve)"
UNIT = "steps/s"
MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")

# DRAM bytes of the tensor-core trailing update per algorithmic byte (the
# trailing triangle read and written once in FP32), from the ncu capture of
# every update launch of a kuhn3d_24 step summarised in
# profiles/k_update_tcp_kuhn3d_24.md (4.513 GB / 2.949 GB; the full-size
# launches are too large to capture); set to None when the kernel changes
UPDATE_DRAM_PER_ALGO_BYTE = 1.53


def measure_peaks(torch):
    """Dense peaks of this GPU measured in this run with library GEMMs (CUDA
    events, best of several after warm-up): FP32 inputs with TF32 allowed
    (the tensor-core rate the FP32 fronts' tcgen05 kind::tf32 MMAs run at) and
    FP64 (the rate the plain FP64 path's DFMA updates are bounded by)."""
    out = {}
    old = torch.backends.cuda.matmul.allow_tf32
    try:
        for name, dt, n, reps, tf32 in (("tf32", torch.float32, 8192, 6, True), ("fp64", torch.float64, 4096, 3, False)):
            torch.backends.cuda.matmul.allow_tf32 = tf32
            a = torch.randn(n, n, dtype=dt, device="cuda")
            b = torch.randn(n, n, dtype=dt, device="cuda")
            c = a @ b
            best = None
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b, out=c)
                e1.record()
                e1.synchronize()
                ms = e0.elapsed_time(e1)
                best = ms if best is None else min(best, ms)
            out[name + "_tflops"] = 2.0 * n ** 3 / (best * 1e-3) / 1e12
            out[name + "_how"] = f"torch.matmul {n}^3 {'fp32 with TF32 allowed' if tf32 else 'fp64'}, best of {reps}"
            del a, b, c
    finally:
        torch.backends.cuda.matmul.allow_tf32 = old
        torch.cuda.empty_cache()
    return out


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="kuhn3d_40")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--fp64-steps", type=int, default=1, help="timed steps of the plain FP64 path (0: skip)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-sample", default="kuhn3d_12", help="oracle sample workload")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="oracle baseline time (0: skip it)")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--batch-workload", default="batch2d_256",
                    help="batched form: many uneven 2D instances in one graph-captured step ('' skips)")
    ap.add_argument("--warm-workload", default="rbf3d_40", help="learned warm start form ('' skips)")
    ap.add_argument("--scale-workload", default="kuhn3d_80",
                    help="largest single-GPU mixed-precision workload, timed once ('' skips)")
    ap.add_argument("--warm-snapshots", type=int, default=128)
    ap.add_argument("--warm-tests", type=int, default=6)
    ap.add_argument("--warm-train-steps", type=int, default=3000)
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"sgn_bench_clocks_{os.getpid()}_{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        busy = [v for v in sm if v > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_state(sample: str, seed: int):
    """A smaller mesh of the same family at its oracle equilibrium."""
    from oracle import equilibrium as EQ
    from sgn_inputs import make_preset
    prob = make_preset(sample, seed=seed)
    x, _ = EQ.newton(prob, prob.p0)
    return prob, x


def oracle_step(prob, x):
    """One SGN step of the CPU oracle, as it stands: element blocks and a
    SuperLU solve of the saddle-point system."""
    from oracle import system as S
    b = S.blocks(prob, x, prob.p0)
    S.sgn_step(b, "kkt")


def oracle_info(sample, prob, n, dt):
    N = 2 * prob.n_free * prob.dim + prob.n_elem
    return {"kind": "oracle", "cores": os.cpu_count(),
            "sample": f"{sample}: {prob.n_elem} elements, N={N}; {n} steps in {dt:.1f} s "
                      f"(NumPy elements + SciPy SuperLU, host cores; equilibrium computed before timing)"}


def oracle_step_rate(sample: str, seconds: float, seed: int):
    prob, x = oracle_state(sample, seed)
    n, t0 = 0, time.perf_counter()
    while True:
        oracle_step(prob, x)
        n += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return n / dt, oracle_info(sample, prob, n, dt)


def run_reference(args):
    ws, rank, local = dist_env()
    if ws > 1 and rank != 0:
        return
    from sgn_inputs import make_preset
    prob_s, x_s = oracle_state(args.cpu_sample, args.seed)
    for _ in range(max(args.warmup, 0)):
        oracle_step(prob_s, x_s)
    t0 = time.perf_counter()
    n = 0
    for _ in range(args.steps):
        oracle_step(prob_s, x_s)
        n += 1
    dt = time.perf_counter() - t0
    value = n / dt
    info = oracle_info(args.cpu_sample, prob_s, n, dt)
    info["value"] = value
    info["unit"] = UNIT
    prob = make_preset(args.workload)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / max(n, 1), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "sample": args.cpu_sample,
                       "note": "the oracle cannot factor the full workload in minutes; each step runs the sample"},
            "cpu_baseline": info,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def _timed(torch, fn):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = fn()
    torch.cuda.synchronize()
    return r, time.perf_counter() - t0


def _batch_instances(args):
    """The batched workload's instances (batch2d_<n>: n plane-strain grids,
    sides U{10..60})."""
    from sgn_inputs import batch2d_instances
    kind, _, n = args.batch_workload.rpartition("_")
    if kind != "batch2d":
        raise ValueError(f"batched workload must be batch2d_<n>, not {args.batch_workload}")
    return batch2d_instances(int(n), seed=args.seed)


def form_batched(P, torch, args):
    """Many uneven plane-strain instances behind one handle (sgn_batch_setup:
    one elimination forest): the mixed step as one CUDA-graph launch
    (assemble, factor, solve, 4 refinement solves) against the stepwise plain
    FP64 path on the same batch; per-instance residuals from the library."""
    subs = _batch_instances(args)
    from paper_2107_03285_gb300 import autotune
    tuned = autotune.lookup(subs, P.MIXED)
    leaf, panel = tuned if tuned else (0, 0)
    s = P.SGN.from_batch(subs, stores=P.STORE_FP64 | P.STORE_MIXED | P.STORE_KFACT | P.STORE_KFACT_MIXED,
                         leaf_nodes=leaf, panel=panel)
    try:
        p0 = np.concatenate([sub.p0 for sub in subs])
        fext = np.concatenate([sub.fext for sub in subs])
        (x64, r64), t64e = _timed(torch, lambda: s.equilibrium(p0, fext, precision=P.FP64))
        res64 = s.batch_residuals(P.binding.BATCH_EQUILIBRIUM)
        (x, rep), t_eq = _timed(torch, lambda: s.equilibrium(p0, fext, precision=P.MIXED))
        resm = s.batch_residuals(P.binding.BATCH_EQUILIBRIUM)
        eq64 = {"iters": r64.iters, "residual": r64.residual, "max_instance_residual": float(res64.max()),
                "seconds": t64e, "history": list(r64.history)[:r64.iters + 1],
                "max_abs_dx_vs_mixed": float((x64 - x).abs().max())}
        del x64
        p = torch.as_tensor(p0, device=x.device)
        out = (torch.empty_like(x), torch.empty_like(p), torch.empty_like(x))
        s.step(x, p, P.FP64)
        (_, dp64, _, _, _), t64 = _timed(torch, lambda: s.step(x, p, P.FP64))
        dp64 = dp64.clone()
        for _ in range(3):
            s.step_graph(x, p, P.MIXED, refine_steps=4, out=out, residual=False)
        n = 10
        l0 = s.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        for _ in range(n):
            s.step_graph(x, p, P.MIXED, refine_steps=4, out=out, residual=False)
        e1.record(s.stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / n
        launches = (s.launch_count() - l0) / n
        _, dpg, _, res = s.step_graph(x, p, P.MIXED, refine_steps=4, out=out, residual=True)
        kkt_inst = s.batch_residuals(P.binding.BATCH_KKT)
        err = float(torch.linalg.norm(dpg - dp64) / torch.linalg.norm(dp64))
        k = len(subs)
        sides = [int(round(np.sqrt(sub.n_nodes))) for sub in subs]
        return {"workload": f"{args.batch_workload}: {k} instances (sgn_batch_setup), sides {min(sides)}.."
                            f"{max(sides)}, {s.n_nodes} nodes, {s.n_elem} triangles, N={int(s.info.n_kkt)}",
                "graph_mixed": {"steps_per_s": 1e3 / ms, "instance_steps_per_s": k * 1e3 / ms, "ms_per_step": ms,
                                "launches_per_graph": launches, "kkt_residual": res,
                                "max_instance_kkt_residual": float(kkt_inst.max()),
                                "dp_rel_err_vs_fp64_gpu": err},
                "stepwise_fp64": {"steps_per_s": 1.0 / t64, "ms_per_step": 1e3 * t64},
                "speedup_vs_fp64": (1e3 / ms) * t64,
                "equilibrium_mixed": {"iters": rep.iters, "solves": rep.solves, "residual": rep.residual,
                                      "max_instance_residual": float(resm.max()),
                                      "seconds": t_eq, "history": list(rep.history)[:rep.iters + 1]},
                "equilibrium_fp64": eq64,
                "levels": int(s.info.n_levels), "supernodes": int(s.info.n_supernodes),
                "setup_options": {"leaf_nodes": leaf or 16, "panel": panel or 32,
                                  "source": "autotuned" if tuned else "defaults"}}
    finally:
        s.close()
        torch.cuda.empty_cache()


def form_batched_sharded(P, torch, args, ws, rank):
    """The batched workload split over the ranks (cost-balanced, no data
    exchange): every rank builds and times its own share as one graph step;
    the batch's rate is set by the slowest rank."""
    from paper_2107_03285_gb300 import shard
    subs = _batch_instances(args)
    sides = [int(round(np.sqrt(sub.n_nodes))) for sub in subs]
    parts = shard.partition(shard.instance_costs(sides), ws)
    mine = [subs[i] for i in parts[rank]]
    s = P.SGN.from_batch(mine, stores=P.STORE_MIXED | P.STORE_KFACT_MIXED)
    try:
        p0 = np.concatenate([sub.p0 for sub in mine])
        fext = np.concatenate([sub.fext for sub in mine])
        x, rep = s.equilibrium(p0, fext, precision=P.MIXED)
        p = torch.as_tensor(p0, device=x.device)
        out = (torch.empty_like(x), torch.empty_like(p), torch.empty_like(x))
        for _ in range(3):
            s.step_graph(x, p, P.MIXED, refine_steps=4, out=out, residual=False)
        n = 10
        torch.distributed.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        for _ in range(n):
            s.step_graph(x, p, P.MIXED, refine_steps=4, out=out, residual=False)
        e1.record(s.stream)
        e1.synchronize()
        ms = shard.max_over_ranks(e0.elapsed_time(e1) / n, device=x.device)
        k = len(subs)
        return {"workload": f"{args.batch_workload} over {ws} ranks (cost-balanced, no collective on the data path)",
                "instances_per_rank": [int(len(q)) for q in parts], "ms_per_step_slowest_rank": ms,
                "steps_per_s": 1e3 / ms, "instance_steps_per_s": k * 1e3 / ms, "scaling": "strong"}
    finally:
        s.close()
        torch.cuda.empty_cache()


def form_scale(P, torch, args):
    """The 80^3-node cube in the mixed path (FP32 fronts on the tensor cores,
    FP64 refinement): mixed Newton to the equilibrium, then timed SGN steps;
    the FP64 path does not fit beside it (its fronts alone need 298 GB) and
    would take minutes per factorization, so accuracy is shown by the FP64
    residual of the full system and the inertia."""
    from sgn_inputs import make_preset
    prob = make_preset(args.scale_workload, seed=args.seed)
    (s, t_setup) = _timed(torch, lambda: P.SGN.from_problem(prob, stores=P.STORE_MIXED | P.STORE_KFACT_MIXED))
    try:
        (x, rep), t_eq = _timed(torch, lambda: s.equilibrium(prob.p0, prob.fext, precision=P.MIXED))
        p = torch.as_tensor(prob.p0, device=x.device)
        out = (torch.empty_like(x), torch.empty_like(p), torch.empty_like(x))
        s.assemble(x, p)
        frep = s.factor(P.MIXED)
        _, _, _, srep = s.solve(P.RHS_KKT, out=out)
        n = 2
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(n):
            s.assemble(x, p)
            s.factor(P.MIXED, report=False)
            s.solve(P.RHS_KKT, report=False, out=out)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / n
        n_x = prob.n_free * prob.dim
        return {"workload": f"{args.scale_workload}: {prob.n_elem} tets, {prob.n_nodes} nodes, "
                            f"N={int(s.info.n_kkt)}",
                "precision": "mixed", "steps_per_s": 1e3 / ms, "ms_per_step": ms,
                "factor_tflops": s.info.factor_flops / (ms * 1e-3) / 1e12,
                "device_gb": s.buf.numel() / 1e9, "setup_and_bind_s": t_setup,
                "kkt_residual": srep.residual, "refine_steps": srep.refine_steps,
                "inertia_ok": (frep.n_pos, frep.n_neg, frep.n_zero) == (n_x + prob.n_elem, n_x, 0),
                "factor_flops": s.info.factor_flops, "nnz_factor": s.info.nnz_factor,
                "equilibrium_mixed": {"iters": rep.iters, "residual": rep.residual, "seconds": t_eq}}
    finally:
        s.close()
        torch.cuda.empty_cache()


def form_warm_start(P, torch, args):
    """Learned warm start on the RBF-parameterised cube: equilibria at seeded
    designs theta ~ N(0, 0.3^2) as snapshots (mixed Newton from the rest
    shape), randomised-SVD basis, BF16 MLP trained by the library's AdamW
    kernels, then Newton on held-out designs from (a) the rest shape, (b) the
    previous iterate (the equilibrium of a design one step away) and (c) the
    better of the learned prediction and (b)."""
    from sgn_inputs import draw_thetas, make_preset
    prob = make_preset(args.warm_workload, seed=args.seed)
    ns, nt = args.warm_snapshots, args.warm_tests
    s = P.SGN.from_problem(prob, stores=P.STORE_KFACT_MIXED)
    n_modes = min(128, ns - 1)
    ws = P.WarmStart(s, prob.meta["rbf_centers"], prob.meta["rbf_width"], n_modes=n_modes, hidden=512,
                     max_snap=ns, batch=min(64, ns))
    try:
        # designs whose Newton solve does not converge (the far tail of theta)
        # are replaced by further draws, and counted
        spare = max(8, ns // 16)
        thetas_all = draw_thetas(prob, ns + nt + spare, seed=args.seed + 101)
        X = torch.as_tensor(prob.X, device="cuda")
        snaps = torch.empty((ns,) + tuple(X.shape), dtype=torch.float64, device="cuda")
        cold_it, cold_t, kept, failed = [], [], [], []
        for i in range(ns + spare):
            if len(kept) == ns:
                break
            (x, rep), dt = _timed(torch, lambda: s.equilibrium(ws.rbf_params(thetas_all[i]), prob.fext,
                                                               precision=P.MIXED))
            if not rep.converged:
                failed.append({"iters": rep.iters, "residual": rep.residual})
                continue
            snaps[len(kept)] = x - X
            kept.append(i)
            cold_it.append(rep.iters)
            cold_t.append(dt)
        if len(kept) < ns:
            raise RuntimeError(f"only {len(kept)} of {ns} snapshot equilibria converged: {failed[:4]}")
        used = set(kept)
        rest = [i for i in range(len(thetas_all)) if i not in used and i > kept[-1]]
        thetas = np.concatenate([thetas_all[kept], thetas_all[rest[:nt]]])
        _, t_basis = _timed(torch, lambda: ws.fit_basis(snaps, seed=1))
        steps = args.warm_train_steps
        loss, t_train = _timed(torch, lambda: ws.train(thetas[:ns], snaps, steps=steps, lr=1e-3,
                                                       weight_decay=1e-5, seed=2))
        rng = np.random.default_rng(args.seed + 7)
        arms = ("rest", "learned", "prev_small", "learned_or_prev_small", "prev_large", "learned_or_prev_large")
        res = {a: [] for a in arms}

        def rec(arm, r, t, used=None):
            e = {"iters": r.iters, "initial_residual": r.initial_residual, "residual": r.residual,
                 "converged": bool(r.converged), "seconds": t}
            if used is not None:
                e["used_learned"] = bool(used)
            res[arm].append(e)

        for th in thetas[ns:]:
            pd = ws.rbf_params(th)
            (_, r), t = _timed(torch, lambda: s.equilibrium(pd, prob.fext, precision=P.MIXED))
            rec("rest", r, t)
            (_, r, used), t = _timed(torch, lambda: ws.equilibrium(th, prob.fext, precision=P.MIXED))
            rec("learned", r, t, used)
            # previous iterate: the equilibrium of a design one SGN step away
            # (small: 10% of theta's spread per coefficient; large: 50%)
            for tag, sig in (("small", 0.03), ("large", 0.15)):
                xp, _ = s.equilibrium(ws.rbf_params(th + rng.normal(0.0, sig, size=th.shape)), prob.fext,
                                      precision=P.MIXED)
                (_, r), t = _timed(torch, lambda: s.equilibrium(pd, prob.fext, x0=xp, precision=P.MIXED))
                rec("prev_" + tag, r, t)
                (_, r, used), t = _timed(torch, lambda: ws.equilibrium(th, prob.fext, x_prev=xp,
                                                                        precision=P.MIXED))
                rec("learned_or_prev_" + tag, r, t, used)

        def summ(v):
            out = {"mean_iters": float(np.mean([e["iters"] for e in v])),
                   "median_initial_residual": float(np.median([e["initial_residual"] for e in v])),
                   "max_final_residual": float(max(e["residual"] for e in v)),
                   "all_converged": all(e["converged"] for e in v),
                   "mean_seconds": float(np.mean([e["seconds"] for e in v]))}
            if "used_learned" in v[0]:
                out["used_learned"] = int(sum(e["used_learned"] for e in v))
            return out
        out = {k: summ(v) for k, v in res.items()}
        return {"workload": f"{args.warm_workload}: {prob.n_elem} tets, {prob.n_nodes} nodes, "
                            f"{prob.meta['n_rbf']} RBF coefficients",
                "size": (f"{ns} snapshots" + (" (as configured)" if ns >= 4096 else " (reduced from 4,096)") +
                         f", {n_modes} modes, MLP {prob.meta['n_rbf']}-512-512-{n_modes}, {steps} AdamW steps; "
                         f"held-out designs: {nt}"),
                "snapshots": {"mean_iters": float(np.mean(cold_it)), "mean_seconds": float(np.mean(cold_t)),
                              "not_converged": len(failed), "not_converged_sample": failed[:4]},
                "basis_seconds": t_basis, "train_seconds": t_train, "train_final_loss": loss,
                "newton_from": out,
                "iters_saved_vs_rest": out["rest"]["mean_iters"] - out["learned"]["mean_iters"],
                "iters_saved_vs_prev_small": out["prev_small"]["mean_iters"]
                - out["learned_or_prev_small"]["mean_iters"],
                "iters_saved_vs_prev_large": out["prev_large"]["mean_iters"]
                - out["learned_or_prev_large"]["mean_iters"]}
    finally:
        ws.close()
        s.close()
        torch.cuda.empty_cache()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    import __graft_entry__
    __graft_entry__.build()
    import paper_2107_03285_gb300 as P
    from sgn_inputs import make_preset

    prob = make_preset(args.workload, seed=args.seed)
    prec = P.MIXED if args.precision == "mixed" else P.FP64
    stores = P.STORE_KFACT | P.STORE_FP64 | (P.STORE_MIXED | P.STORE_KFACT_MIXED if prec == P.MIXED else 0)
    from paper_2107_03285_gb300 import autotune
    tuned = autotune.lookup(prob, prec)
    leaf, panel = tuned if tuned else (0, 0)
    t_setup = time.perf_counter()
    s = P.SGN.from_problem(prob, stores=stores, leaf_nodes=leaf, panel=panel)
    t_setup = time.perf_counter() - t_setup
    buf_gb = s.buf.numel() / 1e9
    info = s.info
    # forward simulation to the equilibrium the step is taken at (reported separately)
    (xeq, nrep), t_eq = _timed(torch, lambda: s.equilibrium(prob.p0, prob.fext, precision=prec))
    equilibrium = {"precision": args.precision, "iters": nrep.iters, "residual": nrep.residual, "seconds": t_eq}
    if prec == P.MIXED:
        (x64, r64), t64 = _timed(torch, lambda: s.equilibrium(prob.p0, prob.fext, precision=P.FP64))
        equilibrium["fp64"] = {"iters": r64.iters, "residual": r64.residual, "seconds": t64,
                               "max_abs_dx_vs_mixed": float((x64 - xeq).abs().max())}
        del x64
    p = torch.as_tensor(prob.p0, device=dev)
    out = (torch.empty_like(xeq), torch.empty_like(p), torch.empty_like(xeq))

    def step(precision):
        s.assemble(xeq, p)
        s.factor(precision, report=False)
        return s.solve(P.RHS_KKT, report=False, out=out)

    # plain FP64 GPU path: reference accuracy and its own rate
    fp64 = None
    dp64 = None
    if args.fp64_steps > 0 or prec == P.FP64:
        step(P.FP64)
        torch.cuda.synchronize()
        dp64 = out[1].clone()
        if args.fp64_steps > 0 and prec != P.FP64:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.fp64_steps):
                step(P.FP64)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.fp64_steps
            fp64 = {"steps_per_s": 1e3 / ms, "ms_per_step": ms,
                    "factor_tflops": info.factor_flops / (ms * 1e-3) / 1e12}

    for _ in range(args.warmup):
        step(prec)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = s.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        torch.cuda.nvtx.range_push("sgn_timed")
        e0.record()
        for _ in range(args.steps):
            step(prec)
        e1.record()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    launches = s.launch_count() - launches0
    ms = e0.elapsed_time(e1) / args.steps
    if ws > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
        torch.distributed.barrier()
    value = ws * 1e3 / ms
    dp = out[1].clone()
    # the dominant kernel kind (trailing update) timed in separate steps (CUDA
    # events around every launch inside the captured factorization graph), so
    # that the headline steps above run without profiling events
    prof_steps = 2
    s.profile(1)
    for _ in range(prof_steps):
        step(prec)
    torch.cuda.synchronize()
    prof_launches, prof_seconds, prof_flops = s.profile_read()["update"]
    s.profile(0)
    # phases of one unprofiled step (CUDA events between the calls)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record()
    s.assemble(xeq, p)
    ev[1].record()
    s.factor(prec, report=False)
    ev[2].record()
    s.solve(P.RHS_KKT, report=False, out=out)
    ev[3].record()
    torch.cuda.synchronize()
    phases = {"assemble_ms": ev[0].elapsed_time(ev[1]), "factor_ms": ev[1].elapsed_time(ev[2]),
              "solve_ms": ev[2].elapsed_time(ev[3]), "source": "one unprofiled step, events between the calls"}
    # per-kernel-kind breakdown of one extra (profiled) step
    s.profile(0xFF)
    s.assemble(xeq, p)
    s.factor(prec, report=False)
    s.solve(P.RHS_KKT, report=False, out=out)
    torch.cuda.synchronize()
    kinds = {k: {"launches": v[0], "ms": 1e3 * v[1], "tflops": (v[2] / v[1] / 1e12) if v[1] > 0 and v[2] > 0 else None}
             for k, v in s.profile_read().items() if v[0] > 0}
    s.profile(0)
    dp_err = float(torch.linalg.norm(dp - dp64) / torch.linalg.norm(dp64)) if dp64 is not None else None
    _, _, _, srep = s.solve(P.RHS_KKT, report=True, out=out)

    # end to end through the C ABI with host buffers (H2D of x, p; D2H of dx, dp, dl)
    xh = torch.empty(tuple(xeq.shape), dtype=torch.float64, pin_memory=True)
    xh.copy_(xeq)
    ph = torch.empty(tuple(p.shape), dtype=torch.float64, pin_memory=True)
    ph.copy_(p)
    xnp, pnp = xh.numpy(), ph.numpy()
    e2e = None  # --e2e-steps 0: not measured
    if args.e2e_steps > 0:
        s.step_host(xnp, pnp, prec)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            s.step_host(xnp, pnp, prec)
        e2e_dt = (time.perf_counter() - t0) / args.e2e_steps
        e2e = {"value": ws / e2e_dt, "unit": UNIT, "h2d_bytes_per_step": int(xnp.nbytes + pnp.nbytes),
               "d2h_bytes_per_step": int(2 * xnp.nbytes + pnp.nbytes)}

    sharded = None
    if ws > 1 and args.batch_workload:
        s.close()
        torch.cuda.empty_cache()
        try:
            sharded = form_batched_sharded(P, torch, args, ws, rank)
        except Exception as e:  # reported, not hidden
            sharded = {"error": f"{type(e).__name__}: {e}"}
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    peaks = json.load(open(MEASURED)) if os.path.exists(MEASURED) else {}
    run_peaks = measure_peaks(torch)
    hbm = peaks.get("hbm_gbs") or 6800.0
    hbm_src = "of measured (MEASURED_PEAKS.json hbm_gbs)" if peaks.get("hbm_gbs") else "of fallback 6.8 TB/s"
    fp32 = prec == P.MIXED
    achieved = prof_flops / prof_seconds / 1e12 if prof_seconds > 0 else None
    upd_launch_flops = prof_flops / max(prof_launches, 1)
    if fp32:
        peak = run_peaks["tf32_tflops"]
        roofline = {"kernel": "k_update_tcp (tcgen05 3xTF32 trailing Schur update, TMEM accumulators)",
                    "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak if achieved else None,
                    "peak_source": "of measured in this run: " + run_peaks["tf32_how"],
                    "tensor_pipe_frac_3xtf32": 3 * achieved / peak if achieved else None,
                    "note": "achieved counts useful FP32 flops (2 x lower-triangle entries x inner dimension per "
                            "outer block, summed on the host) over the update launches' CUDA-event time in "
                            f"{prof_steps} profiled steps; 3xTF32 issues three TF32 MMAs per product"}
        # algorithmic bytes of an update launch: the C tile read and written
        # (FP32) plus the four K-major operand arrays of the block (FP32)
        if UPDATE_DRAM_PER_ALGO_BYTE is not None:
            algo_b = upd_launch_flops / (2.0 * 256) * 8.0
            roofline["traffic"] = UPDATE_DRAM_PER_ALGO_BYTE * algo_b
            roofline["traffic_source"] = ("DRAM bytes per algorithmic byte from the ncu capture in "
                                          "profiles/k_update_tcp_kuhn3d_24.md, scaled to this workload's mean launch")
        else:
            roofline["traffic"] = None
    else:
        peak = run_peaks["fp64_tflops"]
        roofline = {"kernel": "k_update (FP64 DFMA trailing Schur update)", "bound": "alu", "achieved": achieved,
                    "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak if achieved else None,
                    "traffic": None, "peak_source": "of measured in this run: " + run_peaks["fp64_how"]}
    roofline["launches_per_step"] = prof_launches / prof_steps
    roofline["share_of_step"] = prof_seconds / prof_steps / (ms * 1e-3)
    # HBM-bound phases: algorithmic bytes per step over their event-timed phase
    d, ne, nn = prob.dim, prob.n_elem, prob.n_nodes
    nnz_upper = (int(info.nnz_kkt) + int(info.n_kkt)) // 2
    asm_bytes = ne * (4 * (d + 1) + 8 * (d * d + 2)) + nn * 8 * d + nnz_upper * 8 + int(info.n_kkt) * 8
    n_solves = 1 + srep.refine_steps
    solve_bytes = n_solves * 2 * int(info.nnz_factor) * (4 if fp32 else 8)
    hbm_phases = {
        "assembly": {"bytes_per_step": asm_bytes, "ms": phases["assemble_ms"],
                     "gbs": asm_bytes / (phases["assemble_ms"] * 1e-3) / 1e9,
                     "frac": asm_bytes / (phases["assemble_ms"] * 1e-3) / 1e9 / hbm, "peak_gbs": hbm,
                     "peak_source": hbm_src,
                     "bytes": "n_e (4 (d+1) + 8 (d^2 + 2)) + n_nodes 8 d + nnz_upper(KKT) 8 + N 8"},
        "solves": {"bytes_per_step": solve_bytes, "solves_per_step": n_solves, "ms": phases["solve_ms"],
                   "gbs": solve_bytes / (phases["solve_ms"] * 1e-3) / 1e9,
                   "frac": solve_bytes / (phases["solve_ms"] * 1e-3) / 1e9 / hbm, "peak_gbs": hbm,
                   "peak_source": hbm_src,
                   "bytes": "solves x 2 nnz(L) x (4 FP32 | 8 FP64); the phase also holds the FP64 residuals"},
    }
    if ws == 1 and args.cpu_seconds > 0:
        cpu_rate, cpu_info = oracle_step_rate(args.cpu_sample, args.cpu_seconds, args.seed)
        cpu_info["value"] = cpu_rate
        cpu_info["unit"] = UNIT
    else:
        cpu_info = None  # the oracle baseline is timed at N = 1 only (--cpu-seconds 0: not at all)
    N = int(info.n_kkt)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if fp32 else "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {prob.n_elem} tets, {prob.n_nodes} nodes, N={N} saddle-point "
                               f"unknowns, p = per-tet log-modulus",
                   "precision": args.precision, "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU",
                   "setup_options": {"leaf_nodes": leaf or 16, "panel": panel or 32,
                                     "source": "autotuned (paper_2107_03285_gb300/tuned.json)" if tuned
                                     else "defaults"},
                   "l2": f"not flushed: the step's working set ({buf_gb:.1f} GB) exceeds L2",
                   "dp_rel_err_vs_fp64_gpu": dp_err, "refine_steps": srep.refine_steps,
                   "kkt_residual": srep.residual,
                   "refine_history": [float(v) for v in list(srep.history)[:srep.refine_steps + 1]],
                   "factor_flops": info.factor_flops,
                   "nnz_factor": info.nnz_factor, "fp64_path": fp64,
                   "phases": phases, "kernel_kinds_profiled_step": kinds, "setup_s": info.setup_seconds, "bind_s": t_setup,
                   "hbm_phases": hbm_phases, "measured_peaks": run_peaks,
                   "equilibrium": equilibrium},
        "roofline": roofline,
        "cpu_baseline": cpu_info,
        "e2e": e2e,
        "clocks": clk.summary(),
        "gpu_launches": launches,
    }
    if s.h is not None:
        s.close()
    del s
    torch.cuda.empty_cache()
    if sharded is not None:
        line["config"]["forms"] = {"batched_sharded": sharded}
    if ws == 1:
        forms = {}
        for name, fn, wl in (("batched", form_batched, args.batch_workload),
                             ("learned_warm_start", form_warm_start, args.warm_workload),
                             ("scale", form_scale, args.scale_workload)):
            if not wl:
                continue
            try:
                forms[name] = fn(P, torch, args)
            except Exception as e:  # a form that fails is reported, not hidden
                forms[name] = {"error": f"{type(e).__name__}: {e}"}
        line["config"]["forms"] = forms
    print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
