#!/usr/bin/env python
"""Benchmark: nnz/s to a 1e-8 relative residual on one GB300 per rank.

Workload (default): R-MAT scale 26, edge factor 16 (2^30 sampled edges),
(a, b, c, d) = (.57, .19, .19, .05), symmetrised, deduplicated, unit weights,
largest component kept (n = 32.8M, nnz(L) = 2.1e9), generated on the device.
A step is one pass of the whole path on that graph: hierarchy setup
(elimination, strength, aggregation, Galerkin, eigenvalue estimates, coarsest
pseudo-inverse), then one PCG solve with the FP64 V-cycle and one with the
FP32 hierarchy inside FP64 PCG, each to ||b - L x|| / ||b|| <= 1e-8 in FP64.

value = nnz(L_0) / T_solve(FP64), whole job (summed over ranks, each rank
solving its own replica; timings are the max over ranks). The FP32-hierarchy
solve, setup time, setup-inclusive throughput and each result's error against
a 1e-12 solve are reported beside it; the 1M-vertex Chung-Lu graph and the
64 x 64 grid run as secondary legs with errors against the oracle.

--impl reference times the FP64 oracle on the host cores instead, on a
bounded sample of the same workload.
"""

from __future__ import annotations

import argparse
import datetime
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "nnz/s to 1e-8 rel-res, FP32-hier vs FP64 on same GB300; serve p50/p99 ms"
UNIT = "nnz/s"
TOL = 1e-8
L2_BYTES = 129 * 2 ** 20
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e nominal, for the fraction of nominal



def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["lg", "reference"], default="lg")
    ap.add_argument("--workload", default="rmat_26")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-multi-rhs", action="store_true")
    ap.add_argument("--multi-rhs-k", type=int, default=32)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-kcycle", action="store_true")
    ap.add_argument("--no-wda", action="store_true")
    ap.add_argument("--no-ordering", action="store_true")
    ap.add_argument("--no-secondary", action="store_true")
    ap.add_argument("--no-many", action="store_true")
    ap.add_argument("--many-graphs", type=int, default=608)
    ap.add_argument("--serve-graphs", type=int, default=256)
    ap.add_argument("--serve-nmax", type=int, default=2000000)
    ap.add_argument("--serve-requests", type=int, default=600)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-load", type=float, default=0.8)
    ap.add_argument("--serve-headline-only", action="store_true",
                    help="serve only the headline load, least work first (for long runs: --serve-requests 10000)")
    return ap.parse_args()


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        # a replica that fails ends the others' next barrier with an error
        # after this long instead of holding every GPU of the job
        timeout = datetime.timedelta(seconds=float(os.environ.get("BENCH_PG_TIMEOUT_S", "600")))
        dist.init_process_group(backend=backend, timeout=timeout)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def allreduce_max(vals, world):
    if world == 1:
        return list(vals)
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor(vals, dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.cpu().tolist()


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("lg_rows.cuh", "lg_cycle.cu", "lg_common.cuh"):
        with open(os.path.join(ROOT, "paper_1705_06266_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(workload):
    """DRAM bytes per launch of the dominant kernel from a committed ncu summary,
    or None when there is none or the kernel source changed since it was taken."""
    path = os.path.join(ROOT, "profiles", f"k_rows_lap_{workload}.txt")
    if not os.path.exists(path):
        return None, None
    fields = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            fields[k.strip()] = v.strip()
    if fields.get("kernel_source_hash") != kernel_source_hash():
        return None, fields.get("kernel_source_hash")
    try:
        return float(fields["dram_bytes_per_launch"]), fields.get("kernel_source_hash")
    except (KeyError, ValueError):
        return None, None


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(device)], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=10)
        except Exception:
            self.p.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# The bounded sample the oracle is timed on for the R-MAT scale-26 workload:
# an R-MAT graph of the same recipe (edge factor 16, (a, b, c) = (.57, .19,
# .19), symmetrised, deduplicated, unit weights, largest component) at scale
# 20, generated with torch on the host so that both arms time the same graph.
SAMPLE_SCALE = 20


def rmat_sample():
    import torch

    from paper_1705_06266_gb300 import inputs

    n, rp, cl, w = inputs.rmat_device(SAMPLE_SCALE, seed=1, device="cpu")
    return inputs.Graph(n, rp.numpy(), cl.numpy(), w.numpy(), name=f"rmat_{SAMPLE_SCALE}_16_host_torch")


def cpu_baseline(workload_name, g, b, note=""):
    """The oracle as it stands, single-threaded, on a bounded sample of the
    workload: its setup untimed, one FP64 PCG solve to 1e-8 timed."""
    import oracle

    oracle.build()
    t0 = time.perf_counter()
    h = oracle.Hierarchy(g)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    x, st, it, rel = h.pcg(b, tol=TOL)
    t_solve = time.perf_counter() - t0
    return {
        "value": g.nnz / t_solve, "unit": UNIT, "cores": 1, "kind": "oracle",
        "sample": f"{note}{g.name} (n={g.n}, nnz(L)={g.nnz}), one right-hand side: oracle setup "
                  f"{t_setup:.1f} s untimed, one FP64 PCG solve to 1e-8 timed ({it} iterations, "
                  f"relres {rel:.2e})",
        "solve_s": t_solve, "setup_s": t_setup,
    }


def rel_err(x, ref):
    """Relative 2-norm error of x against ref, both with their means removed
    (the solution of a Laplacian system is unique up to a constant)."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    d = (x - x.mean()) - (ref - ref.mean())
    return float(np.linalg.norm(d) / np.linalg.norm(ref - ref.mean()))


_GRAPHS = {}


def workload(inputs, name):
    """inputs.workload(name), generated once per run."""
    if name not in _GRAPHS:
        _GRAPHS[name] = inputs.workload(name)
    return _GRAPHS[name]


def multi_rhs_leg(lg, inputs, torch, dev, k):
    """k right-hand sides solved together (FP32 hierarchy, SpMM cycles, FP64
    outer CG) against the same k solved one after another, on the R-MAT scale
    20 graph and the 128^3 grid. Device-resident B and X; each figure is the
    solve's own event time."""
    out = {}
    for name in ("rmat_20", "grid3d_128"):
        g = workload(inputs, name)
        B = inputs.rhs(g.n, k, seed=3)
        Bd = torch.from_numpy(np.ascontiguousarray(B.T)).to(dev)  # column-major n x k
        Xd = torch.zeros_like(Bd)
        torch.cuda.synchronize()
        h = lg.lg_setup(g.n, g.rowptr, g.col, g.w, lg.options())
        lg.lg_set_precision(h, lg.FP32_HIER)
        lg.lg_solve_batch(h, k, Bd, g.n, Xd, g.n, TOL)  # warm-up (plans, workspace)
        lg.lg_solve(h, Bd[0], Xd[0], TOL)
        torch.cuda.synchronize()
        infos = lg.lg_solve_batch(h, k, Bd, g.n, Xd, g.n, TOL)
        batch_ms = infos[0].solve_ms
        seq_ms, seq_it = 0.0, []
        for c in range(k):
            inf = lg.lg_solve(h, Bd[c], Xd[c], TOL)
            seq_ms += inf.solve_ms
            seq_it.append(inf.iterations)
        nlev = lg.lg_hier_info(h).levels
        levels = [lg.lg_level_info(h, l) for l in range(nlev)]
        sched = [lg.lg_batch_plan(h, l) for l in range(nlev)]
        lg.lg_destroy(h)
        # the same batched solve on the fixed schedule (no timing-based choices: stretches of 256 entries, E = 4)
        hf = lg.lg_setup(g.n, g.rowptr, g.col, g.w, lg.options(autotune=0))
        lg.lg_set_precision(hf, lg.FP32_HIER)
        lg.lg_solve_batch(hf, k, Bd, g.n, Xd, g.n, TOL)
        torch.cuda.synchronize()
        fixed_ms = lg.lg_solve_batch(hf, k, Bd, g.n, Xd, g.n, TOL)[0].solve_ms
        lg.lg_destroy(hf)
        out[name] = {
            "n": g.n, "nnz": g.nnz, "k": k,
            "levels": [{q: lv[q] for q in ("kind", "n", "nnz", "nc")} for lv in levels],
            "batched_ms": batch_ms, "batched_nnz_per_s": g.nnz * k / (batch_ms * 1e-3),
            "batched_iterations_max": max(i.iterations for i in infos),
            "batched_relres_max": max(i.relres for i in infos),
            "sequential_ms": seq_ms, "sequential_nnz_per_s": g.nnz * k / (seq_ms * 1e-3),
            "sequential_iterations_max": max(seq_it),
            "speedup": seq_ms / batch_ms,
            "schedule": [dict(s, level=l) for l, s in enumerate(sched) if s["op_ch"] or s["w_ch"]],
            "fixed_schedule_ms": fixed_ms, "tuned_vs_fixed": fixed_ms / batch_ms,
        }
    return out


def kcycle_leg(lg, inputs, torch, dev):
    """The K-cycle (Section 3.7) beside the V-cycle: single right-hand-side
    solves to 1e-8 from device-resident b, in both precisions, on the 1M
    Chung-Lu graph and on the 128^3 grid (where the V-cycle needs many
    iterations)."""
    out = {}
    for name in ("chung_lu_1m", "grid3d_128"):
        g = workload(inputs, name)
        b = inputs.rhs(g.n, seed=2)
        bd = torch.from_numpy(b).to(dev)
        xd = torch.zeros_like(bd)
        torch.cuda.synchronize()
        row = {"n": g.n, "nnz": g.nnz}
        for cyc in ((0, 1) if name == "grid3d_128" else (1,)):
            h = lg.lg_setup(g.n, g.rowptr, g.col, g.w, lg.options(kcycle=cyc))
            tag = "k" if cyc else "v"
            for pname, prec in (("fp64", lg.FP64), ("fp32", lg.FP32_HIER)):
                lg.lg_set_precision(h, prec)
                lg.lg_solve(h, bd, xd, TOL)  # warm-up (graph capture)
                inf = lg.lg_solve(h, bd, xd, TOL)
                row[f"{tag}_{pname}_ms"] = inf.solve_ms
                row[f"{tag}_{pname}_iterations"] = inf.iterations
                row[f"{tag}_{pname}_nnz_per_s"] = g.nnz / (inf.solve_ms * 1e-3)
            lg.lg_destroy(h)
        out[name] = row
    return out


def wda_leg(lg, inputs, torch, dev):
    """Work per digit of accuracy (Section 2.3.1) on a synthetic suite of the
    paper's graph families at ~10^5 vertices, FP64 solves to 1e-8, for the
    V-cycle, the K-cycle and the V-cycle with four elimination rounds."""
    suite = [
        ("grid2d_300", lambda: inputs.grid2d(300, 300)),
        ("grid3d_45", lambda: inputs.grid3d(45, 45, 45)),
        ("chung_lu_100k", lambda: inputs.chung_lu(100000, m_target=500000, seed=11)),
        ("rmat_17", lambda: inputs.rmat(17, seed=11)),
        ("random_100k", lambda: inputs.random_graph(100000, 6, seed=11)),
        ("road_like_400", lambda: inputs.road_like(400, 400, seed=11)),
    ]
    configs = [("v", {}), ("k", {"kcycle": 1}), ("v_elim4", {"elim_rounds": 4})]
    out = {"graphs": {}}
    for name, make in suite:
        g = make()
        b = inputs.rhs(g.n, seed=2)
        bd = torch.from_numpy(b).to(dev)
        xd = torch.zeros_like(bd)
        torch.cuda.synchronize()
        row = {"n": g.n, "nnz": g.nnz}
        for tag, kw in configs:
            h = lg.lg_setup(g.n, g.rowptr, g.col, g.w, lg.options(**kw))
            lg.lg_solve(h, bd, xd, TOL)
            inf = lg.lg_solve(h, bd, xd, TOL)
            row[tag] = {"iterations": inf.iterations, "work_units": inf.work_units,
                        "wda": inf.work_units / -math.log10(max(inf.relres, 1e-300)),
                        "solve_ms": inf.solve_ms, "levels": inf.levels}
            lg.lg_destroy(h)
        out["graphs"][name] = row
    for tag, _ in configs:
        out[f"median_wda_{tag}"] = statistics.median(r[tag]["wda"] for r in out["graphs"].values())
    out["note"] = ("WDA = work_units / -log10(relres); work in finest-residual units counted from operator "
                   "nonzeros (lg_info.work_units)")
    return out


def ordering_leg(lg, torch, dev, graphs):
    """Vertex orderings (Section 3.3 uses a random one): the caller's, by
    descending degree (the default) and random; setup and FP64/FP32 solves."""
    out = {}
    for name, g, b in graphs:
        bd = torch.from_numpy(b).to(dev)
        xd = torch.zeros_like(bd)
        torch.cuda.synchronize()
        row = {}
        for tag, code in (("caller", 0), ("degree", 1), ("random", 2)):
            h = lg.lg_setup(g.n, g.rowptr, g.col, g.w, lg.options(reorder=code))
            r = {"setup_ms": lg.lg_hier_info(h).setup_ms}
            for pname, prec in (("fp64", lg.FP64), ("fp32", lg.FP32_HIER)):
                lg.lg_set_precision(h, prec)
                lg.lg_solve(h, bd, xd, TOL)
                inf = lg.lg_solve(h, bd, xd, TOL)
                r[f"{pname}_ms"] = inf.solve_ms
                r[f"{pname}_iterations"] = inf.iterations
            lg.lg_destroy(h)
            row[tag] = r
        out[name] = row
    return out


def secondary_leg(lg, inputs, torch, dev, name, flush, oracle_ref):
    """Another configuration of the metric: setup, then FP64 and FP32-hierarchy
    solves to 1e-8 from device-resident b (median of 3, L2 flushed before
    each), with each result's error against the oracle's solution: the dense
    direct solve on the 64 x 64 grid, the oracle's own PCG to 1e-12 on larger
    graphs."""
    g = workload(inputs, name)
    b = inputs.rhs(g.n, seed=2)
    rp, cl, w = (torch.from_numpy(a).to(dev) for a in (g.rowptr, g.col, g.w))
    bd = torch.from_numpy(b).to(dev)
    xd = torch.zeros_like(bd)
    torch.cuda.synchronize()
    out = {"n": g.n, "nnz": g.nnz}
    setups = []
    for _ in range(3):
        flush.fill_(1.0)
        h = lg.lg_setup(g.n, rp, cl, w, lg.options())
        setups.append(lg.lg_hier_info(h).setup_ms)
        lg.lg_destroy(h)
    out["setup_ms"] = sorted(setups)[1]
    h = lg.lg_setup(g.n, rp, cl, w, lg.options())
    xs = {}
    for tag, prec in (("fp64", lg.FP64), ("fp32", lg.FP32_HIER)):
        lg.lg_set_precision(h, prec)
        lg.lg_solve(h, bd, xd, TOL)  # warm-up (graph capture)
        runs = []
        for _ in range(3):
            flush.fill_(2.0)
            runs.append(lg.lg_solve(h, bd, xd, TOL))
        inf = sorted(runs, key=lambda i: i.solve_ms)[1]
        xs[tag] = xd.cpu().numpy()
        out[tag] = {"solve_ms": inf.solve_ms, "iterations": inf.iterations, "relres": inf.relres,
                    "nnz_per_s": g.nnz / (inf.solve_ms * 1e-3)}
    out["fp32_speedup"] = out["fp64"]["solve_ms"] / out["fp32"]["solve_ms"]
    lg.lg_destroy(h)
    if oracle_ref:
        import oracle

        oracle.build()
        if g.n <= 4096:
            ref = oracle.dense_solve(g, b)
            out["x_reference"] = "oracle dense direct solve (pinv of L)"
        else:
            ref, st, it, rel = oracle.Hierarchy(g).pcg(b, tol=1e-12, maxit=1000)
            out["x_reference"] = f"oracle FP64 PCG to 1e-12 ({it} iterations, relres {rel:.1e})"
        for tag in xs:
            out[tag]["x_err_vs_oracle"] = rel_err(xs[tag], ref)
    return out


def serve_leg(lg, inputs, args, torch, dev):
    """Continuous batching over resident hierarchies (the serving workload):
    graphs of log-uniform sizes over four families, generated on the device
    and set up as FP32-only hierarchies (option fp32_only); a burst of
    requests measures the saturation rate, then Poisson arrivals at 0.5, 0.8
    and 0.95 of it give the latency percentiles (submission to completion,
    host B and X) and the served solves per second."""
    t0 = time.perf_counter()
    mix = inputs.serving_mix_device(args.serve_graphs, 1000, args.serve_nmax, seed=5, device=str(dev))
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    hs = []
    for name, n, rp, cl, w in mix:
        hs.append(lg.Hierarchy(n=n, rowptr=rp, col=cl, w=w, precision=lg.FP32_HIER, fp32_only=1))
    setup_s = time.perf_counter() - t0
    sizes = [m[1] for m in mix]
    nnzs = [int(m[3].numel()) + m[1] for m in mix]
    del mix
    torch.cuda.empty_cache()
    rng = np.random.Generator(np.random.PCG64(11))
    # one column-major block of 8 right-hand sides per graph; a request of k takes its first k
    blocks = [np.ascontiguousarray(inputs.rhs(n, 8, seed=20 + q).T) for q, n in enumerate(sizes)]

    def requests(count):
        return [(int(rng.integers(0, len(hs))), int(rng.integers(1, 9))) for _ in range(count)]

    # one server for every load point: the hierarchies are registered once (which builds their
    # multi-column plans and a ready workspace each); the statistics restart for each run
    t0 = time.perf_counter()
    sv = lg.lg_serve_create(lg.serve_options(slots=args.serve_slots, precision=lg.FP32_HIER,
                                             hbm_budget_bytes=120e9, policy=lg.SERVE_LEAST_WORK))
    for H in hs:
        lg.lg_serve_register(sv, H.h)
    register_s = time.perf_counter() - t0

    def run(reqs, rate):
        lg.lg_serve_reset_stats(sv)
        live, rhs, failed = {}, 0, 0
        t0 = time.perf_counter()
        arrival = 0.0
        for gi, k in reqs:
            if rate:
                arrival += rng.exponential(1.0 / rate)
                while time.perf_counter() - t0 < arrival:
                    for t in list(live):
                        done, info = lg.lg_serve_poll(sv, t)
                        if done:
                            failed += info.status != lg.OK
                            del live[t]
            X = np.empty((k, sizes[gi]))
            t = lg.lg_serve_submit(sv, hs[gi].h, k, blocks[gi][:k], X, TOL)
            live[t] = X
            rhs += k
        while live:
            for t in list(live):
                done, info = lg.lg_serve_poll(sv, t)
                if done:
                    failed += info.status != lg.OK
                    del live[t]
        span = time.perf_counter() - t0
        return lg.lg_serve_stats(sv), span, rhs, failed

    def closed_loop(reqs):
        """slots requests in flight at all times (a new one as one completes): the capacity
        without queueing, hence without merging."""
        lg.lg_serve_reset_stats(sv)
        live, rhs, nxt = {}, 0, 0
        t0 = time.perf_counter()
        while nxt < len(reqs) or live:
            while nxt < len(reqs) and len(live) < args.serve_slots:
                gi, k = reqs[nxt]
                X = np.empty((k, sizes[gi]))
                live[lg.lg_serve_submit(sv, hs[gi].h, k, blocks[gi][:k], X, TOL)] = X
                rhs += k
                nxt += 1
            for t in list(live):
                done, info = lg.lg_serve_poll(sv, t)
                if done:
                    del live[t]
        return lg.lg_serve_stats(sv), time.perf_counter() - t0, rhs

    n_probe = min(max(100, args.serve_requests // 4), 400)
    st_c, span_c, rhs_c = closed_loop(requests(n_probe))
    cap_rps = n_probe / span_c
    burst = requests(n_probe)  # every request queued at once: the most merging
    st_b, span_b, rhs_b, fail_b = run(burst, None)
    sat_rps = len(burst) / span_b
    loads = {}
    for load in sorted({args.serve_load} if args.serve_headline_only else {0.5, args.serve_load, 0.95}):
        rate = load * cap_rps
        st, span, rhs, failed = run(requests(args.serve_requests), rate)
        loads[load] = (rate, st, span, rhs, failed)
    arrival = None
    if not args.serve_headline_only:  # the headline load again in arrival order (bounded bypass), for comparison
        lg.lg_serve_set_policy(sv, lg.SERVE_ARRIVAL)
        st_a, span_a, rhs_a, fail_a = run(requests(args.serve_requests), args.serve_load * cap_rps)
        arrival = {"load": args.serve_load, "p50_ms": st_a.p50_ms, "p99_ms": st_a.p99_ms,
                   "solves_per_s": rhs_a / span_a, "groups": int(st_a.groups), "failed": int(st_a.failed + fail_a)}
    resident = sum(lg.lg_hier_bytes(H.h)[0] for H in hs)
    lg.lg_serve_destroy(sv)
    for H in hs:
        H.close()
    rate, st, span, rhs, failed = loads[args.serve_load]
    return {
        "p50_ms": st.p50_ms, "p99_ms": st.p99_ms, "mean_ms": st.mean_ms, "max_ms": st.max_ms,
        "solves_per_s": rhs / span, "requests_per_s": args.serve_requests / span,
        "offered_rps": rate, "capacity_rps": cap_rps, "capacity_solves_per_s": rhs_c / span_c,
        "capacity_p50_ms": st_c.p50_ms, "saturation_rps": sat_rps, "saturation_solves_per_s": rhs_b / span_b,
        "saturation_p50_ms": st_b.p50_ms, "saturation_p99_ms": st_b.p99_ms,
        "saturation_groups": int(st_b.groups), "saturation_packed_groups": int(st_b.packed_groups),
        "saturation_phase_ms": {"workspaces_made": int(st_b.workspaces_made), "workspace": st_b.workspace_ms,
                                "copy": st_b.copy_ms, "solve": st_b.solve_ms, "span": span_b * 1e3},
        "by_load": {f"{ld:g}": {"offered_rps": v[0], "p50_ms": v[1].p50_ms, "p99_ms": v[1].p99_ms,
                                "solves_per_s": v[3] / v[2], "requests": args.serve_requests,
                                "groups": int(v[1].groups), "packed_groups": int(v[1].packed_groups),
                                "failed": int(v[1].failed + v[4])}
                    for ld, v in loads.items()},
        "arrival_order": arrival,
        "completed": int(st.completed),
        "failed": int(sum(v[1].failed + v[4] for v in loads.values()) + st_b.failed + fail_b +
                      (arrival["failed"] if arrival else 0)),
        "requests": args.serve_requests, "graphs": len(hs),
        "vertices_resident": int(sum(sizes)), "nnz_resident": int(sum(nnzs)),
        "resident_bytes": float(resident), "generate_s": gen_s, "setup_s": setup_s, "register_s": register_s,
        "config": f"{len(hs)} resident graphs, n log-uniform in [1000, {args.serve_nmax}], type uniform over "
                  f"2D grid / 3D grid / Chung-Lu 2.1 / R-MAT ef16 (power-law members generated on the device); "
                  f"FP32-only hierarchies; k uniform in 1..8; tol 1e-8; {args.serve_slots} slots; policy least "
                  f"work first with aging (arrival order at the headline load in arrival_order); HBM budget "
                  f"120 GB; capacity = completion rate of {n_probe} requests with one in flight per slot (no "
                  f"queue, no merging); saturation = completion rate of a burst of {len(burst)} queued at once (the "
                  f"most merging); then Poisson arrivals at "
                  f"{'' if args.serve_headline_only else '0.5, '}{args.serve_load} (headline)"
                  f"{'' if args.serve_headline_only else ' and 0.95'} x capacity, "
                  f"{args.serve_requests} requests each; latency = submission to completion with host B and X",
    }


def many_leg(lg, inputs, count):
    """Many small graphs, one right-hand side each (host b and x): one
    lg_solve_many launch against one lg_solve call per graph, on the same
    hierarchies (FP32 hierarchy)."""
    graphs = inputs.serving_mix(count, 500, 5000, seed=31)
    hs = [lg.Hierarchy(g, precision=lg.FP32_HIER) for g in graphs]
    handles = [H.h for H in hs]
    bs = [inputs.rhs(g.n, seed=40 + q) for q, g in enumerate(graphs)]
    xs = [np.zeros(g.n) for g in graphs]
    lg.lg_solve_many(handles, bs, xs, TOL)  # warm-up (builds the device views)
    packed = []
    for _ in range(3):
        t0 = time.perf_counter()
        infos = lg.lg_solve_many(handles, bs, xs, TOL)
        packed.append(time.perf_counter() - t0)
    for H, b, x in zip(hs, bs, xs):  # warm-up (captures each handle's solve graph)
        lg.lg_solve(H.h, b, x, TOL)
    t0 = time.perf_counter()
    single = [lg.lg_solve(H.h, b, x, TOL) for H, b, x in zip(hs, bs, xs)]
    seq_s = time.perf_counter() - t0
    for H in hs:
        H.close()
    p_s = sorted(packed)[1]
    nnz = sum(g.nnz for g in graphs)
    its = sorted(i.iterations for i in infos)
    return {
        "graphs": count, "solves_per_s": count / p_s, "nnz_per_s": nnz / p_s, "wall_ms": p_s * 1e3,
        "launch_ms": infos[0].solve_ms,
        "sequential_solves_per_s": count / seq_s, "speedup_vs_sequential": seq_s / p_s,
        "iterations_median": its[len(its) // 2], "iterations_max": its[-1],
        "iterations_equal_to_lg_solve": sum(a.iterations == b.iterations for a, b in zip(infos, single)),
        "max_relres": max(i.relres for i in infos), "failed": sum(i.status != lg.OK for i in infos),
        "vertices": int(sum(g.n for g in graphs)), "nnz": int(nnz),
        "config": f"{count} graphs, n log-uniform in [500, 5000], type uniform over 2D grid / 3D grid / "
                  f"Chung-Lu 2.1 / R-MAT ef16; one right-hand side each; tol 1e-8; FP32 hierarchy; host b and "
                  f"x; wall time of the call (median of 3) against one lg_solve per graph",
    }


def run_reference(args, world, rank):
    """The oracle as it stands on the host cores, on a bounded sample of the
    workload (each step one FP64 PCG solve to 1e-8, the oracle's setup
    untimed); under torchrun only rank 0 runs it."""
    if rank != 0:
        return
    import oracle
    from paper_1705_06266_gb300 import inputs

    oracle.build()
    if args.workload == "rmat_26":
        g = rmat_sample()
        note = (f"R-MAT scale {SAMPLE_SCALE} of the scale-26 recipe (edge factor 16, a=.57 b=.19 c=.19, "
                f"symmetrised, deduplicated, unit weights, largest component; torch on the host) as the "
                f"bounded sample: ")
    else:
        g = inputs.workload(args.workload)
        note = ""
    b = inputs.rhs(g.n, seed=2)
    h = oracle.Hierarchy(g)
    times = []
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        x, st, it, rel = h.pcg(b, tol=TOL)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
    mean = sum(times) / len(times)
    value = g.nnz / mean
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "rhs": 1, "tol": TOL, "precision": "fp64",
                   "parallelism": "replicas"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{note}{g.name} (n={g.n}, nnz(L)={g.nnz}); each step one FP64 PCG solve "
                                   f"to 1e-8 ({it} iterations) on one host core, oracle setup untimed"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def load_main(args, inputs, torch, dev):
    """The main workload on the device: (description, n, nnz, rowptr, col, w,
    host b, host graph or None). R-MAT scale 26 is generated on the device
    (host generation of 2^30 sampled edges would not fit the bench's time)."""
    if args.workload == "rmat_26":
        t0 = time.perf_counter()
        n, rp, cl, w = inputs.rmat_device(26, seed=1, device=str(dev))
        torch.cuda.synchronize()
        gen_s = time.perf_counter() - t0
        desc = {"graph": "rmat_26_16", "generate_s": gen_s,
                "recipe": "R-MAT scale 26, edge factor 16 (2^30 sampled edges), a=.57 b=.19 c=.19 d=.05, "
                          "symmetrised, deduplicated, self-loops dropped, unit weights, largest component "
                          "kept; generated on the device (seed 1)"}
        g = None
    else:
        g = workload(inputs, args.workload)
        n = g.n
        rp, cl, w = (torch.from_numpy(a).to(dev) for a in (g.rowptr, g.col, g.w))
        desc = {"graph": g.name}
    nnz = int(cl.numel()) + n
    return desc, n, nnz, rp, cl, w, inputs.rhs(n, seed=2), g


def main():
    t_main = time.perf_counter()
    args = parse()
    world, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch

    from paper_1705_06266_gb300 import _build, inputs, lg

    _build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    desc, n, nnz, rp, cl, w, b, g_host = load_main(args, inputs, torch, dev)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        bd = torch.from_numpy(b).to(dev)
        x64 = torch.zeros(n, dtype=torch.float64, device=dev)
        x32 = torch.zeros(n, dtype=torch.float64, device=dev)
        opts = lg.options(stream=stream.cuda_stream)

        def per_level(h, nlev):
            """Per level: the Laplacian passes, then the W = L P passes (profile slots nlev + l)."""
            out = []
            for l in range(2 * nlev):
                p = lg.lg_profile_read(h, l)
                out.append((p.total_ms, p.bytes, p.launches))
            return out

        def step(profile):
            flush.fill_(1.0)
            h = lg.lg_setup(n, rp, cl, w, opts)
            hi = lg.lg_hier_info(h)
            res = {}
            for tag, prec, x in (("fp64", lg.FP64, x64), ("fp32", lg.FP32_HIER, x32)):
                lg.lg_set_precision(h, prec)
                flush.fill_(2.0)
                res[tag] = lg.lg_solve(h, bd, x, TOL)  # graph-driven, unprofiled: the timed solve
                if profile and tag == "fp64":  # the same solve again with every operator pass bracketed by events
                    lg.lg_profile(h, True)
                    flush.fill_(3.0)
                    lg.lg_solve(h, bd, x, TOL)
                    res[tag + "_prof"] = per_level(h, hi.levels)
                    lg.lg_profile(h, False)
            nb = lg.lg_hier_bytes(h)
            lv = [dict(lg.lg_level_info(h, l), **lg.lg_level_plan(h, l)) for l in range(hi.levels)]
            lg.lg_destroy(h)
            return hi, res["fp64"], res["fp32"], res.get("fp64_prof"), nb, lv

        for _ in range(args.warmup):
            step(False)
        stream.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        clocks = Clocks(local)
        launches0 = lg.lg_kernel_launches()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        t0 = time.perf_counter()
        recs = [step(True) for _ in range(args.steps)]
        ev1.record(stream)
        stream.synchronize()
        wall = time.perf_counter() - t0
        torch.cuda.synchronize()
        barrier(world)
        clk = clocks.stop()
        launches = lg.lg_kernel_launches() - launches0
        step_ms = ev0.elapsed_time(ev1) / args.steps

        # After the timed region, on one more (bitwise identical) hierarchy:
        # its setup's stage times (from the library's setup log), the FP32
        # per-level pass table, each result's error against an FP64 solve to
        # 1e-12, and the end-to-end solves from host buffers.
        log_path = os.path.join(tempfile.gettempdir(), f"lg_setup_{os.getpid()}.jsonl")
        os.environ["LG_LOG"] = log_path
        try:
            h = lg.lg_setup(n, rp, cl, w, opts)
        finally:
            del os.environ["LG_LOG"]
        setup_stages = None
        try:
            with open(log_path) as f:
                setup_stages = json.loads(f.readlines()[-1]).get("stages_ms")
            os.remove(log_path)
        except (OSError, ValueError, IndexError):
            pass
        nlev = lg.lg_hier_info(h).levels
        lg.lg_set_precision(h, lg.FP32_HIER)
        lg.lg_profile(h, True)
        flush.fill_(3.0)
        lg.lg_solve(h, bd, x32, TOL)
        prof32 = per_level(h, nlev)
        lg.lg_profile(h, False)
        lg.lg_solve(h, bd, x32, TOL)
        x32_full = x32.clone()  # compared with the FP32-only hierarchy's solve below
        lg.lg_set_precision(h, lg.FP64)
        lg.lg_solve(h, bd, x64, TOL)
        xref = torch.zeros_like(x64)
        ref_info = lg.lg_solve(h, bd, xref, 1e-12, check=False)
        errs = {"fp64": rel_err(x64.cpu().numpy(), xref.cpu().numpy()),
                "fp32": rel_err(x32.cpu().numpy(), xref.cpu().numpy())}
        del xref

        # end to end through the C ABI with host buffers (pinned), per step:
        # H2D of b, the solve, D2H of x, all inside the timed call
        bh = torch.from_numpy(b).pin_memory()
        xh = torch.zeros(n, dtype=torch.float64).pin_memory()
        bnp, xnp = bh.numpy(), xh.numpy()
        e2e = {}
        for tag, prec in (("fp64", lg.FP64), ("fp32", lg.FP32_HIER)):
            lg.lg_set_precision(h, prec)
            lg.lg_solve(h, bnp, xnp, TOL)
            ts = []
            for _ in range(args.e2e_steps):
                t1 = time.perf_counter()
                lg.lg_solve(h, bnp, xnp, TOL)
                ts.append(time.perf_counter() - t1)
            e2e[tag] = sum(ts) / len(ts)
        lg.lg_destroy(h)
        del bh, xh
        setup_e2e = None
        if g_host is not None:
            t1 = time.perf_counter()
            h2 = lg.lg_setup(g_host.n, g_host.rowptr, g_host.col, g_host.w, lg.options())
            setup_e2e = time.perf_counter() - t1
            lg.lg_destroy(h2)

        # the same solves with post-smoothing from f - L x instead of the W = L P pass
        h0 = lg.lg_setup(n, rp, cl, w, lg.options(stream=stream.cuda_stream, lp_residual=0))
        direct = {}
        for tag, prec, x in (("fp64", lg.FP64, x64), ("fp32", lg.FP32_HIER, x32)):
            lg.lg_set_precision(h0, prec)
            ms = []
            for _ in range(3):
                flush.fill_(2.0)
                ms.append(lg.lg_solve(h0, bd, x, TOL).solve_ms)
            direct[tag] = sorted(ms)[1]
        lg.lg_destroy(h0)
        # the FP32-only hierarchy (option fp32_only): its footprint and its FP32-hierarchy solve, which must give the
        # bits of the full hierarchy's
        hl = lg.lg_setup(n, rp, cl, w, lg.options(stream=stream.cuda_stream, precision=lg.FP32_HIER, fp32_only=1))
        xl = torch.zeros_like(x32)
        flush.fill_(2.0)
        lg.lg_solve(hl, bd, xl, TOL)
        flush.fill_(2.0)
        inf_l = lg.lg_solve(hl, bd, xl, TOL)
        lean = {"hierarchy_bytes": lg.lg_hier_bytes(hl)[0], "workspace_bytes": lg.lg_hier_bytes(hl)[1],
                "fp32_solve_ms": inf_l.solve_ms, "iterations": inf_l.iterations,
                "same_bits_as_full": bool(torch.equal(xl, x32_full))}
        lg.lg_destroy(hl)
        del xl, x32_full
        stream.synchronize()
    del rp, cl, w, bd, x64, x32
    torch.cuda.synchronize()
    torch.cuda.empty_cache()

    # the other configurations the metric names, after the timed region
    oracle_ref = world == 1 and not args.no_cpu_baseline
    second = {}
    if not args.no_secondary:
        for name in ("chung_lu_1m", "grid2d_64"):
            if name != args.workload:
                second[name] = secondary_leg(lg, inputs, torch, dev, name, flush, oracle_ref)
    multi = None if args.no_multi_rhs else multi_rhs_leg(lg, inputs, torch, dev, args.multi_rhs_k)
    kcyc = None if args.no_kcycle else kcycle_leg(lg, inputs, torch, dev)
    wda = None if args.no_wda else wda_leg(lg, inputs, torch, dev)
    order = None
    if not args.no_ordering:
        graphs = []
        for name in ("chung_lu_1m", "rmat_20"):
            gg = workload(inputs, name)
            graphs.append((name, gg, inputs.rhs(gg.n, seed=2)))
        order = ordering_leg(lg, torch, dev, graphs)
    serve = None if args.no_serve else serve_leg(lg, inputs, args, torch, dev)
    many = None if args.no_many else many_leg(lg, inputs, args.many_graphs)
    del flush

    setup_ms = sum(r[0].setup_ms for r in recs) / len(recs)
    solve64_ms = sum(r[1].solve_ms for r in recs) / len(recs)
    solve32_ms = sum(r[2].solve_ms for r in recs) / len(recs)
    mx = allreduce_max([step_ms, setup_ms, solve64_ms, solve32_ms, e2e["fp64"], e2e["fp32"]], world)
    step_ms, setup_ms, solve64_ms, solve32_ms, e2e64_s, e2e32_s = mx
    value = world * nnz / (solve64_ms * 1e-3)

    # roofline of the dominant kernel: the operator row pass of the level with the most device time
    nlev = len(recs[0][3]) // 2
    tot = [[0.0, 0.0, 0] for _ in range(nlev)]
    for r in recs:
        for l, (ms, by, la) in enumerate(r[3][:nlev]):
            tot[l][0] += ms
            tot[l][1] += by
            tot[l][2] += la
    dom = max(range(nlev), key=lambda l: tot[l][0])
    d_ms, d_bytes, d_launch = tot[dom]
    peak, peak_kind = measured_peak()
    achieved = d_bytes / (d_ms * 1e-3) / 1e9 if d_ms > 0 else 0.0
    traffic, _ = ncu_traffic(args.workload)
    wpass = [[sum(r[3][nlev + l][q] for r in recs) for q in range(3)] for l in range(nlev)]
    all_ms = sum(t[0] for t in tot) + sum(t[0] for t in wpass)
    all_bytes = sum(t[1] for t in tot) + sum(t[1] for t in wpass)
    i64, i32 = recs[-1][1], recs[-1][2]
    # per-level operator-pass table, both precisions (ms per solve, GB/s)
    levels = []
    for l in range(nlev):
        row = dict(recs[-1][5][l])
        ms = sum(r[3][l][0] for r in recs) / len(recs)
        by = sum(r[3][l][1] for r in recs) / len(recs)
        la = sum(r[3][l][2] for r in recs) / len(recs)
        row["fp64_ms_per_solve"] = ms
        row["fp64_launches_per_solve"] = la
        row["fp64_gbs"] = by / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
        wms = sum(r[3][nlev + l][0] for r in recs) / len(recs)
        wby = sum(r[3][nlev + l][1] for r in recs) / len(recs)
        if wms > 0:
            row["fp64_w_pass_ms_per_solve"] = wms
            row["fp64_w_pass_gbs"] = wby / (wms * 1e-3) / 1e9
        ms, by, la = prof32[l]
        row["fp32_ms_per_solve"] = ms
        row["fp32_launches_per_solve"] = la
        row["fp32_gbs"] = by / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
        wms, wby, _ = prof32[nlev + l]
        if wms > 0:
            row["fp32_w_pass_ms_per_solve"] = wms
            row["fp32_w_pass_gbs"] = wby / (wms * 1e-3) / 1e9
        levels.append(row)

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict({"workload": args.workload, "n": n, "nnz": nnz, "rhs": 1, "tol": TOL,
                        "precision": "fp64 (FP32-hierarchy solve reported in fp32_hier)",
                        "step": "setup; FP64 solve; FP64 solve with per-pass events; FP32-hier solve "
                                "(value and fp32_hier from the solves without events)",
                        "l2": "flushed (512 MiB write) before setup and before each solve",
                        "parallelism": "replicas" if world > 1 else "single GPU"}, **desc),
        "solve_ms": solve64_ms, "setup_ms": setup_ms, "setup_stages_ms": setup_stages,
        "iterations": i64.iterations, "relres": i64.relres, "levels": i64.levels,
        "op_complexity": recs[-1][0].op_complexity,
        "setup_inclusive_nnz_per_s": world * nnz / ((setup_ms + solve64_ms) * 1e-3),
        "lp_residual": {"fp64_solve_ms": solve64_ms, "fp64_solve_ms_without": direct["fp64"],
                        "fp32_solve_ms": solve32_ms, "fp32_solve_ms_without": direct["fp32"],
                        "note": "post-smoothing started by one pass over W = L P (default) against a pass "
                                "over L from f - L x (lp_residual = 0, median of 3 solves)"},
        "fp32_hier": {"value": world * nnz / (solve32_ms * 1e-3), "solve_ms": solve32_ms,
                      "iterations": i32.iterations, "relres": i32.relres,
                      "speedup_vs_fp64": solve64_ms / solve32_ms, "x_err": errs["fp32"]},
        "x_err": {"fp64": errs["fp64"], "fp32": errs["fp32"],
                  "reference": f"FP64 solve of the same hierarchy to 1e-12 ({ref_info.iterations} iterations, "
                               f"relres {ref_info.relres:.1e}); relative 2-norm error of the mean-removed x"},
        "tda_ms_per_digit": solve64_ms / -math.log10(max(i64.relres, 1e-300)),
        "wda": i64.work_units / -math.log10(max(i64.relres, 1e-300)),
        "hierarchy_bytes": recs[-1][4][0], "workspace_bytes": recs[-1][4][1], "fp32_only": lean,
        "e2e": {"value": world * nnz / e2e64_s, "unit": UNIT, "h2d_bytes_per_step": 8 * n,
                "d2h_bytes_per_step": 8 * n, "fp32_hier_value": world * nnz / e2e32_s,
                "setup_from_host_ms": None if setup_e2e is None else setup_e2e * 1e3,
                "note": "lg_solve with pinned host b and x: H2D of b, solve, D2H of x inside the timed call"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                     "whole_solve_frac": (all_bytes / len(recs)) / (solve64_ms * 1e-3) / 1e9 / peak,
                     "whole_solve_note": "algorithmic bytes of every operator pass of one FP64 solve (per-pass "
                                         "events) over the event-free FP64 solve time; vector kernels not counted",
                     "kernel": f"k_rows<double, LapTerm, *> operator passes of level {dom} "
                               f"({tot[dom][2] // len(recs)} per solve) in the timed FP64 solves",
                     "launches": d_launch, "avg_launch_us": d_ms * 1e3 / max(d_launch, 1),
                     "bytes_per_launch": d_bytes / max(d_launch, 1), "peak_kind": peak_kind,
                     "share_of_solve": d_ms / (solve64_ms * len(recs)),
                     "all_levels_achieved": all_bytes / (all_ms * 1e-3) / 1e9 if all_ms > 0 else 0.0},
        "levels": levels,
        "clocks": clk,
        "gpu_launches": launches,
        "wall_s_timed": wall,
    }
    for key, val in (("secondary", second), ("multi_rhs", multi), ("kcycle", kcyc), ("wda", wda),
                     ("ordering", order), ("serve", serve), ("many_small", many)):
        if val:
            line[key] = val
    if world == 1 and not args.no_cpu_baseline:
        if args.workload == "rmat_26":
            gs = rmat_sample()
            line["cpu_baseline"] = cpu_baseline(
                args.workload, gs, inputs.rhs(gs.n, seed=2),
                note=f"R-MAT scale {SAMPLE_SCALE} of the scale-26 recipe (torch on the host) as the bounded "
                     f"sample: ")
        else:
            line["cpu_baseline"] = cpu_baseline(args.workload, g_host, b)
    line["bench_wall_s"] = time.perf_counter() - t_main
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
