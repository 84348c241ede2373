"""Per-level operator pass timing: builds the hierarchy of one graph and
times y = L_l x on each chosen level with CUDA events (L2 flushed before each
pass), in FP64 and in FP32, through lg_level_apply (the cycle's own row plans
and kernels). Prints one JSON line per level with the pass time and the
algorithmic bytes it moves as GB/s.

    python -m paper_1705_06266_gb300.passes --rmat 26 --levels 0,1,3
    python -m paper_1705_06266_gb300.passes --workload chung_lu_1m
    python -m paper_1705_06266_gb300.passes --complete 4500 --levels 0 --reps 1
    python -m paper_1705_06266_gb300.passes --workload rmat_20 --levels none --batch 32

Algorithmic bytes of a pass: the column ids (4 per entry), the weights (8 or
4 per entry, none for a constant-weight finest operator), the row pointers
(8 per row), x once and y once (and the FP64 row sums)."""

from __future__ import annotations

import argparse
import json
import time


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    src = ap.add_mutually_exclusive_group()
    src.add_argument("--rmat", type=int, help="R-MAT scale (device generator, edge factor 16, unit weights)")
    src.add_argument("--workload", help="a named workload of the inputs module (host generator)")
    src.add_argument("--complete", type=int, help="complete graph on this many vertices, uniform weights")
    ap.add_argument("--levels", default="", help="comma-separated levels (default: every non-coarsest level)")
    ap.add_argument("--reps", type=int, default=5, help="timed passes per level and precision (median kept)")
    ap.add_argument("--prec", choices=["both", "fp64", "fp32"], default="both")
    ap.add_argument("--batch", type=int, default=0,
                    help="also time one multi-column V-cycle (lg_vcycle_batch) on this many columns")
    ap.add_argument("--opt", action="append", default=[], metavar="NAME=VALUE",
                    help="an lg_options field for the setup (repeatable), e.g. --opt row_sorts=0")
    ap.add_argument("--setups", type=int, default=1, help="setups to run (the last one is kept; the median "
                    "setup time is printed)")
    ap.add_argument("--lib", default=None, help="path of the library to load (default: build the package's)")
    a = ap.parse_args(argv)

    import torch

    from . import _build, inputs, lg

    if a.lib:
        lg.LIB_PATH = a.lib
    else:
        _build.build()
    dev = torch.device("cuda", 0)
    t0 = time.time()
    if a.workload or a.complete:
        g = inputs.workload(a.workload) if a.workload else inputs.complete(a.complete, weights="uniform", seed=5)
        n = g.n
        rp, cl, w = (torch.from_numpy(v).to(dev) for v in (g.rowptr, g.col, g.w))
    else:
        n, rp, cl, w = inputs.rmat_device(a.rmat if a.rmat else 20, seed=1, device="cuda")
    torch.cuda.synchronize()
    print(json.dumps({"generate_s": time.time() - t0, "n": n, "nnz": int(cl.numel()) + n}), flush=True)
    st = torch.cuda.Stream(device=dev)
    extra = {}
    for kv in a.opt:
        k, v = kv.split("=", 1)
        extra[k] = float(v) if "." in v else int(v)
    times = []
    h = None
    for _ in range(max(1, a.setups)):
        if h is not None:
            lg.lg_destroy(h)
        h = lg.lg_setup(n, rp, cl, w, lg.options(stream=st.cuda_stream, **extra))
        times.append(lg.lg_hier_info(h).setup_ms)
    del rp, cl, w
    hi = lg.lg_hier_info(h)
    print(json.dumps({"setup_ms": sorted(times)[len(times) // 2], "setup_ms_all": times, "levels": hi.levels,
                      "options": extra}), flush=True)
    flush = torch.empty(2 * 129 * 2**20 // 4, dtype=torch.float32, device=dev)
    if a.levels == "none":
        want = []
    else:
        want = [int(v) for v in a.levels.split(",")] if a.levels else list(range(hi.levels - 1))
    for lv in want:
        if lv < 0 or lv >= hi.levels - 1:
            continue
        d = dict(lg.lg_level_info(h, lv), **lg.lg_level_plan(h, lv))
        nl, nnzl = d["n"], d["nnz"]
        row = {"level": lv, "kind": d["kind"], "n": nl, "nnz": nnzl, "E": d.get("E"),
               "seg_tiles": d.get("seg_tiles"), "const_weights": bool(d.get("const_weights", 0))}
        for tag, prec, dt, wb in (("fp64", lg.FP64, torch.float64, 8), ("fp32", lg.FP32_HIER, torch.float32, 4)):
            if a.prec not in ("both", tag):
                continue
            x = torch.randn(nl, dtype=dt, device=dev)
            y = torch.empty(nl, dtype=dt, device=dev)
            lg.lg_level_apply(h, lv, prec, x, y)
            ts = []
            for _ in range(a.reps):
                flush.fill_(1.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(st)
                lg.lg_level_apply(h, lv, prec, x, y)
                e1.record(st)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            ms = sorted(ts)[len(ts) // 2]
            wbytes = 0 if row["const_weights"] else wb
            by = nnzl * (4 + wbytes) + (nl + 1) * 8 + nl * wb * 2 + (nl * 8 if wb == 8 else 0)
            row[tag + "_ms"] = ms
            row[tag + "_gbs"] = by / (ms * 1e-3) / 1e9
        print(json.dumps(row), flush=True)
    if a.batch > 0:
        k = a.batch
        row = {"batch": k, "n": n}
        F = torch.randn(k, n, dtype=torch.float64, device=dev)
        F -= F.mean(dim=1, keepdim=True)
        X = torch.empty_like(F)
        for tag, prec in (("fp64", lg.FP64), ("fp32", lg.FP32_HIER)):
            if a.prec not in ("both", tag):
                continue
            lg.lg_vcycle_batch(h, k, F, n, X, n, prec)
            ts = []
            for _ in range(a.reps):
                flush.fill_(1.0)
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                lg.lg_vcycle_batch(h, k, F, n, X, n, prec)
                ts.append(time.perf_counter() - t1)
            row[tag + "_cycle_ms"] = sorted(ts)[len(ts) // 2] * 1e3
        print(json.dumps(row), flush=True)
    lg.lg_destroy(h)


if __name__ == "__main__":
    main()
