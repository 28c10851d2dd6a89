"""Sweep of the Sinkhorn row configurations; writes the tuning table.

    python -m paper_2404_08970_gb300.tune [--out PATH] [--n ROWS] [--reps R]

Each built-in row-length range of each dtype is split into two halves.  For
the longest rows of a half, a synthetic 1D problem (n rows, uniform marginals,
k = 1, eps = 1e-2, one mirror-descent step of 20 Sinkhorn iterations) is
solved with every candidate configuration (gw_tune_candidates).  A candidate
is kept only if the solve reports no device error and its plan matches the
built-in configuration's plan (relative max difference at most 1e-4 for
float, 1e-10 for double: the configurations differ only in the order of the
row reductions).  The fastest kept candidate (CUDA events on the solve's
stream, best of R graph-launched solves) becomes the half's entry.  The table
goes to tune_table.txt beside the library unless --out says otherwise; the
library loads it at the first context creation of a process.
"""
from __future__ import annotations

import argparse
import datetime
import os

from . import _lib as L

# Built-in row-length ranges (the boundaries of the built-in choice).
RANGES = {
    L.GW_F32: [(1, 384), (385, 512), (513, 768), (769, 1024), (1025, 1536), (1537, 2048), (2049, 3072),
               (3073, 4096), (4097, 6144), (6145, 8192), (8193, 12288), (12289, 16384)],
    L.GW_F64: [(1, 256), (257, 1024), (1025, 4096), (4097, 10240)],
}
TOL = {L.GW_F32: 1e-4, L.GW_F64: 1e-10}
# Rows of the synthetic problems: a single solve then spreads bands of about 54
# rows over the GPU's SMs, close to the bands of large single solves and of
# batched problems (at least 512 KB each).  With 2048 rows (14-row bands) the
# per-band start-up decides, and configurations that stream fewer rows at once
# win there but lose in batched passes.
ROWS = 8192


def halves(lo: int, hi: int):
    if hi - lo < 64:
        return [(lo, hi)]
    mid = (lo + hi) // 2
    return [(lo, mid), (mid + 1, hi)]


def sweep(n: int = ROWS, reps: int = 3, log=print):
    import numpy as np
    import torch

    ctx = L.Context(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    entries, notes = [], []
    for dtype, ranges in RANGES.items():
        tdt = torch.float32 if dtype == L.GW_F32 else torch.float64
        for lo, hi in ranges:
            for a, b in halves(lo, hi):
                m = b
                u = torch.full((n,), 1.0 / n, dtype=torch.float64, device=dev)
                v = torch.full((m,), 1.0 / m, dtype=torch.float64, device=dev)
                prob = L.problem(dim=1, nx=n, ny=m, hx=1.0 / n, hy=1.0 / m, k=1, eps=1e-2, n_outer=1, n_inner=20,
                                 dtype=dtype)
                plans, times = {}, {}
                for cfg in L.gw_tune_candidates(L.GW_TUNE_SINKHORN, dtype, m):
                    L.gw_tune_clear()
                    L.gw_tune_set(L.GW_TUNE_SINKHORN, dtype, a, b, cfg)
                    T = torch.empty((n, m), dtype=tdt, device=dev)
                    try:
                        ctx.gw_solve(prob, u, v, T, stream=stream)  # captures the graph
                        ctx.gw_ctx_check(stream)
                        best = float("inf")
                        for _ in range(reps):
                            e0 = torch.cuda.Event(enable_timing=True)
                            e1 = torch.cuda.Event(enable_timing=True)
                            e0.record(stream)
                            ctx.gw_solve(prob, u, v, T, stream=stream)
                            e1.record(stream)
                            e1.synchronize()
                            best = min(best, e0.elapsed_time(e1))
                        ctx.gw_ctx_check(stream)
                    except L.GWError as ex:
                        notes.append(f"dtype {dtype} m {m} config {cfg}: {ex}")
                        continue
                    plans[cfg] = T.double().cpu().numpy()
                    times[cfg] = best
                L.gw_tune_clear()
                base = L.gw_tune_config(L.GW_TUNE_SINKHORN, dtype, m)
                if base not in plans:
                    notes.append(f"dtype {dtype} m {m}: the built-in configuration {base} failed; range skipped")
                    continue
                ref = plans[base]
                scale = float(np.max(np.abs(ref)))
                kept = {}
                for cfg, P in plans.items():
                    err = float(np.max(np.abs(P - ref))) / scale
                    if err <= TOL[dtype]:
                        kept[cfg] = times[cfg]
                    else:
                        notes.append(f"dtype {dtype} m {m} config {cfg}: plan differs by {err:.2e}; dropped")
                win = min(kept, key=kept.get)
                entries.append((dtype, a, b, win, {c: round(t, 4) for c, t in times.items()}))
                log(f"dtype {dtype} rows {a}..{b}: {win} (ms {entries[-1][4]})")
    ctx.close()
    return entries, notes


def write_table(path: str, entries, notes, n: int, reps: int, device_name: str) -> None:
    """Writes the table in the format gw_tune_load reads."""
    name = device_name
    when = datetime.datetime.now(datetime.timezone.utc).strftime("%Y-%m-%dT%H:%M:%SZ")
    lines = [f"# Sinkhorn row configurations tuned on {name}, {when}",
             f"# n = {n} rows, best of {reps} solves of one mirror-descent step x 20 iterations",
             "# kernel dtype m_lo m_hi config   (ms per candidate)"]
    for dtype, a, b, win, ms in entries:
        lines.append(f"{L.GW_TUNE_SINKHORN} {dtype} {a} {b} {win}   # {ms}")
    lines += [f"# {t}" for t in notes]
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(os.path.dirname(L.LIB_PATH), "tune_table.txt"))
    ap.add_argument("--n", type=int, default=ROWS)
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args()
    import torch
    entries, notes = sweep(args.n, args.reps)
    write_table(args.out, entries, notes, args.n, args.reps, torch.cuda.get_device_name(0))
    print(f"wrote {args.out}: {len(entries)} entries, {len(notes)} notes")
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
