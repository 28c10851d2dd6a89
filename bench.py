"""Benchmark of the structured GW gradient on GB300.

Default workload: 1D uniform grids n = m = 8192, k = 1, uniform marginals, a
random positive coupling T with those marginals (float32 on the device),
spacing h = 1/n.  One step = one gradient evaluation G = L(C_X,C_Y) (x) T
through the C ABI (gw_grad, target marginals).  T and G are 268 MB each,
larger than the 129 MB L2, so no L2 flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  Under torchrun every rank runs the same workload on
its own GPU (independent replicas, weak scaling); rank 0 prints.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "GW grad evals/s fast vs dense (%roofline); served solves/s + p50/p99"
UNIT = "grad evals/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--m", type=int, default=0, help="columns of the gradient workload (default: n)")
    ap.add_argument("--k", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solve", dest="solve", action="store_false")
    ap.add_argument("--no-2d", dest="grid2d", action="store_false")
    ap.add_argument("--no-3d", dest="grid3d", action="store_false")
    ap.add_argument("--no-variants", dest="variants", action="store_false")
    ap.add_argument("--no-batch", dest="batch", action="store_false")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--no-serve", dest="serve", action="store_false")
    ap.add_argument("--serve-count", type=int, default=1500)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--oracle-sample", type=int, default=0, help=argparse.SUPPRESS)
    return ap.parse_args()


def max_over_ranks(x: float, device=None) -> float:
    """Largest value of x over the ranks of the process group (x itself
    without one).  Every rank calls it."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, units_per_rank: int, ms_max: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (replicas do equal work, weak scaling)."""
    return world * units_per_rank / (ms_max / 1e3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(n, k, m=None):
    """The gradient workload: n x m grids (m = n unless given), uniform
    marginals, the random positive coupling, h = 1/n and 1/m."""
    from paper_2404_08970_gb300 import inputs as I
    if m is None or m == n:
        return I.workload_1d_grad(n, k, "uniform", seed=0)
    import numpy as np
    rng = np.random.default_rng(0)
    u, v = I.uniform_weights(n), I.uniform_weights(m)
    return dict(T=I.random_coupling(u, v, rng), u=u, v=v, hx=1.0 / n, hy=1.0 / m, k=k)


L2_BYTES = 126 * 2 ** 20


def config(n, k, extra=None, m=None):
    m = n if m is None else m
    mb = 4 * n * m / 1e6
    l2 = (f"inputs larger than L2 ({mb:.0f} MB T, {mb:.0f} MB G)" if 4 * n * m > L2_BYTES else
          f"inputs fit in L2 ({mb:.1f} MB T, {mb:.1f} MB G): not a valid bench size, for profiling only")
    shape = f"n=m={n}" if m == n else f"n={n}, m={m}"
    c = {"workload": f"1D uniform grids {shape}, k={k}, uniform marginals, random positive coupling, h=1/n; "
                     f"one structured gradient evaluation per step",
         "n": n, "m": m, "k": k, "marginals": "target (uniform)", "l2": l2,
         "global_batch": 1, "parallelism": "replicas"}
    if extra:
        c.update(extra)
    return c


# ---------------------------------------------------------------------------
# CPU oracle timing (baseline leg and the reference arm)
# ---------------------------------------------------------------------------

def oracle_rows_time(T64, u, v, k, h, rows):
    """Times the FP64 oracle's gradient rows (definition: c_x + c_y - 2 D_X T D_Y)."""
    import numpy as np
    from oracle import gw_oracle as O
    n, m = T64.shape
    idx = np.arange(n, dtype=np.float64)
    t0 = time.perf_counter()
    sel = np.arange(rows)
    DXr = (h ** k) * np.abs(idx[sel][:, None] - idx[None, :]) ** k
    DY = O.grid_dist_1d(m, h, k)
    cy = (DY * DY) @ v
    O.grad_rows(DXr, DY, T64, (DXr * DXr) @ u, cy)
    return time.perf_counter() - t0


def oracle_rows(T64, u, v, k, hx, hy, rows):
    """Rows `rows` of the FP64 oracle gradient with target marginals."""
    import numpy as np
    from oracle import gw_oracle as O
    n, m = T64.shape
    idx = np.arange(n, dtype=np.float64)
    sel = np.asarray(rows)
    DXr = (hx ** k) * np.abs(idx[sel][:, None] - idx[None, :]) ** k
    DY = O.grid_dist_1d(m, hy, k)
    return O.grad_rows(DXr, DY, T64, (DXr * DXr) @ u, (DY * DY) @ v)


def cpu_oracle_rate(w, budget_s=15.0):
    """Gradient evals/s of the oracle on the host, from a timed sample of rows
    (the full dense gradient at n = 8192 takes minutes in FP64)."""
    import numpy as np
    T64 = w["T"]
    n = T64.shape[0]
    rows = 16
    t = oracle_rows_time(T64, w["u"], w["v"], w["k"], w["hx"], rows)
    # Grow the sample until it costs about budget_s/2.
    while t < budget_s / 4 and rows < n:
        rows = min(n, rows * 4)
        t = oracle_rows_time(T64, w["u"], w["v"], w["k"], w["hx"], rows)
    rate = (rows / n) / t
    return rate, rows, t


# ---------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------

class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        import tempfile
        fd, self.path = tempfile.mkstemp(prefix="gw_clocks_", suffix=".csv")
        os.close(fd)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "50", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.5)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        if not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        try:
            os.remove(self.path)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def kernel_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu record, or
    None if the kernel source changed since the record was taken."""
    import hashlib
    rec = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(rec):
        return None
    d = json.load(open(rec))
    e = d.get(kernel)
    if not e:
        return None
    h = hashlib.sha1()
    for f in e["sources"]:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return e["dram_bytes"] if h.hexdigest() == e["sha1"] else None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs"), d.get("bf16_tflops"), "measured"
    return 6800.0, 1900.0, "fallback"


def bench_2d(ctx, L, dev, stream, barrier, steps, with_solve):
    """2D grids 64 x 64 against 96 x 96 (n = 4096, m = 9216), squared
    Euclidean cost on the unit square, |N(0,1)| image marginals: structured
    gradient vs the dense BF16 path, and the solve at eps = 5e-3, 20 x 100."""
    import numpy as np
    import torch
    from paper_2404_08970_gb300 import inputs as I
    w = I.workload_2d(64, 96, "sqeuclid", seed=0)
    rng = I.rng_for(1)
    T = I.random_coupling(w["u"], w["v"], rng).astype(np.float32)
    n, m = T.shape
    dT = torch.from_numpy(T).to(dev)
    dG = torch.empty_like(dT)
    du = torch.from_numpy(w["u"]).to(dev)
    dv = torch.from_numpy(w["v"]).to(dev)
    prob = L.problem(dim=2, nx=64, ny=96, hx=w["hx"], hy=w["hy"], k=1, cost=L.GW_COST_SQEUCLID, dtype=L.GW_F32)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        for _ in range(3):
            fn()
        barrier()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        barrier()
        return e0.elapsed_time(e1) / reps

    grad = lambda: ctx.gw_grad(prob, du, dv, dT, dG, L.GW_MARG_TARGET, stream)
    gms = timed(grad, steps)
    ctx.gw_ctx_profile(True)
    ctx.gw_ctx_profile_report(reset=True)
    for _ in range(steps):
        grad()
    barrier()
    prof = ctx.gw_ctx_profile_report(reset=True)
    ctx.gw_ctx_profile(False)
    ctx.gw_ctx_check(stream)
    hbm_peak, _, peak_kind = measured_peaks()
    roof = {}
    for kname in ("g2_rows", "g2_epi"):
        if kname in prof:
            avg = prof[kname]["ms"] / max(1, prof[kname]["launches"])
            gbs = 4.0 * n * m / (avg / 1e3) / 1e9  # g2_rows reads T, g2_epi writes G: 4 B per element each
            roof[kname] = {"avg_launch_ms": avg, "achieved_gbs": gbs, "frac": gbs / hbm_peak,
                           "peak_kind": f"hbm_gbs of {peak_kind}"}
    dense = lambda: ctx.gw_grad_dense(prob, du, dv, dT, dG, L.GW_MARG_TARGET, L.GW_DENSE_BF16, stream)
    try:
        dms = timed(dense, 5)
    except Exception as ex:
        dms = None
        roof["dense_error"] = str(ex)[:200]
    # Manhattan distance squared (k = 2): the two-pass image-transform path.
    powk = {}
    try:
        probk = L.problem(dim=2, nx=64, ny=96, hx=w["hx"], hy=w["hy"], k=2, cost=L.GW_COST_POW, dtype=L.GW_F32)
        gradk = lambda: ctx.gw_grad(probk, du, dv, dT, dG, L.GW_MARG_TARGET, stream)
        kms = timed(gradk, steps)
        ctx.gw_ctx_profile(True)
        ctx.gw_ctx_profile_report(reset=True)
        for _ in range(steps):
            gradk()
        barrier()
        kprof = ctx.gw_ctx_profile_report(reset=True)
        ctx.gw_ctx_profile(False)
        ctx.gw_ctx_check(stream)
        kroof = {}
        for kname in ("g2k_rows", "g2k_cols"):
            if kname in kprof:
                avg = kprof[kname]["ms"] / max(1, kprof[kname]["launches"])
                gbs = 8.0 * n * m / (avg / 1e3) / 1e9  # each pass reads and writes n*m floats
                kroof[kname] = {"avg_launch_ms": avg, "achieved_gbs": gbs, "frac": gbs / hbm_peak,
                                "peak_kind": f"hbm_gbs of {peak_kind}"}
        powk = {"workload": "same grids and T, Manhattan distance squared (k=2), fp32",
                "grad_evals_per_s": 1e3 / kms, "grad_ms": kms,
                "whole_gradient_gbs_16B": 16.0 * n * m / (kms / 1e3) / 1e9,
                "kernels": kprof, "roofline": kroof}
    except Exception as ex:
        powk = {"error": str(ex)[:200]}
    out = {"workload": "2D grids 64x64 vs 96x96 (n=4096, m=9216), squared Euclidean, unit square, "
                       "|N(0,1)| image marginals, random positive coupling, fp32",
           "manhattan_k2": powk,
           "grad_evals_per_s": 1e3 / gms, "grad_ms": gms, "whole_gradient_gbs": 8.0 * n * m / (gms / 1e3) / 1e9,
           "kernels": prof, "roofline": roof,
           "dense_bf16_evals_per_s": (1e3 / dms) if dms else None,
           "structured_over_dense_bf16": (dms / gms) if dms else None}
    if with_solve:
        dTs = torch.empty_like(dT)
        stats = torch.zeros(8, dtype=torch.float64, device=dev)
        sprob = L.problem(dim=2, nx=64, ny=96, hx=w["hx"], hy=w["hy"], k=1, cost=L.GW_COST_SQEUCLID, eps=5e-3,
                          n_outer=20, n_inner=100, dtype=L.GW_F32)
        solve = lambda: ctx.gw_solve(sprob, du, dv, dTs, None, None, stats, stream=stream)
        solve()
        barrier()
        sms = timed(solve, 1)
        ctx.gw_ctx_check(stream)
        out["solve"] = {"schedule": "eps=5e-3, 20 x 100", "solves_per_s": 1e3 / sms, "ms": sms,
                        "gw_value": float(stats[1].item()), "col_marginal_err": float(stats[5].item())}
    return out


def bench_3d(ctx, L, dev, stream, barrier, steps, with_solve):
    """3D grids 16^3 against 21^3 (n = 4096, m = 9261), squared Euclidean cost
    on the unit cube, |N(0,1)| voxel marginals: structured gradient vs the
    dense BF16 path, and the solve at eps = 5e-3, 20 x 100."""
    import numpy as np
    import torch
    from paper_2404_08970_gb300 import inputs as I
    sx, sy = 16, 21
    w = I.workload_3d(sx, sy, "sqeuclid", seed=0)
    T = I.random_coupling(w["u"], w["v"], I.rng_for(1)).astype(np.float32)
    n, m = T.shape
    dT = torch.from_numpy(T).to(dev)
    dG = torch.empty_like(dT)
    du = torch.from_numpy(w["u"]).to(dev)
    dv = torch.from_numpy(w["v"]).to(dev)
    prob = L.problem(dim=3, nx=sx, ny=sy, hx=w["hx"], hy=w["hy"], k=1, cost=L.GW_COST_SQEUCLID, dtype=L.GW_F32)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        for _ in range(3):
            fn()
        barrier()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        barrier()
        return e0.elapsed_time(e1) / reps

    grad = lambda: ctx.gw_grad(prob, du, dv, dT, dG, L.GW_MARG_TARGET, stream)
    gms = timed(grad, steps)
    ctx.gw_ctx_profile(True)
    ctx.gw_ctx_profile_report(reset=True)
    for _ in range(steps):
        grad()
    barrier()
    prof = ctx.gw_ctx_profile_report(reset=True)
    ctx.gw_ctx_profile(False)
    ctx.gw_ctx_check(stream)
    hbm_peak, _, peak_kind = measured_peaks()
    roof = {}
    for kname in ("g3_rows", "g3_epi"):
        if kname in prof:
            avg = prof[kname]["ms"] / max(1, prof[kname]["launches"])
            gbs = 4.0 * n * m / (avg / 1e3) / 1e9  # g3_rows reads T, g3_epi writes G: 4 B per element each
            roof[kname] = {"avg_launch_ms": avg, "achieved_gbs": gbs, "frac": gbs / hbm_peak,
                           "peak_kind": f"hbm_gbs of {peak_kind}"}
    # The dense comparison: cuBLAS BF16 and the library's tcgen05 BF16 kernel
    # (zero-padded rows; 21^3 columns are not a multiple of 8), the better one.
    dense_ms = {}
    for name, prec in (("cublas_bf16", L.GW_DENSE_BF16), ("tc_bf16", L.GW_DENSE_TC_BF16)):
        try:
            dense_ms[name] = timed(lambda: ctx.gw_grad_dense(prob, du, dv, dT, dG, L.GW_MARG_TARGET, prec, stream), 5)
        except Exception as ex:
            roof[f"dense_{name}_error"] = str(ex)[:200]
    dms = min(dense_ms.values()) if dense_ms else None
    out = {"workload": f"3D grids {sx}^3 vs {sy}^3 (n={n}, m={m}), squared Euclidean, unit cube, "
                       "|N(0,1)| voxel marginals, random positive coupling, fp32",
           "grad_evals_per_s": 1e3 / gms, "grad_ms": gms, "whole_gradient_gbs": 8.0 * n * m / (gms / 1e3) / 1e9,
           "kernels": prof, "roofline": roof,
           "dense_ms": dense_ms,
           "dense_bf16_evals_per_s": (1e3 / dms) if dms else None,
           "structured_over_dense_bf16": (dms / gms) if dms else None}
    if with_solve:
        dTs = torch.empty_like(dT)
        stats = torch.zeros(8, dtype=torch.float64, device=dev)
        sprob = L.problem(dim=3, nx=sx, ny=sy, hx=w["hx"], hy=w["hy"], k=1, cost=L.GW_COST_SQEUCLID, eps=5e-3,
                          n_outer=20, n_inner=100, dtype=L.GW_F32)
        solve = lambda: ctx.gw_solve(sprob, du, dv, dTs, None, None, stats, stream=stream)
        solve()
        barrier()
        sms = timed(solve, 1)
        ctx.gw_ctx_check(stream)
        out["solve"] = {"schedule": "eps=5e-3, 20 x 100", "solves_per_s": 1e3 / sms, "ms": sms,
                        "gw_value": float(stats[1].item()), "col_marginal_err": float(stats[5].item())}
    return out


def bench_variants(ctx, L, dev, stream, barrier):
    """The method's variants on 1D grids, one timed call each after a warm-up
    call: entropic unbalanced GW (rho = 1) and mirror descent with tau = 2 eps
    and warm-started Sinkhorn at n = m = 4096 (eps = 1e-2, 20 x 100), mixed
    exponents (k_X, k_Y) = (1, 2) in the gradient at 8192^2, and the
    fixed-support barycenter of three grids (N = 1024; 1024, 2048 and 4096
    points; 3 rounds of 5 x 50)."""
    import numpy as np
    import torch
    from paper_2404_08970_gb300 import inputs as I
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=1):
        fn()
        barrier()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        barrier()
        return e0.elapsed_time(e1) / reps

    out = {}
    n = 4096
    w = I.workload_1d_grad(n, 1, "uniform", seed=0)
    du = torch.from_numpy(w["u"]).to(dev)
    dv = torch.from_numpy(w["v"]).to(dev)
    T = torch.empty(n, n, dtype=torch.float32, device=dev)
    stats = torch.zeros(8, dtype=torch.float64, device=dev)
    passes_bytes = 4.0 * n * n * 20 * 100
    for name, kw in (("ugw_solve", dict(rho=1.0)), ("tau_warm_solve", dict(tau=2e-2, warm_start=1))):
        prob = L.problem(dim=1, nx=n, ny=n, hx=1.0 / n, hy=1.0 / n, k=1, eps=1e-2, n_outer=20, n_inner=100,
                         dtype=L.GW_F32, **kw)
        try:
            ms = timed(lambda: ctx.gw_solve(prob, du, dv, T, None, None, stats, stream=stream))
            ctx.gw_ctx_check(stream)
            out[name] = {"workload": f"1D n = m = {n}, k = 1, uniform marginals, eps = 1e-2, 20 x 100, fp32, {kw}",
                         "ms": ms, "solves_per_s": 1e3 / ms, "pi_stream_gbs": passes_bytes / (ms / 1e3) / 1e9,
                         "value": float(stats[1].item())}
        except Exception as ex:
            out[name] = {"error": str(ex)[:200]}
    nm = 8192
    wm = I.workload_1d_grad(nm, 1, "uniform", seed=1)
    dT = torch.from_numpy(wm["T"].astype(np.float32)).to(dev)
    dG = torch.empty_like(dT)
    dum = torch.from_numpy(wm["u"]).to(dev)
    dvm = torch.from_numpy(wm["v"]).to(dev)
    probm = L.problem(dim=1, nx=nm, ny=nm, hx=1.0 / nm, hy=1.0 / nm, k=1, ky=2, dtype=L.GW_F32)
    try:
        ms = timed(lambda: ctx.gw_grad(probm, dum, dvm, dT, dG, L.GW_MARG_TARGET, stream), 20)
        out["mixed_k_gradient"] = {"workload": "1D n = m = 8192, (k_X, k_Y) = (1, 2), fp32", "ms": ms,
                                   "grad_evals_per_s": 1e3 / ms, "gbs_8B": 8.0 * nm * nm / (ms / 1e3) / 1e9}
    except Exception as ex:
        out["mixed_k_gradient"] = {"error": str(ex)[:200]}
    del dT, dG
    N, ns = 1024, [1024, 2048, 4096]
    rng = I.rng_for(2)
    ps = [torch.from_numpy(I.dirichlet(q, 1.0, rng)).to(dev) for q in ns]
    dp = torch.from_numpy(I.uniform_weights(N)).to(dev)
    C0 = np.abs(np.arange(N)[:, None] - np.arange(N)[None, :]) / N
    dC = torch.from_numpy(C0).to(dev, torch.float32)
    bst = torch.zeros(8 * len(ns), dtype=torch.float64, device=dev)
    bprob = L.gw_barycenter_problem(len(ns), N, 1, L.GW_F32, 1e-2, 3, 5, 50)

    def bary():
        dC.copy_(torch.from_numpy(C0).to(dev, torch.float32))
        ctx.gw_barycenter(bprob, ns, [1.0 / q for q in ns], [1.0, 1.0, 1.0], ps, dp, dC, bst, stream)

    try:
        ms = timed(bary)
        ctx.gw_ctx_check(stream)
        out["barycenter"] = {"workload": "N = 1024 barycenter of 1D grids of 1024, 2048, 4096 points, k = 1, "
                                         "eps = 1e-2, 3 rounds x 5 x 50, fp32", "ms": ms,
                             "rounds_per_s": 3e3 / ms}
    except Exception as ex:
        out["barycenter"] = {"error": str(ex)[:200]}
    return out


def bench_batch(ctx, L, dev, stream, barrier, count):
    """`count` independent 1D problems, n and m log-uniform in [256, 8192], k in
    {1, 2}, uniform marginals, eps = 1e-2, 20 x 100: one gw_solve_batch call
    (one graph launch after the first call captures it)."""
    import numpy as np
    import torch
    from paper_2404_08970_gb300 import inputs as I
    ws = I.workload_batch(count, seed=0)
    probs = [L.problem(dim=1, nx=w["nx"], ny=w["ny"], hx=w["hx"], hy=w["hy"], k=w["k"], eps=w["eps"],
                       n_outer=w["n_outer"], n_inner=w["n_inner"], dtype=L.GW_F32) for w in ws]
    u = [torch.from_numpy(w["u"]).to(dev) for w in ws]
    v = [torch.from_numpy(w["v"]).to(dev) for w in ws]
    T = [torch.empty(w["nx"], w["ny"], dtype=torch.float32, device=dev) for w in ws]
    st = [torch.zeros(8, dtype=torch.float64, device=dev) for w in ws]
    t0 = time.perf_counter()
    ctx.gw_solve_batch(probs, u, v, T, st, stream=stream)  # builds and launches the graph
    barrier()
    t_first = time.perf_counter() - t0
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.gw_solve_batch(probs, u, v, T, st, stream=stream)
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    ctx.gw_ctx_check(stream)
    nm = float(sum(w["nx"] * w["ny"] for w in ws))
    passes = sum(w["n_outer"] * w["n_inner"] for w in ws) / count
    vals = torch.stack(st)[:, 1].cpu().numpy()
    return {"workload": f"{count} 1D problems, n,m log-uniform in [256, 8192], k in {{1,2}}, uniform marginals, "
                        "eps=1e-2, 20 x 100, fp32; one gw_solve_batch call (one CUDA graph)",
            "problems": count, "ms": ms, "problems_per_s": count / (ms / 1e3),
            "sum_nm": nm, "sinkhorn_stream_gbs": 4.0 * nm * passes / (ms / 1e3) / 1e9,
            "first_call_s_incl_capture": t_first, "all_values_finite": bool(np.all(np.isfinite(vals)))}


# Size classes of served requests by n*m (points of X times points of Y).
SIZE_CLASSES = [("nm<1e6", 0, 1e6), ("1e6<=nm<1e7", 1e6, 1e7), ("1e7<=nm<1e8", 1e7, 1e8), ("nm>=1e8", 1e8, 1e30)]


def bench_serve(L, device, count, slots=8):
    """Serving: requests of four kinds (1D/2D, GW/fused GW), N per space
    log-uniform in [128, 16384], eps = 1e-2, 10 x 50, through gw_submit /
    gw_poll with a 40 GB budget and 8 slots.  Saturated throughput (all
    submitted at once), then latency with Poisson arrivals at 2000/s and at
    0.8 x the measured throughput; the first 100 requests of each phase are
    warm-up and excluded from the percentiles."""
    import numpy as np
    from paper_2404_08970_gb300 import inputs as I
    reqs = I.workload_serve(count, rate=2000.0, seed=0)
    srv = L.Server(device, hbm_budget_bytes=40 << 30, max_slots=slots)

    def prob(r):
        return L.problem(dim=r["dim"], nx=r["nx"], ny=r["ny"], hx=r["hx"], hy=r["hy"], k=r["k"],
                         cost=L.GW_COST_SQEUCLID if r["cost"] == "sqeuclid" else L.GW_COST_POW, eps=r["eps"],
                         n_outer=r["n_outer"], n_inner=r["n_inner"], theta=r["theta"],
                         feat_dim=0 if r.get("phi") is None else r["phi"].shape[1], dtype=L.GW_F32)

    probs = [prob(r) for r in reqs]
    sizes = [(r["nx"] ** 2 if r["dim"] == 2 else r["nx"]) * (r["ny"] ** 2 if r["dim"] == 2 else r["ny"])
             for r in reqs]

    def run(arrivals):
        t0 = time.perf_counter()
        tickets = []
        for r, p, a in zip(reqs, probs, arrivals):
            if a is not None:
                while time.perf_counter() - t0 < a:
                    pass
            tickets.append(srv.submit(p, r["u"], r["v"], r.get("phi"), r.get("psi")))
        lat, bad = {}, 0
        while len(lat) < len(tickets):
            for i, t in enumerate(tickets):
                if i in lat:
                    continue
                res = srv.poll(t)
                if res is not None:
                    lat[i] = res[2]
                    bad += res[0] != L.GW_OK
            time.sleep(0.001)
        wall = time.perf_counter() - t0
        keep = range(100, len(tickets)) if len(tickets) > 100 else range(len(tickets))
        la = np.array([lat[i] for i in keep])
        run.by_class = {}
        for name, lo, hi in SIZE_CLASSES:
            sel = [lat[i] for i in keep if lo <= sizes[i] < hi]
            if sel:
                run.by_class[name] = {"count": len(sel), "p50_s": float(np.percentile(sel, 50)),
                                      "p99_s": float(np.percentile(sel, 99))}
        return wall, la, bad

    try:
        run([None] * min(64, count))  # warm-up: allocator pool, module loads
        wall, la, bad = run([None] * count)
        cap = count / wall
        out = {"workload": f"{count} requests: 1D GW, 1D FGW, 2D GW, 2D FGW (1/4 each), N per space log-uniform in "
                           "[128, 16384], 2D side round(sqrt(N)), FGW theta=0.5 with 16-dim N(0,1) features, "
                           f"eps=1e-2, 10 x 50, fp32; budget 40 GB, {slots} slots",
               "saturated_solves_per_s": cap, "saturated_wall_s": wall, "errors": int(bad),
               "mean_nm": float(np.mean([(r["nx"] ** 2 if r["dim"] == 2 else r["nx"]) *
                                         (r["ny"] ** 2 if r["dim"] == 2 else r["ny"]) for r in reqs]))}
        arr = [r["arrival"] for r in reqs]
        wall, la, bad = run(arr)
        out["at_2000_per_s"] = {"p50_s": float(np.percentile(la, 50)), "p99_s": float(np.percentile(la, 99)),
                                "errors": int(bad), "note": "offered load above capacity: the queue grows"}
        rate = 0.8 * cap
        gaps = np.random.default_rng(1).exponential(1.0 / rate, size=count)
        wall, la, bad = run(list(np.cumsum(gaps)))
        out["at_0.8_capacity"] = {"rate_per_s": rate, "p50_s": float(np.percentile(la, 50)),
                                  "p99_s": float(np.percentile(la, 99)), "errors": int(bad),
                                  "by_size_class": run.by_class}
        return out
    finally:
        srv.close()


# ---------------------------------------------------------------------------
# Arms
# ---------------------------------------------------------------------------

def run_reference(args):
    """The oracle arm: each step is one bounded sample of the workload, the
    first R rows of the FP64 dense-definition gradient, with R chosen so that
    the whole warm-up + timed run takes about REF_RUN_S seconds.  ms_per_step
    is the measured time of one such step; value converts it to whole
    gradients per second (R/n of a gradient per step)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    w = workload(args.n, args.k)
    n = args.n
    t16 = oracle_rows_time(w["T"], w["u"], w["v"], w["k"], w["hx"], 16)
    per_row = max(t16 / 16, 1e-6)
    rows = int(min(n, max(16, REF_RUN_S / max(1, args.steps + args.warmup) / per_row)))
    for _ in range(args.warmup):
        oracle_rows_time(w["T"], w["u"], w["v"], w["k"], w["hx"], rows)
    times = [oracle_rows_time(w["T"], w["u"], w["v"], w["k"], w["hx"], rows) for _ in range(args.steps)]
    tot = sum(times)
    value = args.steps * (rows / n) / tot
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "step": f"first {rows} of {n} rows of one gradient ({rows / n:.4f} of a gradient evaluation)",
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config(n, args.k),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{rows} of {n} gradient rows per step (dense FP64 definition, numpy), "
                                       f"{1e3 * tot / args.steps:.0f} ms per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


REF_RUN_S = 90.0


def single_thread_oracle(w, rows):
    """Seconds for `rows` oracle gradient rows in a child process limited to
    one BLAS/OpenMP thread (the paper times single-threaded).  None if the
    child fails."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               BLIS_NUM_THREADS="1", VECLIB_MAXIMUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", str(rows), "--n", str(w["T"].shape[0]),
           "--k", str(w["k"])]
    try:
        out = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=300)
        return float(json.loads(out.stdout.strip().splitlines()[-1])["seconds"])
    except Exception:
        return None


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2404_08970_gb300 import _lib as L

    n, k = args.n, args.k
    m = args.m or n
    w = workload(n, k, m)
    ctx = L.Context(local)
    dev = torch.device("cuda", local)
    T32 = torch.from_numpy(w["T"].astype(np.float32))
    dT = T32.to(dev)
    dG = torch.empty_like(dT)
    du = torch.from_numpy(w["u"]).to(dev)
    dv = torch.from_numpy(w["v"]).to(dev)
    prob = L.problem(dim=1, nx=n, ny=m, hx=w["hx"], hy=w["hy"], k=k, dtype=L.GW_F32)
    stream = torch.cuda.current_stream(dev)

    def step():
        ctx.gw_grad(prob, du, dv, dT, dG, L.GW_MARG_TARGET, stream)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    clocks = Clocks(local)
    clocks.start()  # sampled from warm-up through the dense and solve sections
    for _ in range(max(3, args.warmup)):
        step()
    ctx.gw_ctx_check(stream)
    barrier()

    # Timed region: K gradients, each one graph launch of the library.
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    ctx.gw_ctx_check(stream)
    # Per-kernel durations for the roofline: the same K gradients again with
    # the library's per-kernel CUDA events on (eager launches bracketed by
    # events on this stream; the kernels are the same, only the gaps grow).
    ctx.gw_ctx_profile(True)
    ctx.gw_ctx_profile_report(reset=True)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    barrier()
    ms_profiled = e0.elapsed_time(e1)
    prof = ctx.gw_ctx_profile_report(reset=True)
    ctx.gw_ctx_profile(False)
    ctx.gw_ctx_check(stream)

    ms_max = max_over_ranks(ms, dev)
    per_step = ms_max / args.steps
    value = job_rate(world, args.steps, ms_max)

    # Roofline of the dominant kernel (largest total time).
    hbm_peak, bf16_peak, peak_kind = measured_peaks()
    dom = max(prof.items(), key=lambda kv: kv[1]["ms"]) if prof else (None, None)
    launches = sum(v["launches"] for v in prof.values()) if prof else 0
    nm = n * m
    roof = None
    if dom[0]:
        avg_ms = dom[1]["ms"] / max(1, dom[1]["launches"])
        alg_bytes = 8.0 * nm  # read T + write G, 4 B each (k1c) -- the gradient's algorithmic bytes
        achieved = alg_bytes / (avg_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": dom[0], "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "peak_kind": f"hbm_gbs of {peak_kind}",
                "traffic": kernel_traffic(dom[0]) if n == 8192 and m == 8192 and k == 1 else None,
                "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": avg_ms,
                "timing": "kernel durations from CUDA events in a second region of the same K gradients "
                          f"launched eagerly ({ms_profiled / args.steps:.4f} ms per gradient there)"}
    whole_gbs = 8.0 * nm / (per_step / 1e3) / 1e9

    # End to end through gw_grad_host: page-locked host u, v, T in, G out, every
    # step (the library pipelines one step's copy-in with the previous step's
    # gradient and copy-out over two device slots).  Timed on the host clock
    # from the first call to the synchronisation after the last.
    hT = T32.pin_memory()
    hG = torch.empty_like(hT).pin_memory()
    hu = torch.from_numpy(w["u"]).pin_memory()
    hv = torch.from_numpy(w["v"]).pin_memory()
    e_steps = max(3, min(args.steps, 20))
    for _ in range(3):
        ctx.gw_grad_host(prob, hu, hv, hT, hG, L.GW_MARG_TARGET, stream)
    ctx.gw_ctx_check(stream)
    barrier()
    t0 = time.perf_counter()
    for _ in range(e_steps):
        ctx.gw_grad_host(prob, hu, hv, hT, hG, L.GW_MARG_TARGET, stream)
    barrier()
    e_ms = max_over_ranks(1e3 * (time.perf_counter() - t0), dev)
    ctx.gw_ctx_check(stream)
    e2e = {"value": job_rate(world, e_steps, e_ms), "unit": UNIT, "h2d_bytes_per_step": 4 * nm + 16 * n,
           "d2h_bytes_per_step": 4 * nm, "api": "gw_grad_host (C ABI, page-locked host buffers)",
           "ms_per_step": e_ms / e_steps, "copy_gbs_per_direction": 4 * nm / (e_ms / e_steps / 1e3) / 1e9}

    # Dense comparison (cuBLAS, materialised distance matrices) on the same T.
    dense = {}
    for name, prec in (("bf16", L.GW_DENSE_BF16), ("tf32", L.GW_DENSE_TF32), ("tc_bf16", L.GW_DENSE_TC_BF16),
                       ("tc_tf32", L.GW_DENSE_TC_TF32)):
        try:
            for _ in range(2):
                ctx.gw_grad_dense(prob, du, dv, dT, dG, L.GW_MARG_TARGET, prec, stream)
            barrier()
            ds = 5
            e0.record(stream)
            for _ in range(ds):
                ctx.gw_grad_dense(prob, du, dv, dT, dG, L.GW_MARG_TARGET, prec, stream)
            e1.record(stream)
            barrier()
            dms = e0.elapsed_time(e1) / ds
            dense[name] = {"evals_per_s": 1e3 / dms, "ms": dms,
                           "tflops": 2.0 * n * m * (n + m) / (dms / 1e3) / 1e12}
        except Exception as ex:  # reported, not hidden
            dense[name] = {"error": str(ex)[:200]}
    # The structured gradient in FP64 on the same T (the paper's precision).
    try:
        dT64 = dT.double()
        dG64 = torch.empty_like(dT64)
        prob64 = L.problem(dim=1, nx=n, ny=m, hx=w["hx"], hy=w["hy"], k=k, dtype=L.GW_F64)
        for _ in range(3):
            ctx.gw_grad(prob64, du, dv, dT64, dG64, L.GW_MARG_TARGET, stream)
        barrier()
        e0.record(stream)
        for _ in range(10):
            ctx.gw_grad(prob64, du, dv, dT64, dG64, L.GW_MARG_TARGET, stream)
        e1.record(stream)
        barrier()
        ctx.gw_ctx_check(stream)
        f64ms = e0.elapsed_time(e1) / 10
        structured_f64 = {"evals_per_s": 1e3 / f64ms, "ms": f64ms,
                          "whole_gradient_gbs": 16.0 * nm / (f64ms / 1e3) / 1e9,
                          "note": "same T widened to double; 16 B per element (read T, write G)"}
        del dT64, dG64
    except Exception as ex:
        structured_f64 = {"error": str(ex)[:200]}
    best = max((d.get("evals_per_s", 0.0) for d in dense.values()), default=0.0)
    dense["structured_over_best_dense"] = (value / world) / best if best > 0 else None

    # Sampled rows of each form's output (one untimed evaluation each), compared
    # with the FP64 oracle in the CPU leg below.
    with_cpu = rank == 0 and world == 1 and not args.no_cpu_baseline
    err_rows = sorted({r for r in (0, 1, n // 152, n // 152 + 1, n // 2 - 1, n // 2, n - 2, n - 1) if 0 <= r < n})
    gpu_rows = {}
    if with_cpu:
        sel = torch.tensor(err_rows, device=dev)
        step()
        barrier()
        gpu_rows["structured_f32"] = dG.index_select(0, sel).double().cpu().numpy()
        for name, prec in (("bf16", L.GW_DENSE_BF16), ("tf32", L.GW_DENSE_TF32), ("tc_bf16", L.GW_DENSE_TC_BF16),
                           ("tc_tf32", L.GW_DENSE_TC_TF32)):
            if "ms" not in dense.get(name, {}):
                continue
            ctx.gw_grad_dense(prob, du, dv, dT, dG, L.GW_MARG_TARGET, prec, stream)
            barrier()
            gpu_rows["dense_" + name] = dG.index_select(0, sel).double().cpu().numpy()
        ctx.gw_ctx_check(stream)

    # Full entropic GW solve on the same grids (20 outer x 100 Sinkhorn), one run.
    solve = None
    if args.solve:
        w_s = workload(n, k, m)
        dTs = torch.empty_like(dT)
        stats = torch.zeros(8, dtype=torch.float64, device=dev)
        sprob = L.problem(dim=1, nx=n, ny=m, hx=w_s["hx"], hy=w_s["hy"], k=k, eps=1e-2, n_outer=20,
                          n_inner=100, dtype=L.GW_F32)
        ctx.gw_solve(sprob, du, dv, dTs, None, None, stats, stream=stream)  # captures the graph
        barrier()
        e0.record(stream)
        ctx.gw_solve(sprob, du, dv, dTs, None, None, stats, stream=stream)
        e1.record(stream)
        barrier()
        sms = e0.elapsed_time(e1)
        # Per-kernel breakdown from a second, eagerly launched and traced solve.
        ctx.gw_ctx_profile(True)
        ctx.gw_ctx_profile_report(reset=True)
        ctx.gw_solve(sprob, du, dv, dTs, None, None, stats, stream=stream)
        barrier()
        sprof = ctx.gw_ctx_profile_report(reset=True)
        ctx.gw_ctx_profile(False)
        ctx.gw_ctx_check(stream)
        sk = sprof.get("sk_pass", {"ms": 0.0, "launches": 1})
        sk_ms = sk["ms"] / max(1, sk["launches"])
        grad_ms = sum(v["ms"] for kk, v in sprof.items() if kk.startswith("k1") or kk.startswith("marg")) / 20.0
        other = sms - 20 * grad_ms
        dense_grad_ms = min((d["ms"] for d in dense.values() if isinstance(d, dict) and "ms" in d), default=None)
        solve = {"workload": "same grids, eps=1e-2, 20 mirror-descent steps x 100 Sinkhorn iterations, fp32",
                 "solves_per_s": 1e3 / sms, "ms": sms, "gw_value": float(stats[1].item()),
                 "sk_pass_ms": sk_ms, "sk_pass_gbs": 4.0 * nm / (sk_ms / 1e3) / 1e9 if sk_ms > 0 else None,
                 "gradient_ms_per_step": grad_ms,
                 "dense_solves_per_s_estimate": (1e3 / (other + 20 * dense_grad_ms)) if dense_grad_ms else None,
                 "note": "Sinkhorn passes dominate the solve (2000 passes vs 20 gradients); the dense estimate "
                         "replaces only the 20 gradients by the best dense gradient time"}

    grid2d = bench_2d(ctx, L, dev, stream, barrier, min(args.steps, 20), args.solve) if args.grid2d else None
    grid3d = bench_3d(ctx, L, dev, stream, barrier, min(args.steps, 20), args.solve) if args.grid3d else None
    variants = bench_variants(ctx, L, dev, stream, barrier) if args.variants else None
    batch = bench_batch(ctx, L, dev, stream, barrier, args.batch_count) if args.batch else None
    serve = bench_serve(L, local, args.serve_count, args.serve_slots) if args.serve else None

    clk = clocks.stop()

    cpu = None
    errs = None
    if with_cpu:
        rate, rows, t = cpu_oracle_rate(w)
        cpu = {"value": rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{rows} of {n} rows of the FP64 dense-definition gradient (numpy), {t:.1f} s"}
        st_rows = max(16, min(n, int(rows * 8.0 / max(t, 1e-3) / max(1, os.cpu_count()))))
        t1 = single_thread_oracle(w, st_rows)
        if t1:
            cpu["single_thread"] = {"value": (st_rows / n) / t1, "unit": UNIT, "cores": 1,
                                    "sample": f"{st_rows} of {n} rows, {t1:.1f} s, one BLAS thread"}
        # The oracle reads the same FP32 values of T as the GPU paths.
        Gs = oracle_rows(T32.numpy().astype(np.float64), w["u"], w["v"], k, w["hx"], w["hy"], err_rows)
        den = float(np.max(np.abs(Gs)))
        errs = {name: float(np.max(np.abs(g - Gs)) / den) for name, g in gpu_rows.items()}
        errs["rows"] = err_rows
        errs["metric"] = "max|G - G*| / max|G*| over the sampled rows; G* = FP64 oracle on the same FP32 T"

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config(n, k, m=m),
                "roofline": roof, "whole_gradient_gbs": whole_gbs, "cpu_baseline": cpu, "e2e": e2e,
                "clocks": clk, "gpu_launches": launches, "kernels": prof, "dense": dense,
                "structured_f64": structured_f64,
                "errors_vs_fp64": errs, "solve": solve,
                "grid2d": grid2d, "grid3d": grid3d, "variants": variants, "batch": batch, "serve": serve}
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.oracle_sample:
        # Child of single_thread_oracle: time `rows` oracle rows, print seconds.
        w = workload(args.n, args.k)
        t = oracle_rows_time(w["T"], w["u"], w["v"], w["k"], w["hx"], args.oracle_sample)
        print(json.dumps({"seconds": t}))
        return 0
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
