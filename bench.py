"""Benchmark: PCG time to 1e-8 relative residual on the 256x256-patch biharmonic PUM problem.

Workload (synthetic, seeded): biharmonic Delta^2 u = f on the unit square, PUM with
256 x 256 patches (stretch 1.5), local Legendre degree p = 3 (block size 10, 655,360
unknowns), 9 levels with Galerkin coarse operators, adaptive block-FSAI (P0 = lower
block pattern of A, t_max = 6, tau = 1), fourth-kind Chebyshev smoothing of degree 3 in
a V(3,3) cycle, outer PCG from x0 = 0 to ||r|| / ||b|| <= 1e-8.  f is a Fourier series
with 8 x 8 modes, coefficients N(0,1) (seed 1) scaled by (a^2 + b^2)^-1.

A step is one PCG solve to 1e-8 with the hierarchy set up and b resident in HBM.  The
headline form smooths in FP32 (A, P, G and smoother vectors in float32, FP32 accumulation)
under FP64 flexible PCG; the plain FP64 form is timed beside it.  The working set is
larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Rank 0 prints one JSON line.  Under torchrun (N > 1) every rank solves its own replica
(the solver does not shard): replicas only.
"""
from __future__ import annotations

import argparse
import functools
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import pum_inputs as pin  # noqa: E402

METRIC = "PCG time to 1e-8 rel. residual; smoother GB/s vs HBM peak, vs FP64 plain"
UNIT = "ms"
WORKLOAD = pin.BIHARMONIC_256
RTOL = 1e-8


def algorithmic_bytes(info, smooth_bytes, g_bytes, vec_bytes, iterate_bytes):
    """Algorithmic bytes of one launch of each finest-level kernel class: matrix values and
    int32 column indices once, each vector operand once (iterate_bytes: the FP64 iterate
    the smoother's epilogue accumulates into)."""
    d = info["d"]
    N = info["n"] * d
    G = info["nnzb_G"] * (d * d * g_bytes + 4)
    out = {
        "resid": info["nnzb_A"] * (d * d * smooth_bytes + 4) + 3 * N * vec_bytes,   # e, b read; r write
        "pcg_ap": info["nnzb_A"] * (d * d * 8 + 4) + 2 * N * 8,                        # A (FP64), p read; q write
        # FP64 A on the FP64 iterate and right-hand side, FP32 result
        "resid64": info["nnzb_A"] * (d * d * 8 + 4) + 2 * N * iterate_bytes + N * vec_bytes,
    }
    if info.get("fused_fsai"):
        # G read once: values and columns, r read, partial products G_ji^T t_j written (d FP32 per block)
        out["g"] = G + N * vec_bytes + info["nnzb_G"] * d * 4
        # partial products and their int32 slot positions read; p, e read and written; iterate read + write
        out["gt"] = info["nnzb_G"] * (d * 4 + 4) + 4 * N * vec_bytes + 2 * N * iterate_bytes
    else:
        out["g"] = G + 2 * N * vec_bytes                                                # r read; t write
        # t, p, e read; p, e write; iterate read + write
        out["gt"] = G + 5 * N * vec_bytes + 2 * N * iterate_bytes
    return out


ROOFLINE = {  # roofline kernel per FSAI form: class, description, ncu summary, sources it was taken from
    True: ("g", "g: fused FSAI partial products G_ji^T t_j (G read once), finest level, FP32",
           "profiles/fsai_fused_partial_biharmonic256.md",
           ("paper_2509_06744_gb300/csrc/gg.cu", "paper_2509_06744_gb300/csrc/bulk.cuh",
            "paper_2509_06744_gb300/csrc/kernels_common.cuh")),
    False: ("gt", "gt: G^T t + Chebyshev-4 update, finest level, FP32", None, ()),  # no committed capture
}


def profiled_traffic(profile, sources):
    """DRAM bytes per launch of the roofline kernel from its committed ncu summary, or None when
    there is none or the kernel sources have changed since that capture (the summary records
    their hash)."""
    import hashlib
    import re
    if profile is None:
        return None
    try:
        text = open(os.path.join(ROOT, profile)).read()
        h = hashlib.sha256()
        for s in sources:
            h.update(open(os.path.join(ROOT, s), "rb").read())
        if f"kernel_source_sha256: {h.hexdigest()}" not in text:
            return None
        return int(re.search(r"traffic_bytes_per_launch: (\d+)", text).group(1))
    except (OSError, AttributeError):
        return None


def max_over_ranks(value: float, device: str) -> float:
    """The largest value over the ranks of the default process group (the job's time is its
    slowest replica's)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs (raw samples kept as CSV in
    $PUM_CLOCKS_DIR, default the system temporary directory)."""

    def __init__(self, index):
        import tempfile
        self.index = index
        self.proc = None
        out_dir = os.environ.get("PUM_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"clocks_bench_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


@functools.lru_cache(maxsize=1)
def _oracle_setup():
    """The oracle's hierarchy and smoother set-up for the 16x16-patch version of the workload."""
    from oracle import pum as opum
    from oracle import solver
    m, levels = 16, 5
    pr = WORKLOAD
    f = opum.fourier_source(pin.fourier_coefficients(pr.rhs_seed), pr.rhs_decay)
    h = opum.build_hierarchy(m, pr.p, pr.equation, levels, f=f, constants=pr.nitsche)
    st = solver.build_setup(h, k=pr.cheb_k, mode="adaptive", P0=pr.fsai_p0, t_max=pr.t_max, tau=pr.tau)
    return m, h, st


def oracle_sample(seconds_budget: float = 20.0):
    """Time the FP64 oracle's PCG (V(3,3), adaptive block-FSAI t_max = 6) on the 16x16-patch
    version of the workload and scale to the full problem: per-iteration time grows with the
    number of unknowns (multilevel work is linear in N)."""
    from oracle import solver
    pr = WORKLOAD
    m, h, st = _oracle_setup()
    t0, c0 = time.perf_counter(), os.times()
    reps, iters = 0, 0
    while True:
        res = solver.solve(st, h.b, rtol=RTOL)
        reps += 1
        iters += res.iters
        if time.perf_counter() - t0 >= seconds_budget:
            break
    dt = time.perf_counter() - t0
    c1 = os.times()
    busy = (c1.user + c1.system - c0.user - c0.system) / max(dt, 1e-9)  # threads busy on average (BLAS)
    per_iter_per_dof = dt / iters / (m * m * pr.d)
    # the oracle's time for the whole workload: per-iteration cost scaled by unknowns (multilevel
    # work is linear in N) times the sample's own iteration count (nearly size-independent)
    per_solve_ms = per_iter_per_dof * pr.n_dofs * res.iters * 1e3
    return per_solve_ms, {"sample": f"oracle FP64 PCG on the 16x16-patch problem (2,560 unknowns, 5 levels, same "
                                    f"FSAI/smoother settings), {reps} solves of {res.iters} iterations in {dt:.1f} s; "
                                    f"time per iteration scaled by unknowns to {pr.n_dofs:,} and multiplied by "
                                    f"{res.iters} iterations",
                          "cores": max(1, round(busy)), "kind": "oracle",
                          "cores_note": f"process CPU time / wall time = {busy:.1f} (NumPy/SciPy BLAS threads) of "
                                        f"{len(os.sched_getaffinity(0))} cores available"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_sample(seconds_budget=0.0)  # one untimed solve each
    vals, meta = [], None
    for _ in range(args.steps):
        v, meta = oracle_sample(seconds_budget=max(2.0, 60.0 / max(args.steps + args.warmup, 1)))
        vals.append(v)
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": value, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD.name, "unknowns": WORKLOAD.n_dofs,
                       "note": "oracle FP64 solve time of the workload from a bounded sample"},
            "cpu_baseline": dict(meta, value=value, unit=UNIT),
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def measure_variants(H, pr, b, stream, steps):
    """The paper's cycle/smoother comparisons on the same workload: the convergence factor rho_A
    of the stationary V(k,k), V(2k,0) and Richardson-smoothed V(k,k) cycles (6 cycles from a
    U(-1,1) error, FP64 form: in the FP32 form the smoother's rounding, weighted by the
    operator's conditioning in the A-norm, is of the size of the smallest factors), and the
    V(2k,0) cycle under BiCGStab (FP32 form, time to 1e-8)."""
    import torch
    kw = dict(p0=pr.fsai_p0, adaptive=pr.adaptive, t_max=pr.t_max, tau=pr.tau, k=pr.cheb_k)
    e0 = torch.tensor(pin.uniform_vector(pr.n_dofs, 5), dtype=torch.float64, device="cuda")
    out = {"rho_A": {"precision": "f64"}}
    for name, extra in (("v2k0", dict(cycle="v2k0")), ("richardson_vkk", dict(smoother="richardson")),
                        ("vkk", {})):
        H.setup(**kw, **extra)
        out["rho_A"][name] = H.convergence_factor(e0, 6)
    H.setup(**kw, cycle="v2k0", smooth="f32", g="f32")
    x = torch.zeros_like(b)
    for _ in range(2):
        H.bicgstab(b, x, rtol=RTOL, maxit=200)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(steps):
        rep = H.bicgstab(b, x, rtol=RTOL, maxit=200)
    ev1.record(stream)
    torch.cuda.synchronize()
    out["v2k0_bicgstab"] = {"ms_per_solve": ev0.elapsed_time(ev1) / steps, "iters": rep["iters"],
                            "cycles_per_solve": 2 * rep["iters"], "solves": steps, "precision": "f32 form"}
    for name, fn in (("anisotropic", lambda: measure_anisotropic(H.ctx, pr, stream, steps)),
                     ("batch", lambda: measure_batch(H.ctx))):
        try:
            out[name] = fn()
        except Exception as ex:  # noqa: BLE001
            out[name] = {"error": f"{type(ex).__name__}: {ex}"}
    return out


def measure_batch(ctx, n_workers: int = 16, rhs: int = 16):
    """The batched uneven workload: 64 biharmonic instances (sides 32/64/96/128, p = 2 or 3, drawn
    by seed 3), adaptive FSAI (t_max = 6), FP32 form, 16 N(0,1) right-hand sides each: 1024 PCG
    solves to 1e-8, run concurrently by 16 worker contexts and, for comparison, by one."""
    import torch
    import paper_2509_06744_gb300 as pum
    insts = pin.batch_instances()
    workers = pum.make_workers(n_workers)
    t0 = time.perf_counter()
    Hs = [pum.Hierarchy.assemble(ctx, 4, it.p, it.m, it.n_levels, f_coef=pin.fourier_coefficients(3),
                                 nitsche=pin.NITSCHE_CONSTANTS[4]) for it in insts]
    pum.setup_batch(workers, Hs, p0="lower", adaptive=True, t_max=6, k=3, smooth="f32", g="f32")
    t_setup = time.perf_counter() - t0
    items = []
    for i, (H, it) in enumerate(zip(Hs, insts)):
        for r in range(rhs):
            b = torch.tensor(pin.normal_vector(it.n_dofs, 1000 * i + r), device="cuda")
            items.append((H, b, torch.zeros_like(b)))
    unknowns = sum(it.n_dofs for it in insts) * rhs
    torch.cuda.synchronize()  # the workers' streams read what torch's stream wrote
    res = {"instances": len(insts), "rhs_per_instance": rhs, "solves": len(items), "setup_s": t_setup}
    for name, ws in (("concurrent", workers), ("one_worker", workers[:1])):
        pum.solve_batch(ws, items[:len(insts)], rtol=RTOL, flexible=True)  # warm-up (graphs)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps = pum.solve_batch(ws, items, rtol=RTOL, flexible=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        res[name] = {"workers": len(ws), "s": dt, "solves_per_s": len(items) / dt,
                     "unknown_solves_per_s": unknowns / dt, "max_iters": max(r["iters"] for r in reps)}
    for H in Hs:
        H.close()
    for w in workers:
        w.close()
    return res


def measure_anisotropic(ctx, pr, stream, steps):
    """Example 5.2 at 128x128 patches (the paper's level 7): kappa = 10, theta = pi/3, p = 3,
    adaptive block-FSAI from the diagonal (t_max = 6), FP32 form, V(3,3) under PCG."""
    import torch
    import paper_2509_06744_gb300 as pum
    m, levels = 128, 8
    S = pin.anisotropy_tensor(pin.ANISO_KAPPA, pin.ANISO_THETA)
    b = torch.zeros(m * m * pr.d, dtype=torch.float64, device="cuda")
    Ha = pum.Hierarchy.assemble(ctx, pr.equation, pr.p, m, levels, f_coef=pin.fourier_coefficients(pr.rhs_seed),
                                f_decay=pr.rhs_decay, nitsche=pr.nitsche, b=b, aniso=S)
    Ha.setup(p0="diag", adaptive=True, t_max=6, k=pr.cheb_k, smooth="f32", g="f32")
    x = torch.zeros_like(b)
    for _ in range(2):
        Ha.pcg(b, x, rtol=RTOL, maxit=200, flexible=True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(steps):
        rep = Ha.pcg(b, x, rtol=RTOL, maxit=200, flexible=True)
    ev1.record(stream)
    torch.cuda.synchronize()
    Ha.close()
    return {"workload": "anisotropic biharmonic p=3 128x128 patches, kappa=10, theta=pi/3, 8 levels",
            "unknowns": m * m * pr.d, "ms_per_solve": ev0.elapsed_time(ev1) / steps, "pcg_iters": rep["iters"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="skip the V(2k,0) / Richardson measurements")
    ap.add_argument("--profile", action="store_true",
                    help="FP32 form only: one solve bracketed by cudaProfilerStart/Stop (for ncu "
                         "--profile-from-start off); prints the launch count")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)

    import paper_2509_06744_gb300 as pum

    pr = WORKLOAD
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)  # torch ops and the library share one stream
    ctx = pum.Context(local, stream=stream.cuda_stream)
    N = pr.n_dofs
    b = torch.zeros(N, dtype=torch.float64, device="cuda")
    t_setup = time.perf_counter()
    if args.profile:
        H = pum.Hierarchy.assemble(ctx, pr.equation, pr.p, pr.finest_m, pr.n_levels,
                                   f_coef=pin.fourier_coefficients(pr.rhs_seed), f_decay=pr.rhs_decay,
                                   nitsche=pr.nitsche, b=b)
        H.setup(p0=pr.fsai_p0, adaptive=pr.adaptive, t_max=pr.t_max, tau=pr.tau, k=pr.cheb_k, smooth="f32",
                g="f32")
        x = torch.zeros_like(b)
        for _ in range(args.warmup):
            H.pcg(b, x, rtol=RTOL, maxit=200, flexible=True)
        torch.cuda.synchronize()
        l0 = ctx.launches
        torch.cuda.profiler.start()
        rep = H.pcg(b, x, rtol=RTOL, maxit=200, flexible=True)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"profile": "one FP32-smoothing PCG solve", "launches": ctx.launches - l0,
                          "iters": rep["iters"]}), flush=True)
        return
    H = pum.Hierarchy.assemble(ctx, pr.equation, pr.p, pr.finest_m, pr.n_levels,
                               f_coef=pin.fourier_coefficients(pr.rhs_seed), f_decay=pr.rhs_decay,
                               nitsche=pr.nitsche, b=b)
    t_asm = time.perf_counter() - t_setup
    # plain FP64 form
    H.setup(p0=pr.fsai_p0, adaptive=pr.adaptive, t_max=pr.t_max, tau=pr.tau, k=pr.cheb_k, smooth="f64")
    t_fsai = time.perf_counter() - t_setup - t_asm
    x = torch.zeros_like(b)

    def timed_solves(n, flexible):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = []
        for _ in range(n):
            torch.cuda.synchronize()
            ev0.record(stream)
            rep = H.pcg(b, x, rtol=RTOL, maxit=200, flexible=flexible)
            ev1.record(stream)
            torch.cuda.synchronize()
            reps.append((ev0.elapsed_time(ev1), rep))
        return reps

    timed_solves(args.warmup, False)
    plain = timed_solves(args.steps, False)
    plain_ms = statistics.median(r[0] for r in plain)
    plain_iters = plain[-1][1]["iters"]
    x64 = x.clone()
    # headline form: FP32 smoothing with FP64 iterates and residuals, FP64 PCG
    H.setup(p0=pr.fsai_p0, adaptive=pr.adaptive, t_max=pr.t_max, tau=pr.tau, k=pr.cheb_k, smooth="f32", g="f32")
    timed_solves(args.warmup, True)
    # timed region: events around the roofline kernel class only
    info = H.info(0)
    roof_tk, roof_desc, roof_profile, roof_sources = ROOFLINE[bool(info["fused_fsai"])]
    ctx.timing(True, [roof_tk])
    ctx.timing_reset()
    launches0 = ctx.launches
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        reps = []
        for _ in range(args.steps):
            reps.append(H.pcg(b, x, rtol=RTOL, maxit=200, flexible=True))
        ev1.record(stream)
        torch.cuda.synchronize()
    total_ms = ev0.elapsed_time(ev1)
    launches = ctx.launches - launches0
    kt_live = ctx.timing_read()
    if world > 1:
        total_ms = max_over_ranks(total_ms, "cuda")
    ms_per_solve = total_ms / args.steps
    iters = reps[-1]["iters"]
    # per-class breakdown from an instrumented repeat of the same solves
    ctx.timing(True)
    ctx.timing_reset()
    for _ in range(args.steps):
        H.pcg(b, x, rtol=RTOL, maxit=200, flexible=True)
    kt = ctx.timing_read()
    ctx.timing(False)
    # accuracy of the fast form against the plain FP64 solution (equal accuracy check)
    rel_vs_plain = float(torch.linalg.norm(x - x64) / torch.linalg.norm(x64))
    r = torch.zeros_like(b)
    H.residual(0, b, x, r)
    true_rel = float(torch.linalg.norm(r) / torch.linalg.norm(b))

    # end to end through the C-ABI with host buffers (pinned), copies inside the timed region
    b_host = b.cpu().pin_memory()
    x_host = torch.zeros(N, dtype=torch.float64).pin_memory()
    bd, xd = torch.empty_like(b), torch.empty_like(b)
    e2e = []
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bd.copy_(b_host, non_blocking=True)
        H.pcg(bd, xd, rtol=RTOL, maxit=200, flexible=True)
        x_host.copy_(xd, non_blocking=True)
        stream.synchronize()
        if i >= args.warmup:
            e2e.append((time.perf_counter() - t0) * 1e3)
    e2e_ms = statistics.median(e2e)

    # roofline of the FSAI kernel that streams G (the finest-level class with the largest total
    # time), its launch durations taken live over the timed region
    ab = algorithmic_bytes(info, 4, 4, 4, 8)
    peak, peak_kind = load_peaks()
    n_l, ms_l = kt_live[roof_tk]
    achieved = ab[roof_tk] / (ms_l / n_l * 1e-3) / 1e9
    kernels = {k: {"launches": v[0], "avg_us": (v[1] / v[0] * 1e3) if v[0] else None,
                   "GBps": (ab[k] / (v[1] / v[0] * 1e-3) / 1e9) if v[0] else None,
                   "total_ms_per_solve": v[1] / args.steps} for k, v in kt.items()}
    dom = max(("resid", "g", "gt", "resid64"), key=lambda k: kt[k][1])
    variants = None
    if not args.no_variants:
        try:  # extra measurements: a failure there must not cost the headline line
            variants = measure_variants(H, pr, b, stream, max(3, args.steps // 4))
        except Exception as ex:  # noqa: BLE001
            variants = {"error": f"{type(ex).__name__}: {ex}"}

    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline:
        v, meta = oracle_sample()
        cpu = dict(meta, value=v, unit=UNIT)
    line = {
        "metric": METRIC, "value": ms_per_solve, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_solve, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": pr.name, "unknowns": N, "levels": pr.n_levels, "pcg": "flexible FP64",
                   "smoother": "FP32 A/P/G and correction vectors, FP32 accumulation; FP64 iterates, "
                               "residuals and prolongation", "rtol": RTOL,
                   "l2": "working set larger than L2 (no flush)", "parallelism": "replicas only"},
        "pcg_iters": iters, "true_relres": true_rel, "rel_diff_vs_fp64_plain": rel_vs_plain,
        "fp64_plain": {"ms_per_solve": plain_ms, "pcg_iters": plain_iters, "dtype": "f64"},
        "setup_s": {"assembly_and_galerkin": t_asm, "fsai_lanczos_fp64": t_fsai},
        "kernels_finest": kernels,
        "roofline": {"kernel": roof_desc, "bound": "hbm",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": profiled_traffic(roof_profile, roof_sources),
                     "peak_source": peak_kind, "algorithmic_bytes_per_launch": ab[roof_tk], "launches_timed": n_l,
                     "largest_total_class": dom},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_ms, "unit": UNIT, "h2d_bytes_per_step": N * 8, "d2h_bytes_per_step": N * 8},
        "job_solves_per_s": world * args.steps / (total_ms * 1e-3),  # all replicas' solves / slowest rank's time
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "variants": variants,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
