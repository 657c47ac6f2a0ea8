#!/usr/bin/env python
"""Benchmark: supernodal selected inversion on one GB300.

Workload (default): 3D 7-point Laplacian on a 40^3 grid (N = 64000), diagonal
6 + U(0,1), geometric nested dissection, relaxed supernodes (<= 128 columns,
<= 10% explicit zeros), real FP64, synthetic and seeded.  One step = one
selected inversion: normalization (L_KK^{-1}, Dinv, Lhat), the root-to-leaf
traversal (gather of A^{-1}_{C,C}, A^{-1}_{C,K}, A^{-1}_{K,K}) and the
write-back, on a plan built once for the pattern; the factors come from the
library's GPU LDL^T, outside the timed region.

Metric: GFLOP/s of the algorithmic count F = sum_K 2c^2 s + 2cs^2 + cs^2 + s^3
(same F for every variant), time per step, fraction of the FP64 roof.
Multi-GPU: replicas only (one independent selected inversion per rank).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.070   # SMs x FP64 FMA/clk/SM x flop/FMA x GHz = 1258.6
METRIC = "selinv time and FP64 GFLOP/s (% of peak); batched & adjoint vs plain on one GB300"
WORKLOADS = {
    1: "2D 5-point Laplacian 63x63 (N=3969) + 0.1 I, nested dissection, fundamental supernodes <=64 cols, FP64, plain selinv",
    2: "3D 7-point Laplacian 40^3 (N=64000), diag 6+U(0,1), nested dissection, relaxed supernodes <=128 cols / <=10% zeros, FP64, plain selinv",
    3: "DFT-like complex symmetric H - zS, 1024 atoms x 16 basis functions (N=16384), z=-0.2+0.05i, complex128, plain selinv",
    5: "3D variable-coefficient diffusion 24^3 (N=13824), theta=exp(0.5 N(0,1)), relaxed supernodes, FP64, plain selinv",
}
WORKLOAD = WORKLOADS[2]


def workload_name(cfg: int) -> str:
    return WORKLOADS.get(cfg, f"synthetic configuration {cfg}")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the plain / batched / adjoint comparison runs")
    ap.add_argument("--batch-poles", type=int, default=40)
    ap.add_argument("--schedule", type=int, default=1, help="0 plain, 1 level, 2 persistent")
    ap.add_argument("--autotune", type=int, default=1,
                    help="1: the library's autotuner picks its options on the first (untimed) call")
    ap.add_argument("--fast", type=int, default=1,
                    help="FP64-exact tensor-core contraction for s >= 16 -- 1: tcgen05, 2: mma.sync; 0: DFMA only")
    ap.add_argument("--oz-min-s", type=int, default=None,
                    help="narrowest tensor-core supernode (with --autotune 0; the autotuner picks its own)")
    ap.add_argument("--split-target", type=int, default=None, help="k-split: CTAs per SM on narrow levels")
    ap.add_argument("--split-min-steps", type=int, default=None, help="k-split: smallest k-range in 16-row steps")
    return ap.parse_args()


def reduce_max_over_ranks(value: float) -> float:
    """Max of `value` over all ranks (one process per GPU; replicas only, so
    this timing reduction is the only cross-rank communication)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, max_ms: float) -> float:
    """Whole-job throughput: the units all ranks processed / the slowest rank's time."""
    return world * units_per_rank / (max_ms * 1e-3)


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


KERNEL_SOURCES = {
    "k_selinv_oz": ("kernels_ozaki.cu", "common.cuh"),
    "k_selinv_tc": ("kernels_tc.cu", "kernels_tc_wide.cu", "tc_digits.cuh", "umma.cuh", "fixedpoint.cuh",
                    "common.cuh"),
    "k_diag": ("kernels_ozaki.cu", "common.cuh"),
    "k_diag_tc": ("kernels_tc.cu", "tc_digits.cuh", "umma.cuh", "fixedpoint.cuh", "common.cuh"),
}
DEFAULT_SOURCES = ("kernels_selinv.cu", "tile_gemm.cuh", "common.cuh")


def measured_peaks():
    """Roofline denominators: the machine's measured copy bandwidth and dense bf16
    rate, else the recipe's fallback figures."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "source": "of measured (MEASURED_PEAKS.json bf16_tflops)"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "of fallback (1.9 PFLOP/s)"}


def code_text(src: str) -> str:
    """C++/CUDA source without its comments and with whitespace collapsed:
    what the compiler sees of it (string literals here hold no comment
    markers)."""
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return " ".join(src.split())


def kernel_source_hash(kernel: str) -> str:
    """Hash of the code (comments and whitespace aside) of the sources that
    define `kernel`: a traffic figure taken on other code no longer applies."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES.get(kernel, DEFAULT_SOURCES):
        with open(os.path.join(ROOT, "paper_1604_02528_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(code_text(fh.read()).encode())
    return h.hexdigest()[:16]


def options_tag(o) -> str:
    """The options that decide a schedule's launch set (which supernodes run on
    the tensor cores and how their k-ranges split)."""
    return f"oz{o.oz_min_s}-st{o.split_target}-sm{o.split_min_steps}"


def ncu_traffic(kernel: str, tag: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the current kernel sources with the same launch set (the
    options tag); else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    want = kernel_source_hash(kernel)
    for line in open(path):
        parts = line.split()
        if len(parts) >= 4 and parts[0] == kernel and parts[1] == want and parts[3] == tag:
            return float(parts[2])
    return None


def time_calls(fn, stream, warmup, steps, flush=None):
    """Mean device time (ms) of fn() on `stream` over `steps` calls after
    `warmup`, CUDA events around each call, L2 flushed between calls."""
    import torch
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            fn()
    stream.synchronize()
    tot = 0.0
    for _ in range(steps):
        if flush is not None:
            with torch.cuda.stream(stream):
                flush.fill_(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a.record(stream)
            fn()
            b.record(stream)
        stream.synchronize()
        tot += a.elapsed_time(b)
    return tot / steps


def variant_plain(ctx, dt, L, D, Z, stream, flush, N):
    """The plain per-supernode traversal (one launch chain per supernode)."""
    o = N.selinv_default_opts()
    o.schedule = N.SELINV_SCHED_PLAIN
    N.selinv_plan_set_opts(ctx.plan, o)
    ms = time_calls(lambda: N.selinv_numeric(ctx.plan, dt, L, D, Z, stream), stream, 1, 2, flush)
    N.selinv_plan_set_opts(ctx.plan, N.selinv_default_opts())
    return ms


def variant_schedule(ctx, dt, L, D, Z, stream, flush, N, schedule, fast):
    """Another schedule / contraction choice on the same inputs."""
    o = N.selinv_default_opts()
    o.schedule = schedule
    o.fast_contraction = fast
    N.selinv_plan_set_opts(ctx.plan, o)
    ms = time_calls(lambda: N.selinv_numeric(ctx.plan, dt, L, D, Z, stream), stream, 2, 3, flush)
    N.selinv_plan_set_opts(ctx.plan, N.selinv_default_opts())
    return ms


def variant_batched(dev, stream, flush, N, npoles, lap_scale):
    """Pole shifts A - z_l I of the 40^3 pattern (complex) plus uneven
    Laplacians (real): one batched call vs one call per problem."""
    import torch
    import synth
    from paper_1604_02528_gb300.api import SelInvContext
    base = synth.make_config(4)
    e, eta = synth.pole_shifts()
    idx = np.linspace(0, len(e) - 1, npoles).round().astype(int)
    probs = [base.with_values(synth.problems.shifted_values(base, complex(e[l], eta[l]))) for l in idx]
    probs += synth.batch_laplacians(lap_scale)
    base_ctx = SelInvContext.from_problem(base)
    ctxs, Ls, Ds, Zs, dts, flops = [], [], [], [], [], 0.0
    for q in probs:
        c = base_ctx if q.n == base.n and q.values.dtype.kind == "c" else SelInvContext.from_problem(q)
        L, D = c.factor(torch.from_numpy(q.values).to(dev))
        ctxs.append(c); Ls.append(L); Ds.append(D); Zs.append(torch.empty_like(L))
        dts.append(N.SELINV_C128 if q.values.dtype.kind == "c" else N.SELINV_F64)
        flops += c.stats(dts[-1])[0]
    torch.cuda.synchronize()
    plans = [c.plan for c in ctxs]
    t_batched = time_calls(lambda: N.selinv_numeric_batched(plans, dts, Ls, Ds, Zs, stream), stream, 1, 5, flush)
    def each():
        for c, d, L, D, Z in zip(ctxs, dts, Ls, Ds, Zs):
            N.selinv_numeric(c.plan, d, L, D, Z, stream)
    t_each = time_calls(each, stream, 1, 5, flush)
    # pole-expansion sum over the diagonal of the pole shifts (after the timings: the
    # selection restricts the shared plan, which then needs every supernode anyway)
    poles = [i for i, c in enumerate(ctxs) if c is base_ctx]
    diag = np.arange(base.n)
    pos = torch.from_numpy(N.selinv_plan_select(base_ctx.plan, diag, diag)).to(dev)
    w = np.exp(1j * np.linspace(0.0, np.pi, len(poles)))
    out = torch.empty(base.n, dtype=torch.complex128, device=dev)
    t_pole = time_calls(lambda: N.selinv_pole_sum([dts[i] for i in poles], [Zs[i] for i in poles], w, pos, out,
                                                  stream), stream, 3, 10, flush)
    N.selinv_plan_select(base_ctx.plan, [], [])
    flops_c = sum(c.stats(d)[0] for c, d in zip(ctxs, dts) if d != N.SELINV_F64)
    return {"problems": f"{npoles} complex pole shifts of the 40^3 pattern + 8 Laplacians (side x {lap_scale})",
            "timed_calls": 5, "flops_per_call": flops, "complex_flops_per_call": flops_c,
            "batched_ms": round(t_batched, 3), "one_call_per_problem_ms": round(t_each, 3),
            "speedup": round(t_each / t_batched, 3), "gflops": round(flops / t_batched / 1e6, 2),
            "pole_sum_diag_ms": round(t_pole, 4)}


def variant_config(dev, stream, flush, N, cfg, steps_level, steps_plain):
    """Another configuration on its own: the level schedule (autotuned on the
    first, untimed call) against the plain per-supernode traversal, both
    timed with L2 flushed between calls."""
    import torch
    import synth
    from paper_1604_02528_gb300.api import SelInvContext
    p = synth.make_config(cfg)
    ctx = SelInvContext.from_problem(p)
    dt = N.SELINV_C128 if p.values.dtype.kind == "c" else N.SELINV_F64
    L, D = ctx.factor(torch.from_numpy(p.values).to(dev))
    Z = torch.empty_like(L)
    ctx.set_options(autotune=1)
    N.selinv_numeric(ctx.plan, dt, L, D, Z, stream)
    stream.synchronize()
    if ctx.status() != 0:
        raise RuntimeError(f"configuration {cfg} reported a device error")
    topts = N.selinv_plan_get_opts(ctx.plan)
    topts.autotune = 0
    N.selinv_plan_set_opts(ctx.plan, topts)
    t_level = time_calls(lambda: N.selinv_numeric(ctx.plan, dt, L, D, Z, stream), stream, 3, steps_level, flush)
    o = N.selinv_default_opts()
    o.schedule = N.SELINV_SCHED_PLAIN
    N.selinv_plan_set_opts(ctx.plan, o)
    t_plain = time_calls(lambda: N.selinv_numeric(ctx.plan, dt, L, D, Z, stream), stream, 1, steps_plain, flush)
    F, B = ctx.stats(dt)
    return {"workload": workload_name(cfg), "dtype": "c128" if dt != N.SELINV_F64 else "f64",
            "n": p.n, "nsuper": ctx.nsuper, "flops_per_step": F, "bytes_per_step": B,
            "level_ms": round(t_level, 4), "level_steps": steps_level,
            "plain_ms": round(t_plain, 4), "plain_steps": steps_plain,
            "level_over_plain_speedup": round(t_plain / t_level, 3),
            "gflops": round(F / t_level / 1e6, 2),
            "contraction": {0: "FP64 DFMA", 1: "tcgen05", 2: "mma.sync"}[topts.fast_contraction],
            "oz_min_s": topts.oz_min_s}


def variant_selection(ctx, dt, L, D, Z, stream, flush, N):
    """Subset selection: the diagonal of the first eighth of the columns (one
    corner of the nested-dissection order) -- only their ancestor chains run."""
    cols = np.arange(ctx.n // 8)
    N.selinv_plan_select(ctx.plan, cols, cols)
    active = N.selinv_plan_get(ctx.plan, "active")
    ms = time_calls(lambda: N.selinv_numeric(ctx.plan, dt, L, D, Z, stream), stream, 2, 3, flush)
    N.selinv_plan_select(ctx.plan, [], [])
    return {"selected": f"diagonal of columns 0..{ctx.n // 8 - 1}", "supernodes_run": int(active.sum()),
            "supernodes": int(active.size), "ms": round(ms, 3)}


def variant_adjoint(dev, stream, flush, N):
    """Forward (selected inversion, autotuned) vs reverse mode (selinv_adjoint +
    selinv_factor_adjoint) on the 24^3 diffusion workload."""
    import torch
    import synth
    from paper_1604_02528_gb300.api import SelInvContext
    p = synth.make_config(5)
    ctx = SelInvContext.from_problem(p)
    ctx.set_options(autotune=1)          # the forward's options are tuned on its first call (untimed)
    L, D = ctx.factor(torch.from_numpy(p.values).to(dev))
    Z = torch.empty_like(L)
    N.selinv_numeric(ctx.plan, N.SELINV_F64, L, D, Z, stream)
    stream.synchronize()
    W = torch.randn(Z.shape, dtype=torch.float64, device=dev)
    Lb, Db = torch.empty_like(L), torch.empty_like(D)
    Ab = torch.empty(p.nnz_lower, dtype=torch.float64, device=dev)
    t_fwd = time_calls(lambda: N.selinv_numeric(ctx.plan, N.SELINV_F64, L, D, Z, stream), stream, 2, 5, flush)
    t_adj = time_calls(lambda: N.selinv_adjoint(ctx.plan, N.SELINV_F64, L, D, Z, W, Lb, Db, stream),
                       stream, 2, 5, flush)
    t_fadj = time_calls(lambda: N.selinv_factor_adjoint(ctx.plan, N.SELINV_F64, L, D, Lb, Db, Ab, stream),
                        stream, 2, 5, flush)
    F = ctx.stats(N.SELINV_F64)[0]
    return {"workload": "3D diffusion 24^3 (N=13824), relaxed supernodes", "forward_ms": round(t_fwd, 3),
            "selinv_adjoint_ms": round(t_adj, 3), "factor_adjoint_ms": round(t_fadj, 3),
            "adjoint_over_forward": round((t_adj + t_fadj) / t_fwd, 3),
            "forward_gflops": round(F / t_fwd / 1e6, 2)}


def sample_kmin(sym, flops_target):
    """Smallest K such that the root-side supernodes K..N carry ~flops_target."""
    s, c = sym.sizes()
    F = (2 * c * c * s + 2 * c * s * s + c * s * s + s ** 3).astype(np.float64)
    acc = np.cumsum(F[::-1])
    idx = int(np.searchsorted(acc, flops_target))
    kmin = max(0, sym.nsuper - 1 - idx)
    return kmin, float(F[kmin:].sum())


def oracle_sample_setup(problem):
    import oracle
    sym = oracle.symbolic_for(problem)
    L, D = oracle.ldlt(problem, sym)
    return sym, L, D


def oracle_sample_run(sym, L, D, kmin, threads=1):
    """Wall time of the oracle's Alg. 1 over the supernodes K >= kmin; with
    threads > 1 the supernodes of one tree level run on that many host
    threads at a time (the same per-supernode steps, bit for bit)."""
    import oracle
    t = time.perf_counter()
    if threads > 1:
        oracle.selinv_levels(sym, L, D, threads, kmin=kmin)
    else:
        oracle.selinv_top(sym, L, D, kmin)
    return time.perf_counter() - t


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def host_cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                k = line.split(":")[0].strip().lower()
                if k in ("model name", "cpu part"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def run_reference(args):
    """The CPU oracle, as it stands, on bounded root-side samples of the workload."""
    rank, world, _ = dist_info()
    if rank != 0:
        return
    import synth
    p = synth.make_config(args.config)
    sym, L, D = oracle_sample_setup(p)
    kmin, fs = sample_kmin(sym, 3.0e9)
    cores = host_cores()
    for _ in range(args.warmup):
        oracle_sample_run(sym, L, D, kmin, cores)
    times = [oracle_sample_run(sym, L, D, kmin, cores) for _ in range(args.steps)]
    tot = sum(times)
    value = fs * len(times) / tot / 1e9
    sample = (f"supernodes {kmin}..{sym.nsuper - 1} of {sym.nsuper} (root side of the tree), "
              f"{fs:.3e} of {sample_kmin(sym, 1e30)[1]:.3e} flops per step, each tree level on "
              f"{cores} host threads ({host_cpu_model()})")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GFLOP/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * tot / len(times), 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.config), "sample": sample},
            "cpu_baseline": {"value": round(value, 4), "unit": "GFLOP/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 4), "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="gloo")
    if args.impl == "reference":
        run_reference(args)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    import torch
    import synth
    from paper_1604_02528_gb300 import _native as N
    from paper_1604_02528_gb300.api import SelInvContext

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    p = synth.make_config(args.config)
    ctx = SelInvContext.from_problem(p)
    o = N.selinv_default_opts()
    o.schedule = args.schedule
    o.fast_contraction = args.fast
    o.autotune = args.autotune
    if args.oz_min_s is not None:
        o.oz_min_s = args.oz_min_s
    if args.split_target is not None:
        o.split_target = args.split_target
    if args.split_min_steps is not None:
        o.split_min_steps = args.split_min_steps
    N.selinv_plan_set_opts(ctx.plan, o)
    dt = N.SELINV_C128 if p.values.dtype.kind == "c" else N.SELINV_F64
    A = torch.from_numpy(p.values).to(dev)
    L, D = ctx.factor(A)
    torch.cuda.synchronize()
    if ctx.status() != 0:
        raise RuntimeError("factorization reported a device error")
    F, B = ctx.stats(dt)
    Z = torch.empty_like(L)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > L2 (129 MB)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            N.selinv_numeric(ctx.plan, dt, L, D, Z, stream)
    stream.synchronize()
    if ctx.status() != 0:
        raise RuntimeError("selected inversion reported a device error")
    topts = N.selinv_plan_get_opts(ctx.plan)      # the options the autotuner kept
    topts.autotune = 0

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = N.selinv_launch_count()
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            for i in range(args.steps):
                flush.fill_(i & 0xFF)          # evict L2 between timed steps (outside events)
                ev[i][0].record(stream)
                N.selinv_numeric(ctx.plan, dt, L, D, Z, stream)
                ev[i][1].record(stream)
        stream.synchronize()
    torch.cuda.synchronize()
    launches = N.selinv_launch_count() - launches0
    times = [a.elapsed_time(b) for a, b in ev]
    tot_ms = reduce_max_over_ranks(sum(times))
    ms_step = tot_ms / args.steps
    value = whole_job_rate(F, world, ms_step) / 1e9

    # roofline of the dominant kernel, timed live with CUDA events per launch
    kms, kcnt = N.selinv_numeric_profile(ctx.plan, dt, L, D, Z, stream)
    sp = np.asarray(ctx.analysis["super_ptr"], np.int64)
    rp = np.asarray(ctx.analysis["rowptr"], np.int64)
    s_ = np.diff(sp).astype(np.float64)
    c_ = np.diff(rp).astype(np.float64) - s_
    mult = 1.0 if dt == N.SELINV_F64 else 4.0
    oz = (s_ >= max(16, topts.oz_min_s)) & (dt == N.SELINV_F64) & bool(topts.fast_contraction)
    peaks = measured_peaks()
    dom = int(np.argmax(kms))
    name = N.PROFILE_KINDS[dom]
    # algorithmic flops of the supernodes each kernel kind processes
    f_of = {"k_selinv": mult * float(((2 * c_ * c_ * s_ + 2 * c_ * s_ * s_) * ~oz).sum()),
            "k_selinv_oz": mult * float((2 * c_ * c_ * s_ * oz).sum()),
            "k_selinv_tc": mult * float((2 * c_ * c_ * s_ * oz).sum()),
            "k_selinv_persist": mult * float((2 * c_ * c_ * s_ + 2 * c_ * s_ * s_).sum()),
            "k_diag": mult * float((2 * c_ * s_ * s_ * oz).sum()),
            "k_lhat": mult * float((c_ * s_ * s_ * ~oz).sum()),
            "k_lhat_oz": mult * float((c_ * s_ * s_ * oz).sum()),
            "k_linv_digits": 0.0,
            "k_linv": mult * float((s_ ** 3 / 3 + (s_ ** 3 / 3) * (s_ <= 32)).sum()),
            "k_dinv": mult * float(((s_ ** 3 / 3) * (s_ > 32)).sum()),
            "k_lhat_digits": 0.0,
            "k_tc_reduce": 0.0,
            "k_diag_fin": 0.0,
            "k_push_diag": mult * float((2 * c_ * s_ * s_).sum()),
            "k_push": mult * float((2 * c_ * c_ * s_).sum()),
            "k_diag_tc": mult * float((2 * c_ * s_ * s_ * oz).sum()),
            "k_selinv_tiny": mult * float(((2 * c_ * c_ * s_ + 2 * c_ * s_ * s_) * ~oz * (s_ <= 8) * (c_ <= 64)).sum())}
    f_dom = f_of[name]
    achieved = f_dom / (kms[dom] * 1e-3) / 1e9 if kms[dom] > 0 else None
    traffic = ncu_traffic(name, options_tag(topts))
    if name in ("k_selinv_oz", "k_selinv_tc", "k_diag", "k_diag_tc", "k_lhat_oz"):
        # FP64-exact products on bf16 tensor cores: 28 digit-pair products per FP64 product
        peak, unit, bound = peaks["bf16_tflops"], "TFLOP/s", "tensor"
        ach = 28.0 * f_dom / (kms[dom] * 1e-3) / 1e12 if kms[dom] > 0 else None
        note = (f"dense bf16 peak {peaks['source']} (burst: the kernel is timed inside one "
                f"selected inversion); achieved counts the 28 bf16 digit-pair products per FP64 multiply-add")
    else:
        peak, unit, bound, ach = FP64_PEAK_GFLOPS, "GFLOP/s", "alu", achieved
        note = "FP64 FMA pipe: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (measured DFMA loop 1204)"
    roof = {"bound": bound, "achieved": round(ach, 3) if ach else None, "peak": peak, "unit": unit,
            "frac": round(ach / peak, 4) if ach else None, "traffic": traffic,
            "traffic_options": options_tag(topts), "kernel": name,
            "kernel_ms_per_step": round(kms[dom], 3), "launches_per_step": int(kcnt[dom]),
            "fp64_equiv_gflops": round(achieved, 2) if achieved else None,
            "kernel_ms_all": {k: round(v, 3) for k, v in zip(N.PROFILE_KINDS, kms)},
            "peak_note": note}

    # end to end through the C ABI from host buffers (selinv_numeric_host):
    # H2D of L and D from pinned memory, selected inversion, D2H of A^{-1},
    # every step.  The plan
    # (symbolic analysis, device tables, schedule, captured graph) is built
    # once for the pattern, as a user inverting many matrices of one pattern
    # does (the pole expansion of Sec. I); its one-time cost is reported
    # beside the number.
    Lh = L.cpu().pin_memory()
    Dh = D.cpu().pin_memory()
    Zh = torch.empty(Z.shape, dtype=Z.dtype).pin_memory()
    a = ctx.analysis
    e2e_steps = max(3, min(args.steps, 10))
    Ld = torch.empty_like(L)
    Dd = torch.empty_like(D)
    Zd = torch.empty_like(Z)
    torch.cuda.synchronize()
    tp = time.perf_counter()
    plan = N.selinv_symbolic(p.n, a["nsuper"], a["super_ptr"], a["sparent"], a["rowptr"], a["rows"], topts)

    def e2e_step():
        # host L, D in and A^-1 out through the library's host-buffer call:
        # the top levels' panels first, the rest copied in while the top
        # levels are traversed, A^-1 copied out level group by level group
        N.selinv_numeric_host(plan, dt, Lh, Dh, Zh, Ld, Dd, Zd, stream)
        stream.synchronize()

    e2e_step()   # the first call on the plan also builds its schedule and graph
    plan_ms = 1e3 * (time.perf_counter() - tp)
    e2e_step()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    # the same steps pipelined, as a stream of matrices of one pattern would
    # run: the inversions one after the other on one stream (they share the
    # plan's workspace), the copies of step i + 1's inputs and of step i - 1's
    # result on two copy streams beside it, double-buffered
    cs_in, cs_out = torch.cuda.Stream(), torch.cuda.Stream()
    bufs = [(Ld, Dd, Zd, Zh), (torch.empty_like(L), torch.empty_like(D), torch.empty_like(Z),
                               torch.empty(Z.shape, dtype=Z.dtype).pin_memory())]
    ev_in = [torch.cuda.Event() for _ in range(2)]     # inputs of a buffer landed
    ev_done = [torch.cuda.Event() for _ in range(2)]   # the inversion of a buffer finished
    ev_out = [torch.cuda.Event() for _ in range(2)]    # the result of a buffer was read back
    def pipe_run(steps):
        for i in range(steps + 1):
            if i < steps:
                b = i % 2
                Lb_, Db_, Zb_, Zhb = bufs[b]
                with torch.cuda.stream(cs_in):
                    if i >= 2:
                        cs_in.wait_event(ev_done[b])   # the buffer's previous inversion read its inputs
                    Lb_.copy_(Lh, non_blocking=True)
                    Db_.copy_(Dh, non_blocking=True)
                    ev_in[b].record(cs_in)
                stream.wait_event(ev_in[b])
                if i >= 2:
                    stream.wait_event(ev_out[b])       # its previous result was read back
                N.selinv_numeric(plan, dt, Lb_, Db_, Zb_, stream)
                ev_done[b].record(stream)
            if i >= 1:
                q = (i - 1) % 2
                with torch.cuda.stream(cs_out):
                    cs_out.wait_event(ev_done[q])
                    bufs[q][3].copy_(bufs[q][2], non_blocking=True)
                    ev_out[q].record(cs_out)
    pipe_run(2)   # untimed: the first calls with the second buffer set build what they need
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    pipe_run(e2e_steps)
    torch.cuda.synchronize()
    pipe_s = (time.perf_counter() - t1) / e2e_steps
    del plan
    esz = L.element_size()
    e2e = {"value": round(world * F / e2e_s / 1e9, 4), "unit": "GFLOP/s",
           "h2d_bytes_per_step": int((L.numel() + D.numel()) * esz),
           "d2h_bytes_per_step": int(Z.numel() * esz),
           "ms_per_step": round(1e3 * e2e_s, 3),
           "includes": "selinv_numeric_host every step: H2D of L and D from pinned memory, the "
                       "selected inversion, D2H of A^-1 (the copies overlapped with the traversal inside "
                       "the call), then a stream synchronization",
           "plan_once_ms": round(plan_ms, 3),
           "plan_once": "selinv_symbolic from host arrays + first call (schedule, device tables, graph) + one step",
           "pipelined": {"value": round(world * F / pipe_s / 1e9, 4), "ms_per_step": round(1e3 * pipe_s, 3),
                         "how": "same steps, copies of the next inputs and the previous result on two "
                                "copy streams beside the inversions, double-buffered"}}

    variants = None
    if not args.no_variants:
        variants = {"level_ms": round(ms_step, 3)}
        variants["plain_ms"] = round(variant_plain(ctx, dt, L, D, Z, stream, flush, N), 3)
        variants["level_over_plain_speedup"] = round(variants["plain_ms"] / ms_step, 3)
        variants["level_dfma_ms"] = round(variant_schedule(ctx, dt, L, D, Z, stream, flush, N,
                                                           N.SELINV_SCHED_LEVEL, 0), 3)
        variants["persistent_dfma_ms"] = round(variant_schedule(ctx, dt, L, D, Z, stream, flush, N,
                                                                N.SELINV_SCHED_PERSISTENT, 0), 3)
        variants["push_dfma_ms"] = round(variant_schedule(ctx, dt, L, D, Z, stream, flush, N,
                                                          N.SELINV_SCHED_PUSH, 0), 3)
        variants["selection"] = variant_selection(ctx, dt, L, D, Z, stream, flush, N)
        variants["batched"] = variant_batched(dev, stream, flush, N, args.batch_poles, 1.0)
        variants["adjoint"] = variant_adjoint(dev, stream, flush, N)
        variants["config1"] = variant_config(dev, stream, flush, N, 1, 50, 20)
        variants["config3"] = variant_config(dev, stream, flush, N, 3, 10, 3)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle as it stands: (i) the whole selected inversion with each
        # tree level on all host cores; (ii) one core on a root-side sample
        sym, Lo, Do = oracle_sample_setup(p)
        cores = host_cores()
        secs_all = oracle_sample_run(sym, Lo, Do, 0, cores)
        kmin, fs = sample_kmin(sym, 1.2e10)
        secs = oracle_sample_run(sym, Lo, Do, kmin)
        cpu = {"value": round(F / secs_all / 1e9, 4), "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
               "sample": f"the whole selected inversion ({F:.3e} flops, {secs_all:.1f} s), the supernodes of "
                         f"each tree level on {cores} host threads ({host_cpu_model()})",
               "single_core": {"value": round(fs / secs / 1e9, 4), "unit": "GFLOP/s", "cores": 1,
                               "sample": f"root-side supernodes {kmin}..{sym.nsuper - 1} of {sym.nsuper}, "
                                         f"{fs:.3e} of {F:.3e} flops, {secs:.1f} s"}}

    clocks = clk.summary()
    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 3), "unit": "GFLOP/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 3),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "c128" if dt == N.SELINV_C128 else "f64", "data": "synthetic",
                "config": {"workload": workload_name(args.config), "n": p.n, "nsuper": ctx.nsuper, "nnz_L": ctx.nnz,
                           "flops_per_step": F, "bytes_per_step": B,
                           "schedule": ["plain", "level", "persistent"][args.schedule],
                           "contraction": {0: "FP64 DFMA", 1: "tcgen05 fp16, FP64-exact slicing",
                                           2: "mma.sync fp16, FP64-exact slicing"}[topts.fast_contraction],
                           "options": {"autotuned": bool(args.autotune), "split_target": topts.split_target,
                                       "split_min_steps": topts.split_min_steps, "oz_min_s": topts.oz_min_s},
                           "l2": "flushed between timed steps (256 MB write)",
                           "parallelism": "replicas" if world > 1 else "single GPU",
                           "fp64_frac": round(value / world / FP64_PEAK_GFLOPS, 4)},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "variants": variants,
                "gpu_launches": int(launches), "clocks": clocks}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
