#!/usr/bin/env python3
"""Leapfrog throughput of scheme 2 (arXiv 2302.04979) on one GB300, in DoF-steps/s.

Workload: unit-cube PEC cavity, identity map, spline degree p = 3, 64^3
elements (N_e + N_h = 1,685,970 degrees of freedom), permittivity piecewise
constant on a seeded 8^3 grid of element blocks (uniform in [1, 9)), mu = 1,
seeded random initial D, divergence-free random B, J = 0, dt = 0.5 x the CFL
limit.  One step = one full kick-drift-kick leapfrog step (curl, Hodge apply,
pairing solve for both fields) in FP64.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --profile FORM     # eager steps of the workload for profiler captures

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
(the slow, plain implementation the tests check against) on the host cores.
For N > 1 (torchrun) every rank runs its own independent cavity (replicas, no
collective in the data path); value = all ranks' DoF-steps / max rank time.
Beside the headline FP64 number the line carries the mixed form, the other
cavity configurations (shorter runs of the same protocol) and the batched
64-cavity configuration, each with its DoF-steps/s.
"""
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "leapfrog DoF-steps/s (p=3, 64^3) FP64 vs mixed; % HBM/tensor roofline"
UNIT = "DoF-steps/s"
P, NEL, EPS_BLOCKS, SEED = 3, 64, (8, 8, 8), 2302
L2_FLUSH_BYTES = 256 << 20
# algorithmic bytes of one FP64 step per degree of freedom at p = 3, 64^3 (each kernel reads its
# inputs once and writes its outputs once; the survey's kernel-by-kernel count)
STEP_BYTES_PER_DOF = 89.0


# ------------------------------------------------------------------ peaks (roofline denominators)
def _unit_peaks():
    """CUDA-core peaks from unit counts and the maximum SM clock: 152 SMs x (2 FP64 | 128 FP32)
    FMA lanes per clock x 2 flop x 2.07 GHz."""
    return {"fp64_tflops": 152 * 2 * 2 * 2.07e9 / 1e12, "fp32_tflops": 152 * 128 * 2 * 2.07e9 / 1e12}


def load_peaks():
    """HBM copy bandwidth and BF16 dense throughput measured on this machine (MEASURED_PEAKS.json),
    else the documented fallback (6.8 TB/s, 1.9 PFLOP/s); CUDA-core peaks from unit counts."""
    peaks = dict(_unit_peaks())
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        m = json.load(open(path))
        peaks.update(hbm_gbs=float(m["hbm_gbs"]), bf16_tflops=float(m["bf16_tflops"]),
                     bf16_tflops_sustained=float(m.get("bf16_tflops_sustained", m["bf16_tflops"])),
                     source="of measured (MEASURED_PEAKS.json)")
    except (OSError, KeyError, ValueError):
        peaks.update(hbm_gbs=6800.0, bf16_tflops=1900.0, bf16_tflops_sustained=1700.0, source="of fallback")
    return peaks


# ------------------------------------------------------------------ kernel functions and their rooflines
# kernel class (smx_kernel_times) -> (kernel function, arithmetic pipe, the roof it is rated against).
# The rated roof is the survey's bound for that kernel: HBM for the curls, casts and the FP32 mass
# applies, the FP64 pipe for the FP64 Hodge and line kernels, the FP32 pipe for the FP32 dense line
# products, and the BF16 tensor pipe for the digit-sliced products.
KERNEL_FUNCTION = {
    "curl_primal": ("curl_plane_kernel<double>", "fp64", "hbm"),
    "curl_dual": ("curl_plane_kernel<double>", "fp64", "hbm"),
    "hodge_block": ("hodge_block_kernel", "fp64", "alu"), "hodge_quad": ("hodge_quad_kernel", "fp64", "alu"),
    "solve_x": ("solve_axis_kernel", "fp64", "alu"), "solve_y": ("solve_axis_kernel", "fp64", "alu"),
    "solve_z": ("solve_axis_kernel", "fp64", "alu"),
    "mass_solve_x": ("mass_solve_axis_kernel", "fp64", "alu"),
    "mass_solve_y": ("mass_solve_axis_kernel", "fp64", "alu"),
    "mass_solve_z": ("mass_solve_axis_kernel", "fp64", "alu"),
    "line_f64tc_x": ("mode_digit_kernel<7 digits>", "tensor", "tensor"),
    "line_f64tc_y": ("mode_digit_kernel<7 digits>", "tensor", "tensor"),
    "line_f64tc_z": ("mode_digit_kernel<7 digits>", "tensor", "tensor"),
    "curl_primal_f32": ("curl_plane_kernel<float>", "fp32", "hbm"),
    "curl_dual_f32": ("curl_plane_kernel<float>", "fp32", "hbm"),
    "hodge_block_f32": ("hodge_block_f32_kernel", "fp32", "hbm"),
    "hodge_quad_f32": ("hodge_quad_f32_kernel", "fp32", "hbm"),
    "line_f32_x": ("mode_f32_kernel", "fp32", "alu"), "line_f32_y": ("mode_f32_kernel", "fp32", "alu"),
    "line_f32_z": ("mode_f32_kernel", "fp32", "alu"),
    "line_f32tc_x": ("mode_digit_kernel<4 digits>", "tensor4", "tensor"),
    "line_f32tc_y": ("mode_digit_kernel<4 digits>", "tensor4", "tensor"),
    "line_f32tc_z": ("mode_digit_kernel<4 digits>", "tensor4", "tensor"),
    "cast": ("cast kernels", "fp32", "hbm"),
    "residual": ("band_apply_kernel", "fp64", "alu"),
}
# digit products per FP64-equivalent multiply-add of a dense line product: levels 0..6 of seven
# digits (28) in the FP64 form, levels 0..3 of four digits (10) in the mixed form's tensor option
DIGIT_PAIRS = {"tensor": 28, "tensor4": 10}

# DRAM bytes (read + write) per launch from one ncu capture of each kernel function at this
# workload (files under profiles/; cold caches before each launch, outputs stay in L2).  A
# kernel that changed since its capture is left out (traffic null).
NCU_TRAFFIC = {
    "mass_solve_axis_kernel": None, "solve_axis_kernel": None, "hodge_block_kernel": 13.51e6,
    "mode_f32_kernel": None, "hodge_block_f32_kernel": 13.51e6,
    "mode_digit_kernel<7 digits>": 7.05e6, "mode_digit_kernel<4 digits>": 4.70e6,
}


def kernel_rooflines(table, peaks):
    """Group per-class event times (kernel_table) by kernel function and rate each function
    against every roof it has: HBM (algorithmic bytes) and its arithmetic pipe (FP64 or FP32
    CUDA cores, or the BF16 tensor pipe for the digit-sliced products).  'bound' and 'frac' are
    the rated roof of KERNEL_FUNCTION; 'binding' is the roof with the largest fraction (attainable
    time = max over resources of work / peak).  Returns (list sorted by total time, the dominant
    function's entry)."""
    funcs = {}
    for cls, v in table.items():
        if cls not in KERNEL_FUNCTION:
            continue
        name, roof, rated = KERNEL_FUNCTION[cls]
        f = funcs.setdefault(name, {"kernel": name, "roof": roof, "rated": rated, "classes": [], "launches": 0,
                                    "total_ms": 0.0, "flops": 0.0, "bytes": 0.0})
        f["classes"].append(cls)
        f["launches"] += v["launches"]
        f["total_ms"] += v["total_ms"]
        f["flops"] += v["flops_per_launch"] * v["launches"]
        f["bytes"] += v["bytes_per_launch"] * v["launches"]
    out = []
    total = sum(f["total_ms"] for f in funcs.values()) or 1.0
    for f in funcs.values():
        sec = f["total_ms"] * 1e-3
        gbs = f["bytes"] / sec / 1e9
        fr = {"hbm": gbs / peaks["hbm_gbs"]}
        if f["roof"] == "fp64":
            ach = f["flops"] / sec / 1e12
            fr["alu"] = ach / peaks["fp64_tflops"]
            alu = {"achieved": ach, "peak": peaks["fp64_tflops"], "unit": "TFLOP/s",
                   "peak_source": "FP64 unit count x clock (152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz)"}
        elif f["roof"] == "fp32":
            ach = f["flops"] / sec / 1e12
            fr["alu"] = ach / peaks["fp32_tflops"]
            alu = {"achieved": ach, "peak": peaks["fp32_tflops"], "unit": "TFLOP/s",
                   "peak_source": "FP32 unit count x clock (152 SMs x 128 FMA/clk x 2 flop x 2.07 GHz)"}
        else:
            ach = DIGIT_PAIRS[f["roof"]] * f["flops"] / sec / 1e12
            fr["tensor"] = ach / peaks["bf16_tflops"]
            alu = {"achieved": ach, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                   "peak_source": "BF16 dense, cuBLAS burst " + peaks["source"],
                   "work": "%d BF16 digit products x 2 n flops per line entry (padding not counted)"
                           % DIGIT_PAIRS[f["roof"]], "fp64_equivalent_tflops": f["flops"] / sec / 1e12}
        binding = max(fr, key=fr.get)
        bound = f["rated"]
        ent = {"kernel": f["kernel"], "classes": f["classes"], "launches": f["launches"],
               "avg_us": 1e3 * f["total_ms"] / f["launches"], "share": f["total_ms"] / total,
               "bound": bound, "frac": fr[bound], "fracs": fr, "binding": binding, "hbm_gbs": gbs,
               "hbm_peak_gbs": peaks["hbm_gbs"], "arith": alu,
               "traffic": NCU_TRAFFIC.get(f["kernel"])}
        out.append(ent)
    out.sort(key=lambda e: -e["share"])
    return out, (out[0] if out else None)


def roofline_line(dom, peaks):
    """The 'roofline' object of the JSON line for the dominant kernel function, per launch."""
    if dom is None:
        return None
    if dom["bound"] == "hbm":
        roof = {"bound": "hbm", "achieved": dom["hbm_gbs"], "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "peak_source": "HBM copy bandwidth " + peaks["source"]}
    else:
        a = dom["arith"]
        roof = {"bound": "tensor" if dom["bound"] == "tensor" else "alu", "achieved": a["achieved"], "peak": a["peak"],
                "unit": a["unit"], "peak_source": a["peak_source"]}
    roof.update(kernel=dom["kernel"], frac=roof["achieved"] / roof["peak"], traffic=dom["traffic"],
                avg_us_per_launch=dom["avg_us"], launches=dom["launches"], share=dom["share"])
    return roof


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the GPU is busy."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            cmd = ["nvidia-smi", "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits", "-lms", "100"]
            if self.gpu_id is not None:
                cmd += ["-i", str(self.gpu_id)]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def reduce_max(value, world):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value, world):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_rate(units_this_rank, seconds_this_rank, world):
    """Whole-job throughput: all ranks' units / the slowest rank's time (max over ranks)."""
    return reduce_sum(units_this_rank, world) / reduce_max(seconds_this_rank, world)


def init_dist(world):
    """One process per GPU: NCCL when CUDA is present, gloo otherwise (CPU runs of the host logic)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")


# ------------------------------------------------------------------ CPU oracle timing
def oracle_setup():
    from oracle import maxwell as mx
    from paper_2302_04979_gb300 import synth
    eps = ("blocks", synth.block_material(SEED, EPS_BLOCKS, 1.0, 9.0))
    S = mx.Scheme2(P, NEL, eps=eps)
    d = synth.uniform(SEED + 1, S.N_e, -1.0, 1.0)
    b = S.D1 @ synth.uniform(SEED + 2, S.N_e, -1.0, 1.0)
    e = S.e_from_d(d)
    return S, d, b, e


def threads_available():
    try:
        from threadpoolctl import threadpool_info
        return int(max((i.get("num_threads", 1) for i in threadpool_info()), default=1))
    except Exception:
        return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def _limit_threads(n):
    """Context manager limiting the BLAS/LAPACK pools to n threads (no-op if threadpoolctl is missing)."""
    try:
        from threadpoolctl import threadpool_limits
        return threadpool_limits(limits=n)
    except Exception:
        import contextlib
        return contextlib.nullcontext()


def time_oracle_steps(S, d, b, e, nsteps_max, budget_s, threads=None):
    """Oracle leapfrog steps on the full workload: (DoF-steps/s, steps, wall s, effective cores).
    The effective core count is process CPU time / wall time over the timed steps (numpy's
    elementwise work is single-threaded; only the LAPACK line solves use the BLAS pool)."""
    dt = 1e-3
    ctx = _limit_threads(threads) if threads else _limit_threads(None)
    with ctx:
        c0, t0 = time.process_time(), time.perf_counter()
        n = 0
        while n < nsteps_max:
            d, b, e, _ = S.step(d, b, e, dt, 1)
            n += 1
            if time.perf_counter() - t0 > budget_s:
                break
        el = time.perf_counter() - t0
        cpu = time.process_time() - c0
    return (S.N_e + S.N_h) * n / el, n, el, cpu / el


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_baseline(budget_s=12.0, max_steps=8):
    """The oracle as it stands, timed on the host cores: all cores (BLAS pool) and single-threaded."""
    t0 = time.perf_counter()
    S, d, b, e = oracle_setup()
    setup = time.perf_counter() - t0
    S.step(d, b, e, 1e-3, 1)   # warm-up (first LAPACK calls)
    r_all, n_all, el_all, eff = time_oracle_steps(S, d, b, e, max_steps, budget_s)
    r_one, n_one, el_one, _ = time_oracle_steps(S, d, b, e, max_steps, budget_s, threads=1)
    host = "%s, %d cpus" % (cpu_model(), os.cpu_count() or 0)
    return {"value": r_all, "unit": UNIT, "cores": round(eff, 1), "kind": "oracle",
            "sample": "%d full 64^3 FP64 leapfrog steps of the oracle (%.1f s) after 1 warm-up step, BLAS pool of %d "
                      "threads (effective cores = CPU time / wall time); setup %.1f s not timed; host %s"
                      % (n_all, el_all, threads_available(), setup, host),
            "single_thread": {"value": r_one, "unit": UNIT, "cores": 1,
                              "sample": "%d full 64^3 steps (%.1f s), BLAS pool limited to 1 thread"
                                        % (n_one, el_one)}}


def run_reference(args, rank, world):
    if rank != 0:
        return
    S, d, b, e = oracle_setup()
    budget = max(20.0, min(150.0, 2.0 * (args.steps + args.warmup)))
    S.step(d, b, e, 1e-3, 1)
    rate, n, el, eff = time_oracle_steps(S, d, b, e, args.steps, budget)
    sample = ("%d of the %d requested steps on the full 64^3 workload (%.1f s), warm-up 1; host %s, %d cpus, BLAS "
              "pool %d threads" % (n, args.steps, el, cpu_model(), os.cpu_count() or 0, threads_available()))
    out = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / n, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(S.N_e, S.N_h),
           "cpu_baseline": {"value": rate, "unit": UNIT, "cores": round(eff, 1), "kind": "oracle", "sample": sample},
           "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def workload_config(ne, nh, extra=None):
    cfg = {"workload": "PEC cavity, identity map, p=3, 64^3 elements, eps 8^3 blocks U[1,9), mu=1",
           "p": P, "nel": [NEL] * 3, "N_e": ne, "N_h": nh, "dof": ne + nh,
           "initial": "seeded random d, divergence-free random b, J=0", "dt": "0.5 x CFL",
           "l2": "flushed between timed steps (256 MiB write)", "parallelism": "replicas"}
    if extra:
        cfg.update(extra)
    return cfg


# ------------------------------------------------------------------ GPU arm
def kernel_table(ctx, smx, ktimes):
    """Per-kernel-class launches, time, share and algorithmic work per launch."""
    mode = {smx.FIELD_B: ctx.hodge_mode(smx.FIELD_B), smx.FIELD_D: ctx.hodge_mode(smx.FIELD_D)}
    sol = [f for f, m in ((smx.FIELD_H, mode[smx.FIELD_B]), (smx.FIELD_E, mode[smx.FIELD_D])) if m != 2]
    sep = [f for f, m in ((smx.FIELD_H, mode[smx.FIELD_B]), (smx.FIELD_E, mode[smx.FIELD_D])) if m == 2]
    both = [smx.FIELD_H, smx.FIELD_E]
    fields = {"curl_primal": [smx.FIELD_B], "curl_dual": [smx.FIELD_D],
              "hodge_block": [f for f in (smx.FIELD_B, smx.FIELD_D) if mode[f] == 0],
              "hodge_quad": [f for f in (smx.FIELD_B, smx.FIELD_D) if mode[f] == 1],
              "solve_x": sol, "solve_y": sol, "solve_z": sol,
              "mass_solve_x": sep, "mass_solve_y": sep, "mass_solve_z": sep,
              "curl_primal_f32": [smx.FIELD_B], "curl_dual_f32": [smx.FIELD_D],
              "hodge_block_f32": [f for f in (smx.FIELD_B, smx.FIELD_D) if mode[f] == 0],
              "hodge_quad_f32": [f for f in (smx.FIELD_B, smx.FIELD_D) if mode[f] == 1],
              "line_f32_x": both, "line_f32_y": both, "line_f32_z": both,
              "line_f32tc_x": both, "line_f32tc_y": both, "line_f32tc_z": both,
              "line_f64tc_x": both, "line_f64tc_y": both, "line_f64tc_z": both, "cast": both,
              "residual": both}
    kern = {}
    for name, (ms, cnt) in ktimes.items():
        if cnt == 0 or name not in fields:
            continue
        works = []
        for f in fields[name]:
            try:
                works.append(ctx.kernel_work(name, f))
            except smx.SmxError:
                pass
        if not works:
            continue
        fl = sum(w[0] for w in works) / len(works)
        by = sum(w[1] for w in works) / len(works)
        avg_ms = ms / cnt
        kern[name] = {"launches": cnt, "total_ms": ms, "avg_us": 1e3 * avg_ms,
                      "tflops": fl / (avg_ms * 1e-3) / 1e12, "gbs": by / (avg_ms * 1e-3) / 1e9,
                      "flops_per_launch": fl, "bytes_per_launch": by}
    total_k = sum(v["total_ms"] for v in kern.values())
    for v in kern.values():
        v["share"] = v["total_ms"] / total_k if total_k else None
    return kern


def time_steps(ctx, state, dt, steps, flush, stream, world, jhat=None, amp=None):
    """K single steps, L2 flushed before each, CUDA events on the launching stream; (sum ms, launches)."""
    import torch
    d, b, e, h = state
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    launches0 = ctx.launch_count()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed_region")
    for k in range(steps):
        flush.fill_(float(k))
        starts[k].record(stream)
        ctx.step(d, b, e, h, dt, 1, jhat=jhat, amp=amp)   # same pointers every step: one captured graph
        ends[k].record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    return sum(s.elapsed_time(t) for s, t in zip(starts, ends)), ctx.launch_count() - launches0


def steady_and_kernels(ctx, smx, state, dt, steps, flush, stream):
    """Steady state (K steps in one call) and per-kernel event times over K flushed single steps."""
    import torch
    d, b, e, h = state
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    ctx.step(d, b, e, h, dt, steps)
    s1.record(stream)
    torch.cuda.synchronize()
    ctx.set_timing(True)
    for k in range(steps):
        flush.fill_(float(k))
        ctx.step(d, b, e, h, dt, 1)
    kt = ctx.kernel_times()
    ctx.set_timing(False)
    return s0.elapsed_time(s1), kernel_table(ctx, smx, kt)


def make_state(ctx, smx, dev, seed):
    """Seeded random d, divergence-free b = D^1 (random), e consistent with d, h = 0 (device)."""
    import torch
    from paper_2302_04979_gb300 import synth
    d0 = torch.as_tensor(synth.uniform(seed, ctx.N_e, -1.0, 1.0)).to(dev)
    b0 = torch.zeros(ctx.N_h, dtype=torch.float64, device=dev)
    ctx.curl_primal(torch.as_tensor(synth.uniform(seed + 1, ctx.N_e, -1.0, 1.0)).to(dev), b0, 1.0)
    e0 = torch.empty(ctx.N_e, dtype=torch.float64, device=dev)
    ctx.hodge_star(smx.FIELD_D, d0, e0)
    return d0, b0, e0, torch.zeros(ctx.N_h, dtype=torch.float64, device=dev)


def other_configs(smx, dev, stream, flush, steps):
    """The other single-cavity configurations, same protocol (L2 flushed before each single step,
    CUDA events), fewer steps: DoF-steps/s of the FP64 form and of both mixed forms."""
    import torch
    from paper_2302_04979_gb300 import synth
    specs = [
        ("cube p=2, 8^3, eps=mu=1", dict(p=2, nel=8), False),
        ("curved (sine bump 0.05) p=3, 32^3, Gaussian-bump eps, pulse source", dict(
            p=3, nel=32, geometry="sine_bump", amplitude=0.05, eps=synth.GaussianBumps(SEED)), True),
        ("identity p=4, 64^3, eps 8^3 blocks U[1,9)", dict(
            p=4, nel=64, eps=("blocks", synth.block_material(SEED, EPS_BLOCKS, 1.0, 9.0))), False),
    ]
    res = {}
    for name, kw, source in specs:
        ent = {}
        for prec in ("fp64", "mixed", "mixed_refined"):
            ctx = smx.Context(precision=prec, **kw).bind(dev)
            ctx.set_stream(stream)
            st = make_state(ctx, smx, dev, SEED + 5)
            dt = 0.5 * ctx.cfl(iters=200, tol=1e-6)
            jhat = amp = None
            if source:
                shapes = [ctx.comp_shape(smx.FIELD_D, c) for c in range(3)]
                jhat = torch.as_tensor(synth.bump_coefficients(SEED, shapes)).to(dev)
                amp = torch.as_tensor(synth.source_amplitudes(dt, steps)).to(dev)
            for _ in range(3):
                ctx.step(*st, dt, 1, jhat=jhat, amp=amp)
            ms, _ = time_steps(ctx, st, dt, steps, flush, stream, 1, jhat=jhat, amp=amp)
            dof = ctx.N_e + ctx.N_h
            ent[prec] = {"value": dof * steps / (ms * 1e-3), "ms_per_step": ms / steps}
            ent["dof"] = dof
            del ctx
        ent["steps"] = steps
        res[name] = ent
    return res


def batched_config(smx, dev, stream, nsteps, precision="fp64", dts=None):
    """64 independent cavities of seeded uneven sizes (nel in [16, 48], even) and degrees p in
    {2, 3, 4}, each with its own permittivity on a 2^3 block grid (U[1, 4)) and Gaussian-pulse
    source; one persistent launch per step after autotuning; DoF-steps/s over nsteps steps.
    precision "fp64" or "mixed_refined"; dts: the time steps (0.5 x CFL of the FP64 form, computed
    here when not given)."""
    import torch
    from paper_2302_04979_gb300 import synth
    nel = 16 + 2 * (synth.splitmix64(4040, 64) % 17).astype(int)
    p = 2 + (synth.splitmix64(4041, 64) % 3).astype(int)
    ctxs, keep = [], []
    for k in range(64):
        ctx = smx.Context(int(p[k]), int(nel[k]), eps=("blocks", synth.block_material(4100 + k, (2, 2, 2), 1.0, 4.0)),
                          precision=precision)
        ctx.bind(dev)
        ctx.set_stream(stream)
        ctxs.append(ctx)
    batch = smx.Batch(ctxs, device=dev)
    out_dts = []
    for k, ctx in enumerate(ctxs):
        st = make_state(ctx, smx, dev, 5000 + 10 * k)
        dt = dts[k] if dts is not None else 0.5 * ctx.cfl(iters=100, tol=1e-4)
        out_dts.append(dt)
        shapes = [ctx.comp_shape(smx.FIELD_D, c) for c in range(3)]
        jhat = torch.as_tensor(synth.bump_coefficients(4200 + k, shapes)).to(dev)
        amp = torch.as_tensor(synth.source_amplitudes(dt, nsteps + 8)).to(dev)
        batch.set_state(k, *st, dt, jhat=jhat, amp=amp)
        keep.append((st, jhat, amp, dt))
    lw = batch.autotune(steps=2)
    for k, ctx in enumerate(ctxs):   # restart the amplitude index after the autotuner
        st, jhat, amp, dt = keep[k]
        batch.set_state(k, *st, dt, jhat=jhat, amp=amp)
    batch.step(2)
    batch.status()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s0.record(stream)
    batch.step(nsteps)
    s1.record(stream)
    batch.status()
    ms = s0.elapsed_time(s1)
    dof = sum(c.N_e + c.N_h for c in ctxs)
    return {"value": dof * nsteps / (ms * 1e-3), "ms_per_step": ms / nsteps, "unit": UNIT, "steps": nsteps,
            "cavities": 64, "dof": int(dof), "line_warps": lw,
            "dtype": "f64" if precision == "fp64" else "f32 operators, f64 residual refinement, f64 state",
            "note": "one persistent cooperative launch per step (CUDA-graph replay); the state of all cavities "
                    "(%.0f MB) is larger than L2" % (sum(8 * 2 * (c.N_e + c.N_h) for c in ctxs) / 1e6)}, out_dts


def scheme1_comparison(smx, dev, stream, eps, steps, dt2):
    """Scheme 1 (mass-matrix Hodge stars, Sec. 3.3) on the same workload: ms per step (eager, the CG
    reads its residual on the host every few iterations), CG iterations, and its CFL limit beside
    scheme 2's (Sec. 5.2), so the per-step and whole-run costs of the two schemes compare."""
    import torch
    ctx = smx.Context(P, NEL, eps=eps, mu=1.0, scheme1=True).bind(dev)
    ctx.set_stream(stream)
    st = make_state(ctx, smx, dev, SEED + 9)
    e1 = torch.empty_like(st[2])
    ctx.scheme1_star(smx.FIELD_D, st[0], e1, tol=1e-12)
    st = (st[0], st[1], e1, st[3])
    dt1 = ctx.cfl_scheme1(iters=60, tol=1e-4, cg_tol=1e-10)
    dt = 0.5 * dt1
    iters = ctx.step_scheme1(*st, dt, 1, tol=1e-12)
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    iters = max(iters, ctx.step_scheme1(*st, dt, steps, tol=1e-12))
    s1.record(stream)
    torch.cuda.synchronize()
    ms = s0.elapsed_time(s1) / steps
    dof = ctx.N_e + ctx.N_h
    return {"value": dof / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": steps, "max_cg_iterations": iters,
            "cg_tol": 1e-12, "dt_max": dt1, "dt_max_scheme2": dt2,
            "note": "scheme 1 of the paper (Sec. 3.3): Hodge stars by preconditioned CG on the 1-form masses; "
                    "same workload, FP64"}


def run_ours(args, rank, world, local):
    import torch
    from paper_2302_04979_gb300 import smx, synth

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (there is no CPU fallback)")
    peaks = load_peaks()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    eps = ("blocks", synth.block_material(SEED, EPS_BLOCKS, 1.0, 9.0))
    ctx = smx.Context(P, NEL, eps=eps, mu=1.0).bind(dev)
    stream = torch.cuda.Stream(device=dev)   # non-default: smx_step replays a captured CUDA graph
    torch.cuda.set_stream(stream)
    ctx.set_stream(stream)
    ne, nh = ctx.N_e, ctx.N_h
    dof = ne + nh
    d0, b0, e0, _ = make_state(ctx, smx, dev, SEED + 1 + 17 * rank)
    dt = 0.5 * ctx.cfl(iters=400, tol=1e-8)
    flush = torch.empty(L2_FLUSH_BYTES // 8, dtype=torch.float64, device=dev)
    state = (d0.clone(), b0.clone(), e0.clone(), torch.zeros(nh, dtype=torch.float64, device=dev))

    for _ in range(args.warmup):
        ctx.step(*state, dt, 1)
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    gpu_index = None
    try:
        gpu_index = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_index = None
    sampler = ClockSampler(gpu_index)
    sampler.start()
    time.sleep(0.3)

    # ---- FP64 form: timed region
    total_ms, launches = time_steps(ctx, state, dt, args.steps, flush, stream, world)
    total_ms = reduce_max(total_ms, world)
    value = reduce_sum(dof * args.steps, world) / (total_ms * 1e-3)
    steady_ms, kern = steady_and_kernels(ctx, smx, state, dt, args.steps, flush, stream)
    steady_ms = reduce_max(steady_ms, world)

    # ---- mixed form on the same workload and protocol (FP32 operators, FP64 state)
    mctx = smx.Context(P, NEL, eps=eps, mu=1.0, precision="mixed").bind(dev)
    mctx.set_stream(stream)
    mstate = (d0.clone(), b0.clone(), e0.clone(), torch.zeros(nh, dtype=torch.float64, device=dev))
    for _ in range(args.warmup):
        mctx.step(*mstate, dt, 1)
    m_ms, m_launches = time_steps(mctx, mstate, dt, args.steps, flush, stream, world)
    m_ms = reduce_max(m_ms, world)
    m_steady, mkern = steady_and_kernels(mctx, smx, mstate, dt, args.steps, flush, stream)
    m_steady = reduce_max(m_steady, world)
    # the same mixed step with the dense line operators on the FP32 CUDA cores ((hi, lo) operator pairs)
    mctx.set_mode_kernel("simt")
    for _ in range(args.warmup):
        mctx.step(*mstate, dt, 1)
    s_ms, _ = time_steps(mctx, mstate, dt, args.steps, flush, stream, world)
    s_ms = reduce_max(s_ms, world)
    mctx.set_mode_kernel("auto")
    mctx.device_status()
    ctx.device_status()
    # the refined mixed form: one refinement sweep of each Kronecker solve with an FP64 residual
    rctx = smx.Context(P, NEL, eps=eps, mu=1.0, precision="mixed_refined").bind(dev)
    rctx.set_stream(stream)
    rstate = (d0.clone(), b0.clone(), e0.clone(), torch.zeros(nh, dtype=torch.float64, device=dev))
    for _ in range(args.warmup):
        rctx.step(*rstate, dt, 1)
    r_ms, r_launches = time_steps(rctx, rstate, dt, args.steps, flush, stream, world)
    r_ms = reduce_max(r_ms, world)
    _, rkern = steady_and_kernels(rctx, smx, rstate, dt, min(args.steps, 50), flush, stream)
    rctx.device_status()
    del rctx

    # ---- the other configurations and the batched one (rank 0 of a single-GPU run only)
    configs = batched = None
    s1 = None
    if world == 1 and not args.no_extra:
        configs = other_configs(smx, dev, stream, flush, max(20, min(args.steps, 200)))
        batched, bdts = batched_config(smx, dev, stream, 300)
        batched["refined"], _ = batched_config(smx, dev, stream, 300, precision="mixed_refined", dts=bdts)
        s1 = scheme1_comparison(smx, dev, stream, eps, 5, 2.0 * dt)
        s1["step_time_ratio_vs_scheme2"] = s1["ms_per_step"] / (total_ms / args.steps)
    clocks = sampler.stop()

    # ---- end to end through the host-buffer C call (copies inside the timed region)
    hd = state[0].cpu().pin_memory()
    hb = state[1].cpu().pin_memory()
    he = state[2].cpu().pin_memory()
    hh = state[3].cpu().pin_memory()
    ctx.step_host(hd, hb, he, hh, dt, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.step_host(hd, hb, he, hh, dt, 1)
    e2e_s = reduce_max(time.perf_counter() - t0, world)
    e2e = {"value": reduce_sum(dof * args.steps, world) / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": 8 * (2 * ne + nh), "d2h_bytes_per_step": 8 * (2 * ne + 2 * nh),
           "call": "smx_step_host (pinned host d, b, e in; d, b, e, h out; nsteps=1 per call)"}

    # ---- rooflines: every kernel function against its own roofs; the dominant one is the headline
    kfr, dom = kernel_rooflines(kern, peaks)
    mkfr, mdom = kernel_rooflines(mkern, peaks)
    step_bytes = STEP_BYTES_PER_DOF * dof
    step_hbm = {"bytes_per_step": step_bytes, "per_dof": STEP_BYTES_PER_DOF,
                "achieved_gbs": step_bytes / (total_ms / args.steps * 1e-3) / 1e9, "peak_gbs": peaks["hbm_gbs"]}
    step_hbm["frac"] = step_hbm["achieved_gbs"] / peaks["hbm_gbs"]

    out = None
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "line_operators": "auto: per star the kernel measured faster (digit-sliced tensor-core products or "
                                 "banded FP64 recurrences)",
               "config": workload_config(ne, nh), "gpu_launches": launches, "clocks": clocks, "e2e": e2e,
               "roofline": roofline_line(dom, peaks), "kernels_frac": kfr, "step_hbm": step_hbm,
               "kernels": kern,
               "steady_state": {"value": reduce_sum(dof * args.steps, world) / (steady_ms * 1e-3),
                                "ms_per_step": steady_ms / args.steps,
                                "note": "K steps in one smx_step call, no L2 flush (state L2-resident)"},
               "mixed": {"value": reduce_sum(dof * args.steps, world) / (m_ms * 1e-3), "unit": UNIT,
                         "ms_per_step": m_ms / args.steps, "dtype": "f32 data, operators exact to 31 bits (four-digit tensor-core products), f64 state",
                         "gpu_launches": m_launches, "roofline": roofline_line(mdom, peaks), "kernels_frac": mkfr,
                         "kernels": mkern, "line_operators": mctx.mode_kernel(),
                         "cuda_core_line_operators": {"value": reduce_sum(dof * args.steps, world) / (s_ms * 1e-3),
                                                      "ms_per_step": s_ms / args.steps,
                                                      "note": "same step, dense line operators on the FP32 CUDA "
                                                              "cores (operator as FP32 (hi, lo) pairs)"},
                         "speedup_vs_fp64": total_ms / m_ms,
                         "refined": {"value": reduce_sum(dof * args.steps, world) / (r_ms * 1e-3),
                                     "ms_per_step": r_ms / args.steps, "gpu_launches": r_launches,
                                     "dtype": "f32 operators, one refinement sweep per Kronecker solve with an "
                                              "f64 residual, f64 state and star outputs",
                                     "kernels_frac": kernel_rooflines(rkern, peaks)[0]},
                         "steady_state": {"value": reduce_sum(dof * args.steps, world) / (m_steady * 1e-3),
                                          "ms_per_step": m_steady / args.steps}}}
        if configs is not None:
            out["configs"] = configs
        if batched is not None:
            out["batched"] = batched
        if s1 is not None:
            out["scheme1"] = s1
    return out


def run_profile(form):
    """A few eager leapfrog steps of the benchmark workload, for profiler captures: one Hodge star
    and two single steps on the default stream (no CUDA graph, so ncu sees every launch).
    fp64 (default line operators), fp64-tc (every FP64 line operator on the tensor cores),
    fp64-banded (banded FP64 recurrences), mixed (default: four-digit tensor-core line operators),
    mixed-simt (FP32 CUDA-core line operators)."""
    import torch
    from paper_2302_04979_gb300 import smx, synth
    eps = ("blocks", synth.block_material(SEED, EPS_BLOCKS, 1.0, 9.0))
    prec = "mixed" if form.startswith("mixed") else "fp64"
    ctx = smx.Context(P, NEL, eps=eps, mu=1.0, precision=prec).bind()
    if form == "fp64-tc":
        ctx.set_mode_kernel("tensor")
    elif form in ("fp64-banded", "mixed-simt"):
        ctx.set_mode_kernel("simt")
    d, b, e, h = make_state(ctx, smx, "cuda", SEED + 1)
    for _ in range(2):
        ctx.step(d, b, e, h, 1e-3, 1)
    torch.cuda.synchronize()
    ctx.device_status()
    print(form, "ok", float(d.norm()))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the other configurations and the batched run")
    ap.add_argument("--profile", choices=["fp64", "fp64-tc", "fp64-banded", "mixed", "mixed-simt"])
    args = ap.parse_args()
    if args.profile:
        run_profile(args.profile)
        return
    if args.warmup < 3:
        args.warmup = 3
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local)
        init_dist(world)
    out = run_ours(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline()
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
