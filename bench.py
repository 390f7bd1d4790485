#!/usr/bin/env python3
"""Leapfrog throughput of scheme 2 (arXiv 2302.04979) on one GB300, in DoF-steps/s.

Workload: unit-cube PEC cavity, identity map, spline degree p = 3, 64^3
elements (N_e + N_h = 1,685,970 degrees of freedom), permittivity piecewise
constant on a seeded 8^3 grid of element blocks (uniform in [1, 9)), mu = 1,
seeded random initial D, divergence-free random B, J = 0, dt = 0.5 x the CFL
limit.  One step = one full kick-drift-kick leapfrog step (curl, Hodge apply,
pairing solve for both fields) in FP64.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
(the slow, plain implementation the tests check against) on the host cores.
For N > 1 (torchrun) every rank runs its own independent cavity (replicas, no
collective in the data path); value = all ranks' DoF-steps / max rank time.
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
# GB300 FP64 CUDA-core peak from unit counts and clock: 152 SMs x 2 DFMA lanes/clk x 2 flop x 2.07 GHz
# (the nominal 1.25 TFLOP/s; the repository's FMA probe measures 1.19)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
L2_FLUSH_BYTES = 256 << 20


def workload_config(ne, nh, extra=None):
    cfg = {"workload": "PEC cavity, identity map, p=3, 64^3 elements, eps 8^3 blocks U[1,9), mu=1",
           "p": P, "nel": [NEL] * 3, "N_e": ne, "N_h": nh, "dof": ne + nh,
           "initial": "seeded random d, divergence-free random b, J=0", "dt": "0.5 x CFL",
           "l2": "flushed between timed steps (256 MiB write)", "parallelism": "replicas"}
    if extra:
        cfg.update(extra)
    return cfg


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


def job_rate(units_this_rank, seconds_this_rank, world):
    """Whole-job throughput: all ranks' units / the slowest rank's time (max over ranks)."""
    return reduce_sum(units_this_rank, world) / reduce_max(seconds_this_rank, world)


def init_dist(world):
    """One process per GPU: NCCL when CUDA is present, gloo otherwise (CPU runs of the host logic)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")


def reduce_sum(value, world):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


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


def threads_used():
    try:
        from threadpoolctl import threadpool_info
        n = max((i.get("num_threads", 1) for i in threadpool_info()), default=1)
        return int(n)
    except Exception:
        return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def time_oracle(nsteps_max, budget_s, warmup=1):
    """Oracle leapfrog on the full workload: (DoF-steps/s, steps timed, seconds)."""
    S, d, b, e = oracle_setup()
    dt = 1e-3
    for _ in range(warmup):
        d, b, e, _ = S.step(d, b, e, dt, 1)
    t0 = time.perf_counter()
    n = 0
    while n < nsteps_max:
        d, b, e, _ = S.step(d, b, e, dt, 1)
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    return (S.N_e + S.N_h) * n / el, n, el, S.N_e, S.N_h


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def run_reference(args, rank, world):
    if rank != 0:
        return
    rate, n, el, ne, nh = time_oracle(args.steps, budget_s=120.0, warmup=min(args.warmup, 1))
    cores = threads_used()
    sample = ("%d of the %d requested steps on the full 64^3 workload (%.1f s), warm-up %d; host %s, %d cpus"
              % (n, args.steps, el, min(args.warmup, 1), cpu_model(), os.cpu_count() or 0))
    out = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / n, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(ne, nh),
           "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ GPU arm
HBM_PEAK_GBS = 6793.1   # MEASURED_PEAKS.json hbm_gbs (copy bandwidth)
BF16_PEAK_TFLOPS = 1992.0  # MEASURED_PEAKS.json bf16_tflops (cuBLAS burst)
DIGIT_PAIRS = 28           # digit products (levels 0..6 of seven digits) per FP64 dense line product

# DRAM bytes (read + write) per launch from one ncu capture of each kernel at this
# workload (profiles/fp64_step_p3_64cube.md, profiles/mixed_step_p3_64cube.md,
# profiles/digit_line_p3_64cube.md; cold caches, outputs stay in L2).  Kept only while
# the kernel is unchanged since the capture.
NCU_TRAFFIC = {
    "mass_solve_x": 6.90e6, "mass_solve_y": 6.90e6, "mass_solve_z": 6.90e6,
    "solve_x": 6.72e6, "solve_y": 6.72e6, "solve_z": 6.72e6,
    "hodge_block": 13.51e6,
    # mixed step, CUDA-core line operators (x passes read FP64 input)
    "line_f32_x": 6.93e6, "line_f32_y": 3.56e6, "line_f32_z": 3.56e6,
    "hodge_block_f32": 13.51e6,
    # FP64 line operators on the tensor cores (profiles/digit_line_p3_64cube.md)
    "line_f64tc_x": 7.15e6, "line_f64tc_y": 7.15e6, "line_f64tc_z": 7.15e6,
}


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
              "line_f32_x": both, "line_f32_y": both, "line_f32_z": both,
              "line_f64tc_x": both, "line_f64tc_y": both, "line_f64tc_z": both}
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
                      "fp64_tflops": fl / (avg_ms * 1e-3) / 1e12, "gbs": by / (avg_ms * 1e-3) / 1e9,
                      "flops_per_launch": fl, "bytes_per_launch": by}
    total_k = sum(v["total_ms"] for v in kern.values())
    for v in kern.values():
        v["share"] = v["total_ms"] / total_k if total_k else None
    return kern


def time_steps(ctx, state, dt, steps, flush, stream, world):
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
        ctx.step(d, b, e, h, dt, 1)
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


def run_ours(args, rank, world, local):
    import torch
    from paper_2302_04979_gb300 import smx, synth

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (there is no CPU fallback)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    eps = ("blocks", synth.block_material(SEED, EPS_BLOCKS, 1.0, 9.0))
    ctx = smx.Context(P, NEL, eps=eps, mu=1.0).bind(dev)
    stream = torch.cuda.Stream(device=dev)   # non-default: smx_step replays a captured CUDA graph
    torch.cuda.set_stream(stream)
    ctx.set_stream(stream)
    ne, nh = ctx.N_e, ctx.N_h
    dof = ne + nh
    d0 = torch.as_tensor(synth.uniform(SEED + 1 + 17 * rank, ne, -1.0, 1.0)).to(dev)
    b0 = torch.zeros(nh, dtype=torch.float64, device=dev)
    ctx.curl_primal(torch.as_tensor(synth.uniform(SEED + 2 + 17 * rank, ne, -1.0, 1.0)).to(dev), b0, 1.0)
    e0 = torch.empty(ne, dtype=torch.float64, device=dev)
    ctx.hodge_star(smx.FIELD_D, d0, e0)
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
    # the same mixed step with the dense line operators on the tensor cores (exact four-digit slicing)
    mctx.set_mode_kernel("tensor")
    for _ in range(args.warmup):
        mctx.step(*mstate, dt, 1)
    s_ms, _ = time_steps(mctx, mstate, dt, args.steps, flush, stream, world)
    s_ms = reduce_max(s_ms, world)
    mctx.set_mode_kernel("simt")
    mctx.device_status()
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

    # ---- roofline of the dominant kernel: the FP64 kernels are bound by the FP64 pipe; the
    # digit-sliced line operators by the BF16 tensor pipe (28 digit products of 2 n flops per entry)
    dom = max(kern, key=lambda n: kern[n]["total_ms"])
    if dom.startswith("line_f64tc"):
        tc = DIGIT_PAIRS * kern[dom]["fp64_tflops"]
        roof = {"kernel": dom, "bound": "tensor", "achieved": tc, "peak": BF16_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": tc / BF16_PEAK_TFLOPS, "traffic": NCU_TRAFFIC.get(dom),
                "peak_source": "MEASURED_PEAKS.json bf16_tflops (of measured, burst)",
                "work": "28 BF16 digit products x 2 n flops per line entry (no padding counted)",
                "fp64_equivalent_tflops": kern[dom]["fp64_tflops"], "hbm_gbs": kern[dom]["gbs"]}
    else:
        roof = {"kernel": dom, "bound": "alu", "achieved": kern[dom]["fp64_tflops"], "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": kern[dom]["fp64_tflops"] / FP64_PEAK_TFLOPS,
                "traffic": NCU_TRAFFIC.get(dom),
                "peak_source": "FP64 unit count x clock (152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz); "
                               "MEASURED_PEAKS.json has no FP64 entry; the FMA probe measured 1.19 TFLOP/s",
                "hbm_gbs": kern[dom]["gbs"]}
    mdom = max(mkern, key=lambda n: mkern[n]["total_ms"])
    mroof = {"kernel": mdom, "bound": "hbm", "achieved": mkern[mdom]["gbs"], "peak": HBM_PEAK_GBS, "unit": "GB/s",
             "frac": mkern[mdom]["gbs"] / HBM_PEAK_GBS, "traffic": NCU_TRAFFIC.get(mdom),
             "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}

    out = None
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "line_operators": "auto: at this size the separable star of B on the tensor cores (exact BF16 "
                                 "digit products), the sweeps after the block Hodge apply of D as FP64 banded "
                                 "recurrences",
               "config": workload_config(ne, nh), "gpu_launches": launches, "clocks": clocks, "e2e": e2e,
               "roofline": roof, "kernels": kern,
               "steady_state": {"value": reduce_sum(dof * args.steps, world) / (steady_ms * 1e-3),
                                "ms_per_step": steady_ms / args.steps,
                                "note": "K steps in one smx_step call, no L2 flush (state L2-resident)"},
               "mixed": {"value": reduce_sum(dof * args.steps, world) / (m_ms * 1e-3), "unit": UNIT,
                         "ms_per_step": m_ms / args.steps, "dtype": "f32 operators (split coefficients), f64 state",
                         "gpu_launches": m_launches, "roofline": mroof, "kernels": mkern,
                         "line_operators": "FP32 CUDA cores, (hi, lo) operator coefficients",
                         "tensor_line_operators": {"value": reduce_sum(dof * args.steps, world) / (s_ms * 1e-3),
                                                   "ms_per_step": s_ms / args.steps,
                                                   "note": "same step, dense line operators on the tcgen05 tensor "
                                                           "cores (exact four-digit slicing, one FP32 rounding)"},
                         "speedup_vs_fp64": total_ms / m_ms,
                         "steady_state": {"value": reduce_sum(dof * args.steps, world) / (m_steady * 1e-3),
                                          "ms_per_step": m_steady / args.steps}}}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
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
            rate, n, el, _, _ = time_oracle(3, budget_s=25.0, warmup=0)
            out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads_used(), "kind": "oracle",
                                   "sample": "%d full 64^3 leapfrog steps of the FP64 oracle (%.1f s) on %s"
                                             % (n, el, cpu_model())}
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
