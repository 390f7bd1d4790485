"""A few leapfrog steps of the benchmark workload, for profiler captures.

p = 3, 64^3 elements, identity map, permittivity on a seeded 8^3 block grid,
mu = 1; one Hodge star and two single steps per form, kernels launched
eagerly on the default stream (no CUDA graph), so ncu sees every launch.
"mixed" uses the default (FP32 CUDA-core) line operators, "mixed-tc" the
tensor-core ones; "fp64-tc" the FP64 form with the digit-sliced tensor-core
line operators, "fp64-banded" the FP64 line recurrences.

  python paper_2302_04979_gb300/probe/step_driver.py [fp64|fp64-tc|fp64-banded|mixed|mixed-tc|both]
"""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))


def main(forms):
    import torch
    from paper_2302_04979_gb300 import smx, synth
    eps = ("blocks", synth.block_material(2302, (8, 8, 8), 1.0, 9.0))
    for form in forms:
        prec = "mixed" if form.startswith("mixed") else "fp64"
        ctx = smx.Context(3, 64, eps=eps, mu=1.0, precision=prec).bind()
        if form in ("mixed-tc", "fp64-tc"):
            ctx.set_mode_kernel("tensor")
        elif form == "fp64-banded":
            ctx.set_mode_kernel("simt")
        d = torch.as_tensor(synth.uniform(1, ctx.N_e, -1.0, 1.0)).cuda()
        b = torch.zeros(ctx.N_h, dtype=torch.float64, device="cuda")
        e = torch.empty_like(d)
        h = torch.zeros_like(b)
        ctx.hodge_star(smx.FIELD_D, d, e)
        for _ in range(2):
            ctx.step(d, b, e, h, 1e-3, 1)
        torch.cuda.synchronize()
        print(form, "ok", float(d.norm()))


if __name__ == "__main__":
    arg = sys.argv[1] if len(sys.argv) > 1 else "both"
    main(["fp64", "mixed"] if arg == "both" else [arg])
