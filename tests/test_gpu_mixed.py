"""Mixed-precision leapfrog (FP32 operators, FP64 state) against the FP64 oracle.

The contract for this form is a relative L2 error of at most 1e-5 per field
against the FP64 oracle after the stated step count, with the drift of the
conserved energy W stated.  The errors measured here are printed (pytest -s)
and asserted against that bound.  Both mixed forms are covered: "mixed" (FP32
stars) and "mixed_refined" (each Kronecker solve refined once with an FP64
residual, FP64 star outputs); the refined star must also be markedly closer.
"""
import numpy as np
import pytest

from oracle import hodge
from oracle import maxwell as mx
from paper_2302_04979_gb300 import synth
from tests.gpu_util import rel_l2, to_dev, to_host

pytestmark = pytest.mark.gpu

CASES = {
    "cube_p2_te111": dict(p=2, nel=8, steps=100, init="te111"),
    "p3_blocks_ragged": dict(p=3, nel=(12, 9, 10), eps=("blocks", synth.block_material(3, (3, 3, 2), 1.0, 9.0)),
                             mu=1.5, steps=60, init="random"),
    "p4_aniso_elementwise": dict(p=(4, 3, 2), nel=(10, 7, 9), eps=2.0,
                                 mu=("blocks", synth.block_material(4, (10, 7, 9), 1.0, 4.0)), steps=40,
                                 init="random"),
    # lines longer than the dense mode-product limit (80): the banded FP32 line recurrences run instead
    "p2_long_lines": dict(p=2, nel=(90, 4, 3), eps=("blocks", synth.block_material(6, (3, 2, 1), 1.0, 4.0)),
                          steps=40, init="random"),
    # curved map and pointwise material: the FP32 quadrature Hodge
    "p3_curved_bumps": dict(p=3, nel=(6, 5, 7), geometry="sine_bump", eps=synth.GaussianBumps(5), steps=40,
                            init="random"),
    "p2_pointwise": dict(p=2, nel=(7, 6, 5), eps=lambda x, y, z: 1.0 + x + 0.5 * y * z,
                         mu=lambda x, y, z: 2.0 - 0.5 * z, steps=40, init="random"),
}


def _scheme(case):
    geom = hodge.SineBumpMap(0.05) if case.get("geometry") == "sine_bump" else hodge.IdentityMap()
    return mx.Scheme2(case["p"], case["nel"], geometry=geom, eps=case.get("eps", 1.0), mu=case.get("mu", 1.0))


def _context(smx, case, precision="mixed"):
    return smx.Context(case["p"], case["nel"], geometry=case.get("geometry", "identity"), eps=case.get("eps", 1.0),
                       mu=case.get("mu", 1.0), precision=precision).bind()


PRECISIONS = ("mixed", "mixed_refined")


def _setup(case):
    S = _scheme(case)
    if case["init"] == "te111":
        d = S.project_2form("D", mx.te111_E(0.0))
        b = np.zeros(S.N_h)
    else:
        d = synth.uniform(70, S.N_e, -1.0, 1.0)
        b = S.D1 @ synth.uniform(71, S.N_e, -1.0, 1.0)
    e = S.e_from_d(d)
    dt = 0.5 * S.cfl(tol=1e-8)[0]
    return S, d, b, e, dt


KERNELS = ("tensor", "simt")


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("name", sorted(CASES))
def test_mixed_against_oracle(name, kernel, precision):
    import torch
    from paper_2302_04979_gb300 import smx
    case = CASES[name]
    S, d, b, e, dt = _setup(case)
    n = case["steps"]
    ref = S.step(d, b, e, dt, n)
    ctx = _context(smx, case, precision)
    ctx.set_mode_kernel(kernel)
    dd, bd, ed = to_dev(d), to_dev(b), to_dev(e)
    hd = torch.zeros(S.N_h, dtype=torch.float64, device="cuda")
    ctx.step(dd, bd, ed, hd, dt, n)
    ctx.device_status()
    errs = [rel_l2(to_host(g), w) for g, w in zip((dd, bd, ed, hd), ref)]
    W0 = S.energy(d, b, e, dt)[1]
    W1 = S.energy(to_host(dd), to_host(bd), to_host(ed), dt)[1]
    print("\n%s %s (%s) after %d steps: rel L2 d %.2e b %.2e e %.2e h %.2e; W drift %.2e"
          % (name, precision, kernel, n, *errs, abs(W1 - W0) / W0))
    assert max(errs) < 1e-5
    assert abs(W1 - W0) / W0 < 1e-5


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("name", sorted(CASES))
def test_mixed_hodge_star_against_oracle(name, kernel, precision):
    """One mixed-precision Hodge star (K_1^{-1} M~ d and K~_1^{-1} M b) against the oracle's FP64 one.

    Every stage rounds its data to FP32 once (the CUDA-core operators carry FP64 accuracy in
    their (hi, lo) terms; the tensor-core digit products are exact on 31-bit fixed-point lines
    and round once), so one star stays within a few FP32 roundings: 2e-6.  The refined star
    removes the solve's rounding (FP64 residual, one FP32 correction, FP64 output); what is
    left is the FP32 arithmetic of the mass apply: 1e-6 (5e-8 to 5e-7 measured)."""
    import torch
    from paper_2302_04979_gb300 import smx
    case = CASES[name]
    S = _scheme(case)
    d = synth.uniform(80, S.N_e, -1.0, 1.0)
    b = synth.uniform(81, S.N_h, -1.0, 1.0)
    ctx = _context(smx, case, precision)
    ctx.set_mode_kernel(kernel)
    e_dev = torch.empty(S.N_e, dtype=torch.float64, device="cuda")
    h_dev = torch.empty(S.N_h, dtype=torch.float64, device="cuda")
    ctx.hodge_star_mixed(smx.FIELD_D, to_dev(d), e_dev)
    ctx.hodge_star_mixed(smx.FIELD_B, to_dev(b), h_dev)
    ctx.device_status()
    ee, eh = rel_l2(to_host(e_dev), S.e_from_d(d)), rel_l2(to_host(h_dev), S.h_from_b(b))
    print("\n%s %s star (%s): rel L2 e %.2e h %.2e" % (name, precision, kernel, ee, eh))
    bound = 1e-6 if precision == "mixed_refined" else 2e-6
    assert ee < bound and eh < bound


def test_mixed_kernels_agree_at_64cube():
    """The benchmark workload's mixed Hodge stars: tensor-core (four-digit) and FP32 CUDA-core kernels
    agree to FP32 rounding."""
    import torch
    from paper_2302_04979_gb300 import smx
    eps = ("blocks", synth.block_material(2302, (8, 8, 8), 1.0, 9.0))
    ctx = smx.Context(3, 64, eps=eps, precision="mixed").bind()
    d = to_dev(synth.uniform(82, ctx.N_e, -1.0, 1.0))
    b = to_dev(synth.uniform(83, ctx.N_h, -1.0, 1.0))
    out = {}
    for kernel in KERNELS:
        ctx.set_mode_kernel(kernel)
        e = torch.empty(ctx.N_e, dtype=torch.float64, device="cuda")
        h = torch.empty(ctx.N_h, dtype=torch.float64, device="cuda")
        ctx.hodge_star_mixed(smx.FIELD_D, d, e)
        ctx.hodge_star_mixed(smx.FIELD_B, b, h)
        ctx.device_status()
        out[kernel] = (to_host(e), to_host(h))
    de = rel_l2(out["tensor"][0], out["simt"][0])
    dh = rel_l2(out["tensor"][1], out["simt"][1])
    print("\n64^3 mixed star, tensor vs simt: rel L2 e %.2e h %.2e" % (de, dh))
    assert de < 1e-6 and dh < 1e-6


def test_mixed_star_requires_mixed_context():
    import torch
    from paper_2302_04979_gb300 import smx
    ctx = smx.Context(2, 4).bind()
    x = torch.zeros(ctx.N_e, dtype=torch.float64, device="cuda")
    with pytest.raises(smx.SmxError) as ei:
        ctx.hodge_star_mixed(smx.FIELD_D, x, x.clone())
    assert ei.value.status == smx.ESTATE


@pytest.mark.slow
def test_mixed_64cube_against_oracle():
    """The benchmark workload: 2 steps against the oracle, then W drift over 1000 GPU steps."""
    import torch
    from paper_2302_04979_gb300 import smx
    eps = ("blocks", synth.block_material(2302, (8, 8, 8), 1.0, 9.0))
    S = mx.Scheme2(3, 64, eps=eps)
    d = synth.uniform(2303, S.N_e, -1.0, 1.0)
    b = S.D1 @ synth.uniform(2304, S.N_e, -1.0, 1.0)
    e = S.e_from_d(d)
    dt = 2e-3
    ref = S.step(d, b, e, dt, 2)
    ctx = smx.Context(3, 64, eps=eps, precision="mixed").bind()
    dd, bd, ed = to_dev(d), to_dev(b), to_dev(e)
    hd = torch.zeros(S.N_h, dtype=torch.float64, device="cuda")
    ctx.step(dd, bd, ed, hd, dt, 2)
    errs = [rel_l2(to_host(g), w) for g, w in zip((dd, bd, ed, hd), ref)]
    print("\n64^3 mixed after 2 steps: rel L2 d %.2e b %.2e e %.2e h %.2e" % tuple(errs))
    assert max(errs) < 1e-5
    ctx64 = smx.Context(3, 64, eps=eps).bind()   # FP64 energy of the mixed trajectory
    W0 = ctx64.energy(to_dev(d), to_dev(b), to_dev(e), dt)[1]
    dd, bd, ed = to_dev(d), to_dev(b), to_dev(e)
    ctx.step(dd, bd, ed, hd, dt, 1000)
    W1 = ctx64.energy(dd, bd, ed, dt)[1]
    print("64^3 mixed: W drift over 1000 steps %.2e" % (abs(W1 - W0) / W0))
    assert abs(W1 - W0) / W0 < 1e-4
