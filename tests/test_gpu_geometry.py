"""A general geometry map given by a host callback (SMX_GEOM_CALLBACK, Sec. 2.3) on the GPU: the
Hodge stars and leapfrog steps through the callback map against the oracle with the same map
(1e-11), the callback sine bump against the built-in one, and the refined mixed form on the
sheared domain (1e-5), and scheme 1 on the quarter coaxial cable (Sec. 5.1.2), whose polar map and
degree-2 NURBS patch both run through the callback."""
import numpy as np
import pytest

from oracle import maxwell as mx
from paper_2302_04979_gb300 import synth
from tests.gpu_util import rel_l2, to_dev, to_host

pytestmark = pytest.mark.gpu

MAPS = {"sine_bump": synth.SineBumpMap(0.05), "shear": synth.ShearMap(), "coax": synth.QuarterCoaxMap(),
        "coax_nurbs": synth.QuarterCoaxNURBS()}


def _case(name, p=3, nel=(6, 5, 7)):
    eps = synth.GaussianBumps(17)
    S = mx.Scheme2(p, nel, geometry=MAPS[name], eps=eps)
    d = synth.uniform(60, S.N_e, -1.0, 1.0)
    b = S.D1 @ synth.uniform(61, S.N_e, -1.0, 1.0)
    e = S.e_from_d(d)
    dt = 0.5 * S.cfl(tol=1e-8)[0]
    jhat = synth.uniform(62, S.N_e, -1.0, 1.0)
    amps = synth.uniform(63, 12, -1.0, 1.0)
    return S, eps, d, b, e, dt, jhat, amps


def _steps(ctx, S, d, b, e, dt, n, jhat, amps):
    import torch
    st = [to_dev(d), to_dev(b), to_dev(e), torch.zeros(S.N_h, dtype=torch.float64, device="cuda")]
    ctx.step(*st, dt, n, jhat=to_dev(jhat), amp=to_dev(amps))
    ctx.device_status()
    return [to_host(t) for t in st]


@pytest.mark.parametrize("name", sorted(MAPS))
def test_callback_map_stars_and_steps_match_oracle(name):
    import torch
    from paper_2302_04979_gb300 import smx
    S, eps, d, b, e, dt, jhat, amps = _case(name)
    ctx = smx.Context(3, (6, 5, 7), geometry=MAPS[name], eps=eps).bind()
    assert ctx.hodge_mode(smx.FIELD_D) == 1 and ctx.hodge_mode(smx.FIELD_B) == 1   # quadrature Hodge
    x = synth.uniform(64, S.N_e, -1.0, 1.0)
    y = synth.uniform(65, S.N_h, -1.0, 1.0)
    ed = torch.empty(S.N_e, dtype=torch.float64, device="cuda")
    hd = torch.empty(S.N_h, dtype=torch.float64, device="cuda")
    ctx.hodge_star(smx.FIELD_D, to_dev(x), ed)
    ctx.hodge_star(smx.FIELD_B, to_dev(y), hd)
    assert rel_l2(to_host(ed), S.e_from_d(x)) < 1e-11
    assert rel_l2(to_host(hd), S.h_from_b(y)) < 1e-11
    got = _steps(ctx, S, d, b, e, dt, 12, jhat, amps)
    want = S.step(d, b, e, dt, 12, jhat=jhat, amps=amps)
    errs = [rel_l2(g, w) for g, w in zip(got, want)]
    print("\n%s callback map, 12 steps vs oracle: rel L2 d %.2e b %.2e e %.2e h %.2e" % (name, *errs))
    assert max(errs) < 1e-11


def test_callback_sine_bump_equals_builtin():
    from paper_2302_04979_gb300 import smx
    S, eps, d, b, e, dt, jhat, amps = _case("sine_bump")
    a = smx.Context(3, (6, 5, 7), geometry=MAPS["sine_bump"], eps=eps).bind()
    c = smx.Context(3, (6, 5, 7), geometry="sine_bump", amplitude=0.05, eps=eps).bind()
    ga = _steps(a, S, d, b, e, dt, 12, jhat, amps)
    gc = _steps(c, S, d, b, e, dt, 12, jhat, amps)
    for u, v in zip(ga, gc):
        assert rel_l2(u, v) < 1e-13


def test_refined_mixed_on_sheared_domain():
    from paper_2302_04979_gb300 import smx
    S, eps, d, b, e, dt, jhat, amps = _case("shear")
    ctx = smx.Context(3, (6, 5, 7), geometry=MAPS["shear"], eps=eps, precision="mixed_refined").bind()
    got = _steps(ctx, S, d, b, e, dt, 12, jhat, amps)
    want = S.step(d, b, e, dt, 12, jhat=jhat, amps=amps)
    errs = [rel_l2(g, w) for g, w in zip(got, want)]
    print("\nshear map, refined mixed, 12 steps vs oracle: rel L2 d %.2e b %.2e e %.2e h %.2e" % tuple(errs))
    assert max(errs) < 1e-5


def test_scheme1_on_quarter_coax_matches_oracle():
    """Scheme 1 (mass-matrix Hodge stars) on the quarter coaxial cable through the callback map:
    the 1-form masses are not Kronecker products there, so every solve iterates."""
    import torch
    from oracle import scheme1
    from paper_2302_04979_gb300 import smx
    m = MAPS["coax"]
    S = scheme1.Scheme1(3, (4, 3, 4), geometry=m)
    ctx = smx.Context(3, (4, 3, 4), geometry=m, scheme1=True).bind()
    d = synth.uniform(70, S.N_e, -1.0, 1.0)
    b = S.D1 @ synth.uniform(71, S.N_e, -1.0, 1.0)
    e = S.e_from_d(d)
    dt = 0.5 * S.cfl(tol=1e-8)[0]
    want = S.step(d, b, e, dt, 6)
    st = [to_dev(d), to_dev(b), to_dev(e), torch.zeros(S.N_h, dtype=torch.float64, device="cuda")]
    iters = ctx.step_scheme1(*st, dt, 6, tol=1e-13)
    errs = [rel_l2(to_host(g), w) for g, w in zip(st, want)]
    print("\ncoax scheme 1, 6 steps vs oracle: rel L2 d %.2e b %.2e e %.2e h %.2e; max CG iterations %d" % (*errs, iters))
    assert max(errs) < 1e-10 and iters > 1
