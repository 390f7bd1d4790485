"""Scheme 1 (mass-matrix Hodge stars, Sec. 3.3) on the GPU against the oracle's scheme 1
(oracle/scheme1.py, pinned by tests/test_oracle_scheme1.py): the Hodge stars, whole steps with a
source, the energy and the CFL limit, on the identity map with constant and block material and on
the curved sine-bump map with pointwise material; the CG iteration counts (one iteration where the
preconditioner is exact up to the material constant)."""
import numpy as np
import pytest

from oracle import hodge, scheme1
from paper_2302_04979_gb300 import synth
from tests.gpu_util import rel_l2, to_dev, to_host

pytestmark = pytest.mark.gpu

CASES = {
    "identity_const": dict(p=3, nel=(5, 4, 6), eps=2.5, mu=1.5),
    "identity_blocks": dict(p=(2, 3, 2), nel=(6, 4, 6), eps=("blocks", synth.block_material(21, (3, 2, 2), 1.0, 9.0)),
                            mu=1.0),
    "curved_pointwise": dict(p=2, nel=(4, 5, 4), geometry="sine_bump", eps=synth.GaussianBumps(22),
                             mu=lambda x, y, z: 1.0 + 0.5 * x * y),
    "p4_blocks": dict(p=4, nel=(4, 4, 4), eps=("blocks", synth.block_material(23, (2, 2, 2), 1.0, 4.0)), mu=2.0),
}


def _pair(case):
    from paper_2302_04979_gb300 import smx
    geom = hodge.SineBumpMap(0.05) if case.get("geometry") == "sine_bump" else None
    S = scheme1.Scheme1(case["p"], case["nel"], geometry=geom, eps=case["eps"], mu=case["mu"])
    ctx = smx.Context(case["p"], case["nel"], geometry=case.get("geometry", "identity"), amplitude=0.05,
                      eps=case["eps"], mu=case["mu"], scheme1=True).bind()
    return S, ctx


@pytest.mark.parametrize("name", sorted(CASES))
def test_scheme1_stars_match_oracle(name):
    import torch
    from paper_2302_04979_gb300 import smx
    S, ctx = _pair(CASES[name])
    d = synth.uniform(31, S.N_e, -1.0, 1.0)
    b = synth.uniform(32, S.N_h, -1.0, 1.0)
    e = torch.empty(S.N_e, dtype=torch.float64, device="cuda")
    h = torch.empty(S.N_h, dtype=torch.float64, device="cuda")
    it_e = ctx.scheme1_star(smx.FIELD_D, to_dev(d), e, tol=1e-13)
    it_h = ctx.scheme1_star(smx.FIELD_B, to_dev(b), h, tol=1e-13)
    ee, eh = rel_l2(to_host(e), S.e_from_d(d)), rel_l2(to_host(h), S.h_from_b(b))
    print("\n%s scheme-1 stars: rel L2 e %.2e (%d CG iterations) h %.2e (%d)" % (name, ee, it_e, eh, it_h))
    assert ee < 1e-11 and eh < 1e-11
    if name == "identity_const":
        assert it_e == 1 and it_h == 1   # the preconditioner is the mass up to the material constant
    else:
        assert it_e > 1


@pytest.mark.parametrize("name", sorted(CASES))
def test_scheme1_steps_match_oracle(name):
    import torch
    S, ctx = _pair(CASES[name])
    rng = np.random.default_rng(5)
    d = rng.standard_normal(S.N_e)
    b = S.D1 @ rng.standard_normal(S.N_e)
    e = S.e_from_d(d)
    dt = 0.5 * S.cfl(tol=1e-9)[0]
    n = 8
    jhat = synth.uniform(33, S.N_e, -1.0, 1.0)
    amps = synth.uniform(34, n, -1.0, 1.0)
    want = S.step(d, b, e, dt, n, jhat=jhat, amps=amps)
    st = [to_dev(d), to_dev(b), to_dev(e), torch.zeros(S.N_h, dtype=torch.float64, device="cuda")]
    iters = ctx.step_scheme1(*st, dt, n, jhat=to_dev(jhat), amp=to_dev(amps), tol=1e-13)
    errs = [rel_l2(to_host(g), w) for g, w in zip(st, want)]
    print("\n%s scheme 1, %d steps: rel L2 d %.2e b %.2e e %.2e h %.2e; max CG iterations %d" % (name, n, *errs, iters))
    assert max(errs) < 1e-10
    # energy with the pairing matrices (Sec. 3.3) against the oracle's mass-matrix form, at the
    # synchronised time (the step returns h at the half step: take the star of the final b)
    from paper_2302_04979_gb300 import smx
    hb = torch.empty_like(st[3])
    ctx.scheme1_star(smx.FIELD_B, st[1], hb, tol=1e-13)
    Eg = ctx.energy_scheme1(st[0], st[1], st[2], hb)
    Eo = S.energy(want[0], want[1])[0]
    assert abs(Eg - Eo) < 1e-10 * abs(Eo)


def test_scheme1_cfl_matches_oracle_and_exceeds_scheme2():
    """Sec. 5.2: the GPU power iteration gives the oracle's dt_max; at p = 4 it is larger than the
    scheme-2 limit of the same mesh (scheme 1 decays more slowly with p)."""
    case = CASES["p4_blocks"]
    S, ctx = _pair(case)
    dt_o = S.cfl(tol=1e-10)[0]
    dt_g = ctx.cfl_scheme1(iters=400, tol=1e-10)
    dt2 = ctx.cfl(iters=400, tol=1e-10)
    print("\np=4 4^3: scheme-1 dt_max %.6f (oracle %.6f), scheme-2 %.6f" % (dt_g, dt_o, dt2))
    assert abs(dt_g - dt_o) < 1e-6 * dt_o
    assert dt_g > 1.5 * dt2


def test_scheme1_requires_its_tables():
    import torch
    from paper_2302_04979_gb300 import smx
    ctx = smx.Context(2, 3).bind()
    x = torch.zeros(ctx.N_e, dtype=torch.float64, device="cuda")
    with pytest.raises(smx.SmxError) as err:
        ctx.scheme1_star(smx.FIELD_D, x, torch.empty_like(x))
    assert err.value.status == smx.ESTATE
