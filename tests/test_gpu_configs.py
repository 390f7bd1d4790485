"""GPU against the oracle at the full sizes of the benchmark configurations.

* cube p=2, 8^3, TE_111 initial data, 100 steps at 0.5 x CFL: every field
  compared after all 100 steps (1e-11), W conserved, error to the exact mode;
* curved p=3, 32^3, Gaussian-bump permittivity, Gaussian-pulse current: every
  field after all 500 driven steps against the oracle (FP64 1e-11, both
  mixed forms 1e-5), and the discrete Gauss laws (D^2 b = 0, continuity for
  D~^2 d);
* p=3, 64^3, 8^3-block permittivity (the benchmark workload) and p=4, 64^3:
  every field against the oracle after 50 and 25 steps (the oracle needs
  seconds per step at this size), both mixed forms after 50 steps, then 1000
  GPU steps with W conserved to round-off.
The oracle trajectories are computed once per session and shared by the tests.
Inputs come from the seeded generators and the oracle (projections, CFL);
nothing expected is produced by the CUDA path.
"""
import numpy as np
import pytest

from oracle import forms3d, hodge, maxwell as mx
from paper_2302_04979_gb300 import synth
from tests.gpu_util import rel_l2, to_dev, to_host

pytestmark = pytest.mark.gpu


def _run_gpu(ctx, d, b, e, dt, nsteps, jhat=None, amps=None):
    import torch
    dd, bd, ed = to_dev(d), to_dev(b), to_dev(e)
    hd = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    ctx.step(dd, bd, ed, hd, dt, nsteps, jhat=None if jhat is None else to_dev(jhat),
             amp=None if amps is None else to_dev(amps))
    return dd, bd, ed, hd


def test_cube_p2_te111_100_steps():
    from paper_2302_04979_gb300 import smx
    S = mx.Scheme2(2, 8)
    ctx = smx.Context(2, 8).bind()
    d = S.project_2form("D", mx.te111_E(0.0))
    b = np.zeros(S.N_h)
    e = S.e_from_d(d)
    dt = 0.5 * S.cfl()[0]
    ref = S.step(d, b, e, dt, 100)
    got = _run_gpu(ctx, d, b, e, dt, 100)
    for g, w in zip(got, ref):
        assert rel_l2(to_host(g), w) < 1e-11
    E0, W0 = ctx.energy(to_dev(d), to_dev(b), to_dev(e), dt)
    E1, W1 = ctx.energy(got[0], got[1], got[2], dt)
    assert abs(W1 - W0) <= 1e-13 * W0
    assert abs(E0 - 0.125) < 5e-3          # discrete energy of the projected mode vs 1/2 int |E|^2 = 1/8
    T = 100 * dt
    err, nrm = S.l2_error("E", to_host(got[2]), mx.te111_E(T))
    assert err / nrm < 0.3                  # p=2 on 8^3: dispersion-dominated, loose by design


# ---------------------------------------------------------------- oracle trajectories (computed once)
_CACHE = {}


def _curved_case(nsteps):
    """Config 2: sine-bump map (0.05), p=3, 32^3, Gaussian-bump permittivity, Gaussian-pulse current
    projected by the oracle, dt = 0.003 (about 0.5 x CFL), zero initial fields; the oracle's fields
    after nsteps steps (computed once per session)."""
    key = ("curved", nsteps)
    if key not in _CACHE:
        bumps = synth.GaussianBumps(2302)
        S = mx.Scheme2(3, 32, geometry=hodge.SineBumpMap(0.05), eps=bumps)
        jhat = S.project_2form("D", synth.pulse_profile(synth.pulse_centre(2302), 0.05), rtol=1e-10)
        d, b, e = np.zeros(S.N_e), np.zeros(S.N_h), np.zeros(S.N_e)
        dt = 0.003
        amps = synth.source_amplitudes(dt, nsteps, f0=1.0, tau=0.25, t0=0.75)
        ref = S.step(d, b, e, dt, nsteps, jhat=jhat, amps=amps)
        _CACHE[key] = dict(S=S, bumps=bumps, jhat=jhat, d=d, b=b, e=e, dt=dt, amps=amps, ref=ref)
    return _CACHE[key]


CURVED_STEPS = 500


@pytest.mark.slow
def test_curved_p3_32cube_pulse():
    """FP64 against the oracle after all 500 driven steps (1e-11), and the discrete Gauss laws
    (D^2 b = 0; continuity for D~^2 d) on the GPU fields."""
    from paper_2302_04979_gb300 import smx
    c = _curved_case(CURVED_STEPS)
    S, dt, amps = c["S"], c["dt"], c["amps"]
    ctx = smx.Context(3, 32, geometry="sine_bump", amplitude=0.05, eps=c["bumps"]).bind()
    got = _run_gpu(ctx, c["d"], c["b"], c["e"], dt, CURVED_STEPS, jhat=c["jhat"], amps=amps)
    errs = [rel_l2(to_host(g), w) for g, w in zip(got, c["ref"])]
    print("\ncurved 32^3 FP64 vs oracle after %d steps: rel L2 d %.2e b %.2e e %.2e h %.2e" % (CURVED_STEPS, *errs))
    assert max(errs) < 1e-11
    D2, Dt2 = forms3d.div_matrix("B", S.p, S.nel), forms3d.div_matrix("D", S.p, S.nel)
    dn, bn = to_host(got[0]), to_host(got[1])
    scale = np.abs(dn).max()
    assert scale > 0
    assert np.abs(D2 @ bn).max() <= 1e-12 * max(np.abs(bn).max(), 1.0)
    expected = -dt * amps.sum() * (Dt2 @ c["jhat"])
    assert np.abs(Dt2 @ dn - expected).max() <= 1e-11 * max(np.abs(expected).max(), scale)


@pytest.mark.slow
@pytest.mark.parametrize("precision", ["mixed_refined", "mixed"])
def test_curved_p3_32cube_pulse_mixed(precision):
    """Config 2 in both mixed forms against the FP64 oracle after all 500 driven steps, with the
    drift of W (evaluated in FP64) stated.  The refined form (one refinement sweep of each
    Kronecker solve with an FP64 residual, FP64 star outputs) and the plain form (FP32 star outputs,
    no refinement), both with their default line operators (four-digit tensor-core products), meet
    the 1e-5 contract (measured 4.6e-6 and 5.3e-6).  With the FP32 CUDA-core line operators instead,
    the plain form reached 1.3e-5 on the electric 1-form here."""
    from paper_2302_04979_gb300 import smx
    c = _curved_case(CURVED_STEPS)
    S, dt = c["S"], c["dt"]
    ctx = smx.Context(3, 32, geometry="sine_bump", amplitude=0.05, eps=c["bumps"], precision=precision).bind()
    got = _run_gpu(ctx, c["d"], c["b"], c["e"], dt, CURVED_STEPS, jhat=c["jhat"], amps=c["amps"])
    errs = [rel_l2(to_host(g), w) for g, w in zip(got, c["ref"])]
    W_ref = S.energy(*c["ref"][:3], dt)[1]
    W_got = S.energy(to_host(got[0]), to_host(got[1]), to_host(got[2]), dt)[1]
    print("\ncurved 32^3 %s vs oracle after %d steps: rel L2 d %.2e b %.2e e %.2e h %.2e; W %.9e vs %.9e (rel %.2e)"
          % (precision, CURVED_STEPS, *errs, W_got, W_ref, abs(W_got - W_ref) / abs(W_ref)))
    assert max(errs) < 1e-5
    D2 = forms3d.div_matrix("B", S.p, S.nel)
    bn = to_host(got[1])
    assert np.abs(D2 @ bn).max() <= 1e-6 * max(np.abs(bn).max(), 1.0)


def _big_case(p, nsteps):
    """The benchmark workload (p=3) and config 3 (p=4): 64^3, permittivity on 8^3 seeded blocks in
    [1, 9), random d, divergence-free random b; the oracle's fields after nsteps steps."""
    key = ("big", p, nsteps)
    if key not in _CACHE:
        eps = ("blocks", synth.block_material(2302, (8, 8, 8), 1.0, 9.0))
        S = mx.Scheme2(p, 64, eps=eps)
        d = synth.uniform(2303, S.N_e, -1.0, 1.0)
        b = S.D1 @ synth.uniform(2304, S.N_e, -1.0, 1.0)
        e = S.e_from_d(d)
        # about 0.55 x CFL: the oracle's CFL at 16^3 is 0.0145 (p=3) and 0.0086 (p=4), linear in h
        dt = 2e-3 if p == 3 else 1.2e-3
        ref = S.step(d, b, e, dt, nsteps)
        _CACHE[key] = dict(S=S, eps=eps, d=d, b=b, e=e, dt=dt, ref=ref)
    return _CACHE[key]


BIG_STEPS = {3: 50, 4: 25}


@pytest.mark.slow
@pytest.mark.parametrize("p", [3, 4])
def test_64cube_block_eps(p):
    """Every field against the oracle after 50 (p=3, the benchmark workload) and 25 (p=4) steps
    (1e-11), with the default line operators and with the banded recurrences; then 1000 GPU steps
    with W conserved to round-off."""
    from paper_2302_04979_gb300 import smx
    n = BIG_STEPS[p]
    c = _big_case(p, n)
    ctx = smx.Context(p, 64, eps=c["eps"]).bind()
    for kernel in ("auto", "simt"):
        ctx.set_mode_kernel(kernel)
        got = _run_gpu(ctx, c["d"], c["b"], c["e"], c["dt"], n)
        errs = [rel_l2(to_host(g), w) for g, w in zip(got, c["ref"])]
        print("\n64^3 p=%d FP64 (%s) vs oracle after %d steps: rel L2 d %.2e b %.2e e %.2e h %.2e"
              % (p, kernel, n, *errs))
        assert max(errs) < 1e-11
    ctx.set_mode_kernel("auto")
    d, b, e, dt = c["d"], c["b"], c["e"], c["dt"]
    E0, W0 = ctx.energy(to_dev(d), to_dev(b), to_dev(e), dt)
    got = _run_gpu(ctx, d, b, e, dt, 1000)
    E1, W1 = ctx.energy(got[0], got[1], got[2], dt)
    assert abs(W1 - W0) <= 1e-12 * W0
    assert np.isfinite(E1) and E1 < 10 * E0


@pytest.mark.slow
@pytest.mark.parametrize("precision", ["mixed", "mixed_refined"])
def test_64cube_mixed_against_oracle(precision):
    """The benchmark workload in both mixed forms against the oracle after 50 steps (1e-5), W drift
    (in FP64) stated."""
    from paper_2302_04979_gb300 import smx
    n = BIG_STEPS[3]
    c = _big_case(3, n)
    ctx = smx.Context(3, 64, eps=c["eps"], precision=precision).bind()
    got = _run_gpu(ctx, c["d"], c["b"], c["e"], c["dt"], n)
    errs = [rel_l2(to_host(g), w) for g, w in zip(got, c["ref"])]
    S = c["S"]
    W0 = S.energy(c["d"], c["b"], c["e"], c["dt"])[1]
    W1 = S.energy(to_host(got[0]), to_host(got[1]), to_host(got[2]), c["dt"])[1]
    print("\n64^3 p=3 %s vs oracle after %d steps: rel L2 d %.2e b %.2e e %.2e h %.2e; W drift %.2e"
          % (precision, n, *errs, abs(W1 - W0) / W0))
    assert max(errs) < 1e-5
