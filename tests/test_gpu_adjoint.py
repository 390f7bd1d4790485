"""Reverse mode on the GPU (smx_step_adjoint behind torch.autograd) against the oracle's
discrete adjoint (oracle/adjoint.py, itself pinned by finite differences), and against
central finite differences of the GPU loss at the full adjoint configuration."""
import numpy as np
import pytest

from oracle import adjoint, hodge, maxwell
from paper_2302_04979_gb300 import synth
from tests.gpu_util import rel_l2

pytestmark = pytest.mark.gpu


def _small(geometry):
    p, nel, blocks, nsteps = 2, (4, 4, 6), (2, 2, 3), 6
    geom = hodge.SineBumpMap(0.05) if geometry == "sine_bump" else None
    S0 = maxwell.Scheme2(p, nel, geometry=geom)
    xr = synth.uniform(90, 9, 0.05, 0.95).reshape(3, 3)
    jhat = synth.uniform(91, S0.N_e, -1.0, 1.0)
    d0 = synth.uniform(92, S0.N_e, -1.0, 1.0)
    b0 = S0.D1 @ synth.uniform(93, S0.N_e, -1.0, 1.0)
    eps = synth.uniform(94, int(np.prod(blocks)), 1.0, 4.0).reshape(blocks[::-1])
    dt = 0.4 * S0.cfl(tol=1e-8)[0]
    amps = synth.uniform(95, nsteps, -1.0, 1.0)
    P = adjoint.MisfitProblem(p, nel, geom, eps, 1.0, jhat, adjoint.Receivers(p, nel, xr), dt, nsteps, d0, b0)
    obs = P.forward(eps * (1.0 + 0.1 * synth.uniform(96, eps.size, -1.0, 1.0).reshape(eps.shape)), amps)[3]
    return dict(p=p, nel=nel, geometry=geometry, eps=eps, xr=xr, d0=d0, b0=b0, jhat=jhat, dt=dt, nsteps=nsteps,
                amps=amps, obs=obs, P=P)


def _gpu_grad(case, checkpoint_every=None, precision="fp64"):
    import torch
    from paper_2302_04979_gb300 import adjoint as gadj
    prob = gadj.LeapfrogProblem(case["p"], case["nel"], case["eps"], case["xr"], case["d0"], case["b0"], case["jhat"],
                                case["dt"], case["nsteps"], geometry=case["geometry"], precision=precision)
    if checkpoint_every:
        prob.k = checkpoint_every
    eps_t = torch.tensor(case["eps"], dtype=torch.float64, requires_grad=True)
    amps_t = torch.tensor(case["amps"], dtype=torch.float64, device="cuda", requires_grad=True)
    obs = torch.as_tensor(case["obs"]).cuda()
    traces = gadj.LeapfrogTraces.apply(eps_t, amps_t, prob)
    loss = gadj.misfit(traces, obs, case["dt"])
    loss.backward()
    return float(loss), eps_t.grad.numpy(), amps_t.grad.cpu().numpy(), prob


@pytest.mark.parametrize("geometry", ["identity", "sine_bump"])
def test_gradient_matches_oracle(geometry):
    case = _small(geometry)
    loss_ref, geps_ref, gamp_ref = case["P"].gradient(case["eps"], case["amps"], case["obs"])
    loss, geps, gamp, _ = _gpu_grad(case)
    print("\n%s: loss %.6e vs %.6e; rel L2 grad eps %.2e, amps %.2e"
          % (geometry, loss, loss_ref, rel_l2(geps, geps_ref), rel_l2(gamp, gamp_ref)))
    assert abs(loss - loss_ref) <= 1e-11 * loss_ref
    assert rel_l2(geps, geps_ref) < 1e-10
    assert rel_l2(gamp, gamp_ref) < 1e-10


@pytest.mark.parametrize("geometry", ["identity", "sine_bump"])
def test_refined_mixed_gradient_matches_oracle(geometry):
    """The refined mixed form's forward and reverse steps (FP32 operators, one FP64-residual
    refinement of every Kronecker solve and of every transposed one) against the oracle's FP64
    gradient: the remaining difference is the FP32 arithmetic of the mass applies."""
    case = _small(geometry)
    loss_ref, geps_ref, gamp_ref = case["P"].gradient(case["eps"], case["amps"], case["obs"])
    loss, geps, gamp, _ = _gpu_grad(case, precision="mixed_refined")
    print("\n%s refined mixed: loss rel %.2e; rel L2 grad eps %.2e, amps %.2e"
          % (geometry, abs(loss - loss_ref) / loss_ref, rel_l2(geps, geps_ref), rel_l2(gamp, gamp_ref)))
    assert abs(loss - loss_ref) <= 1e-5 * loss_ref
    assert rel_l2(geps, geps_ref) < 1e-5
    assert rel_l2(gamp, gamp_ref) < 1e-5


def test_plain_mixed_has_no_reverse_step():
    import torch
    from paper_2302_04979_gb300 import smx
    ctx = smx.Context(2, 3, eps=("blocks", np.ones((1, 1, 1))), precision="mixed").bind()
    v = torch.zeros(ctx.N_e, dtype=torch.float64, device="cuda")
    w = torch.zeros(ctx.N_h, dtype=torch.float64, device="cuda")
    with pytest.raises(smx.SmxError) as err:
        ctx.step_adjoint(v, v, v.clone(), w, 0.01)
    assert err.value.status == smx.ESTATE


def test_checkpoint_spacing_does_not_change_the_gradient():
    case = _small("sine_bump")
    _, g1, a1, _ = _gpu_grad(case, checkpoint_every=1)
    _, g3, a3, _ = _gpu_grad(case, checkpoint_every=4)
    assert rel_l2(g3, g1) < 1e-13 and rel_l2(a3, a1) < 1e-13


@pytest.mark.slow
def test_adjoint_configuration_finite_differences():
    """48^3, p=3, sine-bump map, permittivity on a 16^3 block grid (seeded U[1,4)), 500 steps,
    32 seeded receivers, misfit against traces of a perturbed permittivity: the adjoint
    gradient against central differences of the GPU loss in 8 seeded directions (1e-6)."""
    import torch
    from paper_2302_04979_gb300 import adjoint as gadj, smx
    p, nel, nb, nsteps = 3, 48, 16, 500
    eps = synth.uniform(2310, nb ** 3, 1.0, 4.0).reshape(nb, nb, nb)
    probe = smx.Context(p, nel, geometry="sine_bump", amplitude=0.05, eps=("blocks", eps))
    N_e, N_h = probe.N_e, probe.N_h
    shapes = [probe.comp_shape(smx.FIELD_D, c) for c in range(3)]
    del probe
    xr = synth.uniform(2311, 96, 0.05, 0.95).reshape(32, 3)
    jhat = synth.bump_coefficients(2312, shapes)
    d0, b0 = np.zeros(N_e), np.zeros(N_h)
    # about 0.5 x the CFL limit: 0.0126 at 16^3 for this map with eps in [1, 4), linear in h (Sec. 5.2)
    dt = 0.002
    amps = synth.source_amplitudes(dt, nsteps, f0=1.0, tau=0.25, t0=0.75)
    prob = gadj.LeapfrogProblem(p, nel, eps, xr, d0, b0, jhat, dt, nsteps, geometry="sine_bump")
    amps_dev = torch.as_tensor(amps).cuda()
    prob.set_eps(eps * (1.0 + 0.05 * synth.uniform(2313, eps.size, -1.0, 1.0).reshape(eps.shape)))
    obs = prob.forward(amps_dev)
    eps_t = torch.tensor(eps, dtype=torch.float64, requires_grad=True)
    amps_t = amps_dev.clone().requires_grad_(True)
    traces = gadj.LeapfrogTraces.apply(eps_t, amps_t, prob)
    loss = gadj.misfit(traces, obs, dt)
    loss.backward()
    geps, gamp = eps_t.grad.numpy(), amps_t.grad.cpu().numpy()

    def L(e, a):
        prob.set_eps(e)
        return float(gadj.misfit(prob.forward(torch.as_tensor(a).cuda()), obs, dt))

    worst = 0.0
    fds = []
    for k in range(8):
        ve = synth.normal(2400 + k, eps.size).reshape(eps.shape)
        va = synth.normal(2500 + k, nsteps)
        h = 2e-5
        fd = (L(eps + h * ve, amps + h * va) - L(eps - h * ve, amps - h * va)) / (2 * h)
        an = float(np.sum(geps * ve) + gamp @ va)
        worst = max(worst, abs(fd - an) / abs(an))
        print("direction %d: FD %.10e adjoint %.10e rel %.2e" % (k, fd, an, abs(fd - an) / abs(an)))
        fds.append(fd)
    assert worst < 1e-6
    # the refined mixed form's gradient (forward and reverse in its arithmetic) against the same
    # FP64 central differences
    probm = gadj.LeapfrogProblem(p, nel, eps, xr, d0, b0, jhat, dt, nsteps, geometry="sine_bump",
                                 precision="mixed_refined")
    eps_m = torch.tensor(eps, dtype=torch.float64, requires_grad=True)
    amps_m = amps_dev.clone().requires_grad_(True)
    lossm = gadj.misfit(gadj.LeapfrogTraces.apply(eps_m, amps_m, probm), obs, dt)
    lossm.backward()
    gm_eps, gm_amp = eps_m.grad.numpy(), amps_m.grad.cpu().numpy()
    worst_m = 0.0
    for k in range(8):
        ve = synth.normal(2400 + k, eps.size).reshape(eps.shape)
        va = synth.normal(2500 + k, nsteps)
        an = float(np.sum(gm_eps * ve) + gm_amp @ va)
        worst_m = max(worst_m, abs(fds[k] - an) / abs(fds[k]))
        print("direction %d: refined mixed adjoint %.10e rel to FP64 FD %.2e" % (k, an, abs(fds[k] - an) / abs(fds[k])))
    print("loss FP64 %.12e, refined mixed %.12e" % (float(loss), float(lossm)))
    assert worst_m < 1e-5   # measured 0.4e-6 .. 3.3e-6


@pytest.mark.parametrize("geometry", ["identity", "sine_bump"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_material_update_survives_rebind(geometry, precision):
    """smx_set_material_blocks rewrites the device tables and their host copy: the Hodge apply
    matches the oracle with the new permittivity (1e-12) right after the update and after the
    workspace is bound again (which uploads the host copy), for the block-Kronecker (identity)
    and the quadrature (curved) Hodge; a second update works from the first's values."""
    import torch
    from paper_2302_04979_gb300 import smx
    p, nel, blocks = 2, (4, 6, 4), (2, 3, 2)
    geom = hodge.SineBumpMap(0.05) if geometry == "sine_bump" else None
    vals = [synth.uniform(70 + k, int(np.prod(blocks)), 1.0, 6.0).reshape(blocks[::-1]) for k in range(3)]
    ctx = smx.Context(p, nel, geometry=geometry, eps=("blocks", vals[0]), precision=precision).bind()
    x = torch.as_tensor(synth.uniform(80, ctx.N_e, -1.0, 1.0)).cuda()
    y = torch.empty_like(x)
    for k in (1, 2):
        ctx.set_material_blocks(vals[k])
        want = maxwell.Scheme2(p, nel, geometry=geom, eps=("blocks", vals[k])).M_eps.apply(x.cpu().numpy())
        for rebind in (False, True):
            if rebind:
                ctx.bind()
            ctx.hodge_apply(smx.FIELD_D, x, y)
            torch.cuda.synchronize()
            assert rel_l2(y.cpu().numpy(), want) < 1e-12, (k, rebind)
