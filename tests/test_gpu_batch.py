"""Batched cavities: one persistent launch per step (smx_batch_*) against the oracle
(oracle.maxwell.Scheme2.step, element-wise, 1e-11), against the same cavities stepped one by
one with smx_step, and the bounded grid barrier's failure path (SMX_ETIMEOUT, then correct
steps again)."""
import numpy as np
import pytest

from paper_2302_04979_gb300 import synth
from tests.gpu_util import rel_l2, to_dev, to_host

pytestmark = pytest.mark.gpu


def _cavity(smx, torch, spec, seed):
    ctx = smx.Context(spec["p"], spec["nel"], eps=spec["eps"], mu=spec.get("mu", 1.0)).bind()
    d = to_dev(synth.uniform(seed, ctx.N_e, -1.0, 1.0))
    b = torch.zeros(ctx.N_h, dtype=torch.float64, device="cuda")
    ctx.curl_primal(to_dev(synth.uniform(seed + 1, ctx.N_e, -1.0, 1.0)), b, 1.0)
    e = torch.empty_like(d)
    ctx.hodge_star(smx.FIELD_D, d, e)
    h = torch.zeros_like(b)
    return ctx, [d, b, e, h]


SMALL = [
    dict(p=2, nel=(6, 5, 7), eps=("blocks", synth.block_material(1, (3, 5, 1), 1.0, 4.0))),
    dict(p=3, nel=8, eps=2.0, mu=1.5),
    dict(p=4, nel=(5, 6, 4), eps=("blocks", synth.block_material(2, (5, 3, 2), 1.0, 4.0))),
    dict(p=3, nel=(9, 8, 10), eps=("blocks", synth.block_material(3, (3, 2, 5), 1.0, 4.0))),
]


def test_batch_matches_single_cavity_steps():
    import torch
    from paper_2302_04979_gb300 import smx
    nsteps = 20
    cavs = [_cavity(smx, torch, s, 10 * i) for i, s in enumerate(SMALL)]
    ref = []
    for k, (ctx, st) in enumerate(cavs):
        dt = 0.5 * ctx.cfl(iters=300, tol=1e-8)
        jhat = to_dev(synth.uniform(77 + k, ctx.N_e, -1.0, 1.0)) if k % 2 == 0 else None
        amp = to_dev(synth.uniform(88 + k, nsteps, -1.0, 1.0)) if jhat is not None else None
        mine = [t.clone() for t in st]
        ctx.step(*mine, dt, nsteps, jhat=jhat, amp=amp)
        ref.append((mine, dt, jhat, amp))
    batch = smx.Batch([c for c, _ in cavs])
    for k, (ctx, st) in enumerate(cavs):
        _, dt, jhat, amp = ref[k]
        batch.set_state(k, *st, dt, jhat=jhat, amp=amp)
    batch.step(nsteps)
    batch.status()
    for k, (ctx, st) in enumerate(cavs):
        errs = [rel_l2(to_host(g), to_host(w)) for g, w in zip(st, ref[k][0])]
        print("\ncavity %d (p=%s nel=%s): rel L2 d %.2e b %.2e e %.2e h %.2e" % (k, SMALL[k]["p"], SMALL[k]["nel"], *errs))
        assert max(errs) < 1e-13


def test_autotune_keeps_state():
    import torch
    from paper_2302_04979_gb300 import smx
    cavs = [_cavity(smx, torch, s, 10 * i) for i, s in enumerate(SMALL[:2])]
    batch = smx.Batch([c for c, _ in cavs])
    for k, (ctx, st) in enumerate(cavs):
        batch.set_state(k, *st, 1e-3)
    before = [[to_host(t) for t in st] for _, st in cavs]
    lw = batch.autotune(steps=2)
    assert lw in (1, 2, 4, 8)
    for (ctx, st), b0 in zip(cavs, before):
        for t, t0 in zip(st, b0):
            assert np.array_equal(to_host(t), t0)
    batch.step(3)
    batch.status()


@pytest.mark.slow
def test_batched_configuration_64_cavities():
    """64 cavities of seeded uneven sizes (nel in [16, 48], even) and degrees p in {2, 3, 4}, each
    with its own permittivity on a 2^3 block grid (seeded U[1, 4)) and its own Gaussian-pulse
    source, 300 steps in persistent launches after autotuning; 8 sampled cavities against
    single-cavity runs."""
    import time
    import torch
    from paper_2302_04979_gb300 import smx
    nsteps = 300
    nel = 16 + 2 * (synth.splitmix64(4040, 64) % 17).astype(int)
    p = 2 + (synth.splitmix64(4041, 64) % 3).astype(int)
    cavs, extra = [], []
    for k in range(64):
        spec = dict(p=int(p[k]), nel=int(nel[k]), eps=("blocks", synth.block_material(4100 + k, (2, 2, 2), 1.0, 4.0)))
        ctx, st = _cavity(smx, torch, spec, 5000 + 10 * k)
        dt = 0.5 * ctx.cfl(iters=200, tol=1e-6)
        shapes = [ctx.comp_shape(smx.FIELD_D, c) for c in range(3)]
        jhat = to_dev(synth.bump_coefficients(4200 + k, shapes))
        amp = to_dev(synth.source_amplitudes(dt, nsteps, f0=1.0, tau=0.25, t0=0.75))
        cavs.append((ctx, st))
        extra.append((dt, jhat, amp, [t.clone() for t in st]))
    batch = smx.Batch([c for c, _ in cavs])
    for k, (ctx, st) in enumerate(cavs):
        batch.set_state(k, *st, extra[k][0], jhat=extra[k][1], amp=extra[k][2])
    lw = batch.autotune(steps=2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    batch.step(nsteps)
    batch.status()
    el = time.perf_counter() - t0
    dof = sum(c.N_e + c.N_h for c, _ in cavs)
    print("\n64 cavities, %d DoF, %d steps: %.3f s, %.3e DoF-steps/s (line warps %d)" % (dof, nsteps, el,
                                                                                       dof * nsteps / el, lw))
    for k in range(0, 64, 8):
        ctx, st = cavs[k]
        dt, jhat, amp, mine = extra[k]
        ctx.step(*mine, dt, nsteps, jhat=jhat, amp=amp)
        errs = [rel_l2(to_host(g), to_host(w)) for g, w in zip(st, mine)]
        assert max(errs) < 1e-12, (k, errs)


ORACLE_CASES = [
    dict(p=2, nel=(5, 7, 4), eps=("blocks", synth.block_material(11, (5, 7, 2), 1.0, 4.0)), source=False),
    dict(p=4, nel=(6, 4, 5), eps=("blocks", synth.block_material(12, (3, 2, 5), 1.0, 4.0)), source=True),
    dict(p=3, nel=(7, 6, 9), eps=2.5, mu=1.25, source=True),
]


def _oracle_inputs(spec, seed, nsteps):
    from oracle import maxwell as mx
    S = mx.Scheme2(spec["p"], spec["nel"], eps=spec["eps"], mu=spec.get("mu", 1.0))
    d = synth.uniform(seed, S.N_e, -1.0, 1.0)
    b = S.D1 @ synth.uniform(seed + 1, S.N_e, -1.0, 1.0)
    e = S.e_from_d(d)
    dt = 0.5 * S.cfl(tol=1e-8)[0]
    jhat = synth.uniform(seed + 2, S.N_e, -1.0, 1.0) if spec["source"] else None
    amps = synth.uniform(seed + 3, nsteps, -1.0, 1.0) if spec["source"] else None
    return S, d, b, e, dt, jhat, amps


def _set_batch(batch, cases, inputs):
    import torch
    states, keep = [], []
    for k, (S, d, b, e, dt, jhat, amps) in enumerate(inputs):
        st = [to_dev(d), to_dev(b), to_dev(e), torch.zeros(S.N_h, dtype=torch.float64, device="cuda")]
        jd = to_dev(jhat) if jhat is not None else None
        ad = to_dev(amps) if amps is not None else None
        batch.set_state(k, *st, dt, jhat=jd, amp=ad)
        states.append(st)
        keep.append((jd, ad))
    return states, keep


def test_batch_matches_oracle():
    """Three uneven cavities (p = 2, 4, 3; anisotropic nel; block and constant material; two with a
    source) stepped together by the persistent kernel, each against the oracle element-wise."""
    from paper_2302_04979_gb300 import smx
    nsteps = 12
    inputs = [_oracle_inputs(s, 300 + 10 * k, nsteps) for k, s in enumerate(ORACLE_CASES)]
    ctxs = [smx.Context(s["p"], s["nel"], eps=s["eps"], mu=s.get("mu", 1.0)).bind() for s in ORACLE_CASES]
    batch = smx.Batch(ctxs)
    states, keep = _set_batch(batch, ORACLE_CASES, inputs)
    batch.step(nsteps)
    batch.status()
    for k, (S, d, b, e, dt, jhat, amps) in enumerate(inputs):
        want = S.step(d, b, e, dt, nsteps, jhat=jhat, amps=amps)
        errs = [rel_l2(to_host(g), w) for g, w in zip(states[k], want)]
        print("\ncavity %d vs oracle: rel L2 d %.2e b %.2e e %.2e h %.2e" % (k, *errs))
        assert max(errs) < 1e-11, (k, errs)


def test_batch_barrier_timeout_then_recovers():
    """With a zero wait limit the grid barriers give up: smx_batch_status reports SMX_ETIMEOUT
    (the failure is made on the device by the time limit, not by a fault), later launches of the
    same call return at entry, and after the status call and the limit restored the batch steps
    correctly again (against the oracle, 1e-11)."""
    from paper_2302_04979_gb300 import smx
    nsteps = 6
    cases = ORACLE_CASES[:2]
    inputs = [_oracle_inputs(s, 400 + 10 * k, nsteps) for k, s in enumerate(cases)]
    ctxs = [smx.Context(s["p"], s["nel"], eps=s["eps"], mu=s.get("mu", 1.0)).bind() for s in cases]
    batch = smx.Batch(ctxs)
    states, keep = _set_batch(batch, cases, inputs)
    batch.set_wait_limit(0.0)
    batch.step(nsteps)
    with pytest.raises(smx.SmxError) as err:
        batch.status()
    assert err.value.status == smx.ETIMEOUT
    batch.status()   # cleared
    batch.set_wait_limit(1.0)
    states, keep = _set_batch(batch, cases, inputs)   # fresh state; resets the step counter
    batch.step(nsteps)
    batch.status()
    for k, (S, d, b, e, dt, jhat, amps) in enumerate(inputs):
        want = S.step(d, b, e, dt, nsteps, jhat=jhat, amps=amps)
        errs = [rel_l2(to_host(g), w) for g, w in zip(states[k], want)]
        assert max(errs) < 1e-11, (k, errs)


GENERAL_CASES = [
    # curved map: quadrature mass applies for both stars
    dict(p=2, nel=(4, 5, 4), geometry="sine_bump", eps=synth.GaussianBumps(41), mu=1.0, source=True),
    # identity map, pointwise permittivity (quadrature star of D) and block permeability (block star of B)
    dict(p=3, nel=(5, 4, 6), eps=lambda x, y, z: 1.0 + x * y + z, mu=("blocks", synth.block_material(42, (5, 2, 3),
                                                                                                   1.0, 3.0)),
         source=False),
    # anisotropic degrees and elements, constant material (fused stars)
    dict(p=(4, 2, 3), nel=(3, 7, 5), eps=1.7, mu=1.2, source=True),
]


def _general_inputs(spec, seed, nsteps):
    from oracle import hodge, maxwell as mx
    geom = hodge.SineBumpMap(0.05) if spec.get("geometry") == "sine_bump" else None
    S = mx.Scheme2(spec["p"], spec["nel"], geometry=geom, eps=spec["eps"], mu=spec["mu"])
    d = synth.uniform(seed, S.N_e, -1.0, 1.0)
    b = S.D1 @ synth.uniform(seed + 1, S.N_e, -1.0, 1.0)
    e = S.e_from_d(d)
    dt = 0.5 * S.cfl(tol=1e-8)[0]
    jhat = synth.uniform(seed + 2, S.N_e, -1.0, 1.0) if spec["source"] else None
    amps = synth.uniform(seed + 3, nsteps, -1.0, 1.0) if spec["source"] else None
    return S, d, b, e, dt, jhat, amps


@pytest.mark.parametrize("graphs", [False, True])
def test_batch_general_cavities_match_oracle(graphs):
    """Curved and quadrature-material cavities with anisotropic degrees in one batch, stepped in
    two calls (eager launches, or CUDA-graph replays on a non-default stream with the step index
    in a device counter), each cavity against the oracle element-wise."""
    import torch
    from paper_2302_04979_gb300 import smx
    nsteps = 10
    inputs = [_general_inputs(s, 500 + 10 * k, nsteps) for k, s in enumerate(GENERAL_CASES)]
    stream = torch.cuda.Stream() if graphs else None
    ctxs = []
    for s in GENERAL_CASES:
        c = smx.Context(s["p"], s["nel"], geometry=s.get("geometry", "identity"), amplitude=0.05, eps=s["eps"],
                        mu=s["mu"]).bind()
        if stream is not None:
            c.set_stream(stream)
        ctxs.append(c)
    batch = smx.Batch(ctxs)
    batch.set_graphs(graphs)
    states, keep = _set_batch(batch, GENERAL_CASES, inputs)
    torch.cuda.synchronize()
    batch.step(nsteps // 2)
    batch.step(nsteps // 2)   # a second call: the graph of 5 launches replayed, the counter at step 5
    batch.status()
    for k, (S, d, b, e, dt, jhat, amps) in enumerate(inputs):
        want = S.step(d, b, e, dt, nsteps, jhat=jhat, amps=amps)
        errs = [rel_l2(to_host(g), w) for g, w in zip(states[k], want)]
        print("\ngeneral cavity %d (graphs %s) vs oracle: rel L2 d %.2e b %.2e e %.2e h %.2e" % (k, graphs, *errs))
        assert max(errs) < 1e-11, (k, errs)


REFINED_CASES = GENERAL_CASES + [
    # block permittivity on the identity map (block-Kronecker FP32 mass of D), a source
    dict(p=2, nel=(5, 7, 4), eps=("blocks", synth.block_material(13, (5, 7, 2), 1.0, 4.0)), mu=1.0, source=True),
]


def _refined_contexts(smx, cases, stream):
    ctxs = []
    for s in cases:
        c = smx.Context(s["p"], s["nel"], geometry=s.get("geometry", "identity"), amplitude=0.05, eps=s["eps"],
                        mu=s["mu"], precision="mixed_refined").bind()
        if stream is not None:
            c.set_stream(stream)
        ctxs.append(c)
    return ctxs


@pytest.mark.parametrize("graphs", [False, True])
def test_refined_batch_matches_oracle(graphs):
    """The refined mixed form (FP32 operators, one FP64-residual refinement of each Kronecker solve)
    in one persistent launch per step: curved, quadrature-material, block and constant-material
    cavities with anisotropic degrees, stepped in two calls, each against the FP64 oracle after 10
    steps (the mixed contract, 1e-5), and against the same cavity stepped alone in the refined form
    (its dense line operators against the batch's banded FP32 recurrences: 1e-5)."""
    import torch
    from paper_2302_04979_gb300 import smx
    nsteps = 10
    inputs = [_general_inputs(s, 700 + 10 * k, nsteps) for k, s in enumerate(REFINED_CASES)]
    stream = torch.cuda.Stream() if graphs else None
    ctxs = _refined_contexts(smx, REFINED_CASES, stream)
    batch = smx.Batch(ctxs)
    batch.set_graphs(graphs)
    states, keep = _set_batch(batch, REFINED_CASES, inputs)
    torch.cuda.synchronize()
    batch.step(nsteps // 2)
    batch.step(nsteps // 2)
    batch.status()
    torch.cuda.synchronize()
    for k, (S, d, b, e, dt, jhat, amps) in enumerate(inputs):
        want = S.step(d, b, e, dt, nsteps, jhat=jhat, amps=amps)
        errs = [rel_l2(to_host(g), w) for g, w in zip(states[k], want)]
        single = [to_dev(d), to_dev(b), to_dev(e), torch.zeros(S.N_h, dtype=torch.float64, device="cuda")]
        torch.cuda.synchronize()
        ctxs[k].step(*single, dt, nsteps, jhat=keep[k][0], amp=keep[k][1])
        torch.cuda.synchronize()
        diff = [rel_l2(to_host(g), to_host(w)) for g, w in zip(states[k], single)]
        print("\nrefined cavity %d (graphs %s) vs oracle: rel L2 d %.2e b %.2e e %.2e h %.2e; vs single refined %.2e"
              % (k, graphs, *errs, max(diff)))
        assert max(errs) < 1e-5, (k, errs)
        assert max(diff) < 1e-5, (k, diff)


def test_refined_batch_rejects_mixed_precisions():
    from paper_2302_04979_gb300 import smx
    a = smx.Context(2, 4, precision="mixed_refined").bind()
    b = smx.Context(2, 4).bind()
    with pytest.raises(smx.SmxError) as err:
        smx.Batch([a, b])
    assert err.value.status == smx.EINVAL
    with pytest.raises(smx.SmxError):
        smx.Batch([smx.Context(2, 4, precision="mixed").bind()])


def test_batched_configuration_64_cavities_refined():
    """The batched configuration in the refined mixed form: 64 cavities of seeded uneven sizes (nel
    in [16, 48], even) and degrees p in {2, 3, 4}, each with its own 2^3-block permittivity (seeded
    U[1, 4)) and Gaussian-pulse source, 300 steps in persistent launches after autotuning.  8 sampled
    cavities against the same cavity stepped alone in FP64 (the FP64 path is within 1e-11 of the
    oracle, tests/test_gpu_configs.py; the oracle itself would take minutes per cavity here), and
    against the same cavity stepped alone in the refined form.
    The refined form's error is that of its FP32 mass applies (the Kronecker solves are refined to
    about 1e-12; the tile passes use compensated FP32 sums): after 300 driven steps it measures
    7.3e-7 (p = 2), 1.4e-6 to 1.7e-6 (p = 3) and 4.3e-6 to 5.2e-6 (p = 4) against FP64 on these
    cavities, in the batch and in single runs alike: the mixed contract, 1e-5.  Two mixed runs of
    one cavity that differ only in the summation order of their FP64 atomics drift apart up to
    that error (a last-bit difference flips the FP32 rounding of an entry, whose error then
    propagates), so the batch and the single refined run are compared at 2e-5."""
    import time
    import torch
    from paper_2302_04979_gb300 import smx
    nsteps = 300
    nel = 16 + 2 * (synth.splitmix64(4040, 64) % 17).astype(int)
    p = 2 + (synth.splitmix64(4041, 64) % 3).astype(int)
    cavs, extra = [], []
    for k in range(64):
        eps = ("blocks", synth.block_material(4100 + k, (2, 2, 2), 1.0, 4.0))
        ctx = smx.Context(int(p[k]), int(nel[k]), eps=eps, precision="mixed_refined").bind()
        fctx, st = _cavity(smx, torch, dict(p=int(p[k]), nel=int(nel[k]), eps=eps), 5000 + 10 * k)
        dt = 0.5 * fctx.cfl(iters=200, tol=1e-6)
        shapes = [ctx.comp_shape(smx.FIELD_D, c) for c in range(3)]
        jhat = to_dev(synth.bump_coefficients(4200 + k, shapes))
        amp = to_dev(synth.source_amplitudes(dt, nsteps, f0=1.0, tau=0.25, t0=0.75))
        cavs.append((ctx, st))
        extra.append((dt, jhat, amp, [t.clone() for t in st], fctx if k % 8 == 0 else None))
    batch = smx.Batch([c for c, _ in cavs])
    for k, (ctx, st) in enumerate(cavs):
        batch.set_state(k, *st, extra[k][0], jhat=extra[k][1], amp=extra[k][2])
    lw = batch.autotune(steps=2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    batch.step(nsteps)
    batch.status()
    el = time.perf_counter() - t0
    dof = sum(c.N_e + c.N_h for c, _ in cavs)
    print("\n64 cavities, refined mixed, %d DoF, %d steps: %.3f s, %.3e DoF-steps/s (line warps %d)"
          % (dof, nsteps, el, dof * nsteps / el, lw))
    worst = []
    for k in range(0, 64, 8):
        ctx, st = cavs[k]
        dt, jhat, amp, mine, fctx = extra[k]
        ref = [t.clone() for t in mine]
        fctx.step(*ref, dt, nsteps, jhat=jhat, amp=amp)
        ctx.step(*mine, dt, nsteps, jhat=jhat, amp=amp)
        errs = [rel_l2(to_host(g), to_host(w)) for g, w in zip(st, ref)]
        diff = [rel_l2(to_host(g), to_host(w)) for g, w in zip(st, mine)]
        serr = [rel_l2(to_host(g), to_host(w)) for g, w in zip(mine, ref)]
        print("cavity %d (p=%d nel=%d): batch vs FP64 rel L2 %.2e (single refined vs FP64 %.2e); batch vs single "
              "refined %.2e" % (k, p[k], nel[k], max(errs), max(serr), max(diff)))
        worst.append((k, max(errs), max(serr), max(diff)))
    for k, eb, es, ed in worst:
        assert eb < 1e-5 and es < 1e-5 and ed < 2e-5, (k, eb, es, ed)
