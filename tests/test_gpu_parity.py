"""GPU parity of every hot-path stage against the FP64 oracle, through the C ABI.

Meshes are small enough for the oracle to finish in seconds but span several
Hodge tiles (8 elements) and solve CTAs (32 lines) with ragged tails, all
supported degrees, anisotropic degrees/meshes, the block-Kronecker and the
quadrature Hodge paths, and a source term.

Tolerances (relative L2): 1e-12 for a single stage, 1e-11 for composites
(Hodge star = mass apply + solve) and for the fields after many leapfrog
steps (the FP64 contract); integer index work (the
incidence pattern and numbering) is checked bit-exactly on integer data.
"""
import numpy as np
import pytest

from oracle import forms3d, hodge, maxwell as mx
from paper_2302_04979_gb300 import synth
from tests.gpu_util import rel_l2, to_dev, to_host

pytestmark = pytest.mark.gpu

CASES = {
    "p2_cube_n8": dict(p=2, nel=8),
    "p3_blocks_ragged": dict(p=3, nel=(12, 9, 10), eps=("blocks", synth.block_material(3, (3, 3, 2), 1.0, 9.0)), mu=1.5),
    "p4_aniso_elementwise": dict(p=(4, 3, 2), nel=(10, 7, 9), eps=2.0,
                                 mu=("blocks", synth.block_material(4, (10, 7, 9), 1.0, 4.0))),
    "p3_curved_bumps": dict(p=3, nel=(6, 5, 7), geometry="sine_bump", eps=synth.GaussianBumps(5)),
    "p2_pointwise": dict(p=2, nel=(9, 8, 7), eps=lambda x, y, z: 1.0 + x * y + z * z),
    "p5_small": dict(p=5, nel=(3, 4, 2), eps=3.0, mu=0.5),
    "p6_one_element": dict(p=6, nel=(1, 2, 1)),
}

# Solves amplify rounding by the condition numbers of the 1D pairing factors:
# about 30 for p <= 4, 1e2 for p = 5 and 4e2 for p = 6 (oracle, Sec. 4.1
# matrices), and a 3D Kronecker solve multiplies three of them (kappa eps is
# about 7e-9 at p = 6).  The FP64 contract (1e-11) is stated for the
# configurations' degrees p <= 4; p = 5, 6 get the same bound scaled by the
# growth of that product.  Measured on GB300, every p = 5, 6 error but one sits
# below the unscaled bound; the exception is the star of B at p = 6,
# 3.3e-11 (the printed errors show it).
COND_SCALE = {5: 10.0, 6: 100.0}


def cond_scale(name):
    p = CASES[name]["p"]
    return COND_SCALE.get(int(np.max(p)), 1.0)


def _oracle(case):
    geom = hodge.SineBumpMap(0.05) if case.get("geometry") == "sine_bump" else hodge.IdentityMap()
    return mx.Scheme2(case["p"], case["nel"], geometry=geom, eps=case.get("eps", 1.0), mu=case.get("mu", 1.0))


def _gpu(case):
    from paper_2302_04979_gb300 import smx
    return smx.Context(case["p"], case["nel"], geometry=case.get("geometry", "identity"),
                       eps=case.get("eps", 1.0), mu=case.get("mu", 1.0)).bind()


@pytest.fixture(scope="module", params=sorted(CASES))
def pair(request):
    case = CASES[request.param]
    return request.param, _oracle(case), _gpu(case)


def test_sizes(pair):
    _, S, G = pair
    assert (G.N_e, G.N_h) == (S.N_e, S.N_h)


def test_curl_integer_exact(pair):
    """The incidence pattern is bit-exact: integer data stays integer and equals D^1 e, D~^1 h."""
    _, S, G = pair
    rng = np.random.default_rng(0)
    e = rng.integers(-1000, 1000, S.N_e).astype(np.float64)
    b = rng.integers(-1000, 1000, S.N_h).astype(np.float64)
    bd = to_dev(b)
    G.curl_primal(to_dev(e), bd, 1.0)
    assert np.array_equal(to_host(bd), b + S.D1 @ e)
    h = rng.integers(-1000, 1000, S.N_h).astype(np.float64)
    d = rng.integers(-1000, 1000, S.N_e).astype(np.float64)
    j = rng.integers(-1000, 1000, S.N_e).astype(np.float64)
    dd = to_dev(d)
    G.curl_dual(to_dev(h), dd, 1.0, to_dev(j), 3.0)
    assert np.array_equal(to_host(dd), d + S.Dt1 @ h - 3.0 * j)


def test_curl_scaled(pair):
    _, S, G = pair
    e, b = synth.uniform(1, S.N_e, -1, 1), synth.uniform(2, S.N_h, -1, 1)
    bd = to_dev(b)
    G.curl_primal(to_dev(e), bd, -0.37)
    assert rel_l2(to_host(bd), b - 0.37 * (S.D1 @ e)) < 1e-15


def test_hodge_apply(pair):
    import torch
    _, S, G = pair
    from paper_2302_04979_gb300 import smx
    for field, M, n in ((smx.FIELD_B, S.M_mu, S.N_h), (smx.FIELD_D, S.M_eps, S.N_e)):
        x = synth.uniform(10 + field, n, -1, 1)
        y = torch.empty(n, dtype=torch.float64, device="cuda")
        G.hodge_apply(field, to_dev(x), y)
        assert rel_l2(to_host(y), M.apply(x)) < 1e-13


def test_pairing_solve(pair):
    import torch
    name, S, G = pair
    from paper_2302_04979_gb300 import smx
    for which, key, n in ((smx.FIELD_E, "K1", S.N_e), (smx.FIELD_H, "Kt1", S.N_h)):
        y = synth.uniform(20 + which, n, -1, 1)
        x = torch.empty(n, dtype=torch.float64, device="cuda")
        G.pairing_solve(which, to_dev(y), x)
        err = rel_l2(to_host(x), S.kron_solve(key, y))
        print("\n%s pairing solve %s: rel L2 %.2e (bound %.0e)" % (name, key, err, 1e-12 * cond_scale(name)))
        assert err < 1e-12 * cond_scale(name)
        # in place
        yd = to_dev(y)
        G.pairing_solve(which, yd, yd)
        assert rel_l2(to_host(yd), S.kron_solve(key, y)) < 1e-12 * cond_scale(name)


def test_hodge_star(pair):
    import torch
    name, S, G = pair
    from paper_2302_04979_gb300 import smx
    d = synth.uniform(30, S.N_e, -1, 1)
    e = torch.empty(S.N_e, dtype=torch.float64, device="cuda")
    G.hodge_star(smx.FIELD_D, to_dev(d), e)
    # a mass apply followed by a Kronecker solve: the FP64 field tolerance 1e-11
    err = rel_l2(to_host(e), S.e_from_d(d))
    print("\n%s Hodge star of D: rel L2 %.2e" % (name, err))
    assert err < 1e-11 * cond_scale(name)
    b = synth.uniform(31, S.N_h, -1, 1)
    h = torch.empty(S.N_h, dtype=torch.float64, device="cuda")
    G.hodge_star(smx.FIELD_B, to_dev(b), h)
    err = rel_l2(to_host(h), S.h_from_b(b))
    print("%s Hodge star of B: rel L2 %.2e" % (name, err))
    assert err < 1e-11 * cond_scale(name)


def test_leapfrog_steps_with_source(pair):
    import torch
    name, S, G = pair
    from paper_2302_04979_gb300 import smx
    nsteps = 25
    d = synth.uniform(40, S.N_e, -1, 1)
    b = S.D1 @ synth.uniform(41, S.N_e, -1, 1)
    e = S.e_from_d(d)
    jhat = synth.uniform(42, S.N_e, -1, 1)
    dt = 0.02 / max(np.max(S.nel), 1)
    amps = synth.source_amplitudes(dt, nsteps)
    ref = S.step(d, b, e, dt, nsteps, jhat=jhat, amps=amps)
    dd, bd, ed = to_dev(d), to_dev(b), to_dev(e)
    hd = torch.zeros(S.N_h, dtype=torch.float64, device="cuda")
    G.step(dd, bd, ed, hd, dt, nsteps, jhat=to_dev(jhat), amp=to_dev(amps))
    errs = [rel_l2(to_host(got), want) for got, want in zip((dd, bd, ed, hd), ref)]
    print("\n%s %d steps: rel L2 d %.2e b %.2e e %.2e h %.2e" % (name, nsteps, *errs))
    assert max(errs) < 1e-11 * cond_scale(name)



def test_step_host(pair):
    """smx_step_host: the same steps from host buffers, pinned and pageable, with the copies in and
    out inside the call; equal to smx_step on device buffers up to the atomics' summation order
    (1e-13) and within the FP64 contract of the oracle."""
    import torch
    name, S, G = pair
    nsteps = 5
    d = synth.uniform(60, S.N_e, -1, 1)
    b = S.D1 @ synth.uniform(61, S.N_e, -1, 1)
    e = S.e_from_d(d)
    jhat = synth.uniform(62, S.N_e, -1, 1)
    dt = 0.02 / max(np.max(S.nel), 1)
    amps = synth.source_amplitudes(dt, nsteps)
    ref = S.step(d, b, e, dt, nsteps, jhat=jhat, amps=amps)
    jd, ad = to_dev(jhat), to_dev(amps)
    dd, bd, ed = to_dev(d), to_dev(b), to_dev(e)
    hd = torch.zeros(S.N_h, dtype=torch.float64, device="cuda")
    G.step(dd, bd, ed, hd, dt, nsteps, jhat=jd, amp=ad)
    dev = [to_host(t) for t in (dd, bd, ed, hd)]
    for pinned in (True, False):
        host = [torch.from_numpy(v.copy()) for v in (d, b, e)] + [torch.zeros(S.N_h, dtype=torch.float64)]
        if pinned:
            host = [t.pin_memory() for t in host]
        G.step_host(*host, dt, nsteps, jhat=jd, amp=ad)
        got = [t.numpy() for t in host]
        assert max(rel_l2(g, w) for g, w in zip(got, dev)) < 1e-13
        assert max(rel_l2(g, w) for g, w in zip(got, ref)) < 1e-11 * cond_scale(name)

def test_energy(pair):
    _, S, G = pair
    d = synth.uniform(50, S.N_e, -1, 1)
    b = S.D1 @ synth.uniform(51, S.N_e, -1, 1)
    e = S.e_from_d(d)
    dt = 0.01
    Eh, W = G.energy(to_dev(d), to_dev(b), to_dev(e), dt)
    rEh, rW = S.energy(d, b, e, dt)
    assert abs(Eh - rEh) <= 1e-12 * abs(rEh)
    assert abs(W - rW) <= 1e-12 * abs(rW)


def test_nonfinite_detected(pair):
    _, S, G = pair
    from paper_2302_04979_gb300 import smx
    d = synth.uniform(60, S.N_e, -1, 1)
    d[S.N_e // 2] = np.nan
    with pytest.raises(smx.SmxError) as err:
        G.energy(to_dev(d), to_dev(np.zeros(S.N_h)))
    assert err.value.status == smx.ENONFINITE


@pytest.mark.parametrize("name", ["p2_cube_n8", "p3_blocks_ragged"])
def test_cfl_matches_oracle(name):
    case = CASES[name]
    S, G = _oracle(case), _gpu(case)
    ref = S.cfl(tol=1e-13, iters=3000)[0]
    got = G.cfl(iters=3000, tol=1e-13)
    assert abs(got - ref) <= 1e-7 * ref


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_step_graph_replay(precision):
    """smx_step on a non-default stream: captured into a CUDA graph on the first call, replayed after."""
    import torch
    from paper_2302_04979_gb300 import smx
    case = CASES["p3_blocks_ragged"]
    S = _oracle(case)
    G = smx.Context(case["p"], case["nel"], eps=case["eps"], mu=case["mu"], precision=precision).bind()
    stream = torch.cuda.Stream()
    G.set_stream(stream)
    d = synth.uniform(80, S.N_e, -1, 1)
    b = S.D1 @ synth.uniform(81, S.N_e, -1, 1)
    e = S.e_from_d(d)
    dt, nsteps = 0.01, 3
    ref = S.step(d, b, e, dt, 2 * nsteps)
    dd, bd, ed = to_dev(d), to_dev(b), to_dev(e)
    hd = torch.zeros(S.N_h, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    n0 = G.launch_count()
    G.step(dd, bd, ed, hd, dt, nsteps)   # capture + first replay
    n1 = G.launch_count()
    G.step(dd, bd, ed, hd, dt, nsteps)   # replay of the cached graph
    n2 = G.launch_count()
    stream.synchronize()
    assert n1 - n0 == n2 - n1 > 0
    tol = 1e-11 if precision == "fp64" else 1e-5
    for got, want in zip((dd, bd, ed, hd), ref):
        assert rel_l2(to_host(got), want) < tol
