"""FP64 line operators on the tensor cores (exact digit slicing) through the C ABI.

The FP64 context applies each Hodge star's per-axis line operator (A^{-1}, or
A^{-1} M for a separable star; Eq. kroninverse) as a dense product on the
tcgen05 tensor cores, with every line and operator row cut into seven
balanced base-256 digits and each digit level accumulated exactly.  These
tests hold it to the FP64 contract: against the FP64 oracle, against the
banded FP64 recurrences ("simt") on the same context, on inputs with a wide
dynamic range inside each line, on exact zeros, at the scale extremes of the
normal range, and over many leapfrog steps of the p = 3, 64^3 workload.
"""
import numpy as np
import pytest

from oracle import hodge, maxwell as mx
from paper_2302_04979_gb300 import synth
from tests.gpu_util import rel_l2, to_dev, to_host

pytestmark = pytest.mark.gpu

CASES = {
    "p2_cube_n8": dict(p=2, nel=8),
    "p3_blocks_ragged": dict(p=3, nel=(12, 9, 10), eps=("blocks", synth.block_material(3, (3, 3, 2), 1.0, 9.0)), mu=1.5),
    "p4_aniso": dict(p=(4, 3, 2), nel=(10, 7, 9), eps=2.0, mu=0.7),
    "p3_curved_bumps": dict(p=3, nel=(6, 5, 7), geometry="sine_bump", eps=synth.GaussianBumps(5)),
    "p6_one_element": dict(p=6, nel=(1, 2, 1)),
    "p3_long_lines": dict(p=3, nel=(75, 4, 3), eps=1.3),
}


def _ctx(case, **kw):
    from paper_2302_04979_gb300 import smx
    return smx.Context(case["p"], case["nel"], geometry=case.get("geometry", "identity"),
                       eps=case.get("eps", 1.0), mu=case.get("mu", 1.0), **kw).bind()


def _oracle(case):
    geom = hodge.SineBumpMap(0.05) if case.get("geometry") == "sine_bump" else hodge.IdentityMap()
    return mx.Scheme2(case["p"], case["nel"], geometry=geom, eps=case.get("eps", 1.0), mu=case.get("mu", 1.0))


def _star(G, field, x, kernel):
    from paper_2302_04979_gb300 import smx
    G.set_mode_kernel(kernel)
    out = to_dev(np.zeros(G.N_e if field == smx.FIELD_D else G.N_h))
    G.hodge_star(field, to_dev(x), out)
    G.device_status()
    return to_host(out)


@pytest.fixture(scope="module", params=sorted(CASES))
def trio(request):
    case = CASES[request.param]
    return request.param, _oracle(case), _ctx(case)


def _auto_uses_digits(case, separable):
    """The rule of smx_set_mode_kernel's SMX_MODE_AUTO for an FP64 star."""
    p = np.broadcast_to(case["p"], 3)
    nel = np.broadcast_to(case["nel"], 3)
    maxlen = int(np.max(nel + p - 1))
    return maxlen >= 48 and (separable or int(np.max(p)) - 1 >= 3 or maxlen >= 64)


def test_auto_selection(trio):
    """The default ("auto") runs the tensor-core products where they were measured faster: lines of
    at least 48 entries, for a separable star, and from degree 4 or 64-entry lines for the sweeps
    after a mass apply."""
    from paper_2302_04979_gb300 import smx
    name, S, G = trio
    G.set_mode_kernel("auto")
    for field, n in ((smx.FIELD_D, G.N_e), (smx.FIELD_B, G.N_h)):
        G.set_timing(True)
        G.kernel_times()
        out = to_dev(np.zeros(n))
        G.hodge_star(field, to_dev(np.random.default_rng(7).standard_normal(n)), out)
        t = G.kernel_times()
        G.set_timing(False)
        tc = sum(t["line_f64tc_" + a][1] for a in "xyz")
        want = _auto_uses_digits(CASES[name], G.hodge_mode(field) == 2)
        assert tc == (3 if want else 0), (field, tc)


def test_uses_tensor_kernel(trio):
    """Every line of these meshes has at most 80 entries, so the FP64 stars run on the tensor cores."""
    from paper_2302_04979_gb300 import smx
    _, S, G = trio
    G.set_mode_kernel("tensor")
    G.set_timing(True)
    G.kernel_times()
    x = np.random.default_rng(1).standard_normal(G.N_e)
    out = to_dev(np.zeros(G.N_e))
    G.hodge_star(smx.FIELD_D, to_dev(x), out)
    t = G.kernel_times()
    G.set_timing(False)
    assert all(t["line_f64tc_" + a][1] == 1 for a in "xyz")
    assert all(t["mass_solve_" + a][1] == 0 and t["solve_" + a][1] == 0 for a in "xyz")


@pytest.mark.parametrize("field", ["D", "B"])
def test_star_against_oracle_and_banded(trio, field):
    from paper_2302_04979_gb300 import smx
    name, S, G = trio
    fid = smx.FIELD_D if field == "D" else smx.FIELD_B
    n = G.N_e if field == "D" else G.N_h
    x = np.random.default_rng(2).standard_normal(n)
    ref = S.e_from_d(x) if field == "D" else S.h_from_b(x)
    tc = _star(G, fid, x, "tensor")
    band = _star(G, fid, x, "simt")
    scale = 100.0 if name == "p6_one_element" else 1.0
    e_or, e_band = rel_l2(tc, ref), rel_l2(tc, band)
    print("\n%s star %s: tensor vs oracle %.2e, tensor vs banded %.2e, banded vs oracle %.2e"
          % (name, field, e_or, e_band, rel_l2(band, ref)))
    assert e_or <= 1e-11 * scale
    assert e_band <= 1e-12 * scale


def test_wide_dynamic_range(trio):
    """Entries spanning e^{+-12} inside each line: the per-line fixed point keeps 55 bits of the largest."""
    from paper_2302_04979_gb300 import smx
    name, S, G = trio
    rng = np.random.default_rng(3)
    x = rng.standard_normal(G.N_e) * np.exp(rng.uniform(-12.0, 12.0, G.N_e))
    ref = S.e_from_d(x)
    tc = _star(G, smx.FIELD_D, x, "tensor")
    scale = 100.0 if name == "p6_one_element" else 1.0
    assert rel_l2(tc, ref) <= 1e-11 * scale


def test_zero_and_scale_extremes(trio):
    """A zero input gives exact zeros.  A separable star (three digit passes, nothing else) is
    bit-deterministic and exactly homogeneous under powers of two far into the normal range: the
    digits of a line depend only on its entries' ratios to its largest.  (A non-separable star
    first scatters the mass apply with FP64 atomics, whose summation order varies by an ulp from
    run to run, so it is checked only for zeros.)"""
    from paper_2302_04979_gb300 import smx
    name, S, G = trio
    assert not np.any(_star(G, smx.FIELD_D, np.zeros(G.N_e), "tensor"))
    assert not np.any(_star(G, smx.FIELD_B, np.zeros(G.N_h), "tensor"))
    fields = [f for f in (smx.FIELD_D, smx.FIELD_B) if G.hodge_mode(f) == 2]
    if not fields:
        return
    field = fields[0]
    rng = np.random.default_rng(4)
    x = rng.standard_normal(G.N_e if field == smx.FIELD_D else G.N_h)
    base = _star(G, field, x, "tensor")
    again = _star(G, field, x, "tensor")
    assert np.array_equal(base, again), "not deterministic: %d entries differ" % np.count_nonzero(base != again)
    for k in (-900, -400, 400, 900):
        scaled = _star(G, field, np.ldexp(x, k), "tensor")
        want = np.ldexp(base, k)
        bad = np.flatnonzero(scaled != want)
        if len(bad):
            i = bad[0]
            print("\n%s k=%d: %d of %d differ; first %d: %r vs %r; max rel %.2e" % (
                name, k, len(bad), len(want), i, scaled[i], want[i],
                np.max(np.abs(scaled[bad] - want[bad]) / np.maximum(np.abs(want[bad]), 1e-300))))
        assert len(bad) == 0, k


def test_leapfrog_steps_against_oracle(trio):
    """Twenty-five steps with a source on the tensor-core path against the oracle's leapfrog."""
    import torch
    from paper_2302_04979_gb300 import smx
    name, S, G = trio
    nsteps = 25
    d = synth.uniform(40, S.N_e, -1, 1)
    b = S.D1 @ synth.uniform(41, S.N_e, -1, 1)
    e = S.e_from_d(d)
    jhat = synth.uniform(42, S.N_e, -1, 1)
    dt = 0.02 / max(np.max(S.nel), 1)
    amps = synth.source_amplitudes(dt, nsteps)
    ref = S.step(d, b, e, dt, nsteps, jhat=jhat, amps=amps)
    G.set_mode_kernel("tensor")
    dd, bd, ed = to_dev(d), to_dev(b), to_dev(e)
    hd = torch.zeros(S.N_h, dtype=torch.float64, device="cuda")
    G.step(dd, bd, ed, hd, dt, nsteps, jhat=to_dev(jhat), amp=to_dev(amps))
    G.device_status()
    scale = 100.0 if name == "p6_one_element" else 1.0
    for got, want in zip((dd, bd, ed, hd), ref):
        assert rel_l2(to_host(got), want) < 1e-11 * scale


def test_metric_workload_tensor_vs_banded():
    """p = 3, 64^3 with block permittivity: 200 steps on the tensor cores against the banded FP64
    recurrences, and the conserved energy W over those steps."""
    import torch
    from paper_2302_04979_gb300 import smx
    G = smx.Context(3, 64, eps=("blocks", synth.block_material(7, (8, 8, 8), 1.0, 9.0)), mu=1.0).bind()
    rng = np.random.default_rng(6)
    d0, b0 = rng.standard_normal(G.N_e), rng.standard_normal(G.N_h)
    x = rng.standard_normal(G.N_e)
    e_tc = _star(G, smx.FIELD_D, x, "tensor")
    e_bd = _star(G, smx.FIELD_D, x, "simt")
    print("\n64^3 star of D, tensor vs banded: %.2e" % rel_l2(e_tc, e_bd))
    assert rel_l2(e_tc, e_bd) <= 1e-13
    h_tc = _star(G, smx.FIELD_B, b0, "tensor")
    h_bd = _star(G, smx.FIELD_B, b0, "simt")
    assert rel_l2(h_tc, h_bd) <= 1e-13
    dt, nsteps = 2e-3, 200
    runs = {}
    for kernel in ("tensor", "simt"):
        G.set_mode_kernel(kernel)
        dd, bd = to_dev(d0), to_dev(b0)
        ed, hd = to_dev(np.zeros(G.N_e)), to_dev(np.zeros(G.N_h))
        G.hodge_star(smx.FIELD_D, dd, ed)
        w0 = G.energy(dd, bd, ed, dt)[1]
        G.step(dd, bd, ed, hd, dt, nsteps)
        w1 = G.energy(dd, bd, ed, dt)[1]
        G.device_status()
        runs[kernel] = (to_host(dd), to_host(bd), abs(w1 - w0) / abs(w0))
        torch.cuda.synchronize()
    ed_, eb_ = rel_l2(runs["tensor"][0], runs["simt"][0]), rel_l2(runs["tensor"][1], runs["simt"][1])
    print("64^3 after %d steps, tensor vs banded: d %.2e b %.2e; W drift tensor %.2e banded %.2e"
          % (nsteps, ed_, eb_, runs["tensor"][2], runs["simt"][2]))
    assert ed_ <= 1e-11 and eb_ <= 1e-11
    assert runs["tensor"][2] <= 1e-11
