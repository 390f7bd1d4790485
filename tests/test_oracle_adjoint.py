"""Pins of the oracle's discrete adjoint (oracle/adjoint.py) against things other than itself:
transposes by dot-product identities, the per-block mass derivative by summation and by
finite differences of the mass apply, and the full gradient by central finite differences
of the loss in seeded directions."""
import numpy as np
import pytest

from oracle import adjoint, forms3d, hodge, maxwell
from paper_2302_04979_gb300 import synth


def _problem(geometry=None, nsteps=5, p=2, nel=4, blocks=(2, 2, 2)):
    S0 = maxwell.Scheme2(p, nel, geometry=geometry)
    rng = np.random.default_rng(5)
    xr = synth.uniform(90, 9, 0.05, 0.95).reshape(3, 3)
    rec = adjoint.Receivers(p, nel, xr)
    jhat = synth.uniform(91, S0.N_e, -1.0, 1.0)
    d0 = synth.uniform(92, S0.N_e, -1.0, 1.0)
    b0 = S0.D1 @ synth.uniform(93, S0.N_e, -1.0, 1.0)
    eps = synth.uniform(94, int(np.prod(blocks)), 1.0, 4.0).reshape(blocks)
    dt = 0.4 * S0.cfl(tol=1e-8)[0]
    P = adjoint.MisfitProblem(p, nel, geometry, eps, 1.3, jhat, rec, dt, nsteps, d0, b0)
    amps = synth.uniform(95, nsteps, -1.0, 1.0)
    # observations from a perturbed permittivity
    obs = P.forward(eps * (1.0 + 0.1 * synth.uniform(96, eps.size, -1.0, 1.0).reshape(blocks)), amps)[3]
    return P, eps, amps, obs


def test_transposed_kron_solve_dot_product():
    S = maxwell.Scheme2((2, 3, 2), (3, 4, 2))
    for which, rf, cf in (("K1", "D", "E"), ("Kt1", "B", "H")):
        y = synth.uniform(1, forms3d.field_size(rf, S.p, S.nel), -1, 1)
        x = synth.uniform(2, forms3d.field_size(cf, S.p, S.nel), -1, 1)
        lhs = x @ S.kron_solve(which, y)
        rhs = y @ adjoint.MisfitProblem.kron_solve_T(S, which, x)
        assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0)


def test_dual_curl_is_primal_transpose():
    p, nel = (3, 2, 2), (2, 3, 4)
    D1, Dt1 = forms3d.curl_matrix("E", p, nel), forms3d.curl_matrix("H", p, nel)
    assert abs(Dt1 - D1.T).max() == 0.0


@pytest.mark.parametrize("geom", [None, hodge.SineBumpMap(0.05)])
def test_block_bilinear_is_mass_derivative(geom):
    P, eps, amps, obs = _problem(geometry=geom, nsteps=1)
    z = synth.uniform(3, forms3d.field_size("D", P.p, P.nel), -1, 1)
    d = synth.uniform(4, z.size, -1, 1)
    g = P.block_bilinear(z, d)
    # summed over blocks: the unit-weight mass
    assert abs(g.sum() - z @ P.M1.apply(d)) <= 1e-13 * abs(g.sum())
    # each block: central difference of z^T M~_{1/eps} d in eps_c is -g_c / eps_c^2 (exact: 1/eps is smooth)
    for c in [(0, 0, 0), (1, 0, 1)]:
        h = 1e-5 * eps[c]
        ep, em = eps.copy(), eps.copy()
        ep[c] += h
        em[c] -= h
        Mp = hodge.HodgeMass("D", P.p, P.nel, P.geometry, ("blocks", ep))
        Mm = hodge.HodgeMass("D", P.p, P.nel, P.geometry, ("blocks", em))
        fd = (z @ Mp.apply(d) - z @ Mm.apply(d)) / (2 * h)
        assert abs(fd - (-g[c] / eps[c] ** 2)) <= 1e-7 * abs(fd)


def test_receivers_match_interpolation():
    p, nel = (3, 2, 2), (3, 2, 4)
    g = hodge.QuadGrid(p, nel, hodge.IdentityMap())
    idx = (1, 2, 5)  # a Gauss point (z, y, x indices)
    xr = np.array([[g.pts[0][idx[2]], g.pts[1][idx[1]], g.pts[2][idx[0]]]])
    rec = adjoint.Receivers(p, nel, xr)
    e = synth.uniform(7, forms3d.field_size("E", p, nel), -1, 1)
    es = forms3d.split("E", e, p, nel)
    want = [hodge.interpolate(*g.basis("E", c), es[c])[idx] for c in range(3)]
    np.testing.assert_allclose(rec(e), want, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("geom", [None, hodge.SineBumpMap(0.05)])
def test_gradient_matches_central_differences(geom):
    P, eps, amps, obs = _problem(geometry=geom)
    loss, geps, gamp = P.gradient(eps, amps, obs)
    assert loss > 0
    for k in range(4):  # seeded directions in (eps, amps)
        ve = synth.normal(100 + k, eps.size).reshape(eps.shape)
        va = synth.normal(200 + k, amps.size)
        h = 1e-4
        lp = P.loss(eps + h * ve, amps + h * va, obs)
        lm = P.loss(eps - h * ve, amps - h * va, obs)
        fd = (lp - lm) / (2 * h)
        an = float(np.sum(geps * ve) + gamp @ va)
        assert abs(fd - an) <= 1e-6 * abs(an), (k, fd, an)


def test_source_gradient_is_exact_for_a_quadratic():
    """L is quadratic in the amplitudes: the central difference is exact up to rounding."""
    P, eps, amps, obs = _problem(nsteps=4)
    loss, geps, gamp = P.gradient(eps, amps, obs)
    for n in range(4):
        h = 0.5
        ap, am = amps.copy(), amps.copy()
        ap[n] += h
        am[n] -= h
        fd = (P.loss(eps, ap, obs) - P.loss(eps, am, obs)) / (2 * h)
        assert abs(fd - gamp[n]) <= 1e-9 * max(abs(gamp).max(), 1e-300)
