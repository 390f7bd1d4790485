"""Pins of the oracle's univariate layer (Sec. 2.3, Sec. 4.1) against independent sources.

* scipy.interpolate.BSpline (library B-spline evaluation) for the Cox-de Boor basis;
* sympy's exact piecewise-polynomial B-splines for the pairing matrices G-hat, M-hat;
* the calculus facts the paper states: derivatives of splines are +-1 incidence
  matrices in the chosen bases, and 1D integration by parts
  M-hat d + d~^T G-hat = 0 (Eq. disc_int_by_parts1 in one dimension);
* hand-derived closed forms for p = 2, one element (tests/golden/pairing_p2_nel1.txt).
"""
import os

import numpy as np
import pytest
from scipy.interpolate import BSpline

from oracle import splines

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CASES = [(p, nel) for p in (2, 3, 4, 5) for nel in (1, 2, 3, 7)]


@pytest.mark.parametrize("p,nel", CASES)
def test_bspline_matches_scipy(p, nel):
    xi = splines.open_knot_vector(p, nel)
    x = np.random.default_rng(p * 31 + nel).uniform(0, 1, 57)
    B = splines.bspline_values(xi, p, x)
    n = len(xi) - p - 1
    assert B.shape == (57, n) and n == nel + p
    for i in range(n):
        c = np.zeros(n)
        c[i] = 1.0
        ref = BSpline(xi, c, p, extrapolate=False)(x)
        np.testing.assert_allclose(B[:, i], ref, atol=1e-14)
    np.testing.assert_allclose(B.sum(axis=1), 1.0, atol=1e-14)  # partition of unity


@pytest.mark.parametrize("p,nel", CASES)
def test_curry_schoenberg_unit_integral(p, nel):
    for kind in ("P1", "D1"):
        x, w = splines.element_quadrature(nel, p + 3)
        V = splines.space_values(kind, p, nel, x)
        np.testing.assert_allclose(w @ V, 1.0, atol=1e-13)


@pytest.mark.parametrize("p,nel", CASES)
def test_derivative_is_incidence(p, nel):
    """d/dx sum_i c_i phi_i = sum_j (d c)_j psi_j in the paper's basis choice (Sec. 4.1)."""
    rng = np.random.default_rng(100 * p + nel)
    x = rng.uniform(0, 1, 41)
    xi = splines.open_knot_vector(p, nel)
    # primal: S_p,0 (B-splines) -> S_{p-1}(Xi') (CS)
    c = rng.standard_normal(nel + p - 2)
    full = np.concatenate([[0.0], c, [0.0]])
    deriv = BSpline(xi, full, p).derivative()(x)
    ours = splines.space_values("P1", p, nel, x) @ (splines.incidence_primal(p, nel) @ c)
    np.testing.assert_allclose(ours, deriv, atol=1e-11 * max(1, nel))
    # dual: S_{p-1}(Xi') (B-splines) -> S_{p-2}(Xi'') (CS)
    a = rng.standard_normal(nel + p - 1)
    deriv = BSpline(xi[1:-1], a, p - 1).derivative()(x)
    ours = splines.space_values("D1", p, nel, x) @ (splines.incidence_dual(p, nel) @ a)
    np.testing.assert_allclose(ours, deriv, atol=1e-11 * max(1, nel))


@pytest.mark.parametrize("p,nel", CASES)
def test_integration_by_parts_1d(p, nel):
    G, M = splines.G_hat(p, nel), splines.M_hat(p, nel)
    d, dt = splines.incidence_primal(p, nel), splines.incidence_dual(p, nel)
    assert np.abs(M @ d + dt.T @ G).max() < 1e-14 * nel
    # invertible (inf-sup, Sec. 4.1) and banded with half-bandwidth p-1
    assert np.linalg.cond(G) < 1e3 and np.linalg.cond(M) < 1e3
    for A in (G, M):
        i, j = np.nonzero(np.abs(A) > 1e-15)
        assert np.abs(i - j).max() <= p - 1


def _sympy_pairing(p, nel):
    sympy = pytest.importorskip("sympy")
    from sympy.functions.special.bsplines import bspline_basis_set
    X = sympy.Symbol("x")
    xi = [sympy.Integer(0)] * (p + 1) + [sympy.Rational(k, nel) for k in range(1, nel)] + [sympy.Integer(1)] * (p + 1)

    def cs(knots, deg):
        out = []
        for i, b in enumerate(bspline_basis_set(deg, knots, X)):
            out.append(sympy.Rational(deg + 1) / (knots[i + deg + 1] - knots[i]) * b)
        return out

    def integ(f):
        # integrate piece by piece on each element (exact rational arithmetic)
        tot = 0
        for k in range(nel):
            lo, hi = sympy.Rational(k, nel), sympy.Rational(k + 1, nel)
            mid = (lo + hi) / 2
            piece = sympy.piecewise_fold(f).subs(X, X)
            expr = piece.rewrite(sympy.Piecewise)
            # pick the polynomial active at the element midpoint
            if isinstance(expr, sympy.Piecewise):
                poly = next(e for e, cnd in expr.args if bool(cnd.subs(X, mid)))
            else:
                poly = expr
            tot += sympy.integrate(poly, (X, lo, hi))
        return tot

    P0 = bspline_basis_set(p, xi, X)[1:-1]
    P1 = cs(xi[1:-1], p - 1)
    D0 = bspline_basis_set(p - 1, xi[1:-1], X)
    D1 = cs(xi[2:-2], p - 2) if p > 2 else [
        sympy.Piecewise((sympy.Integer(nel), (X >= sympy.Rational(k, nel)) & (X <= sympy.Rational(k + 1, nel))),
                        (0, True)) for k in range(nel)]
    G = np.array([[float(integ(a * b)) for b in P0] for a in D1])
    M = np.array([[float(integ(a * b)) for b in P1] for a in D0])
    return G, M


@pytest.mark.parametrize("p,nel", [(2, 2), (3, 2), (3, 3), (4, 2)])
def test_pairing_matrices_exact(p, nel):
    """G-hat and M-hat against exact rational integrals of sympy's B-splines."""
    G, M = _sympy_pairing(p, nel)
    np.testing.assert_allclose(splines.G_hat(p, nel), G, atol=1e-14)
    np.testing.assert_allclose(splines.M_hat(p, nel), M, atol=1e-14)


def _read_golden(name):
    mats, cur = {}, None
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            if line.startswith("["):
                cur = line.strip("[]")
                mats[cur] = []
            else:
                mats[cur].append([eval(tok, {}, {}) for tok in line.split()])
    return {k: np.array(v, dtype=np.float64) for k, v in mats.items()}


def test_pairing_golden_p2_one_element():
    g = _read_golden("pairing_p2_nel1.txt")
    np.testing.assert_allclose(splines.G_hat(2, 1), g["G_hat"], atol=1e-15)
    np.testing.assert_allclose(splines.M_hat(2, 1), g["M_hat"], atol=1e-15)
    np.testing.assert_allclose(splines.incidence_primal(2, 1), g["d"], atol=0)
    np.testing.assert_allclose(splines.incidence_dual(2, 1), g["d_tilde"], atol=0)


def test_gauss_rule_exactness():
    for q in range(1, 8):
        z, w = splines.gauss_legendre_01(q)
        for k in range(2 * q):
            assert abs(w @ z ** k - 1.0 / (k + 1)) < 1e-14
