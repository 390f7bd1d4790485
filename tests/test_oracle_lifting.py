"""Pins of the oracle's lifting of inhomogeneous tangential boundary data (Sec. 3.5), CPU only.

What fixes each part independently of the oracle's own formulas:
  * the whole spaces X^1_h, X^2_h: their operators restricted to the interior
    coefficients are exactly the homogeneous ones, the curl of a field with
    zero tangential trace has zero normal trace, and d o d = 0 on the whole
    complex (integers);
  * the local projection: the trace of a discrete field comes back exactly,
    and the sum of the separable terms equals the lift of the data itself
    (linearity);
  * the lifted leapfrog: with zero data it is scheme 2; on a plane wave that
    crosses the cube (tangential E nonzero on four faces) it converges at the
    rates of Sec. 5.1 (E ~ h^p, D ~ h^(p-1)) on the identity and the curved
    map, while scheme 2 without the lifting does not converge at all;
  * scheme 1 with the lifting (Sec. 3.5's first form): its whole-space
    operators restrict to scheme 1's, zero data gives scheme 1's step, and the
    plane wave converges at the same rates;
  * the coaxial cable of Sec. 5.1.2 on its degree-2 NURBS map: the TEM mode,
    with the data lifted on the planes x = 0, y = 0 and z = 0, 1, converges as
    the paper reports for both schemes, E ~ h^p and H ~ h^(p-1).
"""
import numpy as np
import pytest

from oracle import forms3d, hodge, lifting, maxwell, splines
from paper_2302_04979_gb300 import synth


def _eval_full(vec, field, p, nel, X, Y, Z):
    """Components (3, len(X)) of a vector of 'EF' or 'BF' at parametric points (plain basis sums)."""
    p, nel = forms3d.as3(p), forms3d.as3(nel)
    parts = forms3d.split(field, vec, p, nel)
    out = []
    for c in range(3):
        k = forms3d.FIELD_KINDS[field][c]
        bx = splines.space_values(k[0], p[0], nel[0], X)
        by = splines.space_values(k[1], p[1], nel[1], Y)
        bz = splines.space_values(k[2], p[2], nel[2], Z)
        out.append(np.einsum("qi,qj,qk,kji->q", bx, by, bz, parts[c]))
    return np.array(out)


P, NEL = (3, 2, 2), (3, 4, 2)


def test_whole_space_operators_restrict_to_the_homogeneous_ones():
    e_in, e_bd = lifting.index_sets("EF", P, NEL)
    b_in, b_bd = lifting.index_sets("BF", P, NEL)
    assert len(e_in) == forms3d.field_size("E", P, NEL) and len(b_in) == forms3d.field_size("B", P, NEL)
    D1F = forms3d.curl_matrix("EF", P, NEL).toarray()
    D1 = forms3d.curl_matrix("E", P, NEL).toarray()
    assert np.array_equal(D1F[np.ix_(b_in, e_in)], D1)
    # a field with zero tangential trace has a curl with zero normal trace
    assert not np.any(D1F[np.ix_(b_bd, e_in)])
    K1F = lifting.pairing_K1_full(P, NEL).toarray()
    np.testing.assert_allclose(K1F[:, e_in], forms3d.pairing_matrix("K1", P, NEL).toarray(), rtol=0, atol=1e-15)
    M = lifting.MassToFull(P, NEL, hodge.SineBumpMap(0.05), 1.5)
    Mb = hodge.HodgeMass("B", P, NEL, hodge.SineBumpMap(0.05), 1.5)
    x = np.random.default_rng(3).standard_normal(len(b_in))
    xf = np.zeros(forms3d.field_size("BF", P, NEL))
    xf[b_in] = x
    np.testing.assert_allclose(M.apply(xf), Mb.apply(x), rtol=1e-14, atol=1e-15)


def test_whole_complex_d_of_d_is_zero():
    G = forms3d.grad_matrix(P, NEL, full=True)
    D1F = forms3d.curl_matrix("EF", P, NEL)
    Dv = forms3d.div_matrix("BF", P, NEL)
    assert (D1F @ G).count_nonzero() == 0 and (Dv @ D1F).count_nonzero() == 0
    # the full 1D incidence without its boundary columns is the homogeneous one
    assert np.array_equal(splines.incidence_full(4, 3)[:, 1:-1], splines.incidence_primal(4, 3))


def test_lift_reproduces_the_trace_of_a_discrete_field():
    u = np.random.default_rng(1).standard_normal(forms3d.field_size("EF", P, NEL))

    def E(x, y, z):
        shp = np.shape(x)
        return _eval_full(u, "EF", P, NEL, *(np.ravel(v) for v in (x, y, z))).reshape((3,) + shp)

    L = lifting.lift(P, NEL, hodge.IdentityMap(), E)
    e_in, e_bd = lifting.index_sets("EF", P, NEL)
    np.testing.assert_allclose(L[e_bd], u[e_bd], rtol=0, atol=1e-13)
    assert not np.any(L[e_in])


def test_lift_of_a_constant_field_on_the_curved_map():
    """Constants lie in the trace space; on the sine-bump map the faces' tangential Jacobian is the
    identity, so the lifted field's tangential trace equals the physical tangential field."""
    const = np.array([1.0, -2.0, 0.5])

    def E(x, y, z):
        return np.array([const[k] * np.ones_like(x) for k in range(3)])

    L = lifting.lift(P, NEL, hodge.SineBumpMap(0.05), E)
    rng = np.random.default_rng(5)
    for a in range(3):
        for side in (0.0, 1.0):
            pts = rng.uniform(0.0, 1.0, (3, 50))
            pts[a] = side
            vals = _eval_full(L, "EF", P, NEL, *pts)
            for c in range(3):
                if c != a:
                    np.testing.assert_allclose(vals[c], const[c], rtol=0, atol=1e-13)


def test_separable_terms_sum_to_the_lift_of_the_data():
    terms = [(lifting.lift(P, NEL, hodge.IdentityMap(), Em), g) for Em, g in lifting.plane_wave_boundary()]
    for t in (0.0, 0.3, 0.77):
        direct = lifting.lift(P, NEL, hodge.IdentityMap(), lifting.plane_wave(t)[0])
        summed = sum(g(t) * v for v, g in terms)
        np.testing.assert_allclose(summed, direct, rtol=0, atol=1e-13)


def test_zero_data_is_scheme_2():
    L = lifting.LiftedScheme2(P, NEL, geometry=hodge.SineBumpMap(0.05), eps=2.0, mu=1.5)
    S = L.S
    rng = np.random.default_rng(0)
    d = rng.standard_normal(S.N_e)
    b = S.D1 @ rng.standard_normal(S.N_e)
    e = S.e_from_d(d)
    ref = S.step(d, b, e, 0.01, 5)
    bF = np.zeros(L.N_bf)
    bF[L.b_in] = b
    got = L.step(d, bF, e, 0.0, 0.01, 5)
    for g, w in zip((got[0], got[1][L.b_in], got[2], got[3]), ref):
        assert np.linalg.norm(g - w) <= 1e-13 * np.linalg.norm(w)
    assert not np.any(got[1][L.b_bd])


def _plane_wave_errors(p, nel, geometry, lifted=True, T=0.5, scheme=2, frac=0.1):
    """Relative L2 errors (E, D) of the discrete solution against the plane wave at time T
    (dt = frac h; frac = 0.1 is about a third of scheme 2's CFL limit)."""
    E0, B0 = lifting.plane_wave(0.0)
    ET, _ = lifting.plane_wave(T)
    nst = int(round(T / (frac / nel)))
    dt = T / nst
    if lifted:
        cls = lifting.LiftedScheme2 if scheme == 2 else lifting.LiftedScheme1
        L = cls(p, nel, geometry=geometry, boundary=lifting.plane_wave_boundary())
        S = L.S
        d = S.project_2form("D", E0)
        b = S.project_2form("BF", B0)
        d, b, e0, _ = L.step(d, b, L.e0_from_d(d, 0.0), 0.0, dt, nst)
        ee = S.l2_error("EF", L.e_full(e0, T), ET)
    else:
        S = maxwell.Scheme2(p, nel, geometry=geometry)
        d = S.project_2form("D", E0)
        b = S.project_2form("B", B0)
        d, b, e, _ = S.step(d, b, S.e_from_d(d), dt, nst)
        ee = S.l2_error("E", e, ET)
    ed = S.l2_error("D", d, ET)
    return ee[0] / ee[1], ed[0] / ed[1]


@pytest.mark.parametrize("p,geometry", [(2, "identity"), (3, "identity"), (2, "sine_bump")])
def test_plane_wave_converges_at_order_p(p, geometry):
    geom = hodge.SineBumpMap(0.05) if geometry == "sine_bump" else hodge.IdentityMap()
    errs = np.array([_plane_wave_errors(p, n, geom) for n in (2, 4, 8)])
    rates = np.log2(errs[1] / errs[2])
    assert rates[0] > p - 0.25            # E ~ h^p
    assert rates[1] > p - 1 - 0.1         # D ~ h^(p-1)
    assert errs[2, 0] < 0.02


def test_without_the_lifting_the_wave_is_lost():
    lifted = _plane_wave_errors(2, 8, hodge.IdentityMap())[0]
    homogeneous = _plane_wave_errors(2, 8, hodge.IdentityMap(), lifted=False)[0]
    assert lifted < 0.02 and homogeneous > 0.5


def test_scheme1_whole_space_operators_and_zero_data():
    """Scheme 1 (Sec. 3.3) with the lifting: K_2 and M^1_eps on the whole spaces restrict to the
    homogeneous ones, and with zero data the lifted step is scheme 1's."""
    L = lifting.LiftedScheme1(P, NEL, geometry=hodge.SineBumpMap(0.05), eps=2.0, mu=1.5)
    S = L.S1
    assert np.array_equal(L.K2F[:, L.b_in].toarray(), S.K2.toarray())
    np.testing.assert_allclose(L.M1F[L.e_in][:, L.e_in].toarray(), S.M1.matrix().toarray(), rtol=0, atol=1e-14)
    rng = np.random.default_rng(0)
    d = rng.standard_normal(S.N_e)
    b = S.D1 @ rng.standard_normal(S.N_e)
    e = S.e_from_d(d)
    ref = S.step(d, b, e, 0.01, 5)
    bF = np.zeros(L.N_bf)
    bF[L.b_in] = b
    got = L.step(d, bF, e, 0.0, 0.01, 5)
    for g, w in zip((got[0], got[1][L.b_in], got[2], got[3]), ref):
        assert np.linalg.norm(g - w) <= 1e-13 * np.linalg.norm(w)


@pytest.mark.parametrize("p,frac", [(2, 0.05), (3, 0.025)])
def test_scheme1_plane_wave_converges_at_order_p(p, frac):
    """Scheme 1's leapfrog error dominates at dt = h/10 for p = 3 (rate 2.5 there, 3.1 at h/40):
    smaller steps keep the spatial rate visible."""
    errs = np.array([_plane_wave_errors(p, n, hodge.IdentityMap(), scheme=1, frac=frac) for n in (2, 4, 8)])
    rates = np.log2(errs[1] / errs[2])
    assert rates[0] > p - 0.25 and rates[1] > p - 1 - 0.1


@pytest.mark.parametrize("scheme,p,frac", [(2, 2, 0.1), (2, 3, 0.1), (1, 2, 0.05)])
def test_coax_tem_mode_converges_on_the_nurbs_map(scheme, p, frac):
    geom = synth.QuarterCoaxNURBS()
    cls = lifting.LiftedScheme2 if scheme == 2 else lifting.LiftedScheme1
    T = 0.5
    errs = []
    for n in (2, 4, 8):
        L = cls(p, n, geometry=geom, boundary=lifting.coax_tem_boundary())
        S = L.S
        E0, B0 = lifting.coax_tem(0.0)
        nst = int(round(T / (frac / n)))
        dt = T / nst
        d, b = S.project_2form("D", E0), S.project_2form("BF", B0)
        d, b, e0, h = L.step(d, b, L.e0_from_d(d, 0.0), 0.0, dt, nst)
        ET, _ = lifting.coax_tem(T)
        _, Bh = lifting.coax_tem(T - dt / 2)  # h is the half-step value; H = B here
        ee = S.l2_error("EF", L.e_full(e0, T), ET)
        eh = S.l2_error("H", h, Bh)
        errs.append((ee[0] / ee[1], eh[0] / eh[1]))
    errs = np.array(errs)
    rates = np.log2(errs[1] / errs[2])
    assert rates[0] > p - 0.25 and rates[1] > p - 1 - 0.1


def test_both_schemes_reach_errors_of_the_same_size_on_the_cable():
    """Sec. 5.1.2: on the cable the two schemes' errors are of very similar size, neither clearly
    ahead (here within a factor of three at p = 2 on 4 elements per direction)."""
    geom = synth.QuarterCoaxNURBS()
    T, n = 0.5, 4
    nst = int(round(T / (0.05 / n)))
    dt = T / nst
    errs = []
    for cls in (lifting.LiftedScheme2, lifting.LiftedScheme1):
        L = cls(2, n, geometry=geom, boundary=lifting.coax_tem_boundary())
        E0, B0 = lifting.coax_tem(0.0)
        d, b = L.S.project_2form("D", E0), L.S.project_2form("BF", B0)
        d, b, e0, _ = L.step(d, b, L.e0_from_d(d, 0.0), 0.0, dt, nst)
        ee = L.S.l2_error("EF", L.e_full(e0, T), lifting.coax_tem(T)[0])
        errs.append(ee[0] / ee[1])
    assert 1 / 3 < errs[0] / errs[1] < 3
