"""Pins of the oracle's scheme-2 leapfrog (Sec. 3.4, Sec. 4.2, Sec. 5).

* Kronecker solve (Eq. kroninverse + vec identity) against a sparse direct
  solve of the assembled pairing matrix;
* the modified energy W is conserved to round-off (derived from
  Eq. disc_int_by_parts2 and Eq. pairing_transpose), E_h oscillates;
* Gauss laws: D^2 b is invariant, D~^2 d obeys the discrete continuity law
  exactly (Eq. maxwell_discrete with d o d = 0);
* convergence to the closed-form TE_111 cavity mode at the rates of Sec. 5.1
  (E ~ h^p, H ~ h^{p-1}) on the unit cube and on the curved sine-bump map;
* the CFL limit against a dense eigen-solve, linear in h, falling with p
  (Sec. 5.2), and a stability check just above and below it;
* the TE_111 mode itself against Maxwell's equations by finite differences.
"""
import numpy as np
import pytest

from oracle import forms3d, hodge, maxwell as mx


@pytest.mark.parametrize("p,nel", [((2, 2, 2), (3, 2, 2)), ((3, 3, 3), (2, 3, 2)), ((4, 2, 3), (2, 2, 3))])
def test_kron_solve_equals_direct(p, nel):
    S = mx.Scheme2(p, nel)
    rng = np.random.default_rng(0)
    y = rng.standard_normal(S.N_e)
    np.testing.assert_allclose(S.kron_solve("K1", y), S.direct_solve("K1", y), rtol=0, atol=1e-11)
    y = rng.standard_normal(S.N_h)
    np.testing.assert_allclose(S.kron_solve("Kt1", y), S.direct_solve("Kt1", y), rtol=0, atol=1e-11)


def _random_state(S, seed):
    rng = np.random.default_rng(seed)
    d = rng.standard_normal(S.N_e)
    b = S.D1 @ rng.standard_normal(S.N_e)  # a discretely divergence-free b
    return d, b, S.e_from_d(d)


@pytest.mark.parametrize("geom", [hodge.IdentityMap(), hodge.SineBumpMap(0.05)])
def test_modified_energy_conserved(geom):
    eps = ("blocks", np.array([[[1.0, 4.0], [2.0, 3.0]], [[5.0, 1.5], [2.5, 9.0]]]))
    S = mx.Scheme2((3, 2, 3), (4, 2, 4), geometry=geom, eps=eps, mu=lambda x, y, z: 1.0 + 0.5 * x * y)
    d, b, e = _random_state(S, 1)
    dt = 0.9 * S.cfl()[0]
    E0, W0 = S.energy(d, b, e, dt)
    Ws, Es = [W0], [E0]
    for _ in range(20):
        d, b, e, _ = S.step(d, b, e, dt, 5)
        E, W = S.energy(d, b, e, dt)
        Ws.append(W)
        Es.append(E)
    Ws, Es = np.array(Ws), np.array(Es)
    assert np.abs(Ws - W0).max() / W0 < 1e-13
    assert np.abs(Es - E0).max() / E0 > 1e-6   # E_h itself oscillates under the leapfrog


def test_gauss_laws():
    S = mx.Scheme2(3, 3, eps=2.0)
    d, b, e = _random_state(S, 2)
    rng = np.random.default_rng(3)
    jhat = rng.standard_normal(S.N_e)
    amps = rng.standard_normal(7)
    dt = 0.5 * S.cfl()[0]
    D2, Dt2 = forms3d.div_matrix("B", S.p, S.nel), forms3d.div_matrix("D", S.p, S.nel)
    d1, b1, e1, _ = S.step(d, b, e, dt, 7, jhat=jhat, amps=amps)
    assert np.abs(D2 @ b1).max() < 1e-12 and np.abs(D2 @ b).max() < 1e-12
    expected = Dt2 @ d - dt * amps.sum() * (Dt2 @ jhat)
    np.testing.assert_allclose(Dt2 @ d1, expected, atol=1e-11)


def test_te111_solves_maxwell():
    """curl E = -dB/dt and curl H = dD/dt for the closed-form mode (eps = mu = 1), by finite differences."""
    rng = np.random.default_rng(4)
    x, y, z = rng.uniform(0.1, 0.9, (3, 10))
    t, h = 0.37, 1e-5

    def curl(F, x, y, z):
        def d(a, comp):
            dx = [h if k == a else 0.0 for k in range(3)]
            return (F(x + dx[0], y + dx[1], z + dx[2])[comp] - F(x - dx[0], y - dx[1], z - dx[2])[comp]) / (2 * h)
        return np.array([d(1, 2) - d(2, 1), d(2, 0) - d(0, 2), d(0, 1) - d(1, 0)])

    dEdt = (mx.te111_E(t + h)(x, y, z) - mx.te111_E(t - h)(x, y, z)) / (2 * h)
    dHdt = (mx.te111_H(t + h)(x, y, z) - mx.te111_H(t - h)(x, y, z)) / (2 * h)
    np.testing.assert_allclose(curl(mx.te111_H(t), x, y, z), dEdt, atol=1e-6)
    np.testing.assert_allclose(curl(mx.te111_E(t), x, y, z), -dHdt, atol=1e-6)


def _cavity_errors(p, nel, geom, T=0.25):
    S = mx.Scheme2(p, nel, geometry=geom)
    nsteps = int(np.ceil(T / 0.002))
    dt = T / nsteps
    d = S.project_2form("D", mx.te111_E(0.0))
    b = np.zeros(S.N_h)
    e = S.e_from_d(d)
    E0 = S.energy(d, b)[0]
    d, b, e, _ = S.step(d, b, e, dt, nsteps)
    eE, nE = S.l2_error("E", e, mx.te111_E(T))
    eH, nH = S.l2_error("H", S.h_from_b(b), mx.te111_H(T))
    return eE / nE, eH / nH, E0


@pytest.mark.slow
@pytest.mark.parametrize("geom", [hodge.IdentityMap(), hodge.SineBumpMap(0.05)])
@pytest.mark.parametrize("p", [2, 3])
def test_cavity_convergence_rates(p, geom):
    """Sec. 5.1: E converges as h^p and H as h^{p-1} in L2, also on a curved map."""
    errs = [_cavity_errors(p, nel, geom) for nel in (2, 4, 8)]
    rE = np.log2(errs[1][0] / errs[2][0])
    rH = np.log2(errs[1][1] / errs[2][1])
    assert rE > p - 0.3, (rE, errs)
    assert rH > p - 1 - 0.2, (rH, errs)
    assert errs[2][0] < errs[1][0] < errs[0][0]
    # discrete energy at t=0 approaches the exact 1/8 (1/2 int |E|^2)
    assert abs(errs[2][2] - 0.125) < abs(errs[0][2] - 0.125)
    assert abs(errs[2][2] - 0.125) < 2e-2


def test_cfl_power_iteration_vs_dense():
    S = mx.Scheme2((2, 3, 2), (2, 2, 3), eps=("blocks", np.array([[[2.0]], [[3.0]], [[1.0]]])))
    dtm, lam = S.cfl()
    ev = np.linalg.eigvals(S.lmat_dense())
    assert np.abs(ev.imag).max() < 1e-8 * ev.real.max()  # similar to a symmetric PSD matrix
    np.testing.assert_allclose(lam, ev.real.max(), rtol=1e-9)


def test_cfl_scaling_and_stability():
    """dt_max is linear in h (Sec. 5.2) and decreases with p; the step is stable just below it."""
    dts = [mx.Scheme2(3, nel).cfl(tol=1e-9)[0] for nel in (4, 8)]
    assert 1.8 < dts[0] / dts[1] < 2.2
    dtp = [mx.Scheme2(p, 6).cfl(tol=1e-9)[0] for p in (2, 3, 4)]
    assert dtp[0] > dtp[1] > dtp[2]
    S = mx.Scheme2(2, 4)
    dtm = S.cfl()[0]
    d, b, e = _random_state(S, 7)
    E0 = S.energy(d, b)[0]
    ok = S.step(d, b, e, 0.98 * dtm, 400)
    bad = S.step(d, b, e, 1.05 * dtm, 400)
    assert S.energy(ok[0], ok[1])[0] < 10 * E0
    assert S.energy(bad[0], bad[1])[0] > 1e3 * E0


def test_energy_oscillation_shrinks_with_h_and_p():
    """Sec. 5.1.1 (energy against time, TE mode, dt from the CFL condition): the leapfrog's
    oscillation of E_h shrinks when the mesh is refined and when the degree is raised, and so does
    the gap between the mean discrete energy and the exact 1/8."""
    stats = {}
    for p, nel in [(3, 2), (3, 4), (4, 2), (4, 4)]:
        S = mx.Scheme2(p, nel)
        d = S.project_2form("D", mx.te111_E(0.0))
        b = np.zeros(S.N_h)
        e = S.e_from_d(d)
        dt = 0.5 * S.cfl(tol=1e-8)[0]
        n = int(np.ceil(2 * np.pi / mx.OMEGA_TE111 / dt))  # one period
        Es = []
        for _ in range(n):
            d, b, e, _ = S.step(d, b, e, dt, 1)
            Es.append(S.energy(d, b)[0])
        Es = np.array(Es)
        stats[(p, nel)] = ((Es.max() - Es.min()) / Es.mean(), abs(Es.mean() - 0.125) / 0.125)
    for i in range(2):  # 0: oscillation amplitude, 1: error of the mean energy
        assert stats[(3, 4)][i] < 0.5 * stats[(3, 2)][i]
        assert stats[(4, 4)][i] < 0.5 * stats[(4, 2)][i]
        assert stats[(4, 2)][i] < stats[(3, 2)][i] and stats[(4, 4)][i] < stats[(3, 4)][i]
