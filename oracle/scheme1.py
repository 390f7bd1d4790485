"""Scheme 1 of the paper: leapfrog with mass-matrix solves (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper passages followed:
  * Sec. 3.3, Eq. def_hodge_discrete1 and Eq. discrete1_ampere,
    Eq. discrete1_hodge_eps, Eq. discrete1_faraday, Eq. discrete1_hodge_mu:
        d' = D~^1 h - j,   M^1_eps e = K~_2 d,
        b' = -D^1 e,       M~^1_mu h = K_2 b,
    with M^1_eps the mass matrix of X^1_{h,0} weighted by eps and M~^1_mu that
    of X~^1 weighted by mu.  The Hodge stars here map 1-forms to 2-forms, so
    the material weights the 1-form inner product directly (not its inverse).
  * K~_2 pairs X^1_{h,0} with X~^2 and K_2 pairs X~^1 with X^2_{h,0}: the
    same wedge integrals as K_1 and K~_1 with rows and columns exchanged
    (a 1-form and a 2-form commute under the wedge product in 3D), so
    K~_2 = K_1^T and K_2 = K~_1^T (Eq. pairing_transpose).
  * 1-forms pull back with u = J^{-T} u^ (Sec. 2.3), so the mass entries are
        int gamma u_i . u_j dx = int gamma u^_i^T (J^T J)^{-1} u^_j det J dx^.
  * Time stepping: the same kick-drift-kick leapfrog as scheme 2 (the reading
    of Sec. 4.2 / Sec. 5 used throughout), with d and b stepped:
        b <- b - dt/2 D^1 e;  h <- (M~^1_mu)^{-1} K_2 b;
        d <- d + dt (D~^1 h - s j);  e <- (M^1_eps)^{-1} K~_2 d;
        b <- b - dt/2 D^1 e.
  * Energy (Sec. 3.3, energy conservation): E_h = 1/2 (e^T M^1 e + h^T M~^1 h)
    = 1/2 (e^T K~_2 d + h^T K_2 b); the kick-drift-kick update conserves
    W = E_h - dt^2/8 c^T K~_1 (M~^1)^{-1} K_2 c with c = D^1 e, the analogue of
    scheme 2's modified energy (same symplectic structure).
  * Sec. 5.2: the CFL limit of this scheme, by power iteration as for scheme 2.

The mass solves are written out as their plain definition: a sparse direct
solve of the assembled mass matrix (splu).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import forms3d, hodge


class OneFormMass:
    """Mass matrix of the 1-form space of ``field`` ('E': X^1_{h,0}, 'H': X~^1) weighted by gamma.

    gamma is eps for E (Eq. discrete1_hodge_eps) and mu for H (Eq. discrete1_hodge_mu),
    given as the material spec (number, ('blocks', array) or callable of the physical point).
    """

    def __init__(self, field, p, nel, geometry, material_spec):
        assert field in ("E", "H")
        self.field = field
        self.p, self.nel = forms3d.as3(p), forms3d.as3(nel)
        g = hodge.QuadGrid(self.p, self.nel, geometry)
        self.grid = g
        gamma = hodge.material_at(material_spec, *g.phys, g.elem_index, self.nel)
        if np.any(~np.isfinite(gamma)) or np.any(gamma <= 0):
            raise ValueError("material must be finite and positive")
        JtJ = np.einsum("ki...,kj...->...ij", g.J, g.J)
        inv = np.moveaxis(np.linalg.inv(JtJ), (-2, -1), (0, 1))
        # G_cc' = w * gamma * (J^T J)^{-1}_cc' * det J at every grid point
        self.G = inv * (gamma * g.W * g.detJ)[None, None]
        self.B = [g.basis(field, c) for c in range(3)]

    def apply(self, x):
        """y = M x, matrix-free: interpolate, weight by the metric, integrate back."""
        xs = forms3d.split(self.field, np.asarray(x, dtype=np.float64), self.p, self.nel)
        U = [hodge.interpolate(*self.B[c], xs[c]) for c in range(3)]
        ys = []
        for c in range(3):
            V = self.G[c, 0] * U[0] + self.G[c, 1] * U[1] + self.G[c, 2] * U[2]
            ys.append(hodge.integrate(*self.B[c], V))
        return forms3d.join(ys)

    def matrix(self):
        """Assembled sparse M = sum_cc' B_c^T diag(G_cc') B_c'."""
        Bk = [forms3d._kron3(*[sp.csr_matrix(m) for m in self.B[c]]) for c in range(3)]
        blocks = [[None] * 3 for _ in range(3)]
        for c in range(3):
            for c2 in range(3):
                blocks[c][c2] = (Bk[c].T @ sp.diags(self.G[c, c2].reshape(-1)) @ Bk[c2]).tocsr()
        return sp.bmat(blocks, format="csr")


class Scheme1:
    """All operators of scheme 1 on one mesh; vectors are flat FP64 numpy arrays (d, e: N_e; b, h: N_h)."""

    def __init__(self, p, nel, geometry=None, eps=1.0, mu=1.0):
        self.p, self.nel = forms3d.as3(p), forms3d.as3(nel)
        self.geometry = geometry if geometry is not None else hodge.IdentityMap()
        self.D1 = forms3d.curl_matrix("E", self.p, self.nel)
        self.Dt1 = forms3d.curl_matrix("H", self.p, self.nel)
        self.Kt2 = forms3d.pairing_matrix("K1", self.p, self.nel).T.tocsr()   # X^1_{h,0} x X~^2
        self.K2 = forms3d.pairing_matrix("Kt1", self.p, self.nel).T.tocsr()   # X~^1 x X^2_{h,0}
        self.Kt1 = forms3d.pairing_matrix("Kt1", self.p, self.nel)
        self.M1 = OneFormMass("E", self.p, self.nel, self.geometry, eps)
        self.Mt1 = OneFormMass("H", self.p, self.nel, self.geometry, mu)
        self._lu_e = spla.splu(self.M1.matrix().tocsc())
        self._lu_h = spla.splu(self.Mt1.matrix().tocsc())
        self.N_e = forms3d.field_size("E", self.p, self.nel)
        self.N_h = forms3d.field_size("H", self.p, self.nel)

    # ---- discrete Hodge stars of scheme 1 (Eq. discrete1_hodge_eps / _mu)
    def e_from_d(self, d):
        return self._lu_e.solve(self.Kt2 @ np.asarray(d, dtype=np.float64))

    def h_from_b(self, b):
        return self._lu_h.solve(self.K2 @ np.asarray(b, dtype=np.float64))

    def step(self, d, b, e, dt, nsteps=1, jhat=None, amps=None):
        """Advance (d, b, e) by nsteps kick-drift-kick steps; returns (d, b, e, h) (h at the half step)."""
        d, b, e = (np.array(v, dtype=np.float64, copy=True) for v in (d, b, e))
        h = None
        for n in range(nsteps):
            b = b - 0.5 * dt * (self.D1 @ e)
            h = self.h_from_b(b)
            rhs = self.Dt1 @ h
            if jhat is not None:
                rhs = rhs - amps[n] * jhat
            d = d + dt * rhs
            e = self.e_from_d(d)
            b = b - 0.5 * dt * (self.D1 @ e)
        return d, b, e, h

    def energy(self, d, b, e=None, dt=0.0):
        """(E_h, W): E_h = 1/2 (e^T M^1 e + h^T M~^1 h) with e, h the Hodge stars of d and b."""
        e_d = self.e_from_d(d)
        h_b = self.h_from_b(b)
        Eh = 0.5 * (e_d @ self.M1.apply(e_d) + h_b @ self.Mt1.apply(h_b))
        if e is None:
            return Eh, Eh
        c = self.D1 @ e
        W = Eh - dt * dt / 8.0 * (c @ (self.Kt1 @ self.h_from_b(c)))
        return Eh, W

    def cfl(self, iters=500, tol=1e-12, seed=0):
        """dt_max = 2/sqrt(lambda_max) of T = D~^1 S_H D^1 S_E (S_E d = e_from_d, S_H b = h_from_b), by
        power iteration in the inner product of A = K_1 S_E (for which T is self-adjoint)."""
        rng = np.random.default_rng(seed)
        K1 = self.Kt2.T
        v = rng.standard_normal(self.N_e)
        lam_old = lam = 0.0
        for _ in range(iters):
            Av = K1 @ self.e_from_d(v)
            w = self.Dt1 @ self.h_from_b(self.D1 @ self.e_from_d(v))
            lam = (Av @ w) / (Av @ v)
            v = w / np.sqrt(w @ (K1 @ self.e_from_d(w)))
            if abs(lam - lam_old) <= tol * abs(lam):
                break
            lam_old = lam
        return 2.0 / np.sqrt(lam), lam

    def step_matrix_dense(self):
        """Dense T = D~^1 S_H D^1 S_E for tiny meshes (pins the power iteration)."""
        n = self.N_e
        T = np.zeros((n, n))
        for i in range(n):
            v = np.zeros(n)
            v[i] = 1.0
            T[:, i] = self.Dt1 @ self.h_from_b(self.D1 @ self.e_from_d(v))
        return T
