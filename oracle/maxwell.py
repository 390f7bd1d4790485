"""Scheme 2 of the paper: leapfrog with pairing solves (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper passages followed:
  * Sec. 3.4, Eq. discrete2_ampere, Eq. discrete2_hodge_eps,
    Eq. discrete2_faraday, Eq. discrete2_hodge_mu: the semi-discrete system
        d' = D~^1 h - j,   K_1 e = M~^2_{1/eps} d,
        b' = -D^1 e,       K~_1 h = M^2_{1/mu} b.
  * Sec. 4.2 and Sec. 5: a symplectic leapfrog in time.  Reading used here
    (the paper names no variant): the kick-drift-kick (Stormer-Verlet) form
        b <- b - dt/2 D^1 e
        h <- K~_1^{-1} M^2_{1/mu} b
        d <- d + dt (D~^1 h - s(t_n + dt/2) j)
        e <- K_1^{-1} M~^2_{1/eps} d
        b <- b - dt/2 D^1 e
    with D and B both given at t = 0 (Sec. 5.1.1) and e consistent with d.
  * Sec. 4.2, Eq. kroninverse and the vec identity: the pairing solve is
    x = (A_z (x) A_y (x) A_x)^{-1} y computed as 1D LU solves along x, y, z.
    ``direct_solve`` solves the assembled block instead (both give C^{-1} y).
  * Sec. 2.4, Eq. energy_matrix_wedge and Sec. 3.4 (energy with mass
    matrices): E_h = 1/2 (d^T M~ d + b^T M b).  The factor 1/2 follows
    Eq. energy_matrix_wedge; the later mass-matrix restatement drops it.
  * The modified energy W = E_h - dt^2/8 (D^1 e)^T M (D^1 e) is the quantity
    the kick-drift-kick update conserves exactly (derived from
    Eq. disc_int_by_parts2 and Eq. pairing_transpose, which give
    D^1 K_1^{-1} = (D~^1 K~_1^{-1})^T).
  * Sec. 5.2: the CFL limit; for this update dt_max = 2 / sqrt(lambda_max)
    of L M^2 L^T M~^2 with L = D~^1 K~_1^{-1}, by power iteration.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from . import forms3d, hodge


class Scheme2:
    """All operators of scheme 2 on one mesh; vectors are flat FP64 numpy arrays."""

    def __init__(self, p, nel, geometry=None, eps=1.0, mu=1.0):
        self.p, self.nel = forms3d.as3(p), forms3d.as3(nel)
        self.geometry = geometry if geometry is not None else hodge.IdentityMap()
        self.D1 = forms3d.curl_matrix("E", self.p, self.nel)     # E -> B
        self.Dt1 = forms3d.curl_matrix("H", self.p, self.nel)    # H -> D
        self.M_mu = hodge.HodgeMass("B", self.p, self.nel, self.geometry, mu)
        self.M_eps = hodge.HodgeMass("D", self.p, self.nel, self.geometry, eps)
        self.N_e = forms3d.field_size("E", self.p, self.nel)
        self.N_h = forms3d.field_size("H", self.p, self.nel)
        # 1D LU factors (LAPACK, partial pivoting) of every Kronecker factor
        self._lu = {}
        for which in ("K1", "Kt1"):
            self._lu[which] = [[sla.lu_factor(A) for A in forms3d.pairing_factors(which, c, self.p, self.nel)]
                               for c in range(3)]

    # ---- pairing solves (Sec. 4.2)
    def kron_solve(self, which, y):
        """x = K^{-1} y for K = K_1 ('K1', y in the D layout, x in E) or K~_1 ('Kt1', y in B, x in H)."""
        row_field, col_field = {"K1": ("D", "E"), "Kt1": ("B", "H")}[which]
        ys = forms3d.split(row_field, np.asarray(y, dtype=np.float64), self.p, self.nel)
        xs = []
        for c in range(3):
            lux, luy, luz = self._lu[which][c]
            X = ys[c]
            Nz, Ny, Nx = X.shape
            # (A_z (x) A_y (x) A_x)^{-1} = A_z^{-1} (x) A_y^{-1} (x) A_x^{-1}: one 1D solve per line
            X = sla.lu_solve(lux, X.reshape(-1, Nx).T).T.reshape(Nz, Ny, Nx)
            X = np.moveaxis(sla.lu_solve(luy, np.moveaxis(X, 1, 0).reshape(Ny, -1)).reshape(Ny, Nz, Nx), 0, 1)
            X = sla.lu_solve(luz, X.reshape(Nz, -1)).reshape(Nz, Ny, Nx)
            xs.append(X)
        return forms3d.join(xs)

    def direct_solve(self, which, y):
        """x = K^{-1} y by a sparse direct solve of the assembled pairing matrix (for pins)."""
        K = forms3d.pairing_matrix(which, self.p, self.nel)
        return spla.spsolve(K.tocsc(), y)

    # ---- discrete Hodge stars of scheme 2 (Eq. discrete2_hodge_eps / _mu)
    def e_from_d(self, d):
        return self.kron_solve("K1", self.M_eps.apply(d))

    def h_from_b(self, b):
        return self.kron_solve("Kt1", self.M_mu.apply(b))

    # ---- time stepping
    def step(self, d, b, e, dt, nsteps=1, jhat=None, amps=None):
        """Advance (d, b, e) by nsteps kick-drift-kick leapfrog steps; returns (d, b, e, h).

        amps[n] is the source amplitude s(t_n + dt/2) of step n (J = s(t) jhat).
        On entry e must equal K_1^{-1} M~ d; h returned is the half-step value.
        """
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
        """(E_h, W): discrete energy and the modified energy conserved by the leapfrog."""
        Md = self.M_eps.apply(d)
        Mb = self.M_mu.apply(b)
        Eh = 0.5 * (d @ Md + b @ Mb)
        if e is None:
            return Eh, Eh
        c = self.D1 @ e
        W = Eh - dt * dt / 8.0 * (c @ self.M_mu.apply(c))
        return Eh, W

    def cfl(self, iters=500, tol=1e-12, seed=0):
        """dt_max = 2/sqrt(lambda_max(L M L^T M~)), L = D~^1 K~_1^{-1}, by power iteration."""
        rng = np.random.default_rng(seed)
        v = rng.standard_normal(self.N_e)
        lam_old = 0.0
        lam = 0.0
        for _ in range(iters):
            Av = self.M_eps.apply(v)
            w = self.Dt1 @ self.h_from_b(self.D1 @ self.kron_solve("K1", Av))
            # Rayleigh quotient in the M~ inner product (M~ T is symmetric)
            lam = (Av @ w) / (Av @ v)
            v = w / np.sqrt(w @ self.M_eps.apply(w))
            if abs(lam - lam_old) <= tol * abs(lam):
                break
            lam_old = lam
        return 2.0 / np.sqrt(lam), lam

    def lmat_dense(self):
        """Dense L M L^T M~ for tiny meshes (pins the power iteration)."""
        n = self.N_e
        out = np.zeros((n, n))
        for i in range(n):
            v = np.zeros(n)
            v[i] = 1.0
            Av = self.M_eps.apply(v)
            out[:, i] = self.Dt1 @ self.h_from_b(self.D1 @ self.kron_solve("K1", Av))
        return out

    # ---- projection and errors (Sec. 5.1.1: initial data by projection)
    def project_2form(self, field, V, rtol=1e-14):
        """L2 projection of a physical 2-form (vector proxy V(x, y, z) -> (3,...)) onto X~^2 ('D'), X^2_{h,0}
        ('B') or the whole X^2_h ('BF', Sec. 3.5)."""
        M1 = hodge.HodgeMass(field, self.p, self.nel, self.geometry, 1.0)
        g = M1.grid
        Vp = np.asarray(V(*g.phys))
        # int_Omega V . (J v^/det J) dx = int (J^T V) . v^ dx^
        JtV = np.einsum("ki...,k...->i...", g.J, Vp)
        r = forms3d.join([hodge.integrate(*M1.B[c], JtV[c] * g.W) for c in range(3)])
        n = len(r)
        op = spla.LinearOperator((n, n), matvec=M1.apply, dtype=np.float64)
        x, info = spla.cg(op, r, rtol=rtol, atol=0.0, maxiter=20 * n)
        if info != 0:
            raise RuntimeError("projection CG did not converge")
        return x

    def l2_error(self, field, coeffs, exact, extra=2):
        """(||u_h - u||_L2, ||u||_L2) for a 1-form ('E', 'H', 'EF') or 2-form ('D', 'B', 'BF') against exact(x,y,z)."""
        g = hodge.QuadGrid(self.p, self.nel, self.geometry, extra=extra)
        xs = forms3d.split(field, np.asarray(coeffs, dtype=np.float64), self.p, self.nel)
        uh = np.array([hodge.interpolate(*g.basis(field, c), xs[c]) for c in range(3)])
        if field in ("E", "H", "EF"):
            # 1-form: u = J^{-T} u^
            Jinv = np.linalg.inv(np.moveaxis(g.J, (0, 1), (-2, -1)))
            u = np.einsum("...ki,k...->i...", Jinv, uh)
        else:
            # 2-form: u = J u^ / det J
            u = np.einsum("ik...,k...->i...", g.J, uh) / g.detJ
        ue = np.asarray(exact(*g.phys))
        dens = g.W * g.detJ
        err = np.sqrt(np.sum(dens * np.sum((u - ue) ** 2, axis=0)))
        nrm = np.sqrt(np.sum(dens * np.sum(ue ** 2, axis=0)))
        return err, nrm


# ---------------------------------------------------------------- closed-form cavity mode

OMEGA_TE111 = np.sqrt(3.0) * np.pi


def te111_E(t):
    """E of the (1,1,1) TE mode of the unit-cube PEC cavity, eps = mu = 1 (solves Eq. ampere/faraday)."""
    def f(x, y, z):
        c = np.cos(OMEGA_TE111 * t)
        return np.array([np.cos(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z) * c,
                         -np.sin(np.pi * x) * np.cos(np.pi * y) * np.sin(np.pi * z) * c,
                         0.0 * x])
    return f


def te111_H(t):
    """H of the same mode: H = -(1/sqrt 3) (sx cy cz, cx sy cz, -2 cx cy sz) sin(omega t)."""
    def f(x, y, z):
        s = -np.sin(OMEGA_TE111 * t) / np.sqrt(3.0)
        sx, sy, sz = np.sin(np.pi * x), np.sin(np.pi * y), np.sin(np.pi * z)
        cx, cy, cz = np.cos(np.pi * x), np.cos(np.pi * y), np.cos(np.pi * z)
        return np.array([sx * cy * cz * s, cx * sy * cz * s, -2.0 * cx * cy * sz * s])
    return f
