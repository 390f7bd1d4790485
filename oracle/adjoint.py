"""Discrete adjoint of the scheme-2 leapfrog: gradient of a receiver misfit (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper defines the forward problem only; the gradient here is the exact
derivative of a loss of the discrete forward map, written out in reverse
order.  No adjoint PDE is discretised, so the result is pinned by central
finite differences of the same loss.

Forward map, one step (the kick-drift-kick reading of Sec. 4.2 / Sec. 5, see
``oracle.maxwell``; S_E = K_1^{-1} M~^2_{1/eps}, S_H = K~_1^{-1} M^2_{1/mu},
Eq. discrete2_hodge_eps / discrete2_hodge_mu, a = dt/2):
    b'      = b_n - a D^1 S_E d_n
    d_{n+1} = d_n + dt (D~^1 S_H b' - s_n jhat)          (Eq. discrete2_ampere)
    b_{n+1} = b' - a D^1 S_E d_{n+1}                     (Eq. discrete2_faraday)

Parameters: the permittivity as values eps_c on a grid of element blocks
(the 'blocks' material, one value per block of parametric elements) and the
source amplitudes s_n.

Loss: L = 1/2 dt sum_{n=1..N} |R e_n - y_n|^2, e_n = S_E d_n, where R
evaluates the parametric components of the discrete electric 1-form
(X^1_{h,0}: component c has the primal S_{p-1} space along axis c and the
boundary-reduced S_p along the others) at receiver points x^_r.

Reverse sweep (ebar_n = dt R^T (R e_n - y_n); dbar, bbar the derivatives of L
with respect to the state):
    dbar_N = S_E^T ebar_N,  bbar_N = 0
    for n = N-1 .. 0:
        w     = dbar_{n+1} - a S_E^T D^1^T bbar_{n+1}
        sbar_n = -dt jhat^T w
        bbar' = bbar_{n+1} + dt S_H^T D~^1^T w
        dbar_n = w - a S_E^T D^1^T bbar' (+ S_E^T ebar_n for n >= 1)
        bbar_n = bbar'
with S_E^T = M~ K_1^{-T}, S_H^T = M K~_1^{-T} (the masses are symmetric).
Every use of S_E(eps) against a vector ybar and a state d adds, for block c,
    dL/deps_c += ybar^T dS_E/deps_c d = -(1/eps_c^2) (K_1^{-T} ybar)^T M~1_c d,
M~1_c the unit-weight mass restricted to the elements of block c.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import forms3d, hodge, maxwell, splines


class Receivers:
    """R: the 3 parametric components of the discrete E field at points xhat (nr x 3) in [0,1]^3.

    Row 3 r + c of R holds the tensor-product basis of E component c evaluated at xhat_r.
    """

    def __init__(self, p, nel, xhat):
        self.p, self.nel = forms3d.as3(p), forms3d.as3(nel)
        xhat = np.atleast_2d(np.asarray(xhat, dtype=np.float64))
        self.nr = xhat.shape[0]
        offs = forms3d.comp_offsets("E", self.p, self.nel)
        rows, cols, vals = [], [], []
        for r in range(self.nr):
            for c in range(3):
                kinds = forms3d.FIELD_KINDS["E"][c]
                v = [splines.space_values(kinds[a], self.p[a], self.nel[a], xhat[r, a:a + 1])[0] for a in range(3)]
                Nz, Ny, Nx = forms3d.comp_shape("E", c, self.p, self.nel)
                full = np.einsum("k,j,i->kji", v[2], v[1], v[0]).reshape(-1)
                nz = np.nonzero(full)[0]
                rows += [3 * r + c] * len(nz)
                cols += list(offs[c] + nz)
                vals += list(full[nz])
        N_e = forms3d.field_size("E", self.p, self.nel)
        self.R = sp.csr_matrix((vals, (rows, cols)), shape=(3 * self.nr, N_e))

    def __call__(self, e):
        return self.R @ e


class MisfitProblem:
    """Receiver-misfit loss of N leapfrog steps and its exact gradient (full-storage reverse sweep)."""

    def __init__(self, p, nel, geometry, eps_blocks, mu, jhat, receivers, dt, nsteps, d0, b0):
        self.p, self.nel = forms3d.as3(p), forms3d.as3(nel)
        self.geometry = geometry if geometry is not None else hodge.IdentityMap()
        self.mu, self.jhat, self.rec = mu, np.asarray(jhat, dtype=np.float64), receivers
        self.dt, self.nsteps = float(dt), int(nsteps)
        self.d0, self.b0 = np.asarray(d0, dtype=np.float64), np.asarray(b0, dtype=np.float64)
        self.shape = np.asarray(eps_blocks).shape
        # unit-weight electric mass: its quadrature metric, for the per-block bilinear forms
        self.M1 = hodge.HodgeMass("D", self.p, self.nel, self.geometry, 1.0)
        g = self.M1.grid
        bz, by, bx = self.shape
        ez, ey, ex = g.elem_index
        self.block_of_point = ((ez // (self.nel[2] // bz)) * by + (ey // (self.nel[1] // by))) * bx + \
            (ex // (self.nel[0] // bx))

    def scheme(self, eps_blocks):
        return maxwell.Scheme2(self.p, self.nel, self.geometry, eps=("blocks", np.asarray(eps_blocks)), mu=self.mu)

    # ---- forward
    def forward(self, eps_blocks, amps, obs=None):
        """States d_0..d_N, b_0..b_N, receiver traces R e_1..R e_N and the loss (if obs is given)."""
        S = self.scheme(eps_blocks)
        d, b = self.d0.copy(), self.b0.copy()
        e = S.e_from_d(d)
        ds, bs, traces = [d], [b], []
        for n in range(self.nsteps):
            d, b, e, _ = S.step(d, b, e, self.dt, 1, jhat=self.jhat, amps=[amps[n]])
            ds.append(d)
            bs.append(b)
            traces.append(self.rec(e))
        traces = np.array(traces)
        loss = None if obs is None else 0.5 * self.dt * float(np.sum((traces - obs) ** 2))
        return S, ds, bs, traces, loss

    def loss(self, eps_blocks, amps, obs):
        return self.forward(eps_blocks, amps, obs)[4]

    # ---- transposed operators
    @staticmethod
    def kron_solve_T(S, which, y):
        """z = K^{-T} y: the 1D LU solves of ``Scheme2.kron_solve`` with the transposed factors."""
        row_field, col_field = {"K1": ("D", "E"), "Kt1": ("B", "H")}[which]
        ys = forms3d.split(col_field, np.asarray(y, dtype=np.float64), S.p, S.nel)
        zs = []
        for c in range(3):
            lux, luy, luz = S._lu[which][c]
            X = ys[c]
            Nz, Ny, Nx = X.shape
            X = sla.lu_solve(lux, X.reshape(-1, Nx).T, trans=1).T.reshape(Nz, Ny, Nx)
            X = np.moveaxis(sla.lu_solve(luy, np.moveaxis(X, 1, 0).reshape(Ny, -1), trans=1).reshape(Ny, Nz, Nx), 0, 1)
            X = sla.lu_solve(luz, X.reshape(Nz, -1), trans=1).reshape(Nz, Ny, Nx)
            zs.append(X)
        return forms3d.join(zs)

    def block_bilinear(self, z, d):
        """Per block c: z^T M~1_c d (unit-weight mass restricted to the block's elements), shape of the blocks."""
        M = self.M1
        zs = forms3d.split("D", z, self.p, self.nel)
        xs = forms3d.split("D", d, self.p, self.nel)
        Uz = [hodge.interpolate(*M.B[c], zs[c]) for c in range(3)]
        Ud = [hodge.interpolate(*M.B[c], xs[c]) for c in range(3)]
        val = sum(Uz[c] * M.G[c, c2] * Ud[c2] for c in range(3) for c2 in range(3))
        out = np.bincount(self.block_of_point.reshape(-1), weights=val.reshape(-1), minlength=int(np.prod(self.shape)))
        return out.reshape(self.shape)

    # ---- gradient
    def gradient(self, eps_blocks, amps, obs):
        """(loss, dL/deps_blocks, dL/damps) by the reverse sweep of the module docstring."""
        eps = np.asarray(eps_blocks, dtype=np.float64)
        S, ds, bs, traces, loss = self.forward(eps, amps, obs)
        dt, a, N = self.dt, 0.5 * self.dt, self.nsteps
        ebar = [None] + [dt * (self.rec.R.T @ (traces[n - 1] - obs[n - 1])) for n in range(1, N + 1)]
        geps = np.zeros(self.shape)
        gamp = np.zeros(N)

        def SET(ybar, d):  # S_E^T ybar, and the eps pair of (ybar, d)
            nonlocal geps
            z = self.kron_solve_T(S, "K1", ybar)
            geps = geps - self.block_bilinear(z, d) / eps ** 2
            return S.M_eps.apply(z)

        dbar = SET(ebar[N], ds[N])
        bbar = np.zeros_like(self.b0)
        for n in range(N - 1, -1, -1):
            w = dbar + SET(-a * (S.Dt1 @ bbar), ds[n + 1])     # D^1^T = D~^1
            gamp[n] = -dt * float(self.jhat @ w)
            zb = self.kron_solve_T(S, "Kt1", S.D1 @ w)          # D~^1^T = D^1
            bbar = bbar + dt * S.M_mu.apply(zb)
            y = -a * (S.Dt1 @ bbar)
            if n >= 1:
                y = y + ebar[n]
            dbar = w + SET(y, ds[n])
        return loss, geps, gamp
