"""Prescribed tangential trace of E by a lifting: scheme 2 with inhomogeneous boundary data (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper passages followed:
  * Sec. 3.5: E_h = E_{h,0} + E_{h,b} with E_{h,0} in X^1_{h,0} and the lifting
    E_{h,b} in X^1_h, spanned by the basis functions whose tangential trace is
    not zero and obtained by a local projection of the boundary data onto the
    trace space.  Scheme 2's Hodge star of D becomes the square solve
        (K_1)_0 e_0 = M~^2_{1/eps} d - (K_1)_b e_b ,
    with K_1 = ((K_1)_0  (K_1)_b) the pairing of X~^2 with the whole X^1_h,
    its columns split into interior and boundary functions.  B_h lives in the
    whole X^2_h, D^1 maps X^1_h to X^2_h, and M^2_{1/mu} takes its columns in
    X^2_h while its rows stay the test functions of X^2_{h,0}: these matrices
    are applied, never inverted.
  * Sec. 3.5, scheme 1: with M^1_eps on the whole X^1_h split into blocks,
    the star of D becomes M^1_{eps,00} e_0 = K~_2 d - M^1_{eps,0b} e_b, and
    K_2 in the star of B takes its columns in X^2_h.
  * Sec. 5.1.2: boundary data that is a separable function of space and time
    is lifted once; every step multiplies the lifted coefficient vectors by
    the known functions of time.
  * Time stepping: the kick-drift-kick leapfrog of ``maxwell.Scheme2`` with
    the whole field E_h in both half kicks of B: its boundary part at t_n in
    the first and at t_{n+1} in the second, where the star of D also takes
    e_b(t_{n+1}).

Reading of the local projection (the paper refers to the literature for it):
the data is the tangential trace of the pulled-back 1-form, u^ = J^T E, on the
faces of the parametric cube, projected in the parametric L2 inner product
hierarchically: first along each edge (a 1D projection onto the P1 space along
the edge gives the edge coefficients), then on each face with the edge
coefficients held fixed (a 2D projection per face and tangential component
gives the remaining face coefficients).  The trace of a discrete field is
reproduced exactly.

Index sets: a coefficient of component c of X^1_h (field 'EF') is a boundary
coefficient when its index along one of the two axes other than c is 0 or
n - 1 (the only B-splines of S_p(Xi) that do not vanish on that face); the
others, in their natural order, are the coefficients of X^1_{h,0} (field 'E').
Likewise for X^2_h ('BF') against X^2_{h,0} ('B'), along the axis of the
component.
"""
import numpy as np
import scipy.sparse as sp


from . import forms3d, hodge, maxwell, scheme1, splines


# ---------------------------------------------------------------- index sets

def interior_mask(full_field, c, p, nel):
    """Boolean array (N_z, N_y, N_x) of component c of 'EF' or 'BF': True on interior coefficients."""
    p, nel = forms3d.as3(p), forms3d.as3(nel)
    kinds = forms3d.FIELD_KINDS[full_field][c]
    shape = forms3d.comp_shape(full_field, c, p, nel)
    mask = np.ones(shape, dtype=bool)
    for a in range(3):
        if kinds[a] != "PF":
            continue
        n = splines.space_dim("PF", p[a], nel[a])
        ax = 2 - a  # array axis of parametric axis a (arrays are (z, y, x))
        sl = [slice(None)] * 3
        sl[ax] = 0
        mask[tuple(sl)] = False
        sl[ax] = n - 1
        mask[tuple(sl)] = False
    return mask


def index_sets(full_field, p, nel):
    """(interior, boundary) flat index arrays into a vector of ``full_field``.

    The interior entries, in their order, form the vector of the homogeneous
    space ('E' for 'EF', 'B' for 'BF').
    """
    off = forms3d.comp_offsets(full_field, p, nel)
    inner, bnd = [], []
    for c in range(3):
        m = interior_mask(full_field, c, p, nel).reshape(-1)
        idx = np.arange(m.size) + off[c]
        inner.append(idx[m])
        bnd.append(idx[~m])
    return np.concatenate(inner), np.concatenate(bnd)


# ---------------------------------------------------------------- local projection of the trace

def _axis_view(arr):
    """View of a (N_z, N_y, N_x) component array indexed [x, y, z]."""
    return arr.transpose(2, 1, 0)


def _pulled_back_tangential(geometry, E, pts, c):
    """Component c of u^ = J^T E at parametric points pts = (X, Y, Z) (any common shape)."""
    X, Y, Z = pts
    J = geometry.jacobian(X, Y, Z)
    Ev = np.asarray(E(*geometry(X, Y, Z)))
    return sum(J[k, c] * Ev[k] for k in range(3))


def lift(p, nel, geometry, E, extra=2):
    """Lifting of the tangential trace of the physical 1-form E(x, y, z) -> (3, ...): a vector of X^1_h
    ('EF') whose boundary coefficients come from the hierarchical local projection (edges, then faces)
    and whose interior coefficients are zero."""
    p, nel = forms3d.as3(p), forms3d.as3(nel)
    out = np.zeros(forms3d.field_size("EF", p, nel))
    comps = forms3d.split("EF", out, p, nel)  # views into out
    # 1D rules and bases along each axis (q = p + 1 + extra points per element)
    rule, P1v, PFv, MP1, MPF = {}, {}, {}, {}, {}
    for a in range(3):
        x, w = splines.element_quadrature(nel[a], p[a] + 1 + extra)
        rule[a] = (x, w)
        P1v[a] = splines.space_values("P1", p[a], nel[a], x)
        PFv[a] = splines.space_values("PF", p[a], nel[a], x)
        MP1[a] = P1v[a].T @ (w[:, None] * P1v[a])
        MPF[a] = PFv[a].T @ (w[:, None] * PFv[a])
    # edges: component c along axis c, at the ends of the two other axes
    for c in range(3):
        a1, a2 = (c + 1) % 3, (c + 2) % 3
        n1, n2 = splines.space_dim("PF", p[a1], nel[a1]), splines.space_dim("PF", p[a2], nel[a2])
        x, w = rule[c]
        V = _axis_view(comps[c])
        for s1 in (0, n1 - 1):
            for s2 in (0, n2 - 1):
                pts = [None] * 3
                pts[c] = x
                pts[a1] = np.full_like(x, 0.0 if s1 == 0 else 1.0)
                pts[a2] = np.full_like(x, 0.0 if s2 == 0 else 1.0)
                u = _pulled_back_tangential(geometry, E, pts, c)
                coef = np.linalg.solve(MP1[c], P1v[c].T @ (w * u))
                idx = [None] * 3
                idx[c] = slice(None)
                idx[a1], idx[a2] = s1, s2
                V[tuple(idx)] = coef
    # faces: normal axis a, tangential component c, third axis b; edge coefficients held fixed
    for a in range(3):
        na = splines.space_dim("PF", p[a], nel[a])
        for sa in (0, na - 1):
            for c in ((a + 1) % 3, (a + 2) % 3):
                b = 3 - a - c
                nb = splines.space_dim("PF", p[b], nel[b])
                xc, wc = rule[c]
                xb, wb = rule[b]
                XC, XB = np.meshgrid(xc, xb, indexing="ij")
                pts = [None] * 3
                pts[c], pts[b] = XC, XB
                pts[a] = np.full_like(XC, 0.0 if sa == 0 else 1.0)
                u = _pulled_back_tangential(geometry, E, pts, c)
                # R[j, m] = sum over points of phi^c_j B^b_m u w
                R = P1v[c].T @ (u * wc[:, None] * wb[None, :]) @ PFv[b]
                V = _axis_view(comps[c])
                idx = [None] * 3
                idx[a], idx[c], idx[b] = sa, slice(None), slice(None)
                face = V[tuple(idx)]  # (n_c - 1, n_b): indexed [j along c, m along b]
                if c > b:
                    face = face.T  # keep [j, m] whatever the array order of c and b
                inner = np.arange(1, nb - 1)
                ends = np.array([0, nb - 1])
                # (M_c (x) M_b[inner, inner]) x = R[:, inner] - (M_c (x) M_b[inner, ends]) x_ends
                A = np.kron(MP1[c], MPF[b][np.ix_(inner, inner)])
                rhs = R[:, inner] - MP1[c] @ face[:, ends] @ MPF[b][np.ix_(inner, ends)].T
                sol = np.linalg.solve(A, rhs.reshape(-1)).reshape(MP1[c].shape[0], len(inner))
                face[:, inner] = sol
    return out


# ---------------------------------------------------------------- operators on the whole spaces

class MassToFull:
    """M^2_{1/mu} with rows on X^2_{h,0} ('B') and columns on the whole X^2_h ('BF') (Sec. 3.5).

    The same metric and quadrature as ``hodge.HodgeMass('B', ...)``; only the
    basis the argument is interpolated with changes.
    """

    def __init__(self, p, nel, geometry, mu):
        self.rows = hodge.HodgeMass("B", p, nel, geometry, mu)
        self.p, self.nel = self.rows.p, self.rows.nel
        self.Bcol = [self.rows.grid.basis("BF", c) for c in range(3)]

    def apply(self, x):
        xs = forms3d.split("BF", np.asarray(x, dtype=np.float64), self.p, self.nel)
        U = [hodge.interpolate(*self.Bcol[c], xs[c]) for c in range(3)]
        G = self.rows.G
        ys = []
        for c in range(3):
            V = G[c, 0] * U[0] + G[c, 1] * U[1] + G[c, 2] * U[2]
            ys.append(hodge.integrate(*self.rows.B[c], V))
        return forms3d.join(ys)


def pairing_K1_full(p, nel):
    """K_1 with its columns on the whole X^1_h: block c = Kronecker product of the 1D pairings of the
    D-component kinds (rows) with the 'EF'-component kinds (columns) (Eq. tensor_K, Sec. 3.5)."""
    p, nel = forms3d.as3(p), forms3d.as3(nel)
    blocks = []
    for c in range(3):
        rk, ck = forms3d.FIELD_KINDS["D"][c], forms3d.FIELD_KINDS["EF"][c]
        f = [splines.pairing_1d(rk[a], ck[a], p[a], nel[a]) for a in range(3)]
        blocks.append(forms3d._kron3(f[0], f[1], f[2]))
    return sp.block_diag(blocks, format="csr")


# ---------------------------------------------------------------- the lifted leapfrog

class LiftedScheme2:
    """Scheme 2 with the tangential trace of E prescribed on the whole boundary (Sec. 3.5).

    ``boundary`` is a list of (E_m, g_m): the boundary data is
    sum_m g_m(t) E_m(x) on the boundary, E_m a physical 1-form (callable of the
    physical point, returning (3, ...)) and g_m a function of time (Sec. 5.1.2).
    The state is (d, b, e_0): d on X~^2, b on the whole X^2_h ('BF'), e_0 the
    X^1_{h,0} part of E_h; E_h = e_0 + e_b(t) on X^1_h.
    """

    def __init__(self, p, nel, geometry=None, eps=1.0, mu=1.0, boundary=()):
        self.S = maxwell.Scheme2(p, nel, geometry=geometry, eps=eps, mu=mu)
        self.p, self.nel, self.geometry = self.S.p, self.S.nel, self.S.geometry
        self.D1F = forms3d.curl_matrix("EF", self.p, self.nel)     # X^1_h -> X^2_h
        self.Dt1 = self.S.Dt1
        self.M_mu = MassToFull(self.p, self.nel, self.geometry, mu)
        self.M_eps = self.S.M_eps
        self.e_in, self.e_bd = index_sets("EF", self.p, self.nel)
        self.b_in, self.b_bd = index_sets("BF", self.p, self.nel)
        self.K1b = pairing_K1_full(self.p, self.nel)[:, self.e_bd]
        self.N_ef = forms3d.field_size("EF", self.p, self.nel)
        self.N_bf = forms3d.field_size("BF", self.p, self.nel)
        self.terms = [(lift(self.p, self.nel, self.geometry, Em)[self.e_bd], g) for Em, g in boundary]

    def e_b(self, t):
        """Boundary coefficients of the lifting at time t."""
        out = np.zeros(len(self.e_bd))
        for vec, g in self.terms:
            out = out + g(t) * vec
        return out

    def e_full(self, e0, t):
        """E_h on X^1_h: e_0 on the interior coefficients, e_b(t) on the boundary ones."""
        out = np.zeros(self.N_ef)
        out[self.e_in] = e0
        out[self.e_bd] = self.e_b(t)
        return out

    def e0_from_d(self, d, t):
        """(K_1)_0 e_0 = M~^2_{1/eps} d - (K_1)_b e_b(t), by the 1D sweeps of (K_1)_0 = K_1 (Sec. 3.5)."""
        return self.S.kron_solve("K1", self.M_eps.apply(d) - self.K1b @ self.e_b(t))

    def h_from_b(self, b):
        """K~_1 h = M^2_{1/mu} b with b on the whole X^2_h (Sec. 3.5)."""
        return self.S.kron_solve("Kt1", self.M_mu.apply(b))

    def step(self, d, b, e0, t0, dt, nsteps=1, jhat=None, amps=None):
        """nsteps kick-drift-kick steps from time t0; returns (d, b, e_0, h) (h at the last half step)."""
        d, b, e0 = (np.array(v, dtype=np.float64, copy=True) for v in (d, b, e0))
        h = None
        for n in range(nsteps):
            t = t0 + n * dt
            b = b - 0.5 * dt * (self.D1F @ self.e_full(e0, t))
            h = self.h_from_b(b)
            rhs = self.Dt1 @ h
            if jhat is not None:
                rhs = rhs - amps[n] * jhat
            d = d + dt * rhs
            e0 = self.e0_from_d(d, t + dt)
            b = b - 0.5 * dt * (self.D1F @ self.e_full(e0, t + dt))
        return d, b, e0, h


class LiftedScheme1(LiftedScheme2):
    """Scheme 1 (Sec. 3.3) with the tangential trace of E prescribed (Sec. 3.5); same state and
    time levels as ``LiftedScheme2``.

    Stars: M~^1_mu h = K_2 b with K_2 pairing X~^1 (rows) with the whole X^2_h,
    and M^1_{eps,00} e_0 = K~_2 d - M^1_{eps,0b} e_b(t), both solved directly
    (sparse LU of the assembled interior blocks, as ``scheme1.Scheme1``).
    """

    def __init__(self, p, nel, geometry=None, eps=1.0, mu=1.0, boundary=()):
        super().__init__(p, nel, geometry=geometry, eps=eps, mu=mu, boundary=boundary)
        self.S1 = scheme1.Scheme1(self.p, self.nel, geometry=self.geometry, eps=eps, mu=mu)
        # M^1_eps on the whole X^1_h (rows and columns), then its interior rows
        g = self.S1.M1.grid
        Bf = [g.basis("EF", c) for c in range(3)]
        Bk = [forms3d._kron3(*[sp.csr_matrix(m) for m in Bf[c]]) for c in range(3)]
        G = self.S1.M1.G
        blocks = [[(Bk[c].T @ sp.diags(G[c, c2].reshape(-1)) @ Bk[c2]).tocsr() for c2 in range(3)]
                  for c in range(3)]
        self.M1F = sp.bmat(blocks, format="csr")
        self.M1_0b = self.M1F[self.e_in][:, self.e_bd]
        # K_2: X~^1 rows against the whole X^2_h
        kb = []
        for c in range(3):
            rk, ck = forms3d.FIELD_KINDS["H"][c], forms3d.FIELD_KINDS["BF"][c]
            f = [splines.pairing_1d(rk[a], ck[a], self.p[a], self.nel[a]) for a in range(3)]
            kb.append(forms3d._kron3(f[0], f[1], f[2]))
        self.K2F = sp.block_diag(kb, format="csr")

    def e0_from_d(self, d, t):
        """M^1_{eps,00} e_0 = K~_2 d - M^1_{eps,0b} e_b(t) (Sec. 3.5, scheme 1)."""
        return self.S1._lu_e.solve(self.S1.Kt2 @ np.asarray(d, dtype=np.float64) - self.M1_0b @ self.e_b(t))

    def h_from_b(self, b):
        """M~^1_mu h = K_2 b with b on the whole X^2_h."""
        return self.S1._lu_h.solve(self.K2F @ np.asarray(b, dtype=np.float64))


# ---------------------------------------------------------------- a travelling wave through the cube

def plane_wave(t, k=np.pi):
    """E = (0, sin k(x - t), 0), B = H = D = (0, 0, sin k(x - t)) with eps = mu = 1: an exact solution of
    Maxwell's equations whose tangential E does not vanish on the faces x = 0, 1 and z = 0, 1.
    Returns (E, B) as callables of the physical point."""
    def E(x, y, z):
        return np.array([0.0 * x, np.sin(k * (x - t)), 0.0 * x])

    def B(x, y, z):
        return np.array([0.0 * x, 0.0 * x, np.sin(k * (x - t))])
    return E, B


def plane_wave_boundary(k=np.pi):
    """The plane wave's E as two separable terms: sin k(x - t) = sin kx cos kt - cos kx sin kt."""
    def E1(x, y, z):
        return np.array([0.0 * x, np.sin(k * x), 0.0 * x])

    def E2(x, y, z):
        return np.array([0.0 * x, np.cos(k * x), 0.0 * x])
    return [(E1, lambda t: np.cos(k * t)), (E2, lambda t: -np.sin(k * t))]


# ---------------------------------------------------------------- the TEM mode of the coaxial cable

def coax_tem(t, k=np.pi):
    """TEM mode of a coaxial line along z with eps = mu = 1 (Sec. 5.1.2; the textbook mode):
    E = (x, y, 0) / r^2 sin k(z - t), B = H = (-y, x, 0) / r^2 sin k(z - t).  E is normal to the
    cylinders r = const (PEC there) and tangential to the planes x = 0, y = 0 and z = const, where
    the lifting carries it.  Returns (E, B) as callables of the physical point."""
    def E(x, y, z):
        s = np.sin(k * (z - t)) / (x * x + y * y)
        return np.array([x * s, y * s, 0.0 * x])

    def B(x, y, z):
        s = np.sin(k * (z - t)) / (x * x + y * y)
        return np.array([-y * s, x * s, 0.0 * x])
    return E, B


def coax_tem_boundary(k=np.pi):
    """The TEM mode's E as two separable terms: sin k(z - t) = sin kz cos kt - cos kz sin kt."""
    def E1(x, y, z):
        s = np.sin(k * z) / (x * x + y * y)
        return np.array([x * s, y * s, 0.0 * x])

    def E2(x, y, z):
        s = np.cos(k * z) / (x * x + y * y)
        return np.array([x * s, y * s, 0.0 * x])
    return [(E1, lambda t: np.cos(k * t)), (E2, lambda t: -np.sin(k * t))]
