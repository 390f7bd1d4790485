"""Geometry map, materials and the discrete Hodge mass matrices (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper passages followed:
  * Sec. 2.3: single-patch map F : (0,1)^3 -> Omega and the pullback of
    k-forms.  For 2-forms the vector proxy pulls back with the Piola rule
    v = J v^ / det J, for 1-forms with u = J^{-T} u^ (J = DF).
  * Sec. 3.4, Eq. discrete2_hodge_eps / Eq. discrete2_hodge_mu: the mass
    matrices of the 2-form spaces, M~^2_{1/eps} on X~^2 (field D) and
    M^2_{1/mu} on X^2_{h,0} (field B).  Entry (i, j) is
        int_Omega gamma  v_i . v_j dx
      = int_(0,1)^3 gamma(F(x^)) v^_i^T (J^T J / det J) v^_j dx^ ,
    gamma = 1/eps or 1/mu.
  * Quadrature: q = p+1 Gauss-Legendre points per element and direction
    (the paper does not state the rule; this reading is exact for the
    identity map with element-wise constant material).

The mass apply writes the definition out: interpolate the tensor-product
basis at the quadrature points (einsum over the three 1D evaluation matrices),
multiply by weight x metric, integrate back against the same basis.
"""
import numpy as np
import scipy.sparse as sp

from . import forms3d, splines


# ---------------------------------------------------------------- geometry

class IdentityMap:
    """F(x^) = x^ (the unit-cube cavity of Sec. 5.1.1)."""

    def __call__(self, X, Y, Z):
        return X, Y, Z

    def jacobian(self, X, Y, Z):
        J = np.zeros((3, 3) + np.shape(X))
        for a in range(3):
            J[a, a] = 1.0
        return J


class SineBumpMap:
    """F_i(x^) = x^_i + a sin(pi x^) sin(pi y^) sin(pi z^): maps the unit cube onto itself.

    J_ij = delta_ij + a dS/dx^_j with S = sin(pi x^) sin(pi y^) sin(pi z^).
    """

    def __init__(self, amplitude=0.05):
        self.a = float(amplitude)

    def __call__(self, X, Y, Z):
        S = np.sin(np.pi * X) * np.sin(np.pi * Y) * np.sin(np.pi * Z)
        return X + self.a * S, Y + self.a * S, Z + self.a * S

    def jacobian(self, X, Y, Z):
        sx, sy, sz = np.sin(np.pi * X), np.sin(np.pi * Y), np.sin(np.pi * Z)
        cx, cy, cz = np.cos(np.pi * X), np.cos(np.pi * Y), np.cos(np.pi * Z)
        g = [np.pi * cx * sy * sz, np.pi * sx * cy * sz, np.pi * sx * sy * cz]
        J = np.zeros((3, 3) + np.shape(X))
        for i in range(3):
            for j in range(3):
                J[i, j] = (1.0 if i == j else 0.0) + self.a * g[j]
        return J


def det3(J):
    return (J[0, 0] * (J[1, 1] * J[2, 2] - J[1, 2] * J[2, 1])
            - J[0, 1] * (J[1, 0] * J[2, 2] - J[1, 2] * J[2, 0])
            + J[0, 2] * (J[1, 0] * J[2, 1] - J[1, 1] * J[2, 0]))


# ---------------------------------------------------------------- material

def material_at(spec, Xp, Yp, Zp, elem_index, nel):
    """Material value at quadrature points.

    spec: a number (constant), ('blocks', array (b_z, b_y, b_x)) piecewise
    constant on a grid of element blocks aligned with the parametric mesh
    (nel divisible by the block counts), or a callable of the physical point
    (vectorised).  elem_index = (ez, ey, ex) index arrays of each point.
    """
    if callable(spec):
        return np.asarray(spec(Xp, Yp, Zp), dtype=np.float64) * np.ones_like(Xp)
    if isinstance(spec, tuple) and spec[0] == "blocks":
        vals = np.asarray(spec[1], dtype=np.float64)
        bz, by, bx = vals.shape
        ez, ey, ex = elem_index
        nel = forms3d.as3(nel)
        if nel[0] % bx or nel[1] % by or nel[2] % bz:
            raise ValueError("block grid must align with the elements")
        return vals[ez // (nel[2] // bz), ey // (nel[1] // by), ex // (nel[0] // bx)]
    return float(spec) * np.ones_like(Xp)


# ---------------------------------------------------------------- quadrature grid

class QuadGrid:
    """Tensor-product Gauss grid: q_a = p_a + 1 points per element along axis a (plus ``extra``)."""

    def __init__(self, p, nel, geometry, extra=0):
        self.p, self.nel = forms3d.as3(p), forms3d.as3(nel)
        self.q = tuple(self.p[a] + 1 + extra for a in range(3))
        self.pts, self.wts, self.elem = [], [], []
        for a in range(3):
            x, w = splines.element_quadrature(self.nel[a], self.q[a])
            self.pts.append(x)
            self.wts.append(w)
            self.elem.append(np.arange(len(x)) // self.q[a])
        Z, Y, X = np.meshgrid(self.pts[2], self.pts[1], self.pts[0], indexing="ij")
        self.X, self.Y, self.Z = X, Y, Z
        EZ, EY, EX = np.meshgrid(self.elem[2], self.elem[1], self.elem[0], indexing="ij")
        self.elem_index = (EZ, EY, EX)
        self.W = self.wts[2][:, None, None] * self.wts[1][None, :, None] * self.wts[0][None, None, :]
        self.geometry = geometry
        self.J = geometry.jacobian(X, Y, Z)
        self.detJ = det3(self.J)
        if np.any(self.detJ <= 0):
            raise ValueError("map is not orientation preserving at some quadrature point")
        self.phys = geometry(X, Y, Z)

    def basis(self, field, c):
        """1D evaluation matrices (x, y, z) of component c's basis at the grid points."""
        kinds = forms3d.FIELD_KINDS[field][c]
        return [splines.space_values(kinds[a], self.p[a], self.nel[a], self.pts[a]) for a in range(3)]


def interpolate(Bx, By, Bz, Xc):
    """Values of sum_kji X[k,j,i] phi^z_k phi^y_j phi^x_i at the grid: shape (Qz, Qy, Qx)."""
    return np.einsum("zk,yj,xi,kji->zyx", Bz, By, Bx, Xc, optimize=True)


def integrate(Bx, By, Bz, V):
    """Transpose of ``interpolate``: sum over grid points of V times each basis function."""
    return np.einsum("zk,yj,xi,zyx->kji", Bz, By, Bx, V, optimize=True)


# ---------------------------------------------------------------- Hodge mass

class HodgeMass:
    """Mass matrix of the 2-form space of ``field`` ('B': X^2_{h,0}, 'D': X~^2, 'BF': the whole X^2_h
    of Sec. 3.5) weighted by gamma.

    gamma is 1/mu for B (Eq. discrete2_hodge_mu) and 1/eps for D
    (Eq. discrete2_hodge_eps); ``gamma_spec`` is given as the material
    (mu or eps), and the reciprocal is taken here.
    """

    def __init__(self, field, p, nel, geometry, material_spec, invert=True):
        assert field in ("B", "D", "BF")
        self.field = field
        self.p, self.nel = forms3d.as3(p), forms3d.as3(nel)
        g = QuadGrid(self.p, self.nel, geometry)
        self.grid = g
        mat = material_at(material_spec, *g.phys, g.elem_index, self.nel)
        if np.any(~np.isfinite(mat)) or np.any(mat <= 0):
            raise ValueError("material must be finite and positive")
        gamma = 1.0 / mat if invert else mat
        J = g.J
        JtJ = np.einsum("ki...,kj...->ij...", J, J)
        # G_cc' = w * gamma * (J^T J)_cc' / det J at every grid point
        self.G = JtJ * (gamma * g.W / g.detJ)[None, None]
        self.B = [g.basis(field, c) for c in range(3)]
        self.shapes = [forms3d.comp_shape(field, c, self.p, self.nel) for c in range(3)]

    def apply(self, x):
        """y = M x, matrix-free (definition of the mass entries, Sec. 3.4)."""
        xs = forms3d.split(self.field, np.asarray(x, dtype=np.float64), self.p, self.nel)
        U = [interpolate(*self.B[c], xs[c]) for c in range(3)]
        ys = []
        for c in range(3):
            V = self.G[c, 0] * U[0] + self.G[c, 1] * U[1] + self.G[c, 2] * U[2]
            ys.append(integrate(*self.B[c], V))
        return forms3d.join(ys)

    def matrix(self):
        """Assembled sparse M = sum_cc' B_c^T diag(G_cc') B_c' (small meshes only)."""
        Bk = [forms3d._kron3(*[sp.csr_matrix(m) for m in self.B[c]]) for c in range(3)]
        blocks = [[None] * 3 for _ in range(3)]
        for c in range(3):
            for c2 in range(3):
                blocks[c][c2] = (Bk[c].T @ sp.diags(self.G[c, c2].reshape(-1)) @ Bk[c2]).tocsr()
        return sp.bmat(blocks, format="csr")
