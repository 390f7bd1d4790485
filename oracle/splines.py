"""Univariate spline spaces of the primal and dual complexes (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper passages followed:
  * Sec. 2.3: p-open knot vector Xi; Xi' and Xi'' drop the first and last
    knot once and twice; S_p(Xi) -> S_{p-1}(Xi') -> S_{p-2}(Xi'') by
    differentiation; homogeneous boundary conditions drop the first and last
    function of S_p(Xi).
  * Sec. 4.1 (after Eq. tensor_K's scalar form): scaled Curry-Schoenberg (CS)
    basis for the primal S_{p-1}(Xi') and the dual S_{p-2}(Xi''), standard
    B-splines for the primal S_p(Xi) and the dual S_{p-1}(Xi'); with that
    choice differentiation is a +-1 incidence matrix (Remark after
    Table 1 on incidence matrices).
  * Sec. 4.1: G-hat pairs the dual S_{p-2}(Xi'') (rows) with the primal
    S_p(Xi) (columns); M-hat pairs the dual S_{p-1}(Xi') (rows, B-splines)
    with the primal S_{p-1}(Xi') (columns, CS).
  * Sec. 5: maximal smoothness (simple interior knots), uniform elements.

The four univariate space kinds are named after where they sit in 3D:
  'P0'  primal S_p(Xi) with the two boundary functions removed (B-splines)
  'P1'  primal S_{p-1}(Xi')  (Curry-Schoenberg)
  'D0'  dual   S_{p-1}(Xi')  (B-splines)
  'D1'  dual   S_{p-2}(Xi'') (Curry-Schoenberg)
With n = nel + p: dim P0 = n-2, dim P1 = n-1, dim D0 = n-1, dim D1 = n-2.
A fifth kind, 'PF', is the whole primal S_p(Xi) (n B-splines, boundary
functions kept): the spaces X^1_h and X^2_h of Sec. 3.5, where the tangential
trace of E is prescribed by a lifting instead of set to zero.  Function 0
(n-1) is the only one that is nonzero at x = 0 (x = 1).
"""
import numpy as np

SPACE_KINDS = ("P0", "P1", "D0", "D1", "PF")


def open_knot_vector(p, nel):
    """Uniform p-open knot vector on [0,1] with simple interior knots (Sec. 2.3, Sec. 5)."""
    if p < 2 or nel < 1:
        raise ValueError("need p >= 2 and nel >= 1")
    inner = np.arange(1, nel, dtype=np.float64) / nel
    return np.concatenate([np.zeros(p + 1), inner, np.ones(p + 1)])


def bspline_values(knots, degree, x):
    """All B-splines of the given degree on ``knots`` at points ``x``.

    Plain Cox-de Boor recursion (textbook definition).  Returns an array of
    shape (len(x), len(knots) - degree - 1).  Points are expected strictly
    inside (0,1) or at interior non-knot positions; a point equal to 1 is
    assigned to the last non-empty knot span.
    """
    t = np.asarray(knots, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    m = len(t) - 1  # number of knot spans (possibly empty)
    B = np.zeros((len(x), m))
    for s in range(m):
        if t[s] < t[s + 1]:
            inside = (x >= t[s]) & (x < t[s + 1])
            B[inside, s] = 1.0
    # right end: x == last knot belongs to the last non-empty span
    last = max(s for s in range(m) if t[s] < t[s + 1])
    B[x == t[-1], last] = 1.0
    for k in range(1, degree + 1):
        Bn = np.zeros((len(x), m - k))
        for i in range(m - k):
            left_den = t[i + k] - t[i]
            right_den = t[i + k + 1] - t[i + 1]
            if left_den > 0:
                Bn[:, i] += (x - t[i]) / left_den * B[:, i]
            if right_den > 0:
                Bn[:, i] += (t[i + k + 1] - x) / right_den * B[:, i + 1]
        B = Bn
    return B


def curry_schoenberg_values(knots, degree, x):
    """Curry-Schoenberg basis: B-splines scaled by (k+1)/(t_{i+k+1}-t_i), each integrates to 1."""
    t = np.asarray(knots, dtype=np.float64)
    B = bspline_values(t, degree, x)
    nf = B.shape[1]
    scale = np.array([(degree + 1) / (t[i + degree + 1] - t[i]) for i in range(nf)])
    return B * scale[None, :]


def space_degree(kind, p):
    return {"P0": p, "P1": p - 1, "D0": p - 1, "D1": p - 2, "PF": p}[kind]


def space_dim(kind, p, nel):
    n = nel + p
    return {"P0": n - 2, "P1": n - 1, "D0": n - 1, "D1": n - 2, "PF": n}[kind]


def space_values(kind, p, nel, x):
    """Values of the basis of one univariate space kind at points x, shape (len(x), dim)."""
    xi = open_knot_vector(p, nel)
    if kind == "P0":
        return bspline_values(xi, p, x)[:, 1:-1]
    if kind == "PF":
        return bspline_values(xi, p, x)
    if kind == "P1":
        return curry_schoenberg_values(xi[1:-1], p - 1, x)
    if kind == "D0":
        return bspline_values(xi[1:-1], p - 1, x)
    if kind == "D1":
        return curry_schoenberg_values(xi[2:-2], p - 2, x)
    raise ValueError(kind)


def gauss_legendre_01(q):
    """q-point Gauss-Legendre rule on [0,1] (library routine numpy.polynomial.legendre.leggauss)."""
    z, w = np.polynomial.legendre.leggauss(q)
    return 0.5 * (z + 1.0), 0.5 * w


def element_quadrature(nel, q):
    """Per-element q-point Gauss rule on the uniform mesh of [0,1]: points and weights, element-major."""
    z, w = gauss_legendre_01(q)
    h = 1.0 / nel
    pts = (np.arange(nel)[:, None] + z[None, :]) * h
    wts = np.broadcast_to(w[None, :] * h, (nel, q))
    return pts.reshape(-1), np.array(wts).reshape(-1)


def pairing_1d(row_kind, col_kind, p, nel, q=None):
    """Univariate pairing (Gram) matrix  int_0^1 phi_i psi_j dx  between two space kinds.

    Sec. 4.1: G-hat = pairing_1d('D1', 'P0'), M-hat = pairing_1d('D0', 'P1').
    Element-wise Gauss quadrature with q = p+1 points is exact for these
    piecewise polynomials (degree at most 2p).
    """
    q = p + 1 if q is None else q
    x, w = element_quadrature(nel, q)
    R = space_values(row_kind, p, nel, x)
    C = space_values(col_kind, p, nel, x)
    return R.T @ (w[:, None] * C)


def G_hat(p, nel):
    """G-hat of Sec. 4.1: dual S_{p-2}(Xi'') CS rows x primal S_p(Xi) (BC removed) columns."""
    return pairing_1d("D1", "P0", p, nel)


def M_hat(p, nel):
    """M-hat of Sec. 4.1: dual S_{p-1}(Xi') B-spline rows x primal S_{p-1}(Xi') CS columns."""
    return pairing_1d("D0", "P1", p, nel)


def mass_1d(kind, p, nel):
    """Univariate L2 mass matrix of one space kind (used to check the Hodge closed form)."""
    return pairing_1d(kind, kind, p, nel)


def incidence_primal(p, nel):
    """1D derivative P0 -> P1 in the chosen bases: (d c)_j = c_j - c_{j-1}, BC entries zero.

    Shape (n-1, n-2).  Derivation: d/dx B_{i,p} = D_{i-1} - D_i with D the CS
    basis of S_{p-1}(Xi') (Remark on incidence matrices after Table 1;
    Sec. 4.1 basis choice).
    """
    n = nel + p
    Dm = np.zeros((n - 1, n - 2))
    for j in range(n - 1):
        if j < n - 2:
            Dm[j, j] = 1.0
        if j - 1 >= 0:
            Dm[j, j - 1] = -1.0
    return Dm


def incidence_full(p, nel):
    """1D derivative PF -> P1 on the whole S_p(Xi): (d c)_k = c_{k+1} - c_k.  Shape (n-1, n).

    The same identity d/dx B_{i,p} = D_{i-1} - D_i as ``incidence_primal``, with
    the boundary functions kept (Sec. 3.5: D^1 between X^1_h and X^2_h).
    ``incidence_primal`` is this matrix without its first and last column.
    """
    n = nel + p
    Dm = np.zeros((n - 1, n))
    for k in range(n - 1):
        Dm[k, k + 1] = 1.0
        Dm[k, k] = -1.0
    return Dm


def incidence_dual(p, nel):
    """1D derivative D0 -> D1 in the chosen bases: (d c)_k = c_{k+1} - c_k.  Shape (n-2, n-1)."""
    n = nel + p
    Dm = np.zeros((n - 2, n - 1))
    for k in range(n - 2):
        Dm[k, k + 1] = 1.0
        Dm[k, k] = -1.0
    return Dm


def pairing_kind(row_kind, col_kind):
    """Which univariate pairing a (row kind, column kind) pair is, as (name, transposed)."""
    table = {
        ("D1", "P0"): ("G", False),
        ("D0", "P1"): ("M", False),
        ("P0", "D1"): ("G", True),
        ("P1", "D0"): ("M", True),
    }
    return table[(row_kind, col_kind)]
