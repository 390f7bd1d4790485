"""Tensor-product primal and dual complexes in 3D (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper passages followed:
  * Sec. 2.3, Eq. cd-iga-tp-drchlt / Eq. cd-iga-tp-nmnn: primal complex of
    mixed degree p, p-1 with homogeneous BC, dual complex of degree p-1, p-2.
  * Sec. 2.4 (field placement): E in X^1_{h,0}, B in X^2_{h,0}, H in X~^1,
    D in X~^2.
  * Sec. 2.4 (pairing matrices) and Sec. 4.1, Eq. tensor_K, Eq. tensor_Ktilde:
    K_1 = blockdiag(C_1, C_2, C_3), C_1 = G^3 (x) G^2 (x) M^1, ... and
    K~_1 = blockdiag of the transposed factors.
  * Sec. 4.2, vec convention: the first direction (x) runs fastest, so a
    Kronecker product A_z (x) A_y (x) A_x acts on a component stored as a
    C-ordered array of shape (N_z, N_y, N_x).
  * Remark on incidence matrices after Table 1: D^k and D~^k are Kronecker
    products of 1D incidence matrices and identities.
  * Sec. 3.5: with a prescribed tangential trace of E, E_h and B_h live in the
    whole X^1_h and X^2_h ('EF', 'BF': the 'PF' kind in place of 'P0') and
    D^1 maps X^1_h to X^2_h.

Component k of a 2-form is the coefficient of dy^dz, dz^dx, dx^dy for
k = 0, 1, 2; component k of a 1-form is that of dx, dy, dz.  A global vector
concatenates the three components, each flattened with x fastest.
"""
import numpy as np
import scipy.sparse as sp

from . import splines

# univariate space kind per axis (x, y, z) for each component of each field
FIELD_KINDS = {
    "E": (("P1", "P0", "P0"), ("P0", "P1", "P0"), ("P0", "P0", "P1")),
    "B": (("P0", "P1", "P1"), ("P1", "P0", "P1"), ("P1", "P1", "P0")),
    "H": (("D1", "D0", "D0"), ("D0", "D1", "D0"), ("D0", "D0", "D1")),
    "D": (("D0", "D1", "D1"), ("D1", "D0", "D1"), ("D1", "D1", "D0")),
    # the whole primal spaces X^1_h, X^2_h (boundary functions kept, Sec. 3.5)
    "EF": (("P1", "PF", "PF"), ("PF", "P1", "PF"), ("PF", "PF", "P1")),
    "BF": (("PF", "P1", "P1"), ("P1", "PF", "P1"), ("P1", "P1", "PF")),
    # 3-forms (targets of the divergence), single component
    "B3": (("P1", "P1", "P1"),),
    "D3": (("D1", "D1", "D1"),),
}


def as3(v):
    v = tuple(int(a) for a in np.broadcast_to(np.asarray(v), (3,)))
    return v


def comp_shape(field, c, p, nel):
    """Array shape (N_z, N_y, N_x) of component c of a field."""
    p, nel = as3(p), as3(nel)
    kinds = FIELD_KINDS[field][c]
    return tuple(splines.space_dim(kinds[a], p[a], nel[a]) for a in (2, 1, 0))


def comp_sizes(field, p, nel):
    return [int(np.prod(comp_shape(field, c, p, nel))) for c in range(len(FIELD_KINDS[field]))]


def comp_offsets(field, p, nel):
    s = comp_sizes(field, p, nel)
    return list(np.concatenate([[0], np.cumsum(s)]).astype(np.int64))


def field_size(field, p, nel):
    return int(sum(comp_sizes(field, p, nel)))


def split(field, v, p, nel):
    """Split a global vector into per-component arrays of shape (N_z, N_y, N_x)."""
    off = comp_offsets(field, p, nel)
    return [v[off[c]:off[c + 1]].reshape(comp_shape(field, c, p, nel)) for c in range(len(off) - 1)]


def join(parts):
    return np.concatenate([np.asarray(a).reshape(-1) for a in parts])


def _kron3(Ax, Ay, Az):
    """Az (x) Ay (x) Ax as a sparse matrix (x fastest)."""
    out = sp.kron(sp.csr_matrix(Az), sp.kron(sp.csr_matrix(Ay), sp.csr_matrix(Ax)), format="csr")
    out.eliminate_zeros()
    return out


def _axis_operator(op1d, axis, in_kinds, p, nel):
    """Apply a 1D operator along one axis and the identity along the other two."""
    mats = []
    for a in range(3):
        if a == axis:
            mats.append(sp.csr_matrix(op1d))
        else:
            mats.append(sp.identity(splines.space_dim(in_kinds[a], p[a], nel[a]), format="csr"))
    return _kron3(mats[0], mats[1], mats[2])


def _derivative_1d(kind, p, nel):
    if kind == "P0":
        return splines.incidence_primal(p, nel)
    if kind == "PF":
        return splines.incidence_full(p, nel)
    if kind == "D0":
        return splines.incidence_dual(p, nel)
    raise ValueError("no derivative from kind " + kind)


def curl_matrix(src, p, nel):
    """3D incidence for the curl: D^1 (src='E', E -> B; src='EF', X^1_h -> X^2_h) or D~^1 (src='H', H -> D).

    (curl u)_c = d_{c+1} u_{c+2} - d_{c+2} u_{c+1}, indices mod 3
    (Eq. maxwell_discrete; Remark on incidence matrices after Table 1).
    """
    p, nel = as3(p), as3(nel)
    kinds = FIELD_KINDS[src]
    dst = {"E": "B", "H": "D", "EF": "BF"}[src]
    in_sizes = comp_sizes(src, p, nel)
    out_sizes = comp_sizes(dst, p, nel)
    blocks = [[None] * 3 for _ in range(3)]
    for c in range(3):
        for c_in in range(3):
            blocks[c][c_in] = sp.csr_matrix((out_sizes[c], in_sizes[c_in]))
        a1, a2 = (c + 1) % 3, (c + 2) % 3
        # + d_{a1} u_{a2}
        d1 = _derivative_1d(kinds[a2][a1], p[a1], nel[a1])
        blocks[c][a2] = blocks[c][a2] + _axis_operator(d1, a1, kinds[a2], p, nel)
        # - d_{a2} u_{a1}
        d2 = _derivative_1d(kinds[a1][a2], p[a2], nel[a2])
        blocks[c][a1] = blocks[c][a1] - _axis_operator(d2, a2, kinds[a1], p, nel)
    out = sp.bmat(blocks, format="csr")
    out.eliminate_zeros()
    return out


def grad_matrix(p, nel, dual=False, full=False):
    """3D incidence D^0 (primal, 0-forms of S_p,0^3 -> E; full=True: S_p^3 -> X^1_h) or D~^0 (dual, S_{p-1}^3 -> H)."""
    p, nel = as3(p), as3(nel)
    k0 = "D0" if dual else ("PF" if full else "P0")
    kinds0 = (k0, k0, k0)
    dst = "H" if dual else ("EF" if full else "E")
    rows = []
    for c in range(3):
        d = _derivative_1d(k0, p[c], nel[c])
        rows.append([_axis_operator(d, c, kinds0, p, nel)])
    out = sp.bmat(rows, format="csr")
    out.eliminate_zeros()
    assert out.shape[0] == field_size(dst, p, nel)
    return out


def div_matrix(src, p, nel):
    """3D incidence for the divergence: D^2 (src='B') or D~^2 (src='D'); div u = sum_c d_c u_c."""
    p, nel = as3(p), as3(nel)
    kinds = FIELD_KINDS[src]
    blocks = []
    for c in range(3):
        d = _derivative_1d(kinds[c][c], p[c], nel[c])
        blocks.append(_axis_operator(d, c, kinds[c], p, nel))
    out = sp.hstack(blocks, format="csr")
    out.eliminate_zeros()
    return out


def pairing_factor(row_kind, col_kind, p, nel):
    """The univariate factor of a pairing block: G-hat, M-hat or a transpose (Sec. 4.1)."""
    name, transposed = splines.pairing_kind(row_kind, col_kind)
    A = splines.G_hat(p, nel) if name == "G" else splines.M_hat(p, nel)
    return A.T if transposed else A


def pairing_factors(which, c, p, nel):
    """1D factors (x, y, z) of block c of K_1 (which='K1') or K~_1 (which='Kt1').

    K_1 pairs X~^2 (rows, field D) with X^1_{h,0} (columns, field E), Eq. tensor_K;
    K~_1 pairs X^2_{h,0} (rows, field B) with X~^1 (columns, field H), Eq. tensor_Ktilde.
    """
    p, nel = as3(p), as3(nel)
    row_field, col_field = {"K1": ("D", "E"), "Kt1": ("B", "H")}[which]
    rk, ck = FIELD_KINDS[row_field][c], FIELD_KINDS[col_field][c]
    return [pairing_factor(rk[a], ck[a], p[a], nel[a]) for a in range(3)]


def pairing_block(which, c, p, nel):
    f = pairing_factors(which, c, p, nel)
    return _kron3(f[0], f[1], f[2])


def pairing_matrix(which, p, nel):
    """K_1 or K~_1 assembled as a block-diagonal sparse matrix (Sec. 4.1)."""
    return sp.block_diag([pairing_block(which, c, p, nel) for c in range(3)], format="csr")
