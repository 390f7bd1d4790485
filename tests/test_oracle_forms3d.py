"""Pins of the oracle's 3D complexes, incidence and pairing matrices (Sec. 2.3-2.4, Sec. 4.1).

* dim X^k_{h,0} = dim X~^{3-k} (Sec. 2.3, after Eq. cd-iga-tp-nmnn);
* d o d = 0 exactly, in integers (Sec. 2.1, Sec. 3.1);
* discrete integration by parts, Eq. disc_int_by_parts2 for k = 1, 2, 3 with
  the signs (-1)^{4-k}, and Eq. pairing_transpose K~_1 = K_2^T;
* the Kronecker blocks of K_1 and K~_1 (Eq. tensor_K, Eq. tensor_Ktilde)
  against a brute-force wedge integral over the 3D mesh (explicit loops).
"""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import forms3d, splines

MESHES = [((2, 2, 2), (2, 2, 2)), ((3, 2, 4), (3, 2, 1)), ((2, 3, 3), (1, 2, 3)), ((4, 4, 4), (2, 2, 2))]


@pytest.mark.parametrize("p,nel", MESHES)
def test_dimensions_pair(p, nel):
    assert forms3d.field_size("E", p, nel) == forms3d.field_size("D", p, nel)
    assert forms3d.field_size("B", p, nel) == forms3d.field_size("H", p, nel)
    for c in range(3):
        assert forms3d.comp_shape("E", c, p, nel) == forms3d.comp_shape("D", c, p, nel)
        assert forms3d.comp_shape("B", c, p, nel) == forms3d.comp_shape("H", c, p, nel)


@pytest.mark.parametrize("p,nel", MESHES)
def test_d_of_d_is_zero_exactly(p, nel):
    for dual in (False, True):
        G = forms3d.grad_matrix(p, nel, dual=dual)
        C = forms3d.curl_matrix("H" if dual else "E", p, nel)
        Dv = forms3d.div_matrix("D" if dual else "B", p, nel)
        for A in (G, C, Dv):
            assert set(np.unique(A.data)) <= {-1.0, 1.0}  # integer +-1 incidence
        assert abs(C @ G).max() == 0.0
        assert abs(Dv @ C).max() == 0.0


def _k0(p, nel):
    return forms3d._kron3(*[splines.G_hat(p[a], nel[a]) for a in range(3)])


def _k3(p, nel):
    return forms3d._kron3(*[splines.M_hat(p[a], nel[a]) for a in range(3)])


@pytest.mark.parametrize("p,nel", MESHES)
def test_integration_by_parts(p, nel):
    """(D~^{3-k})^T K_{k-1} = (-1)^{4-k} K_k D^{k-1}, k = 1, 2, 3 (Eq. disc_int_by_parts2)."""
    K1 = forms3d.pairing_matrix("K1", p, nel)
    K2 = forms3d.pairing_matrix("Kt1", p, nel).T   # Eq. pairing_transpose
    K0, K3 = _k0(p, nel), _k3(p, nel)
    D0, D1, D2 = forms3d.grad_matrix(p, nel), forms3d.curl_matrix("E", p, nel), forms3d.div_matrix("B", p, nel)
    Dt0, Dt1, Dt2 = forms3d.grad_matrix(p, nel, True), forms3d.curl_matrix("H", p, nel), forms3d.div_matrix("D", p, nel)
    tol = 1e-14 * max(nel) * 10
    assert abs(Dt2.T @ K0 + K1 @ D0).max() < tol       # k = 1: sign (-1)^3
    assert abs(Dt1.T @ K1 - K2 @ D1).max() < tol       # k = 2: sign (-1)^2
    assert abs(Dt0.T @ K2 + K3 @ D2).max() < tol       # k = 3: sign (-1)^1


def _brute_pairing(row_field, col_field, p, nel):
    """int (row basis) . (col basis) over (0,1)^3 by loops over elements and Gauss points."""
    q = max(p) + 2
    z, w = splines.gauss_legendre_01(q)
    sizes_r = forms3d.comp_sizes(row_field, p, nel)
    sizes_c = forms3d.comp_sizes(col_field, p, nel)
    K = np.zeros((sum(sizes_r), sum(sizes_c)))
    ro, co = forms3d.comp_offsets(row_field, p, nel), forms3d.comp_offsets(col_field, p, nel)
    for c in range(3):
        rk, ck = forms3d.FIELD_KINDS[row_field][c], forms3d.FIELD_KINDS[col_field][c]
        rs, cs = forms3d.comp_shape(row_field, c, p, nel), forms3d.comp_shape(col_field, c, p, nel)
        for ez, ey, ex in itertools.product(range(nel[2]), range(nel[1]), range(nel[0])):
            for qz, qy, qx in itertools.product(range(q), range(q), range(q)):
                pt = ((ex + z[qx]) / nel[0], (ey + z[qy]) / nel[1], (ez + z[qz]) / nel[2])
                wt = w[qx] * w[qy] * w[qz] / (nel[0] * nel[1] * nel[2])
                vr = [splines.space_values(rk[a], p[a], nel[a], [pt[a]])[0] for a in range(3)]
                vc = [splines.space_values(ck[a], p[a], nel[a], [pt[a]])[0] for a in range(3)]
                for (k, j, i) in itertools.product(range(rs[0]), range(rs[1]), range(rs[2])):
                    fr = vr[2][k] * vr[1][j] * vr[0][i]
                    if fr == 0.0:
                        continue
                    row = ro[c] + (k * rs[1] + j) * rs[2] + i
                    for (kk, jj, ii) in itertools.product(range(cs[0]), range(cs[1]), range(cs[2])):
                        fc = vc[2][kk] * vc[1][jj] * vc[0][ii]
                        if fc != 0.0:
                            K[row, co[c] + (kk * cs[1] + jj) * cs[2] + ii] += wt * fr * fc
    return K


@pytest.mark.parametrize("p,nel", [((2, 2, 2), (2, 1, 2)), ((3, 2, 2), (1, 2, 1))])
def test_pairing_blocks_vs_wedge_integral(p, nel):
    K1 = forms3d.pairing_matrix("K1", p, nel).toarray()
    Kt1 = forms3d.pairing_matrix("Kt1", p, nel).toarray()
    np.testing.assert_allclose(K1, _brute_pairing("D", "E", p, nel), atol=1e-14)
    np.testing.assert_allclose(Kt1, _brute_pairing("B", "H", p, nel), atol=1e-14)


def test_curl_layout_explicit():
    """The first row block of D^1 is  d_y E_z - d_z E_y  with x fastest (Eq. maxwell_discrete)."""
    p, nel = (2, 3, 2), (2, 2, 3)
    D1 = forms3d.curl_matrix("E", p, nel)
    rng = np.random.default_rng(5)
    e = rng.standard_normal(forms3d.field_size("E", p, nel))
    Ex, Ey, Ez = forms3d.split("E", e, p, nel)
    Bx = forms3d.split("B", D1 @ e, p, nel)[0]
    Nz, Ny, Nx = Bx.shape
    ref = np.zeros_like(Bx)
    for k in range(Nz):
        for j in range(Ny):
            for i in range(Nx):
                # primal incidence: (d c)_j = c_j - c_{j-1}, entries outside the BC range are zero
                ezj = Ez[k, j, i] if j < Ez.shape[1] else 0.0
                ezm = Ez[k, j - 1, i] if j - 1 >= 0 else 0.0
                eyk = Ey[k, j, i] if k < Ey.shape[0] else 0.0
                eym = Ey[k - 1, j, i] if k - 1 >= 0 else 0.0
                ref[k, j, i] = (ezj - ezm) - (eyk - eym)
    np.testing.assert_allclose(Bx, ref, rtol=0, atol=4e-16 * np.abs(e).max())
