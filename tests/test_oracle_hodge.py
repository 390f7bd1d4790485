"""Pins of the oracle's Hodge mass matrices (Sec. 3.4, 2-form pullback of Sec. 2.3).

* identity map, constant material: M equals gamma times the Kronecker product of
  univariate mass matrices of each component's spaces (closed form);
* identity map, block-constant material: the sum over blocks of the same
  Kronecker products restricted to the block's elements (closed form);
* the matrix-free apply against the assembled matrix and against a brute-force
  per-entry quadrature loop on a curved 2-element mesh;
* symmetry and positive definiteness (the property the energy proof uses);
* the sine-bump map's Jacobian against finite differences of the map.
"""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import forms3d, hodge, splines


def _element_mass_1d(kind, p, nel, elems):
    """Univariate mass matrix restricted to a subset of elements."""
    x, w = splines.element_quadrature(nel, p + 1)
    e = np.arange(len(x)) // (p + 1)
    keep = np.isin(e, elems)
    V = splines.space_values(kind, p, nel, x[keep])
    return V.T @ (w[keep][:, None] * V)


@pytest.mark.parametrize("field", ["B", "D"])
@pytest.mark.parametrize("p,nel", [((2, 2, 2), (3, 2, 2)), ((3, 2, 4), (2, 3, 2))])
def test_identity_constant_is_kronecker(field, p, nel):
    gam = 2.5
    H = hodge.HodgeMass(field, p, nel, hodge.IdentityMap(), 1.0 / gam)  # gamma = 1/material
    M = H.matrix().toarray()
    blocks = []
    for c in range(3):
        kinds = forms3d.FIELD_KINDS[field][c]
        m = [splines.mass_1d(kinds[a], p[a], nel[a]) for a in range(3)]
        blocks.append(gam * np.kron(m[2], np.kron(m[1], m[0])))
    ref = np.zeros_like(M)
    off = forms3d.comp_offsets(field, p, nel)
    for c in range(3):
        ref[off[c]:off[c + 1], off[c]:off[c + 1]] = blocks[c]
    np.testing.assert_allclose(M, ref, atol=1e-14 * np.abs(ref).max())


def test_identity_block_material_closed_form():
    p, nel = (3, 3, 3), (4, 2, 4)
    vals = np.array([[[1.0, 3.0]], [[2.0, 5.0]]])  # blocks (b_z, b_y, b_x) = (2, 1, 2)
    H = hodge.HodgeMass("D", p, nel, hodge.IdentityMap(), ("blocks", vals))
    M = H.matrix().toarray()
    off = forms3d.comp_offsets("D", p, nel)
    for c in range(3):
        kinds = forms3d.FIELD_KINDS["D"][c]
        ref = 0.0
        for bz, by, bx in itertools.product(range(2), range(1), range(2)):
            ex = np.arange(bx * 2, bx * 2 + 2)
            ey = np.arange(by * 2, by * 2 + 2)
            ez = np.arange(bz * 2, bz * 2 + 2)
            mx_ = _element_mass_1d(kinds[0], p[0], nel[0], ex)
            my_ = _element_mass_1d(kinds[1], p[1], nel[1], ey)
            mz_ = _element_mass_1d(kinds[2], p[2], nel[2], ez)
            ref = ref + (1.0 / vals[bz, by, bx]) * np.kron(mz_, np.kron(my_, mx_))
        blk = M[off[c]:off[c + 1], off[c]:off[c + 1]]
        np.testing.assert_allclose(blk, ref, atol=1e-14)
        # no coupling between components on the identity map
        for c2 in range(3):
            if c2 != c:
                assert np.abs(M[off[c]:off[c + 1], off[c2]:off[c2 + 1]]).max() == 0.0


def test_sine_bump_jacobian_fd():
    F = hodge.SineBumpMap(0.05)
    rng = np.random.default_rng(3)
    X, Y, Z = rng.uniform(0, 1, (3, 20))
    J = F.jacobian(X, Y, Z)
    h = 1e-6
    for j in range(3):
        dp = [X, Y, Z]
        dm = [X, Y, Z]
        dp = [v + (h if a == j else 0) for a, v in enumerate(dp)]
        dm = [v - (h if a == j else 0) for a, v in enumerate(dm)]
        fd = (np.array(F(*dp)) - np.array(F(*dm))) / (2 * h)
        np.testing.assert_allclose(J[:, j], fd, atol=1e-8)
    det = hodge.det3(J)
    np.testing.assert_allclose(det, np.linalg.det(np.moveaxis(J, (0, 1), (-2, -1))), atol=1e-14)
    # maps the cube onto itself: identity on the boundary faces
    for a in range(3):
        pts = [rng.uniform(0, 1, 5) for _ in range(3)]
        pts[a] = np.zeros(5)
        np.testing.assert_allclose(np.array(F(*pts)), np.array(pts), atol=1e-15)


def test_curved_matrix_vs_bruteforce():
    """Per-entry quadrature with explicit loops, curved map, non-constant material."""
    p, nel = (2, 2, 2), (2, 1, 2)
    geom = hodge.SineBumpMap(0.05)
    mat = lambda x, y, z: 1.0 + x + 2.0 * y * z  # noqa: E731
    H = hodge.HodgeMass("B", p, nel, geom, mat)
    M = H.matrix().toarray()
    q = tuple(pa + 1 for pa in p)
    rules = [splines.gauss_legendre_01(q[a]) for a in range(3)]
    off = forms3d.comp_offsets("B", p, nel)
    shapes = [forms3d.comp_shape("B", c, p, nel) for c in range(3)]
    ref = np.zeros_like(M)
    for ez, ey, ex in itertools.product(range(nel[2]), range(nel[1]), range(nel[0])):
        for qz, qy, qx in itertools.product(range(q[2]), range(q[1]), range(q[0])):
            xh = np.array([(ex + rules[0][0][qx]) / nel[0], (ey + rules[1][0][qy]) / nel[1],
                           (ez + rules[2][0][qz]) / nel[2]])
            wt = rules[0][1][qx] * rules[1][1][qy] * rules[2][1][qz] / np.prod(nel)
            J = geom.jacobian(*[np.array([v]) for v in xh])[:, :, 0]
            xphys = np.array(geom(*xh))
            G = (1.0 / mat(*xphys)) * (J.T @ J) / np.linalg.det(J)
            # list all basis functions (component, flat index, value)
            funcs = []
            for c in range(3):
                kinds = forms3d.FIELD_KINDS["B"][c]
                v = [splines.space_values(kinds[a], p[a], nel[a], [xh[a]])[0] for a in range(3)]
                Nz, Ny, Nx = shapes[c]
                for k, j, i in itertools.product(range(Nz), range(Ny), range(Nx)):
                    val = v[2][k] * v[1][j] * v[0][i]
                    if val != 0.0:
                        funcs.append((c, off[c] + (k * Ny + j) * Nx + i, val))
            for (c1, r1, v1), (c2, r2, v2) in itertools.product(funcs, funcs):
                ref[r1, r2] += wt * v1 * G[c1, c2] * v2
    np.testing.assert_allclose(M, ref, atol=1e-14)
    # apply agrees with the assembled matrix, and M is SPD
    x = np.random.default_rng(1).standard_normal(M.shape[0])
    np.testing.assert_allclose(H.apply(x), M @ x, atol=1e-14)
    np.testing.assert_allclose(M, M.T, atol=1e-15)
    assert np.linalg.eigvalsh(M).min() > 0


def test_apply_matches_matrix_block_material_curved():
    p, nel = (3, 2, 3), (2, 4, 2)
    vals = np.arange(1.0, 9.0).reshape(2, 2, 2)
    H = hodge.HodgeMass("D", p, nel, hodge.SineBumpMap(0.05), ("blocks", vals))
    x = np.random.default_rng(2).standard_normal(forms3d.field_size("D", p, nel))
    M = H.matrix()
    np.testing.assert_allclose(H.apply(x), M @ x, atol=1e-13)
    assert abs(M - M.T).max() < 1e-15


def test_rejects_bad_material():
    with pytest.raises(ValueError):
        hodge.HodgeMass("B", 2, 2, hodge.IdentityMap(), -1.0)
    with pytest.raises(ValueError):
        hodge.HodgeMass("B", 2, 2, hodge.IdentityMap(), ("blocks", np.ones((3, 3, 3))))
