"""A general geometry map given by a host callback (SMX_GEOM_CALLBACK, the single-patch map F of
Sec. 2.3), on the host: the seeded input maps' Jacobians against finite differences, the
library's L2 projection through the callback against the oracle's with the same map, the
callback reproducing the built-in sine-bump map, and the error paths (det J_F <= 0, non-finite
values, a callback that raises).  The GPU side (Hodge stars and steps through the callback map)
is in tests/test_gpu_geometry.py."""
import numpy as np
import pytest

from oracle import maxwell as mx
from paper_2302_04979_gb300 import smx, synth
from tests.gpu_util import rel_l2

MAPS = {"sine_bump": synth.SineBumpMap(0.05), "shear": synth.ShearMap(), "coax": synth.QuarterCoaxMap(),
        "coax_nurbs": synth.QuarterCoaxNURBS()}


def test_nurbs_coax_traces_the_annulus():
    """The degree-2 NURBS patch (Sec. 5.1.2) maps onto the quarter annulus exactly: r = 1 + (sqrt 2 - 1) x^
    at every point, the angle runs monotonically from 0 to pi/2 along y^, and the patch's corners
    are the polar map's."""
    m, polar = synth.QuarterCoaxNURBS(), synth.QuarterCoaxMap()
    x, y, z = synth.uniform(9, 3 * 200, 0.0, 1.0).reshape(3, 200)
    X, Y, Z = m(x, y, z)
    np.testing.assert_allclose(np.hypot(X, Y), 1.0 + (np.sqrt(2.0) - 1.0) * x, rtol=0, atol=1e-15)
    np.testing.assert_array_equal(Z, z)
    ys = np.linspace(0.0, 1.0, 101)
    theta = np.arctan2(*m(np.zeros_like(ys), ys, ys)[1::-1])
    assert theta[0] == 0.0 and abs(theta[-1] - np.pi / 2) < 1e-15 and np.all(np.diff(theta) > 0)
    for cx in (0.0, 1.0):
        for cy in (0.0, 1.0):
            np.testing.assert_allclose(m(cx, cy, 0.5), polar(cx, cy, 0.5), rtol=0, atol=1e-15)


@pytest.mark.parametrize("name", sorted(MAPS))
def test_input_map_jacobian_is_the_derivative(name):
    m = MAPS[name]
    x = synth.uniform(5, 3 * 50, 0.02, 0.98).reshape(3, 50)
    J = m.jacobian(*x)
    h = 1e-6
    for c in range(3):
        xp, xm = x.copy(), x.copy()
        xp[c] += h
        xm[c] -= h
        fd = (np.array(m(*xp)) - np.array(m(*xm))) / (2 * h)
        assert np.abs(fd - J[:, c]).max() < 1e-8


def _vec(x, y, z):
    return np.array([np.cos(1.7 * x) * (1 + y), np.sin(2.3 * y + z) - x * z, np.exp(0.5 * x) * (z - 0.3) + y])


@pytest.mark.parametrize("name", sorted(MAPS))
@pytest.mark.parametrize("field", ["D", "B"])
def test_projection_through_callback_matches_oracle(name, field):
    """The library's host projection with the callback map against the oracle's with the same map
    object (both solve the same Galerkin system to 1e-14 relative residual)."""
    p, nel = 3, (3, 2, 4)
    ctx = smx.Context(p, nel, geometry=MAPS[name])
    S = mx.Scheme2(p, nel, geometry=MAPS[name])
    got = ctx.project(smx.FIELD_D if field == "D" else smx.FIELD_B, _vec)
    want = S.project_2form(field, _vec)
    assert rel_l2(got, want) < 1e-12


def test_callback_reproduces_the_builtin_sine_bump():
    """The sine-bump map through the callback and the built-in one give the same projection."""
    p, nel = 2, (4, 3, 3)
    a = smx.Context(p, nel, geometry=synth.SineBumpMap(0.05)).project(smx.FIELD_D, _vec)
    b = smx.Context(p, nel, geometry="sine_bump", amplitude=0.05).project(smx.FIELD_D, _vec)
    assert rel_l2(a, b) < 1e-14


class _Flip:
    """x -> (-x, y, z): det J = -1 (orientation reversing)."""

    def __call__(self, x, y, z):
        return -x, y, z

    def jacobian(self, x, y, z):
        x = np.asarray(x, dtype=np.float64)
        one, zero = np.ones_like(x), np.zeros_like(x)
        return np.array([[-one, zero, zero], [zero, one, zero], [zero, zero, one]])


class _Bad(synth.ShearMap):
    def jacobian(self, x, y, z):
        J = super().jacobian(x, y, z)
        J[0, 0][0] = np.nan
        return J


class _Raises(synth.ShearMap):
    def __call__(self, x, y, z):
        raise ValueError("no map here")


@pytest.mark.parametrize("mapping", [_Flip(), _Bad(), _Raises()], ids=["det<0", "nan", "raises"])
def test_invalid_maps_are_rejected(mapping):
    # the quadrature tables evaluate the map at every point inside smx_create
    with pytest.raises(smx.SmxError) as err:
        smx.Context(2, 2, geometry=mapping)
    assert err.value.status == smx.EGEOM


def test_null_callback_is_invalid():
    P, keep = smx.make_params(2, 2)
    P.geometry = smx.GEOM_CALLBACK   # no geom_fn
    import ctypes
    h = ctypes.c_void_p()
    assert smx.library().smx_create(ctypes.byref(P), ctypes.byref(h)) == smx.EINVAL
