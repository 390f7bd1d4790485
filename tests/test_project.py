"""smx_project (host L2 projection of a physical 2-form, Sec. 5.1.1) against the oracle.

The library's projection runs on the host in FP64, so these tests need no GPU.
They compare it with the oracle's projection (the same Galerkin problem, solved
by plain CG), check that it reproduces fields that lie in the discrete space
exactly, and check its error paths.
"""
import numpy as np
import pytest

from oracle import hodge, maxwell as mx
from paper_2302_04979_gb300 import smx
from tests.gpu_util import rel_l2


def _field(x, y, z):
    """A smooth vector proxy with no particular alignment to the mesh."""
    return np.array([np.sin(2.1 * x + 0.3) * (1 + y * z), np.cos(1.3 * y) * x - z ** 2, np.exp(0.4 * x * y) * (z - 0.5)])


CASES = [
    ("identity_p2", dict(p=2, nel=(3, 4, 2))),
    ("identity_aniso", dict(p=(3, 2, 4), nel=(2, 3, 2))),
    ("curved_p3", dict(p=3, nel=(3, 2, 3), geometry="sine_bump")),
    ("one_element_axis", dict(p=2, nel=(1, 3, 1))),
    ("high_degree", dict(p=6, nel=(1, 2, 1))),
]


@pytest.mark.parametrize("name,case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("field", ["D", "B"])
def test_projection_matches_oracle(name, case, field):
    """Both sides solve the same Galerkin system to a relative residual of 1e-14, so their mass
    residuals agree to round-off; the coefficients agree to that times the condition number of the
    2-form mass, which grows with the degree (about 1e2 at p <= 4, 1e5 at p = 6)."""
    geom = hodge.SineBumpMap(0.05) if case.get("geometry") == "sine_bump" else hodge.IdentityMap()
    S = mx.Scheme2(case["p"], case["nel"], geometry=geom)
    ctx = smx.Context(case["p"], case["nel"], geometry=case.get("geometry", "identity"), amplitude=0.05)
    got = ctx.project(smx.FIELD_D if field == "D" else smx.FIELD_B, _field)
    want = S.project_2form(field, _field)
    assert got.shape == want.shape
    M1 = hodge.HodgeMass(field, case["p"], case["nel"], geom, 1.0)
    assert rel_l2(M1.apply(got), M1.apply(want)) < 1e-13
    tol = 1e-8 if int(np.max(case["p"])) >= 6 else 1e-11
    assert rel_l2(got, want) < tol


def test_projection_reproduces_a_discrete_field():
    """On the identity map a constant proxy lies in X~^2 and in X^2 (their spaces contain the
    constants per component), so projecting it and evaluating the result gives the constant back."""
    S = mx.Scheme2(2, (3, 2, 3))
    ctx = smx.Context(2, (3, 2, 3))
    const = lambda x, y, z: np.array([1.5 + 0 * x, -0.25 + 0 * y, 2.0 + 0 * z])  # noqa: E731
    d = ctx.project(smx.FIELD_D, const)
    err, nrm = S.l2_error("D", d, const)
    assert err < 1e-12 * nrm


def test_projection_errors():
    ctx = smx.Context(2, 2)
    lib = smx.library()
    assert lib.smx_project(ctx.h, smx.FIELD_E, smx.FIELD_FN(lambda *a: None), None, None) == smx.EINVAL
    with pytest.raises(smx.SmxError):
        ctx.project(smx.FIELD_D, lambda x, y, z: np.array([np.nan * x, y, z]))
    with pytest.raises(smx.SmxError):
        ctx.project(smx.FIELD_D, lambda x, y, z: 1 / 0)
