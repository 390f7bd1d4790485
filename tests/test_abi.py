"""CPU tests of the C ABI: the library loads, exports every symbol include/smx.h
declares, and its host-side setup (DoF numbering, univariate pairing factors,
argument checks) agrees with the oracle.  No device work is launched here."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import forms3d, splines

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def smx():
    from paper_2302_04979_gb300 import build, smx as mod
    if not os.path.exists(mod.LIB_PATH):
        build.build()
    return mod


def test_exports_every_declared_symbol(smx):
    header = open(os.path.join(ROOT, "include", "smx.h")).read()
    declared = set(re.findall(r"^\s*(?:const\s+char\s*\*|int)\s+(smx_\w+)\s*\(", header, re.M))
    assert len(declared) >= 18
    lib = smx.library()
    for name in sorted(declared):
        assert hasattr(lib, name), name


FIELDS = {"E": 0, "B": 1, "H": 2, "D": 3}


@pytest.mark.parametrize("p,nel", [((2, 2, 2), (8, 8, 8)), ((3, 4, 2), (5, 3, 7)), ((4, 4, 4), (1, 2, 3))])
def test_numbering_matches_oracle(smx, p, nel):
    ctx = smx.Context(p, nel)
    assert ctx.N_e == forms3d.field_size("E", p, nel) == forms3d.field_size("D", p, nel)
    assert ctx.N_h == forms3d.field_size("B", p, nel) == forms3d.field_size("H", p, nel)
    for f, fi in FIELDS.items():
        for c in range(3):
            nx, ny, nz = ctx.comp_shape(fi, c)
            assert (nz, ny, nx) == forms3d.comp_shape(f, c, p, nel)


@pytest.mark.parametrize("p,nel", [(2, 1), (2, 7), (3, 4), (4, 9), (5, 3), (6, 2)])
def test_pairing_factors_match_oracle(smx, p, nel):
    ctx = smx.Context(p, nel)
    G, M = splines.G_hat(p, nel), splines.M_hat(p, nel)
    for axis in range(3):
        np.testing.assert_allclose(ctx.factor_matrix(axis, 0), G, atol=1e-14)
        np.testing.assert_allclose(ctx.factor_matrix(axis, 1), M, atol=1e-14)
        np.testing.assert_allclose(ctx.factor_matrix(axis, 2), G.T, atol=1e-14)
        np.testing.assert_allclose(ctx.factor_matrix(axis, 3), M.T, atol=1e-14)


def test_hodge_mode_selection(smx):
    assert smx.Context(3, 4).hodge_mode(smx.FIELD_D) == 2          # constant: separable Kronecker star
    assert smx.Context(3, 8, eps=("blocks", np.ones((2, 2, 2)))).hodge_mode(smx.FIELD_D) == 0
    ctx = smx.Context(3, 4, geometry="sine_bump")
    assert ctx.hodge_mode(smx.FIELD_D) == 1 and ctx.hodge_mode(smx.FIELD_B) == 1
    ctx = smx.Context(3, 4, eps=lambda x, y, z: 1.0 + x)
    assert ctx.hodge_mode(smx.FIELD_D) == 1 and ctx.hodge_mode(smx.FIELD_B) == 2


def test_argument_errors(smx):
    def status(**kw):
        try:
            smx.Context(**kw)
            return smx.OK
        except smx.SmxError as e:
            return e.status
    assert status(p=1, nel=4) == smx.EINVAL
    assert status(p=3, nel=0) == smx.EINVAL
    assert status(p=3, nel=4, eps=-1.0) == smx.EMAT
    assert status(p=3, nel=4, mu=float("nan")) == smx.EMAT
    assert status(p=3, nel=6, eps=("blocks", np.ones((4, 4, 4)))) == smx.EINVAL  # 4 does not divide 6
    assert status(p=3, nel=4, eps=("blocks", -np.ones((2, 2, 2)))) == smx.EMAT
    assert status(p=3, nel=4, geometry="sine_bump", amplitude=0.5) == smx.EGEOM  # det J <= 0 somewhere
    assert status(p=3, nel=4, geometry="sine_bump", eps=lambda x, y, z: 0.0 * x) == smx.EMAT
    assert status(p=7, nel=2) == smx.EINVAL                        # degrees 2..6
    assert status(p=2, nel=(4, 801, 4)) == smx.EINVAL             # at most 800 elements per axis
    assert status(p=3, nel=4, geometry="sine_bump", amplitude=float("nan")) == smx.EINVAL
    assert status(p=(2, 6, 3), nel=(1, 2, 3)) == smx.OK


def test_calls_without_workspace_are_rejected(smx):
    ctx = smx.Context(2, 2)
    lib = smx.library()
    assert lib.smx_hodge_apply(ctx.h, smx.FIELD_B, ctypes.c_void_p(8), ctypes.c_void_p(16)) == smx.ESTATE
    assert lib.smx_step(ctx.h, *([ctypes.c_void_p(8)] * 4), None, None, 0.1, 1) == smx.ESTATE
    assert lib.smx_step_host(ctx.h, *([ctypes.c_void_p(8)] * 4), None, None, 0.1, 1) == smx.ESTATE
    assert lib.smx_bind_workspace(ctx.h, ctypes.c_void_p(256), 16) == smx.ESTATE
    assert lib.smx_bind_workspace(ctx.h, None, 1 << 30) == smx.EINVAL
    assert lib.smx_strerror(smx.EGEOM).startswith(b"geometry")
    assert lib.smx_device_status(ctx.h) == smx.ESTATE
    assert lib.smx_hodge_star_mixed(ctx.h, smx.FIELD_D, ctypes.c_void_p(8), ctypes.c_void_p(16)) == smx.ESTATE
    assert lib.smx_strerror(smx.ETIMEOUT).startswith(b"a device-side wait")


def test_mode_kernel_selection(smx):
    ctx = smx.Context(3, 4, precision="mixed")
    assert ctx.mode_kernel() == "simt"  # the mixed default for lines shorter than 32 entries: CUDA cores
    assert smx.Context(3, (30, 2, 2), precision="mixed").mode_kernel() == "tensor"  # 32-entry lines
    assert smx.Context(3, (29, 2, 2), precision="mixed").mode_kernel() == "simt"
    ctx.set_mode_kernel("tensor")
    assert ctx.mode_kernel() == "tensor"
    ctx.set_mode_kernel("simt")
    assert smx.library().smx_set_mode_kernel(ctx.h, 7) == smx.EINVAL
    ctx.set_mode_kernel("auto")
    assert ctx.mode_kernel() == "simt"
    # FP64: per-star choice by default; digit-sliced tensor-core products or recurrences on request
    f64 = smx.Context(3, 20)
    assert f64.mode_kernel() == "auto"
    f64.set_mode_kernel("tensor")
    assert f64.mode_kernel() == "tensor"
    f64.set_mode_kernel("simt")
    assert f64.mode_kernel() == "simt"
    long_lines = smx.Context(2, (90, 3, 3))
    long_lines.set_mode_kernel("tensor")
    assert long_lines.mode_kernel() == "simt"  # lines of 91 entries: banded recurrences only
    assert smx.library().smx_mode_kernel(None, None) == smx.EINVAL


def test_reverse_mode_and_batch_argument_errors(smx):
    lib = smx.library()
    ctx = smx.Context(2, 4, eps=("blocks", np.full((2, 2, 2), 2.0)))
    v = ctypes.c_void_p(8)
    # reverse mode needs a bound workspace
    assert lib.smx_step_adjoint(ctx.h, v, v, v, v, None, None, 0.1, None, None) == smx.ESTATE
    assert lib.smx_adjoint_terminal(ctx.h, v, v, v, None) == smx.ESTATE
    assert lib.smx_set_material_blocks(ctx.h, smx.FIELD_D, v) == smx.ESTATE
    assert lib.smx_receivers_eval(ctx.h, v, v) == smx.ESTATE
    # receivers: before binding only, points in [0, 1], once
    assert lib.smx_receivers_set(ctx.h, -1, None) == smx.EINVAL
    bad = np.array([[0.5, 1.5, 0.5]])
    assert lib.smx_receivers_set(ctx.h, 1, bad.ctypes.data_as(ctypes.c_void_p)) == smx.EINVAL
    ok = np.array([[0.5, 0.25, 0.75], [0.1, 0.9, 0.3]])
    assert lib.smx_receivers_set(ctx.h, 2, ok.ctypes.data_as(ctypes.c_void_p)) == smx.OK
    assert lib.smx_receivers_set(ctx.h, 2, ok.ctypes.data_as(ctypes.c_void_p)) == smx.ESTATE
    # a batch needs bound contexts
    arr = (ctypes.c_void_p * 1)(ctx.h.value)
    out = ctypes.c_void_p()
    assert lib.smx_batch_create(1, arr, ctypes.byref(out)) == smx.EINVAL
    assert lib.smx_batch_create(0, arr, ctypes.byref(out)) == smx.EINVAL
