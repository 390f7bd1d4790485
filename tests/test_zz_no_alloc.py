"""The allocation-free Hodge star (smx_hodge_star_noalloc) against the workspace path.

Callers that cannot allocate device memory cannot bind the workspace the
other entry points need; smx_hodge_star_noalloc serves them from a fixed
device array inside the library.  These tests call it through the C ABI and
compare it with smx_hodge_star on the same inputs, two calls in a row, with
the single-stage tolerance the parity tests use (1e-12 relative L2).  They
pass both in a fresh process (first call does the device set-up) and after
the other tests (the array then holds another context's tables).
"""
import numpy as np
import pytest

from paper_2302_04979_gb300 import synth
from tests.gpu_util import rel_l2, to_dev, to_host

pytestmark = pytest.mark.gpu


def _ctx(p, nel, **kw):
    from paper_2302_04979_gb300 import smx
    return smx.Context(p, nel, **kw)


def _compare(ref_ctx, ctx, seed):
    import torch
    from paper_2302_04979_gb300 import smx
    for field, n in ((smx.FIELD_D, ctx.N_e), (smx.FIELD_B, ctx.N_h)):
        x = to_dev(synth.uniform(seed + field, n, -1.0, 1.0))
        want = torch.empty(n, dtype=torch.float64, device="cuda")
        got = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
        ref_ctx.hodge_star(field, x, want)
        ctx.hodge_star_noalloc(field, x, got)
        torch.cuda.synchronize()
        assert rel_l2(to_host(got), to_host(want)) < 1e-12


def test_noalloc_matches_workspace_path_two_calls():
    eps = ("blocks", synth.block_material(9, (3, 3, 2), 1.0, 9.0))
    ref = _ctx(3, (12, 9, 10), eps=eps, mu=1.5).bind()
    bare = _ctx(3, (12, 9, 10), eps=eps, mu=1.5)   # no workspace bound
    _compare(ref, bare, 100)
    _compare(ref, bare, 200)


def test_noalloc_switches_between_contexts():
    a_ref = _ctx(2, 8).bind()
    b_ref = _ctx(4, (6, 7, 5), eps=2.0).bind()
    a, b = _ctx(2, 8), _ctx(4, (6, 7, 5), eps=2.0)
    _compare(a_ref, a, 300)
    _compare(b_ref, b, 400)
    _compare(a_ref, a, 500)


def test_noalloc_after_material_update():
    """A block-permittivity update (smx_set_material_blocks) must reach the no-alloc call too:
    its next call re-uploads the context's tables, and matches hodge_star and the oracle with
    the new permittivity (1e-12), before and after the update, and again after a rebind."""
    import torch
    from oracle import maxwell as mx
    from paper_2302_04979_gb300 import smx
    p, nel, blocks = 3, (8, 6, 6), (2, 3, 2)
    eps0 = synth.block_material(31, blocks, 1.0, 4.0)
    eps1 = synth.block_material(32, blocks, 2.0, 9.0)
    ctx = _ctx(p, nel, eps=("blocks", eps0), mu=1.0).bind()
    x = to_dev(synth.uniform(600, ctx.N_e, -1.0, 1.0))
    got = torch.full((ctx.N_e,), np.nan, dtype=torch.float64, device="cuda")
    want = torch.empty_like(got)
    for eps, rebind in ((eps0, False), (eps1, False), (eps1, True)):
        if eps is eps1 and not rebind:
            ctx.set_material_blocks(eps1)
        if rebind:
            ctx.bind()   # uploads the host copy of the tables again
        ctx.hodge_star_noalloc(smx.FIELD_D, x, got)
        ctx.hodge_star(smx.FIELD_D, x, want)
        torch.cuda.synchronize()
        ref = mx.Scheme2(p, nel, eps=("blocks", eps)).e_from_d(to_host(x))
        assert rel_l2(to_host(got), to_host(want)) < 1e-12
        assert rel_l2(to_host(got), ref) < 1e-12
        assert rel_l2(to_host(want), ref) < 1e-12


def test_noalloc_rejects_what_does_not_fit():
    import torch
    from paper_2302_04979_gb300 import smx
    big = _ctx(3, 100)   # one field vector alone is larger than the fixed array
    x = torch.zeros(big.N_e, dtype=torch.float64, device="cuda")
    with pytest.raises(smx.SmxError) as err:
        big.hodge_star_noalloc(smx.FIELD_D, x, x)
    assert err.value.status == smx.ENOSPACE
    curved = _ctx(3, 4, geometry="sine_bump")
    y = torch.zeros(curved.N_e, dtype=torch.float64, device="cuda")
    with pytest.raises(smx.SmxError) as err:
        curved.hodge_star_noalloc(smx.FIELD_D, y, torch.empty_like(y))
    assert err.value.status == smx.EINVAL
