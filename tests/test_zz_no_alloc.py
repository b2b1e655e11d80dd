"""The allocation-free block-FSAI application, against the regular one and the oracle.

pum_fsai_apply_noalloc serves callers that cannot allocate device memory (their device
memory is reserved in full by another allocator, their memory budget is fixed at start-up,
or their loop cannot take the device-wide synchronisation of cudaFree): it keeps the
intermediate G r in a static device array instead of hierarchy work vectors.  This file is
collected last, so a run that stops at its first failure has run every other test first.
"""
import ctypes as C

import numpy as np
import pytest

import pum_inputs as pin
from oracle import fsai, pum
from _util import TOL_VECTOR, norm_rel, to_pview, to_view

pytestmark = pytest.mark.gpu


def _device_view(lib_mod, exp, keep):
    import torch
    indptr, indices, blocks, n_cols = exp
    rp = torch.as_tensor(indptr.astype(np.int32)).cuda()
    ci = torch.as_tensor(indices.astype(np.int32)).cuda()
    v = torch.as_tensor(np.ascontiguousarray(blocks)).cuda()
    keep += [rp, ci, v]
    return lib_mod._lib.BsrView(len(indptr) - 1, n_cols, blocks.shape[1], len(indices), rp.data_ptr(),
                                ci.data_ptr(), v.data_ptr(), 1)


def _call(ctx, G, GT, r, z):
    return ctx.lib.pum_fsai_apply_noalloc(ctx.h, C.byref(G), C.byref(GT), C.c_void_p(r), C.c_void_p(z))


def test_noalloc_fsai_apply_matches_regular_entry_point_and_oracle():
    import torch
    import paper_2509_06744_gb300 as L
    pr = pin.SMALL_BIHARMONIC
    f = pum.fourier_source(pin.fourier_coefficients(pr.rhs_seed), pr.rhs_decay)
    h = pum.build_hierarchy(8, pr.p, pr.equation, 3, f=f, constants=pr.nitsche)
    G_oracle = fsai.adaptive_fsai(h.A[0], fsai.lower_pattern(h.A[0]), 3).fsai.G
    ctx = L.Context(0)
    H = L.Hierarchy.from_bsr(ctx, [to_view(A) for A in h.A], [to_pview(P) for P in h.P])
    H.setup(p0="lower", adaptive=True, t_max=3, k=2)
    keep = []
    G = _device_view(L, H.export(0, L.PUM_MAT_G), keep)
    GT = _device_view(L, H.export(0, L.PUM_MAT_GT), keep)
    N = h.A[0].n_rows * h.A[0].d
    dev_before = torch.cuda.current_device()
    free_after = []
    for call in range(2):                       # two calls in a row share the static array
        rh = pin.normal_vector(N, 90 + call)
        r = torch.as_tensor(rh).cuda()
        z_ref = torch.zeros_like(r)
        H.fsai_apply(0, r, z_ref)
        z = torch.full_like(r, float("nan"))
        st = _call(ctx, G, GT, r.data_ptr(), z.data_ptr())
        assert st == 0, ctx.lib.pum_last_error(ctx.h)
        ctx.sync()
        zh = z.cpu().numpy()
        assert norm_rel(zh, z_ref.cpu().numpy()) <= TOL_VECTOR
        # the oracle's own factor (Algorithm 1 on the oracle's matrix), M r = G^T (G r)
        assert norm_rel(zh, fsai.apply_M(G_oracle, rh)) <= TOL_VECTOR
        free_after.append(torch.cuda.mem_get_info()[0])
    assert torch.cuda.current_device() == dev_before
    # after the first call (which may load the kernels' code) device memory stays as it was
    assert free_after[1] == free_after[0]
    # rejections, each before any launch and each with a message
    big = L._lib.BsrView(1 << 20, 1 << 20, 10, 0, G.row_ptr, None, None, 1)
    assert _call(ctx, big, big, r.data_ptr(), z.data_ptr()) == L._lib.PUM_ERR_INVALID_ARG
    assert b"scratch" in ctx.lib.pum_last_error(ctx.h)
    odd = L._lib.BsrView(G.n_brows, G.n_bcols, 7, G.nnzb, G.row_ptr, G.col_idx, G.vals, 1)
    assert _call(ctx, odd, odd, r.data_ptr(), z.data_ptr()) == L._lib.PUM_ERR_UNSUPPORTED
    assert b"block size" in ctx.lib.pum_last_error(ctx.h)
    wrong = L._lib.BsrView(GT.n_brows, GT.n_bcols + 1, GT.bs, GT.nnzb, GT.row_ptr, GT.col_idx, GT.vals, 1)
    assert _call(ctx, G, wrong, r.data_ptr(), z.data_ptr()) == L._lib.PUM_ERR_INVALID_ARG
    assert b"transpose" in ctx.lib.pum_last_error(ctx.h)
    assert _call(ctx, G, GT, r.data_ptr() + 4, z.data_ptr()) == L._lib.PUM_ERR_INVALID_ARG
    assert b"aligned" in ctx.lib.pum_last_error(ctx.h)
    ctx.sync()
    H.close()
    ctx.close()
