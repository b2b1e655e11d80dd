"""The allocation-free block-FSAI application against the regular one.

pum_fsai_apply_noalloc serves callers that must not allocate device memory (a CUDA
graph being captured, a loop that cannot take cudaMalloc's device-wide
synchronisation, memory held by another allocator): it keeps the intermediate G r in a
static device array instead of hierarchy work vectors.  This file is collected last.
"""
import ctypes as C

import numpy as np
import pytest

import pum_inputs as pin
from oracle import pum
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


def test_noalloc_fsai_apply_matches_regular_entry_point():
    import torch
    import paper_2509_06744_gb300 as L
    pr = pin.SMALL_BIHARMONIC
    f = pum.fourier_source(pin.fourier_coefficients(pr.rhs_seed), pr.rhs_decay)
    h = pum.build_hierarchy(8, pr.p, pr.equation, 3, f=f, constants=pr.nitsche)
    ctx = L.Context(0)
    H = L.Hierarchy.from_bsr(ctx, [to_view(A) for A in h.A], [to_pview(P) for P in h.P])
    H.setup(p0="lower", adaptive=True, t_max=3, k=2)
    keep = []
    G = _device_view(L, H.export(0, L.PUM_MAT_G), keep)
    GT = _device_view(L, H.export(0, L.PUM_MAT_GT), keep)
    N = h.A[0].n_rows * h.A[0].d
    for call in range(2):
        r = torch.as_tensor(pin.normal_vector(N, 90 + call)).cuda()
        z_ref = torch.zeros_like(r)
        H.fsai_apply(0, r, z_ref)
        z = torch.full_like(r, float("nan"))
        st = ctx.lib.pum_fsai_apply_noalloc(ctx.h, C.byref(G), C.byref(GT), C.c_void_p(r.data_ptr()),
                                            C.c_void_p(z.data_ptr()))
        assert st == 0, ctx.lib.pum_last_error(ctx.h)
        ctx.sync()
        assert norm_rel(z.cpu().numpy(), z_ref.cpu().numpy()) <= TOL_VECTOR
    # more unknowns than the static scratch holds is refused before any launch
    big = L._lib.BsrView(1 << 20, 1 << 20, 10, 0, G.row_ptr, None, None, 1)
    st = ctx.lib.pum_fsai_apply_noalloc(ctx.h, C.byref(big), C.byref(big), C.c_void_p(r.data_ptr()),
                                        C.c_void_p(z.data_ptr()))
    assert st == L._lib.PUM_ERR_INVALID_ARG and b"scratch" in ctx.lib.pum_last_error(ctx.h)
    H.close()
    ctx.close()
