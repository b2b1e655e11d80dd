"""Example 5.1's raised space (degree 2 inside, 3 on patches meeting the boundary) on the GPU.

The library keeps one block size per level, so the raised space runs on uniform 10 x 10 blocks
in which the interior patches' 6 unknowns are padded with decoupled unknowns of unit diagonal.
The padded hierarchy is built by the oracle and handed to the library through the C-ABI
(pum_hier_from_bsr): Algorithm 1's patterns match the oracle's bit for bit, the FP64 PCG matches
the oracle solver's iterations, history and solution, the padded unknowns stay exactly zero, and
the real ones solve the raised system.
"""
import numpy as np
import pytest

from oracle import fsai, pum_raise, solver
from _util import TOL_FSAI, TOL_HISTORY, assert_same_pattern, cuda, from_export, host, max_rel, norm_rel, to_pview, to_view

pytestmark = pytest.mark.gpu


def test_raised_space_on_the_uniform_layout_matches_oracle():
    import scipy.sparse.linalg as spla
    import paper_2509_06744_gb300 as lib
    h = pum_raise.padded_hierarchy(8, 2, 3, 3, f=lambda x, y: np.sin(np.pi * x) * np.sin(np.pi * y) + 0.5)
    ctx = lib.Context(0)
    H = lib.Hierarchy.from_bsr(ctx, [to_view(A) for A in h.A], [to_pview(P) for P in h.P])
    H.setup(p0="lower", adaptive=True, t_max=3, tau=1.0, k=2)
    for l in range(len(h.A) - 1):
        ref = fsai.adaptive_fsai(h.A[l], fsai.lower_pattern(h.A[l]), 3).fsai
        G = from_export(H.export(l, lib.PUM_MAT_G))
        assert_same_pattern(G, ref.G)
        assert max_rel(G.blocks, ref.G.blocks) <= TOL_FSAI
    ref = solver.build_setup(h, k=2, mode="adaptive", P0="lower", t_max=3)
    x = cuda(np.zeros_like(h.b))
    rep = H.pcg(cuda(h.b), x, rtol=1e-8, maxit=100)
    res = solver.solve(ref, h.b, rtol=1e-8)
    assert rep["converged"] and rep["iters"] == res.iters
    assert np.max(np.abs(np.array(rep["history"]) - np.array(res.history))) <= TOL_HISTORY
    xh = host(x)
    assert norm_rel(xh, res.x) <= 1e-9
    pad = np.setdiff1d(np.arange(len(h.b)), h.real[0])
    assert np.all(xh[pad] == 0.0)
    xr = spla.spsolve(h.A_raised.tocsc(), h.b_raised)
    assert np.linalg.norm(xh[h.real[0]] - xr) <= 1e-7 * np.linalg.norm(xr)
    H.close()
    ctx.close()
