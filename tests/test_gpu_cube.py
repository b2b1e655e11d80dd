"""The solver path on the biharmonic equation on the unit cube (Example 5.3, d = 20 at p = 3).

The hierarchy (4^3, 2^3 and 1 patch) is assembled by the oracle and handed to the library through
the C-ABI (pum_hier_from_bsr): Algorithm 1's patterns on every smoothed level must be the
oracle's bit for bit, and the FP64 form's PCG must reproduce the oracle solver's iteration count,
residual history and solution.  The library assembles the square only.
"""
import numpy as np
import pytest

from oracle import fsai, pum3d, solver
from _util import TOL_FSAI, TOL_HISTORY, assert_same_pattern, cuda, from_export, host, max_rel, norm_rel, to_pview, to_view

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cube():
    f = lambda x, y, z: np.sin(np.pi * x) * np.sin(2 * np.pi * y) * np.sin(np.pi * z) + 1.0
    return pum3d.build_hierarchy(4, 3, 3, f=f)


def test_cube_adaptive_patterns_and_pcg_match_oracle(cube):
    import paper_2509_06744_gb300 as lib
    ctx = lib.Context(0)
    H = lib.Hierarchy.from_bsr(ctx, [to_view(A) for A in cube.A], [to_pview(P) for P in cube.P])
    H.setup(p0="lower", adaptive=True, t_max=3, tau=1.0, k=2)
    assert H.info(0)["d"] == 20
    for l in range(len(cube.A) - 1):
        ref = fsai.adaptive_fsai(cube.A[l], fsai.lower_pattern(cube.A[l]), 3).fsai
        G = from_export(H.export(l, lib.PUM_MAT_G))
        assert_same_pattern(G, ref.G)
        assert max_rel(G.blocks, ref.G.blocks) <= TOL_FSAI
    ref = solver.build_setup(cube, k=2, mode="adaptive", P0="lower", t_max=3)
    x = cuda(np.zeros_like(cube.b))
    rep = H.pcg(cuda(cube.b), x, rtol=1e-8, maxit=100)
    res = solver.solve(ref, cube.b, rtol=1e-8)
    assert rep["converged"] and rep["iters"] == res.iters
    assert np.max(np.abs(np.array(rep["history"]) - np.array(res.history))) <= TOL_HISTORY
    assert norm_rel(host(x), res.x) <= 1e-9
    H.close()
    ctx.close()
