"""Several right-hand sides at once (pcg_solve_multi, vcycle_apply_multi): every product of the
V(k,k) cycle reads its matrix once for a block of columns.  Per column the FP64 form is the
oracle's cycle and PCG (Section 5, Algorithm 3); the FP32 form is the plain FP32 cycle of the
single-right-hand-side path."""
import numpy as np
import pytest

import pum_inputs as pin
from oracle import solver
from _util import TOL_HISTORY, TOL_VECTOR, cuda, host, norm_rel, to_pview, to_view

pytestmark = pytest.mark.gpu

PR = pin.SMALL_BIHARMONIC


@pytest.fixture(scope="module")
def lib():
    import paper_2509_06744_gb300 as L
    return L


@pytest.fixture(scope="module")
def ctx(lib):
    c = lib.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def pair(lib, ctx, small_biharmonic):
    h = small_biharmonic
    H = lib.Hierarchy.from_bsr(ctx, [to_view(A) for A in h.A], [to_pview(P) for P in h.P])
    H.setup(p0="lower", adaptive=False, k=PR.cheb_k)
    ref = solver.build_setup(h, k=PR.cheb_k, mode="static", P0="lower")
    yield H, ref
    H.close()


def _block(n, nrhs, seed):
    return np.stack([pin.normal_vector(n, seed + c) for c in range(nrhs)])


@pytest.mark.parametrize("nrhs", [3, 7])
def test_multi_cycle_matches_oracle_per_column(pair, nrhs):
    """nrhs = 3 runs in a block of 4 columns, 7 in a block of 16 (the rest zero)."""
    H, ref = pair
    R = _block(PR.n_dofs, nrhs, 500)
    Z = cuda(np.zeros_like(R))
    H.vcycle_multi(cuda(R), Z)
    Zh = host(Z)
    for c in range(nrhs):
        assert norm_rel(Zh[c], solver.vcycle(ref, R[c])) <= TOL_VECTOR, c


def test_multi_pcg_matches_oracle_per_column(pair, small_biharmonic):
    """FP64 form: each column's iteration count and ||r_j|| / ||b|| history are the oracle's single
    solve's (histories within 1e-12), columns converging at different iterations included."""
    H, ref = pair
    h = small_biharmonic
    B = np.stack([h.b, pin.normal_vector(PR.n_dofs, 61), 1e-3 * pin.normal_vector(PR.n_dofs, 62),
                  h.A[0].matvec(pin.normal_vector(PR.n_dofs, 63))])
    X = cuda(np.zeros_like(B))
    reps = H.pcg_multi(cuda(B), X, rtol=1e-8, maxit=100)
    Xh = host(X)
    for c in range(B.shape[0]):
        res = solver.solve(ref, B[c], rtol=1e-8)
        assert reps[c]["converged"] and reps[c]["iters"] == res.iters, c
        assert np.max(np.abs(np.array(reps[c]["history"]) - np.array(res.history))) <= TOL_HISTORY, c
        assert norm_rel(Xh[c], res.x) <= 1e-9, c


def test_multi_fp32_form_matches_single_solves(lib, ctx):
    """FP32 form (plain FP32 cycle, mixed_levels = 0) on 64x64 patches with 16 right-hand sides in
    one block: every column converges in the single-right-hand-side solve's iterations, to its
    solution within the FP32 cycle's rounding."""
    import torch
    m, levels = 64, 5
    b = torch.zeros(m * m * PR.d, dtype=torch.float64, device="cuda")
    H = lib.Hierarchy.assemble(ctx, PR.equation, PR.p, m, levels, f_coef=pin.fourier_coefficients(PR.rhs_seed),
                               f_decay=PR.rhs_decay, nitsche=PR.nitsche, b=b)
    H.setup(p0="lower", adaptive=True, t_max=6, k=3, smooth="f32", g="f32", mixed_levels=0)
    N = b.numel()
    B = torch.tensor(_block(N, 16, 700), device="cuda")
    X = torch.zeros_like(B)
    reps = H.pcg_multi(B, X, rtol=1e-8, maxit=100, flexible=True)
    for c in range(16):
        x1 = torch.zeros(N, dtype=torch.float64, device="cuda")
        rep1 = H.pcg(B[c].contiguous(), x1, rtol=1e-8, maxit=100, flexible=True)
        assert reps[c]["converged"] and abs(reps[c]["iters"] - rep1["iters"]) <= 1, c
        assert float(torch.linalg.norm(X[c] - x1) / torch.linalg.norm(x1)) <= 1e-6, c
    H.close()


def test_multi_rejections(lib, ctx, pair):
    import torch
    H, _ = pair
    R = torch.zeros((17, PR.n_dofs), dtype=torch.float64, device="cuda")
    with pytest.raises(lib.PumError):
        H.vcycle_multi(R, torch.zeros_like(R))          # more than 16 columns
    del torch
