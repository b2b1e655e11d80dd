"""Pins of the Chebyshev smoother, Lanczos, V-cycle and PCG oracles (Section 3.1, Section 5)."""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla

import pum_inputs as pin
from oracle import cheb, rng, solver

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_splitmix64_published_values():
    assert rng.splitmix64(0, 3) == pin.splitmix64_reference_values()


def test_w4_recurrence_and_trigonometric_closed_form():
    """W_k(cos t) = sin((k + 1/2) t) / sin(t / 2); W_k(1) = 2k + 1; W_1 = 2t + 1, W_2 = 4t^2 + 2t - 1."""
    th = np.linspace(0.05, np.pi - 0.05, 101)
    for k in range(0, 9):
        assert np.allclose(cheb.w4(k, np.cos(th)), np.sin((k + 0.5) * th) / np.sin(th / 2), atol=1e-12)
        assert abs(cheb.w4(k, 1.0) - (2 * k + 1)) <= 1e-12
    t = np.linspace(-1, 1, 7)
    g = GOLDEN["w4_first_polynomials"]
    assert np.allclose(cheb.w4(0, t), np.polyval(g["W0"][::-1], t))
    assert np.allclose(cheb.w4(1, t), np.polyval(g["W1"][::-1], t))
    assert np.allclose(cheb.w4(2, t), 4 * t ** 2 + 2 * t - 1)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_algorithm3_error_polynomial_on_diagonal_matrix(k):
    """Eq. (3.6): Algorithm 3 on diagonal A (M = I) gives r_k = W_k(1 - 2 lam/beta)/(2k+1) r_0."""
    lam = np.linspace(0.0, 1.0, 41)[1:]
    beta = 1.0
    A = lambda v: lam * v
    I = lambda v: v
    b = np.ones_like(lam)
    x = cheb.cheb4(A, I, b, None, beta, k)
    r = b - A(x)
    expect = cheb.w4(k, 1.0 - 2.0 * lam / beta) / (2 * k + 1)
    assert np.max(np.abs(r - expect)) <= 1e-14 * (2 * k + 1)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_weighted_minimax_value(k):
    """Lemma 3.3 / Eq. (3.6): max over [0, beta] of sqrt(lam)|p_k(lam)| = sqrt(beta)/(2k+1), attained k+1 times."""
    beta = 2.5
    lam = np.linspace(0.0, beta, 200001)
    w = np.sqrt(lam) * np.abs(cheb.cheb4_residual_polynomial(k, lam, beta))
    assert abs(w.max() - np.sqrt(beta) / (2 * k + 1)) <= 1e-6
    # local maxima reaching the bound: k + 1 alternation points
    peaks = np.sum((w[1:-1] >= w[:-2]) & (w[1:-1] >= w[2:]) & (w[1:-1] > (1 - 1e-6) * w.max()))
    peaks += int(w[-1] > (1 - 1e-6) * w.max())
    assert peaks == k + 1


def test_algorithm3_constants_and_richardson_limit():
    """Algorithm 3: mu0 = 1/3, d = 4/beta; k = 1 is Richardson with weight 4/(3 beta)."""
    g = GOLDEN
    assert g["cheb4_mu0"]["value"] == pytest.approx(1 / 3) and g["cheb4_d_times_beta"]["value"] == 4.0
    rs = np.random.default_rng(2)
    Q = rs.standard_normal((6, 6))
    A = Q @ Q.T + 6 * np.eye(6)
    M = np.diag(1.0 / np.diag(A))
    b = rs.standard_normal(6)
    x0 = rs.standard_normal(6)
    beta = 3.0
    x = cheb.cheb4(lambda v: A @ v, lambda v: M @ v, b, x0, beta, 1)
    assert np.allclose(x, x0 + 4.0 / (3.0 * beta) * M @ (b - A @ x0), atol=1e-14)


def test_preconditioned_error_propagation_is_polynomial_in_MA():
    """With M SPD, e_k = p_k(M A) e_0 for the same fourth-kind polynomial."""
    rs = np.random.default_rng(4)
    Q = rs.standard_normal((8, 8))
    A = Q @ Q.T + np.eye(8)
    R = rs.standard_normal((8, 8))
    M = np.linalg.inv(A + 0.3 * (R @ R.T))
    MA = M @ A
    lam, V = np.linalg.eig(MA)
    beta = 1.01 * np.max(lam.real)
    xs = rs.standard_normal(8)
    b = A @ xs
    x0 = rs.standard_normal(8)
    for k in (2, 3, 4):
        x = cheb.cheb4(lambda v: A @ v, lambda v: M @ v, b, x0, beta, k)
        pk = V @ np.diag(cheb.cheb4_residual_polynomial(k, lam, beta)) @ np.linalg.inv(V)
        assert np.allclose(xs - x, (pk @ (xs - x0)).real, atol=1e-10)


def test_lanczos_recovers_known_extreme_eigenvalue():
    """Lanczos on a diagonal matrix with known spectrum finds lambda_max."""
    n = 500
    lam = np.linspace(1e-3, 1.0, n) ** 2
    lam[-1] = 2.0
    est = cheb.lanczos_lmax(lambda v: lam * v, n, its=GOLDEN["lanczos_iterations"]["value"], seed=3)
    assert abs(est - 2.0) <= 1e-10
    # early termination on an invariant subspace: 3 distinct eigenvalues
    lam3 = np.repeat([1.0, 2.0, 5.0], 10)
    assert abs(cheb.lanczos_lmax(lambda v: lam3 * v, 30, seed=1) - 5.0) <= 1e-12


# ----------------------------------------------------------------- V-cycle / PCG

@pytest.fixture(scope="module")
def static_setup(small_biharmonic):
    return solver.build_setup(small_biharmonic, k=2, mode="static", P0="lower")


def test_vcycle_is_symmetric(static_setup, small_biharmonic):
    """V(k,k) with the same Algorithm 3 polynomial before and after is symmetric: <Bu, v> = <u, Bv>."""
    n = small_biharmonic.A[0].n_rows * 10
    u = pin.normal_vector(n, 1)
    v = pin.normal_vector(n, 2)
    Bu, Bv = solver.vcycle(static_setup, u), solver.vcycle(static_setup, v)
    assert abs(Bu @ v - u @ Bv) <= 1e-12 * np.linalg.norm(Bu) * np.linalg.norm(v)
    # and positive: u^T B u > 0
    assert u @ Bu > 0


def test_vcycle_spectral_radius_below_one(static_setup, small_biharmonic):
    """The stationary V-cycle converges: rho_A < 1 (Example 5.1 measure)."""
    e0 = pin.uniform_vector(small_biharmonic.A[0].n_rows * 10, 5)
    rho = solver.convergence_factor(static_setup, e0, 8)
    assert 0.0 < rho < 0.5


def test_pcg_identity_preconditioner_matches_direct_solve():
    rs = np.random.default_rng(5)
    Q = rs.standard_normal((30, 30))
    A = Q @ Q.T + 30 * np.eye(30)
    b = rs.standard_normal(30)
    res = solver.pcg(lambda v: A @ v, lambda v: v, b, rtol=1e-14, maxit=200)
    xd = np.linalg.solve(A, b)
    assert res.converged and np.linalg.norm(res.x - xd) <= 1e-12 * np.linalg.norm(xd)
    assert res.history[0] == 1.0 and len(res.history) == res.iters + 1


def test_pcg_vcycle_end_to_end_matches_direct(static_setup, small_biharmonic):
    """PCG with the V(2,2) cycle reaches 1e-8 and its solution matches a dense solve."""
    h = small_biharmonic
    res = solver.solve(static_setup, h.b, rtol=1e-8)
    assert res.converged and res.history[-1] <= 1e-8 and res.iters < 30
    A = h.A[0].to_dense()
    xd = sla.solve(A, h.b, assume_a="pos")
    e = res.x - xd
    assert np.sqrt(e @ A @ e) / np.sqrt(xd @ A @ xd) <= 1e-7


# ------------------------------------------- Richardson smoothing, V(2k,0), BiCGStab (Section 5)

def test_richardson_error_polynomial_on_diagonal_matrix():
    """Richardson smoothing (Section 3.1) propagates the error by (I - M A)^k: on diagonal
    matrices, e_k = (1 - m lambda)^k e_0 entry by entry."""
    rs = np.random.default_rng(11)
    lam = rs.uniform(0.1, 3.0, 40)
    m = rs.uniform(0.2, 0.6, 40)
    xs = rs.standard_normal(40)
    x0 = rs.standard_normal(40)
    for k in (1, 2, 5):
        x = cheb.richardson(lambda v: lam * v, lambda v: m * v, lam * xs, x0, k)
        assert np.allclose(xs - x, (1.0 - m * lam) ** k * (xs - x0), atol=1e-12)


@pytest.fixture(scope="module")
def two_level():
    """4x4 patches, 2 levels (160 and 40 unknowns): the coarse solve is exact."""
    from oracle import pum
    f = pum.fourier_source(pin.fourier_coefficients(0), 2.0)
    return pum.build_hierarchy(4, 3, 4, 2, f=f, constants=pin.NITSCHE_CONSTANTS[4])


def _dense(op, n):
    return np.column_stack([op(e) for e in np.eye(n)])


@pytest.mark.parametrize("smoother,cycle", [("cheb4", "vkk"), ("cheb4", "v2k0"), ("richardson", "vkk")])
def test_two_level_error_propagation(two_level, smoother, cycle):
    """I - B A of a two-level cycle is S C S for V(k,k) and C S' for V(2k,0), with the coarse
    correction C = I - P A_c^{-1} P^T A and S = p_k(M A) (Algorithm 3, Eq. (3.6)) or
    (I - M A)^k (Richardson), S' the degree-2k polynomial."""
    h = two_level
    st = solver.build_setup(h, k=2, mode="static", P0="lower")
    st.smoother, st.cycle = smoother, cycle
    A = h.A[0].to_dense()
    n = A.shape[0]
    B = _dense(lambda r: solver.vcycle(st, r), n)
    M = _dense(st.levels[0].M, n)
    P = h.P[0].to_dense()
    C = np.eye(n) - P @ np.linalg.solve(h.A[1].to_dense(), P.T @ A)
    deg = 2 if cycle == "vkk" else 4
    if smoother == "richardson":
        S = np.linalg.matrix_power(np.eye(n) - M @ A, deg)
    else:
        lam, V = np.linalg.eig(M @ A)  # real spectrum (M A is similar to G A G^T)
        S = (V @ np.diag(cheb.cheb4_residual_polynomial(deg, lam.real, st.levels[0].beta)) @ np.linalg.inv(V)).real
    E = S @ C @ S if cycle == "vkk" else C @ S
    assert np.max(np.abs(np.eye(n) - B @ A - E)) <= 1e-8 * np.max(np.abs(E))
    sym = np.max(np.abs(B - B.T)) / np.max(np.abs(B))
    assert (sym <= 1e-10) if cycle == "vkk" else (sym > 1e-3)


def test_bicgstab_solves_and_terminates():
    """BiCGStab (van der Vorst 1992): with the exact inverse as preconditioner one step solves
    the system; with an inexact non-symmetric one it reaches the dense solution."""
    rs = np.random.default_rng(12)
    n = 12
    Q = rs.standard_normal((n, n))
    A = Q @ Q.T + n * np.eye(n)
    b = rs.standard_normal(n)
    xd = np.linalg.solve(A, b)
    res1 = solver.bicgstab(lambda v: A @ v, lambda v: np.linalg.solve(A, v), b, rtol=1e-12)
    assert res1.converged and res1.iters == 1 and np.linalg.norm(res1.x - xd) <= 1e-12 * np.linalg.norm(xd)
    Bn = np.linalg.inv(A + 0.3 * rs.standard_normal((n, n)))  # non-symmetric approximate inverse
    res = solver.bicgstab(lambda v: A @ v, lambda v: Bn @ v, b, rtol=1e-13, maxit=100)
    assert res.converged and np.linalg.norm(res.x - xd) <= 1e-11 * np.linalg.norm(xd)
    assert res.history[0] == 1.0 and len(res.history) == res.iters + 1


def test_bicgstab_with_v2k0_cycle_matches_direct(small_biharmonic):
    h = small_biharmonic
    st = solver.build_setup(h, k=2, mode="static", P0="lower")
    st.cycle = "v2k0"
    res = solver.solve_bicgstab(st, h.b, rtol=1e-10)
    xd = np.linalg.solve(h.A[0].to_dense(), h.b)
    assert res.converged and np.linalg.norm(res.x - xd) <= 1e-7 * np.linalg.norm(xd)


def test_paper_ordering_of_convergence_factors(small_biharmonic):
    """Section 5: Chebyshev smoothing converges faster than Richardson smoothing (rho_A of the
    stationary V(k,k) cycles, static FSAI, k = 2; with non-adaptive FSAI Richardson does not
    converge in any useful sense (rho_A near or above 1), as the paper reports for non-nested
    FSAI below t_max = 9).  The V(2k,0)
    cycle converges too; its ordering against V(k,k) depends on the problem (here it is faster
    only for k = 1) and is not pinned."""
    h = small_biharmonic
    e0 = pin.uniform_vector(h.A[0].n_rows * 10, 5)
    rho = {}
    for smoother, cycle in (("cheb4", "vkk"), ("cheb4", "v2k0"), ("richardson", "vkk")):
        st = solver.build_setup(h, k=2, mode="static", P0="lower")
        st.smoother, st.cycle = smoother, cycle
        rho[(smoother, cycle)] = solver.convergence_factor(st, e0, 8)
    assert rho[("cheb4", "vkk")] < 0.5 and rho[("cheb4", "v2k0")] < 0.5
    assert rho[("richardson", "vkk")] > max(0.9, 2 * rho[("cheb4", "vkk")])
