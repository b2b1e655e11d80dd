"""Pins of the PUM discretisation oracle (Section 4, Examples 5.1, 5.3, 5.4).

Each test checks the oracle against something the paper or the mathematics fixes
independently of the oracle's own arithmetic: the partition-of-unity identity,
polynomial reproduction, printed DoF counts, symmetry and definiteness, the
Nitsche consistency (patch test) and closed-form energies.
"""
import json
import os
from math import comb

import numpy as np
import numpy.polynomial.polynomial as P
import pytest

from oracle import blocks as bk
from oracle import pum

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


# --------------------------------------------------------------------------- P-1

@pytest.mark.parametrize("m", [1, 2, 3, 4, 8])
def test_partition_of_unity_sums_to_one(m):
    """Section 4: 0 <= phi_i <= 1 and sum_i phi_i = 1 on the closed domain."""
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.random(400), [0.0, 1.0], pum.breakpoints_1d(m)])
    vals = np.array([pum.pu_1d(m, a, x, 0) for a in range(m)])
    assert np.all(vals >= 0.0) and np.all(vals <= 1.0)
    assert np.max(np.abs(vals.sum(axis=0) - 1.0)) <= 1e-15
    for r in (1, 2, 3):
        dsum = np.array([pum.pu_1d(m, a, x[:400], r) for a in range(m)]).sum(axis=0)
        assert np.max(np.abs(dsum)) <= 1e-9 * m ** r


@pytest.mark.parametrize("m", [2, 4])
def test_partition_of_unity_is_c2_and_supported_on_patch(m):
    """phi_a, phi_a', phi_a'' are continuous at every breakpoint; phi_a vanishes outside omega_a."""
    eps = 1e-10
    for a in range(m):
        lo, hi = pum.patch_box_1d(m, a)
        assert lo == max((a - 0.25) / m, 0.0) and hi == min((a + 1.25) / m, 1.0)
        out = np.array([lo - 1e-3, hi + 1e-3])
        out = out[(out > 0) & (out < 1)]
        assert np.all(pum.pu_1d(m, a, out, 0) == 0.0)
        for x in pum.breakpoints_1d(m)[1:-1]:
            for r in range(3):
                left = pum.pu_1d(m, a, np.array([x - eps]), r)[0]
                right = pum.pu_1d(m, a, np.array([x + eps]), r)[0]
                scale = (2.0 * m) ** r
                assert abs(left - right) <= 1e-6 * scale * 60


# --------------------------------------------------------------------------- P-2

def _rand_poly(p, seed):
    rng = np.random.default_rng(seed)
    C = np.zeros((p + 1, p + 1))
    for a in range(p + 1):
        for b in range(p + 1 - a):
            C[a, b] = rng.standard_normal()
    return C


def _ev(C, x, y, dx=0, dy=0):
    D = P.polyder(P.polyder(C, dx, axis=0), dy, axis=1) if (dx or dy) else C
    return P.polyval2d(x, y, D)


@pytest.mark.parametrize("m,p", [(2, 2), (4, 3), (3, 5)])
def test_polynomial_reproduction(m, p):
    """Section 4: with u_i = q on every patch, sum_i phi_i u_i = q for q of degree <= p."""
    C = _rand_poly(p, 7)
    coef = pum.local_projection(m, p, lambda x, y: _ev(C, x, y))
    rng = np.random.default_rng(3)
    x, y = rng.random(200), rng.random(200)
    got = pum.evaluate(m, p, coef, x, y)
    assert np.max(np.abs(got - _ev(C, x, y))) <= 1e-12 * np.max(np.abs(C)) * 10
    # a derivative of the reproduced function is reproduced as well
    got_dx = pum.evaluate(m, p, coef, x, y, op={(1, 0): 1.0})
    assert np.max(np.abs(got_dx - _ev(C, x, y, 1, 0))) <= 1e-10 * np.max(np.abs(C)) * 10


@pytest.mark.parametrize("m", [2, 4])
def test_constant_has_unit_coefficients_and_unit_mass(m):
    """The constant 1 has coefficient 1 on each patch's degree-0 function; its L2 norm^2 is |Omega| = 1."""
    p = 3
    d = pum.local_dim(p)
    coef = pum.local_projection(m, p, lambda x, y: np.ones_like(x))
    expect = np.zeros(m * m * d)
    expect[::d] = 1.0
    assert np.max(np.abs(coef - expect)) <= 1e-14
    asm = pum.assemble(m, p, 4, pum.nitsche_gamma(4, p, m))
    assert abs(coef @ asm.M.matvec(coef) - 1.0) <= 1e-13


# --------------------------------------------------------------------------- P-3

def test_dof_counts_printed_in_paper():
    """Example 5.1: 100,336 DoF; Example 5.3: 81,920 DoF; dim V_i = binom(p+d, d)."""
    g = GOLDEN
    assert pum.dof_count(7, 2, p_boundary=3) == g["dof_biharmonic_square_level7_p2_boundary_p3"]["value"]
    assert pum.dof_count(4, 3, dim=3) == g["dof_biharmonic_cube_level4_p3"]["value"]
    assert comb(3 + 3, 3) == g["local_dim_3d"]["p3"] and comb(4 + 3, 3) == g["local_dim_3d"]["p4"]
    assert (2 ** 3) ** 2 == g["patches_level3_2d"]["value"]
    for l in range(1, 9):
        for p in range(1, 6):
            assert pum.dof_count(l, p) == pum.local_dim(p) * 4 ** l
    assert pum.local_dim(3) == 10 and pum.local_dim(5) == 21 and len(pum.basis_exponents(5)) == 21


def test_assembled_sizes_and_stencils(small_biharmonic):
    """Finest level: 3x3 block stencil, (3m-2)^2 blocks; Galerkin levels: 5x5 stencil, (5m-6)^2 blocks."""
    h = small_biharmonic
    for l, (m, A) in enumerate(zip(h.m, h.A)):
        assert A.n_rows == m * m and A.d == 10
        if l == 0:
            assert A.nnzb == (3 * m - 2) ** 2
        elif m >= 2:
            assert A.nnzb == (5 * m - 6) ** 2 if m >= 3 else A.nnzb == (m * m) ** 2
        for i in range(A.n_rows):
            ix, iy = i % m, i // m
            for j in A.row(i):
                jx, jy = j % m, j // m
                r = 1 if l == 0 else 2
                assert abs(jx - ix) <= r and abs(jy - iy) <= r


# --------------------------------------------------------------------------- P-4

@pytest.mark.parametrize("order,p,m", [(4, 3, 2), (4, 3, 4), (4, 3, 8), (6, 5, 2), (6, 5, 4)])
def test_stiffness_symmetric_positive_definite(order, p, m):
    A = pum.assemble(m, p, order, pum.nitsche_gamma(order, p, m), with_mass=False).A.to_dense()
    assert np.max(np.abs(A - A.T)) <= 1e-14 * np.max(np.abs(A))
    np.linalg.cholesky(A)
    assert np.linalg.eigvalsh(A)[0] > 0.0


# --------------------------------------------------------------------------- P-5

def _boundary_data(C, order):
    def normal(x, y):
        nx = np.where(x <= 0.0, -1.0, np.where(x >= 1.0, 1.0, 0.0))
        ny = np.where(y <= 0.0, -1.0, np.where(y >= 1.0, 1.0, 0.0))
        return nx, ny

    def g0(x, y):
        return _ev(C, x, y)

    def g1(x, y):
        nx, ny = normal(x, y)
        return nx * _ev(C, x, y, 1, 0) + ny * _ev(C, x, y, 0, 1)

    def g2(x, y):
        return _ev(C, x, y, 2, 0) + _ev(C, x, y, 0, 2)
    return [g0, g1, g2][: order // 2]


@pytest.mark.parametrize("order,p,m", [(4, 3, 2), (4, 3, 4), (4, 4, 2), (6, 5, 2)])
def test_patch_test_exact_polynomial_solution(order, p, m):
    """Nitsche consistency (Examples 5.1, 5.4): a polynomial solution of degree <= p is reproduced.

    Biharmonic: f = Delta^2 u; triharmonic: f = -Delta^3 u; g_0 = u, g_1 = du/dn, g_2 = Delta u.
    This fixes the signs of every boundary term of a_n and l_n.
    """
    C = _rand_poly(p, 11 + p)
    if order == 4:
        f = lambda x, y: _ev(C, x, y, 4, 0) + 2 * _ev(C, x, y, 2, 2) + _ev(C, x, y, 0, 4)
    else:
        f = lambda x, y: -(_ev(C, x, y, 6, 0) + 3 * _ev(C, x, y, 4, 2) + 3 * _ev(C, x, y, 2, 4) + _ev(C, x, y, 0, 6))
    asm = pum.assemble(m, p, order, pum.nitsche_gamma(order, p, m), f=f, g=_boundary_data(C, order),
                       with_mass=False)
    A = asm.A.to_dense()
    u = np.linalg.solve(A, asm.b)
    exact = pum.local_projection(m, p, lambda x, y: _ev(C, x, y))
    kappa = np.linalg.cond(A)
    assert np.max(np.abs(u - exact)) <= 100 * kappa * 2.2e-16 * np.max(np.abs(exact))


def test_patch_test_fails_with_a_flipped_boundary_sign():
    """The patch test is sharp: flipping the sign of the consistency term breaks it."""
    order, p, m = 4, 3, 2
    C = _rand_poly(p, 14)
    gamma = pum.nitsche_gamma(order, p, m)
    asm = pum.assemble(m, p, order, gamma, f=None, g=_boundary_data(C, order), with_mass=False)
    orig = pum.Equation.boundary_pairs

    def flipped(self, n, gam):
        pairs = orig(self, n, gam)
        return [(a, b, -c) if (a is pum.OP_I and c == 1.0) else (a, b, c) for (a, b, c) in pairs]
    pum.Equation.boundary_pairs = flipped
    try:
        bad = pum.assemble(m, p, order, gamma, f=None, g=_boundary_data(C, order), with_mass=False)
    finally:
        pum.Equation.boundary_pairs = orig
    exact = pum.local_projection(m, p, lambda x, y: _ev(C, x, y))
    good = np.linalg.solve(asm.A.to_dense(), asm.b)
    wrong = np.linalg.solve(bad.A.to_dense(), bad.b)
    assert np.max(np.abs(good - exact)) < 1e-8
    assert np.max(np.abs(wrong - exact)) > 1e-4


# ------------------------------------------------- anisotropic biharmonic (Example 5.2)

S_ANISO = pum.anisotropy(10.0, np.pi / 3)


def test_anisotropy_tensor():
    """S = R(theta) diag(kappa, 1) R(theta)^T: eigenvalue kappa along (cos theta, sin theta)."""
    S = np.array([[S_ANISO[0], S_ANISO[1]], [S_ANISO[1], S_ANISO[2]]])
    v = np.array([np.cos(np.pi / 3), np.sin(np.pi / 3)])
    assert np.allclose(S @ v, 10.0 * v, atol=1e-14)
    assert np.allclose(np.linalg.eigvalsh(S), [1.0, 10.0], atol=1e-13)
    assert pum.anisotropy(1.0, 0.7) == pytest.approx(pum.ISOTROPIC, abs=1e-15)


def test_isotropic_tensor_gives_the_isotropic_form_bitwise():
    m, p = 4, 3
    g = pum.nitsche_gamma(4, p, m)
    f = pum.fourier_source(np.ones((2, 2)), 2.0)
    a = pum.assemble(m, p, 4, g, f=f, with_mass=False)
    b = pum.assemble(m, p, 4, pum.nitsche_gamma(4, p, m, S=pum.ISOTROPIC), f=f, with_mass=False, S=pum.ISOTROPIC)
    assert np.array_equal(a.A.blocks, b.A.blocks) and np.array_equal(a.b, b.b)


@pytest.mark.parametrize("m", [2, 4, 8])
def test_anisotropic_stiffness_spd(m):
    """With gamma^(0) scaled by |S|^2 the anisotropic Nitsche matrix is SPD (kappa = 10)."""
    A = pum.assemble(m, 3, 4, pum.nitsche_gamma(4, 3, m, S=S_ANISO), with_mass=False, S=S_ANISO).A.to_dense()
    assert np.max(np.abs(A - A.T)) <= 1e-14 * np.max(np.abs(A))
    np.linalg.cholesky(A)


@pytest.mark.parametrize("m", [2, 4])
def test_anisotropic_patch_test(m):
    """Example 5.2: a cubic u solves S_ij S_kl u_,ijkl = f with f from u's fourth derivatives
    (zero for cubics, so take p = 4 and a quartic), g_0 = u, g_1 = grad u . (S n): the Nitsche
    solution reproduces u exactly.  A wrong S in any consistency term breaks this."""
    p = 4
    C = _rand_poly(p, 31 + m)
    s11, s12, s22 = S_ANISO
    # S_ij S_kl d_ijkl u = (s11 d_xx + 2 s12 d_xy + s22 d_yy)^2 u
    coef = {(4, 0): s11 * s11, (3, 1): 4 * s11 * s12, (2, 2): 2 * s11 * s22 + 4 * s12 * s12,
            (1, 3): 4 * s12 * s22, (0, 4): s22 * s22}
    f = lambda x, y: sum(c * _ev(C, x, y, a, b) for (a, b), c in coef.items())

    def sn(x, y):
        nx = np.where(x <= 0.0, -1.0, np.where(x >= 1.0, 1.0, 0.0))
        ny = np.where(y <= 0.0, -1.0, np.where(y >= 1.0, 1.0, 0.0))
        return s11 * nx + s12 * ny, s12 * nx + s22 * ny

    def g1(x, y):
        a, b = sn(x, y)
        return a * _ev(C, x, y, 1, 0) + b * _ev(C, x, y, 0, 1)
    g = [lambda x, y: _ev(C, x, y), g1]
    asm = pum.assemble(m, p, 4, pum.nitsche_gamma(4, p, m, S=S_ANISO), f=f, g=g, with_mass=False, S=S_ANISO)
    A = asm.A.to_dense()
    u = np.linalg.solve(A, asm.b)
    exact = pum.local_projection(m, p, lambda x, y: _ev(C, x, y))
    assert np.max(np.abs(u - exact)) <= 100 * np.linalg.cond(A) * 2.2e-16 * np.max(np.abs(exact))
    iso = pum.assemble(m, p, 4, pum.nitsche_gamma(4, p, m, S=S_ANISO), f=f, g=g, with_mass=False)
    assert np.max(np.abs(np.linalg.solve(iso.A.to_dense(), iso.b) - exact)) > 1e-3 * np.max(np.abs(exact))


# --------------------------------------------------------------------------- P-6

@pytest.mark.parametrize("order,p", [(4, 3), (6, 5)])
def test_energy_of_linear_function_is_boundary_penalty(order, p):
    """For linear u, Delta u = 0, so a_n(u,u) = int_dOmega gamma0 u^2 + gamma1 (du/dn)^2 exactly."""
    m = 2
    c0, c1, c2 = 0.3, -1.1, 0.7
    u = lambda x, y: c0 + c1 * x + c2 * y
    gamma = pum.nitsche_gamma(order, p, m)
    A = pum.assemble(m, p, order, gamma, with_mass=False).A
    coef = pum.local_projection(m, p, u)

    def int_sq(a, b):  # int_0^1 (a + b t)^2 dt
        return a * a + a * b + b * b / 3.0
    e_u2 = int_sq(c0, c2) + int_sq(c0 + c1, c2) + int_sq(c0, c1) + int_sq(c0 + c2, c1)
    e_dn2 = 2 * c1 ** 2 + 2 * c2 ** 2
    expect = gamma[0] * e_u2 + gamma[1] * e_dn2
    assert abs(coef @ A.matvec(coef) - expect) <= 1e-12 * expect


# --------------------------------------------------------------------------- P-7

@pytest.mark.parametrize("m_f,p", [(4, 3), (8, 3), (4, 5)])
def test_prolongation_reproduces_polynomials(m_f, p):
    """Section 4: the L2 projection of a degree-p polynomial onto V_i is the polynomial itself."""
    C = _rand_poly(p, 5)
    q = lambda x, y: _ev(C, x, y)
    Pm = pum.prolongation(m_f, p)
    coarse = pum.local_projection(m_f // 2, p, q)
    fine = pum.local_projection(m_f, p, q)
    assert np.max(np.abs(Pm.matvec(coarse) - fine)) <= 1e-12 * np.max(np.abs(fine))
    # fine patch meets at most 2 coarse patches per direction: (2 m_f - 2)^2 blocks
    assert Pm.nnzb == (2 * m_f - 2) ** 2


def test_galerkin_levels_symmetric_positive_definite(small_biharmonic):
    for A in small_biharmonic.A[1:]:
        D = A.to_dense()
        assert np.max(np.abs(D - D.T)) <= 1e-12 * np.max(np.abs(D))
        np.linalg.cholesky(D)


def test_galerkin_product_matches_dense_triple_product(small_biharmonic):
    h = small_biharmonic
    Pd = h.P[1].to_dense()
    Ac = Pd.T @ h.A[1].to_dense() @ Pd
    assert np.max(np.abs(h.A[2].to_dense() - Ac)) <= 1e-12 * np.max(np.abs(Ac))
    # structural pattern of R A P equals the pattern read from the product of the patterns
    pat = bk.product_pattern(bk.product_pattern(h.P[1].transpose().pattern(), h.A[1].pattern()), h.P[1].pattern())
    assert pat == h.A[2].pattern()


def test_anisotropic_neighbourhood_figure_fixture():
    """The printed average neighbourhoods of Example 5.2 (tests/golden/aniso_neighbourhoods.json)
    read as 0.5 x the fraction of rows of F^T S^-1 F containing an offset: the centre is 0.5,
    offsets that every interior row has lose exactly the boundary rows (127/128 per direction at
    level 7), and the figure is point-symmetric (F^T S^-1 F is symmetric)."""
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "aniso_neighbourhoods.json")))
    m = 128
    for name, op in g["opacity"].items():
        assert op["0,0"] == 0.5
        for key in ("0,1", "1,0", "0,-1", "-1,0"):
            assert op[key] == pytest.approx(0.5 * (m - 1) / m, abs=5e-6)
        for key, v in op.items():
            dx, dy = (int(t) for t in key.split(","))
            assert op.get(f"{-dx},{-dy}") == v, (name, key)
            assert v <= 0.5 * (m - abs(dx)) * (m - abs(dy)) / m ** 2 + 5e-6
