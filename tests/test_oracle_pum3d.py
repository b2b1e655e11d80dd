"""Pins of the 3-D PUM oracle (Example 5.3: the biharmonic equation on the unit cube).

Each test checks the oracle against what the mathematics fixes independently of its arithmetic:
the size of the local spaces and the printed DoF count, polynomial reproduction of the local
projection, symmetry and definiteness of the stiffness matrix, and the Nitsche consistency
(patch test: a polynomial solution of degree <= p is reproduced exactly), which fixes the sign
and presence of every face term of the forms.
"""
import json
import os

import numpy as np
import numpy.polynomial.polynomial as P
import pytest

from oracle import pum, pum3d

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _rand_poly3(p, seed):
    rng = np.random.default_rng(seed)
    C = np.zeros((p + 1, p + 1, p + 1))
    for a in range(p + 1):
        for b in range(p + 1 - a):
            for c in range(p + 1 - a - b):
                C[a, b, c] = rng.standard_normal()
    return C


def _ev3(C, x, y, z, dx=0, dy=0, dz=0):
    D = C
    for axis, k in ((0, dx), (1, dy), (2, dz)):
        if k:
            D = P.polyder(D, k, axis=axis)
    return P.polyval3d(x, y, z, D)


def _bilap(C, x, y, z):
    return (_ev3(C, x, y, z, 4, 0, 0) + _ev3(C, x, y, z, 0, 4, 0) + _ev3(C, x, y, z, 0, 0, 4)
            + 2 * (_ev3(C, x, y, z, 2, 2, 0) + _ev3(C, x, y, z, 2, 0, 2) + _ev3(C, x, y, z, 0, 2, 2)))


def _boundary_data3(C):
    def g0(x, y, z):
        return _ev3(C, x, y, z)

    def g1(x, y, z):  # outward normal derivative on the faces of the unit cube
        n = [np.where(v <= 0.0, -1.0, np.where(v >= 1.0, 1.0, 0.0)) for v in (x, y, z)]
        return (n[0] * _ev3(C, x, y, z, 1, 0, 0) + n[1] * _ev3(C, x, y, z, 0, 1, 0)
                + n[2] * _ev3(C, x, y, z, 0, 0, 1))
    return [g0, g1]


def test_local_space_and_dof_count_of_example_5_3():
    """dim V_i = binom(p+3, 3) = 20 at p = 3; level 4 (16^3 patches) has the 81,920 unknowns the
    paper prints."""
    exps = pum3d.basis_exponents(3)
    assert pum3d.local_dim(3) == len(exps) == len(set(exps)) == 20
    assert all(sum(e) <= 3 for e in exps) and all(min(e) >= 0 for e in exps)
    assert 16 ** 3 * pum3d.local_dim(3) == GOLDEN["dof_biharmonic_cube_level4_p3"]["value"]
    assert pum.dof_count(4, 3, dim=3) == GOLDEN["dof_biharmonic_cube_level4_p3"]["value"]


@pytest.mark.parametrize("m,p", [(2, 2), (3, 3)])
def test_local_projection_reproduces_polynomials(m, p):
    """On every patch box the projection's Legendre expansion equals a polynomial of degree <= p."""
    C = _rand_poly3(p, 5 + p)
    coef = pum3d.local_projection(m, p, lambda x, y, z: _ev3(C, x, y, z))
    exps = pum3d.basis_exponents(p)
    d = len(exps)
    rng = np.random.default_rng(9)
    for i in range(m ** 3):
        ix, iy, iz = i % m, (i // m) % m, i // (m * m)
        boxes = [pum.patch_box_1d(m, a) for a in (ix, iy, iz)]
        pts = [lo + (hi - lo) * rng.random(20) for lo, hi in boxes]
        ref = [(2 * v - lo - hi) / (hi - lo) for v, (lo, hi) in zip(pts, boxes)]
        got = sum(coef[i * d + k] * pum.legendre(a, ref[0], 0) * pum.legendre(b, ref[1], 0) * pum.legendre(c, ref[2], 0)
                  for k, (a, b, c) in enumerate(exps))
        assert np.max(np.abs(got - _ev3(C, *pts))) <= 1e-12 * 10 * np.max(np.abs(C))


@pytest.mark.parametrize("m,p", [(2, 2), (2, 3)])
def test_stiffness_symmetric_positive_definite(m, p):
    A = pum3d.assemble(m, p, pum3d.nitsche_gamma(p, m)).A.to_dense()
    assert A.shape == (m ** 3 * pum3d.local_dim(p),) * 2
    assert np.max(np.abs(A - A.T)) <= 1e-12 * np.max(np.abs(A))
    assert np.min(np.linalg.eigvalsh(A)) > 0.0


@pytest.mark.parametrize("m,p", [(2, 2), (2, 3), (2, 4)])
def test_patch_test_exact_polynomial_solution(m, p):
    """Nitsche consistency (Examples 5.1 and 5.3): with f = Delta^2 u, g0 = u and g1 = du/dn the
    discrete solution is u itself for any u of degree <= p (degree 4 exercises the source term)."""
    C = _rand_poly3(p, 11 + p)
    f = (lambda x, y, z: _bilap(C, x, y, z)) if p >= 4 else None
    asm = pum3d.assemble(m, p, pum3d.nitsche_gamma(p, m), f=f, g=_boundary_data3(C))
    A = asm.A.to_dense()
    u = np.linalg.solve(A, asm.b)
    exact = pum3d.local_projection(m, p, lambda x, y, z: _ev3(C, x, y, z))
    kappa = np.linalg.cond(A)
    assert np.max(np.abs(u - exact)) <= 100 * kappa * 2.2e-16 * np.max(np.abs(exact))


def test_patch_test_fails_with_a_flipped_face_sign(monkeypatch):
    """The patch test is sharp: flipping the sign of the consistency term v d_n(Delta u) breaks it."""
    m, p = 2, 3
    C = _rand_poly3(p, 14)
    gamma = pum3d.nitsche_gamma(p, m)
    exact = pum3d.local_projection(m, p, lambda x, y, z: _ev3(C, x, y, z))
    good = pum3d.assemble(m, p, gamma, g=_boundary_data3(C))
    orig = pum3d.boundary_pairs

    def flipped(n, gam):
        return [(a, b, -c) if (a is pum3d.OP_I and c == 1.0) else (a, b, c) for (a, b, c) in orig(n, gam)]
    monkeypatch.setattr(pum3d, "boundary_pairs", flipped)
    bad = pum3d.assemble(m, p, gamma, g=_boundary_data3(C))
    assert np.max(np.abs(np.linalg.solve(good.A.to_dense(), good.b) - exact)) < 1e-8
    assert np.max(np.abs(np.linalg.solve(bad.A.to_dense(), bad.b) - exact)) > 1e-4


@pytest.mark.parametrize("m_f,p", [(2, 2), (4, 3)])
def test_prolongation_reproduces_polynomials(m_f, p):
    """Section 4: the L2 projection of a degree-p polynomial onto V_i is the polynomial itself, so
    P maps the coarse representation of the polynomial to the fine one; a fine patch meets at most
    two coarse patches per direction."""
    C = _rand_poly3(p, 5)
    u = lambda x, y, z: _ev3(C, x, y, z)
    Pm = pum3d.prolongation(m_f, p)
    fine = pum3d.local_projection(m_f, p, u)
    assert np.max(np.abs(Pm.matvec(pum3d.local_projection(m_f // 2, p, u)) - fine)) <= 1e-12 * np.max(np.abs(fine))
    assert Pm.nnzb == (8 if m_f == 2 else (2 * m_f - 2) ** 3)


def test_galerkin_hierarchy_on_the_cube():
    """Two levels (4^3 and 2^3 patches, p = 2): the coarse operator P^T A P is symmetric positive
    definite and equals the dense triple product."""
    h = pum3d.build_hierarchy(4, 2, 2)
    A0, P0, A1 = h.A[0].to_dense(), h.P[0].to_dense(), h.A[1].to_dense()
    assert np.max(np.abs(A1 - P0.T @ A0 @ P0)) <= 1e-12 * np.max(np.abs(A1))
    assert np.max(np.abs(A1 - A1.T)) <= 1e-12 * np.max(np.abs(A1))
    assert np.min(np.linalg.eigvalsh(A1)) > 0.0
