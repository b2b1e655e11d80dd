"""Pins of the raised-degree PUM space (Example 5.1: p = 2 inside, 3 on patches meeting the boundary).

Checked against what the paper and the mathematics fix: the printed count of unknowns, equality
with the uniform-degree assembly when no degree is raised, symmetry and definiteness, and the
Nitsche patch test (a polynomial of degree <= 2 is reproduced exactly).
"""
import json
import os

import numpy as np
import numpy.polynomial.polynomial as P
import pytest

from oracle import pum, pum_raise

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _poly2(seed):
    rng = np.random.default_rng(seed)
    C = np.zeros((3, 3))
    for a in range(3):
        for b in range(3 - a):
            C[a, b] = rng.standard_normal()
    return C


def _ev(C, x, y, dx=0, dy=0):
    D = P.polyder(P.polyder(C, dx, axis=0), dy, axis=1) if (dx or dy) else C
    return P.polyval2d(x, y, D)


def _boundary_data(C):
    def g0(x, y):
        return _ev(C, x, y)

    def g1(x, y):
        nx = np.where(x <= 0.0, -1.0, np.where(x >= 1.0, 1.0, 0.0))
        ny = np.where(y <= 0.0, -1.0, np.where(y >= 1.0, 1.0, 0.0))
        return nx * _ev(C, x, y, 1, 0) + ny * _ev(C, x, y, 0, 1)
    return [g0, g1]


def test_unknowns_of_example_5_1():
    """Level l has 2^l x 2^l patches; the count matches the closed form at small levels and the
    100,336 unknowns the paper prints for its level 7."""
    for level in range(1, 5):
        m = 2 ** level
        assert pum_raise.offsets(pum_raise.patch_degrees(m, 2, 3))[-1] == pum.dof_count(level, 2, 3)
    printed = GOLDEN["dof_biharmonic_square_level7_p2_boundary_p3"]["value"]
    assert pum_raise.offsets(pum_raise.patch_degrees(128, 2, 3))[-1] == printed


@pytest.mark.parametrize("m,p", [(2, 2), (4, 3)])
def test_uniform_degree_equals_the_uniform_assembly(m, p):
    """With no degree raised the space is the uniform one: same matrix and load vector."""
    f = lambda x, y: np.sin(np.pi * x) * np.cos(np.pi * y) + x
    raised = pum_raise.assemble(m, p, p, f=f)
    uniform = pum.assemble(m, p, 4, pum.nitsche_gamma(4, p, m), f=f, with_mass=False)
    A = uniform.A.to_dense()
    assert np.max(np.abs(raised.A.toarray() - A)) <= 1e-13 * np.max(np.abs(A))
    assert np.max(np.abs(raised.b - uniform.b)) <= 1e-13 * np.max(np.abs(uniform.b))


def test_raised_stiffness_symmetric_positive_definite():
    asm = pum_raise.assemble(4, 2, 3)
    A = asm.A.toarray()
    assert asm.degrees.count(3) == 12 and asm.degrees.count(2) == 4
    assert np.max(np.abs(A - A.T)) <= 1e-12 * np.max(np.abs(A))
    assert np.min(np.linalg.eigvalsh(A)) > 0.0


@pytest.mark.parametrize("m", [4, 6])
def test_raised_patch_test(m):
    """Nitsche consistency in the raised space: a quadratic solution (f = Delta^2 u = 0, g0 = u,
    g1 = du/dn) is reproduced exactly, on interior and raised patches alike."""
    C = _poly2(31 + m)
    asm = pum_raise.assemble(m, 2, 3, g=_boundary_data(C))
    A = asm.A.toarray()
    u = np.linalg.solve(A, asm.b)
    exact = pum_raise.local_projection(m, 2, 3, lambda x, y: _ev(C, x, y))
    kappa = np.linalg.cond(A)
    assert np.max(np.abs(u - exact)) <= 100 * kappa * 2.2e-16 * np.max(np.abs(exact))


@pytest.mark.parametrize("m_f", [4, 8])
def test_raised_prolongation_reproduces_quadratics_and_galerkin_is_spd(m_f):
    """Section 4: the L2 projection reproduces a polynomial both spaces contain (degree <= 2), so P
    maps its coarse representation to its fine one; the coarse operator P^T A P of the raised
    spaces is symmetric positive definite."""
    C = _poly2(7)
    u = lambda x, y: _ev(C, x, y)
    Pm = pum_raise.prolongation(m_f, 2, 3)
    fine = pum_raise.local_projection(m_f, 2, 3, u)
    coarse = pum_raise.local_projection(m_f // 2, 2, 3, u)
    assert np.max(np.abs(Pm @ coarse - fine)) <= 1e-12 * np.max(np.abs(fine))
    A = pum_raise.assemble(m_f, 2, 3).A
    Ac = (Pm.T @ A @ Pm).toarray()
    assert np.max(np.abs(Ac - Ac.T)) <= 1e-12 * np.max(np.abs(Ac))
    assert np.min(np.linalg.eigvalsh(Ac)) > 0.0


def test_padded_layout_solves_the_raised_system():
    """The raised space on uniform 10 x 10 blocks (interior patches padded with decoupled unknowns
    of unit diagonal): the multilevel PCG on the padded hierarchy keeps every padded unknown at
    zero and its real unknowns solve the raised system."""
    import scipy.sparse.linalg as spla
    from oracle import solver
    h = pum_raise.padded_hierarchy(8, 2, 3, 3, f=lambda x, y: np.sin(np.pi * x) * np.sin(np.pi * y) + 0.5)
    assert [A.n_rows for A in h.A] == [64, 16, 4] and h.A[0].d == 10
    xr = spla.spsolve(h.A_raised.tocsc(), h.b_raised)
    res = solver.solve(solver.build_setup(h, k=2, mode="adaptive", P0="lower", t_max=3), h.b, rtol=1e-10)
    pad = np.setdiff1d(np.arange(len(h.b)), h.real[0])
    assert res.converged and np.all(res.x[pad] == 0.0)
    assert np.linalg.norm(res.x[h.real[0]] - xr) <= 1e-9 * np.linalg.norm(xr)
