"""Multilevel V(k,k)-cycle and preconditioned CG (Section 5, Example 5.1).

Test infrastructure only (never imported by the CUDA library).

* V(k,k) (Section 5): on every level but the coarsest, pre-smooth with Algorithm 3
  from x0 = 0, restrict the residual with R = P^T, recurse, prolongate and add, and
  post-smooth with the same Algorithm 3 polynomial; the coarsest level is solved
  directly (dense Cholesky).  With the same polynomial before and after, the cycle
  is a symmetric operator, so it can precondition CG.
* PCG: standard preconditioned conjugate gradients from x0 = 0 with one V(k,k)
  cycle as preconditioner, stopped when the recursively updated ||r_k|| / ||b||
  reaches rtol.  The paper runs the cycle as a stationary iteration and names CG
  as the Krylov method for the symmetric cycle (Conclusions).
* ``convergence_factor``: rho_A of Example 5.1 for the stationary cycle run on the
  error equation (b = 0), e_n = (I - B A) e_{n-1}.
* Variants of Section 5: Richardson smoothing instead of Algorithm 3 (``smoother =
  "richardson"``), and the non-symmetric V(2k,0) cycle (``cycle = "v2k0"``: 2k steps of
  pre-smoothing, none after the coarse correction), which cannot precondition CG; the
  Conclusions name BiCGStab for it: ``bicgstab`` is van der Vorst's (1992) BiCGStab with the
  cycle as right preconditioner.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla

from . import blocks as bk
from . import cheb, fsai, pum


@dataclasses.dataclass
class Level:
    A: bk.BlockCSR
    P: bk.BlockCSR | None      # prolongation from the next coarser level (None on the coarsest)
    M: object | None           # callable r -> M r (None on the coarsest)
    beta: float | None
    chol: np.ndarray | None    # dense Cholesky factor on the coarsest level


@dataclasses.dataclass
class Setup:
    levels: list
    k: int
    smoother: str = "cheb4"   # "cheb4" (Algorithm 3) or "richardson"
    cycle: str = "vkk"        # "vkk": V(k,k); "v2k0": V(2k,0)


def make_smoother(A: bk.BlockCSR, mode: str, P0: str, t_max: int, tau: float, nested: bool,
                  tie_rel: float = 1e-9, row_map=map):
    """Block-FSAI smoother of one level: returns (M callable, FSAI object(s)).

    row_map (a map over block rows, e.g. a process pool's) runs Algorithm 1 row by row with
    adaptive_row: the rows of Algorithm 1 are independent, so this equals adaptive_fsai's
    pattern (pinned by a test)."""
    p0 = fsai.lower_pattern(A) if P0 == "lower" else fsai.diag_pattern(A.n_rows)
    if nested:
        nf = fsai.nested_fsai(A, p0, t_max, tau, tie_rel, adaptive=(mode == "adaptive"))
        return nf.apply, nf
    if mode == "adaptive" and row_map is not map:
        rows = list(row_map(_AdaptiveRow(A, p0, t_max, tau, tie_rel), range(A.n_rows)))
        f = fsai.fsai(A, rows)
    elif mode == "adaptive":
        f = fsai.adaptive_fsai(A, p0, t_max, tau, tie_rel).fsai
    else:
        f = fsai.fsai(A, p0)
    return (lambda r, G=f.G: fsai.apply_M(G, r)), f


class _AdaptiveRow:
    """Picklable per-row call of Algorithm 1 (fsai.adaptive_row) for a map over block rows."""

    def __init__(self, A, P0, t_max, tau, tie_rel):
        self.A, self.P0, self.t_max, self.tau, self.tie_rel = A, P0, t_max, tau, tie_rel

    def __call__(self, k):
        return fsai.adaptive_row(self.A, k, self.P0[k], self.t_max, self.tau, self.tie_rel)


def build_setup(h: pum.Hierarchy, k: int, mode: str = "static", P0: str = "lower", t_max: int = 0,
                tau: float = 1.0, nested: bool = False, lanczos_seed: int = 0, row_map=map) -> Setup:
    """FSAI smoothers, Lanczos beta = 1.01 lambda_max(M A) per level, coarse Cholesky."""
    levels = []
    L = len(h.A)
    for l in range(L):
        A = h.A[l]
        if l == L - 1:
            levels.append(Level(A, None, None, None, np.linalg.cholesky(A.to_dense())))
            continue
        Mop, obj = make_smoother(A, mode, P0, t_max, tau, nested, row_map=row_map)
        Gop = _symmetric_form(obj, nested)
        lam = cheb.lanczos_lmax(lambda v: Gop(A, v), A.n_rows * A.d, seed=lanczos_seed + l)
        levels.append(Level(A, h.P[l], Mop, cheb.LANCZOS_SAFETY * lam, None))
    return Setup(levels, k)


def _symmetric_form(obj, nested):
    """v -> G A G^T v, the symmetric form of M A whose spectrum equals that of M A."""
    if nested:
        def op(A, v):
            Gt = obj.F0.to_scipy().T @ (obj.inner.G.to_scipy().T @ v)
            return obj.inner.G.matvec(obj.F0.matvec(A.matvec(Gt)))
        return op

    def op(A, v):
        return obj.G.matvec(A.matvec(obj.G.to_scipy().T @ v))
    return op


def _smooth(setup: Setup, lev: Level, b: np.ndarray, x0, steps: int) -> np.ndarray:
    if setup.smoother == "richardson":
        return cheb.richardson(lev.A.matvec, lev.M, b, x0, steps)
    return cheb.cheb4(lev.A.matvec, lev.M, b, x0, lev.beta, steps)


def vcycle(setup: Setup, r: np.ndarray, l: int = 0) -> np.ndarray:
    """z = B r, one V(k,k) (or V(2k,0)) cycle started on level l."""
    lev = setup.levels[l]
    if lev.chol is not None:
        return sla.cho_solve((lev.chol, True), r)
    pre = setup.k if setup.cycle == "vkk" else 2 * setup.k
    x = _smooth(setup, lev, r, None, pre)
    res = r - lev.A.matvec(x)
    rc = lev.P.to_scipy().T @ res
    ec = vcycle(setup, rc, l + 1)
    x = x + lev.P.matvec(ec)
    if setup.cycle == "vkk":
        x = _smooth(setup, lev, r, x, setup.k)
    return x


@dataclasses.dataclass
class PCGResult:
    x: np.ndarray
    history: list      # ||r_j|| / ||b||, j = 0..iters
    iters: int
    converged: bool


def pcg(Aop, Bop, b: np.ndarray, rtol: float = 1e-8, maxit: int = 500) -> PCGResult:
    """Preconditioned conjugate gradients from x0 = 0 (recursive residual stopping test)."""
    x = np.zeros_like(b)
    r = b.copy()
    nb = float(np.linalg.norm(b))
    hist = [1.0]
    if nb == 0.0:
        return PCGResult(x, hist, 0, True)
    z = Bop(r)
    p = z.copy()
    rz = float(r @ z)
    for it in range(1, maxit + 1):
        q = Aop(p)
        alpha = rz / float(p @ q)
        x = x + alpha * p
        r = r - alpha * q
        hist.append(float(np.linalg.norm(r)) / nb)
        if hist[-1] <= rtol:
            return PCGResult(x, hist, it, True)
        z = Bop(r)
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return PCGResult(x, hist, maxit, False)


def bicgstab(Aop, Bop, b: np.ndarray, rtol: float = 1e-8, maxit: int = 500) -> PCGResult:
    """BiCGStab (van der Vorst 1992) from x0 = 0 with B as right preconditioner; the shadow
    residual is r0 = b.  history holds ||r_j|| / ||b|| after each full step (the stop test);
    a half step whose s already meets rtol ends the iteration there."""
    x = np.zeros_like(b)
    r = b.copy()
    rhat = b.copy()
    nb = float(np.linalg.norm(b))
    hist = [1.0]
    if nb == 0.0:
        return PCGResult(x, hist, 0, True)
    rho_old = alpha = omega = 1.0
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    for it in range(1, maxit + 1):
        rho = float(rhat @ r)
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        ph = Bop(p)
        v = Aop(ph)
        alpha = rho / float(rhat @ v)
        s = r - alpha * v
        if float(np.linalg.norm(s)) / nb <= rtol:
            x = x + alpha * ph
            hist.append(float(np.linalg.norm(s)) / nb)
            return PCGResult(x, hist, it, True)
        sh = Bop(s)
        t = Aop(sh)
        omega = float(t @ s) / float(t @ t)
        x = x + alpha * ph + omega * sh
        r = s - omega * t
        hist.append(float(np.linalg.norm(r)) / nb)
        if hist[-1] <= rtol:
            return PCGResult(x, hist, it, True)
        rho_old = rho
    return PCGResult(x, hist, maxit, False)


def solve_bicgstab(setup: Setup, b: np.ndarray, rtol: float = 1e-8, maxit: int = 500) -> PCGResult:
    A = setup.levels[0].A
    return bicgstab(A.matvec, lambda r: vcycle(setup, r), b, rtol, maxit)


def solve(setup: Setup, b: np.ndarray, rtol: float = 1e-8, maxit: int = 500) -> PCGResult:
    A = setup.levels[0].A
    return pcg(A.matvec, lambda r: vcycle(setup, r), b, rtol, maxit)


def convergence_factor(setup: Setup, e0: np.ndarray, n: int) -> float:
    """rho_A = (e_n^T A e_n / e_0^T A e_0)^(1/(2n)) for the stationary V-cycle on A e = 0."""
    A = setup.levels[0].A
    e = e0.copy()
    for _ in range(n):
        e = e - vcycle(setup, A.matvec(e))
    return float((e @ A.matvec(e)) / (e0 @ A.matvec(e0))) ** (1.0 / (2 * n))
