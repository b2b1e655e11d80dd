"""Fourth-kind Chebyshev smoothing and lambda_max estimation (Section 3.1, Section 5).

Test infrastructure only (never imported by the CUDA library).

* ``cheb4``: Algorithm 3 step by step: r = b - A x0, p = M r, mu = 1/3, d = 4/beta,
  x = x0 + d mu p; then for i = 2..k: r = b - A x, p = mu^2 p + M r, mu = 1/(2 - mu),
  x = x + d mu p.  The residual is recomputed from b - A x in every iteration.
* ``richardson``: Richardson smoothing (Section 3.1), k steps of x = x + M (b - A x),
  so the error propagates by S = (I - M A)^k.
* ``w4``: W_k, the Chebyshev polynomial of the fourth kind, by its three-term
  recurrence W_0 = 1, W_1 = 2t + 1, W_{n+1} = 2t W_n - W_{n-1} (Section 3.1);
  the optimal smoother polynomial of Eq. (3.6) is W_k(1 - 2 lambda / beta) / (2k + 1).
* ``lanczos_lmax``: the Lanczos estimate of lambda_max of the symmetric form
  G A G^T of M A (Section 5: 100 iterations, estimate multiplied by 1.01).  The start
  vector is SplitMix64 U(-1,1), normalised; no reorthogonalisation; the iteration
  stops early when beta_{j+1} <= 1e-14 ||T||; the largest eigenvalue of the
  tridiagonal T comes from LAPACK.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import rng


def cheb4(Aop, Mop, b: np.ndarray, x0: np.ndarray | None, beta: float, k: int) -> np.ndarray:
    """Algorithm 3: k steps of the M-preconditioned fourth-kind Chebyshev iteration."""
    x0 = np.zeros_like(b) if x0 is None else x0
    r = b - Aop(x0)
    p = Mop(r)
    mu = 1.0 / 3.0
    d = 4.0 / beta
    x = x0 + d * mu * p
    for _i in range(2, k + 1):
        r = b - Aop(x)
        p = mu * mu * p + Mop(r)
        mu = 1.0 / (2.0 - mu)
        x = x + d * mu * p
    return x


def richardson(Aop, Mop, b: np.ndarray, x0: np.ndarray | None, k: int) -> np.ndarray:
    """Richardson smoothing (Section 3.1): k repeated applications of the preconditioner."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    for _i in range(k):
        x = x + Mop(b - Aop(x))
    return x


def w4(k: int, t):
    """W_k(t) by the three-term recurrence of the fourth-kind polynomials."""
    t = np.asarray(t, dtype=np.float64)
    w_prev, w = np.ones_like(t), 2.0 * t + 1.0
    if k == 0:
        return w_prev
    for _n in range(1, k):
        w_prev, w = w, 2.0 * t * w - w_prev
    return w


def cheb4_residual_polynomial(k: int, lam, beta: float):
    """p_k(lambda) = W_k(1 - 2 lambda / beta) / (2k + 1) (Eq. (3.6))."""
    return w4(k, 1.0 - 2.0 * np.asarray(lam) / beta) / (2 * k + 1)


LANCZOS_ITS = 100
LANCZOS_SAFETY = 1.01


def lanczos_tridiagonal(op, n: int, its: int, seed: int):
    """Diagonal alpha and off-diagonal beta of the Lanczos tridiagonal matrix of op."""
    v = rng.uniform_pm1(seed, n)
    v = v / np.linalg.norm(v)
    v_prev = np.zeros(n)
    alphas, betas = [], []
    b_prev = 0.0
    for _j in range(min(its, n)):
        w = op(v) - b_prev * v_prev
        a = float(w @ v)
        w = w - a * v
        alphas.append(a)
        bnext = float(np.linalg.norm(w))
        tnorm = max(abs(x) for x in alphas) + (max(betas) if betas else 0.0) + bnext
        if bnext <= 1e-14 * tnorm or len(alphas) == min(its, n):
            break
        betas.append(bnext)
        v_prev, v = v, w / bnext
        b_prev = bnext
    return np.array(alphas), np.array(betas)


def lanczos_lmax(op, n: int, its: int = LANCZOS_ITS, seed: int = 0) -> float:
    """Largest eigenvalue of the Lanczos tridiagonal matrix of op."""
    al, be = lanczos_tridiagonal(op, n, its, seed)
    if len(al) == 1:
        return float(al[0])
    ev = sla.eigvalsh_tridiagonal(al, be)
    return float(ev[-1])
