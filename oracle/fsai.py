"""Block-FSAI oracle: Definition 2.2, Lemma 2.7, Algorithm 1 and Section 2.2.

Test infrastructure only (never imported by the CUDA library).

* ``fsai(A, pattern)``: for every block row k with P~_k = P_k \\ {k},
  F_kk = I, F[k, P~_k] = -A[k, P~_k] A[P~_k, P~_k]^{-1}      (Def. 2.2, eq. for F)
  S_kk = A_kk - A[k, P~_k] A[P~_k, P~_k]^{-1} A[P~_k, k]     (Def. 2.2, Schur complement)
  G = S^{-1/2} F with S^{-1/2} read as L_S^{-1}, S_kk = L_S L_S^T (Cholesky); it gives the
  same M = G^T G = F^T S^{-1} F and diag_B(G A G^T) = I.
* ``adaptive_fsai``: Algorithm 1 in the paper's order.  The admissible set is read
  structurally: c < k with c in the union of the A-patterns of the rows in P_k and
  c not in P_k; ties in the argmin of rho_c are broken by taking the smallest column
  among those within a relative band tie_rel of the minimum, and the stop test
  rho_c* < tau takes the same band (rho_c* < tau (1 - tie_rel)).
* ``nested_fsai``: Section 2.2 with one level of nesting:
  A_1 = F_0 A F_0^T, F_1 the (adaptive) FSAI of A_1 with the same parameters,
  S^ = diag_B(F_1 A_1 F_1^T), M = F^^T S^^{-1} F^ with F^ = F_1 F_0.
  The FSAI of A_1 needs A_1 to be SPD, which the paper takes for granted.  In FP64
  the computed A_1 can lose definiteness (a diagonal block whose Schur-complement
  value is far below the rounding of the triple product).  When any local matrix of
  the inner FSAI (A_1[P~_k, P~_k] or S_kk) fails its Cholesky factorisation, the
  inner level falls back to block Jacobi (the diagonal pattern, Remark 2.4), whose
  blocks diag_B(A_1) = S of the outer FSAI by Lemma 2.3; M is then the plain
  (non-nested) block-FSAI G^T G.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla

from . import blocks as bk


def lower_pattern(A: bk.BlockCSR) -> list[list[int]]:
    """Lower block-triangular part of P(A), diagonal included."""
    return [[c for c in A.pattern()[i] if c <= i] for i in range(A.n_rows)]


def diag_pattern(n: int) -> list[list[int]]:
    return [[i] for i in range(n)]


def dense(A: bk.BlockCSR, rows, cols) -> np.ndarray:
    """A[rows, cols] as a dense matrix (missing blocks are zero)."""
    d = A.d
    out = np.zeros((len(rows) * d, len(cols) * d))
    for a, i in enumerate(rows):
        for b, j in enumerate(cols):
            blk = A.block(i, j)
            if blk is not None:
                out[a * d:(a + 1) * d, b * d:(b + 1) * d] = blk
    return out


@dataclasses.dataclass
class FSAI:
    pattern: list        # P_k (sorted) per block row
    F: bk.BlockCSR
    S: np.ndarray        # (n, d, d) diagonal blocks S_kk
    G: bk.BlockCSR       # L_S^{-1} F

    def logdet_S(self) -> float:
        """sum_k log det S_kk: the pattern-dependent part of the Kaporin measure (Lemma 2.7)."""
        return float(sum(np.linalg.slogdet(s)[1] for s in self.S))


class NotSPD(np.linalg.LinAlgError):
    """A local matrix of Definition 2.2 (A[P~_k, P~_k] or S_kk) is not numerically SPD in FP64."""

    def __init__(self, k: int, what: str):
        super().__init__(f"{what} of block row {k} is not numerically SPD")
        self.row = k


def _require_spd(X: np.ndarray, k: int, what: str) -> None:
    """Definition 2.2 assumes SPD local matrices; in FP64 that is decided by their Cholesky."""
    if not _is_spd(X):
        raise NotSPD(k, what)


def fsai_row(A: bk.BlockCSR, k: int, Pk: list[int]):
    """F row k (dict col -> block), S_kk, per Definition 2.2.

    Raises NotSPD when A[P~_k, P~_k] or S_kk fails its Cholesky factorisation."""
    d = A.d
    Pt = [j for j in Pk if j != k]
    row = {k: np.eye(d)}
    Akk = A.block(k, k)
    if not Pt:
        _require_spd(Akk, k, "S_kk")
        return row, Akk.copy()
    App = dense(A, Pt, Pt)
    _require_spd(App, k, "A[P~_k, P~_k]")
    Akp = dense(A, [k], Pt)
    Apk = dense(A, Pt, [k])
    Fk = -np.linalg.solve(App.T, Akp.T).T          # -A[k,P~] A[P~,P~]^{-1}
    S = Akk - Akp @ np.linalg.solve(App, Apk)
    _require_spd(S, k, "S_kk")
    for b, j in enumerate(Pt):
        row[j] = Fk[:, b * d:(b + 1) * d]
    return row, S


def fsai(A: bk.BlockCSR, pattern: list[list[int]]) -> FSAI:
    """Block-FSAI matrices F, S and G = L_S^{-1} F for a lower pattern (Definition 2.2)."""
    n, d = A.n_rows, A.d
    Fent, Gent = {}, {}
    S = np.zeros((n, d, d))
    for k in range(n):
        assert k in pattern[k] and all(j <= k for j in pattern[k]), "pattern must be lower with diagonal"
        row, S[k] = fsai_row(A, k, pattern[k])
        L = np.linalg.cholesky(S[k])
        J = sla.solve_triangular(L, np.eye(d), lower=True)
        for j, blk in row.items():
            Fent[(k, j)] = blk
            Gent[(k, j)] = J @ blk
    pat = [sorted(p) for p in pattern]
    return FSAI(pat, bk.from_blocks(n, n, d, Fent), S, bk.from_blocks(n, n, d, Gent))


def admissible(A_pattern: list[list[int]], Pk: list[int], k: int) -> list[int]:
    """Structural admissible set of Algorithm 1: {c < k : H_kc not identically 0} minus P_k.

    H = F A has row k supported on the union of the A-pattern rows j in P_k.
    """
    s = set()
    for j in Pk:
        s.update(A_pattern[j])
    return sorted(c for c in s if c < k and c not in Pk)


def rho(A: bk.BlockCSR, k: int, Pk: list[int], c: int) -> float:
    """rho_c = det(W_c - H_kc^T H_kk^{-1} H_kc) / det(W_c) of Lemma 2.8 / Algorithm 1."""
    return row_rhos(A, k, Pk, [c])[c]


def row_rhos(A: bk.BlockCSR, k: int, Pk: list[int], C: list[int]) -> dict:
    """rho_c for every c in C, reusing A[P~_k, P~_k]^{-1} as Algorithm 1 suggests."""
    d = A.d
    Pt = [j for j in Pk if j != k]
    row, _ = fsai_row(A, k, Pk)
    Hkk = sum(blk @ _blk(A, j, k) for j, blk in row.items())
    Ainv = np.linalg.inv(dense(A, Pt, Pt)) if Pt else None
    out = {}
    for c in C:
        # H = F A restricted to row k, column c
        Hkc = sum(blk @ _blk(A, j, c) for j, blk in row.items())
        if Pt:
            W = A.block(c, c) - dense(A, [c], Pt) @ Ainv @ dense(A, Pt, [c])
        else:
            W = A.block(c, c).copy()
        X = W - Hkc.T @ np.linalg.solve(Hkk, Hkc)
        sx, lx = np.linalg.slogdet(X)
        sw, lw = np.linalg.slogdet(W)
        if sx <= 0 or sw <= 0 or not _is_spd(X) or not _is_spd(W):
            continue  # rho_c not computable in FP64: the candidate is not admissible
        out[c] = float(np.exp(lx - lw))
    return out


def _is_spd(X) -> bool:
    """X is numerically symmetric positive definite (its Cholesky factorisation exists)."""
    try:
        np.linalg.cholesky(X)
        return True
    except np.linalg.LinAlgError:
        return False


def _blk(A, i, j):
    b = A.block(i, j)
    return b if b is not None else np.zeros((A.d, A.d))


def choose(rhos: dict, tie_rel: float) -> int:
    """argmin over c of rho_c; among values within (1 + tie_rel) of the minimum take the smallest c."""
    rmin = min(rhos.values())
    return min(c for c, r in rhos.items() if r <= rmin * (1.0 + tie_rel))


def accepts(rho_star: float, tau: float, tie_rel: float) -> bool:
    """Algorithm 1's test rho_c* < tau, with the tie band: a gain below tie_rel relative to tau
    is rounding (with tau = 1, a candidate whose coupling H_kc vanishes to rounding has
    rho_c = 1 up to rounding), so it is not a gain."""
    return rho_star < tau * (1.0 - tie_rel)


@dataclasses.dataclass
class AdaptiveResult:
    fsai: FSAI
    logdet_history: list   # sum_k log det S_kk before each step and at the end


def adaptive_fsai(A: bk.BlockCSR, P0: list[list[int]], t_max: int, tau: float = 1.0,
                  tie_rel: float = 1e-9) -> AdaptiveResult:
    """Algorithm 1 (adaptive block-FSAI)."""
    n = A.n_rows
    Apat = A.pattern()
    P = [sorted(p) for p in P0]
    R = set(range(n))
    hist = []
    for _t in range(t_max):
        hist.append(fsai(A, P).logdet_S())
        for k in sorted(R):
            C = admissible(Apat, P[k], k)
            if not C:
                R.discard(k)
                continue
            rhos = row_rhos(A, k, P[k], C)
            if not rhos:
                R.discard(k)
                continue
            cstar = choose(rhos, tie_rel)
            if accepts(rhos[cstar], tau, tie_rel):
                P[k] = sorted(P[k] + [cstar])
            else:
                R.discard(k)
    final = fsai(A, P)
    hist.append(final.logdet_S())
    return AdaptiveResult(final, hist)


def adaptive_row(A: bk.BlockCSR, k: int, P0k: list[int], t_max: int, tau: float = 1.0,
                 tie_rel: float = 1e-9) -> list[int]:
    """Algorithm 1 for block row k alone.

    The steps of Algorithm 1 only ever change row k's pattern from row k's own scores, so a
    row's final pattern depends on A near that row only; A needs the rows of P_k, of the
    admissible columns and of their A-neighbours (a window around k).
    """
    Apat = A.pattern()
    Pk = sorted(P0k)
    for _t in range(t_max):
        C = admissible(Apat, Pk, k)
        if not C:
            break
        rhos = row_rhos(A, k, Pk, C)
        if not rhos:
            break
        cstar = choose(rhos, tie_rel)
        if accepts(rhos[cstar], tau, tie_rel):
            Pk = sorted(Pk + [cstar])
        else:
            break
    return Pk


def g_row(A: bk.BlockCSR, k: int, Pk: list[int]) -> dict:
    """Row k of G = L_S^{-1} F for the pattern row P_k (Definition 2.2)."""
    row, S = fsai_row(A, k, Pk)
    J = sla.solve_triangular(np.linalg.cholesky(S), np.eye(A.d), lower=True)
    return {j: J @ blk for j, blk in row.items()}


@dataclasses.dataclass
class NestedFSAI:
    F0: bk.BlockCSR
    A1: bk.BlockCSR
    inner: FSAI            # FSAI of A1: its G is G_1 = S^^{-1/2} F_1
    outer_pattern: list
    inner_nested: bool = True   # False: A1 was not numerically SPD and the inner level is block Jacobi

    def logdet_S(self) -> float:
        """sum_k log det S_kk of the inner FSAI (the outer S under the block-Jacobi fallback)."""
        return self.inner.logdet_S()

    def apply(self, r: np.ndarray) -> np.ndarray:
        """z = F0^T G1^T G1 F0 r."""
        t = self.F0.matvec(r)
        u = self.inner.G.matvec(t)
        w = self.inner.G.to_scipy().T @ u
        return self.F0.to_scipy().T @ w


def nested_fsai(A: bk.BlockCSR, P0: list[list[int]], t_max: int, tau: float = 1.0,
                tie_rel: float = 1e-9, adaptive: bool = True) -> NestedFSAI:
    """One level of nesting (Section 2.2) with the same parameters on both levels."""
    outer = adaptive_fsai(A, P0, t_max, tau, tie_rel).fsai if adaptive else fsai(A, P0)
    F0 = outer.F
    A1 = bk.galerkin_product(F0, A, F0.transpose())
    try:
        inner = adaptive_fsai(A1, P0, t_max, tau, tie_rel).fsai if adaptive else fsai(A1, P0)
    except NotSPD:
        return NestedFSAI(F0, A1, block_jacobi_from_schur(outer), outer.pattern, inner_nested=False)
    return NestedFSAI(F0, A1, inner, outer.pattern)


def block_jacobi_from_schur(outer: FSAI) -> FSAI:
    """Inner block Jacobi of A_1 = F_0 A F_0^T (Remark 2.4: F = I, S = diag_B(A_1)), with
    diag_B(A_1) taken as the outer Schur complements S (equal by Lemma 2.3) and its G blocks
    L_S^{-1}; then F_0^T G_1^T G_1 F_0 = G^T G of the outer FSAI."""
    n, d = outer.S.shape[0], outer.S.shape[1]
    ent = {(k, k): sla.solve_triangular(np.linalg.cholesky(outer.S[k]), np.eye(d), lower=True)
           for k in range(n)}
    eye = {(k, k): np.eye(d) for k in range(n)}
    return FSAI(diag_pattern(n), bk.from_blocks(n, n, d, eye), outer.S.copy(), bk.from_blocks(n, n, d, ent))


def apply_M(G: bk.BlockCSR, r: np.ndarray) -> np.ndarray:
    """z = M r = G^T (G r)."""
    return G.to_scipy().T @ (G.matvec(r))


def kaporin_number(B: np.ndarray) -> float:
    """beta(B) = tr(B) / (N det(B)^{1/N}) (Definition 2.4), via log-determinants."""
    N = B.shape[0]
    return float(np.trace(B) / (N * np.exp(np.linalg.slogdet(B)[1] / N)))
