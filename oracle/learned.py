"""Learned candidate scoring for the adaptive block-FSAI pattern (test infrastructure only).

The paper's Algorithm 1 (Section 2.1) grows each block row's pattern one admissible candidate
at a time, choosing the candidate with the smallest rho_c of Lemma 2.8.  The learned form is
an addition of this project, not a method of the paper: a small network scores the
candidates of every block row at once from features of A and of the static FSAI on P0, the
t_max best-scoring candidates join the pattern, and Algorithm 1 stays the fallback and the
judge (a level keeps the learned pattern only when it reaches at least 95% of Algorithm 1's
gain in the Kaporin-type measure sum_k log det S_kk of Lemma 2.7 on a sample of rows).
This module is imported by the tests and never by the CUDA library; it shares no code with it.

* ``candidate_pool``: for block row k with initial pattern P0_k, ring 1 is Algorithm 1's
  admissible set of P0 (c < k in the A-rows of P0_k, not in P0_k); ring 2 adds the c < k in
  the A-rows of ring 1 that are in neither (the columns Algorithm 1 can reach in later steps).
* ``features``: 12 numbers per (row, candidate), all from A and the static FSAI G0 = J F on P0:
    0  ring (1 for ring 1, 0 for ring 2)
    1  log10(1e-30 + a_kc),  a_ij = |A_ij|_F / sqrt(|A_ii|_F |A_jj|_F) (0 when not stored)
    2  log10(1e-30 + g_c), g_c = |L_c^-1 (G0 A)_kc^T|_F^2 with A_cc = L_c L_c^T: the first-order
       gain of adding c (Lemma 2.8: rho_c = 1 - g_c + O(|H|^4) when W_c ~ A_cc)
    3  log10(1e-30 + max over ring-1 c' != c with A_c'c stored of g_c' a_c'c^2)
    4  number of ring-1 gains above g_c (1 + 1e-9) / 10 (ring 2: 1)
    5  g_c / max_ring1 g (0 when that maximum is 0)
    6  |{j in P0_k with A_jc stored}| / |P0_k|
    7  |P0_k| / 16
    8  (c_x - k_x) / 4 and  9  (c_y - k_y) / 4 on the level's m x m patch grid (0 when m = 0)
    10 nnzb(A row k) / max_i nnzb(A row i)
    11 |ring 1 of row k| / 32
  The label of a candidate is 1 when Algorithm 1's final pattern of row k contains it.
* ``MLP``: 12 -> 64 -> 64 -> 1 with ReLU, weights used in BF16 (round to nearest even of the
  FP32 master weights), biases in FP32; the loss is the mean binary cross-entropy of the logit.
  Forward and backward here are in FP64 on the BF16-rounded weights (the gradient of the
  rounded weight is taken as the gradient of the master weight).
* ``adam``: Kingma and Ba (2015), bias-corrected.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import blocks as bk

N_FEATURES = 12
HIDDEN = 64


# --------------------------------------------------------------------------- candidates, features

def candidate_pool(A: bk.BlockCSR, k: int, P0k: list[int]) -> tuple[list[int], list[int]]:
    """(ring 1, ring 2) of block row k, each ascending."""
    pat = A.pattern()
    inP = set(P0k)
    ring1 = sorted({c for j in P0k for c in pat[j] if c < k and c not in inP})
    r1 = set(ring1)
    ring2 = sorted({c for j in ring1 for c in pat[j] if c < k and c not in inP and c not in r1})
    return ring1, ring2


def _fro(X) -> float:
    return float(np.sqrt(np.sum(X * X)))


def features(A: bk.BlockCSR, G0: bk.BlockCSR, P0: list[list[int]], m: int = 0):
    """Rows, columns and the (n_cand, 12) feature matrix of every block row's candidate pool
    (rows ascending, ring 1 then ring 2, each ascending)."""
    n, d = A.n_rows, A.d
    pat = A.pattern()
    nrm = np.array([_fro(A.block(i, i)) for i in range(n)])
    Lc = [np.linalg.cholesky(A.block(i, i)) for i in range(n)]
    max_row = max(len(r) for r in pat)

    def a(i, j):
        b = A.block(i, j)
        return 0.0 if b is None else _fro(b) / np.sqrt(nrm[i] * nrm[j])

    rows, cols, feats = [], [], []
    for k in range(n):
        ring1, ring2 = candidate_pool(A, k, P0[k])
        # (G0 A)_kc for the row's candidates
        g = {}
        for c in ring1 + ring2:
            GA = np.zeros((d, d))
            for j in P0[k]:
                Ajc = A.block(j, c)
                if Ajc is not None:
                    GA += G0.block(k, j) @ Ajc
            Y = np.linalg.solve(Lc[c], GA.T)   # L_c^-1 (G0 A)_kc^T
            g[c] = float(np.sum(Y * Y))
        g1 = [g[c] for c in ring1]
        gmax = max(g1) if g1 else 0.0
        # rank: how many ring-1 gains exceed g_c beyond the tie band (equal gains share a rank)
        rank = {c: sum(1 for c2 in ring1 if g[c2] > g[c] * (1.0 + 1e-9)) for c in ring1}
        kx, ky = (k % m, k // m) if m else (0, 0)
        for ring, cand in ((1, ring1), (0, ring2)):
            for c in cand:
                via = [g[cp] * a(cp, c) ** 2 for cp in ring1 if cp != c and A.block(cp, c) is not None]
                cx, cy = (c % m, c // m) if m else (0, 0)
                f = [float(ring), np.log10(1e-30 + a(k, c)), np.log10(1e-30 + g[c]),
                     np.log10(1e-30 + (max(via) if via else 0.0)),
                     rank[c] / 10.0 if ring == 1 else 1.0,
                     g[c] / gmax if gmax > 0 else 0.0,
                     sum(1 for j in P0[k] if A.block(j, c) is not None) / len(P0[k]),
                     len(P0[k]) / 16.0, (cx - kx) / 4.0, (cy - ky) / 4.0,
                     len(pat[k]) / max_row, len(ring1) / 32.0]
                rows.append(k)
                cols.append(c)
                feats.append(f)
    return np.array(rows, dtype=np.int64), np.array(cols, dtype=np.int64), np.array(feats).reshape(-1, N_FEATURES)


def labels(rows, cols, final_pattern: list[list[int]]) -> np.ndarray:
    """1 for candidates in the row's final Algorithm 1 pattern."""
    sets = [set(p) for p in final_pattern]
    return np.array([1.0 if c in sets[k] else 0.0 for k, c in zip(rows, cols)])


def select(rows, cols, scores, P0: list[list[int]], t_max: int) -> list[list[int]]:
    """Each row's pattern: P0_k plus its t_max best-scoring candidates (ties: smaller column)."""
    out = [list(p) for p in P0]
    by_row = {}
    for k, c, s in zip(rows, cols, scores):
        by_row.setdefault(int(k), []).append((-float(s), int(c)))
    for k, lst in by_row.items():
        lst.sort()
        out[k] = sorted(out[k] + [c for _, c in lst[:t_max]])
    return out


def gate_ratio(ld_learned: np.ndarray, ld_alg1: np.ndarray, ld_p0: np.ndarray) -> float:
    """Shortfall of the learned pattern's Kaporin-measure gain, relative to Algorithm 1's gain
    over P0, on the same rows: sum(ld_learned - ld_alg1) / sum(ld_p0 - ld_alg1) (Lemma 2.7's
    measure is sum_k log det S_kk up to a constant; 0 means Algorithm 1's gain, 1 no gain)."""
    den = float(np.sum(ld_p0 - ld_alg1))
    return float(np.sum(ld_learned - ld_alg1)) / den if den > 0 else 0.0


# --------------------------------------------------------------------------- the network

def bf16(x: np.ndarray) -> np.ndarray:
    """Round FP32 values to BF16 (round to nearest, ties to even), returned as float64."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


@dataclasses.dataclass
class MLP:
    """Master weights (FP32): W1 (64, 12), b1 (64), W2 (64, 64), b2 (64), w3 (64), b3 ()."""
    W1: np.ndarray
    b1: np.ndarray
    W2: np.ndarray
    b2: np.ndarray
    w3: np.ndarray
    b3: np.ndarray

    def params(self):
        return [self.W1, self.b1, self.W2, self.b2, self.w3, self.b3]


def init_mlp(seed: int) -> MLP:
    """He-normal weights, zero biases (FP32)."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x1EA]))
    f32 = np.float32
    return MLP((rng.standard_normal((HIDDEN, N_FEATURES)) * np.sqrt(2.0 / N_FEATURES)).astype(f32),
               np.zeros(HIDDEN, f32), (rng.standard_normal((HIDDEN, HIDDEN)) * np.sqrt(2.0 / HIDDEN)).astype(f32),
               np.zeros(HIDDEN, f32), (rng.standard_normal(HIDDEN) * np.sqrt(1.0 / HIDDEN)).astype(f32),
               np.zeros((), f32))


def _weights(m: MLP, quant: bool):
    q = bf16 if quant else (lambda w: np.asarray(w, dtype=np.float64))
    return q(m.W1), q(m.W2), q(m.w3)


def forward(m: MLP, X: np.ndarray, quant: bool = True):
    """Logits of the rows of X and the activations the backward pass needs (FP64 arithmetic on
    BF16 weights -- the FP32 master weights when quant is False -- and FP32 biases)."""
    W1, W2, w3 = _weights(m, quant)
    z1 = X @ W1.T + m.b1.astype(np.float64)
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + m.b2.astype(np.float64)
    h2 = np.maximum(z2, 0.0)
    logit = h2 @ w3 + float(m.b3)
    return logit, (X, z1, h1, z2, h2)


def loss_and_grad(m: MLP, X: np.ndarray, y: np.ndarray, quant: bool = True):
    """Mean binary cross-entropy of the logits and its gradient for every parameter."""
    logit, (X, z1, h1, z2, h2) = forward(m, X, quant)
    n = X.shape[0]
    # log(1 + e^x) - y x, evaluated stably
    loss = float(np.mean(np.maximum(logit, 0.0) + np.log1p(np.exp(-np.abs(logit))) - y * logit))
    s = 1.0 / (1.0 + np.exp(-logit))
    dlogit = (s - y) / n
    _, W2, w3 = _weights(m, quant)
    g_w3 = h2.T @ dlogit
    g_b3 = np.sum(dlogit)
    dz2 = np.outer(dlogit, w3) * (z2 > 0.0)
    g_W2 = dz2.T @ h1
    g_b2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (z1 > 0.0)
    g_W1 = dz1.T @ X
    g_b1 = dz1.sum(axis=0)
    return loss, [g_W1, g_b1, g_W2, g_b2, g_w3, np.asarray(g_b3)]


def adam(params, grads, state, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam step (Kingma and Ba 2015) in place; state: per-parameter (m, v) pairs, t >= 1."""
    for p, g, (mm, vv) in zip(params, grads, state):
        mm *= beta1
        mm += (1.0 - beta1) * g
        vv *= beta2
        vv += (1.0 - beta2) * g * g
        mhat = mm / (1.0 - beta1 ** t)
        vhat = vv / (1.0 - beta2 ** t)
        p -= (lr * mhat / (np.sqrt(vhat) + eps)).astype(p.dtype)
