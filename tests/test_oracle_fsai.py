"""Pins of the block-FSAI oracle (Definition 2.2, Lemmas 2.3/2.7/2.8, Theorem 2.6, Algorithm 1, Section 2.2)."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.optimize as so

import pum_inputs as pin
from oracle import blocks as bk
from oracle import fsai


def _block_csr_from_dense(A, d):
    n = A.shape[0] // d
    ent = {}
    for i in range(n):
        for j in range(n):
            blk = A[i * d:(i + 1) * d, j * d:(j + 1) * d]
            if np.any(blk != 0.0):
                ent[(i, j)] = blk
    return bk.from_blocks(n, n, d, ent)


@pytest.fixture(scope="module")
def tiny():
    A = pin.spd_block_matrix(6, 3, seed=4, density=0.6)
    return A, _block_csr_from_dense(A, 3)


def _random_lower_pattern(n, seed, density=0.5):
    rng = np.random.default_rng(seed)
    return [sorted({i} | {j for j in range(i) if rng.random() < density}) for i in range(n)]


def test_preconditioned_diagonal_blocks_are_identity(tiny):
    """Lemma 2.3: diag_B(F A) = S = diag_B(F A F^T) and diag_B(G A G^T) = I."""
    A, Ab = tiny
    for seed in range(3):
        pat = _random_lower_pattern(Ab.n_rows, seed)
        f = fsai.fsai(Ab, pat)
        F, G = f.F.to_dense(), f.G.to_dense()
        d = Ab.d
        FA, FAF, GAG = F @ A, F @ A @ F.T, G @ A @ G.T
        for k in range(Ab.n_rows):
            sl = slice(k * d, (k + 1) * d)
            assert np.allclose(FA[sl, sl], f.S[k], rtol=0, atol=1e-12 * np.abs(A).max())
            assert np.allclose(FAF[sl, sl], f.S[k], rtol=0, atol=1e-12 * np.abs(A).max())
            assert np.max(np.abs(GAG[sl, sl] - np.eye(d))) <= 1e-12
        # eq. (2.5): (F A)[k, P~_k] = 0
        for k in range(Ab.n_rows):
            for j in pat[k]:
                if j != k:
                    assert np.max(np.abs(FA[k * d:(k + 1) * d, j * d:(j + 1) * d])) <= 1e-11 * np.abs(A).max()


def test_diagonal_pattern_is_block_jacobi(tiny):
    """Remark 2.4: the diagonal pattern gives F = I, S = diag_B(A)."""
    A, Ab = tiny
    f = fsai.fsai(Ab, fsai.diag_pattern(Ab.n_rows))
    assert np.array_equal(f.F.to_dense(), np.eye(A.shape[0]))
    for k in range(Ab.n_rows):
        L = np.linalg.cholesky(Ab.block(k, k))
        assert np.allclose(f.G.block(k, k), np.linalg.inv(L), atol=1e-13)


def test_full_lower_pattern_is_exact_inverse_factor(tiny):
    """With the full lower pattern G is the inverse block-Cholesky factor: G A G^T = I."""
    A, Ab = tiny
    n = Ab.n_rows
    full = _block_csr_from_dense(A + 0.0 * np.ones_like(A), Ab.d)
    pat = [list(range(i + 1)) for i in range(n)]
    # make every block structurally present
    ent = {(i, j): A[i * 3:(i + 1) * 3, j * 3:(j + 1) * 3] for i in range(n) for j in range(n)}
    full = bk.from_blocks(n, n, 3, ent)
    G = fsai.fsai(full, pat).G.to_dense()
    assert np.max(np.abs(G @ A @ G.T - np.eye(A.shape[0]))) <= 1e-11


def test_kaporin_closed_form(tiny):
    """Lemma 2.7: beta(G A G^T) = (prod det S_kk / det A)^(1/N)."""
    A, Ab = tiny
    N = A.shape[0]
    for seed in range(3):
        f = fsai.fsai(Ab, _random_lower_pattern(Ab.n_rows, seed))
        G = f.G.to_dense()
        direct = fsai.kaporin_number(G @ A @ G.T)
        closed = np.exp((f.logdet_S() - np.linalg.slogdet(A)[1]) / N)
        assert abs(direct - closed) <= 1e-12 * closed


def _beta_of(theta, pat, A, d):
    n = A.shape[0] // d
    G = np.zeros_like(A)
    pos = 0
    for k in range(n):
        for j in pat[k]:
            G[k * d:(k + 1) * d, j * d:(j + 1) * d] = theta[pos:pos + d * d].reshape(d, d)
            pos += d * d
    return fsai.kaporin_number(G @ A @ G.T)


def test_fsai_minimises_kaporin_number_brute_force():
    """Theorem 2.6: no full-rank G~ with the pattern has a smaller Kaporin number (n=3, d=2)."""
    d, n = 2, 3
    A = pin.spd_block_matrix(n, d, seed=9, density=1.0)
    Ab = _block_csr_from_dense(A, d)
    pat = [[0], [0, 1], [1, 2]]
    f = fsai.fsai(Ab, pat)
    G = f.G.to_dense()
    best = fsai.kaporin_number(G @ A @ G.T)
    theta0 = np.concatenate([G[k * d:(k + 1) * d, j * d:(j + 1) * d].ravel() for k in range(n) for j in pat[k]])
    rng = np.random.default_rng(0)
    found = []
    for restart in range(8):
        start = theta0 + rng.standard_normal(theta0.shape) * (0.5 if restart else 0.0)
        res = so.minimize(_beta_of, start, args=(pat, A, d), method="Nelder-Mead",
                          options={"maxiter": 40000, "maxfev": 40000, "xatol": 1e-12, "fatol": 1e-15})
        found.append(res.fun)
        assert res.fun >= best - 1e-12
    assert min(found) <= best + 1e-8
    # random perturbations within the pattern never improve on G
    for _ in range(200):
        th = theta0 + 1e-3 * rng.standard_normal(theta0.shape)
        assert _beta_of(th, pat, A, d) >= best - 1e-14


def test_candidate_gain_formula_matches_rebuilt_fsai(tiny):
    """Lemma 2.8: rho_c = det((F^(c) A F^(c)T)_kk) / det((F A F^T)_kk), F^(c) rebuilt from scratch."""
    A, Ab = tiny
    pat = _random_lower_pattern(Ab.n_rows, 3, density=0.3)
    Apat = [list(range(Ab.n_rows))] * Ab.n_rows
    checked = 0
    for k in range(Ab.n_rows):
        for c in range(k):
            if c in pat[k]:
                continue
            r = fsai.rho(Ab, k, pat[k], c)
            _, S_old = fsai.fsai_row(Ab, k, pat[k])
            _, S_new = fsai.fsai_row(Ab, k, sorted(pat[k] + [c]))
            ratio = np.exp(np.linalg.slogdet(S_new)[1] - np.linalg.slogdet(S_old)[1])
            assert abs(r - ratio) <= 1e-12 * max(ratio, 1e-300) + 1e-14
            assert 0.0 < r <= 1.0 + 1e-12
            checked += 1
    assert checked > 5
    del Apat


def _brute_force_step(Ab, P, k, C):
    """Admissible column with the smallest det of the rebuilt S_kk (ties: smallest column)."""
    vals = {}
    for c in C:
        _, S = fsai.fsai_row(Ab, k, sorted(P[k] + [c]))
        vals[c] = np.linalg.slogdet(S)[1]
    vmin = min(vals.values())
    return min(c for c, v in vals.items() if v <= vmin + 1e-9)


def test_adaptive_greedy_choice_equals_brute_force():
    """Algorithm 1: each added block is the admissible column that minimises det S_kk."""
    A = pin.spd_block_matrix(8, 2, seed=21, density=0.5)
    Ab = _block_csr_from_dense(A, 2)
    Apat = Ab.pattern()
    P = fsai.diag_pattern(Ab.n_rows)
    for _step in range(3):
        newP = [list(p) for p in P]
        for k in range(Ab.n_rows):
            C = fsai.admissible(Apat, P[k], k)
            if not C:
                continue
            rhos = fsai.row_rhos(Ab, k, P[k], C)
            c = fsai.choose(rhos, 1e-9)
            assert c == _brute_force_step(Ab, P, k, C)
            newP[k] = sorted(P[k] + [c])
        P = newP
    res = fsai.adaptive_fsai(Ab, fsai.diag_pattern(Ab.n_rows), 3)
    assert res.fsai.pattern == P


def test_adaptive_logdet_nonincreasing_and_patterns_lower(small_biharmonic):
    """Algorithm 1 on a PUM matrix: sum log det S_kk never increases; rows grow by <= 1 block per step."""
    A = small_biharmonic.A[2]
    P0 = fsai.lower_pattern(A)
    res = fsai.adaptive_fsai(A, P0, 3)
    h = res.logdet_history
    assert all(h[i + 1] <= h[i] + 1e-9 * abs(h[i]) for i in range(len(h) - 1))
    for k, row in enumerate(res.fsai.pattern):
        assert k in row and all(j <= k for j in row)
        assert set(P0[k]) <= set(row) and len(row) <= len(P0[k]) + 3


def test_admissible_set_excludes_current_pattern(tiny):
    """Eq. (2.5): H_kc = 0 on P~_k, so the admissible set never contains P_k."""
    _, Ab = tiny
    Apat = Ab.pattern()
    for k in range(Ab.n_rows):
        Pk = [j for j in Apat[k] if j <= k]
        C = fsai.admissible(Apat, Pk, k)
        assert not set(C) & set(Pk) and all(c < k for c in C)


def test_nested_fsai_identities(small_biharmonic):
    """Section 2.2: S^ = diag_B(F^ A F^^T), diag_B(G^ A G^^T) = I with G^ = G_1 F_0."""
    A = small_biharmonic.A[2]
    nf = fsai.nested_fsai(A, fsai.lower_pattern(A), 2)
    Ad = A.to_dense()
    F0 = nf.F0.to_dense()
    F1 = nf.inner.F.to_dense()
    Fh = F1 @ F0
    T = Fh @ Ad @ Fh.T
    d = A.d
    Gh = nf.inner.G.to_dense() @ F0
    GAG = Gh @ Ad @ Gh.T
    for k in range(A.n_rows):
        sl = slice(k * d, (k + 1) * d)
        assert np.allclose(T[sl, sl], nf.inner.S[k], rtol=0, atol=1e-11 * np.abs(T).max())
        assert np.max(np.abs(GAG[sl, sl] - np.eye(d))) <= 1e-10
    r = np.random.default_rng(0).standard_normal(Ad.shape[0])
    ref = Gh.T @ (Gh @ r)
    assert np.max(np.abs(nf.apply(r) - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_nested_with_diagonal_inner_pattern_equals_plain(small_biharmonic):
    """Section 2.2: a block-Jacobi inner level reproduces the non-nested preconditioner."""
    A = small_biharmonic.A[2]
    P0 = fsai.lower_pattern(A)
    outer = fsai.fsai(A, P0)
    F0 = outer.F
    A1 = bk.galerkin_product(F0, A, F0.transpose())
    inner = fsai.fsai(A1, fsai.diag_pattern(A.n_rows))
    r = np.random.default_rng(1).standard_normal(A.n_rows * A.d)
    Gh = inner.G.to_dense() @ F0.to_dense()
    nested = Gh.T @ (Gh @ r)
    plain = fsai.apply_M(outer.G, r)
    assert np.max(np.abs(nested - plain)) <= 1e-11 * np.max(np.abs(plain))
