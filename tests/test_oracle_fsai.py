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


def _rows_only(A: bk.BlockCSR, rows) -> bk.BlockCSR:
    """A with only the given block rows stored (the others empty): a window of A."""
    keep = set(rows)
    ent = {(i, int(j)): A.blocks[p] for i in keep for p, j in
           zip(range(A.indptr[i], A.indptr[i + 1]), A.row(i))}
    return bk.from_blocks(A.n_rows, A.n_cols, A.d, ent)


def _grid_window(k, m, radius):
    kx, ky = k % m, k // m
    return [iy * m + ix for iy in range(max(ky - radius, 0), min(ky + radius + 1, m))
            for ix in range(max(kx - radius, 0), min(kx + radius + 1, m))]


@pytest.mark.parametrize("p0", ["lower", "diag"])
def test_adaptive_row_equals_adaptive_fsai_on_every_row(small_biharmonic, p0):
    """Algorithm 1 row by row: a row's scores depend on A and its own pattern only, so running
    the steps for one row alone (adaptive_row, used at sizes where the whole matrix is out of
    reach) gives that row of the whole-matrix run; also from a window of A of radius 8 around the
    row (t_max = 6 grows a pattern by at most 6 grid steps, candidates one further)."""
    A = small_biharmonic.A[0]            # 16 x 16 patches, d = 10
    m = 16
    P0 = fsai.lower_pattern(A) if p0 == "lower" else fsai.diag_pattern(A.n_rows)
    whole = fsai.adaptive_fsai(A, P0, 6).fsai.pattern
    grown = 0
    for k in range(A.n_rows):
        row = fsai.adaptive_row(A, k, P0[k], 6)
        assert row == whole[k], f"row {k}"
        grown += len(row) - len(P0[k])
    assert grown >= 3 * A.n_rows          # the rows really grew
    for k in (0, 17, 8 * 16 + 8, 255, 100):
        Aw = _rows_only(A, _grid_window(k, m, 8))
        assert fsai.adaptive_row(Aw, k, P0[k], 6) == whole[k], f"windowed row {k}"


def _inadmissible_candidate_matrix():
    """A = X^T X with X = [[I, I, B], [0, 0, E]] (blocks of 2): block columns 0 and 1 of A are
    equal, so once block 0 is in a row's pattern, block 1 has W_1 = A_11 - A_10 A_00^-1 A_01 = 0
    (exactly: A_00 = A_01 = A_11 = I and B, E hold small integers)."""
    I2 = np.eye(2)
    B = np.array([[1.0, 2.0], [0.0, 1.0]])
    E = np.array([[2.0, 1.0], [1.0, 3.0]])
    X = np.block([[I2, I2, B], [np.zeros((2, 2)), np.zeros((2, 2)), E]])
    return _block_csr_from_dense(X.T @ X, 2)


def test_candidate_without_computable_gain_is_inadmissible():
    """Algorithm 1 assumes SPD A, so every candidate's Schur complement W_c - H^T S^-1 H is SPD.
    In FP64 a candidate whose complement fails its Cholesky factorisation has no rho_c: it is
    skipped, and a row left with no computable candidate retires (it is not grown into a
    singular local system)."""
    Ab = _inadmissible_candidate_matrix()
    r0 = fsai.row_rhos(Ab, 2, [2], [0, 1])
    assert set(r0) == {0, 1} and r0[0] == r0[1] < 1.0          # tie: the smaller column is taken
    assert fsai.choose(r0, 1e-9) == 0
    assert fsai.row_rhos(Ab, 2, [0, 2], [1]) == {}              # W_1 = 0: not computable
    res = fsai.adaptive_fsai(Ab, fsai.diag_pattern(3), 3)
    assert res.fsai.pattern[2] == [0, 2]
    assert fsai.adaptive_row(Ab, 2, [2], 3) == [0, 2]
    # the retained pattern gives a valid FSAI: diag_B(G A G^T) = I on row 2
    G, A = res.fsai.G.to_dense(), Ab.to_dense()
    assert np.max(np.abs((G @ A @ G.T)[4:6, 4:6] - np.eye(2))) <= 1e-12


def _indefinite_a1_matrix():
    """A = X^T X (9 x 9, blocks of 3) with strongly coupled blocks: the adaptive outer FSAI
    (from the diagonal, t_max = 2) succeeds, but the diagonal blocks of the computed
    A_1 = F_0 A F_0^T have lost definiteness to the rounding of the triple product, far beyond
    rounding noise (seeded; the margin is asserted by the test)."""
    rng = np.random.default_rng(165)
    N = 9
    X = np.eye(N) + 1e4 * rng.standard_normal((N, N)) * (rng.random((N, N)) < 0.3)
    X += np.diag(10.0 ** rng.uniform(-6, 0, N))
    A = X.T @ X
    return _block_csr_from_dense(0.5 * (A + A.T), 3)


def test_nested_fsai_falls_back_to_block_jacobi_when_A1_is_not_spd():
    """Section 2.2 on an A whose computed A_1 = F_0 A F_0^T is not numerically SPD: the inner
    FSAI cannot be formed, and the inner level is block Jacobi of A_1 (Remark 2.4) with
    diag_B(A_1) = S of the outer FSAI (Lemma 2.3), so M is the plain block-FSAI G^T G."""
    Ab = _indefinite_a1_matrix()
    P0 = fsai.diag_pattern(Ab.n_rows)
    outer = fsai.adaptive_fsai(Ab, P0, 2).fsai
    A1 = bk.galerkin_product(outer.F, Ab, outer.F.transpose())
    worst = min(np.linalg.eigvalsh(0.5 * (A1.block(k, k) + A1.block(k, k).T))[0] / np.linalg.norm(A1.block(k, k))
                for k in range(Ab.n_rows))
    assert worst < -1e-10                          # indefinite well beyond rounding noise
    with pytest.raises(fsai.NotSPD):
        fsai.adaptive_fsai(A1, P0, 2)
    nf = fsai.nested_fsai(Ab, P0, 2)
    assert not nf.inner_nested
    assert nf.inner.pattern == P0
    assert nf.logdet_S() == pytest.approx(outer.logdet_S(), rel=1e-14)
    r = np.random.default_rng(2).standard_normal(Ab.n_rows * Ab.d)
    plain = fsai.apply_M(outer.G, r)
    assert np.max(np.abs(nf.apply(r) - plain)) <= 1e-12 * np.max(np.abs(plain))


def test_block_jacobi_from_schur_is_block_jacobi_of_A1(small_biharmonic):
    """The fallback's blocks L_S^-1 equal block Jacobi of A_1 (Lemma 2.3: diag_B(F_0 A F_0^T) =
    S) on a matrix where A_1 is well conditioned."""
    A = small_biharmonic.A[2]
    outer = fsai.fsai(A, fsai.lower_pattern(A))
    A1 = bk.galerkin_product(outer.F, A, outer.F.transpose())
    jac = fsai.fsai(A1, fsai.diag_pattern(A.n_rows))
    fb = fsai.block_jacobi_from_schur(outer)
    for k in range(A.n_rows):
        ref = jac.G.block(k, k)
        assert np.max(np.abs(fb.G.block(k, k) - ref)) <= 1e-10 * np.max(np.abs(ref))
    assert fb.logdet_S() == pytest.approx(jac.logdet_S(), rel=1e-10)


def _weak_coupling_matrix(eps):
    """Two blocks of 2: A = [[I, eps I], [eps I, I]]; candidate 0 of row 1 has H_10 = eps I, so
    rho_0 = det(I - eps^2 I) = (1 - eps^2)^2 exactly in real arithmetic."""
    I2 = np.eye(2)
    return _block_csr_from_dense(np.block([[I2, eps * I2], [eps * I2, I2]]), 2)


def test_stop_test_takes_the_tie_band():
    """Algorithm 1 adds c* only when rho_c* < tau; with tau = 1 a candidate coupled to the row by
    rounding alone has rho_c = 1 up to rounding, so the test takes the tie band: rho_c* must be
    below tau (1 - tie_rel).  A gain of 2e-6 is taken, one of 2e-12 is not."""
    strong = _weak_coupling_matrix(1e-3)
    weak = _weak_coupling_matrix(1e-6)
    assert fsai.row_rhos(strong, 1, [1], [0])[0] == pytest.approx((1 - 1e-6) ** 2, rel=1e-14)
    assert 1.0 - fsai.row_rhos(weak, 1, [1], [0])[0] == pytest.approx(2e-12, rel=1e-3)
    assert fsai.adaptive_fsai(strong, fsai.diag_pattern(2), 1).fsai.pattern[1] == [0, 1]
    assert fsai.adaptive_fsai(weak, fsai.diag_pattern(2), 1).fsai.pattern[1] == [1]
    assert fsai.adaptive_row(weak, 1, [1], 1) == [1]
    assert fsai.accepts(1.0 - 2e-9, 1.0, 1e-9) and not fsai.accepts(1.0 - 5e-10, 1.0, 1e-9)
