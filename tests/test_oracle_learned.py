"""Pins of the learned candidate scoring (oracle/learned.py): BF16 rounding, the network's
gradient against finite differences, Adam's closed form, the first-order gain feature against
Lemma 2.8's rho_c, the candidate pools against Algorithm 1's admissible sets, selection and the
gate's measure."""
import numpy as np
import pytest

import pum_inputs as pin
from oracle import blocks as bk
from oracle import fsai, learned


def test_bf16_round_to_nearest_even():
    x = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -8 + 2 ** -20, -2.5, 3.0e-39, 65504.0], np.float32)
    want = [1.0, 1.0, 1 + 2 ** -6, 1 + 2 ** -7, -2.5, None, 65536.0]
    got = learned.bf16(x)
    for g, w, xi in zip(got, want, x):
        if w is not None:
            assert g == w, (xi, g, w)
    # every result has at most 8 significant bits
    assert all(np.float32(g).view(np.uint32) & 0xFFFF == 0 for g in got)


def _batch(seed, n=64):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, learned.N_FEATURES)), (rng.random(n) < 0.3).astype(float)


def test_gradient_matches_finite_differences():
    """Backward pass of the 12-64-64-1 ReLU network with the mean binary cross-entropy, against
    central differences of the loss (FP64 master weights, no BF16 rounding)."""
    m = learned.init_mlp(3)
    for p in m.params():
        p[...] = p.astype(np.float64)
    m = learned.MLP(*[np.asarray(p, dtype=np.float64) for p in m.params()])
    m.b1[...] = 0.05
    m.b2[...] = 0.05
    X, y = _batch(4)
    _, grads = learned.loss_and_grad(m, X, y, quant=False)
    rng = np.random.default_rng(5)
    h = 1e-6
    for p, g in zip(m.params(), grads):
        flat = p.reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = learned.loss_and_grad(m, X, y, quant=False)
            flat[idx] = old - h
            lm, _ = learned.loss_and_grad(m, X, y, quant=False)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - np.reshape(g, -1)[idx]) <= 1e-6 * max(1.0, abs(fd)), (p.shape, idx)


def test_loss_is_the_binary_cross_entropy_of_the_logits():
    m = learned.init_mlp(1)
    X, y = _batch(6, 16)
    logit, _ = learned.forward(m, X)
    p = 1.0 / (1.0 + np.exp(-logit))
    ref = -np.mean(y * np.log(p) + (1 - y) * np.log(1 - p))
    assert learned.loss_and_grad(m, X, y)[0] == pytest.approx(ref, rel=1e-12)


def test_adam_closed_form():
    """With a constant gradient g, the bias-corrected moments are g and g^2, so every step moves
    the parameter by lr g / (|g| + eps)."""
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    state = [(np.zeros(3), np.zeros(3))]
    for t in range(1, 6):
        q = p.copy()
        learned.adam([p], [g], state, t, lr=0.01)
        np.testing.assert_allclose(q - p, 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_first_order_gain_is_one_minus_rho_for_weak_coupling():
    """Feature 2: g_c = |L_c^-1 (G0 A)_kc^T|_F^2 with G0 the block-Jacobi FSAI (P0 = diagonal)
    is tr(A_cc^-1 A_ck A_kk^-1 A_kc), and Lemma 2.8 gives rho_c = det(I - A_cc^-1 A_ck A_kk^-1
    A_kc) = 1 - g_c + O(eps^4) for a coupling of size eps."""
    rng = np.random.default_rng(11)
    d = 3
    S1 = rng.standard_normal((d, d))
    S2 = rng.standard_normal((d, d))
    Akk, Acc = S1 @ S1.T + d * np.eye(d), S2 @ S2.T + d * np.eye(d)
    B = rng.standard_normal((d, d))
    for eps in (1e-2, 1e-3):
        A = np.block([[Acc, eps * B.T], [eps * B, Akk]])  # block 0 = c, block 1 = k
        Ab = bk.from_blocks(2, 2, d, {(i, j): A[i * d:(i + 1) * d, j * d:(j + 1) * d] for i in range(2) for j in range(2)})
        P0 = fsai.diag_pattern(2)
        G0 = fsai.fsai(Ab, P0).G
        rows, cols, X = learned.features(Ab, G0, P0)
        assert list(rows) == [1] and list(cols) == [0]
        g = 10 ** X[0, 2]
        rho = fsai.row_rhos(Ab, 1, [1], [0])[0]
        assert abs((1 - rho) - g) <= 10 * eps ** 4 * max(1.0, np.linalg.norm(B) ** 4)
        assert X[0, 0] == 1.0 and X[0, 5] == 1.0 and X[0, 4] == 0.0


def test_candidate_pool_ring1_is_algorithm1_admissible_set(small_biharmonic):
    A = small_biharmonic.A[1]
    pat = A.pattern()
    P0 = fsai.lower_pattern(A)
    for k in range(A.n_rows):
        r1, r2 = learned.candidate_pool(A, k, P0[k])
        assert r1 == fsai.admissible(pat, P0[k], k)
        assert not set(r1) & set(r2) and all(c < k for c in r2)
        assert set(r2) <= set(c for j in r1 for c in pat[j])


def test_selection_and_gate_ratio():
    P0 = [[0], [0, 1], [2]]
    rows = np.array([1, 2, 2, 2])
    cols = np.array([0, 0, 1, 0])
    got = learned.select([2, 2, 2], [0, 1, 0], [0.5, 0.9, 0.1], [[0], [1], [2]], 1)
    assert got == [[0], [1], [1, 2]]
    got = learned.select(rows[1:], cols[1:] * 0 + np.array([0, 1, 1]), [0.3, 0.3, 0.2], [[0], [1], [2]], 1)
    assert got[2] == [0, 2]      # tie between columns 0 and 1: the smaller column
    assert learned.gate_ratio(np.array([1.0, 2.0]), np.array([0.0, 1.0]), np.array([2.0, 3.0])) == 0.5
    del P0
