"""GPU parity of the learned candidate scoring (an addition to the paper's Algorithm 1, which stays
its fallback and judge): candidate pools, features and labels against the oracle, the network's
logits and gradients against the oracle's FP64 forward and backward, training on the device, the
learned set-up with its gate, and the fallback to Algorithm 1 when the gate fails."""
import numpy as np
import pytest

import pum_inputs as pin
from oracle import fsai, learned, pum
from _util import to_pview, to_view

pytestmark = pytest.mark.gpu

PR = pin.SMALL_BIHARMONIC


@pytest.fixture(scope="module")
def lib():
    import paper_2509_06744_gb300 as L
    return L


@pytest.fixture(scope="module")
def ctx(lib):
    c = lib.Context(0)
    yield c
    c.close()


def _hier(m, levels):
    f = pum.fourier_source(pin.fourier_coefficients(PR.rhs_seed), PR.rhs_decay)
    return pum.build_hierarchy(m, PR.p, PR.equation, levels, f=f, constants=PR.nitsche)


def _gpu_hier(lib, ctx, m, levels):
    """A biharmonic p = 3 hierarchy assembled on the device (m x m patches), with its load vector."""
    import torch
    b = torch.zeros(m * m * PR.d, dtype=torch.float64, device="cuda")
    H = lib.Hierarchy.assemble(ctx, PR.equation, PR.p, m, levels, f_coef=pin.fourier_coefficients(PR.rhs_seed),
                               f_decay=PR.rhs_decay, nitsche=PR.nitsche, b=b)
    return H, b


@pytest.fixture(scope="module")
def small(lib, ctx):
    h = _hier(16, 3)
    H = lib.Hierarchy.from_bsr(ctx, [to_view(A) for A in h.A], [to_pview(P) for P in h.P])
    H.setup(p0="lower", adaptive=True, t_max=6, k=2)
    yield h, H
    H.close()


def _model_dict(m):
    return {"w1": m.W1, "b1": m.b1, "w2": m.W2, "b2": m.b2, "w3": m.w3, "b3": m.b3}


@pytest.mark.parametrize("level", [0, 1])
def test_candidates_features_and_labels_match_oracle(small, level):
    """Pools bit-exact (ring 1 = Algorithm 1's admissible set of P0, ring 2 one step further),
    features within FP32 rounding of the oracle's FP64 values, labels = Algorithm 1's choices."""
    h, H = small
    A = h.A[level]
    P0 = fsai.lower_pattern(A)
    G0 = fsai.fsai(A, P0).G
    m = int(round(np.sqrt(A.n_rows)))                      # the library reads the square grid of patches
    rows, cols, X = learned.features(A, G0, P0, m=m)
    got = H.candidates(level)
    assert np.array_equal(got["row"].cpu().numpy(), rows) and np.array_equal(got["col"].cpu().numpy(), cols)
    Xg = got["x"].cpu().numpy().astype(np.float64)
    assert np.max(np.abs(Xg - X) / np.maximum(1.0, np.abs(X))) <= 1e-5
    ref_pattern = fsai.adaptive_fsai(A, P0, 6).fsai.pattern
    assert np.array_equal(got["y"].cpu().numpy(), learned.labels(rows, cols, ref_pattern))


def test_mlp_logits_and_gradients_match_oracle(lib, ctx, small):
    """Forward: BF16-rounded weights, FP32 accumulation against the oracle's FP64 arithmetic on
    the same rounded weights.  Backward: the mean binary cross-entropy's gradient, FP32 on the
    GPU against FP64 in the oracle (both with the rounding passed through)."""
    import torch
    h, H = small
    cand = H.candidates(0)
    m = learned.init_mlp(7)
    m.b1[...] = 0.01
    m.b2[...] = -0.02
    model = _model_dict(m)
    X = cand["x"].cpu().numpy().astype(np.float64)
    y = cand["y"].cpu().numpy().astype(np.float64)
    logit_ref, _ = learned.forward(m, X)
    logit = ctx.mlp_forward(model, cand["x"]).cpu().numpy()
    assert np.max(np.abs(logit - logit_ref)) <= 1e-4 * max(1.0, np.max(np.abs(logit_ref)))
    loss, grads = ctx.mlp_grad(model, cand["x"], cand["y"])
    loss_ref, grads_ref = learned.loss_and_grad(m, X, y)
    assert loss == pytest.approx(loss_ref, rel=1e-5)
    for name, gr in zip(["w1", "b1", "w2", "b2", "w3", "b3"], grads_ref):
        g = np.asarray(grads[name], dtype=np.float64)
        assert np.max(np.abs(g - gr)) <= 1e-4 * max(np.max(np.abs(gr)), 1e-6), name
    # deterministic: the same call twice gives the same bits
    loss2, grads2 = ctx.mlp_grad(model, cand["x"], cand["y"])
    assert loss2 == loss and all(np.array_equal(grads[k], grads2[k]) for k in grads)
    del torch


@pytest.fixture(scope="module")
def trained(lib, ctx):
    """A model trained on the device on Algorithm 1's choices for the 64x64-patch problem
    (levels with at least 256 block rows)."""
    import torch
    H, _ = _gpu_hier(lib, ctx, 64, 5)
    H.setup(p0="lower", adaptive=True, t_max=6, k=3)
    cs = [H.candidates(l) for l in range(3)]
    x = torch.cat([c["x"] for c in cs]).contiguous()
    y = torch.cat([c["y"] for c in cs]).contiguous()
    m0 = _model_dict(learned.init_mlp(1))
    loss0, _ = ctx.mlp_grad(m0, x, y)
    model, loss = ctx.mlp_train(m0, x, y, epochs=30, batch=4096, lr=3e-3, seed=5)
    H.close()
    return model, loss0, loss, x, y


def test_training_reduces_the_loss(trained):
    model, loss0, loss, x, y = trained
    assert loss < 0.6 * loss0 and loss < 0.3


def test_learned_setup_passes_gate_and_matches_selection(lib, ctx, trained):
    """On the 128x128-patch problem (not a training matrix) the learned pattern passes the gate on
    the levels it scores, each row holds P0 plus its t_max best-scoring candidates (the oracle's
    selection rule applied to the GPU's logits), and PCG converges like Algorithm 1's set-up."""
    import torch
    model = trained[0]
    H, b = _gpu_hier(lib, ctx, 128, 6)
    H.setup(p0="lower", adaptive=True, t_max=6, k=3)
    x = torch.zeros_like(b)
    ref = H.pcg(b, x, rtol=1e-8, maxit=100)
    e0 = torch.tensor(pin.uniform_vector(b.numel(), 5), dtype=torch.float64, device="cuda")
    rho_ref = H.convergence_factor(e0, 6)
    cand = H.candidates(0)
    ctx.set_pattern_model(model)
    H.setup(p0="lower", adaptive=2, t_max=6, k=3)
    info = H.info(0)
    assert info["gate"] >= -1e-12 and info["learned"] == 1 and info["gate"] <= 0.05
    assert H.info(3)["gate"] == -1.0                     # 16x16: Algorithm 1 (below 1024 rows)
    logits = ctx.mlp_forward(model, cand["x"]).cpu().numpy()
    from _util import from_export
    A0 = from_export(H.export(0, lib.PUM_MAT_A))
    P0 = fsai.lower_pattern(A0)
    want = learned.select(cand["row"].cpu().numpy(), cand["col"].cpu().numpy(), logits, P0, 6)
    G = from_export(H.export(0, lib.PUM_MAT_G))
    assert [list(G.row(k)) for k in range(G.n_rows)] == want
    x = torch.zeros_like(b)
    rep = H.pcg(b, x, rtol=1e-8, maxit=100)
    assert rep["converged"] and rep["iters"] <= ref["iters"] + 1
    # the other half of the acceptance rule: the V-cycle's convergence factor within 5% of the
    # one with Algorithm 1's patterns (the set-up's gate measures the Kaporin half per level)
    assert H.convergence_factor(e0, 6) <= 1.05 * rho_ref
    ctx.set_pattern_model(None)
    H.close()


def test_gate_falls_back_to_algorithm1(lib, ctx, small):
    """An untrained network (random weights) picks poor candidates: the gate refuses the level and
    Algorithm 1 runs on every row, so the patterns are Algorithm 1's, bit for bit."""
    import torch
    H, _ = _gpu_hier(lib, ctx, 64, 4)
    H.setup(p0="lower", adaptive=True, t_max=6, k=2)
    from _util import from_export
    ref = from_export(H.export(0, lib.PUM_MAT_G))
    m = learned.init_mlp(2)
    m.w3[...] = -np.abs(m.w3)                          # scores that ignore the gain features
    m.W1[:, 2] = 0.0
    m.W1[:, 5] = 0.0
    ctx.set_pattern_model(_model_dict(m))
    H.setup(p0="lower", adaptive=2, t_max=6, k=2)
    info = H.info(0)
    assert info["learned"] == 0 and info["gate"] > 0.05
    G = from_export(H.export(0, lib.PUM_MAT_G))
    assert np.array_equal(G.indptr, ref.indptr) and np.array_equal(G.indices, ref.indices)
    ctx.set_pattern_model(None)
    with pytest.raises(lib.PumError):
        H.setup(p0="lower", adaptive=2, t_max=6, k=2)    # no model: refused
    H.close()
    del torch
