"""The tensor-core surrogate MLP against the CPU oracle (oracle/mlp.py).

The GPU stores weights W1..W3, inputs and hidden activations in BF16 and
accumulates in FP32; the oracle is evaluated in float64 on the same
BF16-rounded weights and inputs, with its hidden activations rounded to
BF16 as well.  What remains is FP32 accumulation order and, in the
backward pass, the BF16 rounding of dZ the GPU applies before each GEMM:
tolerances are derived from that (about 2^-8 relative per rounding)."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import mlp as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import paper_2406_08496_gb300 as L
    L.build()
    L.load_library()


def bf16_bits(a):
    f = np.asarray(M.bf16_round(a), dtype=np.float32)
    return (f.view(np.uint32) >> 16).astype(np.uint16)


@pytest.mark.parametrize("M_,N,K", [(128, 256, 64), (256, 256, 256), (384, 64, 512), (128, 512, 128),
                                    (1024, 256, 2048)])
def test_gemm_matches_float64(M_, N, K):
    from paper_2406_08496_gb300 import gemm_bf16
    rng = np.random.default_rng(M_ + N + K)
    A = rng.standard_normal((M_, K))
    B = rng.standard_normal((N, K))
    Ab, Bb = M.bf16_round(A), M.bf16_round(B)
    D = gemm_bf16(bf16_bits(A), bf16_bits(B))
    ref = Ab @ Bb.T
    scale = np.abs(Ab) @ np.abs(Bb).T
    err = np.abs(D - ref)
    assert np.all(err <= 2e-6 * scale + 1e-6), float((err / (scale + 1e-9)).max())


def _params(seed):
    p = M.init_params(seed)
    rng = np.random.default_rng(seed + 1)
    for k in p:
        if k.startswith("b"):
            p[k] = rng.standard_normal(p[k].shape) * 0.1
    return p


def _bf16_params(p):
    q = dict(p)
    for k in ("W1", "W2", "W3"):
        q[k] = M.bf16_round(p[k])
    for k in ("b1", "b2", "b3", "W4", "b4"):
        q[k] = np.asarray(p[k], dtype=np.float32).astype(np.float64)
    return q


def _inputs(n, seed, nf=9):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, nf)).astype(np.float32)
    Xp = np.zeros((n, 64))
    Xp[:, :nf] = M.bf16_round(X)
    return X, Xp


U32 = 2.0 ** -24  # unit roundoff of binary32


def forward_bound(q, Xp):
    """Oracle forward (float64, hidden activations rounded to BF16 as the GPU
    stores them) and the per-row tolerance of the GPU's output: one BF16
    rounding unit (2^-8) of the head's absolute mass sum_j |w4_j h3_j|.

    Both sides round the same hidden values to BF16; they differ only where
    the GPU's FP32 sums (and its GELU, within 3.1e-6 of the exact one)
    and the oracle's float64 values fall on opposite sides of a rounding
    boundary, which moves that activation by one BF16 spacing (2^-7 of it
    at most).  Such flips are rare (the FP32 sums are within about 2^-20 of
    the exact ones, against BF16 spacings of 2^-7) and of either sign, so
    their effect on y stays far below one unit of the head's mass -- an FP32
    emulation of the network on these inputs stays below a quarter of it --
    while a wrong row, tile or weight moves y by its own size, about a tenth
    of the mass."""
    h = np.asarray(Xp, np.float64)
    for l in (1, 2, 3):
        z = h @ q[f"W{l}"].T + q[f"b{l}"]
        h = M.bf16_round(M.gelu(z))
    w4, b4 = q["W4"][0], q["b4"][0]
    y = h @ w4 + b4
    return y, 2.0 ** -8 * (np.abs(h) @ np.abs(w4)) + 1e-5


def test_forward_matches_oracle():
    from paper_2406_08496_gb300 import Surrogate
    p = _params(3)
    s = Surrogate(batch=256, seed=0)
    s.set_params(p)
    X, Xp = _inputs(700, 4)  # three batches, the last one partial
    y = s.forward(X)
    ref, bound = forward_bound(_bf16_params(p), Xp)
    assert np.all(np.isfinite(y))
    err = np.abs(y - ref)
    assert np.all(err <= bound), float(np.max(err / bound))
    # the tolerance is small against the outputs themselves
    assert np.median(bound) < 0.1 * np.median(np.abs(ref))


def test_forward_production_size_matches_oracle():
    """The persistent fused forward at the size the assignment loop and the
    benchmark use (131,072-row batches: 1,024 tiles over the SMs, each CTA
    looping over several tiles and wrapping its weight ring), with the
    eleven features of the assignment loop and a partial second batch:
    element by element within the derived bound, and bit for bit equal to
    the same rows pushed through a 256-row model (a row's arithmetic does not
    depend on which CTA or tile computes it)."""
    from paper_2406_08496_gb300 import Surrogate
    nf = 11
    p = _params(8)
    p["W1"] = p["W1"].copy()
    p["W1"][:, nf:] = 0.0
    rows = 131072 + 1000
    X, Xp = _inputs(rows, 9, nf=nf)
    big = Surrogate(n_features=nf, batch=131072, seed=0)
    big.set_params(p)
    y = big.forward(X)
    big.close()
    ref, bound = forward_bound(_bf16_params(p), Xp)
    assert np.all(np.isfinite(y))
    err = np.abs(y - ref)
    assert np.all(err <= bound), (int(np.argmax(err / bound)), float(np.max(err / bound)))
    small = Surrogate(n_features=nf, batch=256, seed=0)
    small.set_params(p)
    pick = np.concatenate([np.arange(0, 2048), np.arange(rows - 2048, rows),
                           np.random.default_rng(10).choice(rows, 4096, replace=False)])
    ys = small.forward(X[pick])
    small.close()
    assert np.array_equal(ys.view(np.uint32), y[pick].view(np.uint32))


def test_gradients_match_oracle():
    from paper_2406_08496_gb300 import Surrogate
    p = _params(5)
    s = Surrogate(batch=256, seed=0)
    s.set_params(p)
    X, Xp = _inputs(200, 6)
    t = np.random.default_rng(7).standard_normal(200).astype(np.float32)
    loss, g = s.grad(X, t)
    q = _bf16_params(p)
    ref_loss = float(np.mean((M.forward(q, Xp, act_round=M.bf16_round) - t) ** 2))
    assert abs(loss - ref_loss) <= 1e-2 * ref_loss
    gr = M.backward(q, Xp, t.astype(np.float64), act_round=M.bf16_round)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4"):
        a, b = g[k].astype(np.float64).reshape(-1), gr[k].reshape(-1)
        if k == "W1":  # padded input columns carry no gradient
            a = a.reshape(256, 64)[:, :9].reshape(-1)
            b = b.reshape(256, 64)[:, :9].reshape(-1)
        rel = np.linalg.norm(a - b) / (np.linalg.norm(b) + 1e-12)
        assert rel < 3e-2, (k, rel)
        # elementwise, at 2^-7 sqrt(K) of the tensor's scale (BF16 rounding of dZ)
        tol = 2 ** -7 * np.sqrt(256) * (np.abs(b) + np.sqrt(np.mean(b * b)))
        assert np.all(np.abs(a - b) <= tol), (k, float(np.max(np.abs(a - b) / tol)))
    assert np.all(g["W1"].reshape(256, 64)[:, 9:] == 0)


F32 = np.float32
ADAM_B1, ADAM_B2, ADAM_EPS = float(F32(0.9)), float(F32(0.999)), float(F32(1e-8))


def _adam_reference(p, grads_seq, lr):
    """The oracle's Adam (float64, on the FP32 constants the kernel holds),
    with a per-element bound on the FP32 evaluation: each step's update
    lr m_hat / (sqrt(v_hat) + eps) takes about a dozen roundings, each within
    2^-24 of the magnitudes it combines (|m| carried as sum of |g| terms so
    that cancellation in m is covered), and the subtraction rounds once more
    within 2^-24 |p|; the bias corrections are rounded once each."""
    q = {k: np.asarray(v, np.float32).astype(np.float64) for k, v in p.items()}
    m = {k: np.zeros_like(v) for k, v in q.items()}
    v = {k: np.zeros_like(v) for k, v in q.items()}
    mabs = {k: np.zeros_like(v) for k, v in q.items()}
    tol = {k: np.zeros_like(v) for k, v in q.items()}
    for t, g in enumerate(grads_seq, start=1):
        g64 = {k: np.asarray(g[k], np.float32).astype(np.float64) for k in q}
        M.adam_step(q, g64, m, v, t, lr, beta1=ADAM_B1, beta2=ADAM_B2, eps=ADAM_EPS)
        for k in q:
            mabs[k] = ADAM_B1 * mabs[k] + (1 - ADAM_B1) * np.abs(g64[k])
            vh = v[k] / (1 - ADAM_B2 ** t)
            step_mag = lr * (mabs[k] / (1 - ADAM_B1 ** t)) / (np.sqrt(vh) + ADAM_EPS)
            tol[k] += 16 * U32 * step_mag + U32 * np.abs(q[k])
    return q, tol


def test_adam_matches_oracle():
    """Three Adam steps on the FP32 master weights with caller-given
    gradients (magnitudes from 1e-9 to 1, both signs, so that eps and the
    bias corrections matter) against the oracle's adam_step, element by
    element within the FP32 evaluation bound."""
    from paper_2406_08496_gb300 import Surrogate
    p = _params(12)
    s = Surrogate(batch=256, seed=0)
    s.set_params(p)
    rng = np.random.default_rng(13)
    grads = []
    for _ in range(3):
        g = {}
        for k, shape in zip(("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4"),
                            [(256, 64), (256,), (256, 256), (256,), (256, 256), (256,), (1, 256), (1,)]):
            mag = 10.0 ** rng.uniform(-9, 0, shape)
            g[k] = (np.sign(rng.standard_normal(shape)) * mag).astype(np.float32)
        grads.append(g)
    lr = 1e-3
    for g in grads:
        s.apply_grads(g, lr)
    got = s.get_params()
    ref, tol = _adam_reference(p, grads, lr)
    for k in ref:
        a = got[k].astype(np.float64).reshape(ref[k].shape)
        err = np.abs(a - ref[k])
        assert np.all(err <= tol[k]), (k, float(np.max(err / tol[k])))
        # the update really happened: weights moved by about lr per step
        assert np.mean(np.abs(a - np.asarray(p[k], np.float32).reshape(ref[k].shape))) > 0.5 * lr
    # the BF16 copies the forward pass reads were refreshed from the new weights
    X, Xp = _inputs(300, 14)
    q = _bf16_params({k: got[k].astype(np.float64).reshape(ref[k].shape) for k in got})
    yref, bound = forward_bound(q, Xp)
    assert np.all(np.abs(s.forward(X) - yref) <= bound)
    s.close()


def test_train_step_is_gradient_then_adam():
    """One lpsim_mlp_train step on a full batch equals the gradient of that
    batch followed by the oracle's Adam step.  The train call sums the batch
    in a shuffled row order and its split-K gradient sums use atomics, so its
    gradient differs from lpsim_mlp_grad's by the FP32 noise of those sums
    (measured here by summing the rows in another order); at t = 1 Adam moves
    each weight by lr g / (|g| + eps), which that noise changes by at most
    2 lr |dg| / |g|."""
    from paper_2406_08496_gb300 import Surrogate
    p = _params(15)
    s = Surrogate(batch=256, seed=0)
    s.set_params(p)
    X, _ = _inputs(256, 16)
    t = np.random.default_rng(17).standard_normal(256).astype(np.float32)
    _, g = s.grad(X, t)
    perm = np.random.default_rng(18).permutation(256)
    _, g2 = s.grad(X[perm], t[perm])
    lr = 1e-3
    s.set_params(p)
    s.train(X, t, steps=1, lr=lr, seed=3)
    got = s.get_params()
    ref, tol = _adam_reference(p, [g], lr)
    for k in ref:
        gk = g[k].astype(np.float64).reshape(ref[k].shape)
        noise = 4 * np.abs(gk - g2[k].astype(np.float64).reshape(ref[k].shape)) + 2 ** -20 * np.sqrt(np.mean(gk ** 2))
        bound = tol[k] + lr * np.minimum(2.0, 2 * noise / (np.abs(gk) + ADAM_EPS))
        a = got[k].astype(np.float64).reshape(ref[k].shape)
        err = np.abs(a - ref[k])
        assert np.all(err <= bound), (k, float(np.max(err / bound)))
    # padded input columns have zero gradient and stay put
    assert np.array_equal(got["W1"][:, 9:], np.asarray(p["W1"], np.float32)[:, 9:])
    s.close()


def test_training_reduces_loss():
    from paper_2406_08496_gb300 import Surrogate
    rng = np.random.default_rng(11)
    X = rng.uniform(-1, 1, (20000, 9)).astype(np.float32)
    t = (np.sin(2 * X[:, 0]) + X[:, 1] * X[:, 2] + 0.5 * np.abs(X[:, 3]) - X[:, 4] ** 2).astype(np.float32)
    s = Surrogate(batch=1024, seed=1)
    losses = s.train(X, t, steps=600, lr=2e-3, seed=2)
    assert np.all(np.isfinite(losses))
    assert losses[-50:].mean() < 0.05 * losses[:5].mean(), (losses[:5].mean(), losses[-50:].mean())
    # the trained network generalises to fresh samples
    Xv = rng.uniform(-1, 1, (4000, 9)).astype(np.float32)
    tv = (np.sin(2 * Xv[:, 0]) + Xv[:, 1] * Xv[:, 2] + 0.5 * np.abs(Xv[:, 3]) - Xv[:, 4] ** 2)
    mse = float(np.mean((s.forward(Xv) - tv) ** 2))
    assert mse < 0.05 * float(np.var(tv)), mse


def test_gelu_within_its_error_bound():
    """The epilogues' GELU and GELU' (normal CDF as a logistic of a fitted
    odd polynomial: |error| < 6.8e-6 and |z| |error| < 3.1e-6 over the fit's
    grid; exact density) against the float64 closed forms, over the range the
    activations take and beyond: the fit's bound plus a few float32
    roundings of each term."""
    import oracle.mlp as M
    from paper_2406_08496_gb300 import gelu_eval
    z = np.concatenate([np.linspace(-12.0, 12.0, 200001), np.random.default_rng(4).standard_normal(100000) * 3.0])
    z = z.astype(np.float32)
    g, dg = gelu_eval(z)
    z64 = z.astype(np.float64)
    ref_g, ref_dg = M.gelu(z64), M.gelu_grad(z64)
    # the fit's 3.1e-6 in z Phi (6.8e-6 in Phi) plus float32 evaluation
    # (hardware exp2 and reciprocal, four fused multiply-adds, a few products)
    tol_g = np.minimum(4e-6, 7.5e-6 * np.abs(z64)) + 3e-7 * np.abs(ref_g) + 1e-30
    tol_dg = 8e-6 + 3e-7 * np.abs(z64)
    assert np.all(np.abs(g - ref_g) <= tol_g), float(np.max(np.abs(g - ref_g) / tol_g))
    assert np.all(np.abs(dg - ref_dg) <= tol_dg), float(np.max(np.abs(dg - ref_dg) / tol_dg))


def test_training_pool_parts_equal_one_upload():
    """Samples appended to the device pool in parts train exactly like the
    same samples given at once (same rows in the same order, same shuffled
    passes for the same seed): parameters equal up to the FP32 noise of the
    split-K gradient sums; the losses fall."""
    from paper_2406_08496_gb300 import Surrogate
    rng = np.random.default_rng(21)
    X = rng.uniform(-1, 1, (5000, 9)).astype(np.float32)
    t = (np.sin(2 * X[:, 0]) + X[:, 1] * X[:, 2]).astype(np.float32)
    p = _params(22)
    a = Surrogate(batch=1024, seed=0)
    a.set_params(p)
    la = a.train(X, t, steps=40, lr=1e-3, seed=5)
    b = Surrogate(batch=1024, seed=0)
    b.set_params(p)
    for part in np.array_split(np.arange(5000), 3):
        b.pool_add(X[part], t[part])
    assert b.pool_size() == 5000
    lb = b.train_pool(40, lr=1e-3, seed=5)
    assert la[-5:].mean() < 0.5 * la[:5].mean()
    # the same rows in the same order: the runs differ only by the split-K
    # atomics' summation order, which Adam can turn into up to a step of lr
    # on a weight whose gradient is near zero; in norm they agree closely
    # (the loss curves too: a single loss may move by ~1e-3 of itself)
    assert np.linalg.norm(la - lb) <= 1e-3 * np.linalg.norm(la), float(np.linalg.norm(la - lb) / np.linalg.norm(la))
    pa, pb = a.get_params(), b.get_params()
    for k in pa:
        d = np.linalg.norm((pa[k] - pb[k]).ravel()) / (np.linalg.norm(pa[k].ravel()) + 1e-6)
        assert d <= 1e-3, (k, d)
        assert np.max(np.abs(pa[k] - pb[k])) <= 40 * 2 * 1e-3, k
    b.pool_clear()
    assert b.pool_size() == 0
    a.close()
    b.close()
