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


def test_forward_matches_oracle():
    from paper_2406_08496_gb300 import Surrogate
    p = _params(3)
    s = Surrogate(batch=256, seed=0)
    s.set_params(p)
    X, Xp = _inputs(700, 4)  # three batches, the last one partial
    y = s.forward(X)
    ref = M.forward(_bf16_params(p), Xp, act_round=M.bf16_round)
    assert np.all(np.isfinite(y))
    assert np.max(np.abs(y - ref)) <= 0.02 * (np.abs(ref).max() + 1.0)
    rel = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    assert rel < 5e-3, rel


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
    """The epilogues' GELU and GELU' (normal CDF by Abramowitz and Stegun
    26.2.17, |error| < 7.5e-8) against the float64 closed forms, over the
    range the activations take and beyond: the bound plus a few float32
    roundings of each term."""
    import oracle.mlp as M
    from paper_2406_08496_gb300 import gelu_eval
    z = np.concatenate([np.linspace(-12.0, 12.0, 200001), np.random.default_rng(4).standard_normal(100000) * 3.0])
    z = z.astype(np.float32)
    g, dg = gelu_eval(z)
    z64 = z.astype(np.float64)
    ref_g, ref_dg = M.gelu(z64), M.gelu_grad(z64)
    # 7.5e-8 of the method plus float32 evaluation (fast reciprocal and
    # exponential, four fused multiply-adds, a few products): 5e-7 in Phi
    tol_g = 5e-7 * np.abs(z64) + 2e-7 * np.abs(ref_g) + 1e-30
    tol_dg = 6e-7 + 2e-7 * np.abs(z64)
    assert np.all(np.abs(g - ref_g) <= tol_g), float(np.max(np.abs(g - ref_g) / tol_g))
    assert np.all(np.abs(dg - ref_dg) <= tol_dg), float(np.max(np.abs(dg - ref_dg) / tol_dg))
