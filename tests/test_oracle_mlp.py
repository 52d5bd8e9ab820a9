"""Pins of the step-proposer oracle (oracle/mlp.py) against things other than itself:
bfloat16 rounding (closed-form tie cases and torch's bfloat16 conversion), GELU (its
closed form at special points and torch's exact-erf GELU), the analytic gradient
(central finite differences with the roundings switched off), the loss at z = 0
(log 2), and AdamW (its closed-form first step and torch.optim.AdamW)."""
import math

import numpy as np
import pytest

from oracle import mlp


def test_bf16_ties_to_even():
    x = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -7, -(1 + 2 ** -8), 3.0e-39, 0.0])
    want = np.array([1.0, 1.0, 1 + 2 ** -6, 1 + 2 ** -7, -1.0, None, 0.0], dtype=object)
    got = mlp.bf16(x)
    for g, w in zip(got, want):
        if w is not None:
            assert g == w


def test_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(0).normal(size=10000).astype(np.float32) * 10.0 ** np.random.default_rng(1).integers(-8, 8, 10000)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x), ref)


def test_gelu_special_points_and_torch():
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert abs(mlp.gelu(np.array([10.0]))[0] - 10.0) < 1e-20
    assert abs(mlp.gelu(np.array([-10.0]))[0]) < 1e-20
    # gelu(1) = Phi(1) = (1 + erf(1/sqrt2)) / 2
    assert abs(mlp.gelu(np.array([1.0]))[0] - 0.8413447460685429) < 1e-15
    torch = pytest.importorskip("torch")
    u = np.linspace(-6, 6, 1001)
    ref = torch.nn.functional.gelu(torch.from_numpy(u)).numpy()
    assert np.max(np.abs(mlp.gelu(u) - ref)) < 1e-14
    # the derivative against a central difference of gelu itself
    h = 1e-6
    fd = (mlp.gelu(u + h) - mlp.gelu(u - h)) / (2 * h)
    assert np.max(np.abs(mlp.gelu_prime(u) - fd)) < 1e-8


def test_loss_at_the_boundary_is_log2():
    p = mlp.init(3).astype(np.float64)
    X = np.random.default_rng(4).normal(size=(5, 12))
    m, _ = mlp.forward(p, X)
    for acc in (0, 1):
        assert abs(mlp.loss(p, X, m, np.full(5, acc), 4.0) - math.log(2.0)) < 1e-12


def test_gradient_matches_finite_differences(monkeypatch):
    """With the bfloat16 roundings replaced by the identity the loss is smooth, and the
    analytic gradient must equal central differences of the loss."""
    monkeypatch.setattr(mlp, "bf16", lambda v: np.asarray(v, dtype=np.float64))
    rng = np.random.default_rng(5)
    p = mlp.init(5).astype(np.float64) + rng.normal(0, 0.01, mlp.NPARAM)
    X = rng.normal(size=(16, 12))
    r = rng.normal(size=16)
    acc = rng.integers(0, 2, 16)
    g, _ = mlp.grad(p, X, r, acc, 4.0)
    idx = np.concatenate([rng.choice(768, 20, replace=False), 768 + np.arange(5),
                          832 + rng.choice(4096, 20, replace=False), 4928 + np.arange(5),
                          4992 + np.arange(5), [5056]])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (mlp.loss(p + e, X, r, acc, 4.0) - mlp.loss(p - e, X, r, acc, 4.0)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(g[i]), (i, fd, g[i])


def test_adamw_first_step_closed_form():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -0.2, 1e-3])
    p1, m1, m2 = mlp.adamw(p, np.zeros(3), np.zeros(3), g, 1, lr=0.01, wd=0.1, eps=1e-12)
    # bias-corrected moments are g and g^2 after one step, so the step is g / (|g| + eps)
    assert np.allclose(p1, p - 0.01 * (g / (np.abs(g) + 1e-12) + 0.1 * p), rtol=0, atol=1e-15)
    assert np.allclose(m1, 0.1 * g) and np.allclose(m2, 0.001 * g * g)


def test_adamw_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(6)
    p = rng.normal(size=50)
    tp = torch.tensor(p.copy(), requires_grad=True)
    opt = torch.optim.AdamW([tp], lr=1e-3, betas=(0.9, 0.999), eps=1e-8, weight_decay=1e-4)
    m1 = np.zeros(50)
    m2 = np.zeros(50)
    q = p.copy()
    for step in range(1, 6):
        g = rng.normal(size=50)
        tp.grad = torch.tensor(g)
        opt.step()
        q, m1, m2 = mlp.adamw(q, m1, m2, g, step, lr=1e-3, wd=1e-4)
    # torch applies the decay before the moment update: p <- p (1 - lr wd); the two
    # orders differ by lr^2 terms only
    assert np.max(np.abs(q - tp.detach().numpy())) < 1e-8
