"""Pins for the surrogate oracle (CPU): gradients against central finite differences on a tiny
network, the parameter layout against the seeded initialiser, and the layer semantics against
hand-built cases."""
import numpy as np
import pytest
import torch

from paper_2202_06516_gb300 import workloads as W


def _tiny(seed=0, B=2, H=16, Wd=16, base=8):
    rng = np.random.default_rng(seed)
    x = np.zeros((B, H, Wd, 8))
    x[..., :3] = rng.uniform(0, 1, size=(B, H, Wd, 3))
    target = rng.uniform(0, 1, size=(B, H, Wd))
    mask = rng.uniform(size=(B, H, Wd)) > 0.3
    p = W.unet_init(base, seed).astype(np.float64)
    p[:] += rng.normal(0, 0.05, size=p.size)  # non-zero biases too
    return p, x, target, mask


def test_parameter_layout_matches_initialiser():
    from oracle import surrogate as S
    for base in (8, 32):
        _, n = S.layer_specs(base)
        assert n == W.unet_init(base, 0).size
        assert [(a, b) for a, b, _ in S.layer_specs(base)[0]] == W.unet_layers(base)


def test_gradient_finite_differences():
    """Autograd gradient of the masked MSE equals central differences on 60 random coordinates
    (every layer's weights and biases and the head are sampled)."""
    from oracle import surrogate as S
    p, x, t, m = _tiny()
    loss, g, _ = S.loss_and_grad(p, x, t, m, 8)
    rng = np.random.default_rng(1)
    convs, n = S.layer_specs(8)
    idx = list(rng.choice(n, size=40, replace=False)) + list(range(n - 9, n))
    o = 0
    for ci, co, _ in convs:  # one weight and one bias per layer
        idx.append(o + 5)
        o += co * 9 * ci
        idx.append(o + 1)
        o += co
    for k in idx:
        h = 1e-6 * max(1.0, abs(p[k]))
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        lp, _, _ = S.loss_and_grad(pp, x, t, m, 8)
        lm, _, _ = S.loss_and_grad(pm, x, t, m, 8)
        fd = (lp - lm) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-5, abs=1e-10), k


def test_layer_semantics():
    """Hand-built checks of the specification: zero convolution weights with unit biases make
    every activation 1 (leaky ReLU of a positive value), so the head sees a constant."""
    from oracle import surrogate as S
    base = 8
    convs, n = S.layer_specs(base)
    p = np.zeros(n)
    # all convolution weights zero, biases one: every activation is 1 after ReLU
    o = 0
    for ci, co, _ in convs:
        o += co * 9 * ci
        p[o:o + co] = 1.0
        o += co
    p[o:o + base] = 0.5
    p[o + base] = -1.0
    x = np.random.default_rng(0).uniform(size=(1, 16, 16, 8))
    phi = S.predict(p, x, base)
    assert np.allclose(phi, 1.0 / (1.0 + np.exp(-(0.5 * base - 1.0))))


def test_leaky_relu_slope():
    """Negative pre-activations pass with slope 0.1: zero weights and biases of -1 make every
    activation -0.1 at the first layer and the output a known constant."""
    from oracle import surrogate as S
    base = 8
    convs, n = S.layer_specs(base)
    p = np.zeros(n)
    o = 0
    ci, co, _ = convs[0]
    o += co * 9 * ci
    p[o:o + co] = -1.0   # first conv: output -0.1 everywhere
    o += co
    ci, co, _ = convs[1]
    # second conv: centre tap weight 1 on channel 0 only -> -0.1 -> leaky -> -0.01 (plus bias 0)
    w = np.zeros((co, 3, 3, ci))
    w[:, 1, 1, 0] = 1.0
    p[o:o + co * 9 * ci] = w.ravel()
    x = np.zeros((1, 16, 16, 8))
    import torch
    layers, _, _ = S.unpack(torch.tensor(p), base)
    t = torch.tensor(x).permute(0, 3, 1, 2)
    a0 = torch.nn.functional.leaky_relu(torch.nn.functional.conv2d(t, layers[0][0], layers[0][1], padding=1), 0.1)
    assert torch.allclose(a0, torch.full_like(a0, -0.1))
    a1 = torch.nn.functional.leaky_relu(torch.nn.functional.conv2d(a0, layers[1][0], layers[1][1], padding=1), 0.1)
    assert torch.allclose(a1[0, :, 5, 5], torch.full((8,), -0.01, dtype=torch.float64))
