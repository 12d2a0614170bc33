"""FP64 CPU oracle of the warm-start U-Net (TEST INFRASTRUCTURE ONLY).

Plain PyTorch CPU operations in float64 (conv2d, average pooling, nearest upsampling, autograd
for gradients); the CUDA library's BF16 network is checked against it. It defines the network
independently from the library: the same specification, written with library primitives.

Specification (shared reading, not shared code): input NHWC with 8 channels (mask, wetting map,
volume plane, five zero channels); levels with base, 2 base, 4 base, 8 base channels; per level
two 3x3 convolutions (padding 1) with leaky ReLU (slope 0.1); 2x2 average pooling between
encoder levels; in the
decoder each level starts with a 3x3 convolution of the 2x nearest-upsampled coarser output,
then two 3x3 convolutions on [that result | encoder skip] (channel concatenation in that order);
a 1x1 head with a sigmoid. Parameters are one flat FP32 vector: for every convolution in
forward order its weight laid out [c_out][ky][kx][c_in] followed by its bias [c_out]; then the
head weight [base] and bias [1].

Parity unpinned by the paper (the paper has no network); pinned instead by finite differences
(tests/test_oracle_surrogate.py), in the exact FP64 mode and, to BF16 precision, in the mode that
rounds the pre-activation gradients.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F


def layer_specs(base: int):
    """(c_in, c_out) of the 3x3 convolutions in forward order, the parameter count, and a tag
    per convolution: 'plain', 'up' (input upsampled 2x) or 'cat' (input concatenated with the
    skip of the same level)."""
    b = base
    convs = [(8, b, "plain"), (b, b, "plain"),
             (b, 2 * b, "plain"), (2 * b, 2 * b, "plain"),
             (2 * b, 4 * b, "plain"), (4 * b, 4 * b, "plain"),
             (4 * b, 8 * b, "plain"), (8 * b, 8 * b, "plain"),
             (8 * b, 4 * b, "up"), (8 * b, 4 * b, "cat"), (4 * b, 4 * b, "plain"),
             (4 * b, 2 * b, "up"), (4 * b, 2 * b, "cat"), (2 * b, 2 * b, "plain"),
             (2 * b, b, "up"), (2 * b, b, "cat"), (b, b, "plain")]
    n = sum(co * 9 * ci + co for ci, co, _ in convs) + b + 1
    return convs, n


def unpack(params: torch.Tensor, base: int):
    convs, n = layer_specs(base)
    assert params.numel() == n
    out, o = [], 0
    for ci, co, _ in convs:
        w = params[o:o + co * 9 * ci].reshape(co, 3, 3, ci).permute(0, 3, 1, 2)
        o += co * 9 * ci
        bb = params[o:o + co]
        o += co
        out.append((w, bb))
    hw = params[o:o + base]
    hb = params[o + base:o + base + 1]
    return out, hw, hb


def _bf16_store(t: torch.Tensor) -> torch.Tensor:
    """The value a BF16 activation store keeps (round to nearest even), passed straight
    through in the backward pass: later layers consume the rounded value."""
    return t + (t.to(torch.bfloat16).to(t.dtype) - t).detach()


class _BF16GradStore(torch.autograd.Function):
    """Identity in the forward pass; in the backward pass the gradient that arrives is rounded to
    BF16 (round to nearest even), as when a BF16-storage network writes the gradient with respect
    to a convolution's pre-activation once and every consumer (the weight gradient, the bias
    gradient and the data gradient of that convolution) reads the rounded copy."""

    @staticmethod
    def forward(ctx, t):
        return t.clone()

    @staticmethod
    def backward(ctx, g):
        return g.to(torch.bfloat16).to(g.dtype)


def forward(params: torch.Tensor, x_nhwc: torch.Tensor, base: int,
            bf16_activations: bool = False, bf16_gradients: bool = False,
            record: list | None = None) -> torch.Tensor:
    """phi (B, H, W) for inputs (B, H, W, 8). bf16_activations: round every stored activation
    (convolution outputs and pooled maps) to BF16, the storage precision of the method's
    BF16-in / FP32-accumulate network. bf16_gradients: round the gradient with respect to every
    convolution's pre-activation (the output gradient times the leaky-ReLU slope) to BF16 before
    it reaches that convolution's weights, bias and input, the other tensor such a network
    stores in BF16. Arithmetic stays FP64 in both modes. record: if a list, every convolution's
    pre-activation (before the leaky ReLU) is appended to it, in forward order."""
    layers, hw, hb = unpack(params, base)
    x = x_nhwc.permute(0, 3, 1, 2)
    st = _bf16_store if bf16_activations else (lambda t: t)
    gst = _BF16GradStore.apply if bf16_gradients else (lambda t: t)

    def conv(t, k):
        z = F.conv2d(t, layers[k][0], layers[k][1], padding=1)
        if record is not None:
            record.append(z.detach())
        return st(F.leaky_relu(gst(z), 0.1))

    pool = lambda t: st(F.avg_pool2d(t, 2))
    s1 = conv(conv(x, 0), 1)
    s2 = conv(conv(pool(s1), 2), 3)
    s3 = conv(conv(pool(s2), 4), 5)
    bt = conv(conv(pool(s3), 6), 7)
    up = lambda t: F.interpolate(t, scale_factor=2, mode="nearest")
    u3 = conv(up(bt), 8)
    d3 = conv(conv(torch.cat([u3, s3], 1), 9), 10)
    u2 = conv(up(d3), 11)
    d2 = conv(conv(torch.cat([u2, s2], 1), 12), 13)
    u1 = conv(up(d2), 14)
    d1 = conv(conv(torch.cat([u1, s1], 1), 15), 16)
    z = torch.einsum("bchw,c->bhw", d1, hw) + hb
    return torch.sigmoid(z)


def loss_fn(params, x, target, mask, base, bf16_activations=False, bf16_gradients=False):
    phi = forward(params, x, base, bf16_activations, bf16_gradients)
    m = mask.to(phi.dtype)
    return ((phi - target) ** 2 * m).sum() / m.sum(), phi


def loss_and_grad(params: np.ndarray, x: np.ndarray, target: np.ndarray, mask: np.ndarray,
                  base: int, bf16_activations: bool = False, bf16_gradients: bool = False):
    """Masked mean squared error on phi and its gradient (FP64, numpy in and out)."""
    p = torch.tensor(params, dtype=torch.float64, requires_grad=True)
    xt = torch.tensor(x, dtype=torch.float64)
    tt = torch.tensor(target, dtype=torch.float64)
    mt = torch.tensor(mask)
    loss, phi = loss_fn(p, xt, tt, mt, base, bf16_activations, bf16_gradients)
    loss.backward()
    return float(loss.item()), p.grad.numpy().copy(), phi.detach().numpy()


def predict(params: np.ndarray, x: np.ndarray, base: int) -> np.ndarray:
    with torch.no_grad():
        return forward(torch.tensor(params, dtype=torch.float64),
                       torch.tensor(x, dtype=torch.float64), base).numpy()
