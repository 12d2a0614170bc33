"""GPU parity of the warm-start surrogate: the tensor-core GEMM against FP64 products of the
same BF16 operands, and the U-Net's forward pass, loss and every gradient against the FP64
oracle (oracle/surrogate.py) on the same BF16-rounded inputs and weights."""
import numpy as np
import pytest

from paper_2202_06516_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2202_06516_gb300 import lbm
    return torch, lbm


@pytest.mark.parametrize("ak,bk", [(1, 1), (1, 0), (0, 0), (0, 1)])
@pytest.mark.parametrize("M,N,K", [(128, 128, 32), (200, 72, 136), (8, 256, 1000), (520, 40, 8)])
def test_gemm_layouts(env, ak, bk, M, N, K):
    torch, lbm = env
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(K, N, generator=g).to(torch.bfloat16)
    want = A.double() @ B.double()
    Ad = (A if ak else A.t()).contiguous().cuda()   # K-major = row-major A; MN-major = A^T rows
    Bd = (B.t() if bk else B).contiguous().cuda()
    lda = K if ak else M
    ldb = K if bk else N
    Cd = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    lbm.lbm_sg_gemm(Ad.data_ptr(), Bd.data_ptr(), M, N, K, ak, bk, lda, ldb, Cd.data_ptr(), N)
    torch.cuda.synchronize()
    got = Cd.double().cpu()
    err = (got - want).abs().max().item() / max(1.0, want.abs().max().item())
    assert err < 2e-6, err


@pytest.mark.parametrize("M,N,K", [(1000, 32, 288), (4096, 64, 576), (1024, 256, 2304),
                                   (384, 300, 72), (129, 130, 64), (640, 512, 1152)])
def test_gemm_tensor_core_shapes(env, M, N, K):
    """K-major x K-major products run on the tcgen05 kernel: every N-tile width (32, 64, 128,
    256), several M and N tiles, K tails inside a 64-wide slice, against FP64 products."""
    torch, lbm = env
    g = torch.Generator().manual_seed(M + 11 * N + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    Bt = torch.randn(N, K, generator=g).to(torch.bfloat16)
    want = A.double() @ Bt.double().t()
    Ad, Bd = A.cuda(), Bt.cuda()   # kept alive until the asynchronous GEMM has run
    Cd = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    lbm.lbm_sg_gemm(Ad.data_ptr(), Bd.data_ptr(), M, N, K, 1, 1, K, K, Cd.data_ptr(), N)
    torch.cuda.synchronize()
    err = (Cd.double().cpu() - want).abs().max().item() / max(1.0, want.abs().max().item())
    # the products of BF16 operands are exact in FP32; the FP32 sum of K of them drifts like a
    # random walk, ~sqrt(K) u of the largest output (u = 2^-24), a few times that at the maximum
    assert err < max(2e-6, 2e-7 * np.sqrt(K)), err


@pytest.mark.parametrize("ak,bk", [(0, 0), (1, 0), (0, 1)])
@pytest.mark.parametrize("M,N,K", [(256, 576, 4096), (32, 288, 20000), (1000, 80, 200)])
def test_gemm_tensor_core_mn_major(env, ak, bk, M, N, K):
    """MN-major operands (the weight gradient's layout, K = pixels) on the tcgen05 kernel:
    several 64-wide swizzle blocks along M and N, partial blocks, long and ragged K."""
    torch, lbm = env
    g = torch.Generator().manual_seed(3 * M + N + 7 * K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(K, N, generator=g).to(torch.bfloat16)
    want = A.double() @ B.double()
    Ad = (A if ak else A.t()).contiguous().cuda()
    Bd = (B.t() if bk else B).contiguous().cuda()
    Cd = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    lbm.lbm_sg_gemm(Ad.data_ptr(), Bd.data_ptr(), M, N, K, ak, bk, K if ak else M,
                    K if bk else N, Cd.data_ptr(), N)
    torch.cuda.synchronize()
    err = (Cd.double().cpu() - want).abs().max().item() / max(1.0, want.abs().max().item())
    assert err < max(2e-6, 2e-7 * np.sqrt(K)), err


def _case(seed=0, B=2, H=32, Wd=32, base=8):
    rng = np.random.default_rng(seed)
    x = np.zeros((B, H, Wd, 8), dtype=np.float32)
    x[..., 0] = rng.uniform(size=(B, H, Wd)) > 0.7
    x[..., 1] = rng.normal(0, 0.5, size=(B, H, Wd))
    x[..., 2] = 0.3
    target = rng.uniform(0, 1, size=(B, H, Wd)).astype(np.float32)
    mask = (x[..., 0] == 0).astype(np.uint8)
    p = W.unet_init(base, seed)
    p = p + rng.normal(0, 0.02, size=p.size).astype(np.float32)
    return x, target, mask, p


def _bf16(a):
    import torch
    return torch.tensor(a).to(torch.bfloat16).double().numpy()


def _gpu_and_oracle(env, x, t, m, p, base, H, Wd=None):
    """One GPU training step without update (gradients only) and the oracle on the same BF16
    inputs and weights the GPU used (convolution weights rounded to BF16; biases and the head
    stay FP32, as in the GPU epilogue and head), in three modes: FP64 throughout, BF16
    activations, and BF16 activations plus BF16 pre-activation gradients (the two tensors the
    GPU stores in BF16)."""
    torch, lbm = env
    from oracle import surrogate as S
    s = lbm.Surrogate(H, Wd or H, base=base, max_batch=2)
    assert s.n == p.size
    s.set_weights(p)
    nb = x.shape[0]
    xd = torch.tensor(x).to(torch.bfloat16).cuda()
    td = torch.tensor(t).cuda()
    md = torch.tensor(m).cuda()
    loss = s.train_step(xd.data_ptr(), td.data_ptr(), md.data_ptr(), nb, 0.0)
    gpu = dict(loss=loss, g=s.weights(grads=True).astype(np.float64), phi=s.phi(nb))
    s.close()
    pw = _bf16(p)
    convs, n = S.layer_specs(base)
    o = 0
    for ci, co, _ in convs:
        o += co * 9 * ci
        pw[o:o + co] = p[o:o + co]
        o += co
    pw[o:] = p[o:]
    xb, tt, mb = _bf16(x), t.astype(np.float64), m.astype(bool)
    ref = {}
    for mode, flags in (("fp64", (False, False)), ("act", (True, False)), ("full", (True, True))):
        l, g, phi = S.loss_and_grad(pw, xb, tt, mb, base, *flags)
        ref[mode] = dict(loss=l, g=g, phi=phi)
    return gpu, ref, pw, xb


def _layers(base):
    """(weight slice, bias slice) of every convolution and the head slice."""
    from oracle import surrogate as S
    convs, _ = S.layer_specs(base)
    out, o = [], 0
    for ci, co, _ in convs:
        out.append((slice(o, o + co * 9 * ci), slice(o + co * 9 * ci, o + co * 9 * ci + co)))
        o += co * 9 * ci + co
    return out, slice(o, o + base + 1)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _cos(a, b):
    return (a @ b) / (np.linalg.norm(a) * np.linalg.norm(b))


CASES = [(8, 32), (8, 48), (16, 64), (32, 64)]  # base, resolution (48: not a power of two)


def _fp32_yardstick(pw, xb, t, m, base):
    """The oracle's BF16-storage network evaluated in FP32 on the CPU (same BF16 inputs and
    weights): how far FP32 arithmetic alone moves the gradients from the FP64 evaluation."""
    import torch
    from oracle import surrogate as S
    pt = torch.tensor(pw.astype(np.float32), requires_grad=True)
    loss, _ = S.loss_fn(pt, torch.tensor(xb.astype(np.float32)), torch.tensor(t),
                        torch.tensor(m.astype(bool)), base, True, True)
    loss.backward()
    return pt.grad.double().numpy()


@pytest.mark.parametrize("regime", ["positive", "negative"])
@pytest.mark.parametrize("base,H", CASES)
def test_gradients_match_bf16_oracle_per_layer(env, base, H, regime):
    _per_layer_check(env, base, H, regime)


def test_tma_fed_levels_at_full_resolution(env):
    """256 x 256, base 32, one image: the 128 x 128 (64 channels), 64 x 64 and 32 x 32 levels
    feed their forward and data-gradient GEMMs with tensor-map (TMA) boxes, the 128 x 128 level
    with single-row boxes of 128 pixels; the per-layer check of
    test_gradients_match_bf16_oracle_per_layer at that size."""
    _per_layer_check(env, 32, 256, "positive", B=1)


@pytest.mark.parametrize("B", [1, 2])
def test_tma_fed_levels_on_a_rectangular_lattice(env, B):
    """128 rows x 256 columns, base 32, one or two images: tiles of whole rows (or half rows) of
    a non-square image through every tensor-map path (forward, data and weight gradients, the
    upsampling layers' even/odd orders, the staged windows of the weight gradient and of the
    32-channel forward and data gradient); with two images the fourth (image) coordinate of
    the boxes and the zero fill at each image's top and bottom rows; the per-layer check of
    test_gradients_match_bf16_oracle_per_layer."""
    _per_layer_check(env, 32, 128, "positive", B=B, Wd=256)


def _per_layer_check(env, base, H, regime, B=2, Wd=None):
    """Every layer's weight and bias gradient against the oracle that stores activations and
    pre-activation gradients in BF16 as the GPU does, with weights chosen so that every
    pre-activation keeps one sign with a wide margin (positive: weights x 0.1, biases +1;
    negative: weights x 0.25, biases -1; margin checked in the oracle). Away from the leaky-ReLU
    kink the differences left are FP32 against FP64 accumulation and the BF16 rounding decisions
    they move, amplified through the 17 layers. The same oracle evaluated in FP32 on the CPU
    shows that amplification: it departs from the FP64 evaluation by up to 1.1e-2 per layer in
    these regimes, with the same per-layer profile as the GPU. So each layer must be within the
    1e-2 relative bound for BF16 gradients, or, where FP32 arithmetic itself does not reach that
    bound, within twice the FP32 evaluation's own departure; 1.5e-2 caps both (measured GPU
    worst 1.25e-2 with the FP32 evaluation at 1.08e-2 on that layer's case). The forward pass
    agrees to ~1e-7 and the head gradient to 1e-4. The oracle without the gradient rounding is
    farther from the GPU, so that mode is what the GPU computes."""
    torch, _ = env
    from oracle import surrogate as S
    x, t, m, p = _case(base=base, H=H, Wd=Wd or H, B=B)
    scale, bias = (0.1, 1.0) if regime == "positive" else (0.25, -1.0)
    p = p.copy()
    layers, head = _layers(base)
    for sw, sb in layers:
        p[sw] *= scale
        p[sb] = bias
    gpu, ref, pw, xb = _gpu_and_oracle(env, x, t, m, p, base, H, Wd)
    rec = []
    S.forward(torch.tensor(pw), torch.tensor(xb), base, bf16_activations=True, record=rec)
    margin = min(float(z.abs().min()) for z in rec)
    assert margin > 0.3 and all(((z > 0).all() if bias > 0 else (z < 0).all()) for z in rec)
    full = ref["full"]
    assert np.abs(gpu["phi"] - full["phi"]).max() < 5e-4
    assert gpu["loss"] == pytest.approx(full["loss"], rel=1e-5)
    assert _rel(gpu["g"][head], full["g"][head]) < 1e-3
    g32 = _fp32_yardstick(pw, xb, t, m, base)
    errs = []
    for k, (sw, sb) in enumerate(layers):
        ew, eb = _rel(gpu["g"][sw], full["g"][sw]), _rel(gpu["g"][sb], full["g"][sb])
        yard = max(_rel(g32[sw], full["g"][sw]), _rel(g32[sb], full["g"][sb]))
        errs.append(max(ew, eb))
        assert max(ew, eb) < min(1.5e-2, max(1e-2, 2.0 * yard)), (k, ew, eb, yard)
    act_only = [max(_rel(gpu["g"][sw], ref["act"]["g"][sw]), _rel(gpu["g"][sb], ref["act"]["g"][sb]))
                for sw, sb in layers]
    assert sum(errs) < sum(act_only)
    print(f"{regime} base {base} H {H}: worst layer {max(errs):.2e} (activation-only oracle "
          f"{max(act_only):.2e})")


@pytest.mark.parametrize("base,H", CASES)
def test_forward_loss_gradients_match_oracle_random_init(env, base, H):
    """Seeded initial weights (pre-activations of both signs). Forward and loss within BF16
    storage of the oracle; gradients: the leaky-ReLU slope switches between 1 and 0.1 at zero,
    and pre-activations within a BF16 rounding step of zero flip with any FP32-level change of
    the inputs (the oracle's own per-layer gradients move by 3-12 % when its weights move by a
    relative 6e-8, see the oracle tests), so here the per-layer check is on direction: cosine > 0.99
    (0.96 at base 32) against the BF16 oracle, > 0.999 (0.99) for the whole gradient."""
    x, t, m, p = _case(base=base, H=H, Wd=H)
    gpu, ref, _, _ = _gpu_and_oracle(env, x, t, m, p, base, H)
    wide = base >= 32
    assert np.abs(gpu["phi"] - ref["fp64"]["phi"]).max() < 2e-2
    assert gpu["loss"] == pytest.approx(ref["fp64"]["loss"], rel=3e-2)
    full = ref["full"]
    assert np.abs(gpu["phi"] - full["phi"]).max() < 1e-3
    assert gpu["loss"] == pytest.approx(full["loss"], rel=1e-4)
    assert _cos(gpu["g"], full["g"]) > (0.99 if wide else 0.999)
    layers, head = _layers(base)
    for k, (sw, sb) in enumerate(layers):
        assert _cos(gpu["g"][sw], full["g"][sw]) > (0.96 if wide else 0.99), k
        assert _cos(gpu["g"][sb], full["g"][sb]) > (0.96 if wide else 0.99), k
    assert _rel(gpu["g"][head], full["g"][head]) < 2e-2


def test_training_reduces_loss(env):
    torch, lbm = env
    x, t, m, p = _case(seed=3, H=32, Wd=32, base=8)
    s = lbm.Surrogate(32, 32, base=8, max_batch=2)
    s.set_weights(p)
    xd = torch.tensor(x).to(torch.bfloat16).cuda()
    td = torch.tensor(t).cuda()
    md = torch.tensor(m).cuda()
    losses = [s.train_step(xd.data_ptr(), td.data_ptr(), md.data_ptr(), 2, 3e-3) for _ in range(60)]
    assert losses[-1] < 0.7 * losses[0]
    s.close()


def test_training_reduces_loss_at_bench_size(env):
    """The warm-start configuration itself (base 32, 256 x 256, batch 8): Adam at lr 1e-3 on one
    fixed batch of drop-like targets (phi in {0, 1}, ~6 % liquid) lowers the loss."""
    torch, lbm = env
    rng = np.random.default_rng(5)
    B, H = 8, 256
    x = np.zeros((B, H, H, 8), dtype=np.float32)
    j, i = np.mgrid[0:H, 0:H]
    t = np.zeros((B, H, H), dtype=np.float32)
    for b in range(B):
        cx, cy, r = rng.uniform(80, 176), rng.uniform(60, 120), rng.uniform(20, 45)
        t[b] = ((i - cx) ** 2 + (j - cy) ** 2 < r * r).astype(np.float32)
        x[b, ..., 0] = (j < 40).astype(np.float32)
        x[b, ..., 2] = (t[b].sum() / H / H)
    m = (x[..., 0] == 0).astype(np.uint8)
    s = lbm.Surrogate(H, H, base=32, max_batch=B)
    s.set_weights(W.unet_init(32, seed=0))
    xd = torch.tensor(x).to(torch.bfloat16).cuda()
    td = torch.tensor(t).cuda()
    md = torch.tensor(m).cuda()
    losses = [s.train_step(xd.data_ptr(), td.data_ptr(), md.data_ptr(), B, 1e-3)
              for _ in range(40)]
    print(losses[0], losses[9], losses[-1])
    assert losses[-1] < 0.5 * losses[0]
    s.close()
