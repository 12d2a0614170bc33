"""GPU test of the learned warm start end to end on a small scale (128 x 128 cases, base-8
network): solver-generated equilibria train the network with the library's kernels, and on
held-out cases its prediction starts closer to the equilibrium than the Eq. 16 cap does."""
import numpy as np
import pytest

from paper_2202_06516_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_warm_start_beats_cold_start_on_held_out_cases():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2202_06516_gb300 import lbm, warmstart as WS
    train_cases = W.warm_cases(48, seed=11, size=128)
    test_cases = W.warm_cases(8, seed=99, size=128)
    x, t, m = WS.generate(train_cases, steps=6000)
    sur = lbm.Surrogate(128, 128, base=8, max_batch=8)
    sur.set_weights(W.unet_init(8, seed=0))
    losses, _ = WS.train(sur, x, t, m, epochs=30, batch=8, lr=2e-3)
    assert losses[-1] < 0.5 * losses[0]
    xe, te, me = WS.generate(test_cases, steps=6000)
    phi = WS.predict(sur, xe)
    # cold start: the Eq. 16 initial field of the same cases
    b, co, neutral = WS.make_batch(test_cases)
    cold = np.zeros_like(te)
    for i, w in enumerate(test_cases):
        ctx = lbm.lbm_batch_instance(b.b, i)
        rho = lbm.lbm_read_fields(ctx, lbm.LBM_FIELD_RHO, w.nx, w.ny)[0]
        cold[i] = np.clip((rho - co["rho_g"]) / (co["rho_l"] - co["rho_g"]), 0, 1)
    b.close()
    err_warm = np.sqrt((((phi - te) * me) ** 2).sum() / me.sum())
    err_cold = np.sqrt((((cold - te) * me) ** 2).sum() / me.sum())
    print(f"RMS phi error to equilibrium: warm {err_warm:.4f}, cold {err_cold:.4f}")
    assert err_warm < err_cold
    sur.close()
