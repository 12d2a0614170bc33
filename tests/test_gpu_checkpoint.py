"""Checkpoint and restart through the C ABI: a lattice restored from lbm_save_state into a fresh
context with the same geometry continues bit for bit like the uninterrupted run; malformed or
mismatched checkpoints are refused without touching the context."""
import numpy as np
import pytest

from helpers import gpu_lattice, oracle_config
from paper_2202_06516_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2202_06516_gb300 import lbm as L
    L.lib()
    return L


def _cfg(O, interp=False):
    w = W.Workload("ckpt", 160, 110, (80.0, 0.0, 35.0), W.tangent_drop(80, 0, 35, 20),
                   mu_rel_circle=-0.02, stripes=(9.0, 0.03), g=(2e-6, -3e-6))
    cfg = oracle_config(O, w)[0]
    if interp:
        cfg.interp_bb = 1
    return cfg


@pytest.mark.parametrize("precision,interp", [(0, False), (1, False), (0, True)])
def test_restart_is_bit_identical(lbm, oracle_mod, precision, interp):
    cfg = _cfg(oracle_mod, interp)
    a = gpu_lattice(lbm, cfg, precision=precision)
    a.step(301)  # odd: the current buffer is the second one
    data = lbm.lbm_save_state(a.ctx)
    assert len(data) == lbm.lib().lbm_state_bytes(a.ctx)
    a.step(199)
    b = gpu_lattice(lbm, cfg, precision=precision)
    b.step(7)  # some other state first; the checkpoint replaces it
    lbm.lbm_load_state(b.ctx, data)
    assert b.info().steps == 301
    b.step(199)
    assert b.info().steps == a.info().steps == 500
    assert np.array_equal(a.rho(), b.rho())
    for u, v in zip(a.velocity(), b.velocity()):
        assert np.array_equal(u, v)
    la, ra = a.measure()
    lb, rb = b.measure()
    assert la.theta == lb.theta and ra.theta == rb.theta
    a.close()
    b.close()


def test_bad_checkpoints_are_refused(lbm, oracle_mod):
    cfg = _cfg(oracle_mod)
    a = gpu_lattice(lbm, cfg)
    a.step(50)
    data = lbm.lbm_save_state(a.ctx)
    rho = a.rho()
    # before lbm_set_geometry
    fresh = lbm.Lattice(cfg.nx, cfg.ny, eos=cfg.eos, Tr=cfg.Tr, k2=cfg.k2, kappa=cfg.kappa,
                        rho_g=cfg.rho_g, rho_l=cfg.rho_l)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_load_state(fresh.ctx, data)
    assert e.value.status == lbm.LBM_ERR_STATE
    fresh.close()
    # truncated, corrupted, other size, other precision
    bad = [data[:-4], b"\0" * 8 + data[8:]]
    other = gpu_lattice(lbm, oracle_config(oracle_mod, W.plain_small())[0])
    bad.append(lbm.lbm_save_state(other.ctx))
    other.close()
    wide = gpu_lattice(lbm, cfg, precision=1)
    bad.append(lbm.lbm_save_state(wide.ctx))
    wide.close()
    for blob in bad:
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_load_state(a.ctx, blob)
        assert e.value.status == lbm.LBM_ERR_ARG
    assert np.array_equal(a.rho(), rho)  # refused loads leave the state alone
    assert a.info().steps == 50
    a.close()
