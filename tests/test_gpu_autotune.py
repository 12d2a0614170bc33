"""GPU checks of the step-kernel autotuners: every compiled variant is timed, the fastest is kept,
and the trial launches leave the simulation state untouched."""
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


def _cfg(O, **over):
    return oracle_config(O, W.plain_small(), **over)[0]


def _batch(lbm, cfgs, tile_auto=False):
    c0 = cfgs[0]
    b = lbm.Batch([(c.nx, c.ny) for c in cfgs], eos=c0.eos, Tr=c0.Tr, k2=c0.k2, kappa=c0.kappa,
                  tau=c0.tau, s_e=c0.s_e, s_eps=c0.s_eps, s_q=c0.s_q, rho_g=c0.rho_g,
                  rho_l=c0.rho_l, tile_auto=tile_auto)
    for i, c in enumerate(cfgs):
        b.set_geometry(i, circle=(c.cx, c.cy, c.R), mu_circle=c.mu_circle, mu_bottom=c.mu_bottom,
                       mu_top=c.mu_top, drop=(c.drop_x, c.drop_y, c.drop_r, c.drop_W))
    return b


@pytest.mark.parametrize("precision,n_variants", [(0, 7), (1, 2)])
def test_autotune_keeps_state_and_picks_fastest(lbm, oracle_mod, precision, n_variants):
    O = oracle_mod
    cfg = _cfg(O, nx=96, ny=64, cx=48, R=20, drop_x=48, drop_y=34.5, drop_r=14)
    lat = gpu_lattice(lbm, cfg, precision=precision)
    lat.step(50)
    rho0 = lat.rho()
    res = lat.autotune(5)
    assert len(res) == n_variants
    assert all(r["us_per_step"] > 0 for r in res)
    assert np.array_equal(lat.rho(), rho0)          # no step was taken
    info = lat.info()
    assert info.steps == 50
    best = min(res, key=lambda r: r["us_per_step"])
    assert (info.tile_x, info.tile_y, info.min_blocks) == (*best["tile"], best["min_blocks"])
    # stepping on with the chosen variant still follows the oracle
    lat.step(150)
    ref = O.Sim(cfg)
    ref.step(200)
    tol = 1e-9 if precision else 2e-5
    assert np.abs(lat.rho() - ref.rho()).max() / cfg.rho_l < tol


def test_tile_auto_tunes_at_first_step(lbm, oracle_mod):
    O = oracle_mod
    cfg = _cfg(O, nx=96, ny=64, cx=48, R=20, drop_x=48, drop_y=34.5, drop_r=14)
    lat = gpu_lattice(lbm, cfg, tile=(lbm.LBM_TILE_AUTO, 0))
    lat.step(130)   # autotune, then two graph chunks and two single launches
    info = lat.info()
    assert info.steps == 130
    assert (info.tile_x, info.tile_y) in {(32, 8), (32, 16), (64, 16), (32, 32)}
    ref = O.Sim(cfg)
    ref.step(130)
    assert np.abs(lat.rho() - ref.rho()).max() / cfg.rho_l < 2e-5


def test_batch_autotune_keeps_state(lbm, oracle_mod):
    O = oracle_mod
    cfgs = [_cfg(O, nx=96, ny=64, cx=48, R=20, drop_x=48, drop_y=34.5, drop_r=14),
            _cfg(O, nx=77, ny=53, cx=38.5, R=20.0, drop_x=38.5, drop_y=34.5, drop_r=14),
            _cfg(O, nx=130, ny=90, cx=65, R=30, drop_x=65, drop_y=30.5 + 15, drop_r=15)]
    b = _batch(lbm, cfgs)
    b.run(200, check_every=100, tol=0.0)
    before = [b.rho(i) for i in range(len(cfgs))]
    res = b.autotune(5)
    tiles = [(32, 8), (32, 16), (64, 16), (32, 32)]
    assert [r["tile"] for r in res] == [t for t in tiles for _ in range(2)]
    assert [r["persistent"] for r in res] == [False, True] * 4
    assert all(r["us_per_step"] > 0 for r in res)
    for i in range(len(cfgs)):
        assert np.array_equal(b.rho(i), before[i])
    steps, _, _ = b.run(200, check_every=100, tol=0.0)
    assert (steps == 400).all()
    for i, c in enumerate(cfgs):
        ref = O.Sim(c)
        ref.step(400)
        assert np.abs(b.rho(i) - ref.rho()).max() / c.rho_l < 2e-5, i


def test_batch_tile_auto_runs(lbm, oracle_mod):
    O = oracle_mod
    c = _cfg(O, nx=96, ny=64, cx=48, R=20, drop_x=48, drop_y=34.5, drop_r=14)
    b = _batch(lbm, [c, c], tile_auto=True)
    steps, _, _ = b.run(300, check_every=100, tol=0.0)
    assert (steps == 300).all()
    ref = O.Sim(c)
    ref.step(300)
    for i in range(2):
        assert np.abs(b.rho(i) - ref.rho()).max() / c.rho_l < 2e-5
