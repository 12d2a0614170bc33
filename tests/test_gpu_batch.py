"""GPU tests of the batched sweep engine (lbm_batch_*): uneven instances advanced by one
persistent kernel must equal independent single-lattice runs bit for bit (same device code and
tile variant), agree with the oracle, and leave the table when converged."""
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


CASES = [  # nx, ny, circle (cx, cy, R), drop r, mu_rel
    (96, 64, (48.0, 0.0, 20.0), 14.0, 0.0),
    (130, 70, (65.0, 0.0, 30.5), 16.0, -0.01),
    (77, 53, (38.5, 0.0, 20.0), 12.0, 0.012),
    (160, 96, (80.0, 0.0, 45.0), 22.0, 0.005),
]


def _cfgs(O):
    out = []
    for nx, ny, circ, r, mu_rel in CASES:
        w = W.Workload("t", nx, ny, circ, W.tangent_drop(circ[0], circ[1], circ[2], r),
                       mu_rel_circle=mu_rel)
        out.append(oracle_config(O, w)[0])
    # a drop at the bottom of a circular cavity (concave substrate)
    out.append(oracle_config(O, W.sweep_instance(40.0, 14.0, 100.0, True))[0])
    return out


def _batch(lbm, cfgs):
    c0 = cfgs[0]
    b = lbm.Batch([(c.nx, c.ny) for c in cfgs], eos=c0.eos, Tr=c0.Tr, k2=c0.k2, kappa=c0.kappa,
                  tau=c0.tau, s_e=c0.s_e, s_eps=c0.s_eps, s_q=c0.s_q, rho_g=c0.rho_g,
                  rho_l=c0.rho_l)
    for i, c in enumerate(cfgs):
        b.set_geometry(i, circle=(c.cx, c.cy, c.R), mu_circle=c.mu_circle, mu_bottom=c.mu_bottom,
                       mu_top=c.mu_top, drop=(c.drop_x, c.drop_y, c.drop_r, c.drop_W),
                       concave=bool(c.concave))
    return b


def test_batch_equals_single_lattices(lbm, oracle_mod):
    cfgs = _cfgs(oracle_mod)
    b = _batch(lbm, cfgs)
    steps, conv, res = b.run(600, check_every=200, tol=0.0)
    assert (steps == 600).all() and not conv.any()
    for i, c in enumerate(cfgs):
        single = gpu_lattice(lbm, c)
        single.step(600)
        assert np.array_equal(b.rho(i), single.rho()), i
        ref = oracle_mod.Sim(c)
        ref.step(600)
        assert np.abs(b.rho(i) - ref.rho()).max() / c.rho_l < 2e-5
    ang = b.measure()
    for i, c in enumerate(cfgs):
        single = gpu_lattice(lbm, c)
        single.step(600)
        l, r = single.measure()
        assert ang[i][0].theta == l.theta and ang[i][1].theta == r.theta
    b.close()


def test_batch_early_exit(lbm, oracle_mod):
    """Instances leave the table when their residual drops below tol; each stops exactly at a
    check and its state equals a single-lattice run of that many steps."""
    cfgs = _cfgs(oracle_mod)
    b = _batch(lbm, cfgs)
    steps, conv, res = b.run(6000, check_every=500, tol=2e-4)
    assert (steps % 500 == 0).all()
    assert conv.any()
    for i in np.nonzero(conv)[0]:
        assert res[i] < 2e-4
    for i in np.nonzero(~conv.astype(bool))[0]:
        assert steps[i] == 6000
    i = int(np.nonzero(conv)[0][0])
    single = gpu_lattice(lbm, cfgs[i])
    single.step(int(steps[i]))
    assert np.array_equal(b.rho(i), single.rho())
    b.close()


def test_batch_mass_conserved(lbm, oracle_mod):
    cfgs = _cfgs(oracle_mod)
    b = _batch(lbm, cfgs)
    m0 = [b.mass(i)["mass"] for i in range(len(cfgs))]
    b.run(1000, check_every=500, tol=0.0)
    for i in range(len(cfgs)):
        assert abs(b.mass(i)["mass"] - m0[i]) / m0[i] < 1e-5
    b.close()


def test_batch_angle_convergence(lbm, oracle_mod):
    """With an angle criterion an instance stops at the first check where both angles moved by
    <= 0.05 degrees since the previous check, for the second check in a row. Replaying the same
    instance alone and measuring at its last three checks shows exactly that, and its final
    state equals the batch's. (The criterion is a stopping rule: a contact line pinned on the
    staircase wall can hold still for two checks and move again later.)"""
    cfgs = _cfgs(oracle_mod)
    b = _batch(lbm, cfgs)
    steps, conv, res = b.run(20000, check_every=500, tol=0.0, angle_tol=0.05)
    assert conv.any()
    ang = b.measure()
    for i in np.nonzero(conv)[0]:
        s = int(steps[i])
        assert 1500 <= s < 20000 and s % 500 == 0
        single = gpu_lattice(lbm, cfgs[i])
        single.step(s - 1000)
        t0 = single.measure()
        single.step(500)
        t1 = single.measure()
        single.step(500)
        t2 = single.measure()
        for side in (0, 1):
            assert abs(t1[side].theta - t0[side].theta) <= 0.05
            assert abs(t2[side].theta - t1[side].theta) <= 0.05
            assert t2[side].theta == ang[i][side].theta
        assert np.array_equal(single.rho(), b.rho(i))
    b.close()
