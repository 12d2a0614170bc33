"""GPU parity of the FP64 reductions (mass, liquid-node count, liquid centroid) against the oracle,
and the failure paths that report an unstable or timed-out run, through the C ABI.

The centroid decides which side of the drop each interface point belongs to (Sec. 3.2, Fig. 1),
so it is compared with the oracle's own centroid (the one its measurement uses) on the same
FP32 field; the mass is compared with the oracle's mass of a lattice started from that field.
Failures are made on the host: a non-finite or non-positive density is written into a host
initial field, and the tensor-core timeout flag is latched by the host hook; nothing faults,
traps or stalls a GPU.
"""
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


def _tilted_cfg(O):
    """A drop pushed sideways on a striped cylinder, so the centroid is off every symmetry axis."""
    w = W.Workload("tilted", 160, 110, (80.0, 0.0, 35.0), W.tangent_drop(80, 0, 35, 20),
                   mu_rel_circle=-0.02, stripes=(9.0, 0.03), g=(4e-6, -2e-6))
    return oracle_config(O, w)[0]


def _oracle_sums(O, cfg, rho):
    """Mass, liquid count and centroid of a field the way the oracle defines them: the oracle's
    total mass of a lattice started from the field (populations summed over fluid nodes) and the
    liquid centroid its contact-angle measurement uses; the count is the number of fluid nodes
    with rho > rho_m."""
    rho_m = 0.5 * (cfg.rho_g + cfg.rho_l)
    sim = O.Sim(cfg, rho0=rho)
    _, _, flag, _ = sim.ext()
    fluid = flag[2:-2] == 0
    _, _, cen = O.measure(cfg, rho, rho_m)
    return sim.mass(), int((fluid & (rho > rho_m)).sum()), cen


@pytest.mark.parametrize("source", ["oracle_field", "gpu_field"])
def test_mass_and_centroid_match_oracle(lbm, oracle_mod, source):
    """lbm_mass against the oracle on identical FP32 densities: mass to 1e-12 (both sum FP64
    values, in different orders), liquid count exactly, centroid to 1e-12."""
    O = oracle_mod
    cfg = _tilted_cfg(O)
    if source == "oracle_field":
        ref = O.Sim(cfg)
        ref.step(1200)
        rho = ref.rho().astype(np.float32).astype(np.float64)
        lat = gpu_lattice(lbm, cfg, rho0=rho)
    else:
        lat = gpu_lattice(lbm, cfg)
        lat.step(1200)
        rho = lat.rho()  # the FP32 density plane, widened exactly
    got = lat.mass()
    mass, n_liq, cen = _oracle_sums(O, cfg, rho)
    assert n_liq > 100
    assert abs(cen[0] - cfg.cx) > 1.0  # the drop has moved off the axis
    assert got["mass"] == pytest.approx(mass, rel=1e-12, abs=0)
    assert got["n_liquid"] == n_liq
    assert got["cx"] == pytest.approx(cen[0], rel=1e-12, abs=0)
    assert got["cy"] == pytest.approx(cen[1], rel=1e-12, abs=0)
    lat.close()


def test_fp64_lattice_mass_matches_oracle_every_step_count(lbm, oracle_mod):
    """FP64 lattice evolved beside the oracle: the device mass sum equals the oracle's mass
    (conserved to round-off on both sides) and the liquid centroids agree to 1e-9 lu."""
    O = oracle_mod
    cfg = _tilted_cfg(O)
    ref = O.Sim(cfg)
    lat = gpu_lattice(lbm, cfg, precision=1)
    rho_m = 0.5 * (cfg.rho_g + cfg.rho_l)
    for n in (0, 300, 700):
        ref.step(n)
        lat.step(n)
        got = lat.mass()
        assert got["mass"] == pytest.approx(ref.mass(), rel=1e-12, abs=0)
        _, _, cen = O.measure(cfg, ref.rho(), rho_m)
        assert abs(got["cx"] - cen[0]) < 1e-9 and abs(got["cy"] - cen[1]) < 1e-9
    lat.close()


@pytest.mark.parametrize("bad", [np.nan, np.inf, -0.25, 0.0])
def test_unstable_density_is_reported(lbm, oracle_mod, bad):
    """A non-finite or non-positive density at one fluid node makes lbm_mass return
    LBM_ERR_UNSTABLE (with the sums of the other nodes still written); a clean field does not."""
    O = oracle_mod
    cfg = oracle_config(O, W.plain_small())[0]
    ref = O.Sim(cfg)
    rho = ref.rho()
    lat = gpu_lattice(lbm, cfg, rho0=rho)
    st, _ = lbm.lbm_mass(lat.ctx, allow_unstable=True)
    assert st == lbm.LBM_OK
    j, i = 100, 17  # a gas node far from the drop and the walls
    bad_rho = rho.copy()
    bad_rho[j, i] = bad
    lat.set_geometry(circle=(cfg.cx, cfg.cy, cfg.R), mu_circle=cfg.mu_circle,
                     mu_bottom=cfg.mu_bottom, mu_top=cfg.mu_top, rho0=bad_rho)
    st, out = lbm.lbm_mass(lat.ctx, allow_unstable=True)
    assert st == lbm.LBM_ERR_UNSTABLE
    assert "non-finite or non-positive" in lbm.lbm_last_error(lat.ctx)
    if np.isfinite(bad):
        fluid = lat.geometry()[0][2:-2] == 0
        assert out["mass"] == pytest.approx(float(bad_rho.astype(np.float32)[fluid].astype(
            np.float64).sum()), rel=1e-12)
    with pytest.raises(lbm.LbmError) as e:
        lat.mass()
    assert e.value.status == lbm.LBM_ERR_UNSTABLE
    lat.close()


def test_batch_isolates_an_unstable_instance(lbm, oracle_mod):
    """An instance started with a NaN density leaves the batched sweep at its first check
    (reported as not converged) while the others run on, bit-identical to their separate runs."""
    O = oracle_mod
    cfgs = []
    for nx, ny, circ, r in [(96, 64, (48.0, 0.0, 20.0), 14.0), (77, 53, (38.5, 0.0, 20.0), 12.0),
                            (130, 70, (65.0, 0.0, 30.5), 16.0)]:
        w = W.Workload("t", nx, ny, circ, W.tangent_drop(circ[0], circ[1], circ[2], r))
        cfgs.append(oracle_config(O, w)[0])
    c0 = cfgs[0]
    b = lbm.Batch([(c.nx, c.ny) for c in cfgs], eos=c0.eos, Tr=c0.Tr, k2=c0.k2, kappa=c0.kappa,
                  tau=c0.tau, s_e=c0.s_e, s_eps=c0.s_eps, s_q=c0.s_q, rho_g=c0.rho_g,
                  rho_l=c0.rho_l)
    bad = 1
    for i, c in enumerate(cfgs):
        rho0 = None
        if i == bad:
            rho0 = O.Sim(c).rho()
            rho0[c.ny - 5, 3] = np.nan
        b.set_geometry(i, circle=(c.cx, c.cy, c.R), mu_circle=c.mu_circle,
                       mu_bottom=c.mu_bottom, mu_top=c.mu_top,
                       drop=(c.drop_x, c.drop_y, c.drop_r, c.drop_W), rho0=rho0)
    steps, conv, res = b.run(1000, check_every=200, tol=0.0)
    assert steps[bad] == 200 and conv[bad] == 0
    for i, c in enumerate(cfgs):
        if i == bad:
            continue
        assert steps[i] == 1000
        single = gpu_lattice(lbm, c)
        single.step(1000)
        assert np.array_equal(b.rho(i), single.rho()), i
        single.close()
    st, _ = lbm.lbm_mass(lbm.lbm_batch_instance(b.b, bad), allow_unstable=True)
    assert st == lbm.LBM_ERR_UNSTABLE
    b.close()


def test_latched_timeout_is_reported_once(lbm):
    """The tensor-core timeout flag, latched from the host as an expired device wait would latch
    it, turns the next surrogate call into LBM_ERR_TIMEOUT; the call after that succeeds."""
    import torch
    s = lbm.Surrogate(32, 32, base=8, max_batch=1)
    rng = np.random.default_rng(3)
    s.set_weights((0.05 * rng.standard_normal(s.n)).astype(np.float32))
    x = torch.zeros((1, 32, 32, 8), dtype=torch.bfloat16, device="cuda")
    phi = torch.zeros((1, 32, 32), dtype=torch.float32, device="cuda")
    s.forward(x.data_ptr(), 1, phi.data_ptr())
    lbm.lbm_sg_inject_timeout()
    with pytest.raises(lbm.LbmError) as e:
        s.forward(x.data_ptr(), 1, phi.data_ptr())
    assert e.value.status == lbm.LBM_ERR_TIMEOUT
    assert "timed out" in str(e.value)
    s.forward(x.data_ptr(), 1, phi.data_ptr())  # reported once, then cleared
    lbm.lbm_sg_inject_timeout()
    a = torch.zeros((128, 64), dtype=torch.bfloat16, device="cuda")
    c = torch.zeros((128, 128), dtype=torch.float32, device="cuda")
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_sg_gemm(a.data_ptr(), a.data_ptr(), 128, 128, 64, 1, 1, 64, 64, c.data_ptr(), 128)
    assert e.value.status == lbm.LBM_ERR_TIMEOUT
    s.close()
