"""GPU parity: the CUDA library against the FP64 oracle, through the C ABI.

Tolerances: geometry, boundary links, candidate links and chosen contact-line links bit-exact;
FP64 fields to 1e-9 of rho_l after hundreds of steps; FP32 fields max|drho| <= 1e-4 rho_l after
the 200 x 120 workload's 3000 steps; contact angles within 0.5 degrees on independently evolved
fields and within 1e-6 degrees on identical fields.
"""
import numpy as np
import pytest

from helpers import gpu_lattice, oracle_config, tanh_drop
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


def _cfg(O, w=None, **over):
    return oracle_config(O, w or W.plain_small(), **over)[0]


# --------------------------------------------------------------------------------- geometry
@pytest.mark.parametrize("case", ["cyl", "stripes", "flat", "halfint", "wrap", "concave",
                                  "concave_wrap"])
def test_geometry_bit_exact(lbm, oracle_mod, case):
    O = oracle_mod
    over = {}
    if case == "stripes":
        over = dict(stripes=1, stripe_arc=7.0, mu_stripe_b=0.5)
    if case == "flat":
        over = dict(has_circle=0)
    if case == "halfint":
        over = dict(nx=77, ny=53, cx=38.5, cy=-0.5, R=20.5, drop_x=38.5, drop_y=40, drop_r=8)
    if case == "wrap":
        over = dict(nx=40, ny=30, cx=2.0, cy=3.0, R=9.0, drop_x=20, drop_y=22, drop_r=5)
    if case == "concave":
        over = dict(nx=96, ny=70, cx=48.0, cy=40.5, R=38.0, concave=1, stripes=1, stripe_arc=7.0,
                    mu_stripe_b=0.5, drop_x=48, drop_y=12, drop_r=10)
    if case == "concave_wrap":
        over = dict(nx=60, ny=50, cx=1.5, cy=26.0, R=32.5, concave=1, drop_x=1.5, drop_y=10,
                    drop_r=6)
    cfg = _cfg(O, **over)
    ref = O.Sim(cfg)
    lat = gpu_lattice(lbm, cfg)
    flags, muw, links = lat.geometry()
    _, _, oflag, omuw = ref.ext()
    assert np.array_equal(flags, oflag)
    assert np.array_equal(muw.astype(np.float32), omuw.astype(np.float32))
    assert np.array_equal(links, ref.links())
    assert lat.info().n_fluid == int((oflag[2:-2] == 0).sum())


# -------------------------------------------------------------------------------- time steps
@pytest.mark.parametrize("tile", [(32, 8), (32, 16)])
def test_fp64_matches_oracle(lbm, oracle_mod, tile):
    """FP64 kernel vs FP64 oracle: same arithmetic up to operation order."""
    O = oracle_mod
    cfg = _cfg(O, nx=77, ny=53, cx=38.5, R=20.0, drop_x=38.5, drop_y=20.5 + 14, drop_r=14,
               gy=-1e-5)
    ref = O.Sim(cfg)
    lat = gpu_lattice(lbm, cfg, precision=1, tile=tile)
    for n in (1, 9, 290):
        ref.step(n)
        lat.step(n)
        err = np.abs(lat.rho() - ref.rho()).max() / cfg.rho_l
        assert err < 1e-9, (n, err)
    ux, uy = lat.velocity()
    oux, ouy, _, _ = ref.velocity_force()
    # the oracle reports the velocity of the state before its last step; step once more
    ref2 = O.Sim(cfg)
    ref2.step(301)
    oux, ouy, _, _ = ref2.velocity_force()
    assert np.abs(ux - oux).max() < 1e-9
    assert np.abs(uy - ouy).max() < 1e-9


@pytest.mark.parametrize("tile", [(32, 8), (32, 16), (64, 16), (32, 32), (32, 16, 5), (32, 8, 6),
                                  (32, 16, 6)])
def test_fp32_matches_oracle_ragged(lbm, oracle_mod, tile):
    """FP32 path on a domain that is not a multiple of any tile (ragged tails in x and y)."""
    O = oracle_mod
    cfg = _cfg(O, nx=77, ny=53, cx=38.5, R=20.0, drop_x=38.5, drop_y=20.5 + 14, drop_r=14)
    ref = O.Sim(cfg)
    ref.step(500)
    lat = gpu_lattice(lbm, cfg, tile=tile[:2], min_blocks=tile[2] if len(tile) > 2 else 0)
    lat.step(500)
    err = np.abs(lat.rho() - ref.rho()).max() / cfg.rho_l
    assert err < 2e-5, err


def test_fp32_plain_workload_3000_steps(lbm, oracle_mod):
    """The 200 x 120 workload (cylinder R = 40, drop r = 25, neutral walls): after 3000 steps
    max |drho| <= 1e-4 rho_l, mass conserved, angles within 0.5 degrees of the oracle's."""
    O = oracle_mod
    cfg = _cfg(O)
    ref = O.Sim(cfg)
    ref.step(3000)
    lat = gpu_lattice(lbm, cfg)
    m0 = lat.mass()["mass"]
    lat.step(3000)
    rho, oref = lat.rho(), ref.rho()
    err = np.abs(rho - oref).max() / cfg.rho_l
    gas = oref < 0.5 * (cfg.rho_g + cfg.rho_l)
    gas_err = np.abs(rho - oref)[gas & (oref > 0)].max() / cfg.rho_g
    print(f"max |drho|/rho_l = {err:.3e}, gas max rel = {gas_err:.3e}")
    assert err <= 1e-4
    m1 = lat.mass()["mass"]
    assert abs(m1 - m0) / m0 < 1e-5
    gl, gr = lat.measure()
    ol, orr, _ = ref.measure()
    assert gl.status == 0 and gr.status == 0
    assert abs(gl.theta - ol.theta) <= 0.5 and abs(gr.theta - orr.theta) <= 0.5


def test_fp64_plain_workload(lbm, oracle_mod):
    """FP64 variant of the 200 x 120 workload, 1000 steps: agreement to 1e-9 of rho_l."""
    O = oracle_mod
    cfg = _cfg(O)
    ref = O.Sim(cfg)
    ref.step(1000)
    lat = gpu_lattice(lbm, cfg, precision=1)
    lat.step(1000)
    assert np.abs(lat.rho() - ref.rho()).max() / cfg.rho_l < 1e-9


def test_small_periodic_domain(lbm, oracle_mod):
    """nx = 8 (the tile and its halo wrap the periodic axis several times)."""
    O = oracle_mod
    mx = O.maxwell(0, 0.7)
    nx, ny = 8, 40
    j = np.arange(ny)[:, None] * np.ones((1, nx))
    rho0 = mx["rho_g"] + (mx["rho_l"] - mx["rho_g"]) * 0.5 * (np.tanh((j - 12) / 2.) -
                                                              np.tanh((j - 28) / 2.))
    cfg = _cfg(O, nx=nx, ny=ny, has_circle=0)
    ref = O.Sim(cfg, rho0)
    ref.step(400)
    lat = gpu_lattice(lbm, cfg, precision=1, rho0=rho0)
    lat.step(400)
    assert np.abs(lat.rho() - ref.rho()).max() / cfg.rho_l < 1e-9


def test_graph_chunks_equal_single_launches(lbm, oracle_mod):
    """Steps replayed from the captured graphs (64, 32, ..., 2 steps from either buffer) equal
    steps launched one by one (bitwise), for step counts that use every graph size and both
    starting buffers."""
    O = oracle_mod
    cfg = _cfg(O, nx=96, ny=64, cx=48, R=20, drop_x=48, drop_y=34.5, drop_r=14)
    a = gpu_lattice(lbm, cfg)
    b = gpu_lattice(lbm, cfg)
    total = 0
    for n in (128 + 3, 37, 126, 1, 20, 63):  # 64+64+2+1, 32+4+1, 64+32+16+8+4+2, 1, 16+4, ...
        a.step(n)
        total += n
        for _ in range(n):
            b.step(1)
        assert np.array_equal(a.rho(), b.rho()), n
    assert a.info().steps == b.info().steps == total


def test_new_geometry_on_a_used_context(lbm, oracle_mod):
    """A context that has stepped (and captured its step graphs) and then gets a new geometry,
    with the same or the interpolated boundary scheme, steps bit for bit like a fresh context
    given that geometry."""
    O = oracle_mod
    first = _cfg(O, nx=96, ny=64, cx=48, R=20, drop_x=48, drop_y=34.5, drop_r=14)
    second = _cfg(O, nx=96, ny=64, cx=40, R=16, drop_x=40, drop_y=16.5 + 12, drop_r=12)
    lat = gpu_lattice(lbm, first)
    lat.step(70)
    for cfg in (second, first):
        for interp in (0, 1):
            cfg.interp_bb = interp
            lat.set_geometry(circle=(cfg.cx, cfg.cy, cfg.R), mu_circle=cfg.mu_circle,
                             mu_bottom=cfg.mu_bottom, mu_top=cfg.mu_top,
                             drop=(cfg.drop_x, cfg.drop_y, cfg.drop_r, cfg.drop_W),
                             boundary=interp)
            fresh = gpu_lattice(lbm, cfg)
            lat.step(75)
            fresh.step(75)
            assert np.array_equal(lat.rho(), fresh.rho()), (cfg.cx, interp)
            fresh.close()
        cfg.interp_bb = 0
    lat.close()


@pytest.mark.parametrize("interp", [0, 1])
def test_same_walls_new_state_on_a_used_context(lbm, oracle_mod, interp):
    """lbm_set_geometry with the walls unchanged (only the drop, or a host rho0) keeps the walls
    on the device and resets the state: the context then steps bit for bit like a fresh one given
    that geometry and start, and its node classes and wall potentials are unchanged; a change of
    one wall field (the wall potential) afterwards rebuilds the walls."""
    O = oracle_mod
    cfg = _cfg(O, nx=96, ny=64, cx=48, R=20, drop_x=48, drop_y=34.5, drop_r=14)
    cfg.interp_bb = interp
    walls = dict(circle=(cfg.cx, cfg.cy, cfg.R), mu_circle=cfg.mu_circle, mu_bottom=cfg.mu_bottom,
                 mu_top=cfg.mu_top, boundary=interp)
    lat = gpu_lattice(lbm, cfg)
    lat.step(60)
    flags0, muw0, _ = lat.geometry()
    # a new drop on the same walls
    cfg.drop_x, cfg.drop_r = 40.0, 12.0
    lat.set_geometry(**walls, drop=(cfg.drop_x, cfg.drop_y, cfg.drop_r, cfg.drop_W))
    flags1, muw1, _ = lat.geometry()
    assert np.array_equal(flags0, flags1) and np.array_equal(muw0, muw1)
    fresh = gpu_lattice(lbm, cfg)
    lat.step(75)
    fresh.step(75)
    assert np.array_equal(lat.rho(), fresh.rho())
    # a host density field on the same walls
    rho0 = fresh.rho()
    lat.set_geometry(**walls, drop=(cfg.drop_x, cfg.drop_y, cfg.drop_r, cfg.drop_W), rho0=rho0)
    fresh.set_geometry(**walls, drop=(cfg.drop_x, cfg.drop_y, cfg.drop_r, cfg.drop_W), rho0=rho0)
    lat.step(40)
    fresh.step(40)
    assert np.array_equal(lat.rho(), fresh.rho())
    fresh.close()
    # one wall field changed: the walls are rebuilt
    cfg.mu_circle = cfg.mu_circle + 0.02
    walls["mu_circle"] = cfg.mu_circle
    lat.set_geometry(**walls, drop=(cfg.drop_x, cfg.drop_y, cfg.drop_r, cfg.drop_W))
    fresh = gpu_lattice(lbm, cfg)
    assert not np.array_equal(lat.geometry()[1], muw0)
    assert np.array_equal(lat.geometry()[1], fresh.geometry()[1])
    lat.step(50)
    fresh.step(50)
    assert np.array_equal(lat.rho(), fresh.rho())
    fresh.close()
    lat.close()


def _concave_cfg(O):
    """Drop started as a near-hemispherical cap at the bottom of a circular cavity (Fig. 2b) of
    radius 60 in a 160 x 100 domain (cut by the top wall), on a hydrophilic wall."""
    cfg, mx, neutral = oracle_config(O, W.plain_small(), nx=160, ny=100, cx=80.0, cy=66.0,
                                     R=60.0, concave=1, drop_x=80.0, drop_y=8.0, drop_r=24.0)
    cfg.mu_circle = neutral + W.mu_rel_for_angle(70.0)
    return cfg


@pytest.mark.parametrize("precision,tol", [(0, 3e-5), (1, 1e-9)])
def test_concave_cavity_matches_oracle(lbm, oracle_mod, precision, tol):
    """Concave substrate: density after 800 steps against the oracle, then the angles measured
    on the independently evolved fields within 0.5 degrees (left line at smaller x)."""
    O = oracle_mod
    cfg = _concave_cfg(O)
    ref = O.Sim(cfg)
    ref.step(800)
    lat = gpu_lattice(lbm, cfg, precision=precision)
    lat.step(800)
    err = np.abs(lat.rho() - ref.rho()).max() / cfg.rho_l
    assert err < tol, err
    gl, gr = lat.measure()
    ol, orr, _ = ref.measure()
    assert gl.status == gr.status == ol.status == orr.status == 0
    assert abs(gl.theta - ol.theta) <= 0.5 and abs(gr.theta - orr.theta) <= 0.5
    assert gl.contact[0] < gr.contact[0]
    assert gl.beta == pytest.approx(gl.theta - gl.alpha)


def test_concave_measure_identical_field_bit_exact(lbm, oracle_mod):
    """On the same FP32-rounded field in a cavity: candidate links, points and distances bit for
    bit, the same contact-line links and the same angles."""
    O = oracle_mod
    mx = O.maxwell(0, 0.7)
    rg, rl = mx["rho_g"], mx["rho_l"]
    for (R, cy, r, yc, dx) in [(60.0, 66.0, 22.0, 8.3, 0.4), (70.5, 75.0, 30.0, 10.0, -1.3)]:
        nx, ny = 170, 100
        rho = tanh_drop(nx, ny, 85.0 + dx, yc, r, rg, rl, 5.0).astype(np.float32).astype(np.float64)
        cfg = _cfg(O, nx=nx, ny=ny, cx=85.0, cy=cy, R=R, concave=1)
        lat = gpu_lattice(lbm, cfg, rho0=rho)
        ids, pd = lat.candidates()
        oids, opd = O.candidates(cfg, rho, 0.5 * (rg + rl))
        assert np.array_equal(ids, oids)
        assert np.array_equal(pd, opd)
        gl, gr = lat.measure()
        ol, orr, _ = O.measure(cfg, rho, 0.5 * (rg + rl))
        for g, o in ((gl, ol), (gr, orr)):
            assert g.status == o.status == 0
            assert (g.link1, g.link2) == (o.link1, o.link2)
            assert g.d1 == o.d1 and g.d2 == o.d2
            assert g.theta == pytest.approx(o.theta, abs=1e-6)
            assert g.beta == pytest.approx(o.beta, abs=1e-6)


def _ibb_cfg(O, **over):
    """Drop on a cylinder (or in a cavity) with the interpolated, mass-corrected bounce-back."""
    cfg, mx, neutral = oracle_config(O, W.plain_small(), nx=96, ny=64, cx=48.0, R=20.5,
                                     drop_x=48.3, drop_y=20.5 + 13.0, drop_r=14.0, interp_bb=1,
                                     stripes=1, stripe_arc=6.0)
    cfg.mu_stripe_b = neutral + 0.02
    for k, v in over.items():
        setattr(cfg, k, v)
    return cfg


@pytest.mark.parametrize("concave,precision,tol", [(0, 1, 1e-9), (0, 0, 3e-5), (1, 1, 1e-9),
                                                   (1, 0, 3e-5)])
def test_interp_bb_matches_oracle(lbm, oracle_mod, concave, precision, tol):
    """Interpolated bounce-back (link fractions from the analytic wall, mass correction) on a
    striped cylinder and in a cavity: density against the oracle after 600 steps, the mass
    conserved, and the angles on the independently evolved fields within 0.5 degrees."""
    O = oracle_mod
    over = dict(concave=concave)
    if concave:
        over.update(cx=48.0, cy=40.0, R=37.0, drop_x=48.3, drop_y=9.0, drop_r=14.0)
    cfg = _ibb_cfg(O, **over)
    ref = O.Sim(cfg)
    ref.step(600)
    lat = gpu_lattice(lbm, cfg, precision=precision)
    m0 = lat.mass()["mass"]
    lat.step(600)
    err = np.abs(lat.rho() - ref.rho()).max() / cfg.rho_l
    assert err < tol, err
    assert abs(lat.mass()["mass"] - m0) / m0 < (1e-12 if precision else 1e-6)
    gl, gr = lat.measure()
    ol, orr, _ = ref.measure()
    assert gl.status == gr.status == ol.status == orr.status == 0
    assert abs(gl.theta - ol.theta) <= 0.5 and abs(gr.theta - orr.theta) <= 0.5


def test_interp_bb_flat_walls_equal_halfway(lbm, oracle_mod):
    """Flat walls only: every link fraction is 1/2 and the interpolated run equals the half-way
    run bit for bit on the GPU too."""
    O = oracle_mod
    cfg = _ibb_cfg(O, has_circle=0, stripes=0, drop_y=10.0)
    a = gpu_lattice(lbm, cfg)
    cfg.interp_bb = 0
    b = gpu_lattice(lbm, cfg)
    a.step(500)
    b.step(500)
    assert np.array_equal(a.rho(), b.rho())


def test_interp_bb_measure_identical_field(lbm, oracle_mod):
    """With interpolated bounce-back the measurement keeps the wall surface R + 1/2: candidate
    points, distances and chosen links bit for bit on an identical field."""
    O = oracle_mod
    mx = O.maxwell(0, 0.7)
    rg, rl = mx["rho_g"], mx["rho_l"]
    nx, ny = 200, 120
    rho = tanh_drop(nx, ny, 100.4, 58.0, 25.0, rg, rl, 5.0).astype(np.float32).astype(np.float64)
    cfg = _cfg(O, nx=nx, ny=ny, cx=100.0, R=40.0, interp_bb=1)
    lat = gpu_lattice(lbm, cfg, rho0=rho)
    ids, pd = lat.candidates()
    oids, opd = O.candidates(cfg, rho, 0.5 * (rg + rl))
    assert np.array_equal(ids, oids) and np.array_equal(pd, opd)
    gl, gr = lat.measure()
    ol, orr, _ = O.measure(cfg, rho, 0.5 * (rg + rl))
    for g, o in ((gl, ol), (gr, orr)):
        assert (g.link1, g.link2) == (o.link1, o.link2)
        assert g.theta == pytest.approx(o.theta, abs=1e-6)
        assert np.hypot(g.contact[0] - 100.0, g.contact[1]) == pytest.approx(40.5, abs=1e-9)


def test_interp_bb_rejected_in_batches(lbm, oracle_mod):
    b = lbm.Batch([(64, 48)], Tr=0.7)
    with pytest.raises(lbm.LbmError):
        b.set_geometry(0, circle=(32.0, 0.0, 10.0), drop=(32.0, 20.0, 6.0, 5.6),
                       boundary=lbm.LBM_BB_INTERP)
    b.close()


# ------------------------------------------------------------------------------ measurement
def test_measure_identical_field_bit_exact(lbm, oracle_mod):
    """On the same (FP32-rounded) density field the GPU finds the same liquid/gas links, points
    and distances bit for bit, picks the same contact-line links and the same angles."""
    O = oracle_mod
    mx = O.maxwell(0, 0.7)
    rg, rl = mx["rho_g"], mx["rho_l"]
    for k, (R, r, yc, dx) in enumerate([(40.0, 25.0, 58.3, 0.3), (30.5, 18.0, 38.0, -1.2),
                                        (45.0, 30.0, 75.0, 0.0)]):
        nx, ny = 200, 120
        rho = tanh_drop(nx, ny, 100.0 + dx, yc, r, rg, rl, 5.0).astype(np.float32).astype(np.float64)
        cfg = _cfg(O, nx=nx, ny=ny, cx=100.0, R=R)
        lat = gpu_lattice(lbm, cfg, rho0=rho)
        ids, pd = lat.candidates()
        oids, opd = O.candidates(cfg, rho, 0.5 * (rg + rl))
        assert np.array_equal(ids, oids)
        assert np.array_equal(pd, opd)
        gl, gr = lat.measure()
        ol, orr, _ = O.measure(cfg, rho, 0.5 * (rg + rl))
        for g, o in ((gl, ol), (gr, orr)):
            assert g.status == o.status == 0
            assert (g.link1, g.link2) == (o.link1, o.link2)
            assert g.d1 == o.d1 and g.d2 == o.d2
            assert g.theta == pytest.approx(o.theta, abs=1e-6)
            assert g.alpha == pytest.approx(o.alpha, abs=1e-6)
            assert g.contact[0] == pytest.approx(o.contact[0], abs=1e-9)


def test_measure_flat_wall(lbm, oracle_mod):
    O = oracle_mod
    mx = O.maxwell(0, 0.7)
    rg, rl = mx["rho_g"], mx["rho_l"]
    nx, ny = 160, 80
    rho = tanh_drop(nx, ny, 80.2, 8.0, 30.0, rg, rl, 6.0).astype(np.float32).astype(np.float64)
    cfg = _cfg(O, nx=nx, ny=ny, has_circle=0)
    lat = gpu_lattice(lbm, cfg, rho0=rho)
    gl, gr = lat.measure()
    ol, orr, _ = O.measure(cfg, rho, 0.5 * (rg + rl))
    assert (gl.link1, gl.link2, gr.link1, gr.link2) == (ol.link1, ol.link2, orr.link1, orr.link2)
    assert gl.theta == pytest.approx(ol.theta, abs=1e-6)
    assert gr.theta == pytest.approx(orr.theta, abs=1e-6)


def test_measure_no_contact(lbm, oracle_mod):
    """A drop far from the substrate has no interface points in the band: NO_CONTACT status."""
    O = oracle_mod
    cfg = _cfg(O, drop_y=95.0, drop_r=12.0)
    lat = gpu_lattice(lbm, cfg)
    st, (l, r) = lbm.lbm_measure_contact_angle(lat.ctx)
    assert st == lbm.LBM_ERR_NO_CONTACT
    assert l.status == lbm.LBM_ERR_NO_CONTACT and r.status == lbm.LBM_ERR_NO_CONTACT


# ---------------------------------------------------------------------------- full size
def test_full_size_sampled(lbm, oracle_mod):
    """2048 x 1024 (cylinder R = 300, drop r = 150, sessile body force), bench launch config:
    50 FP32 steps vs the oracle on every node, mass to FP32 round-off."""
    O = oracle_mod
    w = W.plain_large(0)
    cfg = oracle_config(O, w)[0]
    ref = O.Sim(cfg)
    ref.step(50)
    lat = gpu_lattice(lbm, cfg)
    m0 = lat.mass()["mass"]
    lat.step(50)
    err = np.abs(lat.rho() - ref.rho()).max() / cfg.rho_l
    assert err < 2e-5, err
    m1 = lat.mass()["mass"]
    assert abs(m1 - m0) / m0 < 1e-6


@pytest.mark.parametrize("heterogeneous", [True, False])
def test_hysteresis_full_size(lbm, oracle_mod, heterogeneous):
    """4096 x 1024 hysteresis workload (cylinder R = 800, 40-lu stripes of 60 and 120 degrees or
    uniform 120 degrees, tangential body force), bench launch config: wall chemical potentials
    bit-exact in FP32, 50 FP32 steps vs the oracle on every node."""
    O = oracle_mod
    w = W.hysteresis(heterogeneous)
    cfg = oracle_config(O, w)[0]
    ref = O.Sim(cfg)
    lat = gpu_lattice(lbm, cfg, tile=(lbm.LBM_TILE_AUTO, 0))
    flags, muw, links = lat.geometry()
    _, _, oflag, omuw = ref.ext()
    assert np.array_equal(flags, oflag)
    assert np.array_equal(muw.astype(np.float32), omuw.astype(np.float32))
    ref.step(50)
    lat.step(50)
    err = np.abs(lat.rho() - ref.rho()).max() / cfg.rho_l
    assert err < 2e-5, err


def test_stream_from_torch(lbm, oracle_mod):
    """The library runs on a caller's torch stream."""
    import torch
    O = oracle_mod
    cfg = _cfg(O, nx=96, ny=64, cx=48, R=20, drop_x=48, drop_y=34.5, drop_r=14)
    s = torch.cuda.Stream()
    a = gpu_lattice(lbm, cfg, stream=s)
    b = gpu_lattice(lbm, cfg)
    a.step(100)
    b.step(100)
    assert np.array_equal(a.rho(), b.rho())
    # device-pointer read into torch tensors
    r = torch.zeros(64 * 96, dtype=torch.float64, device="cuda")
    lbm.lbm_read_fields(a.ctx, lbm.LBM_FIELD_RHO, 96, 64, device_out=(r.data_ptr(), None, None))
    torch.cuda.synchronize()
    assert np.array_equal(r.cpu().numpy().reshape(64, 96), a.rho())
    # caller-owned (pinned) host destination
    pinned = torch.zeros((64, 96), dtype=torch.float64, pin_memory=True).numpy()
    got = a.rho(out=pinned)
    assert got is pinned and np.array_equal(pinned, a.rho())
    with pytest.raises(ValueError):
        a.rho(out=np.zeros((64, 96), dtype=np.float32))


# -------------------------------------------------------------------- other model options
def test_carnahan_starling_bgk_matches_oracle(lbm, oracle_mod):
    """Second EOS (Carnahan-Starling, Tr = 0.7) with the BGK collision of Eq. 3."""
    O = oracle_mod
    mx = O.maxwell(1, 0.7)
    k2 = 0.05
    neutral = k2 * mx["mu_sat"]
    cfg = O.Config(nx=96, ny=64, eos=1, collision=1, Tr=0.7, k2=k2, kappa=0.05, tau=1.0,
                   rho_g=mx["rho_g"], rho_l=mx["rho_l"], has_circle=1, cx=48, cy=0, R=20,
                   mu_circle=neutral, mu_bottom=neutral, mu_top=neutral, drop_x=48,
                   drop_y=20.5 + 14, drop_r=14, drop_W=4.0)
    ref = O.Sim(cfg)
    ref.step(300)
    assert np.isfinite(ref.rho()).all()
    for prec, tol in ((1, 1e-9), (0, 2e-5)):
        lat = gpu_lattice(lbm, cfg, precision=prec)
        lat.step(300)
        err = np.abs(lat.rho() - ref.rho()).max() / cfg.rho_l
        assert err < tol, (prec, err)


def test_carnahan_starling_mrt_200x120_3000_steps(lbm, oracle_mod):
    """The 200 x 120 cylinder workload with the Carnahan-Starling EOS (Tr = 0.7) and the MRT
    collision of Eq. 1, 3000 steps: FP32 within 1e-4 of rho_l and FP64 within 1e-9 of rho_l of
    the oracle, mass conserved, both contact angles within 0.5 degrees of the oracle's."""
    O = oracle_mod
    cfg = oracle_config(O, W.plain_small_cs())[0]
    assert cfg.eos == 1 and cfg.collision == 0
    ref = O.Sim(cfg)
    ref.step(3000)
    oref = ref.rho()
    assert np.isfinite(oref).all()
    ol, orr, _ = ref.measure()
    assert ol.status == 0 and orr.status == 0
    for prec, tol in ((0, 1e-4), (1, 1e-9)):
        lat = gpu_lattice(lbm, cfg, precision=prec)
        m0 = lat.mass()["mass"]
        lat.step(3000)
        err = np.abs(lat.rho() - oref).max() / cfg.rho_l
        print(f"precision {prec}: max |drho|/rho_l = {err:.3e}")
        assert err <= tol, (prec, err)
        assert abs(lat.mass()["mass"] - m0) / m0 < (1e-5 if prec == 0 else 1e-12)
        gl, gr = lat.measure()
        assert gl.status == 0 and gr.status == 0
        assert abs(gl.theta - ol.theta) <= 0.5 and abs(gr.theta - orr.theta) <= 0.5
        lat.close()


def test_striped_wetting_and_pendent_gravity(lbm, oracle_mod):
    """Heterogeneous (striped) circle wetting with a body force pulling the drop away from the
    cylinder (pendent arrangement), FP32 vs oracle, 1500 steps."""
    O = oracle_mod
    w = W.Workload("stripes", 160, 110, (80.0, 0.0, 35.0), W.tangent_drop(80, 0, 35, 20),
                   mu_rel_circle=-0.02, stripes=(9.0, 0.03), g=(2e-6, 5e-6))
    cfg = oracle_config(O, w)[0]
    ref = O.Sim(cfg)
    ref.step(1500)
    lat = gpu_lattice(lbm, cfg)
    flags, muw, _ = lat.geometry()
    _, _, _, omuw = ref.ext()
    assert np.array_equal(muw.astype(np.float32), omuw.astype(np.float32))
    lat.step(1500)
    err = np.abs(lat.rho() - ref.rho()).max() / cfg.rho_l
    assert err < 3e-5, err
    gl, gr = lat.measure()
    ol, orr, _ = ref.measure()
    assert abs(gl.theta - ol.theta) <= 0.5 and abs(gr.theta - orr.theta) <= 0.5


@pytest.mark.parametrize("precision,tol", [(0, 3e-5), (1, 1e-9)])
def test_buoyant_body_force_along_periodic_axis(lbm, oracle_mod, precision, tol):
    """Body force (rho - rho_g) g with g along the periodic x axis (plus a normal component) on
    a striped cylinder: density and the reported velocity v = u + F / 2 rho against the oracle
    after 1000 steps, so the reference density enters both the stepping and the force output."""
    O = oracle_mod
    w = W.Workload("buoyant", 160, 110, (80.0, 0.0, 35.0), W.tangent_drop(80, 0, 35, 20),
                   mu_rel_circle=0.02, stripes=(9.0, -0.03), g=(2e-5, -1e-5), buoyant=True)
    cfg = oracle_config(O, w)[0]
    assert cfg.g_rho_ref == cfg.rho_g > 0
    ref = O.Sim(cfg)
    ref.step(1000)
    lat = gpu_lattice(lbm, cfg, precision=precision)
    lat.step(1000)
    err = np.abs(lat.rho() - ref.rho()).max() / cfg.rho_l
    assert err < tol, err
    # the oracle reports the velocity of the state before its last step: step it once more
    ref.step(1)
    oux, ouy, _, _ = ref.velocity_force()
    ux, uy = lat.velocity()
    fluid = ref.ext()[2][2:-2] == 0
    umax = max(np.abs(oux[fluid]).max(), np.abs(ouy[fluid]).max())
    assert umax > 1e-5
    du = max(np.abs(ux - oux)[fluid].max(), np.abs(uy - ouy)[fluid].max())
    assert du < (1e-2 * umax if precision == 0 else 1e-9), (du, umax)


@pytest.mark.parametrize("precision,tol", [(0, 1e-5), (1, 1e-12)])
def test_uniform_coexistence_state_stays_uniform(lbm, oracle_mod, precision, tol):
    """Degenerate case: a uniform liquid at the coexistence density next to neutral walls is an
    exact equilibrium; after 500 steps the density stays uniform to round-off and no flow
    appears."""
    O = oracle_mod
    cfg, mx, _ = oracle_config(O, W.plain_small(), nx=64, ny=48, cx=32.0, R=12.0)
    rho0 = np.full((cfg.ny, cfg.nx), mx["rho_l"])
    lat = gpu_lattice(lbm, cfg, precision=precision, rho0=rho0)
    lat.step(500)
    flags = lat.geometry()[0][2:-2]
    r = lat.rho()[flags == 0]
    assert np.abs(r - mx["rho_l"]).max() / mx["rho_l"] < tol
    ux, uy = lat.velocity()
    assert max(np.abs(ux[flags == 0]).max(), np.abs(uy[flags == 0]).max()) < tol
