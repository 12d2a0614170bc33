"""Pins for the oracle's lattice step, geometry and measurement (CPU only).

Checks against brute force, closed forms and conservation laws rather than against the oracle's
own formulas: geometry by an independent classification, the fourth-order stencils by exactness
on quartics, exact-difference forcing by the momentum it must add, MRT by its reduction to BGK,
mass by conservation, the EOS coupling by flat-interface coexistence and Laplace's law, the
measurement by the closed-form secant construction on exact circular caps.
"""
import numpy as np
import pytest

from helpers import (cap_angle_on_circle, drop_centre_for_angle, exact_secant_angle,
                     oracle_config, tanh_drop)
from paper_2202_06516_gb300 import workloads as W

MODEL_KEYS = ["eos", "Tr", "k2", "kappa", "tau", "s_e", "s_eps", "s_q"]


def _model():
    return {k: W.MODEL[k] for k in MODEL_KEYS}


# ------------------------------------------------------------------ geometry (Sec. 3.1, Fig. 1)
def _brute_flags(nx, ny, circle, concave=False):
    """Independent classification on the extended rows -2..ny+1 (concave: the circle is a cavity,
    solid outside it)."""
    rows = ny + 4
    solid = np.zeros((rows, nx), bool)
    for r in range(rows):
        j = r - 2
        for i in range(nx):
            s = j < 0 or j >= ny
            if circle is not None:
                cx, cy, R = circle
                inside = (i - cx) ** 2 + (j - cy) ** 2 <= R * R
                s = s or (inside != concave)
            solid[r, i] = s
    nb = [(1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
    flags = np.where(solid, 3, 0)
    for r in range(rows):
        for i in range(nx):
            if solid[r, i] and any(0 <= r + dy < rows and not solid[r + dy, (i + dx) % nx]
                                   for dx, dy in nb):
                flags[r, i] = 1
    for r in range(rows):
        for i in range(nx):
            if flags[r, i] == 3 and any(0 <= r + dy < rows and flags[r + dy, (i + dx) % nx] == 1
                                        for dx, dy in nb):
                flags[r, i] = 2
    return flags.astype(np.uint8)


@pytest.mark.parametrize("circle,concave", [(None, 0), ((20.0, 0.0, 9.0), 0), ((17.5, 3.0, 6.5), 0),
                                            ((0.0, 10.0, 7.0), 0), ((20.0, 12.0, 10.5), 1),
                                            ((19.5, 20.0, 17.0), 1), ((0.0, 11.5, 14.0), 1)])
def test_geometry_bruteforce(oracle_mod, circle, concave):
    O = oracle_mod
    nx, ny = 40, 24
    kw = dict(nx=nx, ny=ny, Tr=0.7)
    if circle:
        kw.update(has_circle=1, cx=circle[0], cy=circle[1], R=circle[2], concave=concave)
    s = O.Sim(O.Config(**kw, drop_x=20, drop_y=30, drop_r=2))
    _, _, flag, _ = s.ext()
    assert np.array_equal(flag, _brute_flags(nx, ny, circle, bool(concave)))
    # boundary links: (fluid node, q) with x + e_q solid, in (node, q) order
    ex = [0, 1, 0, -1, 0, 1, -1, -1, 1]
    ey = [0, 0, 1, 0, -1, 1, 1, -1, -1]
    want = []
    for j in range(ny):
        for i in range(nx):
            if flag[j + 2, i] != 0:
                continue
            for q in range(1, 9):
                if flag[j + 2 + ey[q], (i + ex[q]) % nx] != 0:
                    want.append((j * nx + i) * 9 + q)
    assert np.array_equal(s.links(), np.array(want, dtype=np.int64))


def test_wall_mu_assignment(oracle_mod):
    """Layer nodes take the circle's (or stripe's) chemical potential inside the disc and the
    flat wall's below/above the domain; other nodes carry none."""
    O = oracle_mod
    cfg = O.Config(nx=64, ny=40, Tr=0.7, has_circle=1, cx=32, cy=0, R=15, mu_circle=0.5,
                   mu_bottom=-1.0, mu_top=2.0, stripes=1, stripe_arc=5.0, mu_stripe_b=0.25,
                   drop_x=32, drop_y=30, drop_r=3)
    s = O.Sim(cfg)
    _, _, flag, muw = s.ext()
    for r in range(flag.shape[0]):
        j = r - 2
        for i in range(64):
            if flag[r, i] not in (1, 2):
                assert muw[r, i] == 0
                continue
            if (i - 32) ** 2 + j * j <= 225:
                phi = np.arctan2(j, i - 32)
                k = int(np.floor(15 * (phi - np.pi / 2) / 5.0))
                assert muw[r, i] == (0.5 if k % 2 == 0 else 0.25)
            else:
                assert muw[r, i] == (-1.0 if j < 0 else 2.0)


def test_wall_mu_assignment_concave(oracle_mod):
    """In a cavity the circle's potential (and its stripes) belongs to the layer nodes outside the
    circle; layer nodes of the wall rows inside the circle keep the flat walls' values."""
    O = oracle_mod
    cfg = O.Config(nx=64, ny=40, Tr=0.7, has_circle=1, cx=32, cy=22, R=24, concave=1,
                   mu_circle=0.5, mu_bottom=-1.0, mu_top=2.0, stripes=1, stripe_arc=5.0,
                   mu_stripe_b=0.25, drop_x=32, drop_y=10, drop_r=3)
    s = O.Sim(cfg)
    _, _, flag, muw = s.ext()
    seen = set()
    for r in range(flag.shape[0]):
        j = r - 2
        for i in range(64):
            if flag[r, i] not in (1, 2):
                assert muw[r, i] == 0
                continue
            if (i - 32) ** 2 + (j - 22) ** 2 > 24 * 24:
                phi = np.arctan2(j - 22, i - 32)
                k = int(np.floor(24 * (phi - np.pi / 2) / 5.0))
                assert muw[r, i] == (0.5 if k % 2 == 0 else 0.25)
                seen.add("circle")
            else:
                assert muw[r, i] == (-1.0 if j < 0 else 2.0)
                seen.add("wall")
    assert seen == {"circle", "wall"}


def test_wetting_layer_densities_eq14(oracle_mod):
    """Eq. 14 on a random density field, by brute force: a first-layer node takes the D2Q9-weighted
    mean of its fluid neighbours, a second-layer node the weighted mean of its first-layer
    neighbours (the layers of a step are built from the density the step starts from)."""
    O = oracle_mod
    nx, ny = 40, 30
    cfg = O.Config(nx=nx, ny=ny, Tr=0.7, has_circle=1, cx=20.5, cy=4.0, R=9.0, mu_circle=0.1,
                   mu_bottom=0.0, mu_top=0.0, drop_x=20, drop_y=24, drop_r=3)
    rng = np.random.default_rng(5)
    rho0 = 1.0 + rng.random((ny, nx))
    s = O.Sim(cfg, rho0)
    _, _, flag, _ = s.ext()
    s.step(1)
    r_ext, _, _, _ = s.ext()
    ext0 = np.zeros((ny + 4, nx))
    ext0[2:-2] = rho0
    ex = [1, 0, -1, 0, 1, -1, -1, 1]
    ey = [0, 1, 0, -1, 1, 1, -1, -1]
    wq = [1 / 9] * 4 + [1 / 36] * 4
    want = ext0.copy()
    for layer, src in ((1, 0), (2, 1)):
        for r in range(ny + 4):
            for i in range(nx):
                if flag[r, i] != layer:
                    continue
                num = den = 0.0
                for dx, dy, w in zip(ex, ey, wq):
                    rr = r + dy
                    if 0 <= rr < ny + 4 and flag[rr, (i + dx) % nx] == src:
                        num += w * want[rr, (i + dx) % nx]
                        den += w
                assert den > 0
                want[r, i] = num / den
        sel = flag == layer
        assert sel.sum() > 10
        assert np.allclose(r_ext[sel], want[sel], rtol=1e-14, atol=0)


# ------------------------------------------------------- stencils (Eq. 12, fourth-order FD)
def test_chemical_potential_exact_on_quartics(oracle_mod):
    """mu = k^2 psi'(rho) - kappa lap(rho); the fourth-order Laplacian is exact on quartics, so
    on a quartic density field mu matches the analytic Laplacian at interior nodes."""
    O = oracle_mod
    nx, ny = 48, 40
    j, i = np.mgrid[0:ny, 0:nx].astype(float)
    x, y = (i - 20.0) / 20.0, (j - 18.0) / 20.0
    rho = 3.0 + 0.3 * x**4 - 0.2 * x**3 + 0.1 * x + 0.25 * y**4 + 0.15 * y**2 - 0.05 * y**3
    lap = (0.3 * 12 * x**2 - 0.2 * 6 * x) / 400.0 + (0.25 * 12 * y**2 + 0.3 - 0.05 * 6 * y) / 400.0
    m = _model()
    s = O.Sim(O.Config(nx=nx, ny=ny, **m, mu_bottom=0.02, mu_top=0.02), rho)
    s.step(1)
    _, mu, _, _ = s.ext()
    for jj in range(3, ny - 3):
        for ii in range(3, nx - 3):
            want = m["k2"] * O.eos_eval(0, m["Tr"], rho[jj, ii])["mu0"] - m["kappa"] * lap[jj, ii]
            assert mu[jj + 2, ii] == pytest.approx(want, rel=1e-12, abs=1e-14)


def test_force_gradient_fourth_order(oracle_mod):
    """F = -rho grad(mu) + grad(rho)/3 converges at fourth order on a smooth field: halving the
    wavelength-to-lattice ratio raises the error by about 2^4."""
    O = oracle_mod
    m = dict(_model(), kappa=0.0)
    errs = []
    for L in (16.0, 32.0):
        nx, ny = int(4 * L), 48
        j, i = np.mgrid[0:ny, 0:nx].astype(float)
        rho = 3.0 + 0.5 * np.sin(2 * np.pi * i / (4 * L))
        s = O.Sim(O.Config(nx=nx, ny=ny, **m, mu_bottom=0.02, mu_top=0.02), rho)
        s.step(1)
        _, _, fx, fy = s.velocity_force()
        k = 2 * np.pi / (4 * L)
        drho = 0.5 * k * np.cos(k * i)
        mup = np.array([O.eos_eval(0, m["Tr"], r)["dp"] / r for r in rho.ravel()]).reshape(rho.shape)
        want = -rho * m["k2"] * mup * drho + drho / 3.0
        band = slice(5, ny - 5)
        errs.append(np.abs(fx[band] - want[band]).max() / np.abs(want[band]).max())
    assert errs[1] < errs[0] / 10.0


# --------------------------------------------------- collision and forcing (Eq. 1, 3, 13)
@pytest.mark.parametrize("g_rho_ref", [0.0, 0.1, 0.3])
def test_body_force_momentum(oracle_mod, g_rho_ref):
    """Exact-difference forcing adds exactly the force as momentum and no mass: a uniform fluid of
    density 0.3 at rest under acceleration g with body-force reference density rho_ref has
    velocity (1 - rho_ref / 0.3) g after one step (g itself for rho_ref = 0, rest for 0.3)."""
    O = oracle_mod
    m = _model()
    rho0 = np.full((24, 16), 0.3)
    s = O.Sim(O.Config(nx=16, ny=24, **m, gx=3e-4, gy=-2e-4, g_rho_ref=g_rho_ref,
                       mu_bottom=0.0, mu_top=0.0), rho0)
    s.step(1)
    f = s.f()
    ex = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
    ey = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
    rho = f.sum(-1)
    mid = slice(4, 20)
    scale = 1.0 - g_rho_ref / 0.3
    assert np.allclose(rho[mid], 0.3, rtol=1e-13)
    assert np.allclose((f @ ex)[mid] / rho[mid], 3e-4 * scale, rtol=1e-10, atol=1e-14)
    assert np.allclose((f @ ey)[mid] / rho[mid], -2e-4 * scale, rtol=1e-10, atol=1e-14)


@pytest.mark.parametrize("collision,tau", [(0, 1.0), (0, 0.8), (1, 0.9)])
def test_channel_shear_mode_decays_at_the_lattice_viscosity(oracle_mod, collision, tau):
    """The lowest shear mode of the channel, u_x = U sin(pi (y + 1/2) / ny) between the walls at
    y = -1/2 and ny - 1/2, in a uniform liquid (no interface, so no force) decays as
    exp(-nu (pi / ny)^2 t) with the lattice viscosity nu = (tau - 1/2) / 3 of the shear rate
    s_v = 1/tau (Sec. 2.1). This pins the stress rows of the MRT moment basis (equal rates
    reduce MRT to BGK for any invertible basis) and the half-way wall position."""
    O = oracle_mod
    m = _model()
    m.update(tau=tau)
    mx = O.maxwell(m["eos"], m["Tr"])
    neutral = m["k2"] * mx["mu_sat"]
    nx, ny, U = 8, 48, 1e-3
    cfg = O.Config(nx=nx, ny=ny, **m, collision=collision, rho_g=mx["rho_g"], rho_l=mx["rho_l"],
                   mu_bottom=neutral, mu_top=neutral, drop_x=0, drop_y=0, drop_r=1)
    rho0 = np.full((ny, nx), mx["rho_l"])
    s = O.Sim(cfg, rho0)
    # equilibrium populations (Eq. 2) of the mode, as the initial state
    mode = np.sin(np.pi * (np.arange(ny) + 0.5) / ny)
    ux = (U * mode)[:, None].repeat(nx, 1)
    ex = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    eu = ex[None, None, :] * ux[:, :, None]
    f = w * rho0[:, :, None] * (1 + 3 * eu + 4.5 * eu ** 2 - 1.5 * (ux ** 2)[:, :, None])
    s.set_f(f)
    steps = 3000
    s.step(steps)
    s.step(1)   # the reported velocity is that of the state before the last step
    vx, _, _, _ = s.velocity_force()
    amp = (vx.mean(1) * mode).sum() / (mode * mode).sum()
    nu = (tau - 0.5) / 3.0
    want = np.exp(-nu * (np.pi / ny) ** 2 * steps)
    assert amp / U == pytest.approx(want, rel=5e-3)
    # and not the decay of another viscosity (a 10 % error in nu moves it by > 1 %)
    assert abs(amp / U - np.exp(-1.1 * nu * (np.pi / ny) ** 2 * steps)) > 0.01 * want


def test_sound_wave_travels_at_the_model_sound_speed(oracle_mod):
    """A small density wave in the uniform liquid oscillates at omega = c q with the model's
    sound speed c^2 = k^2 p0'(rho_l) + rho_l kappa q^2: the force of Eq. 7, -rho grad(mu) +
    c_s^2 grad(rho), replaces the lattice pressure c_s^2 rho by rho mu (Gibbs-Duhem), and the
    gradient term of Eq. 12 adds the q^2 dispersion. A dropped k^2, a sign error in the c_s^2
    term or a missing Laplacian moves omega by far more than the 5 % tolerance (the fit is ~3 %
    above the continuum value: damping and the half-step lag of the forcing shift it)."""
    from scipy.optimize import curve_fit
    O = oracle_mod
    m = _model()
    mx = O.maxwell(m["eos"], m["Tr"])
    neutral = m["k2"] * mx["mu_sat"]
    nx, ny, eps = 64, 96, 1e-4
    rl = mx["rho_l"]
    q = 2 * np.pi / nx
    rho0 = rl * (1 + eps * np.cos(q * np.arange(nx)))[None, :].repeat(ny, 0)
    cfg = O.Config(nx=nx, ny=ny, **m, rho_g=mx["rho_g"], rho_l=rl, mu_bottom=neutral,
                   mu_top=neutral, drop_x=0, drop_y=0, drop_r=1)
    s = O.Sim(cfg, rho0)
    amps = []
    for _ in range(1200):
        r = s.rho()[ny // 2 - 5: ny // 2 + 5].mean(0)
        amps.append(((r - r.mean()) * np.cos(q * np.arange(nx))).sum() * 2 / nx / (rl * eps))
        s.step(1)
    c2 = m["k2"] * O.eos_eval(m["eos"], m["Tr"], rl)["dp"] + rl * m["kappa"] * q * q
    w0 = np.sqrt(c2) * q
    fit = lambda t, A, g, w, ph: A * np.exp(-g * t) * np.cos(w * t + ph)
    popt, _ = curve_fit(fit, np.arange(len(amps)), np.array(amps), p0=[1, 1e-3, w0, 0])
    assert popt[2] == pytest.approx(w0, rel=0.05)
    assert popt[1] > 0   # damped by the bulk and shear viscosity


@pytest.mark.parametrize("tau", [1.0, 0.8])
def test_mrt_reduces_to_bgk(oracle_mod, tau):
    """With every relaxation rate equal to 1/tau, MRT (Eq. 1) equals BGK (Eq. 3): pins the moment
    matrix and its inverse."""
    O = oracle_mod
    w = W.plain_small()
    cfg_m, _, _ = oracle_config(O, w, nx=80, ny=60, cx=40, R=15, drop_x=40, drop_y=31.5,
                                drop_r=15, tau=tau, s_e=1 / tau, s_eps=1 / tau, s_q=1 / tau)
    cfg_b, _, _ = oracle_config(O, w, nx=80, ny=60, cx=40, R=15, drop_x=40, drop_y=31.5,
                                drop_r=15, tau=tau, collision=1)
    a, b = O.Sim(cfg_m), O.Sim(cfg_b)
    a.step(50)
    b.step(50)
    assert np.allclose(a.f(), b.f(), rtol=1e-11, atol=1e-13)
    # and genuinely different rates change the result
    c = O.Sim(oracle_config(O, w, nx=80, ny=60, cx=40, R=15, drop_x=40, drop_y=31.5,
                            drop_r=15, tau=tau)[0])
    c.step(50)
    assert not np.allclose(a.f(), c.f(), rtol=1e-6)


def test_mass_conservation(oracle_mod):
    """Periodic streaming, half-way bounce-back and mass-neutral forcing conserve mass to
    round-off over the 200 x 120 workload's 3000 steps."""
    O = oracle_mod
    cfg, _, _ = oracle_config(O, W.plain_small())
    s = O.Sim(cfg)
    m0 = s.mass()
    s.step(3000)
    assert abs(s.mass() - m0) / m0 < 1e-11
    assert np.isfinite(s.rho()).all()


def test_carnahan_starling_workload(oracle_mod):
    """The Carnahan-Starling 200 x 120 workload (MRT, Tr = 0.7): mass conserved to round-off over
    its 3000 steps, the mirror-symmetric set-up gives mirror-equal left and right angles, and the
    bulk densities relax toward the CS Maxwell pair (liquid within 3 %, gas within a factor 2:
    the forcing's discrete pressure term shifts the gas, as for PR)."""
    O = oracle_mod
    cfg, mx, _ = oracle_config(O, W.plain_small_cs())
    assert cfg.eos == O.EOS_CS
    s = O.Sim(cfg)
    m0 = s.mass()
    s.step(3000)
    rho = s.rho()
    assert np.isfinite(rho).all()
    assert abs(s.mass() - m0) / m0 < 1e-11
    left, right, cen = s.measure()
    assert left.status == 0 and right.status == 0
    assert abs(left.theta - right.theta) < 1e-9
    assert cen[0] == pytest.approx(cfg.cx, abs=1e-9)
    assert 60.0 < left.theta < 120.0
    liquid = rho[int(cfg.drop_y), int(cfg.drop_x)]
    gas = rho[cfg.ny - 10, 5]
    assert liquid == pytest.approx(mx["rho_l"], rel=0.03)
    assert mx["rho_g"] / 2 < gas < 2 * mx["rho_g"]


@pytest.mark.parametrize("phase", ["liquid", "gas"])
def test_uniform_coexistence_state_is_fixed_point(oracle_mod, phase):
    """A uniform fluid at a coexistence density next to neutral walls (mu_w = k^2 psi'(rho_sat))
    is an exact equilibrium: psi' of either coexistence density equals the wall value, so mu is
    uniform, the Eq. 14 layers copy the fluid density, the force vanishes and the equilibrium
    populations are a fixed point of collision and streaming."""
    O = oracle_mod
    cfg, mx, neutral = oracle_config(O, W.plain_small(), nx=64, ny=48, cx=32.0, R=12.0)
    rho_c = mx["rho_l"] if phase == "liquid" else mx["rho_g"]
    rho0 = np.full((cfg.ny, cfg.nx), rho_c)
    s = O.Sim(cfg, rho0)
    s.step(200)
    r = s.rho()
    fluid = s.ext()[2][2:-2] == 0
    assert np.abs(r[fluid] - rho_c).max() / rho_c < 1e-10
    ux, uy, _, _ = s.velocity_force()
    assert np.abs(ux[fluid]).max() < 1e-12 and np.abs(uy[fluid]).max() < 1e-12


# ------------------------------------------------------ thermodynamics (Eq. 7, 12, Maxwell)
def test_flat_interface_coexistence(oracle_mod):
    """A flat liquid slab equilibrates at the Maxwell liquid density (0.5 %). The gas density
    sits above its Maxwell value: the forcing's discrete pressure term is largest where
    F / rho is, in the gas; it is bounded here (within 30 %) as a regression on the model."""
    O = oracle_mod
    m = _model()
    mx = O.maxwell(0, m["Tr"])
    nx, ny = 4, 120
    j = np.arange(ny)[:, None] * np.ones((1, nx))
    rho0 = mx["rho_g"] + (mx["rho_l"] - mx["rho_g"]) * 0.5 * (np.tanh((j - 30) / 2.) -
                                                              np.tanh((j - 90) / 2.))
    neutral = m["k2"] * mx["mu_sat"]
    s = O.Sim(O.Config(nx=nx, ny=ny, **m, rho_g=mx["rho_g"], rho_l=mx["rho_l"],
                       mu_bottom=neutral, mu_top=neutral), rho0)
    s.step(12000)
    r = s.rho()[:, 0]
    assert r[60] == pytest.approx(mx["rho_l"], rel=5e-3)
    assert mx["rho_g"] < r[5] < 1.3 * mx["rho_g"]
    assert np.allclose(r[:, None], s.rho(), rtol=1e-12)  # stays one-dimensional


@pytest.mark.slow
def test_laplace_law(oracle_mod):
    """Free drops: the pressure jump k^2 (p0(rho_in) - p0(rho_out)) falls as 1/R (Laplace's law):
    Delta p * R agrees within 3 % for R = 16 and 24. The effective tension exceeds the continuum
    sqrt(k^2 kappa) * int sqrt(2 dOmega) drho (the forcing's discrete pressure term widens the
    interface to ~1.9 times the continuum width); it is bounded to 1.0-2.0 times that value."""
    O = oracle_mod
    from scipy.integrate import quad
    m = _model()
    mx = O.maxwell(0, m["Tr"])
    neutral = m["k2"] * mx["mu_sat"]
    dO = lambda r: O.eos_eval(0, m["Tr"], r)["psi"] - mx["mu_sat"] * r + mx["p_sat"]
    S, _ = quad(lambda r: np.sqrt(max(2 * dO(r), 0)), mx["rho_g"], mx["rho_l"], limit=200)
    sigma = np.sqrt(m["k2"] * m["kappa"]) * S
    pr = []
    for r0, N in [(16, 80), (24, 112)]:
        s = O.Sim(O.Config(nx=N, ny=N, **m, rho_g=mx["rho_g"], rho_l=mx["rho_l"],
                           mu_bottom=neutral, mu_top=neutral, drop_x=N / 2, drop_y=N / 2 - 0.5,
                           drop_r=r0, drop_W=4))
        s.step(7000)
        r = s.rho()
        rin, rout = r[N // 2, N // 2], r[N // 2, 2]
        dp = m["k2"] * (O.eos_eval(0, m["Tr"], rin)["p0"] - O.eos_eval(0, m["Tr"], rout)["p0"])
        Rm = np.sqrt(((r - rout) / (rin - rout)).sum() / np.pi)
        pr.append(dp * Rm)
    assert pr[0] == pytest.approx(pr[1], rel=0.03)
    assert 1.0 < pr[1] / sigma < 2.0


# --------------------------------------------------------- measurement (Eq. 15, Fig. 1, 2)
def _synthetic_cases(n, seed, flat=False):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        R = float(rng.integers(30, 120))
        r = float(rng.uniform(25, 60))
        th = float(rng.uniform(40, 140))
        if flat:
            nx = int(2 * r + 60)
            x0 = nx / 2 + rng.uniform(-0.5, 0.5)
            y0 = -0.5 - r * np.cos(np.radians(th))
            out.append((None, nx, int(y0 + r + 20), x0, y0, r, th))
            continue
        nx = int(2 * (R + r) + 40)
        cx = float(nx // 2)
        x0, y0 = drop_centre_for_angle(R + 0.5, r, th, cx, 0.0)
        x0 += rng.uniform(-0.5, 0.5)
        y0 += rng.uniform(-0.5, 0.5)
        D = np.hypot(x0 - cx, y0)
        # keep both contact points on the upper half of the cylinder, inside the domain
        cosg = (D * D + (R + 0.5) ** 2 - r * r) / (2 * D * (R + 0.5))
        if np.degrees(np.arccos(np.clip(cosg, -1, 1))) > 70:
            continue
        out.append(((cx, 0.0, R), nx, int(y0 + r + 20), x0, y0, r,
                    cap_angle_on_circle(R + 0.5, r, D)))
    return out


def _secant_tolerance_deg(a, drop_c, r):
    """How far the Fig. 1 secant through the measured points may turn away from the exact secant:
    each Eq. 15 point sits off the exact interface circle by e (linear interpolation of the tanh
    profile along its link), so the line through them turns by at most (e1 + e2) / |p2 - p1|
    rad; a 20 % margin covers the exact secant's use of the measured distances d1, d2."""
    e1 = abs(np.hypot(a.p1[0] - drop_c[0], a.p1[1] - drop_c[1]) - r)
    e2 = abs(np.hypot(a.p2[0] - drop_c[0], a.p2[1] - drop_c[1]) - r)
    sep = np.hypot(a.p2[0] - a.p1[0], a.p2[1] - a.p1[1])
    return np.degrees(1.2 * (e1 + e2) / sep) + 1e-9


def _synthetic_concave_cases(n, seed):
    """Circular drops resting in a circular cavity (radius Rs = R + 1/2, centre (cx, cy)) at a
    prescribed angle: D^2 = Rs^2 + r^2 + 2 Rs r cos(theta), drop centre straight below the cavity
    centre (plus a sub-node offset), contact points within 60 degrees of the cavity's bottom."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        R = float(rng.integers(60, 160))
        r = float(rng.uniform(20, 0.6 * R))
        th = float(rng.uniform(40, 140))
        Rs = R + 0.5
        D = np.sqrt(Rs * Rs + r * r + 2 * Rs * r * np.cos(np.radians(th)))
        cosg = (D * D + Rs * Rs - r * r) / (2 * D * Rs)   # half-angle of the wetted arc
        if np.degrees(np.arccos(np.clip(cosg, -1, 1))) > 60:
            continue
        nx = int(2 * R + 20)
        cx, cy = float(nx // 2), R + 6.0
        x0 = cx + rng.uniform(-0.5, 0.5)
        y0 = cy - D + rng.uniform(-0.5, 0.5)
        D = np.hypot(x0 - cx, y0 - cy)
        out.append(((cx, cy, R), nx, int(cy + 10), x0, y0, r,
                    cap_angle_on_circle(Rs, r, D, concave=True)))
    return out


def test_measure_synthetic_caps_concave(oracle_mod):
    """The Fig. 1 construction in a cavity (Fig. 2b): on exact circular drops the angle equals the
    closed-form secant through the chosen points, is within the curvature offset of the true
    angle, the contact point lies on the wall surface R + 1/2, and beta = theta - alpha."""
    O = oracle_mod
    mx = O.maxwell(0, 0.7)
    rg, rl = mx["rho_g"], mx["rho_l"]
    rm = 0.5 * (rg + rl)
    for circ, nx, ny, x0, y0, r, th in _synthetic_concave_cases(20, 5):
        cfg = O.Config(nx=nx, ny=ny, Tr=0.7, has_circle=1, cx=circ[0], cy=circ[1], R=circ[2],
                       concave=1)
        sub = ("concave", circ[0], circ[1], circ[2] + 0.5)
        rho = tanh_drop(nx, ny, x0, y0, r, rg, rl, 10.0)
        L, R_, _ = O.measure(cfg, rho, rm)
        for side, a in enumerate((L, R_)):
            assert a.status == 0
            assert abs(a.d1 - 1) <= 0.75 and abs(a.d2 - 2) <= 0.75
            for pt in (a.p1, a.p2):  # Eq. 15 points on the exact interface circle
                assert abs(np.hypot(pt[0] - x0, pt[1] - y0) - r) < 0.012
            sec = exact_secant_angle(sub, (x0, y0), r, a.d1, a.d2, side)
            assert abs(a.theta - sec) <= _secant_tolerance_deg(a, (x0, y0), r)
            assert abs(a.theta - th) <= np.degrees(1.6 * 1.5 / r) + 0.75
            assert np.hypot(a.contact[0] - circ[0], a.contact[1] - circ[1]) == \
                pytest.approx(circ[2] + 0.5, abs=1e-9)
            assert a.beta == pytest.approx(a.theta - a.alpha)
        # left is the smaller-x contact line for a drop at the bottom of the cavity
        assert L.contact[0] < R_.contact[0]


def test_cap_method_closed_form_concave(oracle_mod):
    """Spherical-cap method in a cavity: theta = beta + alpha equals the circle-circle angle."""
    O = oracle_mod
    mx = O.maxwell(0, 0.7)
    rg, rl = mx["rho_g"], mx["rho_l"]
    for circ, nx, ny, x0, y0, r, th in _synthetic_concave_cases(8, 9):
        cfg = O.Config(nx=nx, ny=ny, Tr=0.7, has_circle=1, cx=circ[0], cy=circ[1], R=circ[2],
                       concave=1)
        rho = tanh_drop(nx, ny, x0, y0, r, rg, rl, 6.0)
        cap = O.cap_angle(cfg, rho, 0.5 * (rg + rl))
        assert cap["r"] == pytest.approx(r, abs=0.1)
        assert cap["theta"] == pytest.approx(th, abs=0.5)
        assert cap["theta"] == pytest.approx(cap["beta"] + cap["alpha"], abs=1e-9)


@pytest.mark.parametrize("flat", [False, True])
@pytest.mark.parametrize("width", [10.0, 5.6])
def test_measure_synthetic_caps(oracle_mod, flat, width):
    """On exact circular caps (tanh interface of the paper's width W = 10, and the workloads'
    5.6) every Eq. 15 point lies within 0.012 lu of the exact interface (the level set rho_m of
    the profile is the drop circle; the residue is linear interpolation along the link); the
    measured angle is the Fig. 1 secant through the exact circle points at the chosen distances
    d1, d2, within the turn that those point errors allow (1.2 (e1 + e2) / |p2 - p1| rad: up to
    0.5 deg at W = 10 and 1.6 deg at W = 5.6, where the points can lie 0.8 lu apart); the
    contact point lies on the substrate, and the offset from the true angle is the interface
    curvature over the ~1.5 lu between the wall and the points (a loose sanity bound: 1.6 * 1.5 / r
    rad plus 0.75 deg)."""
    O = oracle_mod
    mx = O.maxwell(0, 0.7)
    rg, rl = mx["rho_g"], mx["rho_l"]
    rm = 0.5 * (rg + rl)
    for circ, nx, ny, x0, y0, r, th in _synthetic_cases(25, 1 if flat else 0, flat):
        kw = dict(nx=nx, ny=ny, Tr=0.7)
        if circ:
            kw.update(has_circle=1, cx=circ[0], cy=circ[1], R=circ[2])
            sub = ("circle", circ[0], circ[1], circ[2] + 0.5)
        else:
            sub = ("flat", -0.5)
        cfg = O.Config(**kw)
        rho = tanh_drop(nx, ny, x0, y0, r, rg, rl, width)
        L, R_, _ = O.measure(cfg, rho, rm)
        for side, a in enumerate((L, R_)):
            assert a.status == 0
            assert 0.5 <= a.d1 <= 2.5 and 0.5 <= a.d2 <= 2.5
            assert abs(a.d1 - 1) <= 0.75 and abs(a.d2 - 2) <= 0.75
            for pt in (a.p1, a.p2):
                assert abs(np.hypot(pt[0] - x0, pt[1] - y0) - r) < 0.012
            sec = exact_secant_angle(sub, (x0, y0), r, a.d1, a.d2, side)
            tol = _secant_tolerance_deg(a, (x0, y0), r)
            assert abs(a.theta - sec) <= tol
            assert abs(a.theta - th) <= np.degrees(1.6 * 1.5 / r) + max(tol, 0.75)
            if circ:
                assert np.hypot(a.contact[0] - circ[0], a.contact[1] - circ[1]) == \
                    pytest.approx(circ[2] + 0.5, abs=1e-9)
                assert a.beta == pytest.approx(a.theta + a.alpha)
            else:
                assert a.contact[1] == -0.5 and a.alpha == 0


def test_measure_mirror_symmetry(oracle_mod):
    """A drop centred on the cylinder's axis gives equal left and right angles."""
    O = oracle_mod
    mx = O.maxwell(0, 0.7)
    rg, rl = mx["rho_g"], mx["rho_l"]
    cfg = O.Config(nx=201, ny=120, Tr=0.7, has_circle=1, cx=100, cy=0, R=40)
    rho = tanh_drop(201, 120, 100.0, 62.3, 27.0, rg, rl, 6.0)
    L, R_, c = O.measure(cfg, rho, 0.5 * (rg + rl))
    assert c[0] == pytest.approx(100.0, abs=1e-12)
    assert L.theta == pytest.approx(R_.theta, abs=1e-9)
    assert L.p1[0] + R_.p1[0] == pytest.approx(200.0, abs=1e-9)


def test_cap_method_closed_form(oracle_mod):
    """Spherical-cap method (Sec. 4.1): on exact caps the fitted radius equals R0 from
    (4H^2 + L^2) / 8H and theta = beta - alpha equals the circle-circle angle."""
    O = oracle_mod
    mx = O.maxwell(0, 0.7)
    rg, rl = mx["rho_g"], mx["rho_l"]
    for circ, nx, ny, x0, y0, r, th in _synthetic_cases(8, 3):
        cfg = O.Config(nx=nx, ny=ny, Tr=0.7, has_circle=1, cx=circ[0], cy=circ[1], R=circ[2])
        rho = tanh_drop(nx, ny, x0, y0, r, rg, rl, 6.0)
        cap = O.cap_angle(cfg, rho, 0.5 * (rg + rl))
        assert cap["R0"] == pytest.approx(cap["r"], rel=1e-9)
        assert cap["r"] == pytest.approx(r, abs=0.1)
        assert cap["theta"] == pytest.approx(th, abs=0.5)


@pytest.mark.slow
def test_equilibrium_present_vs_cap(oracle_mod):
    """Equilibrated drop on a cylinder (neutral wall): the present scheme agrees with the
    spherical-cap method within 2 degrees (Sec. 4.1 reports agreement at relative L2 error
    0.025), both sides agree, and the angle is stationary."""
    O = oracle_mod
    w = W.plain_small()
    cfg, _, _ = oracle_config(O, w, nx=120, ny=80, cx=60, R=30, drop_x=60, drop_y=30.5 + 18,
                              drop_r=18)
    s = O.Sim(cfg)
    s.step(9000)
    L1, R1, _ = s.measure()
    s.step(1000)
    L, R_, _ = s.measure()
    cap = O.cap_angle(cfg, s.rho(), s.rho_m)
    assert L.status == 0 and R_.status == 0
    assert L.theta == pytest.approx(R_.theta, abs=0.2)
    assert L.theta == pytest.approx(cap["theta"], abs=2.0)
    assert L.theta == pytest.approx(L1.theta, abs=0.2)


# ------------------------------------------- interpolated bounce-back (curved-wall variant)
def _in_analytic_solid(x, y, ny, circle, concave):
    """The analytic solid of the interpolated scheme: beyond the flat wall planes, inside the
    disc of radius R + 1/2 (outside it for a cavity)."""
    if y <= -0.5 or y >= ny - 0.5:
        return True
    if circle is None:
        return False
    cx, cy, R = circle
    d2, w2 = (x - cx) ** 2 + (y - cy) ** 2, (R + 0.5) ** 2
    return d2 >= w2 if concave else d2 <= w2      # the wall circle itself counts as solid


def _brute_fraction(i, j, d, ny, circle, concave, n=4001):
    """First s in [0, 1] at which the point (i, j) + s e_d crosses into the analytic solid: a
    scan, then bisection on the first bracket; 1/2 when the segment starts inside it or never
    enters it (no crossing within the link)."""
    ex = [0, 1, 0, -1, 0, 1, -1, -1, 1][d]
    ey = [0, 0, 1, 0, -1, 1, 1, -1, -1][d]
    s = np.linspace(0.0, 1.0, n)
    hit = [k for k in range(n) if _in_analytic_solid(i + s[k] * ex, j + s[k] * ey, ny, circle,
                                                     concave)]
    if not hit or hit[0] == 0:
        return 0.5
    k = hit[0]
    lo, hi = s[k - 1], s[k]
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if _in_analytic_solid(i + mid * ex, j + mid * ey, ny, circle, concave):
            hi = mid
        else:
            lo = mid
    return hi


@pytest.mark.parametrize("circle,concave", [((20.0, 0.0, 9.0), 0), ((17.5, 3.0, 6.5), 0),
                                            ((20.0, 12.0, 10.5), 1), (None, 0)])
def test_link_fraction_bruteforce(oracle_mod, circle, concave):
    """Link fractions of every cut link against a scan-and-bisect of the analytic wall; flat
    walls sit half way."""
    O = oracle_mod
    nx, ny = 40, 24
    kw = dict(nx=nx, ny=ny, Tr=0.7)
    if circle:
        kw.update(has_circle=1, cx=circle[0], cy=circle[1], R=circle[2], concave=concave)
    cfg = O.Config(**kw, drop_x=20, drop_y=30, drop_r=2)
    _, _, flag, _ = O.Sim(cfg).ext()
    ex = [0, 1, 0, -1, 0, 1, -1, -1, 1]
    ey = [0, 0, 1, 0, -1, 1, 1, -1, -1]
    checked = 0
    for j in range(ny):
        for i in range(nx):
            if flag[j + 2, i] != 0:
                continue
            for d in range(1, 9):
                if flag[j + 2 + ey[d], (i + ex[d]) % nx] == 0:
                    continue
                got = O.link_fraction(cfg, i, j, d)
                assert 0.0 <= got <= 1.0
                if not 0 <= i + ex[d] < nx:
                    continue   # across the periodic edge (the circle has no periodic image)
                # the scheme takes walls closer than a tenth of the link at a tenth
                want = max(_brute_fraction(i, j, d, ny, circle, bool(concave)), 0.1)
                assert got == pytest.approx(want, abs=1e-6), (i, j, d)
                checked += 1
    assert checked > 20


def _ibb_cfg(O, **over):
    cfg, mx, neutral = oracle_config(O, W.plain_small(), nx=96, ny=64, cx=48.0, R=20.0,
                                     drop_x=48.0, drop_y=20.0 + 14.0, drop_r=14.0, interp_bb=1)
    for k, v in over.items():
        setattr(cfg, k, v)
    return cfg


def test_interp_bb_reduces_to_halfway_on_flat_walls(oracle_mod):
    """With only flat walls every link fraction is 1/2, where the interpolation returns the
    outgoing population exactly: the interpolated run equals the half-way run bit for bit."""
    O = oracle_mod
    a = O.Sim(_ibb_cfg(O, has_circle=0, drop_y=10.0))
    b = O.Sim(_ibb_cfg(O, has_circle=0, drop_y=10.0, interp_bb=0))
    a.step(300)
    b.step(300)
    assert np.array_equal(a.f(), b.f())


@pytest.mark.parametrize("concave", [0, 1])
def test_interp_bb_conserves_mass_and_differs(oracle_mod, concave):
    """The mass correction keeps the total mass to round-off on a circle (convex and cavity),
    and the scheme is live: the fields differ from the half-way run (by a shift of the contact
    line, a small fraction of the density jump)."""
    O = oracle_mod
    over = dict(concave=concave)
    if concave:
        over.update(cx=48.0, cy=40.0, R=37.0, drop_y=10.0)
    a = O.Sim(_ibb_cfg(O, **over))
    b = O.Sim(_ibb_cfg(O, interp_bb=0, **over))
    m0 = a.mass()
    a.step(400)
    b.step(400)
    assert abs(a.mass() - m0) / m0 < 1e-12
    d = np.abs(a.rho() - b.rho()) / a.cfg.rho_l
    assert d.max() > 1e-6
    assert d.max() < 0.2


def test_interp_bb_keeps_uniform_coexistence_at_rest(oracle_mod):
    """A uniform liquid at the coexistence density around a cylinder is an exact fixed point of
    the interpolated scheme as well (equal populations interpolate to themselves)."""
    O = oracle_mod
    cfg = _ibb_cfg(O)
    mx = O.maxwell(0, cfg.Tr)
    s = O.Sim(cfg, np.full((cfg.ny, cfg.nx), mx["rho_l"]))
    s.step(300)
    _, _, flag, _ = s.ext()
    r = s.rho()[flag[2:-2] == 0]
    assert np.abs(r - mx["rho_l"]).max() / mx["rho_l"] < 1e-12
    ux, uy, _, _ = s.velocity_force()
    assert np.abs(ux[flag[2:-2] == 0]).max() < 1e-12


@pytest.mark.parametrize("concave", [0, 1])
def test_interp_bb_mirror_symmetry(oracle_mod, concave):
    """A configuration symmetric under x -> nx - 1 - x stays symmetric under the interpolated
    scheme to round-off: link fractions, the choice of the node behind and the mass correction
    are direction-consistent (a swapped direction index breaks the mirror)."""
    O = oracle_mod
    nx, ny = 91, 70
    c = (nx - 1) / 2.0
    if concave:
        cfg = _ibb_cfg(O, nx=nx, ny=ny, cx=c, cy=38.0, R=33.5, concave=1, drop_x=c, drop_y=9.0,
                       drop_r=12.0)
    else:
        cfg = _ibb_cfg(O, nx=nx, ny=ny, cx=c, cy=0.0, R=20.5, drop_x=c, drop_y=20.5 + 12.0,
                       drop_r=13.0)
    s = O.Sim(cfg)
    s.step(300)
    r = s.rho()
    assert np.abs(r - r[:, ::-1]).max() / cfg.rho_l < 1e-10
    l, rr, _ = s.measure()
    assert l.status == 0 and rr.status == 0
    assert l.theta == pytest.approx(rr.theta, abs=1e-6)
