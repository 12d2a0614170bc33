"""Host logic of the contact-line mechanics (Sec. 4.5): stripe fractions against brute force and
against the oracle's wall layout, Eq. 18 special cases, the sign convention of Eq. 17, the
transition-band footprint, and the per-sample analysis on a hand-made series."""
import math

import numpy as np
import pytest

from helpers import oracle_config
from paper_2202_06516_gb300 import contact_mechanics as CM
from paper_2202_06516_gb300 import workloads as W


def _brute_odd_fraction(a, b, arc, n=400001):
    s = np.linspace(a, b, n)
    return float((np.floor(s / arc) % 2 == 1).mean())


def test_odd_fraction_matches_brute_force():
    rng = np.random.default_rng(7)
    for _ in range(60):
        arc = float(rng.uniform(3.0, 50.0))
        a = float(rng.uniform(-300.0, 300.0))
        b = a + float(rng.choice([rng.uniform(0.1, arc), rng.uniform(arc, 7 * arc)]))
        got = float(CM.odd_fraction(a, b, arc))
        assert got == pytest.approx(_brute_odd_fraction(a, b, arc), abs=2e-4), (a, b, arc)


def test_odd_fraction_special_cases():
    arc = 40.0
    assert CM.odd_fraction(45.0, 75.0, arc) == 1.0        # inside stripe 1
    assert CM.odd_fraction(-35.0, -5.0, arc) == 1.0       # inside stripe -1 (odd)
    assert CM.odd_fraction(-75.0, -45.0, arc) == 0.0      # inside stripe -2 (even)
    assert CM.odd_fraction(30.0, 50.0, arc) == pytest.approx(0.5)   # straddles 40
    assert CM.odd_fraction(0.0, 4 * arc, arc) == pytest.approx(0.5)
    assert CM.odd_fraction(50.0, 50.0, arc) == 1.0        # zero-length: the point's stripe
    assert CM.odd_fraction(10.0, 10.0, arc) == 0.0


def test_stripe_convention_matches_the_oracle_wall(oracle_mod):
    """The analysis assigns a wall point to the same stripe as the oracle's geometry: every
    wetting-layer node of a striped circle carries the second wall potential exactly when its
    arc coordinate falls on an odd stripe."""
    O = oracle_mod
    w = W.Workload("stripes", 200, 120, (100.0, 0.0, 60.0), W.tangent_drop(100, 0, 60, 20),
                   mu_rel_circle=-0.02, stripes=(9.0, 0.03))
    cfg = oracle_config(O, w)[0]
    sim = O.Sim(cfg)
    _, _, flags, muw = sim.ext()
    j, i = np.nonzero((flags == 1) | (flags == 2))
    j = j - 2                                               # ext rows start at y = -2
    in_disc = (i - cfg.cx) ** 2 + (j - cfg.cy) ** 2 <= cfg.R ** 2
    i, j = i[in_disc], j[in_disc]
    assert i.size > 100
    s = CM.arc_coordinate(i, j, (cfg.cx, cfg.cy, cfg.R))
    odd = CM.odd_fraction(s, s, cfg.stripe_arc) == 1.0
    is_b = muw[j + 2, i] == cfg.mu_stripe_b
    assert odd.any() and (~odd).any()
    assert np.array_equal(odd, is_b)


def test_cassie_baxter_eq18():
    assert CM.cassie_baxter(1.0, 60.0, 120.0) == pytest.approx(60.0)
    assert CM.cassie_baxter(0.0, 60.0, 120.0) == pytest.approx(120.0)
    assert CM.cassie_baxter(0.5, 60.0, 120.0) == pytest.approx(90.0)
    # cos-weighted, not angle-weighted
    want = math.degrees(math.acos(0.25 * math.cos(math.radians(30.0))
                                  + 0.75 * math.cos(math.radians(150.0))))
    assert CM.cassie_baxter(0.25, 30.0, 150.0) == pytest.approx(want)
    # roughness r multiplies the first component only
    want = math.degrees(math.acos(1.2 * 0.5 * 0.5 + 0.5 * -0.5))
    assert CM.cassie_baxter(0.5, 60.0, 120.0, roughness=1.2) == pytest.approx(want)
    phis = np.linspace(0, 1, 11)
    assert np.all(np.diff(CM.cassie_baxter(phis, 60.0, 120.0)) < 0)


def test_young_force_sign_convention():
    """x to the right: advancing (right) angle above equilibrium pushes right (positive); a
    receding (left) angle above equilibrium gives a negative force; magnitudes follow Eq. 17."""
    g = 0.7
    assert CM.young_force_x(100.0, 100.0, g, CM.RIGHT) == 0.0
    fa = CM.young_force_x(120.0, 100.0, g, CM.RIGHT)
    fr = CM.young_force_x(120.0, 100.0, g, CM.LEFT)
    mag = g * abs(math.cos(math.radians(120.0)) - math.cos(math.radians(100.0)))
    assert fa == pytest.approx(mag) and fr == pytest.approx(-mag)
    assert CM.young_force_x(80.0, 100.0, g, CM.RIGHT) < 0
    assert CM.young_force_x(80.0, 100.0, g, CM.LEFT) > 0


def test_interface_footprint_is_the_band_cut():
    """A straight band of thickness w meeting the wall (y = 0) at theta: the two bounding lines
    cross the wall w / sin(theta) apart."""
    for theta in (30.0, 60.0, 90.0, 120.0, 150.0):
        t = math.radians(theta)
        d = np.array([math.cos(t), math.sin(t)])
        n = np.array([-math.sin(t), math.cos(t)])
        w = 7.3
        p0 = w * n                                   # a point of the second line
        x_cut = p0[0] - p0[1] / d[1] * d[0]          # where p0 + s d reaches y = 0
        assert CM.interface_footprint(w, theta) == pytest.approx(abs(x_cut))


def test_equilibrium_angle_and_series_analysis():
    circle, arc, R = (0.0, 0.0, 100.0), 20.0, 100.0

    def point_at(s):                                 # wall surface point at arc coordinate s
        phi = s / R + 0.5 * math.pi
        return (R + 0.5) * math.cos(phi), (R + 0.5) * math.sin(phi)

    # middle of an odd stripe, footprint well inside it: the stripe's own angle
    x, y = point_at(30.0)
    teq, phi = CM.equilibrium_angle(x, y, circle, 120.0, (arc, 60.0), width=4.0, theta_deg=90.0)
    assert phi == 1.0 and teq == pytest.approx(60.0)
    # centred on the border at s = 20: half on each side
    x, y = point_at(20.0)
    teq, phi = CM.equilibrium_angle(x, y, circle, 120.0, (arc, 60.0), width=4.0, theta_deg=90.0)
    assert phi == pytest.approx(0.5) and teq == pytest.approx(90.0)
    # uniform wall
    teq, phi = CM.equilibrium_angle(x, y, circle, 120.0, None)
    assert teq == 120.0 and phi == 0.0

    xl, yl = point_at(30.0)       # left line on an odd (60-degree) stripe
    xr, yr = point_at(-10.0)      # right line on stripe -1: odd as well
    xr2, yr2 = point_at(-30.0)    # stripe -2: even (120 degrees)
    series = np.array([
        [0, 50.0, 0, 70.0, xl, xr, yl, yr],
        [0, 50.0, 0, 125.0, xl, xr2, yl, yr2],
        [5, 0.0, 0, 125.0, 0.0, xr2, 0.0, yr2],
    ])
    res = CM.analyse_series(series, circle, 120.0, (arc, 60.0), gamma=2.0, width=4.0)
    L_, R_ = res["left"], res["right"]
    assert L_["region"].tolist() == [1, 1, -1] and R_["region"].tolist() == [1, 0, 0]
    assert np.isnan(L_["force"][2])
    # receding below its equilibrium angle: positive (the paper's hydrophilic-region case)
    assert L_["force"][0] == pytest.approx(2.0 * (math.cos(math.radians(50)) - 0.5))
    # advancing above equilibrium on the 60-degree stripe: positive
    assert R_["force"][0] > 0
    # advancing at 125 on the 120-degree wall: small positive
    assert R_["force"][1] == pytest.approx(
        2.0 * (math.cos(math.radians(120)) - math.cos(math.radians(125))))


def _arc_points(q, r, circle, concave, n=400):
    """Points of the drop circle (centre q, radius r) lying in the fluid region."""
    t = np.linspace(0, 2 * np.pi, n, endpoint=False)
    p = np.column_stack([q[0] + r * np.cos(t), q[1] + r * np.sin(t)])
    cx, cy, R = circle
    rad = np.hypot(p[:, 0] - cx, p[:, 1] - cy)
    d = (R + 0.5) - rad if concave else rad - (R + 0.5)
    keep = d > 0
    return p[keep], d[keep]


@pytest.mark.parametrize("concave", [False, True])
def test_cap_angle_closed_form(concave):
    """Sec. 4.1 on exact circles: the fitted radius is the drop's, R0 from (4H^2 + L^2)/8H equals
    it, and theta is the circle-circle angle of the law of cosines (convex and cavity)."""
    from helpers import cap_angle_on_circle
    rng = np.random.default_rng(3)
    for _ in range(12):
        R = float(rng.integers(60, 300))
        r = float(rng.uniform(15, 0.5 * R))
        th = float(rng.uniform(40, 140))
        Rs = R + 0.5
        sgn = 1.0 if concave else -1.0
        D = math.sqrt(Rs * Rs + r * r + sgn * 2 * Rs * r * math.cos(math.radians(th)))
        circle = (0.0, 0.0, R)
        q = (0.3, -D) if concave else (0.3, D)
        D = math.hypot(*q)
        p, d = _arc_points(q, r, circle, concave)
        cap = CM.cap_angle(p, d, circle, concave=concave)
        assert cap["r"] == pytest.approx(r, rel=1e-9)
        assert cap["R0"] == pytest.approx(r, rel=1e-7)
        assert cap["theta"] == pytest.approx(cap_angle_on_circle(Rs, r, D, concave), abs=1e-6)


def test_cap_angle_flat_wall():
    r, th = 20.0, 70.0
    q = (5.0, -0.5 - r * math.cos(math.radians(th)))
    t = np.linspace(0, 2 * np.pi, 300, endpoint=False)
    p = np.column_stack([q[0] + r * np.cos(t), q[1] + r * np.sin(t)])
    d = p[:, 1] + 0.5
    cap = CM.cap_angle(p[d > 0], d[d > 0], None)
    assert cap["theta"] == pytest.approx(th, abs=1e-6) and cap["alpha"] == 0


def test_cap_angle_matches_oracle_on_fields(oracle_mod):
    """Host and oracle implementations of Sec. 4.1 on the same synthetic density fields (the
    oracle's Eq. 15 link points as input): same fitted circle and angle."""
    from helpers import tanh_drop
    O = oracle_mod
    mx = O.maxwell(0, 0.7)
    rg, rl = mx["rho_g"], mx["rho_l"]
    rm = 0.5 * (rg + rl)
    cases = [(dict(has_circle=1, cx=100.0, cy=0.0, R=50.0), (100.3, 62.0, 30.0), (0.0, 0.0, 50.0),
              False),
             (dict(has_circle=1, cx=85.0, cy=66.0, R=60.0, concave=1), (85.4, 12.0, 24.0),
              (85.0, 66.0, 60.0), True)]
    for kw, (x0, y0, r), circle, concave in cases:
        cfg = O.Config(nx=200, ny=110, Tr=0.7, **kw)
        rho = tanh_drop(200, 110, x0, y0, r, rg, rl, 6.0)
        ids, pd = O.candidates(cfg, rho, rm)
        circ = (kw["cx"], kw["cy"], kw["R"])
        host = CM.cap_angle(pd[:, :2], pd[:, 2], circ, concave=concave)
        ref = O.cap_angle(cfg, rho, rm)
        assert host["theta"] == pytest.approx(ref["theta"], abs=1e-7)
        assert host["r"] == pytest.approx(ref["r"], rel=1e-9)
