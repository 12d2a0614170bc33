"""Mechanical analysis at a moving contact line (Sec. 4.5).

The unbalanced Young's force of Eq. 17 is evaluated on the contact angles the device measures
(Sec. 3.2), with the equilibrium angle taken from the wettability under the contact region: the
intrinsic angle of a homogeneous stretch of wall, or the modified Cassie-Baxter mean of Eq. 18
where the liquid-gas transition region straddles two wettabilities. The liquid-gas surface
tension comes from Laplace's law on free drops simulated by the CUDA library.

Conventions (the paper states Eq. 17 as a magnitude and fixes the sign in words: x points right,
an advancing angle above its equilibrium value gives a positive force, a receding angle above
it a negative one). The force per unit length on the contact line along the wall, toward the
gas, is gamma (cos theta_eq - cos theta); its x-component is that for the right contact line
and minus that for the left one.

Everything here is host post-processing of a few numbers per measurement; the lattice runs go
through the C ABI (``lbm``)."""
from __future__ import annotations

import math

import numpy as np

from . import lbm as L

LEFT, RIGHT = 0, 1


# ----------------------------------------------------------------------------- wall geometry
def arc_coordinate(x, y, circle):
    """Arc coordinate of a point seen from the circle centre, in the units the geometry uses to
    lay out stripes: R (phi - pi/2), phi = atan2(y - cy, x - cx), counter-clockwise from the
    apex (a wall node belongs to stripe floor(s / arc); even stripes carry the circle's own
    wettability, odd stripes the second one)."""
    cx, cy, R = circle
    return R * (np.arctan2(np.asarray(y, float) - cy, np.asarray(x, float) - cx) - 0.5 * math.pi)


def odd_stripe_length(s, arc):
    """Signed length of [0, s] covered by odd stripes (floor(s'/arc) odd): the antiderivative of
    the odd-stripe indicator, so that the odd length of [a, b] is F(b) - F(a) for any a <= b,
    including negative coordinates."""
    s = np.asarray(s, float)
    p = np.floor(s / (2.0 * arc))
    rem = s - 2.0 * arc * p                      # in [0, 2 arc)
    return p * arc + np.clip(rem - arc, 0.0, arc)


def odd_fraction(s_lo, s_hi, arc):
    """Fraction of the interval [s_lo, s_hi] lying on odd stripes (phi_d of Eq. 18 when the odd
    stripes carry theta_s1)."""
    s_lo, s_hi = np.asarray(s_lo, float), np.asarray(s_hi, float)
    span = s_hi - s_lo
    frac = (odd_stripe_length(s_hi, arc) - odd_stripe_length(s_lo, arc)) / np.where(span > 0,
                                                                                    span, 1.0)
    point = (np.floor(s_lo / arc) % 2 == 1).astype(float)
    return np.where(span > 0, frac, point)


def interface_footprint(width, theta_deg):
    """Length along a wall of a liquid-gas transition band of thickness `width` that meets the
    wall at theta (a straight band cut by a line at angle theta): width / sin theta."""
    return width / np.sin(np.radians(theta_deg))


# ------------------------------------------------------------------------ Eq. 17 and Eq. 18
def cassie_baxter(phi_d, theta_s1_deg, theta_s2_deg, roughness=1.0):
    """Eq. 18: cos theta_eq = r phi_d cos theta_s1 + (1 - phi_d) cos theta_s2 (degrees; r = 1 for
    a smooth wall)."""
    c = (roughness * np.asarray(phi_d, float) * np.cos(np.radians(theta_s1_deg))
         + (1.0 - np.asarray(phi_d, float)) * np.cos(np.radians(theta_s2_deg)))
    return np.degrees(np.arccos(np.clip(c, -1.0, 1.0)))


def young_force_x(theta_deg, theta_eq_deg, gamma, side):
    """x-component of the unbalanced Young's force per unit length (Eq. 17) on the left
    (side = 0) or right (side = 1) contact line."""
    f = gamma * (np.cos(np.radians(theta_eq_deg)) - np.cos(np.radians(theta_deg)))
    return np.where(np.asarray(side) == RIGHT, f, -f)


def equilibrium_angle(contact_x, contact_y, circle, theta_circle_deg, stripes=None,
                      width=0.0, theta_deg=90.0):
    """Equilibrium angle under a contact point on the circle, and phi_d.

    stripes = (arc, theta_stripe_deg) for a wall alternating theta_circle (even stripes) and
    theta_stripe (odd stripes); None for a uniform wall (phi_d = 0). The contact region is the
    footprint of the transition band (`interface_footprint(width, theta)`) centred on the
    contact point, converted from the wall surface (radius R + 1/2) to arc coordinates."""
    x, y = np.asarray(contact_x, float), np.asarray(contact_y, float)
    if stripes is None:
        return np.full(np.broadcast(x, y).shape, float(theta_circle_deg)), np.zeros_like(x + y)
    arc, theta_stripe = stripes
    R = circle[2]
    s = arc_coordinate(x, y, circle)
    half = 0.5 * interface_footprint(width, theta_deg) * R / (R + 0.5)
    phi = odd_fraction(s - half, s + half, arc)
    return cassie_baxter(phi, theta_stripe, theta_circle_deg), phi


# -------------------------------------------------------------------- Laplace surface tension
def _profile_width(row, centre, lo=0.1, hi=0.9):
    """Distance between the hi and lo crossings of a normalised profile that falls from 1 at
    `centre` outward (linear interpolation between nodes)."""
    def crossing(level):
        for i in range(centre, len(row) - 1):
            if row[i] >= level > row[i + 1]:
                return i + (row[i] - level) / (row[i] - row[i + 1])
        raise ValueError("profile does not cross the level")
    return crossing(lo) - crossing(hi)


def laplace_tension(model: dict, radii=(20.0, 30.0), steps: int = 20000, W: float = 5.6,
                    margin: int = 40, precision: int = L.LBM_FP32) -> dict:
    """Liquid-gas surface tension from Laplace's law (2D: Delta p = gamma / R) on free drops run
    by the CUDA library: square periodic-x domains with neutral top and bottom walls, no body
    force, one drop per radius started as the Eq. 16 profile.

    After `steps` steps: Delta p = k^2 (p0(rho_in) - p0(rho_out)) from the host EOS at the drop
    centre and far from it, R from the excess density (area of the drop), the 10-90 % width of
    the interface along the centre row. gamma is the mean of Delta p R; `spread` is the relative
    difference of Delta p R between the radii (Laplace's law holds if it is small).

    model: the keys of ``workloads.MODEL`` (eos, Tr, k2, kappa, tau, s_e, s_eps, s_q)."""
    co = L.lbm_coexistence(model["eos"], model["Tr"])
    neutral = model["k2"] * co["mu_sat"]
    out = []
    for r0 in radii:
        N = int(2 * r0 + 2 * margin)
        lat = L.Lattice(N, N, eos=model["eos"], Tr=model["Tr"], k2=model["k2"],
                        kappa=model["kappa"], tau=model["tau"], s_e=model["s_e"],
                        s_eps=model["s_eps"], s_q=model["s_q"], precision=precision)
        try:
            lat.set_geometry(circle=None, mu_bottom=neutral, mu_top=neutral,
                             drop=(N / 2.0, N / 2.0 - 0.5, float(r0), W))
            lat.step(steps)
            rho = lat.rho()
        finally:
            lat.close()
        c = N // 2
        rin, rout = rho[c, c], rho[c, 2]
        p_in = L.lbm_eos_eval(model["eos"], model["Tr"], rin)["p0"]
        p_out = L.lbm_eos_eval(model["eos"], model["Tr"], rout)["p0"]
        dp = model["k2"] * (p_in - p_out)
        phi = (rho - rout) / (rin - rout)
        Rm = math.sqrt(phi.sum() / math.pi)
        out.append({"r0": float(r0), "N": N, "rho_in": float(rin), "rho_out": float(rout),
                    "dp": float(dp), "R": Rm, "dp_R": float(dp * Rm),
                    "width_10_90": float(_profile_width(phi[c], c))})
    prs = np.array([o["dp_R"] for o in out])
    return {"gamma": float(prs.mean()),
            "spread": float((prs.max() - prs.min()) / prs.mean()) if len(prs) > 1 else 0.0,
            "width_10_90": float(np.mean([o["width_10_90"] for o in out])),
            "drops": out}


# ---------------------------------------------------------------- spherical-cap method (4.1)
def cap_angle(points, d, circle, concave=False, dmin=3.0) -> dict:
    """Spherical-cap estimate of the contact angle (Sec. 4.1), the benchmark the measurement is
    compared with: a circle fitted (algebraic least squares, x^2 + y^2 + D x + E y + F = 0) to
    the drop's interface points farther than dmin from the wall, its chord with the wall
    surface (radius R + 1/2) of length L, the drop height H above the chord along the wall
    normal into the fluid, R0 = (4 H^2 + L^2) / (8 H), tan(beta) = L / (2 (R0 - H)),
    alpha = asin(L / (2 (R + 1/2))) and theta = beta - alpha on a convex wall, beta + alpha in a
    cavity (Fig. 2). circle = (cx, cy, R) or None for the flat bottom wall y = -1/2 (alpha = 0).

    points: (n, 2) interface points (Eq. 15 link points); d: their distances from the wall."""
    p = np.asarray(points, float)[np.asarray(d, float) >= dmin]
    if len(p) < 3:
        raise ValueError("cap_angle: fewer than three interface points away from the wall")
    A = np.column_stack([p[:, 0], p[:, 1], np.ones(len(p))])
    z = -(p[:, 0] ** 2 + p[:, 1] ** 2)
    (Dc, Ec, Fc), *_ = np.linalg.lstsq(A, z, rcond=None)
    qx, qy = -0.5 * Dc, -0.5 * Ec
    rr = math.sqrt(qx * qx + qy * qy - Fc)
    if circle is not None:
        cx, cy, R = circle
        Rs = R + 0.5
        dx, dy = qx - cx, qy - cy
        D = math.hypot(dx, dy)
        if not (abs(Rs - rr) < D < Rs + rr):
            raise ValueError("cap_angle: fitted drop does not cut the wall")
        a = (Rs * Rs - rr * rr + D * D) / (2.0 * D)
        h = math.sqrt(Rs * Rs - a * a)
        mx, my = cx + a * dx / D, cy + a * dy / D          # chord midpoint
        L = 2.0 * h
        nx_, ny_ = (mx - cx) / a, (my - cy) / a            # outward normal of the circle
        if concave:
            nx_, ny_ = -nx_, -ny_
        alpha = math.asin(min(1.0, L / (2.0 * Rs)))
    else:
        dy = -0.5 - qy
        if abs(dy) >= rr:
            raise ValueError("cap_angle: fitted drop does not cut the wall")
        L = 2.0 * math.sqrt(rr * rr - dy * dy)
        mx, my, nx_, ny_, alpha = qx, -0.5, 0.0, 1.0, 0.0
    H = rr + (qx - mx) * nx_ + (qy - my) * ny_
    R0 = (4.0 * H * H + L * L) / (8.0 * H)
    beta = math.atan2(L, 2.0 * (R0 - H))
    theta = beta + alpha if (circle is not None and concave) else beta - alpha
    return {"theta": math.degrees(theta), "beta": math.degrees(beta),
            "alpha": math.degrees(alpha), "L": L, "H": H, "R0": R0, "qx": qx, "qy": qy, "r": rr,
            "points": int(len(p))}


# ------------------------------------------------------------------ intrinsic contact angle
def intrinsic_angle(model: dict, mu_rel: float, R: float = 800.0, r: float = 120.0,
                    steps: int = 40000, samples: int = 10, every: int = 2000,
                    precision: int = L.LBM_FP32, concave: bool = False,
                    boundary: int = L.LBM_BB_HALFWAY, offset=(0.0, 0.0)) -> dict:
    """Equilibrium contact angle a uniform wall of chemical potential neutral + mu_rel produces
    (theta_s of Eq. 18): a drop of radius r started as a 90-degree cap on a cylinder of radius R
    centred on the bottom boundary (convex), or at the bottom of a circular cavity of radius R
    whose lowest wall point sits 5.5 lu above the bottom boundary (concave, Fig. 2b); no body
    force. After `steps` steps the device measures both angles `samples` times, `every` steps
    apart (the contact lines creep across the staircase wall, so single readings scatter by a
    few degrees); returns the means and the scatter. offset shifts the circle centre by
    multiples of 1/2 (a different staircase of the same circle); boundary selects the curved-wall
    scheme (LBM_BB_HALFWAY or LBM_BB_INTERP)."""
    co = L.lbm_coexistence(model["eos"], model["Tr"])
    neutral = model["k2"] * co["mu_sat"]
    if concave:
        nx, ny = int(2 * R + 20), int(3 * r + 40)
        nx += nx % 2
        cx, cy = nx / 2.0 + offset[0], R + 6.0 + offset[1]
        drop_c = (cx, cy - R - 0.5)
    else:
        nx, ny = int(2 * R + 4 * r + 40), int(R + 3 * r + 40)
        nx += nx % 2
        cx, cy = nx / 2.0 + offset[0], 0.0 + offset[1]
        drop_c = (cx, cy + R + 0.5)
    lat = L.Lattice(nx, ny, eos=model["eos"], Tr=model["Tr"], k2=model["k2"],
                    kappa=model["kappa"], tau=model["tau"], s_e=model["s_e"],
                    s_eps=model["s_eps"], s_q=model["s_q"], precision=precision)
    readings = []
    try:
        # 90-degree cap: centre on the wall surface R + 1/2 straight above (convex) or below
        # (concave) the circle centre
        lat.set_geometry(circle=(cx, cy, R), mu_circle=neutral + mu_rel, mu_bottom=neutral,
                         mu_top=neutral, drop=(drop_c[0], drop_c[1], float(r), 5.6),
                         concave=concave, boundary=boundary)
        lat.step(steps)
        for k in range(samples):
            if k:
                lat.step(every)
            left, right = lat.measure()
            if left.status != 0 or right.status != 0:
                raise RuntimeError("intrinsic_angle: no contact line on one side")
            readings.append((left.theta, right.theta))
    finally:
        lat.close()
    a = np.array(readings)
    return {"left": float(a[:, 0].mean()), "right": float(a[:, 1].mean()),
            "theta": float(a.mean()), "scatter": float(a.mean(axis=1).std()),
            "nx": nx, "ny": ny, "R": R, "r": r, "concave": concave,
            "steps": steps + (samples - 1) * every}


# ------------------------------------------------------------------------ series analysis
def analyse_series(series: np.ndarray, circle, theta_circle_deg, stripes, gamma, width):
    """Young's force along a measured angle series.

    series columns: left status, theta_left, right status, theta_right, contact x left, contact
    x right, contact y left, contact y right (one row per measurement). Rows where a side has no
    contact give NaN for that side. Returns per side (left, right) arrays theta_eq, phi_d and
    the force x-component, plus a region label: 0 on the circle's own wettability, 1 on the
    odd stripes, 2 on a border (0 < phi_d < 1)."""
    series = np.asarray(series, float)
    res = {}
    for side, (st, th, cxi, cyi) in ((LEFT, (0, 1, 4, 6)), (RIGHT, (2, 3, 5, 7))):
        ok = series[:, st] == 0
        theta = np.where(ok, series[:, th], np.nan)
        teq, phi = equilibrium_angle(series[:, cxi], series[:, cyi], circle, theta_circle_deg,
                                     stripes, width, np.where(ok, theta, 90.0))
        teq = np.where(ok, teq, np.nan)
        phi = np.where(ok, phi, np.nan)
        force = np.where(ok, young_force_x(theta, teq, gamma, side), np.nan)
        region = np.where(~ok, -1, np.where(phi <= 0.0, 0, np.where(phi >= 1.0, 1, 2)))
        res["left" if side == LEFT else "right"] = {"theta": theta, "theta_eq": teq,
                                                     "phi_d": phi, "force": force,
                                                     "region": region}
    return res
