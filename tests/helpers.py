"""Test-side glue: turns a workload description into oracle parameters (and, for the GPU tests,
into the CUDA library's parameters) with the same resolved numbers on both sides."""
from __future__ import annotations

import numpy as np


def oracle_config(O, w, **over):
    """oracle.Config for a workload; wall chemical potentials resolved from the oracle's own
    coexistence value (neutral wall = k^2 psi'(rho_sat))."""
    m = w.model
    mx = O.maxwell(m["eos"], m["Tr"])
    neutral = m["k2"] * mx["mu_sat"]
    kw = dict(nx=w.nx, ny=w.ny, eos=m["eos"], Tr=m["Tr"], k2=m["k2"], kappa=m["kappa"],
              tau=m["tau"], s_e=m["s_e"], s_eps=m["s_eps"], s_q=m["s_q"], gx=w.g[0], gy=w.g[1],
              rho_g=mx["rho_g"], rho_l=mx["rho_l"], g_rho_ref=mx["rho_g"] if w.buoyant else 0.0,
              mu_bottom=neutral + w.mu_rel_bottom, mu_top=neutral + w.mu_rel_top,
              drop_x=w.drop[0], drop_y=w.drop[1], drop_r=w.drop[2], drop_W=w.drop[3])
    if w.circle is not None:
        kw.update(has_circle=1, cx=w.circle[0], cy=w.circle[1], R=w.circle[2],
                  mu_circle=neutral + w.mu_rel_circle)
    if w.stripes is not None:
        kw.update(stripes=1, stripe_arc=w.stripes[0], mu_stripe_b=neutral + w.stripes[1])
    if w.concave:
        kw.update(concave=1)
    kw.update(over)
    return O.Config(**kw), mx, neutral


def tanh_drop(nx, ny, x0, y0, r, rho_g, rho_l, W):
    """Density field of a circular drop with a tanh interface (the Eq. 16 profile), built in the
    test, used as a synthetic input of known geometry."""
    j, i = np.mgrid[0:ny, 0:nx].astype(np.float64)
    d = np.sqrt((i - x0) ** 2 + (j - y0) ** 2)
    return 0.5 * (rho_g + rho_l) + 0.5 * (rho_g - rho_l) * np.tanh(2.0 * (d - r) / W)


def cap_angle_on_circle(Rs, r, D, concave=False):
    """Contact angle (degrees, through the liquid) of a circular drop of radius r whose centre is
    at distance D from the centre of a circular substrate of radius Rs: cos theta is the dot
    product of the wall normal into the fluid and the drop's outward normal at the contact point,
    which the law of cosines in the triangle (substrate centre, drop centre, contact point) gives
    as (Rs^2 + r^2 - D^2) / (2 Rs r) on a convex circle and its negative in a cavity."""
    c = (Rs**2 + r**2 - D**2) / (2.0 * Rs * r)
    return float(np.degrees(np.arccos(np.clip(-c if concave else c, -1, 1))))


def drop_centre_for_angle(Rs, r, theta_deg, cx=0.0, cy=0.0):
    """Centre of a drop of radius r on top of the circle (cx, cy, Rs) meeting it at theta."""
    D = np.sqrt(Rs**2 + r**2 - 2.0 * Rs * r * np.cos(np.radians(theta_deg)))
    return cx, cy + D


def exact_secant_angle(substrate, drop_c, r, d1, d2, side):
    """Closed-form result of the Fig. 1 construction on an exact circular interface: the points
    of the drop circle (centre drop_c, radius r) at distances d1 and d2 from the substrate, the
    line through them, its intersection with the substrate and the angle (degrees) between that
    line and the substrate tangent pointing into the liquid. substrate = ("circle", cx, cy, Rs),
    ("concave", cx, cy, Rs) (fluid inside the circle) or ("flat", y_wall). side 0 = left,
    1 = right (as seen from the liquid standing on the wall)."""
    qx, qy = drop_c
    concave = substrate[0] == "concave"

    def point_at(d):
        if substrate[0] in ("circle", "concave"):
            _, cx, cy, Rs = substrate
            a = Rs - d if concave else Rs + d
            dx, dy = qx - cx, qy - cy
            D = np.hypot(dx, dy)
            l = (a * a - r * r + D * D) / (2 * D)
            h = np.sqrt(max(a * a - l * l, 0.0))
            mx, my = cx + l * dx / D, cy + l * dy / D
            cands = [(mx + h * dy / D, my - h * dx / D), (mx - h * dy / D, my + h * dx / D)]
            # left = counter-clockwise from the wall normal into the fluid, which is the
            # drop-centre direction on a convex circle and its opposite in a cavity
            def cross(p):
                c = dx * (p[1] - cy) - dy * (p[0] - cx)
                return -c if concave else c
            return max(cands, key=cross) if side == 0 else min(cands, key=cross)
        yw = substrate[1]
        y = yw + d
        hx = np.sqrt(max(r * r - (y - qy) ** 2, 0.0))
        return (qx - hx, y) if side == 0 else (qx + hx, y)

    p1, p2 = np.array(point_at(d1)), np.array(point_at(d2))
    v = (p2 - p1) / np.linalg.norm(p2 - p1)
    if substrate[0] in ("circle", "concave"):
        _, cx, cy, Rs = substrate
        w = p1 - np.array([cx, cy])
        wv = w @ v
        disc = wv * wv - (w @ w - Rs * Rs)
        s = min([-wv - np.sqrt(disc), -wv + np.sqrt(disc)], key=abs)
        C = p1 + s * v
        n = (C - np.array([cx, cy])) / Rs * (-1.0 if concave else 1.0)
        t = np.array([n[1], -n[0]]) if side == 0 else np.array([-n[1], n[0]])
    else:
        t = np.array([1.0, 0.0]) if side == 0 else np.array([-1.0, 0.0])
    return float(np.degrees(np.arccos(np.clip(t @ v, -1, 1))))


MODEL_KEYS = ("eos", "Tr", "k2", "kappa", "tau", "s_e", "s_eps", "s_q")


def gpu_lattice(lbm, cfg, precision=0, tile=(0, 0), rho0=None, stream=None, min_blocks=0):
    """CUDA-library lattice with exactly the numbers of an oracle Config (same coexistence
    densities, wall chemical potentials and initial drop)."""
    lat = lbm.Lattice(cfg.nx, cfg.ny, eos=cfg.eos, Tr=cfg.Tr, k2=cfg.k2, kappa=cfg.kappa,
                      tau=cfg.tau, s_e=cfg.s_e, s_eps=cfg.s_eps, s_q=cfg.s_q, gx=cfg.gx,
                      gy=cfg.gy, rho_g=cfg.rho_g, rho_l=cfg.rho_l, precision=precision,
                      collision=cfg.collision, tile=tile, stream=stream,
                      g_rho_ref=cfg.g_rho_ref, min_blocks=min_blocks)
    lat.set_geometry(circle=(cfg.cx, cfg.cy, cfg.R) if cfg.has_circle else None,
                     mu_circle=cfg.mu_circle,
                     stripes=(cfg.stripe_arc, cfg.mu_stripe_b) if cfg.stripes else None,
                     mu_bottom=cfg.mu_bottom, mu_top=cfg.mu_top,
                     drop=(cfg.drop_x, cfg.drop_y, cfg.drop_r, cfg.drop_W), rho0=rho0,
                     concave=bool(cfg.concave), boundary=int(cfg.interp_bb))
    return lat
