"""Seeded synthetic workloads shared by the oracle tests, the CUDA parity tests and the benchmark.

This module holds parameters and seeded random draws only, none of the method's arithmetic.
Chemical potentials are given relative to the neutral wall value k^2 * psi'(rho_sat) ("mu_rel");
each caller resolves them with its own coexistence solver.

Readings (stated with the workloads they affect):
* Peng-Robinson EOS at Tr = 0.7 (density ratio 145): Tr = 0.6 and 0.65 diverge at tau = 1 with
  every interface width tried, so the reduced temperature is raised.
* k^2 = 0.05 and kappa-hat = 0.0063 (Eq. 12 leaves both open): equilibrium interface 10-90 %
  width 8.5 lu. With k^2 = 0.1 the 2048 x 1024 drop diverges near step 600 (an acoustic wave
  from the relaxing interface focuses at the drop centre); k^2 = 0.05 is stable past 20k steps.
* Eq. 16 interface width W = 5.6 at start, close to the equilibrium profile (W = 2 diverges
  within a few hundred steps).
* The wall surface lies half a link outside the solid disc, at radius R + 1/2. Small drops start
  tangent to it; large drops (r >= 60) start as a 90-degree cap overlapping it, because the
  tangent start leaves a long thin gas film whose rupture diverges (oracle and GPU alike, near
  step 550 for r = 150 on R = 300).
"""
from __future__ import annotations

from dataclasses import dataclass, field, asdict

import math

import numpy as np

# model parameters common to every workload
MODEL = dict(eos=0, Tr=0.7, k2=0.05, kappa=0.0063, tau=1.0, s_e=1.64, s_eps=1.54, s_q=1.9)
W_INIT = 5.6  # Eq. 16 width matched to the equilibrium interface of MODEL


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    circle: tuple | None          # (cx, cy, R) or None for a flat bottom wall
    drop: tuple                   # (x, y, r, W) of the Eq. 16 initial drop
    mu_rel_circle: float = 0.0    # wall chemical potential minus the neutral value
    mu_rel_bottom: float = 0.0
    mu_rel_top: float = 0.0
    stripes: tuple | None = None  # (arc length, mu_rel of the odd stripes)
    g: tuple = (0.0, 0.0)
    buoyant: bool = False         # body force (rho - rho_g) g instead of rho g
    concave: bool = False         # the circle is a cavity (solid outside it, Fig. 2b)
    steps: int = 3000
    measure_every: int = 0
    model: dict = field(default_factory=lambda: dict(MODEL))

    def as_dict(self):
        return asdict(self)


def tangent_drop(cx, cy, R, r, W=W_INIT):
    """Drop of radius r resting on top of the circle (cx, cy, R), tangent to its surface R + 1/2."""
    return (float(cx), float(cy) + R + 0.5 + r, float(r), float(W))


def cap_drop(cx, cy, R, r, theta0=90.0, W=W_INIT):
    """Drop of radius r on top of the circle (cx, cy, R) overlapping its surface R + 1/2 as a cap
    that meets it at theta0 (law of cosines); used for large drops, where a tangent start leaves
    a long thin gas film whose rupture destabilises the run."""
    Rs = R + 0.5
    D = float(np.sqrt(Rs * Rs + r * r - 2.0 * Rs * r * np.cos(np.radians(theta0))))
    return (float(cx), float(cy) + D, float(r), float(W))


def plain_small() -> Workload:
    """200 x 120, cylinder R = 40 centred on the bottom boundary, drop r = 25, neutral walls,
    3000 steps then one measurement."""
    return Workload("plain-200x120-cyl40-drop25", 200, 120, (100.0, 0.0, 40.0),
                    tangent_drop(100, 0, 40, 25), steps=3000)


# Carnahan-Starling variant of the 200 x 120 workload (a = 1, b = 4, Tr = 0.7, density ratio 38.5).
# k^2 = 0.05 and kappa-hat = 0.05 give a 10-90 % interface width close to the PR model's; the
# Eq. 16 start needs W = 4 here (W = 2 diverges within the 3000 steps, as with PR).
MODEL_CS = dict(eos=1, Tr=0.7, k2=0.05, kappa=0.05, tau=1.0, s_e=1.64, s_eps=1.54, s_q=1.9)
W_INIT_CS = 4.0


def plain_small_cs() -> Workload:
    """The 200 x 120 cylinder workload with the Carnahan-Starling EOS and the MRT collision:
    R = 40 centred on the bottom boundary, drop r = 25 tangent to it, neutral walls, 3000 steps
    then one measurement."""
    return Workload("plain-200x120-cyl40-drop25-cs", 200, 120, (100.0, 0.0, 40.0),
                    tangent_drop(100, 0, 40, 25, W=W_INIT_CS), steps=3000, model=dict(MODEL_CS))


def mu_rel_for_angle(theta_deg: float, slope_per_deg: float = 1.5e-3) -> float:
    """Wall chemical potential offset for a target angle from a linear theta(mu_w) calibration
    (Sec. 4.1 reports theta linear in mu_w): mu_rel = slope * (theta - 90). The slope, 1.5e-3
    per degree, is the fitted dtheta/dmu_w of MODEL on the 200 x 120 cylinder workload."""
    return slope_per_deg * (theta_deg - 90.0)


def plain_large(seed: int = 0, pendent: bool = False) -> Workload:
    """2048 x 1024, cylinder R = 300 on the bottom boundary, drop r = 150, body force 1e-6 toward
    the cylinder (sessile) or away from it (pendent), wetting drawn from the seed for a target
    angle in 40-140 degrees, angle measured every 500 steps."""
    rng = np.random.default_rng(seed)
    theta = float(rng.uniform(40.0, 140.0))
    gy = 1e-6 if pendent else -1e-6
    return Workload(f"plain-2048x1024-cyl300-drop150-{'pendent' if pendent else 'sessile'}-s{seed}",
                    2048, 1024, (1024.0, 0.0, 300.0), cap_drop(1024, 0, 300, 150),
                    mu_rel_circle=mu_rel_for_angle(theta), g=(0.0, gy), steps=50000,
                    measure_every=500)


# Wall potential of the hydrophilic stripes of the hysteresis workload. The linear calibration
# (mu_rel_for_angle) is accurate on the hydrophobic side (mu_rel +0.045 gives 116-120 degrees on
# a uniform R = 800 cylinder with an r = 120 drop) but overshoots on the hydrophilic side there
# (mu_rel_for_angle(60) = -0.045 gives 46-50 degrees); -0.03 gives 58-60 degrees.
HYST_MU_REL_60 = -0.03


def hysteresis(heterogeneous: bool = True) -> Workload:
    """Dynamic contact-angle hysteresis on a curved surface (Sec. 4.4): 4096 x 1024, periodic in
    x, cylinder R = 800 whose wall alternates 60- and 120-degree stripes of arc length 40
    (heterogeneous) or is uniformly 120 degrees, drop r = 120 started as a 90-degree cap on top.
    The substrate is tilted by the slope angle 20 degrees: gravity makes 20 degrees with the
    vertical, g = G (sin 20, -cos 20) with G sin 20 = 5e-7 (the tangential component at the top),
    so the normal component keeps the drop pressed to the cylinder while it slides right; at this
    G the uniform-wall drop reaches the foot of the cylinder near the end of the 200k steps. The
    force acts on the density above the gas density (the full weight rho g along the periodic
    axis would drive the gas through the channel without bound). The cylinder centre sits 100 lu
    below the bottom boundary so that the drop fits under the top wall. Advancing (right) and
    receding (left) angles every 100 steps for 200k steps."""
    cx, cy, R, r = 2048.0, -100.0, 800.0, 120.0
    phi = math.radians(20.0)
    G = 5e-7 / math.sin(phi)
    stripes = (40.0, HYST_MU_REL_60) if heterogeneous else None
    name = "hysteresis-4096x1024-cyl800-" + ("stripes60-120" if heterogeneous else "uniform120")
    return Workload(name, 4096, 1024, (cx, cy, R), cap_drop(cx, cy, R, r),
                    mu_rel_circle=mu_rel_for_angle(120.0), stripes=stripes,
                    g=(G * math.sin(phi), -G * math.cos(phi)), buoyant=True, steps=200000, measure_every=100)


def sweep_instance(R: float, r: float, target_deg: float, concave: bool) -> Workload:
    """One drop of radius r at rest on a convex cylinder of radius R centred on the bottom
    boundary, or at the bottom of a circular cavity of radius R whose lowest wall point sits
    5.5 lu above the bottom boundary (Fig. 2b). The drop starts where an exact circle of radius
    r meets the wall surface (R + 1/2) at the target angle (law of cosines; |D| from the
    circle-circle angle), and the wall potential is mu_rel_for_angle(target)."""
    Rs, t = R + 0.5, math.radians(target_deg)
    if concave:
        nx, ny = int(2 * R + 20), int(3 * r + 40)
        nx += nx % 2
        cx, cy = nx / 2.0, R + 6.0
        D = math.sqrt(Rs * Rs + r * r + 2.0 * Rs * r * math.cos(t))
        drop = (cx, cy - D, r, W_INIT)
    else:
        nx, ny = int(2 * R + 4 * r + 40), int(R + 3 * r + 40)
        nx += nx % 2
        cx, cy = nx / 2.0, 0.0
        D = math.sqrt(Rs * Rs + r * r - 2.0 * Rs * r * math.cos(t))
        drop = (cx, cy + D, r, W_INIT)
    kind = "cavity" if concave else "cyl"
    return Workload(f"{kind}{R:g}-r{r:g}-theta{target_deg:g}", nx, ny, (cx, cy, R), drop,
                    mu_rel_circle=mu_rel_for_angle(target_deg), concave=concave,
                    steps=30000, measure_every=1000)


def curvature_sweep(targets=(70.0, 90.0, 110.0, 130.0, 150.0), radii=(150.0, 250.0, 400.0),
                    drops=(30.0, 50.0, 70.0, 100.0)) -> list[Workload]:
    """Grid-independence / curvature sweep (Sec. 4.1-4.2: drops of 30-100 lu on substrates of
    radius 150-400 lu, hydrophilic to superhydrophobic), on convex cylinders and in cavities.
    Drops larger than half the substrate radius are left out so that no wetted arc reaches the
    foot of the cylinder. (A 50-degree target wets the small cylinders into films: the drop
    spreads down the sides and neither the measurement nor a cap fit describes a drop.)"""
    out = []
    for concave in (False, True):
        for t in targets:
            for R in radii:
                for r in drops:
                    if r <= 0.5 * R:
                        out.append(sweep_instance(R, r, t, concave))
    return out


def gravity_sweep(targets=(70.0, 100.0, 140.0), drops=(20.0, 40.0, 60.0, 80.0, 100.0, 120.0),
                  R=150.0, G=1e-6) -> dict:
    """Sessile and pendent drops of growing size on a cylinder (Sec. 4.3): for each wall potential
    and drop radius, a drop started as a 90-degree cap on top of a cylinder of radius R centred on
    the bottom boundary. Three body-force settings share the instances: none, toward the
    cylinder (sessile) and away from it (pendent: the paper's drop beneath the substrate with
    gravity reversed, turned upside down). Returns {"instances": [...], "g": {...}}."""
    out = []
    for t in targets:
        for r in drops:
            nx, ny = int(2 * R + 4 * r + 40), int(R + 4 * r + 40)
            nx += nx % 2
            cx = nx / 2.0
            out.append(Workload(f"cyl{R:g}-r{r:g}-theta{t:g}", nx, ny, (cx, 0.0, R),
                                cap_drop(cx, 0.0, R, r), mu_rel_circle=mu_rel_for_angle(t),
                                steps=60000, measure_every=1000))
    return {"instances": out, "g": {"none": (0.0, 0.0), "sessile": (0.0, -G), "pendent": (0.0, G)}}


def flat_drop(nx=160, ny=80, r=20.0, theta_rel=0.0) -> Workload:
    """Drop on a flat bottom wall (no cylinder)."""
    return Workload(f"flat-{nx}x{ny}-drop{r:g}", nx, ny, None, (nx / 2.0, -0.5 + r, r, W_INIT),
                    mu_rel_bottom=theta_rel)


def batched(n: int = 256, seed: int = 0) -> list[Workload]:
    """Independent instances with domain 128..768 x 128..512, cylinder radius 20..200, drop radius
    15..90 and target angle 30..150 degrees, rejection-resampled until 2 R + 16 <= nx and
    R + 2 r + 8 <= ny (the drawn ranges otherwise overlap the domain walls)."""
    out = []
    for i in range(n):
        rng = np.random.default_rng([seed, i])
        while True:
            nx = int(rng.integers(128, 769))
            ny = int(rng.integers(128, 513))
            R = float(rng.integers(20, 201))
            r = float(rng.integers(15, 91))
            if 2 * R + 16 <= nx and R + 2 * r + 8 <= ny:
                break
        theta = float(rng.uniform(30.0, 150.0))
        cx = float(nx // 2)
        drop = cap_drop(cx, 0, R, r) if r >= 60 else tangent_drop(cx, 0, R, r)
        out.append(Workload(f"batch{seed}-{i}", nx, ny, (cx, 0.0, R), drop,
                            mu_rel_circle=mu_rel_for_angle(theta), steps=40000))
    return out


# ----------------------------------------------------------------------- warm-start surrogate
def unet_layers(base: int = 32):
    """(c_in, c_out) of the U-Net's 3x3 convolutions in forward order (encoder 4 levels of two
    convolutions with base, 2, 4, 8 x base channels; decoder per level one convolution of the
    upsampled coarser output and two on [that | skip]), input with 8 channels."""
    b = base
    return [(8, b), (b, b), (b, 2 * b), (2 * b, 2 * b), (2 * b, 4 * b), (4 * b, 4 * b),
            (4 * b, 8 * b), (8 * b, 8 * b), (8 * b, 4 * b), (8 * b, 4 * b), (4 * b, 4 * b),
            (4 * b, 2 * b), (4 * b, 2 * b), (2 * b, 2 * b), (2 * b, b), (2 * b, b), (b, b)]


def unet_init(base: int = 32, seed: int = 0) -> np.ndarray:
    """Seeded initial weights (He-normal convolutions, zero biases, small head) as one FP32
    vector: per convolution [c_out][ky][kx][c_in] then bias[c_out]; head weight[base], bias[1]."""
    rng = np.random.default_rng(seed)
    out = []
    for ci, co in unet_layers(base):
        out.append(rng.normal(0.0, np.sqrt(2.0 / (9 * ci)), size=co * 9 * ci))
        out.append(np.zeros(co))
    out.append(rng.normal(0.0, 0.01, size=base))
    out.append(np.zeros(1))
    return np.concatenate(out).astype(np.float32)


def warm_cases(n: int, seed: int, size: int = 256):
    """Cases for the warm-start surrogate: the batched ranges (domain 128..768 x 128..512,
    R 20..200, r 15..90, target angle 30..150 degrees) rescaled to a size x size lattice by
    s = size / max(nx, ny), rejection-resampled until the scaled cylinder and drop fit
    (2 R + 16 <= size, R + 2 r + 8 <= size) and the drop keeps r >= 12 (a smaller drop is mostly
    interface at the 8.5 lu interface width). Seeds seed, seed+1, ... give case 0, 1, ..."""
    out = []
    for i in range(n):
        rng = np.random.default_rng([seed, i, 7])
        while True:
            nx = int(rng.integers(128, 769))
            ny = int(rng.integers(128, 513))
            R = float(rng.integers(20, 201))
            r = float(rng.integers(15, 91))
            theta = float(rng.uniform(30.0, 150.0))
            s = size / max(nx, ny)
            Rs = round(2 * R * s) / 2
            rs = r * s
            if Rs >= 4 and 2 * Rs + 16 <= size and Rs + 2 * rs + 8 <= size and rs >= 12:
                break
        cx = size / 2
        drop = cap_drop(cx, 0, Rs, rs) if rs >= 60 else tangent_drop(cx, 0, Rs, rs)
        out.append(Workload(f"warm{seed}-{i}", size, size, (cx, 0.0, Rs), drop,
                            mu_rel_circle=mu_rel_for_angle(theta), steps=20000))
    return out
