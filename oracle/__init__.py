"""FP64 CPU oracle for the multiphase LBM with curved wetting solids (arXiv:2202.06516).

TEST INFRASTRUCTURE ONLY: the slow, literal restatement of the method that the CUDA library is
checked against. Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package. The arithmetic lives in ``lbm_oracle.c`` (plain C, FP64, OpenMP over
rows); this module only builds it and marshals numpy arrays through ctypes. It shares no code with
the CUDA library.

Passages followed: Eq. 1-4 (D2Q9 MRT/BGK collision and streaming), Sec. 2.1 relaxation rates,
Eq. 7 (force), Eq. 10-12 (Peng-Robinson EOS, chemical potential, mesh scaling), Eq. 13
(exact-difference forcing), Eq. 14 (wetting-layer densities), Eq. 15 and Fig. 1 (interface points
and contact point), Fig. 2 (beta = theta + alpha on convex walls), Eq. 16 (initial drop), Sec. 4.1
(spherical-cap method).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field, fields

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

EOS_PR, EOS_CS = 0, 1
MRT, BGK = 0, 1
FLUID, LAYER1, LAYER2, SOLID = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FP contraction, so results are the same on x86 and Arm)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-std=c11", "-D_GNU_SOURCE", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Cfg(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("eos", C.c_int32), ("collision", C.c_int32),
        ("Tr", C.c_double), ("k2", C.c_double), ("kappa", C.c_double), ("tau", C.c_double),
        ("s_e", C.c_double), ("s_eps", C.c_double), ("s_q", C.c_double),
        ("gx", C.c_double), ("gy", C.c_double), ("g_rho_ref", C.c_double),
        ("rho_g", C.c_double), ("rho_l", C.c_double),
        ("has_circle", C.c_int32), ("cx", C.c_double), ("cy", C.c_double), ("R", C.c_double),
        ("mu_circle", C.c_double), ("stripes", C.c_int32), ("stripe_arc", C.c_double),
        ("mu_stripe_b", C.c_double), ("mu_bottom", C.c_double), ("mu_top", C.c_double),
        ("drop_x", C.c_double), ("drop_y", C.c_double), ("drop_r", C.c_double),
        ("drop_W", C.c_double), ("nthreads", C.c_int32), ("concave", C.c_int32),
        ("interp_bb", C.c_int32),
    ]


class _Angle(C.Structure):
    _fields_ = [
        ("status", C.c_int32), ("theta", C.c_double), ("alpha", C.c_double), ("beta", C.c_double),
        ("cx", C.c_double), ("cy", C.c_double), ("p1x", C.c_double), ("p1y", C.c_double),
        ("p2x", C.c_double), ("p2y", C.c_double), ("d1", C.c_double), ("d2", C.c_double),
        ("link1", C.c_int64), ("link2", C.c_int64),
    ]


@dataclass
class Config:
    """Oracle run parameters (lattice units). Defaults: PR EOS, MRT rates of Sec. 2.1."""
    nx: int = 64
    ny: int = 64
    eos: int = EOS_PR
    collision: int = MRT
    Tr: float = 0.7
    k2: float = 0.1
    kappa: float = 0.0126
    tau: float = 1.0
    s_e: float = 1.64
    s_eps: float = 1.54
    s_q: float = 1.9
    gx: float = 0.0
    gy: float = 0.0
    g_rho_ref: float = 0.0
    rho_g: float = 0.0
    rho_l: float = 0.0
    has_circle: int = 0
    cx: float = 0.0
    cy: float = 0.0
    R: float = 0.0
    mu_circle: float = 0.0
    stripes: int = 0
    stripe_arc: float = 40.0
    mu_stripe_b: float = 0.0
    mu_bottom: float = 0.0
    mu_top: float = 0.0
    drop_x: float = 32.0
    drop_y: float = 32.0
    drop_r: float = 10.0
    drop_W: float = 2.0
    nthreads: int = 0
    concave: int = 0
    interp_bb: int = 0

    def _c(self) -> _Cfg:
        c = _Cfg()
        for f in fields(self):
            setattr(c, f.name, getattr(self, f.name))
        return c


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    dp = C.POINTER(C.c_double)
    lib.orc_eos_eval.argtypes = [C.c_int, C.c_double, C.c_double, dp]
    lib.orc_eos_constants.argtypes = [C.c_int, C.c_double, dp]
    lib.orc_maxwell.argtypes = [C.c_int, C.c_double, dp]
    lib.orc_maxwell.restype = C.c_int
    lib.orc_create.argtypes = [C.POINTER(_Cfg), dp]
    lib.orc_create.restype = C.c_void_p
    lib.orc_destroy.argtypes = [C.c_void_p]
    lib.orc_step.argtypes = [C.c_void_p, C.c_int]
    lib.orc_info.argtypes = [C.c_void_p, dp]
    lib.orc_get_rho.argtypes = [C.c_void_p, dp]
    lib.orc_get_ext.argtypes = [C.c_void_p, dp, dp, C.POINTER(C.c_uint8), dp]
    lib.orc_get_f.argtypes = [C.c_void_p, dp]
    lib.orc_set_f.argtypes = [C.c_void_p, dp]
    lib.orc_get_uv.argtypes = [C.c_void_p, dp, dp, dp, dp]
    lib.orc_mass.argtypes = [C.c_void_p]
    lib.orc_mass.restype = C.c_double
    lib.orc_links.argtypes = [C.c_void_p, C.POINTER(C.c_int64), C.c_longlong]
    lib.orc_links.restype = C.c_longlong
    lib.orc_measure.argtypes = [C.POINTER(_Cfg), dp, C.c_double, C.POINTER(_Angle), dp]
    lib.orc_candidates.argtypes = [C.POINTER(_Cfg), dp, C.c_double, C.POINTER(C.c_int64), dp,
                                   C.c_longlong]
    lib.orc_candidates.restype = C.c_longlong
    lib.orc_cap_angle.argtypes = [C.POINTER(_Cfg), dp, C.c_double, C.c_double, dp]
    lib.orc_cap_angle.restype = C.c_int
    lib.orc_threads.restype = C.c_int
    lib.orc_link_fraction.argtypes = [C.POINTER(_Cfg), C.c_int, C.c_int, C.c_int]
    lib.orc_link_fraction.restype = C.c_double
    _lib = lib
    return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def threads() -> int:
    return int(_load().orc_threads())


def eos_eval(eos: int, Tr: float, rho: float) -> dict:
    """psi'(rho) (bulk chemical potential, k = 1), p0, psi and dp0/drho."""
    out = np.zeros(4)
    _load().orc_eos_eval(eos, Tr, rho, _dp(out))
    return {"mu0": out[0], "p0": out[1], "psi": out[2], "dp": out[3]}


def eos_constants(eos: int, Tr: float) -> dict:
    out = np.zeros(5)
    _load().orc_eos_constants(eos, Tr, _dp(out))
    return {"a": out[0], "b": out[1], "R": out[2], "T": out[3], "alpha": out[4]}


def maxwell(eos: int, Tr: float) -> dict:
    """Equal-area coexistence: rho_g, rho_l, p_sat, mu_sat (psi' at coexistence, k = 1)."""
    out = np.zeros(4)
    if _load().orc_maxwell(eos, Tr, _dp(out)) != 0:
        raise ValueError("no coexistence above the critical temperature")
    return {"rho_g": out[0], "rho_l": out[1], "p_sat": out[2], "mu_sat": out[3]}


@dataclass
class Angle:
    status: int
    theta: float
    alpha: float
    beta: float
    contact: tuple
    p1: tuple
    p2: tuple
    d1: float
    d2: float
    link1: int
    link2: int


def _angle(a: _Angle) -> Angle:
    return Angle(a.status, a.theta, a.alpha, a.beta, (a.cx, a.cy), (a.p1x, a.p1y),
                 (a.p2x, a.p2y), a.d1, a.d2, a.link1, a.link2)


def measure(cfg: Config, rho: np.ndarray, rho_m: float):
    """Left and right contact angles of a fluid-domain density field (ny, nx)."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    assert rho.shape == (cfg.ny, cfg.nx)
    out = (_Angle * 2)()
    cen = np.zeros(2)
    c = cfg._c()
    _load().orc_measure(C.byref(c), _dp(rho), rho_m, out, _dp(cen))
    return _angle(out[0]), _angle(out[1]), (cen[0], cen[1])


def candidates(cfg: Config, rho: np.ndarray, rho_m: float):
    """All liquid/gas links in node order: ids (node*4+slot) and (px, py, d) rows."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    cap = 4 * cfg.nx * cfg.ny
    ids = np.zeros(cap, dtype=np.int64)
    pd = np.zeros((cap, 3))
    c = cfg._c()
    n = _load().orc_candidates(C.byref(c), _dp(rho), rho_m,
                               ids.ctypes.data_as(C.POINTER(C.c_int64)), _dp(pd), cap)
    return ids[:n].copy(), pd[:n].copy()


def link_fraction(cfg: Config, i: int, j: int, d: int) -> float:
    """Fraction of the link from fluid node (i, j) along direction d at which it enters the
    analytic solid (interpolated bounce-back)."""
    c = cfg._c()
    return float(_load().orc_link_fraction(C.byref(c), i, j, d))


def cap_angle(cfg: Config, rho: np.ndarray, rho_m: float, dmin: float = 3.0) -> dict:
    """Spherical-cap method of Sec. 4.1 on a density field."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    out = np.zeros(9)
    c = cfg._c()
    if _load().orc_cap_angle(C.byref(c), _dp(rho), rho_m, dmin, _dp(out)) != 0:
        raise ValueError("spherical-cap fit failed")
    keys = ["theta", "beta", "alpha", "L", "H", "R0", "qx", "qy", "r"]
    return dict(zip(keys, out.tolist()))


class Sim:
    """One oracle simulation: geometry, Eq. 16 (or given) initial density, FP64 time steps."""

    def __init__(self, cfg: Config, rho0: np.ndarray | None = None):
        self.cfg = cfg
        self._c = cfg._c()
        lib = _load()
        if rho0 is not None:
            self._rho0 = np.ascontiguousarray(rho0, dtype=np.float64)
            assert self._rho0.shape == (cfg.ny, cfg.nx)
            p = lib.orc_create(C.byref(self._c), _dp(self._rho0))
        else:
            p = lib.orc_create(C.byref(self._c), None)
        if not p:
            raise ValueError("oracle creation failed (no coexistence at this temperature)")
        self._p = C.c_void_p(p)

    def __del__(self):
        if getattr(self, "_p", None) is not None and _lib is not None:
            _lib.orc_destroy(self._p)
            self._p = None

    def step(self, n: int = 1):
        _load().orc_step(self._p, int(n))

    def info(self) -> dict:
        out = np.zeros(8)
        _load().orc_info(self._p, _dp(out))
        return {"rho_g": out[0], "rho_l": out[1], "p_sat": out[2], "mu_sat": out[3],
                "T": out[4], "alpha": out[5], "steps": int(out[6])}

    @property
    def rho_m(self) -> float:
        i = self.info()
        return 0.5 * (i["rho_g"] + i["rho_l"])

    def rho(self) -> np.ndarray:
        out = np.zeros((self.cfg.ny, self.cfg.nx))
        _load().orc_get_rho(self._p, _dp(out))
        return out

    def ext(self):
        """Extended arrays over rows -2..ny+1: rho (incl. wetting layers), mu, flags, mu_w."""
        shp = (self.cfg.ny + 4, self.cfg.nx)
        rho, mu, muw = np.zeros(shp), np.zeros(shp), np.zeros(shp)
        flag = np.zeros(shp, dtype=np.uint8)
        _load().orc_get_ext(self._p, _dp(rho), _dp(mu), flag.ctypes.data_as(C.POINTER(C.c_uint8)),
                            _dp(muw))
        return rho, mu, flag, muw

    def f(self) -> np.ndarray:
        out = np.zeros((self.cfg.ny, self.cfg.nx, 9))
        _load().orc_get_f(self._p, _dp(out))
        return out

    def set_f(self, f: np.ndarray):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.shape == (self.cfg.ny, self.cfg.nx, 9)
        _load().orc_set_f(self._p, _dp(f))

    def velocity_force(self):
        shp = (self.cfg.ny, self.cfg.nx)
        ux, uy, fx, fy = (np.zeros(shp) for _ in range(4))
        _load().orc_get_uv(self._p, _dp(ux), _dp(uy), _dp(fx), _dp(fy))
        return ux, uy, fx, fy

    def mass(self) -> float:
        return float(_load().orc_mass(self._p))

    def links(self) -> np.ndarray:
        cap = 9 * self.cfg.nx * self.cfg.ny
        out = np.zeros(cap, dtype=np.int64)
        n = _load().orc_links(self._p, out.ctypes.data_as(C.POINTER(C.c_int64)), cap)
        return out[:n].copy()

    def measure(self):
        return measure(self.cfg, self.rho(), self.rho_m)
