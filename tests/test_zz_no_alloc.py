"""lbm_mass_noalloc: the density sums for callers that must not allocate device memory.

Some callers cannot call cudaMalloc where they need the sums: a framework whose memory pool owns
every device byte, code that cannot take the implicit synchronisation of cudaMalloc/cudaFree, or
a process that has budgeted the whole GPU. lbm_mass_noalloc keeps its scratch in a fixed device
array inside the library, and the caller passes the density field, the node flags and a device
output. This test calls it through the C ABI on caller-owned torch tensors and checks it against
the existing lbm_mass of a context holding the same field, on two calls in a row (the second
call reuses the scratch the first one left behind). It lives in its own file, collected last.
"""
import ctypes as C

import numpy as np
import pytest

from helpers import gpu_lattice, oracle_config
from paper_2202_06516_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _entry(lbm):
    L = lbm.lib()
    f = L.lbm_mass_noalloc
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_double,
                  C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    return f


def test_noalloc_sums_match_lbm_mass_twice(oracle_mod):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2202_06516_gb300 import lbm
    fn = _entry(lbm)
    cfg = oracle_config(oracle_mod, W.plain_small())[0]
    nx, ny = cfg.nx, cfg.ny
    lat = gpu_lattice(lbm, cfg)
    flags_ext, _, _ = lat.geometry()
    flags = torch.from_numpy(np.ascontiguousarray(flags_ext[2:-2])).cuda()
    rho_m = 0.5 * (cfg.rho_g + cfg.rho_l)
    stream = torch.cuda.current_stream()
    out = torch.full((5,), -1.0, dtype=torch.float64, device="cuda")
    for steps in (100, 137):
        lat.step(steps)
        rho64 = torch.empty(ny * nx, dtype=torch.float64, device="cuda")
        lbm.lbm_read_fields(lat.ctx, lbm.LBM_FIELD_RHO, nx, ny,
                            device_out=(rho64.data_ptr(), None, None))
        rho32 = rho64.to(torch.float32)  # exact: the library's density plane is FP32
        st = fn(rho32.data_ptr(), flags.data_ptr(), nx, ny, nx, rho_m, out.data_ptr(),
                stream.cuda_stream)
        assert st == lbm.LBM_OK, lbm.lbm_last_error(None)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        want = lat.mass()  # the existing entry point, same field
        assert got[0] == pytest.approx(want["mass"], rel=1e-12)
        assert got[1] == want["n_liquid"]
        assert got[2] == pytest.approx(want["cx"], rel=1e-12)
        assert got[3] == pytest.approx(want["cy"], rel=1e-12)
        assert got[4] == 0.0
        # and the oracle's definitions on the same FP32 values: its mass of a lattice started
        # from this field and the liquid centroid its measurement uses
        rho_h = rho32.double().cpu().numpy().reshape(ny, nx)
        omass = oracle_mod.Sim(cfg, rho0=rho_h).mass()
        _, _, ocen = oracle_mod.measure(cfg, rho_h, rho_m)
        fluid = flags_ext[2:-2] == 0
        assert got[0] == pytest.approx(omass, rel=1e-12)
        assert got[1] == int((fluid & (rho_h > rho_m)).sum())
        assert got[2] == pytest.approx(ocen[0], rel=1e-12)
        assert got[3] == pytest.approx(ocen[1], rel=1e-12)
    lat.close()


def test_noalloc_pitch_bad_values_and_lbm_mass_status(oracle_mod):
    """Rows wider than the domain (pitch > nx) whose padding holds sentinel values that would
    show if summed; a NaN and a negative density are counted in out[4], and lbm_mass on a context
    loaded with the same field reports LBM_ERR_UNSTABLE."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2202_06516_gb300 import lbm
    fn = _entry(lbm)
    cfg = oracle_config(oracle_mod, W.plain_small())[0]
    nx, ny = cfg.nx, cfg.ny
    rho_h = oracle_mod.Sim(cfg).rho().astype(np.float32)
    lat = gpu_lattice(lbm, cfg)
    flags_h = np.ascontiguousarray(lat.geometry()[0][2:-2])
    stream = torch.cuda.current_stream()
    rho_m = 0.5 * (cfg.rho_g + cfg.rho_l)
    out = torch.full((5,), -1.0, dtype=torch.float64, device="cuda")

    def call(rho2d, flags2d, pitch):
        st = fn(rho2d.data_ptr(), flags2d.data_ptr(), nx, ny, pitch, rho_m, out.data_ptr(),
                stream.cuda_stream)
        assert st == lbm.LBM_OK, lbm.lbm_last_error(None)
        torch.cuda.synchronize()
        return out.cpu().numpy().copy()

    tight = call(torch.from_numpy(rho_h).cuda(), torch.from_numpy(flags_h).cuda(), nx)
    pitch = nx + 13
    rp = np.full((ny, pitch), 1e30, dtype=np.float32)
    fp = np.zeros((ny, pitch), dtype=np.uint8)  # padding marked fluid: it must still be skipped
    rp[:, :nx] = rho_h
    fp[:, :nx] = flags_h
    wide = call(torch.from_numpy(rp).cuda(), torch.from_numpy(fp).cuda(), pitch)
    assert np.array_equal(tight, wide)
    assert tight[4] == 0.0
    bad = rho_h.copy()
    bad[ny - 10, 7] = np.nan
    bad[ny - 12, 9] = -0.5
    assert flags_h[ny - 10, 7] == 0 and flags_h[ny - 12, 9] == 0
    got = call(torch.from_numpy(bad).cuda(), torch.from_numpy(flags_h).cuda(), nx)
    assert got[4] == 2.0
    lat.set_geometry(circle=(cfg.cx, cfg.cy, cfg.R), mu_circle=cfg.mu_circle,
                     mu_bottom=cfg.mu_bottom, mu_top=cfg.mu_top,
                     rho0=bad.astype(np.float64))
    st, _ = lbm.lbm_mass(lat.ctx, allow_unstable=True)
    assert st == lbm.LBM_ERR_UNSTABLE
    lat.close()


def test_noalloc_rejects_oversize(oracle_mod):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2202_06516_gb300 import lbm
    fn = _entry(lbm)
    big = 4096 + 1
    rho = torch.ones(big * 8, dtype=torch.float32, device="cuda")
    flags = torch.zeros(big * 8, dtype=torch.uint8, device="cuda")
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    st = fn(rho.data_ptr(), flags.data_ptr(), 8, big, 8, 0.5, out.data_ptr(), None)
    assert st == lbm.LBM_ERR_ARG
    assert "LBM_NOALLOC_MAX_ROWS" in lbm.lbm_last_error(None)
