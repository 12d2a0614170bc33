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
