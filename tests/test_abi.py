"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports every entry point that
include/lbm.h declares, and its host-only parts behave (no kernel is launched here)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("lbm_create", "lbm_set_geometry", "lbm_step", "lbm_measure_contact_angle",
              "lbm_read_fields", "lbm_destroy", "lbm_last_error"):
        assert n in names


@pytest.mark.parametrize("lang,std", [("c", "-std=c11"), ("c++", "-std=c++17")])
def test_header_compiles_standalone(lang, std):
    """include/lbm.h is a plain C header: it compiles on its own as C11 and as C++17."""
    import shutil
    import subprocess
    cc = shutil.which("gcc" if lang == "c" else "g++")
    if cc is None:
        pytest.skip("no host compiler")
    r = subprocess.run([cc, "-fsyntax-only", "-x", lang, std, "-Wall", "-Wextra", "-Werror",
                        os.path.join(ROOT, "include", "lbm.h")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_struct_layouts_match_the_binding(tmp_path):
    """Every public struct of include/lbm.h has, in the ctypes binding, the same size and the
    same field offsets as the C compiler gives it (fields are appended over time; a mismatch
    would silently shift every later field)."""
    import shutil
    import subprocess
    from paper_2202_06516_gb300 import lbm
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no host compiler")
    structs = [lbm.lbm_params, lbm.lbm_geometry, lbm.lbm_angle, lbm.lbm_info, lbm.lbm_tune_entry]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lbm.h"', "int main(void) {"]
    for st in structs:
        n = st.__name__
        lines.append(f'printf("{n} size %zu\\n", sizeof({n}));')
        for f, _ in st._fields_:
            lines.append(f'printf("{n} {f} %zu\\n", offsetof({n}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                        str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            n, f, v = line.split()
            got[(n, f)] = int(v)
    for st in structs:
        n = st.__name__
        assert got[(n, "size")] == ctypes.sizeof(st), n
        for f, _ in st._fields_:
            assert got[(n, f)] == getattr(st, f).offset, (n, f)


def test_library_exports_every_declared_symbol():
    from paper_2202_06516_gb300 import _native
    lib = _native.load()
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_coexistence_agrees_with_oracle(oracle_mod):
    """The library's host Maxwell solver (parametrised by mu) and the oracle's (bisection on p)
    are independent; they must agree to near round-off."""
    from paper_2202_06516_gb300 import lbm
    for eos, Tr in [(0, 0.6), (0, 0.7), (0, 0.8), (1, 0.7)]:
        a = lbm.lbm_coexistence(eos, Tr)
        b = oracle_mod.maxwell(eos, Tr)
        for k in ("rho_g", "rho_l", "p_sat", "mu_sat"):
            assert a[k] == pytest.approx(b[k], rel=1e-9), (eos, Tr, k)


def test_eos_eval_agrees_with_oracle(oracle_mod):
    """The library's host EOS (used for Laplace tensions) against the oracle's p0 and psi'."""
    from paper_2202_06516_gb300 import lbm
    for eos, Tr in [(0, 0.6), (0, 0.7), (1, 0.7)]:
        mx = oracle_mod.maxwell(eos, Tr)
        for rho in np.linspace(0.5 * mx["rho_g"], 1.1 * mx["rho_l"], 7):
            a = lbm.lbm_eos_eval(eos, Tr, rho)
            b = oracle_mod.eos_eval(eos, Tr, rho)
            assert a["p0"] == pytest.approx(b["p0"], rel=1e-12, abs=1e-15)
            assert a["dpsi"] == pytest.approx(b["mu0"], rel=1e-12, abs=1e-15)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_eos_eval(0, 0.7, -1.0)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_eos_eval(0, 0.7, 21.0 / 2.0 + 1.0)


def test_coexistence_rejects_supercritical():
    from paper_2202_06516_gb300 import lbm
    with pytest.raises(lbm.LbmError):
        lbm.lbm_coexistence(0, 1.2)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_coexistence(7, 0.7)


def test_create_validates_arguments():
    """Argument errors are reported before any device work, with a message."""
    from paper_2202_06516_gb300 import lbm
    p = lbm.lbm_params(4, 64, 0, 0, 0, 0, 0, 0, 0, 0.7, 0.1, 0.0126, 1.0, 1.64, 1.54, 1.9, 0, 0,
                       0, 0, None)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create(p)
    assert e.value.status == lbm.LBM_ERR_ARG
    assert "nx" in lbm.lbm_last_error(None)
    p.nx, p.tile_x, p.tile_y = 64, 48, 48
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create(p)
    assert e.value.status == lbm.LBM_ERR_ARG


def test_create_rejects_oversized_and_empty_lattices():
    """A lattice whose nine padded planes would exceed 2^31 nodes, and an empty one, are argument
    errors found on the host before any device work."""
    from paper_2202_06516_gb300 import lbm
    for nx, ny in [(60000, 60000), (0, 64), (64, 0)]:
        p = lbm.lbm_params(nx, ny, 0, 0, 0, 0, 0, 0, 0, 0.7, 0.1, 0.0126, 1.0, 1.64, 1.54, 1.9,
                           0, 0, 0, 0, None)
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_create(p)
        assert e.value.status == lbm.LBM_ERR_ARG, (nx, ny)


def test_null_context_is_an_error_not_a_crash():
    from paper_2202_06516_gb300 import lbm
    L = lbm.lib()
    assert L.lbm_step(None, 1) == lbm.LBM_ERR_ARG
    assert L.lbm_measure_contact_angle(None, None) == lbm.LBM_ERR_ARG
    assert L.lbm_state_bytes(None) == 0
    assert L.lbm_save_state(None, None, 0) == lbm.LBM_ERR_ARG
    assert L.lbm_load_state(None, None, 0) == lbm.LBM_ERR_ARG
    L.lbm_destroy(None)


def test_product_path_does_not_import_the_oracle():
    """The CUDA path's package never reaches the oracle."""
    pkg = os.path.join(ROOT, "paper_2202_06516_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "lbm_oracle" not in txt, f


def test_autotune_rejects_null_handles():
    """The autotuners report a NULL handle as an argument error (no device work)."""
    import ctypes as C
    from paper_2202_06516_gb300 import lbm
    L = lbm.lib()
    n = C.c_int32()
    assert L.lbm_autotune(None, 5, None, 0, C.byref(n)) == lbm.LBM_ERR_ARG
    assert L.lbm_batch_autotune(None, 5, None, 0, C.byref(n)) == lbm.LBM_ERR_ARG
