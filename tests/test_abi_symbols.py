"""The C ABI library builds for sm_103a, loads, and exports every function
that include/topo.h declares (no compute calls: no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(topo_\w+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2605_04735_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("topo_create_mesh", "topo_set_density", "topo_solve", "topo_compliance",
                     "topo_sensitivity", "topo_free"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_loads_and_reports_status_strings(libpath):
    from paper_2605_04735_gb300 import topo
    assert topo.status_string(topo.OK) == "ok"
    assert "converged" in topo.status_string(topo.ERR_NOT_CONVERGED)
    o = topo.default_opts()
    assert o.rtol == 1e-8 and o.precision == topo.PREC_FP32
    assert topo.footprint_bytes(96, 32, 32) > 0


def test_noalloc_binding_refuses_arrays_that_do_not_fit_the_grid(libpath):
    """topo_sensitivity_noalloc only sees pointers, so its binding checks the
    lengths against the grid before anything is passed to the library."""
    import numpy as np
    from paper_2605_04735_gb300 import topo
    nx, ny, nz = 4, 2, 2
    ok_u = np.zeros(3 * 5 * 3 * 3)
    ok_r = np.zeros(nx * ny * nz, np.float32)
    ok_d = np.zeros(nx * ny * nz)
    c = np.zeros(1)
    bad = [(ok_u[:-3], ok_r, ok_d, c), (ok_u, ok_r[:-1], ok_d, c), (ok_u, ok_r, ok_d[:-1], c),
           (ok_u, ok_r, ok_d, np.zeros(0))]
    for u, r, d, cc in bad:
        with pytest.raises(ValueError):
            topo.sensitivity_noalloc(nx, ny, nz, u, r, d, cc)
    # the right sizes pass the size check and stop at the device check (host arrays)
    with pytest.raises(TypeError):
        topo.sensitivity_noalloc(nx, ny, nz, ok_u, ok_r, ok_d, c)
