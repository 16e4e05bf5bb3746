"""CPU-side checks of the C ABI: the library builds, loads without a GPU and
exports every function include/cfd.h declares; argument validation that
needs no device."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(cfd_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def built():
    from paper_2209_15333_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    declared = declared_functions()
    assert declared, "no declarations found"
    missing = declared - exported
    assert not missing, missing


def test_library_loads_and_binds(built):
    from paper_2209_15333_gb300 import _lib
    L = _lib.lib()
    for name in declared_functions():
        assert hasattr(L, name)
    assert set(_lib.EXPORTS) == declared_functions()


def test_default_params_and_validation_without_gpu(built):
    from paper_2209_15333_gb300 import _lib
    p = _lib.default_params()
    assert p.gamma == 1.4 and p.theta1 == 0.02 and p.theta2 == 0.1 and p.visc_order == 8
    ctx = C.c_void_p()
    met = (C.c_double * 10)()
    # periodic on one face only: rejected before any device call
    g = _lib.make_grid(8, 8, 8, bc_lo=(0, 0, 0), bc_hi=(3, 0, 0), metric_layout=_lib.METRICS_UNIFORM)
    st = _lib.lib().cfd_create(C.byref(ctx), C.byref(g), C.cast(met, C.c_void_p), 0, C.byref(p), None)
    assert st == _lib.CFD_EINVAL
    assert b"periodic" in _lib.lib().cfd_last_error(None)
    g = _lib.make_grid(4, 8, 8, bc_lo=(3, 0, 0), bc_hi=(3, 0, 0), metric_layout=_lib.METRICS_UNIFORM)
    assert _lib.lib().cfd_create(C.byref(ctx), C.byref(g), C.cast(met, C.c_void_p), 0, C.byref(p), None) == \
        _lib.CFD_EINVAL
    p.visc_order = 7
    g = _lib.make_grid(8, 8, 8, metric_layout=_lib.METRICS_UNIFORM)
    assert _lib.lib().cfd_create(C.byref(ctx), C.byref(g), C.cast(met, C.c_void_p), 0, C.byref(p), None) == \
        _lib.CFD_EINVAL
    assert _lib.lib().cfd_step(None, 0.1, 1) == _lib.CFD_EINVAL
    assert _lib.lib().cfd_sync(None, 1.0) == _lib.CFD_EINVAL
    _lib.lib().cfd_destroy(None)


def test_more_validation_without_gpu(built):
    """Degenerate and unsupported inputs are refused before any device call."""
    from paper_2209_15333_gb300 import _lib
    L = _lib.lib()
    ctx = C.c_void_p()
    met = (C.c_double * 10)()
    mp = C.cast(met, C.c_void_p)

    def create(g, p):
        return L.cfd_create(C.byref(ctx), C.byref(g), mp, 0, C.byref(p), None)

    p = _lib.default_params()
    assert create(_lib.make_grid(0, 8, 8, metric_layout=_lib.METRICS_UNIFORM), p) == _lib.CFD_EINVAL   # empty
    assert create(_lib.make_grid(8, 8, 8, bc_lo=(6, 0, 0), bc_hi=(6, 0, 0), metric_layout=_lib.METRICS_UNIFORM),
                  p) == _lib.CFD_EINVAL                                                               # unknown BC
    q = _lib.default_params(metric_mode=2)
    assert create(_lib.make_grid(8, 8, 8, metric_layout=_lib.METRICS_UNIFORM), q) == _lib.CFD_EINVAL  # unknown mode
    # an x-y plane of 2^31 nodes or more (plane offsets are 32-bit)
    assert create(_lib.make_grid(1 << 16, 1 << 15, 1, metric_layout=_lib.METRICS_UNIFORM), p) == _lib.CFD_EINVAL
    assert b"nx * ny" in L.cfd_last_error(None)
    q = _lib.default_params(metric_mode=_lib.METRIC_FSP)                                   # FSP needs periodic lines
    g = _lib.make_grid(8, 8, 8, bc_lo=(3, 0, 0), bc_hi=(3, 0, 0), metric_layout=_lib.METRICS_UNIFORM)
    assert create(g, q) == _lib.CFD_EUNSUPPORTED
    # a direction with ghost layers needs 2 * 8 + 1 nodes
    g = _lib.make_grid(16, 8, 8, bc_lo=(_lib.BC_HALO, 0, 0), bc_hi=(_lib.BC_HALO, 0, 0),
                       metric_layout=_lib.METRICS_UNIFORM)
    assert create(g, p) == _lib.CFD_EINVAL
    assert b"ghost" in L.cfd_last_error(None)
    q = _lib.default_params(recon_vars=7)
    assert create(_lib.make_grid(8, 8, 8, metric_layout=_lib.METRICS_UNIFORM), q) == _lib.CFD_EINVAL
    q = _lib.default_params(precision=1, weno_eps=0.0)
    assert create(_lib.make_grid(8, 8, 8, metric_layout=_lib.METRICS_UNIFORM), q) == _lib.CFD_EINVAL
    # characteristic reconstruction in an ensemble, and in the allocation-free call
    q = _lib.default_params(recon_vars=1)
    grids = (_lib.CfdGrid * 2)(_lib.make_grid(8, 8, 8, metric_layout=_lib.METRICS_UNIFORM),
                               _lib.make_grid(8, 8, 8, metric_layout=_lib.METRICS_UNIFORM))
    prms = (_lib.CfdParams * 2)(q, q)
    mets = (C.c_void_p * 2)(mp, mp)
    assert L.cfd_create_batch(C.byref(ctx), 2, grids, mets, 0, prms, None) == _lib.CFD_EUNSUPPORTED
    assert L.cfd_set_halo_links(None, None) == _lib.CFD_EINVAL
