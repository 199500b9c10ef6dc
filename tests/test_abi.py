"""The C-ABI library builds for sm_103a, loads, exports every declared entry point,
and rejects bad arguments on the host (no GPU work is issued)."""
import ctypes

import numpy as np
import pytest

from paper_1708_01663_gb300 import build, cisor


@pytest.fixture(scope="module")
def lib():
    build.build()
    return cisor.load()


def test_exports_every_declared_symbol(lib):
    names = cisor.declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_empty_error(lib):
    assert b"sm_103a" in lib.cisor_version()


@pytest.mark.parametrize("kw", [dict(n=4), dict(n=300), dict(T=0), dict(delta=0.0), dict(pad=100),
                                dict(pad=64, n=64), dict(dim=4), dict(dim=1), dict(dim=3, n=200),
                                dict(dim=3, pad=512), dict(tx_kind=2), dict(tx_kind=1)])
def test_create_rejects_bad_geometry(lib, kw):
    ang = np.zeros(12)   # tx_kind = 1 reads T x dim source positions: (0, 0) is inside the grid
    rx = np.ones((3, 2)) * 10
    g = dict(dim=2, n=32, delta=0.125, wavelength=1.0, eps_b=1.0, T=4, M=3, complex_f=0, pad=0)
    g.update(kw)
    geo = cisor.Geometry(g["dim"], g["n"], g["delta"], g["wavelength"], g["eps_b"], g["T"],
                         ang.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), g["M"],
                         rx.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), g["complex_f"], g["pad"],
                         g.get("tx_kind", 0))
    ctx = ctypes.c_void_p()
    st = lib.cisor_create(ctypes.byref(ctx), ctypes.byref(geo), None)
    assert st == cisor.ERR_INVALID_ARG
    assert not ctx.value
    assert cisor.last_error()


def test_null_arguments(lib):
    assert lib.cisor_create(None, None, None) == cisor.ERR_INVALID_ARG
    assert lib.cisor_destroy(None) == cisor.OK
    assert lib.cisor_forward(None, None, None, None, None, None, None, None) == cisor.ERR_INVALID_ARG
    assert lib.cisor_step(None, None, None, None, None) == cisor.ERR_INVALID_ARG
    assert lib.cisor_tv_prox(None, None, None, 0.1, 5, 0.0, 1.0, 0.0, 1.0) == cisor.ERR_INVALID_ARG
