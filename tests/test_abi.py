"""The C ABI library builds, loads without a GPU, exports every entry point that
include/hsg.h declares, and rejects bad arguments on the host before touching
the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libhsg():
    from paper_1204_6192_gb300 import build, hsg
    build.build()
    return hsg.lib()


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "hsg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hsg_[a-z_0-9]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(libhsg):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(libhsg, n), n


def test_default_options(libhsg):
    from paper_1204_6192_gb300 import hsg
    o = hsg.default_options()
    assert (o.precision, o.n_hb_per_step, o.n_or_per_step, o.variant) == (0, 1, 5, 0)


@pytest.mark.parametrize("L,temps,nrep,msg", [
    (5, [0.5, 1.0], 2, "even"),
    (2, [0.5, 1.0], 2, "even"),
    (8, [1.0, 0.5], 2, "increasing"),
    (8, [0.5, float("nan")], 2, "positive"),
    (8, [0.5, 1.0], 0, "n_replicas"),
])
def test_host_side_validation(libhsg, L, temps, nrep, msg):
    from paper_1204_6192_gb300 import hsg
    N = L ** 3
    J = np.ones((N, 3), dtype=np.float32)
    t = np.array(temps, dtype=np.float64)
    ctx = ctypes.c_void_p()
    st = libhsg.hsg_create(ctypes.byref(ctx), L, t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                           len(temps), nrep, J.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), None,
                           1, None)
    assert st == 1
    assert msg in libhsg.hsg_last_error(None).decode()
    assert not ctx.value


def test_nonfinite_coupling_rejected(libhsg):
    L = 4
    J = np.ones((L ** 3, 3), dtype=np.float32)
    J[7, 2] = np.inf
    t = np.array([0.5, 1.0])
    ctx = ctypes.c_void_p()
    st = libhsg.hsg_create(ctypes.byref(ctx), L, t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 2,
                           1, J.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), None, 1, None)
    assert st == 1 and b"non-finite" in libhsg.hsg_last_error(None)


def test_status_strings(libhsg):
    for k in range(6):
        assert libhsg.hsg_status_string(k)
    libhsg.hsg_destroy(None)   # NULL is accepted
