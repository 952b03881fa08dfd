"""Host-side checks of the C ABI that need no GPU.

* the library builds and exports every function ``include/lbm.h`` declares;
* argument validation returns LBM_EINVAL before any device work;
* status strings.
"""

import ctypes
import os
import re

import pytest

from paper_2112_09972_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2112_09972_gb300 import build

    build.build()
    return lbm.load_library()


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", src)))


def test_header_and_binding_agree():
    assert _declared_functions() == sorted(lbm.ABI_FUNCTIONS)


def test_exports_every_declared_function(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_strerror(lib):
    assert lbm.strerror(0) == "ok"
    assert "invalid" in lbm.strerror(-1)
    assert "Mach" in lbm.strerror(-5)


def _create(lib, box=(16, 16, 16), R=4.0, visc=(1 / 6, 1 / 6), G=3.5, **kw):
    o = lbm.lbm_opts()
    lib.lbm_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    b = (ctypes.c_int32 * 3)(*box)
    v = (ctypes.c_double * 2)(*visc)
    h = ctypes.c_void_p(1234)
    rc = lib.lbm_create(ctypes.byref(h), b, R, v, G, ctypes.byref(o))
    return rc, h


@pytest.mark.parametrize(
    "kw",
    [
        dict(box=(3, 16, 16)),             # box below the minimum
        dict(R=7.5),                        # droplet touches the ghost layer (2R > min(box) - 2)
        dict(R=-1.0),
        dict(visc=(0.0, 0.1)),
        dict(visc=(0.1, float("nan"))),
        dict(G=-1.0),
        dict(precision=7),
        dict(bc=5),
        dict(rho_hi=0.5, rho_lo=0.9),       # minority above majority
    ],
)
def test_create_rejects_invalid_arguments(lib, kw):
    rc, h = _create(lib, **kw)
    assert rc == -1
    assert h.value is None  # *out is cleared on failure


def test_null_handles_are_rejected(lib):
    assert lib.lbm_step(None, 1) == -1
    assert lib.lbm_sync(None) == -1
    assert lib.lbm_set_gradient(None, None, 0) == -1
    lib.lbm_destroy(None)  # allowed
