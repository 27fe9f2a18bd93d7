"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function include/ps.h declares, and rejects bad parameters."""
import ctypes
import os

import pytest

from paper_2002_08642_gb300 import binding as B
from paper_2002_08642_gb300 import build as pbuild
from paper_2002_08642_gb300.solver import make_params


@pytest.fixture(scope="module")
def lib():
    pbuild.build()
    return B.lib()


def test_exports_every_declared_symbol(lib):
    names = B.header_symbols()
    assert len(names) >= 15
    raw = ctypes.CDLL(pbuild.LIB)
    for nm in names:
        assert hasattr(raw, nm), nm


def test_supported_sizes(lib):
    sizes = B.ps_supported_n()
    assert {32, 128, 256, 768} <= set(sizes)
    for n in sizes:
        m = n
        while m % 2 == 0:
            m //= 2
        while m % 3 == 0:
            m //= 3
        assert m == 1


def test_workspace_and_validation(lib):
    small = B.ps_workspace_size(make_params(32, 6.28, 0.01, 1.0, 1e-3))
    big = B.ps_workspace_size(make_params(64, 6.28, 0.01, 1.0, 1e-3, precision="fp64"))
    assert 0 < small < big
    with pytest.raises(B.PsError) as e:
        B.ps_workspace_size(make_params(100, 4.0, 0.01, 1.0, 1e-3))
    assert e.value.status == B.PS_EUNSUPPORTED
    bad = make_params(32, 4.0, 0.01, 1.0, 1e-3)
    bad.dt = -1.0
    with pytest.raises(B.PsError) as e:
        B.ps_workspace_size(bad)
    assert e.value.status == B.PS_EINVAL
    bad = make_params(32, 4.0, 0.01, 1.0, 1e-3)
    bad.precision = 7
    with pytest.raises(B.PsError):
        B.ps_workspace_size(bad)


def test_init_rejects_small_or_unaligned_workspace(lib):
    p = make_params(32, 4.0, 0.01, 1.0, 1e-3)
    need = B.ps_workspace_size(p)
    ctx = ctypes.c_void_p(0)
    # no device memory is touched before these checks fail
    assert lib.ps_init(ctypes.byref(p), None, ctypes.c_void_p(4096), need - 256, ctypes.byref(ctx)) == B.PS_ENOMEM
    assert lib.ps_init(ctypes.byref(p), None, ctypes.c_void_p(4096 + 8), need, ctypes.byref(ctx)) == B.PS_EINVAL
    assert lib.ps_init(ctypes.byref(p), None, None, need, ctypes.byref(ctx)) == B.PS_EINVAL
    assert not ctx.value
