"""The C-ABI library loads and exports every symbol include/mpmc.h declares (no GPU needed)."""

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2306_09559_gb300 import build, mpmc
    build.build()
    return mpmc.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "mpmc.h")).read()
    return sorted(set(re.findall(r"^MPMC_API [^(]*?\b(mpmc_\w+)\(", src, flags=re.M)))


def test_every_declared_symbol_is_exported(L):
    from paper_2306_09559_gb300 import mpmc
    declared = _declared()
    assert len(declared) >= 15
    assert declared == mpmc.exported_symbols()
    for name in declared:
        assert hasattr(L, name), name


def test_strerror(L):
    assert L.mpmc_strerror(0) == b"ok"
    assert L.mpmc_strerror(1) == b"invalid argument"
    assert L.mpmc_strerror(99) == b"unknown error"


def test_create_rejects_bad_arguments_before_touching_the_gpu(L):
    h = ctypes.c_void_p()
    links = np.zeros(4 * 16 * 9, dtype=np.complex128)
    ptr = links.ctypes.data_as(ctypes.c_void_p)
    for dims, kappa, prec, bc, code in [((1, 2, 2, 2), 0.1, 0, 1, 1), ((2, 2, 2, 2), float("nan"), 0, 1, 1),
                                       ((2, 2, 2, 2), 0.1, 7, 1, 3), ((2, 2, 2, 2), 0.1, 0, 0, 1)]:
        d = (ctypes.c_int * 4)(*dims)
        assert L.mpmc_create(ctypes.byref(h), d, ptr, kappa, prec, bc) == code
        assert not h.value
    assert L.mpmc_create(None, None, None, 0.1, 0, 1) == 1
    assert L.mpmc_destroy(None) == 0
    assert L.mpmc_last_error(None) == b"null handle"
