"""The C-ABI library builds, loads and exports every symbol include/lhc.h declares
(CPU only: no compute call needs a GPU here)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1711_02384_gb300 import build as B

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")


def _declared():
    names = set()
    for f in os.listdir(HDR):
        if f.endswith(".h"):
            src = open(os.path.join(HDR, f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lhc_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    B.build()
    return ctypes.CDLL(B.LIB)


def test_header_declares_entry_points():
    names = _declared()
    for n in ("lhc_create", "lhc_destroy", "lhc_insertion", "lhc_spectator", "lhc_combine",
              "lhc_momenta", "lhc_strerror"):
        assert n in names


def test_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_and_version(lib):
    lib.lhc_strerror.restype = ctypes.c_char_p
    assert lib.lhc_strerror(0) == b"success"
    assert lib.lhc_strerror(3) == b"request exceeds the HBM budget"
    assert lib.lhc_version() >= 100


def test_momenta_host_helper_matches_paper_count(lib):
    nq = ctypes.c_int(0)
    assert lib.lhc_momenta(8, -1, None, 0, ctypes.byref(nq)) == 0
    assert nq.value == 93
    k = np.zeros((93, 3), dtype=np.int32)
    assert lib.lhc_momenta(8, -1, k.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), 93, ctypes.byref(nq)) == 0
    n2 = (k.astype(int) ** 2).sum(1)
    assert n2.max() == 8 and np.all(np.diff(n2) >= 0) and len({tuple(v) for v in k}) == 93


def test_invalid_arguments_rejected_before_launch(lib):
    lib.lhc_insertion.argtypes = [ctypes.c_void_p] * 13
    # NULL context -> LHC_EINVAL, without touching any device
    assert lib.lhc_insertion(*([None] * 13)) == 1
    assert lib.lhc_combine(None, 0, None, 1, None, 1, 1, 1, None, None, None, 1, 0, None, None) == 1
    assert lib.lhc_momenta(-1, -1, None, 0, None) == 1


def test_binding_loads(lib):
    from paper_1711_02384_gb300 import lhc
    assert lhc.lib() is not None
    k = lhc.momenta(4)
    assert len(k) == 33


def test_server_calls_validate_without_a_gpu(lib):
    lib.lhc_submit.argtypes = [ctypes.c_void_p] * 3
    lib.lhc_poll.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]
    lib.lhc_serve_start.argtypes = [ctypes.c_void_p, ctypes.c_int]
    assert lib.lhc_submit(None, None, None) == 1          # no server for a NULL context -> EINVAL
    assert lib.lhc_poll(None, 1, None) == 7               # LHC_ENOTFOUND
    assert lib.lhc_serve_start(None, 4) == 1


@pytest.mark.parametrize("n2max,cmax", [(3, 1), (4, -1), (8, -1), (9, 3), (16, -1)])
def test_momenta_host_helper_matches_oracle(lib, n2max, cmax):
    """a0 on the host: the library's momentum list (C++) equals the oracle's (numpy), the
    same vectors in the same order (|k|^2, then kx, ky, kz ascending)."""
    from oracle.momenta import momenta
    from paper_1711_02384_gb300 import lhc
    ref = np.asarray(momenta(n2max, None if cmax < 0 else cmax), dtype=np.int32)
    got = np.asarray(lhc.momenta(n2max, cmax), dtype=np.int32)
    assert got.shape == ref.shape and np.array_equal(got, ref)
