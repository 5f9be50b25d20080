"""The C-ABI library loads without a GPU, exports every symbol include/sa.h
declares, and rejects malformed models on the host before any device work."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2511_17245_gb300 import _lib
from paper_2511_17245_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    inc = os.path.join(ROOT, "include")
    names = set()
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            text = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, f)).read(), flags=re.S)
            names |= set(re.findall(r"\b(sa_[a-z_]+)\s*\(", text))
    return sorted(names)


def test_exports_every_declared_symbol():
    lib = _lib.load()
    declared = _declared_functions()
    assert set(declared) == set(_lib.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name
    assert "sm_103a" in _lib.sa_version()


def _create(inst):
    return _lib.sa_model_create(inst["n_vars"], inst["lower"], inst["upper"], inst["term_offsets"],
                                inst["term_vars"], inst["coeffs"], inst["coef_type"])


@pytest.mark.parametrize("case,status", [
    (dict(lo=[3], hi=[1], terms=[[0]], c=[1]), _lib.SA_ERR_INVALID),             # l > u
    (dict(lo=[0], hi=[1], terms=[[1]], c=[1]), _lib.SA_ERR_INVALID),             # index out of range
    (dict(lo=[0], hi=[2 ** 40], terms=[[0]], c=[1]), _lib.SA_ERR_UNSUPPORTED),   # bound beyond int32
    (dict(lo=[0], hi=[1], terms=[[0] * 64], c=[1]), _lib.SA_ERR_UNSUPPORTED),    # exponent 64
    (dict(lo=[-2 ** 20, 0], hi=[2 ** 20, 1], terms=[[0, 0, 0, 1]], c=[2 ** 10]), _lib.SA_ERR_OVERFLOW),
])
def test_host_validation(case, status):
    ct = "i64"
    inst = wl._pack(len(case["lo"]), case["lo"], case["hi"], case["terms"], case["c"], ct)
    with pytest.raises(_lib.SAError) as e:
        _create(inst)
    assert e.value.status == status
    assert _lib.sa_last_error() != ""


def test_nan_coefficient_rejected():
    inst = wl._pack(2, [0, 0], [1, 1], [[0, 1]], [float("nan")], "f64")
    with pytest.raises(_lib.SAError) as e:
        _create(inst)
    assert e.value.status == _lib.SA_ERR_INVALID


def test_bad_offsets_rejected():
    lib = _lib.load()
    h = C.c_void_p()
    lo = np.zeros(2, np.int64)
    hi = np.ones(2, np.int64)
    offs = np.array([0, 2, 1], np.int64)
    tv = np.array([0, 1], np.int32)
    co = np.array([1, 1], np.int32)
    rc = lib.sa_model_create(C.byref(h), 2, lo.ctypes.data, hi.ctypes.data, 2, offs.ctypes.data,
                             tv.ctypes.data, co.ctypes.data, 0)
    assert rc == _lib.SA_ERR_INVALID and not h.value


def test_null_arguments():
    lib = _lib.load()
    assert lib.sa_run(None, None, None, None, None, None) == _lib.SA_ERR_INVALID
    assert lib.sa_energy(None, None, 0, None, None) == _lib.SA_ERR_INVALID
    lib.sa_model_destroy(None)
