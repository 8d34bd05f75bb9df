"""The C-ABI library builds, loads and exports every symbol include/ktune.h
declares; host-side validation that runs before any device call."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def kt():
    from paper_2102_05297_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    from paper_2102_05297_gb300 import ktune
    return ktune


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?[\w ]+?\*?\s*(ktune_\w+)\s*\(", src, re.M))
    return names


def test_header_symbols_exported(kt):
    names = declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(kt.lib, n), n
    assert set(kt.EXPORTED) <= names


def test_abi_version_and_error(kt):
    assert kt.lib.ktune_abi_version() == 100
    assert isinstance(kt.lib.ktune_last_error(), bytes)


def test_early_validation(kt):
    h = C.c_void_p()
    assert kt.lib.ktune_space_create(None, 0, None, C.byref(h)) == kt.KTUNE_EINVAL
    d = kt.ktune_space_desc(0, None, None, None, 0)
    assert kt.lib.ktune_space_create(C.byref(d), 0, None, C.byref(h)) == kt.KTUNE_EINVAL
    nv = (C.c_int * 17)(*([2] * 17))
    vals = (C.c_int64 * 34)(*([0, 1] * 17))
    d = kt.ktune_space_desc(17, nv, vals, None, 0)
    assert kt.lib.ktune_space_create(C.byref(d), 0, None, C.byref(h)) == kt.KTUNE_EINVAL
    assert b"n_params" in kt.lib.ktune_last_error()
    d = kt.ktune_space_desc(1, nv, vals, None, 0)
    assert kt.lib.ktune_space_create(C.byref(d), 7, None, C.byref(h)) == kt.KTUNE_EINVAL
    assert kt.lib.ktune_model_load(None, None, 0, C.byref(h)) == kt.KTUNE_EINVAL
    assert kt.lib.ktune_step(None, None, 5, None, None, None) == kt.KTUNE_EINVAL
    assert kt.lib.ktune_report(None, None, 0) == kt.KTUNE_EINVAL


def test_model_blob_layout(kt):
    import numpy as np
    import struct
    t = {"feature": [0, -1, -1], "threshold": [1, 0, 0], "left": [1, -1, -1],
         "right": [2, -1, -1], "value": [0.0, 1.5, 2.5]}
    b = kt.model_blob({"roles": [0], "trees": [t]})
    assert struct.unpack("<4I", b[:16]) == (kt.MODEL_MAGIC, 1, 1, 1)
    assert len(b) == 16 + 4 + 4 + 3 * 20
    assert np.frombuffer(b[-12:], "<f4").tolist() == [0.0, 1.5, 2.5]


def test_table_blob_layout(kt):
    import numpy as np
    import struct
    t = np.arange(6, dtype=np.float32).reshape(3, 2)
    b = kt.model_blob({"kind": "table", "roles": [0, 1], "table": t})
    assert struct.unpack("<4I", b[:16]) == (kt.MODEL_MAGIC, 1, 2, 2)
    assert struct.unpack("<Q", b[24:32]) == (3,)
    assert np.frombuffer(b[32:], "<f4").tolist() == list(range(6))
