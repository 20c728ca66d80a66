"""CPU checks of the server's C ABI (include/tacsl_serve.h): bad configurations and
arguments are refused before any CUDA call."""
import ctypes as C

import pytest

import paper_2408_06506_b300 as tacsl
from paper_2408_06506_b300 import build
from paper_2408_06506_b300 import serve as sv

INVALID = 1
FAKE = 0x7F0000001000


@pytest.fixture(scope="module")
def lib():
    build.build()
    return sv._lib()


def _sdfs():
    s = tacsl._Sdf()
    s.n[0] = s.n[1] = s.n[2] = 8
    s.voxel = 1e-3
    s.data = FAKE
    arr = (tacsl._Sdf * 1)(s)
    st = tacsl._SdfSet(C.cast(arr, C.POINTER(tacsl._Sdf)), 1)
    st._keep = arr
    return st


@pytest.mark.parametrize("field,value", [("hbm_budget_bytes", 1000), ("max_pads", 0), ("n_streams", 0),
                                         ("n_streams", 9), ("batch_timeout_ms", 0)])
def test_create_rejects_config(lib, field, value):
    cfg = sv._Config(1 << 30, 1024, 2, 1000)
    setattr(cfg, field, value)
    first = (C.c_int64 * 1)(0)
    count = (C.c_int32 * 1)(4)
    h = C.c_void_p()
    st = _sdfs()
    assert lib.tacsl_server_create(C.byref(cfg), C.byref(st), None, FAKE, 4, 1, first, count, C.byref(h)) == INVALID
    assert not h.value


def test_create_rejects_layouts_and_pool(lib):
    cfg = sv._Config(1 << 30, 1024, 2, 1000)
    st = _sdfs()
    h = C.c_void_p()
    first = (C.c_int64 * 1)(2)
    count = (C.c_int32 * 1)(4)
    # layout [2, 6) outside a pool of 4 points
    assert lib.tacsl_server_create(C.byref(cfg), C.byref(st), None, FAKE, 4, 1, first, count, C.byref(h)) == INVALID
    assert lib.tacsl_server_create(C.byref(cfg), C.byref(st), None, None, 4, 1, first, count, C.byref(h)) == INVALID
    assert lib.tacsl_server_create(C.byref(cfg), None, None, FAKE, 8, 1, first, count, C.byref(h)) == INVALID
    assert lib.tacsl_server_create(None, C.byref(st), None, FAKE, 8, 1, first, count, C.byref(h)) == INVALID


def test_null_server_handles(lib):
    rid = C.c_int64()
    assert lib.tacsl_server_submit(None, None, C.byref(rid)) == INVALID
    assert lib.tacsl_server_wait(None, 1, 0, None, None) == INVALID
    assert lib.tacsl_server_get_stats(None, None) == INVALID
    assert lib.tacsl_server_destroy(None) == 0
