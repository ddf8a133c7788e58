"""The C-ABI library builds for sm_103a, loads, exports every entry point that
include/slim_gb300.h declares, and rejects bad arguments on the host (no GPU
work is done here)."""
import ctypes
import os
import re

import pytest

from paper_2512_12945_gb300 import build as B
from paper_2512_12945_gb300 import slim

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                   "slim_gb300.h")


def declared():
    txt = open(HDR).read()
    return sorted(set(re.findall(r"^\s*(?:slim_status|const char\*)\s+(slim_\w+)\s*\(", txt, re.M)))


@pytest.fixture(scope="module")
def L():
    B.build()
    return slim.lib()


def test_exports_every_declared_symbol(L):
    names = declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(slim.EXPORTS)


def test_params_default_and_arg_errors(L):
    p = slim.slim_map_params_default()
    assert p.voxel_size == pytest.approx(0.1) and p.num_classes == 20
    bad = []
    for field, val in [("voxel_size", 0.0), ("trunc", 1.0), ("mode", 5), ("num_classes", 0),
                       ("block_capacity", 0), ("hash_capacity", 8), ("max_points", -1),
                       ("alpha0", -1.0)]:
        q = slim.slim_map_params_default()
        setattr(q, field, val)
        h = ctypes.c_void_p()
        rc = L.slim_map_create(ctypes.byref(q), ctypes.byref(h))
        bad.append((field, rc))
        assert rc == 1, (field, rc)
        assert h.value is None
        assert len(L.slim_last_error()) > 0
    q = slim.slim_map_params_default()
    q.mode = 2
    q.embed_dim = 100
    h = ctypes.c_void_p()
    assert L.slim_map_create(ctypes.byref(q), ctypes.byref(h)) == 1
    assert b"embed_dim" in L.slim_last_error()


def test_null_handles_rejected(L):
    assert L.slim_integrate(None, None, 0, None, None, None) == 1
    assert L.slim_map_sync(None, None) == 1
    assert L.slim_map_destroy(None) == 1
    n = ctypes.c_int64()
    assert L.slim_extract_tsdf(None, None, None, None, None, None, None, 0, ctypes.byref(n), 0,
                               None) == 1
    assert L.slim_map_params_default(None) == 1


def test_params_struct_size_matches_the_binding(L):
    """slim_map_params_default clears the C struct with its own sizeof and
    sets embed_bound (the last field) to 1: with a sentinel-filled buffer
    larger than the binding's struct, it must write exactly the binding's
    size, so the two layouts agree."""
    n = ctypes.sizeof(slim.slim_map_params)
    buf = (ctypes.c_ubyte * (n + 64))(*([0xAB] * (n + 64)))
    assert L.slim_map_params_default(ctypes.cast(buf, ctypes.POINTER(slim.slim_map_params))) == 0
    assert all(b == 0xAB for b in bytes(buf)[n:]), "C struct larger than the binding's"
    p = slim.slim_map_params.from_buffer(buf)
    assert p.embed_bound == 1.0 and p.voxel_size == pytest.approx(0.1)


def test_open_set_embed_bound_range_checked(L):
    """embed_bound must lie in [2^-16, 2^16] for open-set maps (checked on
    the host, nothing allocated)."""
    for b in (0.0, -1.0, 2.0 ** 17):
        q = slim.slim_map_params_default()
        q.mode = 2
        q.embed_dim = 64
        q.embed_bound = b
        h = ctypes.c_void_p()
        assert L.slim_map_create(ctypes.byref(q), ctypes.byref(h)) == 1
        assert b"embed_bound" in L.slim_last_error()
