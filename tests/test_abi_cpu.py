"""Host-side checks of libann (no GPU needed): the library builds and loads,
exports every entry point include/ann.h declares, and rejects bad arguments
and bad index files before touching the device."""
import ctypes
import os
import re
import struct

import numpy as np
import pytest

from paper_2506_15986_gb300 import _build, ann

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return ann.load_library()


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(ann_[a-z0-9_]+)\s*\(", src))
    return names


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert {"ann_load_index", "ann_search_batch", "ann_index_create"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_status_strings(lib):
    for s in range(9):
        assert ann.status_string(s)
    assert ann.status_string(ann.ERR_FORMAT) == "bad index file format"


def test_null_and_bad_arguments(lib):
    out = ctypes.c_void_p()
    assert lib.ann_index_create(None, 0, ctypes.byref(out)) == ann.ERR_INVALID_ARG
    d = ann.ann_index_desc(n=10, dim=3, degree=4, dtype=ann.F32, metric=ann.L2,
                           base=1, graph=1, medoid=0)
    # 3 fp32 = 12 bytes per row: not a multiple of 16
    assert lib.ann_index_create(ctypes.byref(d), 0, ctypes.byref(out)) == ann.ERR_INVALID_ARG
    d = ann.ann_index_desc(n=10, dim=16, degree=4, dtype=ann.U8, metric=ann.IP,
                           base=1, graph=1, medoid=0)
    assert lib.ann_index_create(ctypes.byref(d), 0, ctypes.byref(out)) == ann.ERR_UNSUPPORTED
    d = ann.ann_index_desc(n=10, dim=16, degree=4, dtype=ann.U8, metric=ann.L2,
                           base=1, graph=1, medoid=10)
    assert lib.ann_index_create(ctypes.byref(d), 0, ctypes.byref(out)) == ann.ERR_INVALID_ARG
    p = ann.search_params(10, 64)
    assert lib.ann_search_batch(None, None, 1, None, ctypes.byref(p), None, None, None, None) \
        == ann.ERR_INVALID_ARG
    assert lib.ann_sync_status(None, None) == ann.ERR_INVALID_ARG
    assert lib.ann_free_index(None) == ann.OK


def _write_index(path, n=8, dim=16, degree=4, corrupt=None, truncate=0):
    rng = np.random.default_rng(0)
    base = rng.integers(0, 256, (n, dim)).astype(np.uint8).tobytes()
    graph = rng.integers(-1, n, (n, degree)).astype(np.int32).tobytes()
    h = 14695981039346656037
    for b in base + graph:
        h ^= b
        h = (h * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    hdr = struct.pack("<8sIIqiiiiiIQQQQ", b"GATEANN1", 1, 80, n, dim, degree, 0, 0, 0, 0,
                      len(base), len(graph), 0, h)
    assert len(hdr) == 80
    blob = bytearray(hdr + base + graph)
    if corrupt is not None:
        blob[corrupt] ^= 0x5A
    if truncate:
        blob = blob[:-truncate]
    with open(path, "wb") as f:
        f.write(blob)


def test_index_file_errors_detected_on_host(lib, tmp_path):
    out = ctypes.c_void_p()
    assert lib.ann_load_index(str(tmp_path / "missing").encode(), 0, ctypes.byref(out)) == ann.ERR_IO
    p = tmp_path / "trunc.idx"
    _write_index(p, truncate=5)
    assert lib.ann_load_index(str(p).encode(), 0, ctypes.byref(out)) == ann.ERR_FORMAT
    p = tmp_path / "flip.idx"
    _write_index(p, corrupt=100)  # a base byte: checksum mismatch
    assert lib.ann_load_index(str(p).encode(), 0, ctypes.byref(out)) == ann.ERR_FORMAT
    p = tmp_path / "magic.idx"
    _write_index(p, corrupt=0)
    assert lib.ann_load_index(str(p).encode(), 0, ctypes.byref(out)) == ann.ERR_FORMAT
    p = tmp_path / "short.idx"
    with open(p, "wb") as f:
        f.write(b"GATE")
    assert lib.ann_load_index(str(p).encode(), 0, ctypes.byref(out)) == ann.ERR_FORMAT


def test_index_header_limits_checked_before_allocating(lib, tmp_path):
    # a header whose sizes agree with each other but break the row limits of
    # ann_index_create (rows a multiple of 16 bytes, at most 16 KiB; degree at
    # most ANN_MAX_STEP_CAND) is a format error, found before the loader sizes
    # any buffer from it (no data follows the header)
    out = ctypes.c_void_p()
    for n, dim, degree in ((4, 1 << 30, 4), (4, 17, 4), (4, 16, 129)):
        hdr = struct.pack("<8sIIqiiiiiIQQQQ", b"GATEANN1", 1, 80, n, dim, degree, 0, 0, 0, 0,
                          n * dim, n * degree * 4, 0, 0)
        p = tmp_path / f"hdr_{dim}_{degree}.idx"
        p.write_bytes(hdr)
        assert lib.ann_load_index(str(p).encode(), 0, ctypes.byref(out)) == ann.ERR_FORMAT


def test_release_l2_needs_an_index(lib):
    assert lib.ann_release_l2(None) == ann.ERR_INVALID_ARG
