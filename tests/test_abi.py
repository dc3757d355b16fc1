"""Host-side checks of the C ABI (no GPU needed): the library builds, loads, exports every
symbol include/htruss.h declares, and the binding fails loudly instead of falling back."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "htruss.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2411_06405_gb300 import build, _lib

    build.build()
    return _lib.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(htd_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("htd_build_csr", "htd_h_support", "htd_truss_decompose"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2411_06405_gb300 import _lib

    names = declared_functions()
    for name in names:
        assert hasattr(lib, name), f"{name} declared in htruss.h but not exported"
    assert sorted(_lib.EXPORTED) == names


def test_stats_struct_matches_header(lib):
    from paper_2411_06405_gb300 import _lib

    text = open(HEADER).read()
    body = re.search(r"typedef struct htd_stats \{(.*?)\} htd_stats;", text, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"(int64_t|int32_t|double|float)\s+(\w+);", body)
    ctype = {"int64_t": ctypes.c_int64, "int32_t": ctypes.c_int32, "double": ctypes.c_double,
             "float": ctypes.c_float}
    assert [(n, ctype[t]) for t, n in fields] == list(_lib.HtdStats._fields_)


def _struct_fields(name):
    text = open(HEADER).read()
    body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (name, name), text, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    ctype = {"int64_t": ctypes.c_int64, "int32_t": ctypes.c_int32, "double": ctypes.c_double,
             "float": ctypes.c_float}
    return [(n, ctype[t]) for t, n in re.findall(r"(int64_t|int32_t|double|float)\s+(\w+);", body)]


def test_server_structs_match_header(lib):
    from paper_2411_06405_gb300 import _lib

    assert _struct_fields("htd_request_info") == list(_lib.HtdRequestInfo._fields_)
    assert _struct_fields("htd_server_stats") == list(_lib.HtdServerStats._fields_)
    assert _struct_fields("htd_hindex_stats") == list(_lib.HtdHindexStats._fields_)


def test_footprint_estimate_on_host(lib):
    # host-only: grows with the graph, dense balls when they fit a quarter of free memory
    est = [lib.htd_footprint_estimate(n, 8 * n, 2, 200 << 30) for n in (1000, 10000, 100000)]
    assert est[0] < est[1] < est[2]
    small_free = lib.htd_footprint_estimate(100000, 800000, 2, 1 << 30)
    assert small_free < est[2]  # compact estimate when the dense sets do not fit
    assert lib.htd_footprint_estimate(1000, 8000, 3, 200 << 30) > est[0]  # two ball radii
    assert lib.htd_footprint_estimate(-1, 0, 2, 0) == -1


def test_hindex_rejects_bad_arguments_without_a_device(lib):
    # NULL handle, unknown flags, pruning with asynchronous sweeps: EINVAL before any
    # device work
    assert lib.htd_hindex_decompose_ex(None, 2, 1, -1, 0, None, None, None, None) == 1
    assert lib.htd_hindex_decompose_ex(None, 2, 1, -1, 2, None, None, None, None) == 1
    assert lib.htd_hindex_decompose_ex(None, 2, 4, -1, 1, None, None, None, None) == 1
    assert lib.htd_hindex_decompose(None, 2, 1, -1, None, None, None, None) == 1


def test_server_rejects_bad_arguments_without_a_device(lib):
    out = ctypes.c_void_p()
    assert lib.htd_server_create(0, 0, 0, ctypes.byref(out)) == 1
    assert lib.htd_server_create(4, -5, 0, ctypes.byref(out)) == 1
    rid = ctypes.c_int64()
    assert lib.htd_server_submit(None, 4, None, None, 0, 2, ctypes.byref(rid)) == 1
    done = ctypes.c_int32()
    assert lib.htd_server_poll(None, 1, ctypes.byref(done)) == 1
    lib.htd_server_destroy(None)


def test_status_strings(lib):
    for code in range(7):
        assert lib.htd_status_string(code)


def test_invalid_arguments_rejected_on_host(lib):
    out = ctypes.c_void_p()
    # NULL out pointer, negative n, n above the limit, oversized m_in: all host-side checks
    assert lib.htd_build_csr(4, None, None, 0, 1, None, None) == 1
    assert lib.htd_build_csr(-1, None, None, 0, 1, None, ctypes.byref(out)) == 1
    assert lib.htd_build_csr(2_000_000, None, None, 0, 1, None, ctypes.byref(out)) == 6
    assert lib.htd_build_csr(4, ctypes.c_void_p(8), ctypes.c_void_p(8), 1 << 30, 1, None,
                             ctypes.byref(out)) == 5
    assert not out.value
    assert lib.htd_h_support(None, 2, None, None) == 1
    assert lib.htd_truss_decompose(None, 2, None, None, None, None) == 1


def test_batched_arguments_rejected_on_host(lib):
    import numpy as np

    def call(n, h, off, num=None):
        n = np.asarray(n, dtype=np.int32)
        h = np.asarray(h, dtype=np.int32)
        off = np.asarray(off, dtype=np.int64)
        k = len(n) if num is None else num
        oo = np.zeros(max(len(n), 1), dtype=np.int64)
        om = np.zeros(max(len(n), 1), dtype=np.int64)
        vp = lambda a: ctypes.c_void_p(a.ctypes.data)
        return lib.htd_truss_decompose_batched(k, vp(n), vp(h), vp(off), None, None, 0, 0, None,
                                               vp(oo), vp(om), None, None, None)

    assert call([4], [2], [0, 0], num=-1) == 1          # negative count
    assert call([4], [0], [0, 0]) == 1                  # h below 1
    assert call([4], [9], [0, 0]) == 1                  # h above HTD_MAX_H
    assert call([-1], [2], [0, 0]) == 1                 # negative n
    assert call([4, 4], [2, 2], [0, 3, 1]) == 1         # decreasing offsets
    assert call([4], [2], [1, 3]) == 1                  # offsets not starting at 0
    assert call([2_000_000], [2], [0, 0]) == 6          # n above HTD_MAX_N
    assert call([4], [2], [0, 2]) == 1                  # pairs but NULL device buffers
    assert call([4], [2], [0, 1 << 31]) == 5            # 2 m_in >= 2^31
    assert lib.htd_truss_decompose_batched(0, None, None, None, None, None, 0, 0, None, None,
                                           None, None, None, None) == 0  # empty batch


def test_no_cpu_fallback_without_a_gpu(lib):
    import torch

    import paper_2411_06405_gb300 as htd

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(Exception):
        htd.htd_build_csr(3, torch.tensor([0, 1], dtype=torch.int32),
                          torch.tensor([1, 2], dtype=torch.int32))
