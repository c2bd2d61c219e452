"""The C-ABI library builds, loads, and exports exactly what include/graph.h declares.

No GPU: only host-side entry points that never reach CUDA are called (argument checks,
status strings).
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "graph.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:graph_status|void|const char\*)\s+(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1312_3018_gb300 import _lib, build
    build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("graph_load_csr", "graph_partition", "bfs", "sssp", "pagerank",
                     "graph_free", "graph_strerror"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1312_3018_gb300 import _lib
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in graph.h but not exported"
        assert name in _lib.SIGNATURES, f"{name} missing from the Python binding"
    assert sorted(_lib.SIGNATURES) == declared_functions()


def test_library_is_an_sm103a_build():
    from paper_1312_3018_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
    assert os.path.exists(build.LIB)


def test_status_strings(lib):
    assert lib.graph_strerror(0) == b"success"
    assert lib.graph_strerror(-1) == b"invalid argument"
    assert lib.graph_strerror(-4).startswith(b"bounded wait")
    assert lib.graph_strerror(-99) == b"unknown status"


def test_load_rejects_bad_arguments_before_touching_the_device(lib):
    from paper_1312_3018_gb300 import _lib
    out = ctypes.c_void_p(0)
    off = (ctypes.c_int64 * 2)(0, 0)
    # n = 0
    assert lib.graph_load_csr(0, 0, ctypes.addressof(off), None, None, 0, None,
                              ctypes.byref(out)) == _lib.GRAPH_EINVAL
    # n >= 2^31
    assert lib.graph_load_csr(1 << 31, 0, ctypes.addressof(off), None, None, 0, None,
                              ctypes.byref(out)) == _lib.GRAPH_EINVAL
    # offsets[n] != m (host input)
    cols = (ctypes.c_uint32 * 5)()
    assert lib.graph_load_csr(1, 5, ctypes.addressof(off), ctypes.addressof(cols), None, 0,
                              None, ctypes.byref(out)) == _lib.GRAPH_EINVAL
    assert b"offsets[n]" in lib.graph_last_error()
    # NULL out
    assert lib.graph_load_csr(1, 0, ctypes.addressof(off), None, None, 0, None,
                              None) == _lib.GRAPH_EINVAL
    # bad memory kind
    assert lib.graph_load_csr(1, 0, ctypes.addressof(off), None, None, 7, None,
                              ctypes.byref(out)) == _lib.GRAPH_EINVAL
    # allocator hooks must come in pairs
    rt = _lib.graph_runtime(_lib.ALLOC_FN(lambda b, c: None), _lib.FREE_FN(), None, None)
    assert lib.graph_load_csr(1, 0, ctypes.addressof(off), None, None, 0, ctypes.byref(rt),
                              ctypes.byref(out)) == _lib.GRAPH_EINVAL
    assert out.value is None


def test_algorithms_reject_null_handles(lib):
    from paper_1312_3018_gb300 import _lib
    lv = (ctypes.c_uint32 * 4)()
    assert lib.bfs(None, 0, ctypes.addressof(lv), None, None, None) == _lib.GRAPH_EINVAL
    assert lib.sssp(None, 0, ctypes.addressof(lv), None, None) == _lib.GRAPH_EINVAL
    src = (ctypes.c_uint32 * 1)()
    assert lib.bfs_batch(None, ctypes.addressof(src), 1, ctypes.addressof(lv), None,
                         None) == _lib.GRAPH_EINVAL
    attr = _lib.pagerank_attr(0.85, 10, 0.0, 0, 1, 0, 0)
    assert lib.pagerank(None, ctypes.byref(attr), None, None) == _lib.GRAPH_EINVAL
    assert lib.pagerank_hybrid(None, ctypes.byref(attr), 1, None, None,
                               None) == _lib.GRAPH_EINVAL
    assert lib.graph_partition(None, None) == _lib.GRAPH_EINVAL
    lib.graph_free(None)


def test_binding_constants_match_the_header():
    from paper_1312_3018_gb300 import _lib
    src = open(HEADER).read()
    for name in ("GRAPH_BATCH_MAX", "GRAPH_NOALLOC_MAX_VERTICES", "GRAPH_INF", "GRAPH_MEM_HOST",
                 "GRAPH_MEM_DEVICE", "GRAPH_HYBRID_MAX_THREADS"):
        m = re.search(r"#define\s+%s\s+\(?([0-9xXa-fA-F]+)u?(?:\s*<<\s*(\d+))?" % name, src)
        assert m, name
        val = int(m.group(1), 0) << (int(m.group(2)) if m.group(2) else 0)
        assert getattr(_lib, name) == val, name


def test_python_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1312_3018_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "lib_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        _lib.load()
