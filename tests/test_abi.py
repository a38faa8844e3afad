"""The C ABI library builds for sm_103a, loads without a GPU and exports
every entry point that include/mad.h declares (no compute calls)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(mad_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libmad():
    if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
        pytest.skip("nvcc not available")
    from paper_1506_03872_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_pipeline():
    names = _declared()
    for must in ("mad_build_tables", "mad_sample", "mad_topk", "mad_rescore"):
        assert must in names


def test_every_declared_symbol_is_exported(libmad):
    for name in _declared():
        assert hasattr(libmad, name), name


def test_binding_covers_the_header():
    import paper_1506_03872_gb300 as mad
    assert sorted(mad.EXPORTS) == _declared()


def test_strerror_without_gpu(libmad):
    libmad.mad_strerror.restype = ctypes.c_char_p
    libmad.mad_strerror.argtypes = [ctypes.c_int]
    assert libmad.mad_strerror(0) == b"success"
    assert b"hash" in libmad.mad_strerror(6)


def test_struct_layouts_match_header():
    import paper_1506_03872_gb300 as mad
    assert ctypes.sizeof(mad.mad_pair) == 24
    assert ctypes.sizeof(mad.mad_matrix) == 56
    assert mad.mad_stats_t.device_error.offset + 4 == ctypes.sizeof(mad.mad_stats_t)
