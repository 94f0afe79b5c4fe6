"""The C-ABI library loads and exports every function include/cortex.h declares (no GPU needed:
loading the library makes no CUDA call).  Also checks the binding covers the same names."""
import ctypes
import os
import re

from paper_2406_03762_gb300 import _build, cortex

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "cortex.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w\*\s]+?\b(cortex_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("cortex_build", "cortex_build_batch", "cortex_simulate", "cortex_spikes", "cortex_stats",
                     "cortex_free", "cortex_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol():
    path = _build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(cortex.EXPORTED) == declared_functions()


def test_strerror_without_gpu():
    lib = ctypes.CDLL(_build.build())
    lib.cortex_strerror.restype = ctypes.c_char_p
    assert lib.cortex_strerror(0) == b"ok"
    assert b"timed out" in lib.cortex_strerror(-4)
