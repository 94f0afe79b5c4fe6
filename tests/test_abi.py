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


def test_binding_structs_match_the_header(tmp_path):
    """Sizes and field offsets of the ctypes mirrors equal those the C compiler gives the header's
    structs (the binding marshals them by address)."""
    import shutil
    import subprocess

    import pytest
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = []
    for cname, py in (("cortex_params", cortex.Params), ("cortex_options", cortex.Options),
                      ("cortex_stats_t", cortex.Stats)):
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "cortex.h"\nint main(void) {\n' +
                   "\n".join(lines) + "\nreturn 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-std=c11", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)])
    got = dict((" ".join(l.split()[:2]), int(l.split()[2])) for l in subprocess.check_output([str(exe)]).decode().splitlines())
    for cname, py in (("cortex_params", cortex.Params), ("cortex_options", cortex.Options),
                      ("cortex_stats_t", cortex.Stats)):
        assert got[f"{cname} size"] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[f"{cname} {f}"] == getattr(py, f).offset, (cname, f)


def test_option_checks_before_any_device_call():
    """Invalid options are refused with CORTEX_ERR_ARG before the device is touched: balance 2
    without per-network costs, or with a cost that is not finite and positive."""
    from paper_2406_03762_gb300 import workloads as W
    L = cortex.load()
    specs, seeds = W.small_batch_specs()
    arr = (cortex.Params * len(specs))(*[cortex.params_from_spec(s) for s in specs])
    sd = (ctypes.c_uint64 * len(specs))(*seeds)
    h = ctypes.c_void_p(None)
    for opts in (cortex.make_options(balance=2), cortex.make_options(balance=3),
                 cortex.make_options(balance=2, net_work=[1.0] * (len(specs) - 1) + [0.0]),
                 cortex.make_options(balance=2, net_work=[1.0] * (len(specs) - 1) + [float("nan")])):
        assert L.cortex_build_batch(arr, sd, len(specs), ctypes.byref(opts), None, ctypes.byref(h)) == -1
        assert h.value is None


def test_checkpoint_calls_check_their_arguments_without_gpu():
    L = cortex.load()
    buf = (ctypes.c_float * 4)()
    assert L.cortex_get_ring(None, 0, buf) == -1
    assert L.cortex_set_state(None, 0, None, None, None, None) == -1
    assert L.cortex_set_step(None, 0) == -1
