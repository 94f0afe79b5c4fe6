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


def test_parameter_limits_are_refused_before_any_device_call():
    """Parameters outside the method's domain (CORTEX_ERR_ARG) or beyond the layout's fields
    (CORTEX_ERR_UNSUPPORTED: in-degree in a 16-bit draw index, d_max in the 8-bit delay span, the
    16-bit refractory counter) are refused by the host with a reason, before the device is touched,
    and leave no handle."""
    from paper_2406_03762_gb300 import workloads as W
    L = cortex.load()
    base = W.NetSpec(800, 200, 80, 20)
    cases = [
        (dict(n_exc=0, n_inh=0), cortex.ERR_ARG, "neuron counts"),
        (dict(k_exc=-1), cortex.ERR_ARG, "in-degree"),
        (dict(n_inh=0, k_inh=5), cortex.ERR_ARG, "empty population"),
        (dict(k_exc=60000, k_inh=5536), cortex.ERR_UNSUPPORTED, "in-degree above 65535"),
        (dict(d_min=0), cortex.ERR_ARG, "d_min"),
        (dict(d_min=5, d_max=4), cortex.ERR_ARG, "d_min"),
        (dict(d_max=256), cortex.ERR_UNSUPPORTED, "d_max above 255"),
        (dict(tau_syn=10.0), cortex.ERR_UNSUPPORTED, "singular propagator"),
        (dict(dt=0.0), cortex.ERR_ARG, "positive"),
        (dict(t_ref=3276.8), cortex.ERR_UNSUPPORTED, "refractory counter"),
        (dict(nu_ext_hz=float("nan")), cortex.ERR_ARG, "nu_ext_hz"),
        (dict(weight_dtype=7), cortex.ERR_ARG, "weight_dtype"),
        (dict(e_l=-70.0), cortex.ERR_UNSUPPORTED, "E_L"),
    ]
    for change, code, why in cases:
        p = cortex.params_from_spec(base)
        for k, v in change.items():
            setattr(p, k, v)
        h = ctypes.c_void_p(None)
        rc = L.cortex_build(ctypes.byref(p), 1, None, None, ctypes.byref(h))
        assert rc == code, change
        assert h.value is None, change
        assert why in L.cortex_last_error().decode(), change
    # the limits themselves pass the parameter check: the host-only planner accepts them
    p = cortex.params_from_spec(base)
    p.k_exc, p.k_inh, p.d_max = 60000, 5535, 255
    tb, nb = (ctypes.c_int32 * 1)(), ctypes.c_int32(0)
    assert L.cortex_plan(ctypes.byref(p), 1, None, 152, 232448, tb, ctypes.byref(nb)) == cortex.OK
    assert nb.value >= 1 and 1 <= tb[0] <= base.n
