"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function include/twa.h declares, and rejects bad arguments before it
touches the device."""
import ctypes
import math
import os
import subprocess

import pytest

from paper_2608_10075_b300 import twa


def test_library_exports_every_declared_function():
    names = twa.header_functions()
    assert len(names) >= 12
    L = twa.lib()
    for n in names:
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", twa.LIB_PATH], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert set(names) <= exported
    # nothing but the declared API leaks out of the library
    assert {e for e in exported if e.startswith("twa")} == set(names)


def test_binding_signatures_cover_header():
    assert set(twa.header_functions()) == set(twa._SIGNATURES)


@pytest.mark.parametrize("pyclass,ctype", [(twa.Opts, "twa_opts"), (twa.Obs, "twa_obs"),
                                           (twa.GradReq, "twa_grad_req"), (twa.GradOut, "twa_grad_out"),
                                           (twa.Point, "twa_point")])
def test_struct_layouts_match_header(tmp_path, pyclass, ctype):
    # compile the header with the host C compiler and compare sizes and offsets
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    src = tmp_path / "layout.c"
    fields = [f for f, _ in pyclass._fields_]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "twa.h"', "int main(void) {",
             '  printf("%%zu\\n", sizeof(%s));' % ctype]
    lines += ['  printf("%%zu\\n", offsetof(%s, %s));' % (ctype, f) for f in fields]
    lines += ["  return 0; }"]
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I" + inc, str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert vals[0] == ctypes.sizeof(pyclass)
    assert vals[1:] == [getattr(pyclass, f).offset for f in fields]


def test_defaults():
    o = twa.Opts()
    assert twa.lib().twa_opts_default(ctypes.byref(o)) == 0
    assert (o.precision, o.init_state, o.window_start, o.renormalize, o.clip_negative) == (0, -1, 0.0, 1, 0)
    assert twa.lib().twa_opts_default(None) == -1


@pytest.mark.parametrize("args,frag", [
    ((0, 1.0, 1.0, 1.0, 0.1), "N must"),
    ((70000, 1.0, 1.0, 1.0, 0.1), "N must"),
    ((4, -1.0, 1.0, 1.0, 0.1), "alpha"),
    ((4, math.nan, 1.0, 1.0, 0.1), "alpha"),
    ((4, 1.0, -2.0, 1.0, 0.1), "w must"),
    ((4, 1.0, math.inf, 1.0, 0.1), "w must"),
    ((4, 1.0, 1.0, -1.0, 0.1), "Gamma"),
    ((4, 1.0, 1.0, 1.0, 0.0), "dt"),
    ((4, 1.0, 1.0, 1.0, math.nan), "dt"),
])
def test_init_rejects_bad_parameters(args, frag):
    with pytest.raises(twa.TWAError) as e:
        twa.TWA(*args)
    assert e.value.code == -1 and frag in str(e.value)
    assert frag in twa.last_error(None)


def test_init_rejects_bad_options():
    with pytest.raises(twa.TWAError) as e:
        twa.TWA(4, 1.0, 1.0, 1.0, 0.1, precision=-1)
    assert e.value.code == -1
    with pytest.raises(twa.TWAError) as e:
        twa.TWA(4, 1.0, 1.0, 1.0, 0.1, precision=8)          # one past TWA_PREC_BF16B
    assert e.value.code == -1 and "precision" in str(e.value)
    with pytest.raises(twa.TWAError) as e:
        twa.TWA(4, 1.0, 1.0, 1.0, 0.1, integrator=2)
    assert e.value.code == -1 and "integrator" in str(e.value)
    with pytest.raises(twa.TWAError) as e:
        twa.TWA(4, 1.0, 1.0, 1.0, 0.1, integrator=-1)
    assert e.value.code == -1
    with pytest.raises(twa.TWAError) as e:
        twa.TWA(4, 1.0, 1.0, 1.0, 0.1, init_state=0)
    assert e.value.code == -1
    with pytest.raises(twa.TWAError) as e:
        twa.TWA(4, 1.0, 1.0, 1.0, 0.1, window_start=-1.0)
    assert e.value.code == -1
    with pytest.raises(twa.TWAError) as e:
        twa.TWA(4, 1.0, 1.0, 1.0, 0.1, precision="bf16x3", ws_route="fft", noise_route=3)
    assert e.value.code == -1 and "noise_route" in str(e.value)
    # the circulant draw exists only beside the FFT pump field
    with pytest.raises(twa.TWAError) as e:
        twa.TWA(4, 1.0, 1.0, 1.0, 0.1, precision="bf16x3", noise_route="circulant")
    assert e.value.name == "TWA_EUNSUPPORTED"


def test_precision_and_integrator_constants_match_the_header():
    # the binding's names are the header's values
    import re
    hdr = open(os.path.join(os.path.dirname(twa.LIB_PATH), "..", "include", "twa.h")).read()
    val = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define (TWA_\w+)\s+(-?\d+)", hdr)}
    assert twa.PRECISION == {"fp64": val["TWA_PREC_FP64"], "bf16": val["TWA_PREC_BF16"],
                             "bf16x3": val["TWA_PREC_BF16X3"], "tf32": val["TWA_PREC_TF32"],
                             "fp32": val["TWA_PREC_FP32"], "bf16x2": val["TWA_PREC_BF16X2"],
                             "bf16l2": val["TWA_PREC_BF16L2"], "bf16b": val["TWA_PREC_BF16B"]}
    assert twa.INTEGRATOR == {"heun": val["TWA_INT_HEUN"], "midpoint": val["TWA_INT_MIDPOINT"]}
    import ctypes
    o = twa.Opts()
    ctypes.memset(ctypes.byref(o), 0xFF, ctypes.sizeof(o))   # the defaults overwrite every byte
    twa.lib().twa_opts_default(ctypes.byref(o))
    assert o.integrator == val["TWA_INT_HEUN"] and o.precision == val["TWA_PREC_FP64"]
    assert o.sample_stride == 1 and not o.alloc and not o.free


def test_null_context_calls_are_rejected():
    L = twa.lib()
    assert L.twa_run(None, 4, 1) == -1
    assert L.twa_sync(None) == -1
    assert L.twa_observables(None, None) == -1
    L.twa_destroy(None)


def test_built_for_sm103a():
    # the library carries sm_103a device code only (checked from the build flags)
    from paper_2608_10075_b300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(twa.LIB_PATH)
