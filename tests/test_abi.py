"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/sdc.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

from paper_1910_12578_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sdc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sdc_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_hot_path_calls():
    names = declared_functions()
    for n in ["sdc_init_box", "sdc_advective_term", "sdc_node_integral", "sdc_react_newton", "sdc_step"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = B.build()
    L = ctypes.CDLL(lib)
    for n in declared_functions():
        assert hasattr(L, n), n


def test_status_strings_without_gpu():
    from paper_1910_12578_gb300 import sdc
    L = sdc.load()
    for s in range(7):
        assert L.sdc_status_string(s)
    assert L.sdc_status_string(99) == b"unknown status"


def test_init_rejects_bad_arguments_without_touching_the_gpu():
    """Argument checks run before any CUDA call."""
    from paper_1910_12578_gb300 import sdc
    L = sdc.load()
    out = ctypes.c_void_p()
    assert L.sdc_init_box(None, 1, None, None, None, ctypes.byref(out)) == sdc.SDC_ERR_INVALID_ARG
    boxes = (sdc.Box * 1)()
    boxes[0].dim = 5
    net = sdc.Network()
    prm = sdc.Params()
    assert L.sdc_init_box(boxes, 1, ctypes.byref(net), ctypes.byref(prm), None, ctypes.byref(out)) == \
        sdc.SDC_ERR_INVALID_ARG
    assert out.value is None


def test_binding_structures_match_the_header(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets that
    a C compiler gives the header's struct (compiled here with gcc)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    from paper_1910_12578_gb300 import sdc
    pairs = {"sdc_box": sdc.Box, "sdc_network": sdc.Network, "sdc_params": sdc.Params, "sdc_stats": sdc.Stats,
             "sdc_profile": sdc.Profile, "sdc_tuning": sdc.Tuning}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "sdc.h"', "int main(void) {"]
    for cname, py in pairs.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in py._fields_:
            lines.append(f'    printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in pairs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f in py._fields_:
            assert got[(cname, f[0])] == getattr(py, f[0]).offset, (cname, f[0])


def test_pow_tables_header_is_the_generator_output():
    """sdc_pow_tables.h is exactly what the committed gen_pow_tables.py writes."""
    import subprocess
    import sys
    d = os.path.join(ROOT, "paper_1910_12578_gb300", "csrc")
    out = subprocess.run([sys.executable, "gen_pow_tables.py"], cwd=d, check=True, capture_output=True,
                         text=True).stdout
    assert out == open(os.path.join(d, "sdc_pow_tables.h")).read()


def test_pow_tables_hold_their_defining_values():
    """Every table entry against its definition in double arithmetic (an
    independent check of the generator): 2^(i/256), c_j (1 + (j + 1/2)/128) = 1,
    hi + lo = log2(1/c_j), and the Taylor coefficients."""
    import math
    src = open(os.path.join(ROOT, "paper_1910_12578_gb300", "csrc", "sdc_pow_tables.h")).read()

    def table(name):
        body = re.search(name + r"\[\d+\] = \{(.*?)\};", src, re.S).group(1)
        return [float.fromhex(t.strip()) for t in body.split(",") if t.strip()]

    def const(name):
        return float.fromhex(re.search(r"constexpr double " + name + r" = (\S+);", src).group(1))

    e2 = table("POW_EXP2_T")
    assert len(e2) == 256
    for i, v in enumerate(e2):
        assert abs(v - 2.0 ** (i / 256)) <= 2.3e-16 * v
    c, hi, lo = table("POW_LOG_C"), table("POW_LOG_HI"), table("POW_LOG_LO")
    assert len(c) == len(hi) == len(lo) == 128
    for j in range(128):
        assert abs(c[j] * (1 + (j + 0.5) / 128) - 1) <= 2.3e-16
        assert abs(hi[j] + lo[j] + math.log2(c[j])) <= 4e-16
        assert abs(lo[j]) <= 1.2e-16 * max(hi[j], 2.0 ** -60)
    for n in range(1, 7):
        assert const("POW_LOG_A%d" % n) == pytest.approx((-1) ** (n + 1) / (n * math.log(2)), rel=2e-16)
    for n in range(1, 5):
        assert const("POW_EXP_B%d" % n) == pytest.approx(math.log(2) ** n / math.factorial(n), rel=4e-16)
