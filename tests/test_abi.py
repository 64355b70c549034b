"""Host-side checks of the C ABI: the library loads without a GPU, exports every
function include/gpl1.h declares, and the Python structures match the C
layouts.  No compute call is made here."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_0902_4424_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gpl1.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gpl1_[a-z0-9_]+)\s*\(", txt)))


def test_library_loads_and_exports_every_declared_symbol():
    L = pkg.lib()
    decl = declared_functions()
    assert len(decl) >= 8
    for name in decl:
        assert hasattr(L, name), name
    assert sorted(pkg.EXPORTS) == decl
    out = subprocess.run(["nm", "-D", "--defined-only", pkg.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (gpl1_\w+)", out))
    assert set(decl) <= exported


def test_params_default_are_the_papers():
    prm = pkg.params_default()
    assert (prm.M, prm.theta, prm.beta) == (1, 0.5, 1e-4)
    assert (prm.alpha_min, prm.alpha_max, prm.tau1, prm.M_alpha) == (1e-10, 1e10, 0.5, 2)
    assert prm.alpha0_rule == 0 and prm.max_backtracks == 100 and prm.timeout_ns > 0


def test_struct_layouts_match_header(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text(f'''#include <stdio.h>
#include <stddef.h>
#include "{HEADER}"
int main(void) {{
  printf("%zu %zu %zu\\n", sizeof(gpl1_params), sizeof(gpl1_result), sizeof(gpl1_problem));
  printf("%zu %zu %zu %zu %zu %zu\\n", offsetof(gpl1_params, timeout_ns), offsetof(gpl1_result, fail_iter), offsetof(gpl1_problem, trace_cap),
         offsetof(gpl1_params, method), offsetof(gpl1_params, step), offsetof(gpl1_params, tile));
  return 0;
}}''')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-o", str(exe), str(src)])
    a, b = subprocess.check_output([str(exe)], text=True).split("\n")[:2]
    assert [int(v) for v in a.split()] == [ctypes.sizeof(pkg.Params), ctypes.sizeof(pkg.Result),
                                           ctypes.sizeof(pkg.Problem)]
    assert [int(v) for v in b.split()] == [pkg.Params.timeout_ns.offset, pkg.Result.fail_iter.offset,
                                           pkg.Problem.trace_cap.offset, pkg.Params.method.offset,
                                           pkg.Params.step.offset, pkg.Params.tile.offset]


def test_null_context_is_rejected_without_a_gpu():
    L = pkg.lib()
    assert L.gpl1_last_error(None) == b"null context"
    prm = pkg.params_default()
    res = pkg.Result()
    assert L.gpl1_solve(None, None, 1, ctypes.byref(prm), ctypes.byref(res)) == 1
    assert L.gpl1_project(None, None, None, 1, 10, 1, 10, None, 0, None) == 1


def test_parameter_checks_run_before_any_device_call():
    """gpl1_solve_noalloc checks its parameters on the host before it touches a
    device, so the refusals are visible without a GPU: an engine or tile out of
    range, and the comparison methods (single solves only)."""
    L = pkg.lib()
    res = pkg.Result()
    err = ctypes.create_string_buffer(256)
    for over, word in (({"tile": 4}, b"tile"), ({"tile": -1}, b"tile"), ({"engine": 9}, b"engine"),
                       ({"method": pkg.METHOD_FISTA}, b"ISTA")):
        prm = pkg.params_default(**over)
        st = L.gpl1_solve_noalloc(None, 1, ctypes.byref(prm), ctypes.byref(res), None, err, 256)
        assert st in (1, 7) and word in err.value, (over, st, err.value)
