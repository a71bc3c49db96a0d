"""The C-ABI library loads on a CPU-only host and exports every declared symbol."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header, where=os.path.join(ROOT, "include")):
    txt = open(os.path.join(where, header)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(nef_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2602_02759_gb300 import build
    return ctypes.CDLL(build.build())


PROBE = os.path.join(ROOT, "tests", "tc_probe")


def test_headers_match_binding_lists():
    import paper_2602_02759_gb300 as nef
    assert _declared("nef.h") == sorted(nef.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared("nef.h"):
        assert hasattr(lib, name), name


def test_probe_entry_points_live_only_in_the_test_library(lib):
    """The tensor-core probes (tests/tc_probe/nef_probe.h) are built into the
    test-only libnef_probe.so and are absent from the product library."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("nef_probe_build", os.path.join(PROBE, "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    probe = ctypes.CDLL(mod.build())
    names = _declared("nef_probe.h", PROBE)
    assert names == ["nef_tc_gemm", "nef_tc_gemm_split", "nef_tc_probe"]
    for name in names:
        assert hasattr(probe, name), name
        assert not hasattr(lib, name), name


def test_defaults_and_errors_without_gpu(lib):
    """Calls that need no device work return their documented status codes."""
    import paper_2602_02759_gb300._nef as b
    L = b.load()
    o = b.Options()
    L.nef_default_options(ctypes.byref(o))
    assert o.precision == 0 and o.eps == pytest.approx(1e-10) and o.force_generic == 0
    h = ctypes.c_void_p()
    shapes = (ctypes.c_int64 * 3)(2, 2, 2)
    ranks = (ctypes.c_int64 * 1)(2)
    assert L.nef_plan(b"ir,jr,kr", shapes, 3, ranks, 1, None, ctypes.byref(h)) == 2
    assert b"->" in L.nef_last_error()
    assert L.nef_plan(b"ir,jr,kr->ijk", shapes, 2, ranks, 1, None, ctypes.byref(h)) == 1
    assert L.nef_fit(None, None, None, None, 1.0, 0.0, 1) == 1


@pytest.mark.parametrize("lang,std", [("c", "-std=c11"), ("c++", "-std=c++17")])
def test_headers_are_plain_c(lang, std, tmp_path):
    """The public headers compile on their own as C11 (pedantic) and as C++:
    plain types and pointers only, no CUDA, C++ or torch types."""
    import subprocess
    src = tmp_path / ("h.c" if lang == "c" else "h.cpp")
    src.write_text('#include "nef.h"\n#include "nef_probe.h"\nint main(void) { return 0; }\n')
    cc = "gcc" if lang == "c" else "g++"
    r = subprocess.run([cc, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                        "-I", os.path.join(ROOT, "include"), "-I", PROBE, str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
