"""The C-ABI library builds, loads without a GPU and exports every symbol
that include/sqrtba.h declares (no compute calls here)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sqrtba.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"SQRTBA_API\s+[\w\s\*]*?\b(ba_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def built_lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2103_01843_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ba_create", "ba_linearize", "ba_marginalize_qr", "ba_pcg_solve",
                     "ba_backsubstitute", "ba_eval_cost", "ba_lm_step", "ba_destroy"):
        assert required in names


def test_library_loads_and_exports_all_declared_symbols(built_lib):
    lib = ctypes.CDLL(built_lib)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_match_header(built_lib):
    import paper_2103_01843_gb300 as pkg
    assert sorted(pkg.exported_symbols()) == declared_functions()
    pkg.lib()  # loads, sets argtypes for every declared function


def test_no_internal_symbols_leak(built_lib):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", built_lib], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert exported == set(declared_functions()), exported ^ set(declared_functions())


def test_default_options_without_gpu(built_lib):
    import paper_2103_01843_gb300 as pkg
    o = pkg.default_options()
    assert o.lambda0 == 1e-4 and o.max_lm_iters == 50 and o.func_tol == 1e-6
    assert o.max_cg_iters == 500 and o.cg_eta == 0.1


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_2103_01843_gb300 as pkg
    monkeypatch.setattr(pkg, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(pkg, "_lib", None)
    with pytest.raises(pkg.BAError):
        pkg.lib()
