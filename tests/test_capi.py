"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/tmloops.h (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "tmloops.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_A-Z]*)\s*\(",
                       text, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "return", "sizeof")))


def test_header_declares_the_six_named_calls():
    names = _declared()
    for n in ["tm_dslash", "tm_cg_solve", "z4_noise", "loop_contract_local", "loop_contract_oneD",
              "tsm_combine"]:
        assert n in names


def test_library_builds_loads_and_exports_every_declared_symbol():
    from paper_1401_6749_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1401_6749_gb300 import build
    build.build()
    from paper_1401_6749_gb300 import tmloops
    assert set(_declared()) == set(tmloops.EXPORTED)
    # host-only calls work without a GPU
    assert tmloops.tm_spinor_bytes((4, 4, 4, 4), tmloops.F32, 2) == 256 * 24 * 4 * 2
    assert tmloops.tm_spinor_bytes((4, 4, 4, 4), tmloops.F16, 1) == 256 * 24 * 2
    assert tmloops.tm_launch_count() >= 0
