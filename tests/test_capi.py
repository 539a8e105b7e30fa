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


def test_header_is_plain_c_and_host_calls_link_and_run(tmp_path):
    """A C99 program includes the header with every warning an error, links
    against the library and runs the host-only calls (no GPU needed)."""
    import shutil
    import subprocess
    import pytest
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    from paper_1401_6749_gb300 import build
    lib = build.build()
    src = tmp_path / "main.c"
    src.write_text(r'''
#include <math.h>
#include <stdio.h>
#include "tmloops.h"
int main(void) {
  tm_geom_t g = {{4, 4, 4, 4}};
  if (tm_spinor_bytes(&g, TM_PREC_FF, 2) != (size_t)256 * 24 * 8 * 2) return 1;
  if (tm_spinor_bytes(&g, TM_PREC_F16, 1) != (size_t)256 * 24 * 2) return 2;
  tm_params_t p = {{4, 4, 4, 4}, 0.16, 0.0, 1, 0};
  double out[16 * 4 * 2];
  if (tm_hpe_exact(&p, out) != TM_OK) return 3;
  /* mu = 0: B = 1 and (1 - g)(1 + g) = 0 kills the second order, so
     Tr_t[B - BHB + (BH)^2 B - (BH)^3 B] = 12 x 64 sites on every slice */
  for (int t = 0; t < 4; ++t)
    if (fabs(out[2 * t] - 768.0) > 1e-9 || fabs(out[2 * t + 1]) > 1e-9) return 4;
  p.recon = 7;
  tm_op_t *op = NULL;
  if (tm_op_create(&op, &p, (const double *)out, NULL) != TM_ERR_ARG) return 5;
  if (tm_last_error()[0] == 0) return 6;
  if (tm_mem_reserved(NULL) != TM_ERR_ARG) return 7;
  if (tm_dslash_mma_enable(0) != TM_OK) return 8;  /* switching off needs no device */
  printf("ok\n");
  return 0;
}
''')
    inc = os.path.join(ROOT, "include")
    libdir = os.path.dirname(lib)
    exe = tmp_path / "main"
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", inc, str(src),
                        "-o", str(exe), "-L", libdir, "-ltmloops", "-lm", "-Wl,-rpath," + libdir],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True)
    assert run.returncode == 0 and run.stdout.strip() == "ok", (run.returncode, run.stdout, run.stderr)
