"""The C ABI from C: a C99 program that includes include/tpfa.h (warnings as
errors), links libtpfa.so and calls entry points that reject their arguments
before any CUDA call, so it runs without a GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2408_03452_gb300")

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "tpfa.h"

#define EXPECT(cond) do { if (!(cond)) { printf("failed: %s\n", #cond); return 1; } } while (0)

int main(void) {
  tpfa_ctx* ctx = NULL;
  tpfa_batch* batch = NULL;
  tpfa_unet* net = NULL;
  EXPECT(tpfa_abi_version() > 0);
  EXPECT(strlen(tpfa_strerror(TPFA_EINVAL)) > 0);
  EXPECT(tpfa_create(NULL, &ctx) == TPFA_EINVAL && ctx == NULL);
  EXPECT(tpfa_destroy(NULL) == TPFA_EINVAL);
  EXPECT(cg_solve(NULL, NULL, NULL, NULL, NULL, 1e-8, 10, NULL, NULL) == TPFA_EINVAL);
  EXPECT(tpfa_batch_create(NULL, 0, NULL, &batch) == TPFA_EINVAL && batch == NULL);
  EXPECT(fcg_solve_batch(NULL, NULL, 0, NULL, NULL, NULL, NULL, NULL, NULL, 1e-8, 10, NULL, NULL,
                         NULL, NULL) == TPFA_EINVAL);
  EXPECT(tpfa_unet_create(6, 8, 8, 1, 0, &net) == TPFA_EINVAL && net == NULL);
  EXPECT(tpfa_unet_param_count() == 146625);
  EXPECT(tpfa_restrict_levels(NULL, NULL, 8, 8, 8, 1, 0, NULL) == TPFA_EINVAL);
  EXPECT(tpfa_tc_wait_probe(0, NULL) == TPFA_EINVAL);
  printf("ok\n");
  return 0;
}
"""


def test_header_compiles_as_c99_and_the_library_links(tmp_path):
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("gcc not available")
    lib = os.path.join(PKG, "libtpfa.so")
    if not os.path.exists(lib):
        from paper_2408_03452_gb300 import build
        build.build()
    src = tmp_path / "consumer.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "consumer"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I",
                        os.path.join(ROOT, "include"), str(src), "-L", PKG, "-ltpfa",
                        "-Wl,-rpath," + PKG, "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
