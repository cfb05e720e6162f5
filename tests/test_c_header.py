"""The C ABI from plain C, with no Python or torch in between: include/dgswem.h compiles as strict
C99 with every warning an error, and a program linked against libdgswem.so validates a mesh,
sizes its workspace, refuses a step before attach and rejects a clockwise triangle, using only
the header's types and status codes (no device work: creation is host-only)."""
import os
import shutil
import subprocess

import pytest

from paper_2508_21208_gb300.build import LIB, build_library

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include "dgswem.h"

static dgswem_params defaults(void) {
  dgswem_params p = {0};
  p.p = 1;
  p.precision = DGSWEM_FP64;
  p.g = 9.81;
  p.cfl = 0.3;
  p.tide_period = 44714.0;
  p.pc_hpa = 950.0;
  p.pn_hpa = 1013.0;
  p.rmax_m = 40e3;
  p.holland_b = 1.5;
  p.vt_ms = 5.0;
  p.rho_air = 1.15;
  p.rho_water = 1000.0;
  p.rk_scheme = DGSWEM_RK_SSP22;
  p.flux = DGSWEM_FLUX_LLF;
  return p;
}

int main(void) {
  const double xy[] = {0, 0, 100, 0, 100, 100, 0, 100};
  const int32_t tri[] = {0, 1, 2, 0, 2, 3};
  const int32_t clockwise[] = {0, 2, 1};
  const double hb[] = {10, 10, 10, 10};
  const dgswem_mesh mesh = {4, 2, 0, xy, tri, NULL, NULL};
  const dgswem_mesh bad = {4, 1, 0, xy, clockwise, NULL, NULL};
  const dgswem_params p = defaults();
  dgswem_ctx *c = NULL, *c2 = NULL;
  size_t ws = 0;
  int rc = dgswem_create(&mesh, hb, &p, NULL, NULL, &c);
  int ws_rc = rc == DGSWEM_OK ? dgswem_workspace_size(c, &ws) : rc;
  int step_rc = rc == DGSWEM_OK ? dgswem_step(c, 1) : rc;
  int bad_rc = dgswem_create(&bad, hb, &p, NULL, NULL, &c2);
  dgswem_destroy(c);
  printf("%d %d %zu %d %d %d\n", rc, ws_rc, ws, step_rc, bad_rc, c2 == NULL);
  return 0;
}
"""


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs a C compiler")
def test_header_is_c99_and_the_library_links_from_c(tmp_path):
    build_library()
    src = tmp_path / "use_dgswem.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "use_dgswem"
    libdir = os.path.dirname(LIB)
    subprocess.run(["gcc", "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror",
                    "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe), LIB,
                    f"-Wl,-rpath,{libdir}"], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    rc, ws_rc, ws, step_rc, bad_rc, c2_null = (int(v) for v in out)
    assert rc == 0 and ws_rc == 0 and ws > 0
    assert step_rc == -8           # DGSWEM_ESTATE: no workspace attached yet
    assert bad_rc == -2 and c2_null == 1   # DGSWEM_EMESH, *out left NULL
