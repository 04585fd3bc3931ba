"""The C ABI from plain C: both public headers compile as strict C99 with
every warning an error, a program links against libdgsigma.so and runs.
Without a device, dg_create must return DG_ECUDA with a NULL handle and the
program must end normally; with one, the same program runs a small Sigma
solve (the usage sequence the README shows)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include "dgsigma.h"
#include "dgsurrogate.h"

int main(void) {
  const double cx[2] = {2.0, 7.0}, cy[2] = {2.0, 7.0}, r[2] = {1.0, 1.2};
  const double xy[2] = {5.0, 5.0};
  double sigma[3], mu[2];
  dg_config cfg;
  dg_ctx *ctx = NULL;
  int rc;
  dg_config_default(&cfg);
  cfg.p = 3;
  cfg.precision = DG_FP32;
  rc = dg_create(&cfg, &ctx);
  if (rc != DG_OK) {
    printf("dg_create: %d %s handle=%s\n", rc, dg_strerror(rc), ctx ? "set" : "null");
    return 0;
  }
  rc = dg_set_geometry_disks(ctx, cx, cy, r, 2, 10.0, 32, 3);
  if (rc == DG_OK) rc = dg_set_sources(ctx, xy, 1);
  if (rc == DG_OK) rc = dg_propagate_to(ctx, 0.5);
  if (rc == DG_OK) rc = dg_covariance(ctx, sigma, mu, NULL);
  if (rc != DG_OK) printf("error %d: %s\n", rc, dg_last_error(ctx));
  else printf("sigma %.6e %.6e %.6e\n", sigma[0], sigma[1], sigma[2]);
  dg_destroy(ctx);
  return rc == DG_OK ? 0 : 1;
}
"""


def _compile_and_run(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_1907_06191_gb300 import _build
    lib = _build.build()
    src = tmp_path / "use_dgsigma.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "use_dgsigma"
    libdir = os.path.dirname(lib)
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
           "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
           "-L", libdir, "-ldgsigma", "-Wl,-rpath," + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    return r.stdout.strip()


def _check_sigma(out):
    assert out.startswith("sigma "), out
    sxx, sxy, syy = (float(v) for v in out.split()[1:])
    # free diffusion would give 2 D t = 2 um^2; walls only lower it
    assert 0 < sxx < 2.0 + 1e-6 and 0 < syy < 2.0 + 1e-6 and sxx * syy > sxy ** 2


def test_c_program_compiles_links_and_runs(tmp_path):
    out = _compile_and_run(tmp_path)
    if out.startswith("dg_create"):
        # no usable device here: an error status, no handle, no crash
        assert out == "dg_create: 3 CUDA error handle=null", out
    else:
        _check_sigma(out)


@pytest.mark.gpu
def test_c_program_sigma_solve_on_the_gpu(tmp_path):
    """The plain-C usage sequence (create, disks, start point, propagate_to,
    covariance, destroy) on a device: it must take the solve branch."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _check_sigma(_compile_and_run(tmp_path))
