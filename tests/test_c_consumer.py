"""The boundary is a C ABI: a plain C99 program includes ``include/prc_lbm.h``,
links the shared library and calls its host-only entry points (parameter
set-up and checks, the viscosity-to-relaxation mapping of Eq.
transport-coefficients, workspace sizing).  No GPU is needed for these calls.
A second program (GPU) creates a cavity with lbm_create, steps it with
lbm_step and reads its fields with lbm_fields into host arrays, and compares
them with the FP64 oracle's fields of the same run
(``golden/c_consumer_oracle.txt``, written by
``golden/make_c_consumer_oracle.py``).
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

PROGRAM = r"""
#include <stdio.h>
#include <math.h>
#include "prc_lbm.h"

int main(void)
{
    lbm_params p;
    double w = 0.0;
    size_t bytes = 0;
    if (lbm_params_init(&p, 128, 128, 2.0, 0.1, 0.0088681, 0.0346410, LBM_F32) != LBM_OK) return 1;
    if (lbm_params_check(&p) != LBM_OK) return 2;
    if (lbm_omega_nu(&p, &w) != LBM_OK) return 3;
    /* nu = gamma q^2 c_s*^2 (1/omega - 1/2), q = min(1, r) = 1 */
    if (fabs(p.nu - p.gamma * (1.0 / 3.0) * (1.0 / w - 0.5)) > 1e-15) return 4;
    if (lbm_workspace_bytes(&p, &bytes) != LBM_OK || bytes < (size_t)2 * 9 * 128 * 128 * 4) return 5;
    p.gamma = 1.5; /* outside (0, 1] */
    if (lbm_params_check(&p) != LBM_EINVAL) return 6;
    printf("ok %.12f %zu\n", w, bytes);
    return 0;
}
"""


def test_plain_c_program_uses_the_abi(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    lib_dir = os.path.join(ROOT, "paper_2208_03562_gb300", "_build")
    if not cc:
        pytest.skip("no C compiler")
    if not os.path.exists(os.path.join(lib_dir, "libprc_lbm.so")):
        pytest.skip("library not built")
    src = tmp_path / "consumer.c"
    src.write_text(PROGRAM)
    exe = str(tmp_path / "consumer")
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", exe, "-L", lib_dir, "-lprc_lbm", "-Wl,-rpath," + lib_dir, "-lm"],
                   check=True, capture_output=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0, (out.returncode, out.stderr)
    assert out.stdout.startswith("ok ")


GPU_PROGRAM = r"""
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include "prc_lbm.h"

int main(int argc, char **argv)
{
    int nx, ny, steps;
    if (argc < 2) return 1;
    FILE *f = fopen(argv[1], "r");
    if (!f || fscanf(f, "%d %d %d", &nx, &ny, &steps) != 3) return 1;
    size_t n = (size_t)nx * ny;
    double *want = malloc(3 * n * sizeof(double)), *got = malloc(3 * n * sizeof(double));
    if (!want || !got) return 2;
    for (size_t k = 0; k < n; k++)
        if (fscanf(f, "%lf %lf %lf", &want[k], &want[n + k], &want[2 * n + k]) != 3) return 3;
    fclose(f);
    lbm_t h = NULL;
    if (lbm_create(nx, ny, 0.5, 0.25, 0.01, 0.03, LBM_F64, &h) != LBM_OK) {
        fprintf(stderr, "create: %s\n", lbm_last_error(NULL));
        return 4;
    }
    if (lbm_step(h, steps) != LBM_OK) return 5;
    if (lbm_fields(h, got, got + n, got + 2 * n, 0) != LBM_OK) return 6;
    double num = 0.0, den = 0.0, drho = 0.0;
    for (size_t k = 0; k < n; k++) {
        for (int c = 1; c < 3; c++) {
            double d = got[c * n + k] - want[c * n + k];
            num += d * d;
            den += want[c * n + k] * want[c * n + k];
        }
        double e = fabs(got[k] - want[k]);
        if (e > drho) drho = e;
    }
    lbm_destroy(h);
    printf("rel_l2_u %.3e max_drho %.3e\n", sqrt(num / den), drho);
    free(want);
    free(got);
    return sqrt(num / den) <= 1e-10 && drho <= 1e-12 ? 0 : 7;
}
"""


@pytest.mark.gpu
def test_plain_c_program_steps_a_cavity_and_matches_the_oracle(tmp_path):
    """lbm_create -> lbm_step -> lbm_fields from plain C99 with host arrays:
    FP64 GPU parity bar (1e-10 relative L2 of the velocity) against the
    stored oracle fields."""
    cc = shutil.which("gcc") or shutil.which("cc")
    lib_dir = os.path.join(ROOT, "paper_2208_03562_gb300", "_build")
    if not cc:
        pytest.skip("no C compiler")
    if not os.path.exists(os.path.join(lib_dir, "libprc_lbm.so")):
        pytest.skip("library not built")
    src = tmp_path / "stepper.c"
    src.write_text(GPU_PROGRAM)
    exe = str(tmp_path / "stepper")
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", exe, "-L", lib_dir, "-lprc_lbm", "-Wl,-rpath," + lib_dir, "-lm"],
                   check=True, capture_output=True)
    out = subprocess.run([exe, os.path.join(HERE, "golden", "c_consumer_oracle.txt")], capture_output=True, text=True)
    assert out.returncode == 0, (out.returncode, out.stdout, out.stderr)
    assert out.stdout.startswith("rel_l2_u ")
