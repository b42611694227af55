"""The boundary is a C ABI: a plain C99 program includes ``include/prc_lbm.h``,
links the shared library and calls its host-only entry points (parameter
set-up and checks, the viscosity-to-relaxation mapping of Eq.
transport-coefficients, workspace sizing).  No GPU is needed for these calls.
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
