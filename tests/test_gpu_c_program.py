"""The boundary used from C alone: a C99 program reads links from a file,
fixes them through include/lgf.h on the GPU and prints what lgf_fix returns;
the result must be the oracle's."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1301_3460_gb300 import build, inputs

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include "lgf.h"
#include <stdio.h>
#include <stdlib.h>
int main(int argc, char** argv) {
    int dims[4] = {atoi(argv[2]), atoi(argv[3]), atoi(argv[4]), atoi(argv[5])};
    size_t V = (size_t)dims[0] * dims[1] * dims[2] * dims[3];
    size_t n = 4 * V * 18;
    double* U = malloc(n * sizeof(double));
    FILE* f = fopen(argv[1], "rb");
    if (!f || fread(U, sizeof(double), n, f) != n) return 3;
    fclose(f);
    lgf_ctx* ctx = 0;
    int rc = lgf_create(dims, LGF_FP64, &ctx);
    if (rc != LGF_OK) { printf("create %d %s\n", rc, lgf_strerror(rc)); return 1; }
    rc = lgf_set_links(ctx, U, 0);
    if (rc != LGF_OK) { printf("set_links %d %s\n", rc, lgf_strerror(rc)); return 1; }
    int iters = 0; double F = 0, theta = 0;
    rc = lgf_fix(ctx, 0.08, 1e-15, 5000, &iters, &F, &theta);
    rc = rc == LGF_OK ? lgf_get_links(ctx, U, 0) : rc;
    f = fopen(argv[6], "wb");
    fwrite(U, sizeof(double), n, f);
    fclose(f);
    printf("%d %d %.17g %.17g\n", rc, iters, F, theta);
    lgf_destroy(ctx);
    free(U);
    return 0;
}
"""


def test_c_program_fixes_like_the_oracle(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    lib = build.build()
    src = tmp_path / "fix.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "fix"
    r = subprocess.run(["gcc", "-std=c99", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                        "-o", str(exe), lib, "-Wl,-rpath," + os.path.dirname(lib)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    L = (8, 8, 8, 4)
    U = inputs.rough_gauge_field(L, 0.3, 1234)
    fin, fout = tmp_path / "in.bin", tmp_path / "out.bin"
    U.astype(np.complex128).tofile(fin)
    out = subprocess.run([str(exe), str(fin), *map(str, L), str(fout)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    rc, iters, F, theta = out.stdout.split()
    ref = orc.fix(L, U, alpha=0.08, tol=1e-15, max_iter=5000)
    assert int(rc) == 0 and float(theta) < 1e-15
    assert abs(int(iters) - ref["iters"]) <= 1
    assert float(F) == pytest.approx(ref["F"], rel=1e-12)
    Ug = np.fromfile(fout, np.complex128).reshape(U.shape)
    assert np.max(np.abs(Ug - ref["U"])) < 1e-11
