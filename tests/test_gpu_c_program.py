"""The C ABI from plain C: a C99 program linked against libcunbody.so calls
the Section 3.1 routine (cn_force_host_f64: FP64 host arrays xj, mj, xi,
eps2, a) and cn_force_host, with no Python or PyTorch in the process; its
printed accelerations are compared with the FP64 oracle."""

import os
import subprocess

import numpy as np
import pytest

import oracle
from conftest import ROOT
from gpu_common import e_max, torch_cuda
from paper_astro_ph_0703100_gb300 import synth

pytestmark = pytest.mark.gpu

PROGRAM = r"""
#include <stdio.h>
#include <stdlib.h>
#include "cunbody.h"

int main(int argc, char **argv) {
    const char *path = argv[1];
    int n;
    double eps2;
    FILE *f = fopen(path, "r");
    if (!f || fscanf(f, "%d %lf", &n, &eps2) != 2) return 2;
    double *x = malloc(sizeof(double) * 3 * n), *m = malloc(sizeof(double) * n);
    double *a = malloc(sizeof(double) * 3 * n);
    float *rec = malloc(sizeof(float) * 4 * n), *acc = malloc(sizeof(float) * 3 * n);
    for (int i = 0; i < n; ++i) {
        if (fscanf(f, "%lf %lf %lf %lf", &x[3 * i], &x[3 * i + 1], &x[3 * i + 2], &m[i]) != 4) return 3;
        for (int d = 0; d < 3; ++d) rec[4 * i + d] = (float)x[3 * i + d];
        rec[4 * i + 3] = (float)m[i];
    }
    fclose(f);
    /* the paper's routine: force(xj, mj, xi, eps2, a, ni, nj) */
    cn_status st = cn_force_host_f64(x, m, x, eps2, a, n, n);
    if (st != CN_OK) { fprintf(stderr, "%s: %s\n", cn_status_string(st), cn_last_error_message()); return 4; }
    st = cn_force_host(n, rec, n, rec, (float)eps2, acc, NULL, NULL);
    if (st != CN_OK) { fprintf(stderr, "%s: %s\n", cn_status_string(st), cn_last_error_message()); return 5; }
    printf("%s\n", cn_version());
    for (int i = 0; i < n; ++i)
        printf("%.17g %.17g %.17g %.9g %.9g %.9g\n", a[3 * i], a[3 * i + 1], a[3 * i + 2], acc[3 * i], acc[3 * i + 1],
               acc[3 * i + 2]);
    return 0;
}
"""


def test_c_program_calls_the_paper_routine(tmp_path):
    torch_cuda()  # a GPU is present
    lib_dir = os.path.join(ROOT, "paper_astro_ph_0703100_gb300")
    src = tmp_path / "force.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "force"
    subprocess.run(["gcc", "-std=c99", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    "-L", lib_dir, "-lcunbody", f"-Wl,-rpath,{lib_dir}", "-o", str(exe)], check=True)
    n = 777
    p = synth.plummer(n, 90)
    eps2 = float(np.float32(0.01))
    data = tmp_path / "in.txt"
    with open(data, "w") as f:
        f.write(f"{n} {eps2!r}\n")
        for r in p:
            f.write(" ".join(repr(float(v)) for v in r) + "\n")
    out = subprocess.run([str(exe), str(data)], check=True, capture_output=True, text=True).stdout.splitlines()
    assert out[0]  # the library version string
    vals = np.array([[float(v) for v in line.split()] for line in out[1:]])
    assert vals.shape == (n, 6)
    ref, _ = oracle.force(p, p, eps2, potential=False)
    assert e_max(vals[:, :3], ref) <= 1e-5  # FP64 interface, FP32 records and pairs inside
    assert e_max(vals[:, 3:], ref) <= 1e-5
