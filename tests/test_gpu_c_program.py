"""The C ABI from plain C: C99 programs linked against libcunbody.so, with no
Python or PyTorch in the process. One calls the Section 3.1 routine
(cn_force_host_f64: FP64 host arrays xj, mj, xi, eps2, a) and
cn_force_host; the other builds a gathering interaction-list plan and runs
it on device buffers it allocated with the CUDA runtime. Their printed
accelerations are compared with the FP64 oracle."""

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


LIST_PROGRAM = r"""
#include <stdio.h>
#include <stdlib.h>
#include <stdint.h>
#include <cuda_runtime.h>
#include "cunbody.h"

/* groups of particles against index lists into one source array, from C:
   argv[1] holds n_i n_src n_groups n_entries eps2, the i records, the
   source records, i_offsets, j_begin, j_count and the entries */
int main(int argc, char **argv) {
    FILE *f = fopen(argv[1], "r");
    long long ni, ns, ng, ne;
    double eps2;
    if (!f || fscanf(f, "%lld %lld %lld %lld %lf", &ni, &ns, &ng, &ne, &eps2) != 5) return 2;
    float *pi = malloc(sizeof(float) * 4 * ni), *ps = malloc(sizeof(float) * 4 * ns);
    float *acc = malloc(sizeof(float) * 3 * ni), *e2 = malloc(sizeof(float) * ng);
    int64_t *ioff = malloc(sizeof(int64_t) * (ng + 1)), *jb = malloc(sizeof(int64_t) * ng);
    int64_t *jc = malloc(sizeof(int64_t) * ng);
    int32_t *idx = malloc(sizeof(int32_t) * ne);
    for (long long k = 0; k < 4 * ni; ++k) if (fscanf(f, "%f", &pi[k]) != 1) return 3;
    for (long long k = 0; k < 4 * ns; ++k) if (fscanf(f, "%f", &ps[k]) != 1) return 3;
    for (long long g = 0; g <= ng; ++g) { long long v; if (fscanf(f, "%lld", &v) != 1) return 3; ioff[g] = v; }
    for (long long g = 0; g < ng; ++g) { long long v; if (fscanf(f, "%lld", &v) != 1) return 3; jb[g] = v; }
    for (long long g = 0; g < ng; ++g) { long long v; if (fscanf(f, "%lld", &v) != 1) return 3; jc[g] = v; }
    for (long long e = 0; e < ne; ++e) { int v; if (fscanf(f, "%d", &v) != 1) return 3; idx[e] = v; }
    fclose(f);
    for (long long g = 0; g < ng; ++g) e2[g] = (float)eps2;
    cn_batch_plan *plan = NULL;
    cn_status st = cn_list_plan_create_indexed((int32_t)ng, ioff, jb, jc, e2, idx, ne, ns, NULL, 0, &plan);
    if (st != CN_OK) { fprintf(stderr, "%s: %s\n", cn_status_string(st), cn_last_error_message()); return 4; }
    /* an entry outside the source array is refused on the host */
    int32_t keep = idx[jb[0]];
    idx[jb[0]] = (int32_t)ns;
    cn_batch_plan *bad = NULL;
    if (cn_list_plan_create_indexed((int32_t)ng, ioff, jb, jc, e2, idx, ne, ns, NULL, 0, &bad) != CN_ERR_INVALID_ARG
        || bad != NULL) return 5;
    idx[jb[0]] = keep;
    float *d_pi, *d_ps, *d_acc;
    if (cudaMalloc((void **)&d_pi, sizeof(float) * 4 * ni) != cudaSuccess ||
        cudaMalloc((void **)&d_ps, sizeof(float) * 4 * ns) != cudaSuccess ||
        cudaMalloc((void **)&d_acc, sizeof(float) * 3 * ni) != cudaSuccess) return 6;
    cudaMemcpy(d_pi, pi, sizeof(float) * 4 * ni, cudaMemcpyHostToDevice);
    cudaMemcpy(d_ps, ps, sizeof(float) * 4 * ns, cudaMemcpyHostToDevice);
    st = cn_force_lists(plan, d_pi, d_ps, d_acc, NULL, NULL, 0, NULL);
    if (st != CN_OK) { fprintf(stderr, "%s: %s\n", cn_status_string(st), cn_last_error_message()); return 7; }
    if (cudaMemcpy(acc, d_acc, sizeof(float) * 3 * ni, cudaMemcpyDeviceToHost) != cudaSuccess) return 8;
    if (cn_get_device_status(NULL) != CN_OK) return 9;
    cn_batch_plan_destroy(plan);
    cudaFree(d_pi);
    cudaFree(d_ps);
    cudaFree(d_acc);
    for (long long i = 0; i < ni; ++i) printf("%.9g %.9g %.9g\n", acc[3 * i], acc[3 * i + 1], acc[3 * i + 2]);
    return 0;
}
"""


def test_c_program_runs_index_lists(tmp_path):
    """A C99 program builds a gathering list plan, runs it on device buffers
    it allocated itself, and has an out-of-range entry refused; its
    accelerations are compared with the FP64 oracle group by group."""
    torch_cuda()
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    lib_dir = os.path.join(ROOT, "paper_astro_ph_0703100_gb300")
    src = tmp_path / "lists.c"
    src.write_text(LIST_PROGRAM)
    exe = tmp_path / "lists"
    lib64 = os.path.join(cuda, "lib64")
    subprocess.run(["gcc", "-std=c99", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-I",
                    os.path.join(cuda, "include"), str(src), "-L", lib_dir, "-lcunbody", f"-Wl,-rpath,{lib_dir}",
                    "-L", lib64, "-lcudart", f"-Wl,-rpath,{lib64}", "-o", str(exe)], check=True)
    pos_i, i_off, srcr, j_index, jb, jc = synth.interaction_lists_indexed(1500, 128, 300, seed=12)
    eps2 = float(np.float32(0.001))
    data = tmp_path / "in.txt"
    with open(data, "w") as f:
        f.write(f"{pos_i.shape[0]} {srcr.shape[0]} {len(jc)} {j_index.size} {eps2!r}\n")
        for arr in (pos_i.ravel(), srcr.ravel()):
            f.write(" ".join(repr(float(v)) for v in arr) + "\n")
        for arr in (i_off, jb, jc, j_index):
            f.write(" ".join(str(int(v)) for v in arr) + "\n")
    res = subprocess.run([str(exe), str(data)], capture_output=True, text=True)
    assert res.returncode == 0, (res.returncode, res.stderr[-2000:])
    acc = np.array([[float(v) for v in line.split()] for line in res.stdout.splitlines()])
    assert acc.shape == (pos_i.shape[0], 3)
    for g in range(len(jc)):
        lo, hi = i_off[g], i_off[g + 1]
        ref, _ = oracle.force(pos_i[lo:hi], srcr[j_index[jb[g]:jb[g] + jc[g]]], eps2, potential=False)
        assert e_max(acc[lo:hi], ref) <= 1e-5, g
