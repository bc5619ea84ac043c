"""cn_force_noalloc: the FP32 force for callers that may not allocate device
memory (their own memory manager owns every device allocation, or they
cannot afford the synchronisation an allocation may bring). It takes its
scratch from a fixed array in the library's device image.

Checked here through the C ABI against cn_force (the existing entry point)
and against the FP64 oracle, on two calls in a row, at the FP32 tolerance
the other parity tests use; with the library's allocation step made to fail
(CN_FAULT_INJECT=alloc), so that a pass shows no allocation path was taken;
and in a fresh process, where free device memory is read around the first
no-allocation call. This file is collected last on purpose.
"""

import ctypes
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import oracle
from conftest import ROOT
from gpu_common import dev_tensor, e_max, lib, rel_pot_err, torch_cuda
from paper_astro_ph_0703100_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class _Inject:
    """Sets CN_FAULT_INJECT for the duration of a block (host-side only)."""

    def __init__(self, what):
        self.what = what

    def __enter__(self):
        self.old = os.environ.get("CN_FAULT_INJECT")
        os.environ["CN_FAULT_INJECT"] = self.what

    def __exit__(self, *exc):
        if self.old is None:
            os.environ.pop("CN_FAULT_INJECT", None)
        else:
            os.environ["CN_FAULT_INJECT"] = self.old


def test_noalloc_matches_cn_force_and_oracle_on_two_calls_in_a_row():
    cn = lib()
    torch = torch_cuda()
    L = cn.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [
        # (i set, j set, eps2, with potential)
        (synth.plummer(20000, 1), None, 1e-3, True),
        (synth.plummer(7001, 2), synth.plummer(5003, 3), 0.01, False),
    ]
    for idx, (pi_np, pj_np, eps2, with_pot) in enumerate(cases):
        pj_np = pi_np if pj_np is None else pj_np
        pi = dev_tensor(pi_np)
        pj = dev_tensor(pj_np)
        ref_acc, ref_pot = cn.cn_force(pi, pj, eps2, potential=with_pot)  # existing entry point
        acc = torch.full((pi.shape[0], 3), float("nan"), device="cuda")
        pot = torch.full((pi.shape[0],), float("nan"), device="cuda") if with_pot else None
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        with _Inject("alloc"):  # any library allocation would now fail the call
            st = L.cn_force_noalloc(pi.shape[0], _p(pi), pj.shape[0], _p(pj), eps2, _p(acc), _p(pot), stream)
        assert st == 0, L.cn_last_error_message()
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free_before  # nothing was allocated
        assert cn.cn_get_device_status() == 0
        a = acc.cpu().numpy()
        assert e_max(a, ref_acc.cpu().numpy().astype(np.float64)) <= TOL_F32
        rows = synth.sample_rows(pi_np.shape[0], 1024, seed=31 + idx)
        ref_o, ref_op = oracle.force(pi_np, pj_np, eps2, rows=rows, potential=with_pot)
        assert e_max(a[rows], ref_o) <= TOL_F32
        if with_pot:
            assert rel_pot_err(pot.cpu().numpy(), ref_pot.cpu().numpy()) <= TOL_F32
            assert rel_pot_err(pot.cpu().numpy()[rows], ref_op) <= TOL_F32


def test_noalloc_rejects_problems_beyond_the_static_scratch():
    """2^33 i-particles need more tile counters than the 32 MiB scratch
    holds: rejected on the host. The pointers are real (small) device
    buffers and launches are made to fail on the host, so even a broken
    size check could not start a kernel on them."""
    cn = lib()
    torch = torch_cuda()
    L = cn.load()
    pi = torch.zeros((1024, 4), device="cuda")
    pj = torch.zeros((1024, 4), device="cuda")
    acc = torch.zeros((1024, 3), device="cuda")
    with _Inject("launch"):
        st = L.cn_force_noalloc(1 << 33, _p(pi), 1024, _p(pj), 0.01, _p(acc), None, None)
    assert st == 6  # CN_ERR_WORKSPACE
    assert b"static scratch" in L.cn_last_error_message()


def test_noalloc_python_binding():
    """The binding of the same name: outputs given or allocated by PyTorch."""
    cn = lib()
    torch = torch_cuda()
    q = synth.plummer(3000, 4)
    pi = dev_tensor(q)
    ref, ref_pot = cn.cn_force(pi, pi, 1e-3, potential=True)
    acc = torch.empty((3000, 3), device="cuda")
    a1, _ = cn.cn_force_noalloc(pi, pi, 1e-3, acc_out=acc)
    a2, p2 = cn.cn_force_noalloc(pi, pi, 1e-3, potential=True)
    torch.cuda.synchronize()
    assert a1.data_ptr() == acc.data_ptr()
    assert e_max(a1.cpu().numpy(), ref.cpu().numpy().astype(np.float64)) <= TOL_F32
    assert e_max(a2.cpu().numpy(), ref.cpu().numpy().astype(np.float64)) <= TOL_F32
    assert rel_pot_err(p2.cpu().numpy(), ref_pot.cpu().numpy()) <= TOL_F32
    ref_o, _ = oracle.force(q, q, 1e-3, potential=False)
    assert e_max(a1.cpu().numpy(), ref_o) <= TOL_F32


FRESH = textwrap.dedent(r"""
    import ctypes, sys
    import numpy as np, torch
    sys.path.insert(0, sys.argv[1])
    import paper_astro_ph_0703100_gb300 as cn
    from paper_astro_ph_0703100_gb300 import synth
    L = cn.load()
    p = torch.from_numpy(synth.plummer(9000, 5)).cuda()
    ref, _ = cn.cn_force(p, p, 1e-3)   # sets the device up and loads this kernel
    acc = torch.empty((9000, 3), device="cuda")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    st = L.cn_force_noalloc(9000, ptr(p), 9000, ptr(p), 1e-3, ptr(acc), None, None)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    err = float(np.max(np.abs(acc.cpu().numpy() - ref.cpu().numpy()) / np.linalg.norm(ref.cpu().numpy(), axis=1)[:, None]))
    print(st, free0 - free1, err)
""")


def test_noalloc_first_call_in_a_fresh_process_allocates_nothing():
    """In a new process: after one cn_force call (device set-up and kernel
    load), the process's first cn_force_noalloc call leaves free device
    memory unchanged."""
    torch_cuda()
    out = subprocess.run([sys.executable, "-c", FRESH, ROOT], check=True, capture_output=True, text=True,
                         timeout=300).stdout.split()
    st, allocated, err = int(out[0]), int(out[1]), float(out[2])
    assert st == 0
    assert allocated == 0
    assert err <= TOL_F32
