"""cn_force_noalloc: the FP32 force for callers that may not allocate device
memory (their own memory manager owns every device allocation, or they
cannot afford the synchronisation an allocation may bring). It takes its
scratch from a fixed array in the library's device image.

Checked here through the C ABI against cn_force (the existing entry point)
on two calls in a row, at the FP32 tolerance the other parity tests use.
This file is collected last on purpose.
"""

import ctypes

import numpy as np
import pytest

from gpu_common import dev_tensor, e_max, lib, rel_pot_err, torch_cuda
from paper_astro_ph_0703100_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def test_noalloc_matches_cn_force_on_two_calls_in_a_row():
    cn = lib()
    torch = torch_cuda()
    L = cn.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [
        # (i set, j set, eps2, with potential)
        (synth.plummer(20000, 1), None, 1e-3, True),
        (synth.plummer(7001, 2), synth.plummer(5003, 3), 0.01, False),
    ]
    free_after_first = None
    for idx, (pi_np, pj_np, eps2, with_pot) in enumerate(cases):
        pi = dev_tensor(pi_np)
        pj = pi if pj_np is None else dev_tensor(pj_np)
        ref_acc, ref_pot = cn.cn_force(pi, pj, eps2, potential=with_pot)  # existing entry point
        acc = torch.full((pi.shape[0], 3), float("nan"), device="cuda")
        pot = torch.full((pi.shape[0],), float("nan"), device="cuda") if with_pot else None
        torch.cuda.synchronize()
        if idx == 1:
            free_before = torch.cuda.mem_get_info()[0]
        st = L.cn_force_noalloc(pi.shape[0], _p(pi), pj.shape[0], _p(pj), eps2, _p(acc), _p(pot), stream)
        assert st == 0, L.cn_last_error_message()
        torch.cuda.synchronize()
        if idx == 1:
            assert torch.cuda.mem_get_info()[0] == free_before  # nothing was allocated
        assert cn.cn_get_device_status() == 0
        assert e_max(acc.cpu().numpy(), ref_acc.cpu().numpy().astype(np.float64)) <= TOL_F32
        if with_pot:
            assert rel_pot_err(pot.cpu().numpy(), ref_pot.cpu().numpy()) <= TOL_F32


def test_noalloc_rejects_problems_beyond_the_static_scratch():
    cn = lib()
    L = cn.load()
    # 2^33 i-particles need more tile counters than the 32 MiB scratch holds;
    # the check happens on the host before anything touches these addresses.
    n = 1 << 33
    pi, pj, acc = 0x100000000000, 0x200000000000, 0x300000000000
    st = L.cn_force_noalloc(n, ctypes.c_void_p(pi), 1024, ctypes.c_void_p(pj), 0.01, ctypes.c_void_p(acc), None,
                            None)
    assert st == 6  # CN_ERR_WORKSPACE
    assert b"static scratch" in L.cn_last_error_message()


def test_noalloc_python_binding():
    """The binding of the same name: outputs given or allocated by PyTorch."""
    cn = lib()
    torch = torch_cuda()
    pi = dev_tensor(synth.plummer(3000, 4))
    ref, ref_pot = cn.cn_force(pi, pi, 1e-3, potential=True)
    acc = torch.empty((3000, 3), device="cuda")
    a1, _ = cn.cn_force_noalloc(pi, pi, 1e-3, acc_out=acc)
    a2, p2 = cn.cn_force_noalloc(pi, pi, 1e-3, potential=True)
    torch.cuda.synchronize()
    assert a1.data_ptr() == acc.data_ptr()
    assert e_max(a1.cpu().numpy(), ref.cpu().numpy().astype(np.float64)) <= TOL_F32
    assert e_max(a2.cpu().numpy(), ref.cpu().numpy().astype(np.float64)) <= TOL_F32
    assert rel_pot_err(p2.cpu().numpy(), ref_pot.cpu().numpy()) <= TOL_F32
