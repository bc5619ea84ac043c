"""Launch ordering under programmatic dependent launch.

The library launches its pair and symmetric kernels with programmatic
stream serialization: a kernel may be scheduled while the previous kernel of
the stream is still running, and waits (griddepcontrol.wait) before its
first global memory access. These tests chain library kernels whose second
call reads what the first one wrote, with no host synchronisation between
them, and require the bits of the same calls made one at a time with a
synchronisation after each; in stream order, inside a captured CUDA graph,
and against a process that launches in plain stream order (CN_PDL=0).
"""

import hashlib
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from conftest import ROOT
from gpu_common import dev_tensor, lib, torch_cuda
from paper_astro_ph_0703100_gb300 import synth

pytestmark = pytest.mark.gpu

N_I, N_J, N_2 = 1600, 3000, 500  # call 1 writes 1600 x 3 floats = 1200 float4 records read by call 2


def chain(cn, torch, p, q, buf, seed_fill, sync):
    """Call 1 writes accelerations into buf; call 2 reads buf as its j
    records (x, y, z, m); the symmetric form (its kernel and its merge
    kernel) then runs on the same records."""
    buf.fill_(seed_fill)
    acc1 = buf[: N_I * 3].view(N_I, 3)
    cn.cn_force(p[:N_I], q, 1e-3, acc_out=acc1)
    if sync:
        torch.cuda.synchronize()
    recs = buf.view(-1, 4)[: N_I * 3 // 4]
    out2, _ = cn.cn_force(p[:N_2], recs, 1e-2)
    if sync:
        torch.cuda.synchronize()
    sym, _ = cn.cn_force_symmetric(recs, 1e-2)
    if sync:
        torch.cuda.synchronize()
    return out2, sym


def test_chained_calls_match_synchronised_calls():
    cn = lib()
    torch = torch_cuda()
    buf = torch.empty(N_I * 3, dtype=torch.float32, device="cuda")
    for it in range(20):
        p = dev_tensor(synth.plummer(N_I, 100 + it))
        q = dev_tensor(synth.plummer(N_J, 200 + it))
        ref2, refs = chain(cn, torch, p, q, buf, 7.0, sync=True)
        ref2, refs = ref2.clone(), refs.clone()
        out2, sym = chain(cn, torch, p, q, buf, -3.0, sync=False)
        torch.cuda.synchronize()
        assert cn.cn_get_device_status() == 0
        assert torch.equal(out2, ref2), it
        assert torch.equal(sym, refs), it


def test_chained_adjoint_compensated_and_batched_calls():
    """The adjoint takes as its weights the accelerations a cn_force call
    has just written (its weight-packing kernel and its pair kernel both
    follow that call), the compensated form and a batch plan read records
    that call wrote; no host synchronisation in between, compared bit for
    bit with the same calls synchronised one by one."""
    cn = lib()
    torch = torch_cuda()
    n = 2000
    p = dev_tensor(synth.plummer(n, 41))
    offs = np.array([0, 700, 1200, n * 3 // 4], dtype=np.int64)
    eps2s = np.array([1e-2, 2e-2, 5e-3], dtype=np.float32)
    plan = cn.BatchPlan(offs, eps2s)

    def run(sync):
        w = torch.empty((n, 3), dtype=torch.float32, device="cuda")
        cn.cn_force(p, p, 1e-3, acc_out=w)
        if sync:
            torch.cuda.synchronize()
        gp, gm = cn.cn_force_adjoint(p, 1e-3, w)
        if sync:
            torch.cuda.synchronize()
        recs = w.view(-1, 4)  # n * 3 floats as (n * 3 / 4) records
        dd, _ = cn.cn_force_dd(recs, recs, 1e-2)
        if sync:
            torch.cuda.synchronize()
        ens, _ = plan.run(recs)
        torch.cuda.synchronize()
        return [x.clone() for x in (w, gp, gm, dd, ens)]

    ref = run(True)
    for _ in range(5):
        got = run(False)
        assert cn.cn_get_device_status() == 0
        for a, b in zip(got, ref):
            assert torch.equal(a, b)
    plan.close()


def test_chained_calls_in_a_captured_graph():
    cn = lib()
    torch = torch_cuda()
    p = dev_tensor(synth.plummer(N_I, 5))
    q = dev_tensor(synth.plummer(N_J, 6))
    buf = torch.empty(N_I * 3, dtype=torch.float32, device="cuda")
    ref2, refs = chain(cn, torch, p, q, buf, 7.0, sync=True)
    ref2, refs = ref2.clone(), refs.clone()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        chain(cn, torch, p, q, buf, 1.0, sync=False)  # grows the library workspace on this stream
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            out2, sym = chain(cn, torch, p, q, buf, -3.0, sync=False)
    for _ in range(5):
        g.replay()
    torch.cuda.synchronize()
    assert cn.cn_get_device_status() == 0
    assert torch.equal(out2, ref2)
    assert torch.equal(sym, refs)


SCRIPT = textwrap.dedent(r"""
    import hashlib, sys
    sys.path.insert(0, sys.argv[1])
    import torch
    import paper_astro_ph_0703100_gb300 as cn
    from paper_astro_ph_0703100_gb300 import synth
    n_i, n_j, n_2 = (int(x) for x in sys.argv[2:5])
    d = lambda a: torch.from_numpy(a).cuda()
    p, q = d(synth.plummer(n_i, 5)), d(synth.plummer(n_j, 6))
    buf = torch.zeros(n_i * 3, dtype=torch.float32, device="cuda")
    cn.cn_force(p, q, 1e-3, acc_out=buf.view(n_i, 3))
    recs = buf.view(-1, 4)
    out2, _ = cn.cn_force(p[:n_2], recs, 1e-2)
    sym, _ = cn.cn_force_symmetric(recs, 1e-2)
    torch.cuda.synchronize()
    h = hashlib.sha256(out2.cpu().numpy().tobytes() + sym.cpu().numpy().tobytes()).hexdigest()
    print(h, cn.cn_get_device_status())
""")


def test_plain_stream_order_gives_the_same_bits():
    torch_cuda()
    runs = {}
    for flag in ("0", "1"):
        env = dict(os.environ, CN_PDL=flag)
        res = subprocess.run([sys.executable, "-c", SCRIPT, ROOT, str(N_I), str(N_J), str(N_2)], env=env,
                             capture_output=True, text=True, timeout=300)
        assert res.returncode == 0, res.stderr[-2000:]
        h, status = res.stdout.split()[-2:]
        assert status == "0"
        runs[flag] = h
    assert runs["0"] == runs["1"]
    assert len(runs["0"]) == len(hashlib.sha256().hexdigest())
