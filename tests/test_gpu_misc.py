"""Potential energy, host-memory forms, tuning, probes, failure paths."""

import os

import numpy as np
import pytest

import oracle
from gpu_common import dev_tensor, e_max, lib, torch_cuda
from paper_astro_ph_0703100_gb300 import synth

pytestmark = pytest.mark.gpu


def test_potential_energy_fp32_and_dd():
    cn = lib()
    torch = torch_cuda()
    n = 16384
    p = synth.plummer(n, 101)
    eps2 = float(np.float32(1e-3) ** 2)
    t = dev_tensor(p)
    _, pot = cn.cn_force(t, t, eps2, potential=True)
    _, pot_d = cn.cn_force_dd(t, t, eps2, potential=True)
    w32 = cn.cn_potential_energy(t, pot)
    wdd = cn.cn_potential_energy_dd(t, pot_d)
    torch.cuda.synchronize()
    _, ref_p = oracle.force(p, p, eps2)
    ref_w = oracle.potential_energy(p, ref_p)
    assert float(w32.item()) == pytest.approx(ref_w, rel=1e-6)
    assert float(wdd.item()) == pytest.approx(ref_w, rel=1e-9)
    # same inputs, same result (fixed-order FP64 reduction)
    assert float(cn.cn_potential_energy(t, pot).item()) == float(w32.item())


def test_host_forms():
    cn = lib()
    torch = torch_cuda()
    p = synth.plummer(3000, 77)
    acc_h, pot_h = cn.cn_force_host(p, p, 1e-3, potential=True)
    t = dev_tensor(p)
    acc_d, pot_d = cn.cn_force(t, t, 1e-3, potential=True)
    torch.cuda.synchronize()
    assert np.array_equal(acc_h, acc_d.cpu().numpy()) and np.array_equal(pot_h, pot_d.cpu().numpy())
    # pinned host tensors
    pin = torch.from_numpy(p).pin_memory()
    acc_pin = torch.empty((3000, 3), dtype=torch.float32).pin_memory()
    pot_pin = torch.empty((3000,), dtype=torch.float32).pin_memory()
    cn.cn_force_host(pin, pin, 1e-3, acc_out=acc_pin, pot_out=pot_pin)  # same kernel variant as acc_h
    assert np.array_equal(acc_pin.numpy(), acc_h) and np.array_equal(pot_pin.numpy(), pot_h)
    # the paper's routine: FP64 host arrays, i set != j set
    xj = p[:, :3].astype(np.float64)
    mj = p[:, 3].astype(np.float64)
    xi = synth.plummer(100, 78)[:, :3].astype(np.float64)
    a = cn.cn_force_host_f64(xj, mj, xi, 1e-3)
    pi = np.zeros((100, 4), dtype=np.float32)
    pi[:, :3] = xi
    ref, _ = oracle.force(pi, p, 1e-3, potential=False)
    assert e_max(a, ref) <= 1e-5


def test_tune_roundtrip_and_probe():
    cn = lib()
    t = {"i_per_thread": 2, "threads": 256, "j_tile": 64, "stages": 3, "ctas_per_sm": 0, "chunk_units": 0,
         "j_lanes": 1}
    cn.cn_tune_set("f32", 5000, 7000, t)
    assert cn.cn_tune_get("f32", 5000, 7000) == t
    cn.cn_tune_set("f32", 5000, 7000, None)
    assert cn.cn_tune_get("f32", 5000, 7000) != t
    with pytest.raises(cn.CunbodyError):  # split-j lanes are offered for the FP32 form only
        cn.cn_tune_set("dd", 5000, 7000, dict(t, i_per_thread=1, j_lanes=8))
    peaks = cn.cn_probe_peaks()
    assert peaks["sms"] >= 100
    assert peaks["ffma_per_s"] > 1e12 and peaks["mufu_rsqrt_per_s"] > 1e11 and peaks["pair_mix_per_s"] > 1e11
    assert 500 < peaks["sm_mhz"] < 3000


def test_timeout_path_reports_and_recovers():
    """A wait that nothing completes gives up after the limit; the context stays usable."""
    cn = lib()
    torch = torch_cuda()
    cn.cn_set_wait_limit_ns(2_000_000)  # 2 ms
    try:
        cn.cn_debug_timeout_probe()
        assert cn.cn_get_device_status() == 4  # CN_ERR_TIMEOUT
        assert cn.cn_get_device_status() == 0  # cleared
    finally:
        cn.cn_set_wait_limit_ns(0)
    p = synth.plummer(500, 1)
    t = dev_tensor(p)
    acc, _ = cn.cn_force(t, t, 1e-2)
    torch.cuda.synchronize()
    ref, _ = oracle.force(p, p, 1e-2, potential=False)
    assert e_max(acc.cpu().numpy(), ref) <= 1e-5


def test_host_fault_injection(monkeypatch):
    cn = lib()
    torch = torch_cuda()
    t = dev_tensor(synth.plummer(100, 2))
    monkeypatch.setenv("CN_FAULT_INJECT", "launch")
    with pytest.raises(cn.CunbodyError) as ei:
        cn.cn_force(t, t, 1e-2)
    assert ei.value.code == "CN_ERR_CUDA" and "injected" in str(ei.value)
    monkeypatch.setenv("CN_FAULT_INJECT", "alloc")
    s = torch.cuda.Stream()  # a fresh stream has no library workspace yet
    with pytest.raises(cn.CunbodyError) as ei:
        cn.cn_force(t, t, 1e-2, stream=s)
    assert ei.value.code == "CN_ERR_CUDA"
    monkeypatch.setenv("CN_FAULT_INJECT", "capture")
    with pytest.raises(cn.CunbodyError) as ei:
        cn.cn_force(t, t, 1e-2, stream=torch.cuda.Stream())
    assert ei.value.code == "CN_ERR_WORKSPACE"
    monkeypatch.delenv("CN_FAULT_INJECT")
    acc, _ = cn.cn_force(t, t, 1e-2)
    torch.cuda.synchronize()
    assert torch.isfinite(acc).all()


def test_plan_functions_of_the_binding():
    """The module-level plan functions (the C names) drive the same plans."""
    cn = lib()
    torch = torch_cuda()
    rec, offs, eps2 = synth.ensemble(6, 31, n_lo=100, n_hi=900)
    t = dev_tensor(rec)
    plan = cn.cn_batch_plan_create(offs, eps2)
    n_total, pairs = cn.cn_batch_plan_info(plan)
    assert n_total == rec.shape[0] and pairs == float((np.diff(offs).astype(float) ** 2).sum())
    ws = torch.zeros(max(cn.cn_batch_plan_workspace_bytes(plan), 256), dtype=torch.uint8, device="cuda")
    acc = torch.empty((n_total, 3), device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        cn.cn_batch_plan_capture(plan, t, acc, workspace=ws, stream=s)
        cn.cn_batch_plan_launch(plan, s)
    torch.cuda.synchronize()
    ref, _ = cn.cn_force_batched(plan, t)
    torch.cuda.synchronize()
    assert torch.equal(acc, ref)
    cn.cn_batch_plan_destroy(plan)
    assert cn.cn_status_string(0) and cn.cn_status_string(1) != cn.cn_status_string(0)
    assert isinstance(cn.cn_last_error_message(), str)


def test_concurrent_host_threads_on_separate_streams():
    """Calls from several host threads, each on its own stream (own library
    workspace): results equal the single-threaded ones bit for bit."""
    import threading

    cn = lib()
    torch = torch_cuda()
    sizes = [3000, 20000, 70000, 131072]
    data = [dev_tensor(synth.plummer(n, 40 + n)) for n in sizes]
    eps2 = 1e-3
    ref = []
    for d in data:
        a, _ = cn.cn_force(d, d, eps2)
        ref.append(a)
    torch.cuda.synchronize()
    out = [None] * len(sizes)
    errors = []

    def work(idx):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                for _ in range(3):
                    a, _ = cn.cn_force(data[idx], data[idx], eps2, stream=s)
                s.synchronize()
            out[idx] = a
        except Exception as e:  # noqa: BLE001 - reported below
            errors.append(e)

    threads = [threading.Thread(target=work, args=(i,)) for i in range(len(sizes))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    torch.cuda.synchronize()
    assert cn.cn_get_device_status() == 0
    for a, r in zip(out, ref):
        assert torch.equal(a, r)


def test_tuning_file_save_and_load(tmp_path):
    """cn_tune_save writes this device's entries; after they are cleared,
    cn_tune_load restores them, and a launch uses the restored shape. A
    file naming another device is refused."""
    import json

    cn = lib()
    torch = torch_cuda()
    shape = {"i_per_thread": 4, "threads": 128, "j_tile": 512, "stages": 3, "ctas_per_sm": 0, "chunk_units": 0,
             "j_lanes": 1}
    cn.cn_tune_set("f32", 3000, 3000, shape)
    path = tmp_path / "tune.json"
    try:
        cn.cn_tune_save(str(path))
        doc = json.loads(path.read_text())
        assert doc["format"] == "cunbody-tune-1" and doc["arch"] == "sm_103"
        assert any(e["variant"] == "f32" and e["i_per_thread"] == 4 and e["threads"] == 128 for e in doc["entries"])
        cn.cn_tune_set("f32", 3000, 3000, None)
        assert cn.cn_tune_get("f32", 3000, 3000) != shape
        assert cn.cn_tune_load(str(path)) == len(doc["entries"])
        assert cn.cn_tune_get("f32", 3000, 3000) == shape
        p = dev_tensor(synth.plummer(3000, 12))
        acc, _ = cn.cn_force(p, p, 1e-3)
        torch.cuda.synchronize()
        ref, _ = oracle.force(synth.plummer(3000, 12), synth.plummer(3000, 12), 1e-3, potential=False)
        assert e_max(acc.cpu().numpy(), ref) <= 1e-5
        doc["device"] = "some other GPU"
        other = tmp_path / "other.json"
        other.write_text(json.dumps(doc))
        with pytest.raises(cn.CunbodyError) as ei:
            cn.cn_tune_load(str(other))
        assert ei.value.code == "CN_ERR_UNSUPPORTED_DEVICE"
    finally:
        cn.cn_tune_set("f32", 3000, 3000, None)


def test_binding_rejects_tensors_the_kernels_cannot_read():
    """Tensors that are not contiguous CUDA memory of the records' device are
    refused by the binding before anything reaches the library: host
    potentials for the energy, host or strided workspaces and weights."""
    cn = lib()
    torch = torch_cuda()
    p = dev_tensor(synth.plummer(300, 71))
    acc, pot = cn.cn_force(p, p, 1e-3, potential=True)
    with pytest.raises(TypeError):
        cn.cn_potential_energy(p, pot.cpu())
    with pytest.raises(TypeError):
        cn.cn_force_ws(p, p, 1e-3, torch.zeros(1 << 16, dtype=torch.uint8))
    with pytest.raises(TypeError):
        cn.cn_force_adjoint(p, 1e-3, torch.zeros((300, 3), dtype=torch.float32))
    with pytest.raises(TypeError):
        cn.cn_force_adjoint(p, 1e-3, torch.zeros((3, 300), dtype=torch.float32, device="cuda").t())
    plan = cn.BatchPlan(np.array([0, 100, 300], dtype=np.int64), np.array([1e-3, 1e-3], dtype=np.float32))
    with pytest.raises(TypeError):
        plan.run(p, workspace=torch.zeros(plan.workspace_bytes + 256, dtype=torch.uint8))
    plan.close()
    w = cn.cn_potential_energy(p, pot)  # the valid call still works
    torch.cuda.synchronize()
    assert np.isfinite(float(w.item()))


LOG_SCRIPT = r"""
import sys
sys.path.insert(0, sys.argv[1])
import numpy as np, torch
import paper_astro_ph_0703100_gb300 as cn
from paper_astro_ph_0703100_gb300 import synth
d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
p = d(synth.plummer(5000, 1))
cn.cn_force(p, p, 1e-3)
cn.cn_force_symmetric(p, 1e-3)
pos_i, i_off, src, jidx, jb, jc = synth.interaction_lists_indexed(3000, 256, 700, seed=2)
lx = cn.ListPlan(i_off, jb, jc, 1e-3, j_index=jidx, n_src=src.shape[0])
lx.run(d(pos_i), d(src))
lc = cn.ListPlan(i_off, jb, jc, 1e-3)
lc.run(d(pos_i), d(src[jidx]))
torch.cuda.synchronize()
print("status", cn.cn_get_device_status())
"""


def test_plan_logging_names_each_launch():
    """CN_LOG=1 prints one line per launch on stderr with the entry point,
    variant, sizes, launch shape, grid and units (the index-list form marked
    as such); without it the library prints nothing."""
    import subprocess
    import sys

    from conftest import ROOT

    torch_cuda()
    runs = {}
    for flag in ("1", "0"):
        env = dict(os.environ, CN_LOG=flag)
        res = subprocess.run([sys.executable, "-c", LOG_SCRIPT, ROOT], env=env, capture_output=True, text=True,
                             timeout=300)
        assert res.returncode == 0, res.stderr[-2000:]
        assert res.stdout.split()[-1] == "0"
        runs[flag] = [line for line in res.stderr.splitlines() if line.startswith("[cunbody]")]
    assert runs["0"] == []
    lines = runs["1"]
    force = [x for x in lines if x.startswith("[cunbody] cn_force: variant f32 n_i 5000 n_j 5000")]
    assert len(force) == 1 and "grid " in force[0] and "units " in force[0] and "K " in force[0]
    assert sum(x.startswith("[cunbody] cn_force_symmetric: n 5000") for x in lines) >= 1
    indexed = [x for x in lines if x.startswith("[cunbody] cn_force_lists (index lists): variant batched")]
    plain = [x for x in lines if x.startswith("[cunbody] cn_force_lists: variant batched")]
    assert len(indexed) == 1 and len(plain) == 1
    assert "n_i 3000 n_j 3750" in indexed[0] and "n_i 3000 n_j" in plain[0]
