"""Parity of the batched ensemble launch with the FP64 oracle, per cluster."""

import numpy as np
import pytest

import oracle
from gpu_common import dev_tensor, e_max, lib, rel_pot_err, torch_cuda
from paper_astro_ph_0703100_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5


def small_ensemble():
    sizes = [1, 31, 256, 300, 1000, 0, 513, 2048, 7]
    offs = np.zeros(len(sizes) + 1, dtype=np.int64)
    offs[1:] = np.cumsum(sizes)
    rec = np.concatenate([synth.plummer(n, 40 + c) for c, n in enumerate(sizes)])
    eps2 = np.array([np.float32(synth.plummer_eps(max(n, 1))) ** 2 for n in sizes], dtype=np.float32)
    eps2[0] = 0.0  # a single particle with zero softening: its only pair is the s = 0 self pair
    return rec, offs, eps2


@pytest.mark.parametrize("tune", [
    None,
    {"i_per_thread": 1, "threads": 64, "j_tile": 64, "stages": 2},
    {"i_per_thread": 4, "threads": 128, "j_tile": 256, "stages": 4, "chunk_units": 2},
    {"i_per_thread": 8, "threads": 256, "j_tile": 128, "stages": 5, "chunk_units": 0},
    {"i_per_thread": 2, "threads": 128, "j_tile": 32, "stages": 3, "chunk_units": 1},
])
def test_small_ensemble_all_particles(tune):
    cn = lib()
    torch = torch_cuda()
    rec, offs, eps2 = small_ensemble()
    plan = cn.BatchPlan(offs, eps2, tune=tune, potential=True)
    t = dev_tensor(rec)
    acc, pot = plan.run(t)
    torch.cuda.synchronize()
    assert cn.cn_get_device_status() == 0
    acc, pot = acc.cpu().numpy(), pot.cpu().numpy()
    for c in range(len(offs) - 1):
        lo, hi = offs[c], offs[c + 1]
        if hi == lo:
            continue
        ref_a, ref_p = oracle.force(rec[lo:hi], rec[lo:hi], eps2[c])
        if hi - lo == 1:
            assert np.all(acc[lo:hi] == 0) and np.all(pot[lo:hi] == 0)
            continue
        assert e_max(acc[lo:hi], ref_a) <= TOL_F32, c
        assert rel_pot_err(pot[lo:hi], ref_p) <= TOL_F32, c
    plan.close()


def test_ensemble_c4_sampled_graph_replay_and_per_cluster_launches():
    cn = lib()
    torch = torch_cuda()
    rec, offs, eps2 = synth.ensemble(512, 512)
    t = dev_tensor(rec)
    plan = cn.BatchPlan(offs, eps2)
    acc_direct, _ = plan.run(t)
    stream = torch.cuda.Stream()
    acc_graph = torch.empty_like(acc_direct)
    with torch.cuda.stream(stream):
        ws = plan.new_workspace()
        plan.capture(t, acc_graph, workspace=ws, stream=stream)
        acc_graph.fill_(-1.0)
        plan.launch(stream)
        plan.launch(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    assert torch.equal(acc_direct, acc_graph)
    # per-cluster separate launches agree within tolerance
    sep = torch.empty_like(acc_direct)
    for c in range(512):
        lo, hi = int(offs[c]), int(offs[c + 1])
        cn.cn_force(t[lo:hi], t[lo:hi], float(eps2[c]), acc_out=sep[lo:hi])
    torch.cuda.synchronize()
    a = acc_direct.cpu().numpy()
    s = sep.cpu().numpy()
    assert e_max(a, s.astype(np.float64)) <= 2 * TOL_F32
    # oracle on 64 sampled particles per cluster
    rng = np.random.default_rng(512)
    for c in range(0, 512, 8):
        lo, hi = int(offs[c]), int(offs[c + 1])
        rows = np.sort(rng.choice(hi - lo, size=min(64, hi - lo), replace=False))
        ref, _ = oracle.force(rec[lo:hi], rec[lo:hi], eps2[c], rows=rows, potential=False)
        assert e_max(a[lo:hi][rows], ref) <= TOL_F32, c
    plan.close()


def test_batched_deterministic_and_autotune():
    cn = lib()
    torch = torch_cuda()
    rec, offs, eps2 = small_ensemble()
    t = dev_tensor(rec)
    best = cn.cn_autotune_batched(offs, eps2, t, reps=1)
    assert best["i_per_thread"] in (2, 4, 8)
    plan = cn.BatchPlan(offs, eps2)  # picks up the tuned shape
    a1, _ = plan.run(t)
    a2, _ = plan.run(t)
    torch.cuda.synchronize()
    assert torch.equal(a1, a2)
    plan.close()


@pytest.mark.parametrize("kind", ["small_ragged", "equal"])
def test_default_plan_shapes_small_and_equal_clusters(kind):
    """The plan's default shape for clusters of a few hundred particles (128-
    record j-tiles, i and j padding counted) and for equal clusters (static
    schedule): every cluster against the oracle."""
    cn = lib()
    torch = torch_cuda()
    if kind == "small_ragged":
        rec, offs, eps2 = synth.ensemble(600, 77, n_lo=64, n_hi=512)
    else:
        rec, offs, eps2 = synth.ensemble(200, 78, n_lo=1024, n_hi=1024)
    plan = cn.BatchPlan(offs, eps2)
    acc, _ = plan.run(dev_tensor(rec))
    torch.cuda.synchronize()
    assert cn.cn_get_device_status() == 0
    acc = acc.cpu().numpy()
    for c in range(0, len(offs) - 1, 7):
        lo, hi = offs[c], offs[c + 1]
        ref, _ = oracle.force(rec[lo:hi], rec[lo:hi], eps2[c], potential=False)
        assert e_max(acc[lo:hi], ref) <= TOL_F32, c
    plan.close()
