"""Parity of the interaction-list form (groups of i-particles, each against
its own list of j records: the modified tree algorithm's use of the engine,
Section 4.4) with the FP64 oracle, group by group."""

import numpy as np
import pytest

import oracle
from gpu_common import dev_tensor, e_max, lib, rel_pot_err, torch_cuda
from paper_astro_ph_0703100_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5


def ragged_lists():
    """Groups of uneven size with overlapping, shared and empty lists."""
    rng = np.random.default_rng(17)
    pos_i = synth.plummer(3000, 9)
    sizes = [1, 0, 37, 300, 128, 999, 5, 1530]
    i_off = np.zeros(len(sizes) + 1, dtype=np.int64)
    i_off[1:] = np.cumsum(sizes)
    pool = np.concatenate([synth.plummer(4000, 10), pos_i])  # the list pool also holds the i-particles
    jb = np.array([0, 100, 50, 4000, 10, 2000, 0, 3000], dtype=np.int64)
    jc = np.array([7000, 300, 0, 3000, 1, 2500, 7000, 4000], dtype=np.int64)  # group 2 has an empty list
    eps2 = rng.uniform(1e-4, 1e-2, len(sizes)).astype(np.float32)
    eps2[0] = 0.0
    return pos_i, i_off, pool, jb, jc, eps2


@pytest.mark.parametrize("tune", [None, {"i_per_thread": 1, "threads": 64, "j_tile": 64, "stages": 2},
                                  {"i_per_thread": 4, "threads": 128, "j_tile": 256, "stages": 4, "chunk_units": 3},
                                  {"i_per_thread": 8, "threads": 128, "j_tile": 512, "stages": 1}])
def test_lists_group_by_group(tune):
    cn = lib()
    torch = torch_cuda()
    pos_i, i_off, pool, jb, jc, eps2 = ragged_lists()
    plan = cn.ListPlan(i_off, jb, jc, eps2, tune=tune, potential=True)
    acc, pot = plan.run(dev_tensor(pos_i), dev_tensor(pool))
    torch.cuda.synchronize()
    assert cn.cn_get_device_status() == 0
    acc, pot = acc.cpu().numpy(), pot.cpu().numpy()
    assert plan.pairs == float(sum((i_off[g + 1] - i_off[g]) * jc[g] for g in range(len(jc))))
    for g in range(len(jc)):
        lo, hi = i_off[g], i_off[g + 1]
        if hi == lo:
            continue
        if jc[g] == 0:
            assert np.all(acc[lo:hi] == 0) and np.all(pot[lo:hi] == 0)
            continue
        ref_a, ref_p = oracle.force(pos_i[lo:hi], pool[jb[g]:jb[g] + jc[g]], eps2[g])
        assert e_max(acc[lo:hi], ref_a) <= TOL_F32, g
        assert rel_pot_err(pot[lo:hi], ref_p) <= TOL_F32, g
    plan.close()


def test_tree_like_lists_graph_replay_and_plan_kinds():
    cn = lib()
    torch = torch_cuda()
    pos_i, i_off, lists, jb, jc = synth.interaction_lists(20000, 256, 2048, seed=5)
    eps2 = float(np.float32(0.01) ** 2)
    plan = cn.ListPlan(i_off, jb, jc, eps2)
    ti, tj = dev_tensor(pos_i), dev_tensor(lists)
    direct, _ = plan.run(ti, tj)
    s = torch.cuda.Stream()
    out = torch.empty_like(direct)
    with torch.cuda.stream(s):
        plan.capture(ti, tj, out, stream=s)
        out.fill_(-1)
        plan.launch(s)
    s.synchronize()
    torch.cuda.synchronize()
    assert torch.equal(direct, out)
    a = direct.cpu().numpy()
    for g in range(0, len(jc), 9):
        lo, hi = i_off[g], i_off[g + 1]
        ref, _ = oracle.force(pos_i[lo:hi], lists[jb[g]:jb[g] + jc[g]], eps2, potential=False)
        assert e_max(a[lo:hi], ref) <= TOL_F32, g
    # the C ABI keeps the two plan kinds apart
    import ctypes
    L = cn.load()
    cl = cn.BatchPlan(np.array([0, 10]), np.array([0.01], dtype=np.float32))
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    assert L.cn_force_batched(plan._h, p(ti), p(out), None, None, 0, None) == 1
    assert L.cn_force_lists(cl._h, p(ti), p(tj), p(out), None, None, 0, None) == 1
    cl.close()
    plan.close()
