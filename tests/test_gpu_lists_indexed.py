"""Parity of the gathering interaction-list form: lists given as index
arrays into one source array of particles and tree nodes (the form a tree
walk produces, Section 4.4), with the kernel gathering each j-tile's records
itself. Checked group by group against the FP64 oracle on the gathered
records, and bit for bit against the contiguous list plan of the same launch
shape run on the same records laid out in entry order."""

import numpy as np
import pytest

import oracle
from gpu_common import dev_tensor, e_max, lib, rel_pot_err, torch_cuda
from paper_astro_ph_0703100_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5

TUNES = [None,
         {"i_per_thread": 1, "threads": 64, "j_tile": 64, "stages": 2},
         {"i_per_thread": 2, "threads": 128, "j_tile": 256, "stages": 4, "chunk_units": 3},
         {"i_per_thread": 4, "threads": 128, "j_tile": 128, "stages": 3, "j_lanes": 2},
         {"i_per_thread": 8, "threads": 256, "j_tile": 512, "stages": 4, "j_lanes": 8},
         {"i_per_thread": 8, "threads": 128, "j_tile": 1024, "stages": 1}]


def ragged_indexed(with_guard):
    """Groups of uneven size; lists with repeated entries, lists sharing and
    overlapping entries, an empty list, a group with no i-particles whose
    list holds entries outside the source array (never reached), lists of
    1 to 3100 entries (ragged last j-tiles); with_guard: one group at
    eps2 = 0 (the guarded kernel)."""
    rng = np.random.default_rng(23)
    pos_i = synth.plummer(3000, 31)
    src = np.concatenate([pos_i, synth.plummer(1500, 32)])
    src[3000:, 3] *= 8.0  # heavier "nodes"
    sizes = [1, 0, 37, 300, 128, 999, 5, 1530]
    i_off = np.zeros(len(sizes) + 1, dtype=np.int64)
    i_off[1:] = np.cumsum(sizes)
    lens = [700, 50, 0, 3100, 1, 2000, 333, 1200]
    parts, jb, pos = [], [], 0
    for g, ln in enumerate(lens):
        e = rng.integers(0, src.shape[0], ln).astype(np.int32)
        if g == 3:
            e[::7] = e[0]  # repeats of one record
        if g == 1:
            e[:] = src.shape[0] + 5  # outside the source array: the group has no i-particles
        parts.append(e)
        jb.append(pos)
        pos += ln
    j_index = np.concatenate(parts)
    jb = np.array(jb, dtype=np.int64)
    jc = np.array(lens, dtype=np.int64)
    jb[6], jc[6] = jb[5] + 100, 900  # overlaps group 5's list
    jb[7] = jb[3]  # shares group 3's list start
    eps2 = rng.uniform(1e-4, 1e-2, len(sizes)).astype(np.float32)
    if with_guard:
        eps2[5] = 0.0
    return pos_i, i_off, src, j_index, jb, jc, eps2


@pytest.mark.parametrize("tune", TUNES)
def test_indexed_lists_against_oracle_and_contiguous_plan(tune):
    cn = lib()
    torch = torch_cuda()
    pos_i, i_off, src, j_index, jb, jc, eps2 = ragged_indexed(with_guard=False)
    plan = cn.ListPlan(i_off, jb, jc, eps2, tune=tune, potential=True, j_index=j_index, n_src=src.shape[0])
    acc, pot = plan.run(dev_tensor(pos_i), dev_tensor(src))
    torch.cuda.synchronize()
    assert cn.cn_get_device_status() == 0
    # the contiguous plan on the gathered records, entry order kept
    pool = src[np.clip(j_index, 0, src.shape[0] - 1)]
    ref_plan = cn.ListPlan(i_off, jb, jc, eps2, tune=tune, potential=True)
    acc_c, pot_c = ref_plan.run(dev_tensor(pos_i), dev_tensor(pool))
    torch.cuda.synchronize()
    assert torch.equal(acc, acc_c) and torch.equal(pot, pot_c)
    a, p = acc.cpu().numpy(), pot.cpu().numpy()
    assert plan.pairs == float(sum((i_off[g + 1] - i_off[g]) * jc[g] for g in range(len(jc))))
    for g in range(len(jc)):
        lo, hi = i_off[g], i_off[g + 1]
        if hi == lo:
            continue
        if jc[g] == 0:
            assert np.all(a[lo:hi] == 0) and np.all(p[lo:hi] == 0)
            continue
        recs = src[j_index[jb[g]:jb[g] + jc[g]]]
        ref_a, ref_p = oracle.force(pos_i[lo:hi], recs, eps2[g])
        assert e_max(a[lo:hi], ref_a) <= TOL_F32, g
        assert rel_pot_err(p[lo:hi], ref_p) <= TOL_F32, g
    plan.close()
    ref_plan.close()


def test_indexed_lists_guarded_group_and_no_potential():
    """A group at eps2 = 0 moves the plan onto the guarded kernel (a pair at
    zero separation contributes nothing); the force-only form."""
    cn = lib()
    torch = torch_cuda()
    pos_i, i_off, src, j_index, jb, jc, eps2 = ragged_indexed(with_guard=True)
    plan = cn.ListPlan(i_off, jb, jc, eps2, j_index=j_index, n_src=src.shape[0])
    acc, pot = plan.run(dev_tensor(pos_i), dev_tensor(src))
    torch.cuda.synchronize()
    assert cn.cn_get_device_status() == 0 and pot is None
    a = acc.cpu().numpy()
    for g in range(len(jc)):
        lo, hi = i_off[g], i_off[g + 1]
        if hi == lo or jc[g] == 0:
            continue
        ref_a, _ = oracle.force(pos_i[lo:hi], src[j_index[jb[g]:jb[g] + jc[g]]], eps2[g], potential=False)
        assert e_max(a[lo:hi], ref_a) <= TOL_F32, g
    plan.close()


def test_tree_walk_lists_graph_replay_and_workspace():
    """The benchmark's structure at a smaller size: particles plus tree nodes
    in one source array, groups of 256 with 2048-entry lists; direct run,
    caller workspace and graph replay agree bit for bit."""
    cn = lib()
    torch = torch_cuda()
    pos_i, i_off, src, j_index, jb, jc = synth.interaction_lists_indexed(20000, 256, 2048, seed=7)
    eps2 = float(np.float32(0.01) ** 2)
    plan = cn.ListPlan(i_off, jb, jc, eps2, j_index=j_index)
    assert plan.n_j == src.shape[0]
    ti, ts = dev_tensor(pos_i), dev_tensor(src)
    direct, _ = plan.run(ti, ts)
    ws = plan.new_workspace()
    out_ws, _ = plan.run(ti, ts, workspace=ws)
    s = torch.cuda.Stream()
    out = torch.empty_like(direct)
    with torch.cuda.stream(s):
        plan.capture(ti, ts, out, stream=s)
        out.fill_(-1)
        plan.launch(s)
    s.synchronize()
    torch.cuda.synchronize()
    assert cn.cn_get_device_status() == 0
    assert torch.equal(direct, out) and torch.equal(direct, out_ws)
    a = direct.cpu().numpy()
    for g in range(0, len(jc), 9):
        lo, hi = i_off[g], i_off[g + 1]
        ref, _ = oracle.force(pos_i[lo:hi], src[j_index[jb[g]:jb[g] + jc[g]]], eps2, potential=False)
        assert e_max(a[lo:hi], ref) <= TOL_F32, g
    # a source array shorter than the plan's n_src is refused before launch
    with pytest.raises(ValueError):
        plan.run(ti, ts[:-1])
    plan.close()


# the default shape of gathering plans on these lists (K = 4, lane groups of 4)
SHAPE_BENCH = {"i_per_thread": 4, "threads": 256, "j_tile": 512, "stages": 4, "j_lanes": 4}


def test_full_size_tree_lists_sampled_groups():
    """The benchmark's launch: 131072 particles in groups of 256, each
    against 4096 entries (half particles, half nodes) of a 163840-record
    source array, default plan; sampled groups against the oracle, and the
    whole output bit for bit against the contiguous plan of the same launch
    shape on the gathered records."""
    cn = lib()
    torch = torch_cuda()
    pos_i, i_off, src, j_index, jb, jc = synth.interaction_lists_indexed(131072, 256, 4096, seed=131072)
    eps2 = float(np.float32(0.01) ** 2)
    ti, ts = dev_tensor(pos_i), dev_tensor(src)
    plan = cn.ListPlan(i_off, jb, jc, eps2, j_index=j_index)
    acc, _ = plan.run(ti, ts)
    pinned = cn.ListPlan(i_off, jb, jc, eps2, tune=SHAPE_BENCH, j_index=j_index)
    acc_p, _ = pinned.run(ti, ts)
    ref_plan = cn.ListPlan(i_off, jb, jc, eps2, tune=SHAPE_BENCH)
    acc_c, _ = ref_plan.run(ti, dev_tensor(src[j_index]))
    torch.cuda.synchronize()
    assert cn.cn_get_device_status() == 0
    assert torch.equal(acc_p, acc_c)
    assert torch.equal(acc, acc_p)  # the default is that shape
    a = acc.cpu().numpy()
    for g in (0, 1, 255, 256, 511):
        lo, hi = i_off[g], i_off[g + 1]
        ref, _ = oracle.force(pos_i[lo:hi], src[j_index[jb[g]:jb[g] + jc[g]]], eps2, potential=False)
        assert e_max(a[lo:hi], ref) <= TOL_F32, g
    for p in (plan, pinned, ref_plan):
        p.close()


def test_indexed_plan_refusals_on_the_device():
    cn = lib()
    pos_i, i_off, src, j_index, jb, jc, eps2 = ragged_indexed(with_guard=False)
    bad = j_index.copy()
    bad[jb[3] + 5] = src.shape[0]  # reached by a group with i-particles
    with pytest.raises(RuntimeError):
        cn.ListPlan(i_off, jb, jc, eps2, j_index=bad, n_src=src.shape[0])
    with pytest.raises(ValueError):
        cn.ListPlan(i_off, jb, jc, eps2, j_index=j_index.astype(np.int64) + (1 << 40))
