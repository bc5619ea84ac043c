"""The seeded input generators shared by the oracle and the CUDA path: shapes,
dtypes, ranges and structure of what they hand over (they hold none of the
method's arithmetic). CPU only."""

import numpy as np

from paper_astro_ph_0703100_gb300 import synth


def test_index_lists_structure():
    n, gs, ls = 5000, 256, 700
    pos_i, i_off, src, j_index, jb, jc = synth.interaction_lists_indexed(n, gs, ls, seed=3)
    n_nodes = n // 4
    n_groups = -(-n // gs)
    assert pos_i.shape == (n, 4) and pos_i.dtype == np.float32
    assert src.shape == (n + n_nodes, 4) and src.dtype == np.float32
    assert np.array_equal(src[:n], pos_i)                      # the particles come first, as the i-set
    assert np.all(np.diff(pos_i[:, 0]) >= 0)                   # ordered by x
    assert i_off.dtype == np.int64 and i_off[0] == 0 and i_off[-1] == n and len(i_off) == n_groups + 1
    assert np.all(np.diff(i_off) > 0) and np.all(np.diff(i_off) <= gs)
    assert j_index.dtype == np.int32 and j_index.shape == (n_groups * ls,)
    assert np.array_equal(jb, np.arange(n_groups) * ls) and np.all(jc == ls)
    assert j_index.min() >= 0 and j_index.max() < src.shape[0]
    n_pseudo = ls // 2
    for g in range(n_groups):
        e = j_index[jb[g]:jb[g] + jc[g]]
        parts, nodes = e[:ls - n_pseudo], e[ls - n_pseudo:]
        assert np.all(parts < n) and len(np.unique(parts)) == parts.size
        assert np.all(nodes >= n) and len(np.unique(nodes)) == nodes.size
    assert np.all(src[n:, 3] > 0) and np.all(src[n:, 3] >= src[:n, 3].max())  # nodes carry 1-64x a particle mass


def test_index_lists_are_seeded():
    a = synth.interaction_lists_indexed(3000, 256, 500, seed=9)
    b = synth.interaction_lists_indexed(3000, 256, 500, seed=9)
    c = synth.interaction_lists_indexed(3000, 256, 500, seed=10)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert not np.array_equal(a[3], c[3])


def test_index_lists_with_few_nodes():
    """Fewer nodes than half a list: every node once, the rest particles."""
    pos_i, i_off, src, j_index, jb, jc = synth.interaction_lists_indexed(2000, 128, 400, seed=4, n_nodes=50)
    assert src.shape[0] == 2050
    for g in range(len(jc)):
        e = j_index[jb[g]:jb[g] + jc[g]]
        assert np.sum(e >= 2000) == 50 and len(np.unique(e)) == e.size


def test_contiguous_lists_and_sampled_rows():
    pos_i, i_off, lists, jb, jc = synth.interaction_lists(3000, 256, 600, seed=5)
    assert lists.shape == (len(jc) * 600, 4) and lists.dtype == np.float32
    assert np.array_equal(jb, np.arange(len(jc)) * 600)
    rows = synth.sample_rows(10000, 512, seed=1)
    assert rows.size == 512 and np.all(np.diff(rows) > 0) and rows.min() >= 0 and rows.max() < 10000
