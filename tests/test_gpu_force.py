"""Parity of cn_force / cn_force_dd (CUDA, sm_103a) with the FP64 oracle.

Tolerances (per-particle |a_gpu - a_oracle| / |a_oracle|, max over the
checked particles, Eq. 3), as the target accuracy of each form states:
  plain FP32       <= 1e-5
  compensated      <= 1e-7 (the pair term in FP32 with its roundings
                   recovered, (hi, lo) sums: measured ~1e-9, 1.6e-8 at
                   N = 2^20, so the bound keeps a margin)
Potentials: relative error <= 1e-5 (FP32) / 1e-7 (compensated).
"""

import numpy as np
import pytest

import oracle
from gpu_common import dev_tensor, e_max, lib, rel_pot_err, torch_cuda
from paper_astro_ph_0703100_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5
TOL_DD = 1e-7


def run(cn, pi, pj, eps2, potential=False, dd=False):
    torch = torch_cuda()
    ti, tj = dev_tensor(pi), dev_tensor(pj)
    fn = cn.cn_force_dd if dd else cn.cn_force
    acc, pot = fn(ti, tj, eps2, potential=potential)
    torch.cuda.synchronize()
    assert cn.cn_get_device_status() == 0
    return acc.cpu().numpy(), (pot.cpu().numpy() if pot is not None else None)


def test_c1_plummer_1024_acc_and_potential():
    cn = lib()
    p = synth.plummer(1024, 1001)
    eps2 = float(np.float32(1 / 64) ** 2)
    acc, pot = run(cn, p, p, eps2, potential=True)
    ref_a, ref_p = oracle.force(p, p, eps2)
    assert e_max(acc, ref_a) <= TOL_F32
    assert rel_pot_err(pot, ref_p) <= TOL_F32


@pytest.mark.parametrize("n", [2048])
def test_c2_small_all_i(n):
    cn = lib()
    p = synth.plummer(n, n)
    eps2 = float(np.float32(synth.plummer_eps(n)) ** 2)
    acc, _ = run(cn, p, p, eps2)
    ref, _ = oracle.force(p, p, eps2, potential=False)
    assert e_max(acc, ref) <= TOL_F32


@pytest.mark.parametrize("n", [16384, 131072])
def test_c2_large_sampled_rows_autotuned(n):
    """Full-size runs in the launch shape the benchmark uses (autotuned)."""
    cn = lib()
    torch = torch_cuda()
    p = synth.plummer(n, n)
    eps2 = float(np.float32(synth.plummer_eps(n)) ** 2)
    t = dev_tensor(p)
    cn.cn_autotune("f32", t, t, eps2, reps=2)
    acc, _ = cn.cn_force(t, t, eps2)
    torch.cuda.synchronize()
    rows = synth.sample_rows(n, 4096, seed=n + 1)
    ref, _ = oracle.force(p, p, eps2, rows=rows, potential=False)
    assert e_max(acc.cpu().numpy()[rows], ref) <= TOL_F32
    cn.cn_tune_set("f32", n, n, None)


@pytest.mark.parametrize("n_i,n_j", [(9000, 9000), (14000, 14000), (22000, 22000), (28000, 28000),
                                     (45000, 45000), (14000, 9000), (9000, 22000), (1000000, 50),
                                     (200000, 2000)])
def test_default_shapes_with_fitted_j_tiles(n_i, n_j):
    """Between the measured sizes the default j-tile is fitted to the static
    schedule, so it is often not a power of two (and the last j-tile is
    ragged): sampled rows against the oracle in those default shapes."""
    cn = lib()
    torch = torch_cuda()
    pi, pj = synth.plummer(n_i, n_i + 3), synth.plummer(n_j, n_j + 4)
    eps2 = float(np.float32(synth.plummer_eps(max(n_i, n_j))) ** 2)
    cn.cn_tune_set("f32", n_i, n_j, None)
    shape = cn.cn_tune_get("f32", n_i, n_j)
    acc, _ = cn.cn_force(dev_tensor(pi), dev_tensor(pj), eps2)
    torch.cuda.synchronize()
    assert cn.cn_get_device_status() == 0
    rows = synth.sample_rows(n_i, 1024, seed=n_i + n_j)
    ref, _ = oracle.force(pi, pj, eps2, rows=rows, potential=False)
    assert e_max(acc.cpu().numpy()[rows], ref) <= TOL_F32, shape
    assert shape["j_tile"] % 16 == 0


@pytest.mark.parametrize("n_i,n_j", [(24576, 24576), (20000, 13000), (8192, 8192)])
def test_dd_default_shapes_by_size(n_i, n_j):
    """The compensated form's default shapes: one i-particle per thread below
    N = 12000, K = 4 x 256 with a j-tile fitted to the schedule above 20000
    (432 records at 24576, 528 at 20000 on a 152-SM GB300)."""
    cn = lib()
    torch = torch_cuda()
    pi, pj = synth.plummer(n_i, n_i + 5), synth.plummer(n_j, n_j + 6)
    eps2 = float(np.float32(synth.plummer_eps(max(n_i, n_j))) ** 2)
    cn.cn_tune_set("dd", n_i, n_j, None)
    shape = cn.cn_tune_get("dd", n_i, n_j)
    acc, _ = cn.cn_force_dd(dev_tensor(pi), dev_tensor(pj), eps2)
    torch.cuda.synchronize()
    assert cn.cn_get_device_status() == 0
    rows = synth.sample_rows(n_i, 512, seed=n_i + 7)
    ref, _ = oracle.force(pi, pj, eps2, rows=rows, potential=False)
    assert e_max(acc.cpu().numpy()[rows], ref) <= TOL_DD, shape


@pytest.mark.parametrize("n_i,n_j", [(16384, 16384), (24576, 13000)])
def test_potential_default_shapes_mid_size(n_i, n_j):
    """With the potential the mid-size default takes K = 4 with lane groups
    of 4 (the K = 8 split-j kernel runs short of registers there)."""
    cn = lib()
    torch = torch_cuda()
    pi, pj = synth.plummer(n_i, n_i + 11), synth.plummer(n_j, n_j + 12)
    eps2 = float(np.float32(synth.plummer_eps(max(n_i, n_j))) ** 2)
    cn.cn_tune_set("f32_pot", n_i, n_j, None)
    shape = cn.cn_tune_get("f32_pot", n_i, n_j)
    acc, pot = cn.cn_force(dev_tensor(pi), dev_tensor(pj), eps2, potential=True)
    torch.cuda.synchronize()
    assert cn.cn_get_device_status() == 0
    rows = synth.sample_rows(n_i, 512, seed=n_i + 13)
    ref_a, ref_p = oracle.force(pi, pj, eps2, rows=rows)
    assert e_max(acc.cpu().numpy()[rows], ref_a) <= TOL_F32, shape
    assert rel_pot_err(pot.cpu().numpy()[rows], ref_p) <= TOL_F32, shape


def test_fitted_j_tiles_include_non_powers_of_two():
    """The sizes above exercise j-tiles that are not powers of two (on a
    152-SM GB300: 9000 -> 2304, 14000 -> 1280, 22000 -> 3200, 45000 -> 944)."""
    cn = lib()
    tiles = [cn.cn_tune_get("f32", n, n)["j_tile"] for n in (9000, 14000, 22000, 28000, 45000)]
    assert any(t & (t - 1) for t in tiles), tiles


def test_c2_131072_default_shape_sampled():
    """The benchmark's own launch configuration (the default shape, no
    autotuning) at N = 131072 on 4096 sampled rows, twice in a row."""
    cn = lib()
    torch = torch_cuda()
    n = 131072
    p = synth.plummer(n, n)
    eps2 = float(np.float32(synth.plummer_eps(n)) ** 2)
    t = dev_tensor(p)
    cn.cn_tune_set("f32", n, n, None)
    a1, _ = cn.cn_force(t, t, eps2)
    a2, _ = cn.cn_force(t, t, eps2)
    torch.cuda.synchronize()
    assert torch.equal(a1, a2)
    rows = synth.sample_rows(n, 4096, seed=n + 2)
    ref, _ = oracle.force(p, p, eps2, rows=rows, potential=False)
    assert e_max(a1.cpu().numpy()[rows], ref) <= TOL_F32


SHAPES = [
    (1, 1), (1, 7), (7, 1), (31, 33), (33, 31), (257, 1000), (1000, 777), (3000, 5001), (4097, 2049),
]
TUNES = [
    None,
    {"i_per_thread": 1, "threads": 64, "j_tile": 16, "stages": 2},
    {"i_per_thread": 2, "threads": 128, "j_tile": 64, "stages": 3},
    {"i_per_thread": 4, "threads": 256, "j_tile": 256, "stages": 4},
    {"i_per_thread": 8, "threads": 128, "j_tile": 512, "stages": 6},
    {"i_per_thread": 4, "threads": 64, "j_tile": 128, "stages": 4, "chunk_units": 3},
    {"i_per_thread": 2, "threads": 128, "j_tile": 32, "stages": 4, "ctas_per_sm": 1},
    # split-j shapes: lanes of a warp share one i-particle, shuffle-reduced
    {"i_per_thread": 1, "threads": 128, "j_tile": 256, "stages": 2, "j_lanes": 32},
    {"i_per_thread": 1, "threads": 64, "j_tile": 64, "stages": 3, "j_lanes": 4},
    {"i_per_thread": 1, "threads": 256, "j_tile": 128, "stages": 4, "j_lanes": 16, "chunk_units": 2},
    {"i_per_thread": 1, "threads": 128, "j_tile": 128, "stages": 1, "j_lanes": 16},
    # packed split-j: two i-particles per lane group
    {"i_per_thread": 2, "threads": 128, "j_tile": 256, "stages": 2, "j_lanes": 32},
    {"i_per_thread": 2, "threads": 256, "j_tile": 128, "stages": 4, "j_lanes": 16, "chunk_units": 2},
    {"i_per_thread": 4, "threads": 128, "j_tile": 64, "stages": 1},
]


@pytest.mark.parametrize("tune", TUNES)
@pytest.mark.parametrize("shape", SHAPES)
def test_ragged_shapes_and_launch_shapes(shape, tune):
    cn = lib()
    n_i, n_j = shape
    pj = synth.plummer(n_j, 11 + n_j)
    pi = synth.plummer(n_i, 5 + n_i)  # an i set distinct from the j set
    eps2 = 1e-3
    for variant in ("f32", "f32_pot"):
        cn.cn_tune_set(variant, n_i, n_j, tune)
    try:
        acc, pot = run(cn, pi, pj, eps2, potential=True)
        acc2, _ = run(cn, pi, pj, eps2, potential=False)
    finally:
        for variant in ("f32", "f32_pot"):
            cn.cn_tune_set(variant, n_i, n_j, None)
    ref_a, ref_p = oracle.force(pi, pj, eps2)
    assert e_max(acc, ref_a) <= TOL_F32
    assert e_max(acc2, ref_a) <= TOL_F32
    assert rel_pot_err(pot, ref_p) <= TOL_F32


@pytest.mark.parametrize("tune", [None, {"i_per_thread": 2, "threads": 64, "j_tile": 64, "stages": 3},
                                  {"i_per_thread": 4, "threads": 128, "j_tile": 128, "chunk_units": 5},
                                  {"i_per_thread": 1, "threads": 128, "j_tile": 512, "stages": 3, "j_lanes": 8}])
def test_bitwise_deterministic(tune):
    cn = lib()
    torch = torch_cuda()
    p = synth.plummer(6000, 3)
    t = dev_tensor(p)
    cn.cn_tune_set("f32_pot", 6000, 6000, tune)
    try:
        a1, p1 = cn.cn_force(t, t, 1e-3, potential=True)
        a2, p2 = cn.cn_force(t, t, 1e-3, potential=True)
        torch.cuda.synchronize()
    finally:
        cn.cn_tune_set("f32_pot", 6000, 6000, None)
    assert torch.equal(a1, a2) and torch.equal(p1, p2)


def test_zero_softening_and_coincident_points():
    """eps2 = 0: pairs with zero separation add nothing (no inf/NaN)."""
    cn = lib()
    p = synth.plummer(700, 9)
    p[100:110] = p[50]  # ten exact copies of particle 50
    acc, pot = run(cn, p, p, 0.0, potential=True)
    ref_a, ref_p = oracle.force(p, p, 0.0)
    assert np.all(np.isfinite(acc)) and np.all(np.isfinite(pot))
    assert e_max(acc, ref_a) <= TOL_F32
    assert rel_pot_err(pot, ref_p) <= TOL_F32
    # subnormal eps2 takes the same guarded path
    acc, _ = run(cn, p, p, 1e-40)
    assert np.all(np.isfinite(acc))


def test_potential_excludes_self_and_duplicates_with_softening():
    cn = lib()
    p = synth.plummer(300, 4)
    p[7] = p[3]
    acc, pot = run(cn, p, p, 0.01, potential=True)
    ref_a, ref_p = oracle.force(p, p, 0.01)
    assert rel_pot_err(pot, ref_p) <= TOL_F32
    assert e_max(acc, ref_a) <= TOL_F32


def test_empty_j_set_writes_zeros_and_empty_i_is_noop():
    cn = lib()
    torch = torch_cuda()
    pi = dev_tensor(synth.plummer(50, 1))
    pj = torch.zeros((0, 4), dtype=torch.float32, device="cuda")
    acc = torch.full((50, 3), 7.0, device="cuda")
    pot = torch.full((50,), 7.0, device="cuda")
    cn.cn_force(pi, pj, 0.01, acc_out=acc, pot_out=pot)
    torch.cuda.synchronize()
    assert torch.count_nonzero(acc) == 0 and torch.count_nonzero(pot) == 0
    a0, _ = cn.cn_force(pi[:0], pi, 0.01)
    assert a0.shape == (0, 3)


def test_workspace_form_matches_library_workspace():
    cn = lib()
    torch = torch_cuda()
    p = synth.plummer(5000, 12)
    t = dev_tensor(p)
    nbytes = cn.cn_workspace_bytes("f32_pot", 5000, 5000)
    assert nbytes > 0
    ws = torch.full((nbytes,), 0xAB, dtype=torch.uint8, device="cuda")  # no initialisation needed
    a1, p1 = cn.cn_force_ws(t, t, 1e-3, ws, potential=True)
    ws.fill_(0x5C)  # stale bytes between calls are harmless
    a2, p2 = cn.cn_force_ws(t, t, 1e-3, ws, potential=True)
    a3, p3 = cn.cn_force(t, t, 1e-3, potential=True)
    torch.cuda.synchronize()
    assert torch.equal(a1, a3) and torch.equal(a2, a3) and torch.equal(p1, p3)
    small = torch.zeros(256, dtype=torch.uint8, device="cuda")
    with pytest.raises(cn.CunbodyError) as ei:
        cn.cn_force_ws(t, t, 1e-3, small)
    assert ei.value.code == "CN_ERR_WORKSPACE"


# ------------------------------------------------------------------ compensated form

def test_dd_plummer_all_i():
    cn = lib()
    n = 2048
    p = synth.plummer(n, n)
    eps2 = float(np.float32(synth.plummer_eps(n)) ** 2)
    acc, pot = run(cn, p, p, eps2, potential=True, dd=True)
    ref_a, ref_p = oracle.force(p, p, eps2)
    assert acc.dtype == np.float64
    assert e_max(acc, ref_a) <= TOL_DD
    assert rel_pot_err(pot, ref_p) <= TOL_DD


@pytest.mark.parametrize("shape", [(1, 1), (31, 33), (1000, 777), (4097, 2049)])
def test_dd_ragged(shape):
    cn = lib()
    n_i, n_j = shape
    pj = synth.plummer(n_j, 21 + n_j)
    pi = synth.plummer(n_i, 2 + n_i)
    acc, pot = run(cn, pi, pj, 1e-2, potential=True, dd=True)
    ref_a, ref_p = oracle.force(pi, pj, 1e-2)
    assert e_max(acc, ref_a) <= TOL_DD
    assert rel_pot_err(pot, ref_p) <= TOL_DD


def test_dd_beats_f32_on_plummer_131072_sampled():
    cn = lib()
    n = 131072
    p = synth.plummer(n, n)
    eps2 = float(np.float32(synth.plummer_eps(n)) ** 2)
    rows = synth.sample_rows(n, 2048, seed=77)
    ref, _ = oracle.force(p, p, eps2, rows=rows, potential=False)
    a32, _ = run(cn, p, p, eps2)
    add, _ = run(cn, p, p, eps2, dd=True)
    e32, edd = e_max(a32[rows], ref), e_max(add[rows], ref)
    assert e32 <= TOL_F32
    assert edd <= TOL_DD
    assert edd < e32


def test_dd_c3_hernquist_million_sampled():
    """N = 1,048,576 Hernquist sphere (log-normal masses, eps = 1e-3): the
    compensated form against the oracle on 8192 sampled particles."""
    cn = lib()
    n = 1 << 20
    h = synth.hernquist(n, 1048576)
    eps2 = float(np.float32(1e-3) ** 2)
    rows = synth.sample_rows(n, 8192, seed=8192)
    ref, _ = oracle.force(h, h, eps2, rows=rows, potential=False)
    add, _ = run(cn, h, h, eps2, dd=True)
    a32, _ = run(cn, h, h, eps2)
    edd, e32 = e_max(add[rows], ref), e_max(a32[rows], ref)
    print(f"C3 E_max: compensated {edd:.3e}, plain FP32 {e32:.3e}")
    assert edd <= TOL_DD
    assert e32 <= TOL_F32
    assert edd < e32
