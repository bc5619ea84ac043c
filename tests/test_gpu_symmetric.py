"""Parity of cn_force_symmetric (each unordered pair evaluated once) with the FP64 oracle.

The symmetric form computes the same accelerations as the paper's kernel
(Eq. 1 with the i set equal to the j set), so it is held to the same
per-particle bound E_max <= 1e-5 as the plain FP32 form. Its partial sums
are FP32 (the j-side per tile pair, the i-side per CTA and tile row),
merged in FP64 in a fixed order, so repeated calls with one launch shape
are bitwise equal.
"""

import numpy as np
import pytest

import oracle
from gpu_common import dev_tensor, e_max, lib, rel_pot_err, torch_cuda
from paper_astro_ph_0703100_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


def run(cn, p, eps2, potential=False):
    torch = torch_cuda()
    a, pot = cn.cn_force_symmetric(dev_tensor(p), eps2, potential=potential)
    torch.cuda.synchronize()
    assert cn.cn_get_device_status() == 0
    return (a.cpu().numpy(), pot.cpu().numpy()) if potential else a.cpu().numpy()


TUNES = [None,
         {"i_per_thread": 1, "threads": 64, "j_tile": 16, "stages": 2},
         {"i_per_thread": 2, "threads": 128, "j_tile": 64, "stages": 3},
         {"i_per_thread": 4, "threads": 128, "j_tile": 128, "stages": 1},
         {"i_per_thread": 8, "threads": 128, "j_tile": 256, "stages": 4, "ctas_per_sm": 1},
         {"i_per_thread": 8, "threads": 256, "j_tile": 512, "stages": 2}]


@pytest.mark.parametrize("tune", TUNES)
@pytest.mark.parametrize("n", [1, 2, 33, 1000, 4097])
def test_symmetric_ragged_and_launch_shapes(n, tune):
    cn = lib()
    p = synth.plummer(n, 50 + n)
    # with the potential, tiles of 2048 particles need more shared memory than a CTA has
    with_pot = tune is None or tune["i_per_thread"] * tune["threads"] <= 1024
    cn.cn_tune_set("symmetric", n, n, tune)
    try:
        a = run(cn, p, 1e-3)
        if with_pot:
            a2, pot = run(cn, p, 1e-3, potential=True)
    finally:
        cn.cn_tune_set("symmetric", n, n, None)
    ref, rpot = oracle.force(p, p, 1e-3)
    assert e_max(a, ref) <= TOL
    if with_pot:
        assert e_max(a2, ref) <= TOL
        assert rel_pot_err(pot, rpot) <= TOL


def test_symmetric_potential_rejects_oversized_tiles():
    """An explicit 2048-particle tile cannot hold four sums per particle."""
    cn = lib()
    torch = torch_cuda()
    n = 3000
    cn.cn_tune_set("symmetric", n, n, {"i_per_thread": 8, "threads": 256, "j_tile": 256, "stages": 3})
    try:
        d = dev_tensor(synth.plummer(n, 34))
        with pytest.raises(cn.CunbodyError):
            cn.cn_force_symmetric(d, 1e-3, potential=True)
        a, _ = cn.cn_force_symmetric(d, 1e-3)  # the force alone fits
        torch.cuda.synchronize()
    finally:
        cn.cn_tune_set("symmetric", n, n, None)


def test_symmetric_unequal_masses_many_tiles():
    """Log-normal masses: the i-side (m_j) and j-side (m_i) weights differ per pair."""
    cn = lib()
    n = 20000
    p = synth.hernquist(n, 3)
    cn.cn_tune_set("symmetric", n, n, {"i_per_thread": 2, "threads": 64, "j_tile": 32, "stages": 4})
    try:
        a = run(cn, p, 1e-4)
    finally:
        cn.cn_tune_set("symmetric", n, n, None)
    ref, _ = oracle.force(p, p, 1e-4, potential=False)
    assert e_max(a, ref) <= TOL


def test_symmetric_zero_softening_guard():
    """eps2 = 0 takes the guarded kernel: the self pair contributes nothing."""
    cn = lib()
    n = 777
    p = synth.plummer(n, 8)
    a = run(cn, p, 0.0)
    ref, _ = oracle.force(p, p, 0.0, potential=False)
    assert np.all(np.isfinite(a))
    assert e_max(a, ref) <= TOL


def test_symmetric_deterministic_and_matches_plain_form():
    cn = lib()
    torch = torch_cuda()
    n = 9000
    p = synth.plummer(n, 12)
    d = dev_tensor(p)
    a1, _ = cn.cn_force_symmetric(d, 1e-3)
    a2, _ = cn.cn_force_symmetric(d, 1e-3)
    plain, _ = cn.cn_force(d, d, 1e-3)
    torch.cuda.synchronize()
    assert torch.equal(a1, a2)
    ref, _ = oracle.force(p, p, 1e-3, potential=False)
    assert e_max(a1.cpu().numpy(), ref) <= TOL
    assert e_max(plain.cpu().numpy(), ref) <= TOL


@pytest.mark.parametrize("rows", [1, 2, 3])
def test_symmetric_bands_reproducible_and_close_to_one_band(rows):
    """Banded evaluation (chunk_units = tile rows per band): each launch
    configuration gives bit-identical results when repeated; the band
    launches cut the tile rows into other CTA segments than the one-band
    launch, so the two differ only by the FP32 rounding of those segment
    sums (and both match the oracle)."""
    cn = lib()
    torch = torch_cuda()
    n = 5000
    p = synth.hernquist(n, 9)
    d = dev_tensor(p)
    shape = {"i_per_thread": 2, "threads": 64, "j_tile": 64, "stages": 3}
    cn.cn_tune_set("symmetric", n, n, shape)
    try:
        one, pone = cn.cn_force_symmetric(d, 1e-4, potential=True)
        one2, pone2 = cn.cn_force_symmetric(d, 1e-4, potential=True)
        cn.cn_tune_set("symmetric", n, n, dict(shape, chunk_units=rows))
        banded, pband = cn.cn_force_symmetric(d, 1e-4, potential=True)
        banded2, pband2 = cn.cn_force_symmetric(d, 1e-4, potential=True)
        torch.cuda.synchronize()
    finally:
        cn.cn_tune_set("symmetric", n, n, None)
    assert cn.cn_get_device_status() == 0
    assert torch.equal(one, one2) and torch.equal(pone, pone2)
    assert torch.equal(banded, banded2) and torch.equal(pband, pband2)
    a1 = one.cpu().numpy().astype(np.float64)
    assert e_max(banded.cpu().numpy(), a1) <= 1e-6
    assert rel_pot_err(pband.cpu().numpy(), pone.cpu().numpy()) <= 1e-6
    ref, rpot = oracle.force(p, p, 1e-4)
    assert e_max(banded.cpu().numpy(), ref) <= TOL
    assert rel_pot_err(pband.cpu().numpy(), rpot) <= TOL


def test_symmetric_empty():
    cn = lib()
    torch = torch_cuda()
    a, pot = cn.cn_force_symmetric(torch.empty((0, 4), dtype=torch.float32, device="cuda"), 1e-3, potential=True)
    assert a.shape == (0, 3) and pot.shape == (0,)


def test_symmetric_rejects_j_lanes():
    """Split-j lanes are a plain-form option: the symmetric variant refuses them."""
    import ctypes

    cn = lib()
    t = cn.cn_tune()
    t.i_per_thread, t.threads, t.j_tile, t.stages, t.j_lanes = 1, 128, 128, 2, 4
    assert cn.load().cn_tune_set(9, 100, 100, ctypes.byref(t)) == 1


def test_symmetric_plummer_131072_sampled():
    """The headline system (N = 131072 Plummer, eps = 4 / N^(1/3)) in the default launch shape."""
    cn = lib()
    n = 131072
    p = synth.plummer(n, 1)
    eps2 = float(np.float32(synth.plummer_eps(n)) ** 2)
    a = run(cn, p, eps2)
    rows = synth.sample_rows(n, 512, 7)
    ref, _ = oracle.force(p, p, eps2, rows=rows, potential=False)
    assert e_max(a[rows], ref) <= TOL


def test_symmetric_million_automatic_bands_sampled():
    """N = 2^20: the one-band slot array (8.6 GB) exceeds the 2 GiB budget, so
    the rows run in bands; sampled rows against the oracle."""
    cn = lib()
    n = 1 << 20
    p = synth.plummer(n, 20)
    eps2 = float(np.float32(synth.plummer_eps(n)) ** 2)
    a = run(cn, p, eps2)
    rows = synth.sample_rows(n, 256, 21)
    ref, _ = oracle.force(p, p, eps2, rows=rows, potential=False)
    assert e_max(a[rows], ref) <= TOL


def test_symmetric_potential_coincident_points_and_zero_softening():
    """Duplicated positions in different tiles and eps2 = 0: the potential
    skips pairs at zero separation, the force gets nothing from them."""
    cn = lib()
    p = synth.plummer(700, 31)
    p = np.concatenate([p, p[:90]])
    for eps2 in (0.0, 1e-3):
        a, pot = run(cn, p, eps2, potential=True)
        ref, rpot = oracle.force(p, p, eps2)
        assert np.all(np.isfinite(a)) and np.all(np.isfinite(pot))
        assert e_max(a, ref) <= TOL
        assert rel_pot_err(pot, rpot) <= TOL


def test_symmetric_potential_energy_plummer_131072():
    """W = 1/2 sum m phi from the symmetric potentials at the benchmark size."""
    cn = lib()
    torch = torch_cuda()
    n = 131072
    p = synth.plummer(n, 32)
    eps2 = float(np.float32(synth.plummer_eps(n)) ** 2)
    d = dev_tensor(p)
    _, pot = cn.cn_force_symmetric(d, eps2, potential=True)
    _, pot_plain = cn.cn_force(d, d, eps2, potential=True)
    torch.cuda.synchronize()
    rows = synth.sample_rows(n, 256, 33)
    _, rpot = oracle.force(p, p, eps2, rows=rows)
    assert rel_pot_err(pot.cpu().numpy()[rows], rpot) <= TOL
    w_sym = float(cn.cn_potential_energy(d, pot).item())
    w_plain = float(cn.cn_potential_energy(d, pot_plain).item())
    assert abs(w_sym - w_plain) <= 1e-6 * abs(w_plain)
