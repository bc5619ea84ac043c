"""cn_force_eps_i: a softening per i-particle, read from the 4th slot of its
record (x, y, z, eps2_i) as in the appendix's force driver (IDIM = 4).
Parity with the FP64 oracle at the plain FP32 bound, including particles
with eps2_i = 0 (guarded pairs), and bitwise agreement with cn_force when
every eps2_i is the same."""

import numpy as np
import pytest

import oracle
from gpu_common import dev_tensor, e_max, lib, rel_pot_err, torch_cuda
from paper_astro_ph_0703100_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _with_eps(p, seed, zero_every=0):
    rng = np.random.default_rng(seed)
    q = p.copy()
    q[:, 3] = rng.uniform(1e-4, 5e-2, size=p.shape[0]).astype(np.float32)
    if zero_every:
        q[::zero_every, 3] = 0.0
    return q


TUNES = [None,
         {"i_per_thread": 1, "threads": 64, "j_tile": 64, "stages": 3},
         {"i_per_thread": 2, "threads": 128, "j_tile": 256, "stages": 4},
         {"i_per_thread": 8, "threads": 256, "j_tile": 512, "stages": 4},
         {"i_per_thread": 2, "threads": 256, "j_tile": 256, "stages": 2, "j_lanes": 16},
         {"i_per_thread": 1, "threads": 128, "j_tile": 256, "stages": 1, "j_lanes": 32}]


@pytest.mark.parametrize("tune", TUNES)
@pytest.mark.parametrize("shape", [(1, 1), (33, 700), (1000, 1000), (4097, 2049)])
def test_eps_i_parity(shape, tune):
    cn = lib()
    torch = torch_cuda()
    n_i, n_j = shape
    pj = synth.plummer(n_j, 60 + n_j)
    pi = _with_eps(synth.plummer(n_i, 61 + n_i), 62 + n_i, zero_every=7)
    for v in ("f32_eps_i", "f32_eps_i_pot"):
        cn.cn_tune_set(v, n_i, n_j, tune)
    try:
        a, pot = cn.cn_force_eps_i(dev_tensor(pi), dev_tensor(pj), potential=True)
        a2, _ = cn.cn_force_eps_i(dev_tensor(pi), dev_tensor(pj))
        torch.cuda.synchronize()
    finally:
        for v in ("f32_eps_i", "f32_eps_i_pot"):
            cn.cn_tune_set(v, n_i, n_j, None)
    assert cn.cn_get_device_status() == 0
    ra, rp = oracle.force_eps_i(pi, pj)
    assert e_max(a.cpu().numpy(), ra) <= TOL
    assert e_max(a2.cpu().numpy(), ra) <= TOL
    assert rel_pot_err(pot.cpu().numpy(), rp) <= TOL


def test_eps_i_zero_softening_with_coincident_points():
    """eps2_i = 0 for every particle and duplicated positions: guarded pairs give nothing."""
    cn = lib()
    torch = torch_cuda()
    p = synth.plummer(500, 63)
    p = np.concatenate([p, p[:50]])
    pi = p.copy()
    pi[:, 3] = 0.0
    a, pot = cn.cn_force_eps_i(dev_tensor(pi), dev_tensor(p), potential=True)
    torch.cuda.synchronize()
    assert np.all(np.isfinite(a.cpu().numpy())) and np.all(np.isfinite(pot.cpu().numpy()))
    ra, rp = oracle.force_eps_i(pi, p)
    assert e_max(a.cpu().numpy(), ra) <= TOL
    assert rel_pot_err(pot.cpu().numpy(), rp) <= TOL


@pytest.mark.parametrize("tune", [{"i_per_thread": 8, "threads": 256, "j_tile": 1024, "stages": 4},
                                  {"i_per_thread": 2, "threads": 256, "j_tile": 2048, "stages": 1,
                                   "j_lanes": 32}])
def test_eps_i_uniform_equals_cn_force_bitwise(tune):
    cn = lib()
    torch = torch_cuda()
    n = 2000
    p = synth.plummer(n, 64)
    eps2 = float(np.float32(0.01))
    pi = p.copy()
    pi[:, 3] = np.float32(eps2)
    for v in ("f32", "f32_eps_i"):
        cn.cn_tune_set(v, n, n, tune)
    try:
        a, _ = cn.cn_force(dev_tensor(p), dev_tensor(p), eps2)
        b, _ = cn.cn_force_eps_i(dev_tensor(pi), dev_tensor(p))
        torch.cuda.synchronize()
    finally:
        for v in ("f32", "f32_eps_i"):
            cn.cn_tune_set(v, n, n, None)
    assert torch.equal(a, b)


def test_eps_i_plummer_131072_sampled():
    """Full size in the default launch shape, softening varying by a factor 100."""
    cn = lib()
    torch = torch_cuda()
    n = 131072
    p = synth.plummer(n, 65)
    pi = _with_eps(p, 66)
    a, _ = cn.cn_force_eps_i(dev_tensor(pi), dev_tensor(p))
    torch.cuda.synchronize()
    rows = synth.sample_rows(n, 1024, 67)
    ra, _ = oracle.force_eps_i(pi, p, rows=rows, potential=False)
    assert e_max(a.cpu().numpy()[rows], ra) <= TOL


@pytest.mark.parametrize("n_i,n_j", [(16384, 16384), (20000, 9000)])
def test_eps_i_mid_size_default_shape_sampled(n_i, n_j):
    """Mid sizes, where the plain form's default uses lane groups of 8 with
    eight i-particles; the per-i-softening kernels hold at most two per lane
    group, so the plan takes two (with and without the potential)."""
    cn = lib()
    torch = torch_cuda()
    p = synth.plummer(n_j, n_j + 68)
    pi = _with_eps(synth.plummer(n_i, n_i + 69), 70)
    a, pot = cn.cn_force_eps_i(dev_tensor(pi), dev_tensor(p), potential=True)
    torch.cuda.synchronize()
    assert cn.cn_get_device_status() == 0
    rows = synth.sample_rows(n_i, 512, 71)
    ra, rp = oracle.force_eps_i(pi, p, rows=rows)
    assert e_max(a.cpu().numpy()[rows], ra) <= TOL
    assert rel_pot_err(pot.cpu().numpy()[rows], rp) <= TOL
