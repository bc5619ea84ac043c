"""Systems beyond the benchmark sizes: 64-bit unit and slot indexing, many
split tiles, the symmetric form's bands. Sampled rows against the oracle."""

import numpy as np
import pytest

import oracle
from gpu_common import dev_tensor, e_max, lib, torch_cuda
from paper_astro_ph_0703100_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


def test_plain_force_four_million():
    """N = 2^22 Plummer sphere (1.8e13 pairs, 2^21 x 2^13 units of the default shape)."""
    cn = lib()
    torch = torch_cuda()
    n = 1 << 22
    p = synth.plummer(n, 22)
    eps2 = float(np.float32(synth.plummer_eps(n)) ** 2)
    a, _ = cn.cn_force(dev_tensor(p), dev_tensor(p), eps2)
    torch.cuda.synchronize()
    assert cn.cn_get_device_status() == 0
    rows = synth.sample_rows(n, 128, 23)
    ref, _ = oracle.force(p, p, eps2, rows=rows, potential=False)
    assert e_max(a.cpu().numpy()[rows], ref) <= TOL


def test_symmetric_two_million_in_bands():
    """N = 2^21: 1024 tiles, 32 bands of 32 rows under the 2 GiB slot budget."""
    cn = lib()
    torch = torch_cuda()
    n = 1 << 21
    p = synth.plummer(n, 24)
    eps2 = float(np.float32(synth.plummer_eps(n)) ** 2)
    a, _ = cn.cn_force_symmetric(dev_tensor(p), eps2)
    torch.cuda.synchronize()
    assert cn.cn_get_device_status() == 0
    rows = synth.sample_rows(n, 128, 25)
    ref, _ = oracle.force(p, p, eps2, rows=rows, potential=False)
    assert e_max(a.cpu().numpy()[rows], ref) <= TOL
