"""The packed (f32x2) pair kernels against their scalar forms, bit for bit.

The packed policies (two i-particles per 64-bit register pair) perform the
same lane-level FP32 operations in the same order as the scalar policies, so
on a launch shape where no i-tile is split across CTAs (the whole j set in
one tile, fewer units than resident CTAs) the results must be identical.
K = 1 runs the scalar policy; K = 2, 4, 8 the packed one.
"""

import numpy as np
import pytest

from gpu_common import dev_tensor, lib, torch_cuda
from paper_astro_ph_0703100_gb300 import synth

pytestmark = pytest.mark.gpu

N = 2000
JT = 2048  # one j-tile holds the whole j set


def _shape(k, threads=64):
    return {"i_per_thread": k, "threads": threads, "j_tile": JT, "stages": 1}


def _with_tune(cn, variants, tune, fn):
    for v in variants:
        cn.cn_tune_set(v, N, N, tune)
    try:
        return fn()
    finally:
        for v in variants:
            cn.cn_tune_set(v, N, N, None)


@pytest.mark.parametrize("potential", [False, True])
def test_plain_packed_equals_scalar(potential):
    cn = lib()
    torch = torch_cuda()
    p = dev_tensor(synth.plummer(N, 77))
    v = "f32_pot" if potential else "f32"

    def run():
        a, pot = cn.cn_force(p, p, 1e-3, potential=potential)
        torch.cuda.synchronize()
        return a.cpu().numpy(), (pot.cpu().numpy() if pot is not None else None)

    a1, p1 = _with_tune(cn, [v], _shape(1), run)
    for k in (2, 4, 8):
        ak, pk = _with_tune(cn, [v], _shape(k), run)
        assert np.array_equal(a1, ak), k
        if potential:
            assert np.array_equal(p1, pk), k


@pytest.mark.parametrize("potential", [False, True])
@pytest.mark.parametrize("j_lanes", [8, 16, 32])
def test_splitj_packed_equals_scalar(potential, j_lanes):
    """Split-j shapes: lanes of a group take every j_lanes-th j record; the
    packed form holds two, four or eight i-particles per group."""
    cn = lib()
    torch = torch_cuda()
    p = dev_tensor(synth.plummer(N, 82))
    v = "f32_pot" if potential else "f32"

    def run():
        a, pot = cn.cn_force(p, p, 1e-3, potential=potential)
        torch.cuda.synchronize()
        return a.cpu().numpy(), (pot.cpu().numpy() if pot is not None else None)

    shape = dict(_shape(1, threads=128), j_lanes=j_lanes)
    a1, p1 = _with_tune(cn, [v], shape, run)
    for k in (2, 4, 8):
        ak, pk = _with_tune(cn, [v], dict(shape, i_per_thread=k), run)
        assert np.array_equal(a1, ak), k
        if potential:
            assert np.array_equal(p1, pk), k


@pytest.mark.parametrize("potential", [False, True])
def test_compensated_packed_equals_scalar(potential):
    """The compensated form: K = 1 runs the scalar policy, K = 2 and 4 the
    packed one (the same lane-level operations, selects per half)."""
    cn = lib()
    torch = torch_cuda()
    p = dev_tensor(synth.plummer(N, 83))
    v = "dd_pot" if potential else "dd"

    def run():
        a, pot = cn.cn_force_dd(p, p, 1e-3, potential=potential)
        torch.cuda.synchronize()
        return a.cpu().numpy(), (pot.cpu().numpy() if pot is not None else None)

    a1, p1 = _with_tune(cn, [v], _shape(1), run)
    for k in (2, 4):
        ak, pk = _with_tune(cn, [v], _shape(k), run)
        assert np.array_equal(a1, ak), k
        if potential:
            assert np.array_equal(p1, pk), k


def test_adjoint_packed_equals_scalar():
    cn = lib()
    torch = torch_cuda()
    p = dev_tensor(synth.plummer(N, 78))
    w = dev_tensor(synth.adjoint_weights(N, 79))

    def run():
        gp, gm = cn.cn_force_adjoint(p, 1e-3, w)
        torch.cuda.synchronize()
        return gp.cpu().numpy(), gm.cpu().numpy()

    g1, m1 = _with_tune(cn, ["adjoint"], _shape(1), run)
    for k in (2, 4):
        gk, mk = _with_tune(cn, ["adjoint"], _shape(k), run)
        assert np.array_equal(g1, gk), k
        assert np.array_equal(m1, mk), k


@pytest.mark.parametrize("potential", [False, True])
def test_jerk_packed_equals_scalar(potential):
    cn = lib()
    torch = torch_cuda()
    p = dev_tensor(synth.plummer(N, 80))
    v = dev_tensor(synth.plummer_velocities(N, 81))
    variants = ["jerk", "jerk_pot"]

    def run():
        a, j, pot = cn.cn_force_jerk(p, v, p, v, 1e-3, potential=potential)
        torch.cuda.synchronize()
        return a.cpu().numpy(), j.cpu().numpy(), (pot.cpu().numpy() if pot is not None else None)

    a1, j1, p1 = _with_tune(cn, variants, _shape(1), run)
    for k in (2, 4):
        ak, jk, pk = _with_tune(cn, variants, _shape(k), run)
        assert np.array_equal(a1, ak), k
        assert np.array_equal(j1, jk), k
        if potential:
            assert np.array_equal(p1, pk), k
