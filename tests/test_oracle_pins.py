"""Pins for the FP64 oracle: closed forms, invariants, brute force and the
paper's printed error table. None of them re-types the oracle's formula.

All run on the CPU (no GPU marker) and finish in well under a minute.
"""

import decimal
import math

import numpy as np
import pytest

import oracle
from conftest import load_table
from paper_astro_ph_0703100_gb300 import synth


def rec(xyz, m):
    xyz = np.asarray(xyz, dtype=np.float32).reshape(-1, 3)
    out = np.empty((xyz.shape[0], 4), dtype=np.float32)
    out[:, :3] = xyz
    out[:, 3] = np.asarray(m, dtype=np.float32)
    return out


# ---------------------------------------------------------------- closed forms

def test_two_body_pythagorean_exact():
    """Eq. 1 with one partner on a 3-4-5 / 5-12-13 triangle: exact rationals."""
    m2 = 0.75
    p = rec([[1.0, -2.0, 0.5], [1.0 + 3.0, -2.0 + 4.0, 0.5]], [0.5, m2])
    # eps = 0: |d| = 5, a_1 = m2 (3, 4, 0) / 125, phi_1 = -m2 / 5
    a, phi = oracle.force(p, p, 0.0)
    assert a[0] == pytest.approx([m2 * 3 / 125, m2 * 4 / 125, 0.0], rel=1e-15, abs=0)
    assert phi[0] == pytest.approx(-m2 / 5, rel=1e-15)
    # the partner feels the opposite pull scaled by the other mass
    assert a[1] == pytest.approx([-0.5 * 3 / 125, -0.5 * 4 / 125, 0.0], rel=1e-15, abs=0)
    # eps^2 = 144: softened distance sqrt(25 + 144) = 13
    a, phi = oracle.force(p, p, 144.0)
    assert a[0] == pytest.approx([m2 * 3 / 2197, m2 * 4 / 2197, 0.0], rel=1e-15, abs=0)
    assert phi[0] == pytest.approx(-m2 / 13, rel=1e-15)


def test_direction_and_sign():
    """r_ij = r_j - r_i: the pull points from i toward j (attractive)."""
    p = rec([[0, 0, 0], [0, 0, 2.0]], [1.0, 1.0])
    a, _ = oracle.force(p[:1], p[1:], 0.0)
    assert a[0, 2] == pytest.approx(0.25, rel=1e-15)
    assert a[0, 0] == 0.0 and a[0, 1] == 0.0


def test_octahedron_symmetry():
    """Six unit masses at +-e_k and one mass m0 at the origin.

    Centre: zero force by symmetry. Vertex +e_1: the opposite vertex at
    distance 2, four neighbours at distance sqrt(2) (their transverse pulls
    cancel pairwise) and the centre at distance 1 give, with eps = 0,
    a_x = -(2/8 + 4 * 1/2^(3/2)) - m0.
    """
    m0 = 0.5
    pts = [[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1], [0, 0, 0]]
    p = rec(pts, [1, 1, 1, 1, 1, 1, m0])
    a, phi = oracle.force(p, p, 0.0)
    assert np.abs(a[6]).max() < 1e-15
    ax = -(2.0 / 8.0 + 4.0 / 2.0 ** 1.5) - m0
    assert a[0, 0] == pytest.approx(ax, rel=1e-14)
    assert abs(a[0, 1]) < 1e-15 and abs(a[0, 2]) < 1e-15
    # potential at a vertex: -(1/2 + 4/sqrt(2) + m0/1)
    assert phi[0] == pytest.approx(-(0.5 + 4 / math.sqrt(2) + m0), rel=1e-14)
    # potential at the centre: -6 (six unit masses at distance 1)
    assert phi[6] == pytest.approx(-6.0, rel=1e-15)


def test_self_pair_and_coincident_points():
    """s = 0 pairs add nothing; the potential skips exact zero separations."""
    p = rec([[0.5, 0.5, 0.5], [0.5, 0.5, 0.5], [1.5, 0.5, 0.5]], [1.0, 2.0, 4.0])
    a, phi = oracle.force(p, p, 0.0)
    # particle 0 feels only particle 2 (distance 1 along +x)
    assert a[0] == pytest.approx([4.0, 0.0, 0.0], rel=1e-15)
    assert phi[0] == pytest.approx(-4.0, rel=1e-15)
    # with softening the coincident partner still adds no force (d = 0) and
    # is still excluded from the potential (zero separation)
    a, phi = oracle.force(p, p, 0.25)
    assert a[0] == pytest.approx([4.0 / 1.25 ** 1.5, 0.0, 0.0], rel=1e-15)
    assert phi[0] == pytest.approx(-4.0 / math.sqrt(1.25), rel=1e-15)


def test_empty_sets():
    p = synth.plummer(5, 1)
    a, phi = oracle.force(p, p[:0], 0.01)
    assert np.all(a == 0) and np.all(phi == 0)
    a, phi = oracle.force(p[:0], p, 0.01)
    assert a.shape == (0, 3)


# ---------------------------------------------------------------- brute force

def _decimal_force(p, eps2, prec=50):
    """eps2: one softening for every pair, or one per i-particle."""
    ctx = decimal.Context(prec=prec)
    D = decimal.Decimal
    n = p.shape[0]
    e2s = np.broadcast_to(np.asarray(eps2, dtype=np.float32), (n,))
    out = []
    for i in range(n):
        e2 = D(float(e2s[i]))
        acc = [D(0), D(0), D(0)]
        pot = D(0)
        for j in range(n):
            d = [ctx.subtract(D(float(p[j, k])), D(float(p[i, k]))) for k in range(3)]
            s = ctx.add(ctx.add(ctx.add(ctx.multiply(d[0], d[0]), ctx.multiply(d[1], d[1])),
                                ctx.multiply(d[2], d[2])), e2)
            if s == 0:
                continue
            root = ctx.sqrt(s)
            f = ctx.divide(D(float(p[j, 3])), ctx.multiply(s, root))
            for k in range(3):
                acc[k] = ctx.add(acc[k], ctx.multiply(f, d[k]))
            if any(x != 0 for x in d):
                pot = ctx.subtract(pot, ctx.divide(D(float(p[j, 3])), root))
        out.append(([float(x) for x in acc], float(pot)))
    return out


@pytest.mark.parametrize("n,seed,eps2", [(2, 3, 0.0), (5, 7, 1e-2), (8, 11, 2.0 ** -12), (8, 13, 0.0)])
def test_bruteforce_50_digits(n, seed, eps2):
    rng = np.random.default_rng(seed)
    p = np.empty((n, 4), dtype=np.float32)
    p[:, :3] = rng.normal(size=(n, 3)).astype(np.float32)
    p[:, 3] = rng.uniform(0.1, 2.0, size=n).astype(np.float32)
    a, phi = oracle.force(p, p, eps2)
    ref = _decimal_force(p, eps2)
    for i in range(n):
        assert a[i] == pytest.approx(ref[i][0], rel=1e-14, abs=1e-14 * np.abs(ref[i][0]).max())
        assert phi[i] == pytest.approx(ref[i][1], rel=1e-14)


def test_eps_i_two_body_closed_form():
    """Softening per i-particle (the i record's 4th slot): each particle of a
    3-4-5 pair feels its own softened distance, sqrt(25 + 144) = 13 and 5."""
    m1, m2 = 0.5, 0.75
    pj = rec([[1.0, -2.0, 0.5], [4.0, 2.0, 0.5]], [m1, m2])
    pi = pj.copy()
    pi[:, 3] = [144.0, 0.0]
    a, phi = oracle.force_eps_i(pi, pj)
    assert a[0] == pytest.approx([m2 * 3 / 2197, m2 * 4 / 2197, 0.0], rel=1e-15, abs=0)
    assert phi[0] == pytest.approx(-m2 / 13, rel=1e-15)
    assert a[1] == pytest.approx([-m1 * 3 / 125, -m1 * 4 / 125, 0.0], rel=1e-15, abs=0)
    assert phi[1] == pytest.approx(-m1 / 5, rel=1e-15)


@pytest.mark.parametrize("n,seed", [(6, 17), (8, 19)])
def test_eps_i_bruteforce_50_digits(n, seed):
    rng = np.random.default_rng(seed)
    pj = np.empty((n, 4), dtype=np.float32)
    pj[:, :3] = rng.normal(size=(n, 3)).astype(np.float32)
    pj[:, 3] = rng.uniform(0.1, 2.0, size=n).astype(np.float32)
    eps2 = rng.uniform(0.0, 0.5, size=n).astype(np.float32)
    eps2[0] = 0.0
    pi = pj.copy()
    pi[:, 3] = eps2
    a, phi = oracle.force_eps_i(pi, pj)
    ref = _decimal_force(pj, eps2)
    for i in range(n):
        assert a[i] == pytest.approx(ref[i][0], rel=1e-14, abs=1e-14 * np.abs(ref[i][0]).max())
        assert phi[i] == pytest.approx(ref[i][1], rel=1e-14)


# ---------------------------------------------------------------- invariants

def test_momentum_conservation():
    """Newton's third law: sum_i m_i a_i = 0 when the i and j sets coincide."""
    p = synth.plummer(2000, 5)
    a, _ = oracle.force(p, p, 1e-4, potential=False)
    m = p[:, 3].astype(np.float64)
    total = (m[:, None] * a).sum(axis=0)
    scale = (m * np.linalg.norm(a, axis=1)).sum()
    assert np.abs(total).max() <= 1e-13 * scale


def test_j_permutation_invariance():
    p = synth.plummer(3000, 8)
    perm = np.random.default_rng(1).permutation(p.shape[0])
    rows = np.arange(0, 3000, 7)
    a1, f1 = oracle.force(p, p, 1e-3, rows=rows)
    a2, f2 = oracle.force(p, p[perm], 1e-3, rows=rows)
    assert np.abs(a1 - a2).max() <= 1e-14 * np.abs(a1).max()
    assert np.abs(f1 - f2).max() <= 1e-14 * np.abs(f1).max()


def test_translation_and_mass_scaling():
    """a is invariant under a common shift and linear in the j masses."""
    p = synth.plummer(500, 21)
    # put positions on a 2^-16 grid inside |x| < 64 so that a shift by 1/2 is exact in FP32
    p[:, :3] = np.clip(np.round(p[:, :3] * 65536) / 65536, -63, 63)
    q = p.copy()
    q[:, :3] += np.float32(0.5)
    assert np.array_equal(q[:, :3].astype(np.float64) - 0.5, p[:, :3].astype(np.float64))
    a1, _ = oracle.force(p, p, 1e-2, potential=False)
    a2, _ = oracle.force(q, q, 1e-2, potential=False)
    assert np.abs(a1 - a2).max() <= 1e-13 * np.abs(a1).max()
    r = p.copy()
    r[:, 3] *= np.float32(4.0)
    a3, _ = oracle.force(p, r, 1e-2, potential=False)
    assert np.abs(a3 - 4 * a1).max() <= 1e-14 * np.abs(a1).max()


def test_potential_force_consistency():
    """a = -grad(phi) at external test points (Richardson-extrapolated FD)."""
    src = synth.plummer(400, 31)
    # test points on a 2^-6 grid so that +-h (h = 2^-9, 2^-10) is exact in FP32
    rng = np.random.default_rng(2)
    pts = np.round(rng.uniform(-1, 1, size=(12, 3)) * 64) / 64
    eps2 = 1e-2
    for x in pts:
        a, _ = oracle.force(rec([x], [0.0]), src, eps2, potential=False)
        grad = []
        for k in range(3):
            est = []
            for h in (2.0 ** -9, 2.0 ** -10):
                xp = x.copy(); xp[k] += h
                xm = x.copy(); xm[k] -= h
                _, pp = oracle.force(rec([xp], [0.0]), src, eps2)
                _, pm = oracle.force(rec([xm], [0.0]), src, eps2)
                est.append((pp[0] - pm[0]) / (2 * h))
            grad.append((4 * est[1] - est[0]) / 3)
        assert np.allclose(a[0], -np.array(grad), rtol=1e-7, atol=1e-7 * np.abs(a[0]).max())


# ---------------------------------------------------------------- Plummer sphere

def test_plummer_potential_energy():
    """W = 1/2 sum m_i phi_i -> -3 pi / 32 (G = M = a = 1) as N grows, eps -> 0.

    A finite sample has E[W] = (1 - 1/N)(-3 pi / 32) before softening; the
    seed-to-seed spread at N = 16384 is about 0.6 %.
    """
    n, eps2 = 16384, np.float32(1e-3) ** 2
    target = -3 * math.pi / 32 * (1 - 1 / n)
    ws = []
    for seed in (101, 202, 303, 404):
        p = synth.plummer(n, seed)
        _, phi = oracle.force(p, p, eps2)
        ws.append(oracle.potential_energy(p, phi))
    ws = np.array(ws)
    assert abs(ws.mean() / target - 1) < 0.01
    assert np.all(np.abs(ws / target - 1) < 0.03)


def test_plummer_radial_field():
    """Shell-averaged radial pull vs the analytic -r / (r^2 + 1)^(3/2)."""
    n = 8192
    p = synth.plummer(n, 77)
    a, _ = oracle.force(p, p, np.float32(1e-3) ** 2, potential=False)
    x = p[:, :3].astype(np.float64)
    r = np.linalg.norm(x, axis=1)
    ar = (a * x).sum(axis=1) / r
    for lo, hi in [(0.3, 0.5), (0.5, 0.8), (0.8, 1.2), (1.2, 2.0), (2.0, 3.5)]:
        sel = (r >= lo) & (r < hi)
        model = -r[sel] / (r[sel] ** 2 + 1) ** 1.5
        assert abs(ar[sel].mean() / model.mean() - 1) < 0.03, (lo, hi)


# ---------------------------------------------------------------- adjoint oracle

def _adjoint_case(n=64, seed=5, eps2=0.05):
    p = synth.plummer(n, seed)
    w = synth.adjoint_weights(n, seed + 1)
    return p, w, np.float32(eps2)


def test_adjoint_matches_finite_differences():
    p, w, eps2 = _adjoint_case()
    gp, gm = oracle.adjoint(p, eps2, w)
    for k in (0, 7, 33, 63):
        x0 = p[k, :3].astype(np.float64)
        m0 = float(p[k, 3])
        for c in range(3):
            est = []
            for h in (1e-4, 5e-5):
                xp = x0.copy(); xp[c] += h
                xm = x0.copy(); xm[c] -= h
                est.append((oracle.loss_k(p, eps2, w, k, xp, m0) - oracle.loss_k(p, eps2, w, k, xm, m0)) / (2 * h))
            fd = (4 * est[1] - est[0]) / 3
            assert fd == pytest.approx(gp[k, c], rel=1e-6, abs=1e-9 * np.abs(gp).max())
        h = 1e-3 * m0
        fdm = (oracle.loss_k(p, eps2, w, k, x0, m0 + h) - oracle.loss_k(p, eps2, w, k, x0, m0 - h)) / (2 * h)
        assert fdm == pytest.approx(gm[k], rel=1e-9, abs=1e-12 * np.abs(gm).max())


def test_adjoint_invariants():
    """Translation: sum_k dL/dx_k = 0. Linearity in mass: sum_k m_k dL/dm_k = L.
    With eps = 0, a is homogeneous of degree -2 in positions, so
    sum_k x_k . dL/dx_k = -2 L."""
    p, w, eps2 = _adjoint_case(n=200, seed=9, eps2=0.02)
    a, _ = oracle.force(p, p, eps2, potential=False)
    L = float((w.astype(np.float64) * a).sum())
    gp, gm = oracle.adjoint(p, eps2, w)
    scale = np.abs(gp).sum()
    assert np.abs(gp.sum(axis=0)).max() <= 1e-12 * scale
    assert float((p[:, 3].astype(np.float64) * gm).sum()) == pytest.approx(L, rel=1e-12)
    a0, _ = oracle.force(p, p, 0.0, potential=False)
    L0 = float((w.astype(np.float64) * a0).sum())
    gp0, _ = oracle.adjoint(p, 0.0, w)
    assert float((p[:, :3].astype(np.float64) * gp0).sum()) == pytest.approx(-2 * L0, rel=1e-11)


def test_adjoint_rows_subset():
    p, w, eps2 = _adjoint_case(n=120, seed=3)
    gp, gm = oracle.adjoint(p, eps2, w)
    rows = np.array([5, 17, 119])
    gp2, gm2 = oracle.adjoint(p, eps2, w, rows=rows)
    assert np.array_equal(gp[rows], gp2) and np.array_equal(gm[rows], gm2)


# ---------------------------------------------------------------- paper's error table

@pytest.mark.parametrize("n", [2048, 4096, 8192, 16384])
def test_cumulative_error_trend_matches_table(n):
    """FP32 DIRECT vs FORCE-LOOP errors land in the paper's decade (Table 2).

    The paper does not state its softening; the test program of Section 3.1
    uses eps2 = 0.01, taken here. Inputs, hardware rounding and the sampled
    sphere differ, so the check is a factor-of-3 band, plus the ordering
    DIRECT > FORCE-LOOP > exact sum of FP32 terms.
    """
    table = {int(r[0]): (r[1], r[2]) for r in load_table("cumerror_table.txt")}
    p = synth.plummer(n, n)
    ref, _ = oracle.force(p, p, 0.01, potential=False)
    e_direct = oracle.e_max(oracle.fp32_study(p, p, 0.01, oracle.FP32_DIRECT), ref)
    e_loop = oracle.e_max(oracle.fp32_study(p, p, 0.01, oracle.FP32_FORCE_LOOP, 512), ref)
    e_exact = oracle.e_max(oracle.fp32_study(p, p, 0.01, oracle.FP32_EXACT_SUM), ref)
    t_direct, t_loop = table[n]
    assert t_direct / 3 < e_direct < t_direct * 3
    assert t_loop / 3 < e_loop < t_loop * 3
    assert e_direct > e_loop > e_exact


# ---------------------------------------------------------------- force, jerk, potential (appendix pipeline)

def _vel(v):
    v = np.asarray(v, dtype=np.float32).reshape(-1, 3)
    out = np.zeros((v.shape[0], 4), dtype=np.float32)
    out[:, :3] = v
    return out


def test_jerk_two_body_exact():
    """Partner at d = (3, 4, 0), eps = 0, mass m: with relative velocity
    (0, 0, 1) the jerk is m (0, 0, 1/125); with (1, 0, 0), d.w = 3 and the
    jerk is m [(1, 0, 0)/125 - 9 (3, 4, 0)/3125] = m (-0.00064, -0.01152, 0)."""
    m = 0.5
    p = rec([[0, 0, 0], [3, 4, 0]], [1.0, m])
    for w, expect in (([0, 0, 1], [0, 0, m / 125]), ([1, 0, 0], [-0.00064 * m, -0.01152 * m, 0.0])):
        v = _vel([[0, 0, 0], w])
        a, j, phi = oracle.force_jerk(p, v, p, v, 0.0)
        assert a[0] == pytest.approx([m * 3 / 125, m * 4 / 125, 0.0], rel=1e-15, abs=0)
        assert j[0] == pytest.approx(expect, rel=1e-14, abs=1e-17)
        assert phi[0] == pytest.approx(-m / 5, rel=1e-15)


def test_jerk_is_time_derivative_of_acceleration():
    """j_i = d a_i / dt for straight-line motion x(t) = x + v t
    (Richardson-extrapolated central differences of the oracle's own force)."""
    n = 64
    p = synth.plummer(n, 12)
    v = synth.plummer_velocities(n, 13)
    eps2 = 0.01
    a, j, _ = oracle.force_jerk(p, v, p, v, eps2)
    est = []
    for h in (2.0 ** -10, 2.0 ** -11):
        pp = p.astype(np.float64).copy()
        pm = p.astype(np.float64).copy()
        pp[:, :3] += h * v[:, :3]
        pm[:, :3] -= h * v[:, :3]
        # the oracle takes FP32 records: difference quotients in FP64 need the
        # moved positions exactly, so evaluate the FP64 definition directly
        def acc64(q):
            d = q[None, :, :3] - q[:, None, :3]
            s = (d ** 2).sum(-1) + np.float64(np.float32(eps2))
            w = q[None, :, 3] / (s * np.sqrt(s))
            return (w[:, :, None] * d).sum(1)
        est.append((acc64(pp) - acc64(pm)) / (2 * h))
    fd = (4 * est[1] - est[0]) / 3
    assert np.abs(fd - j).max() <= 1e-8 * np.abs(j).max()
    assert np.abs(acc64(p.astype(np.float64)) - a).max() <= 1e-12 * np.abs(a).max()


def test_jerk_invariants():
    """sum_i m_i j_i = 0 (i set = j set), and a common velocity shift leaves
    the jerk unchanged (it depends on velocity differences only)."""
    n = 500
    p = synth.plummer(n, 31)
    v = synth.plummer_velocities(n, 32)
    _, j, _ = oracle.force_jerk(p, v, p, v, 1e-3)
    m = p[:, 3].astype(np.float64)
    scale = (m * np.linalg.norm(j, axis=1)).sum()
    assert np.abs((m[:, None] * j).sum(0)).max() <= 1e-13 * scale
    v2 = v.copy()
    v2[:, :3] += np.float32(0.25)
    exact = np.array_equal(v2[:, :3].astype(np.float64) - 0.25, v[:, :3].astype(np.float64))
    _, j2, _ = oracle.force_jerk(p, v2, p, v2, 1e-3)
    assert np.abs(j2 - j).max() <= (1e-14 if exact else 1e-6) * np.abs(j).max()
    # the acceleration and potential agree with the force-only oracle
    a0, phi0 = oracle.force(p, p, 1e-3)
    a1, _, phi1 = oracle.force_jerk(p, v, p, v, 1e-3)
    assert np.array_equal(a0, a1) and np.array_equal(phi0, phi1)
