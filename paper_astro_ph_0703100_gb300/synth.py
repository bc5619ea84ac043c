"""Seeded synthetic particle sets shaped like the paper's workloads.

The paper builds its test systems with an external tool (an equal-mass
Plummer sphere, Section 3.3); these generators stand in for it. They hold
none of the force arithmetic: they only draw particle records, which both
the GPU path and the FP64 oracle then consume unchanged.

Every generator draws in FP64 from ``numpy.random.Generator(PCG64(seed))``
in a fixed order and rounds the result once to an FP32 ``(n, 4)`` array of
``(x, y, z, m)`` records (the j-particle record of the appendix driver:
three coordinates and a mass).

Draw order (part of the recipe, so any reimplementation reproduces it):

* radii: ``n`` uniforms, then the directions: ``n`` uniforms for
  ``cos(theta)`` and ``n`` uniforms for ``phi``;
* masses (log-normal sets only): ``n`` standard normals after the
  positions.
"""

from __future__ import annotations

import math

import numpy as np

__all__ = [
    "plummer",
    "hernquist",
    "ensemble_sizes",
    "ensemble",
    "adjoint_weights",
    "sample_rows",
    "plummer_eps",
    "plummer_velocities",
    "interaction_lists",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _open_uniform(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform draws on the open interval (0, 1); exact zeros are redrawn."""
    u = rng.random(n)
    while True:
        bad = u == 0.0
        if not bad.any():
            return u
        u[bad] = rng.random(int(bad.sum()))


def _directions(rng: np.random.Generator, r: np.ndarray) -> np.ndarray:
    n = r.shape[0]
    cos_t = 2.0 * rng.random(n) - 1.0
    phi = 2.0 * math.pi * rng.random(n)
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    out = np.empty((n, 3), dtype=np.float64)
    out[:, 0] = r * sin_t * np.cos(phi)
    out[:, 1] = r * sin_t * np.sin(phi)
    out[:, 2] = r * cos_t
    return out


def _pack(xyz: np.ndarray, m: np.ndarray) -> np.ndarray:
    rec = np.empty((xyz.shape[0], 4), dtype=np.float32)
    rec[:, :3] = xyz.astype(np.float32)
    rec[:, 3] = np.asarray(m, dtype=np.float64).astype(np.float32)
    return rec


def plummer(n: int, seed: int, total_mass: float = 1.0) -> np.ndarray:
    """Equal-mass Plummer sphere, scale radius 1, no truncation.

    Radii invert the cumulative mass M(<r) = r^3 / (1 + r^2)^(3/2):
    r = (X^(-2/3) - 1)^(-1/2) with X uniform on (0, 1).
    """
    if n < 0:
        raise ValueError("n must be >= 0")
    rng = _rng(seed)
    x = _open_uniform(rng, n)
    r = 1.0 / np.sqrt(np.power(x, -2.0 / 3.0) - 1.0)
    xyz = _directions(rng, r)
    m = np.full(n, total_mass / max(n, 1), dtype=np.float64)
    return _pack(xyz, m)


def hernquist(n: int, seed: int, r_max: float = 100.0, lognormal_sigma: float | None = 1.0) -> np.ndarray:
    """Hernquist sphere, scale radius 1, truncated at ``r_max``.

    Cumulative mass M(<r) = r^2 / (1 + r)^2; draw X uniform on
    (0, M(r_max)) and invert: r = sqrt(X) / (1 - sqrt(X)).
    Masses are log-normal, m = exp(Z) with Z ~ N(0, sigma^2), normalised to
    total mass 1 in FP64 before the FP32 cast; ``lognormal_sigma=None``
    gives equal masses 1/n.
    """
    rng = _rng(seed)
    m_max = r_max * r_max / ((1.0 + r_max) * (1.0 + r_max))
    x = _open_uniform(rng, n) * m_max
    sx = np.sqrt(x)
    r = sx / (1.0 - sx)
    xyz = _directions(rng, r)
    if lognormal_sigma is None:
        m = np.full(n, 1.0 / max(n, 1))
    else:
        m = np.exp(lognormal_sigma * rng.standard_normal(n))
        m = m / m.sum()
    return _pack(xyz, m)


def plummer_eps(n: int) -> float:
    """Softening eps = 4 / N^(1/3) used for the scaling runs."""
    return 4.0 / float(n) ** (1.0 / 3.0)


def ensemble_sizes(n_clusters: int, seed: int, n_lo: int = 256, n_hi: int = 16384) -> np.ndarray:
    """Cluster sizes log-uniform on [n_lo, n_hi], rounded to integers."""
    rng = _rng(seed)
    u = rng.random(n_clusters)
    n = np.rint(np.exp(math.log(n_lo) + u * (math.log(n_hi) - math.log(n_lo))))
    return n.astype(np.int64)


def ensemble(n_clusters: int, seed: int, n_lo: int = 256, n_hi: int = 16384):
    """Independent Plummer clusters of uneven size, concatenated.

    Returns ``(records, offsets, eps2)``: FP32 ``(sum N_c, 4)`` records,
    int64 ``offsets`` of length ``n_clusters + 1`` and FP32 per-cluster
    ``eps2 = (4 / N_c^(1/3))^2``. Cluster ``c`` uses seed ``seed + 1 + c``.
    """
    sizes = ensemble_sizes(n_clusters, seed, n_lo, n_hi)
    offsets = np.zeros(n_clusters + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    rec = np.empty((int(offsets[-1]), 4), dtype=np.float32)
    eps2 = np.empty(n_clusters, dtype=np.float32)
    for c in range(n_clusters):
        rec[offsets[c]:offsets[c + 1]] = plummer(int(sizes[c]), seed + 1 + c)
        eps2[c] = np.float32(plummer_eps(int(sizes[c])) ** 2)
    return rec, offsets, eps2


def adjoint_weights(n: int, seed: int) -> np.ndarray:
    """Loss weights w_i ~ N(0, I_3) as FP32 ``(n, 3)``."""
    rng = _rng(seed)
    return rng.standard_normal((n, 3)).astype(np.float32)


def sample_rows(n: int, k: int, seed: int) -> np.ndarray:
    """``k`` distinct row indices out of ``n`` (sorted int64), seeded."""
    rng = _rng(seed)
    k = min(k, n)
    return np.sort(rng.choice(n, size=k, replace=False)).astype(np.int64)


def plummer_velocities(n: int, seed: int, scale: float = 0.5) -> np.ndarray:
    """Seeded isotropic Gaussian velocities as FP32 ``(n, 4)`` records (v, 0).

    A stand-in with the order of magnitude of a virialised Plummer sphere
    (sigma ~ 0.5 in units G = M = a = 1); the jerk is defined for any
    velocities, so no distribution function is sampled.
    """
    rng = _rng(seed)
    v = scale * rng.standard_normal((n, 3))
    out = np.zeros((n, 4), dtype=np.float32)
    out[:, :3] = v.astype(np.float32)
    return out


def interaction_lists(n_particles: int, group_size: int, list_size: int, seed: int, n_pseudo_frac: float = 0.5):
    """A synthetic stand-in for the group / interaction-list structure a
    modified tree code hands to the O(N^2) engine.

    Particles of a Plummer sphere are ordered by their x coordinate and cut
    into consecutive groups of ``group_size``; each group gets a list of
    ``list_size`` j records: a seeded random subset of the particles plus
    "pseudo-particles" (records at random positions carrying larger masses,
    standing in for tree nodes). Returns ``(pos_i, i_offsets, lists, j_begin,
    j_count)`` with FP32 records; lists of consecutive groups are stored back
    to back. No force arithmetic happens here.
    """
    p = plummer(n_particles, seed)
    pos_i = p[np.argsort(p[:, 0], kind="stable")]
    n_groups = -(-n_particles // group_size)
    i_offsets = np.minimum(np.arange(n_groups + 1, dtype=np.int64) * group_size, n_particles)
    rng = _rng(seed + 1)
    n_pseudo = int(list_size * n_pseudo_frac)
    n_real = list_size - n_pseudo
    lists = np.empty((n_groups * list_size, 4), dtype=np.float32)
    for g in range(n_groups):
        blk = lists[g * list_size:(g + 1) * list_size]
        blk[:n_real] = pos_i[rng.choice(n_particles, size=n_real, replace=False)]
        blk[n_real:, :3] = (4.0 * rng.standard_normal((n_pseudo, 3))).astype(np.float32)
        blk[n_real:, 3] = (rng.uniform(1.0, 64.0, n_pseudo) / n_particles).astype(np.float32)
    j_begin = np.arange(n_groups, dtype=np.int64) * list_size
    j_count = np.full(n_groups, list_size, dtype=np.int64)
    return pos_i, i_offsets, lists, j_begin, j_count


def interaction_lists_indexed(n_particles: int, group_size: int, list_size: int, seed: int,
                              n_nodes: int | None = None, n_pseudo_frac: float = 0.5):
    """The same group / list structure with the lists as index arrays, as a
    tree walk produces them: one source array holds the particles (ordered
    by x, as the i-set) followed by ``n_nodes`` pseudo-particle records
    (random positions, 1-64x the particle mass; default ``n_particles //
    4``), and each group's list is ``list_size`` int32 indices into it: a
    seeded subset of the particles without repeats plus a seeded subset of
    the nodes without repeats. Returns ``(pos_i, i_offsets, src, j_index,
    j_begin, j_count)``; ``src[j_index]`` is the list records laid out in
    entry order. No force arithmetic happens here.
    """
    p = plummer(n_particles, seed)
    pos_i = p[np.argsort(p[:, 0], kind="stable")]
    n_nodes = n_particles // 4 if n_nodes is None else n_nodes
    rng = _rng(seed + 2)
    nodes = np.empty((n_nodes, 4), dtype=np.float32)
    nodes[:, :3] = (4.0 * rng.standard_normal((n_nodes, 3))).astype(np.float32)
    nodes[:, 3] = (rng.uniform(1.0, 64.0, n_nodes) / n_particles).astype(np.float32)
    src = np.concatenate([pos_i, nodes])
    n_groups = -(-n_particles // group_size)
    i_offsets = np.minimum(np.arange(n_groups + 1, dtype=np.int64) * group_size, n_particles)
    n_pseudo = min(int(list_size * n_pseudo_frac), n_nodes)
    n_real = list_size - n_pseudo
    j_index = np.empty(n_groups * list_size, dtype=np.int32)
    for g in range(n_groups):
        blk = j_index[g * list_size:(g + 1) * list_size]
        blk[:n_real] = rng.choice(n_particles, size=n_real, replace=False)
        blk[n_real:] = n_particles + rng.choice(n_nodes, size=n_pseudo, replace=False)
    j_begin = np.arange(n_groups, dtype=np.int64) * list_size
    j_count = np.full(n_groups, list_size, dtype=np.int64)
    return pos_i, i_offsets, src, j_index, j_begin, j_count
