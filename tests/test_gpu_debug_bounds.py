"""The bounds-checked build (CN_DEBUG_BOUNDS): every schedule index the pair
kernel reaches (the unit-to-tile lookup, tile descriptors against the i and
j arrays, each bulk copy's range, the chunk range of split tiles) and the
symmetric kernel's unit and segment indices are checked on the device; a
violation would set the device status bit kStatusBadSchedule and stop the
CTA's work (the gathering list kernel also checks every list entry it
copies against the source array). Here the batched, interaction-list,
gathering-list, dynamic-queue and split-j paths, default shapes with
j-tiles fitted to the schedule (and the compensated, adjoint, force-jerk
and banded symmetric forms) run under that build, in a separate process: no
check fires, and the results still match the FP64 oracle.
"""

import json
import os
import subprocess
import sys
import textwrap

import pytest

from conftest import ROOT
from gpu_common import torch_cuda

pytestmark = pytest.mark.gpu

SCRIPT = textwrap.dedent(r"""
    import json, sys
    import numpy as np, torch
    sys.path.insert(0, sys.argv[1])
    import oracle
    import paper_astro_ph_0703100_gb300 as cn
    from paper_astro_ph_0703100_gb300 import synth
    L = cn.load()
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = {"errors": {}, "status": []}
    def status(tag):
        torch.cuda.synchronize()
        out["status"].append([tag, cn.cn_get_device_status()])

    # ensembles: static and dynamic schedules, split-j lane groups
    rec, offs, eps2s = synth.ensemble(24, 31, n_hi=3000)
    for name, tune in [("static", {"i_per_thread": 4, "threads": 128, "j_tile": 256, "stages": 3}),
                       ("dynamic", {"i_per_thread": 2, "threads": 64, "j_tile": 128, "stages": 4, "chunk_units": 5}),
                       ("splitj", {"i_per_thread": 8, "threads": 256, "j_tile": 512, "stages": 3, "j_lanes": 8})]:
        plan = cn.BatchPlan(offs, eps2s, tune=tune)
        acc, _ = plan.run(d(rec))
        status("ensemble " + name)
        a = acc.cpu().numpy(); e = 0.0
        for c in range(0, 24, 5):
            lo, hi = int(offs[c]), int(offs[c + 1])
            ref, _ = oracle.force(rec[lo:hi], rec[lo:hi], eps2s[c], potential=False)
            e = max(e, oracle.e_max(a[lo:hi], ref))
        out["errors"]["ensemble " + name] = e
        plan.close()

    # interaction lists: empty, shared and overlapping lists, guarded (eps2 = 0) and not
    pos_i = synth.plummer(2000, 9)
    pool = np.concatenate([synth.plummer(3000, 10), pos_i])
    sizes = [1, 0, 37, 300, 128, 999, 535]
    i_off = np.zeros(len(sizes) + 1, dtype=np.int64); i_off[1:] = np.cumsum(sizes)
    jb = np.array([0, 100, 50, 3000, 10, 2000, 0], dtype=np.int64)
    jc = np.array([5000, 300, 0, 2000, 1, 2500, 5000], dtype=np.int64)
    for name, eps0 in (("lists guarded", 0.0), ("lists", 1e-3)):
        eps2 = np.full(len(sizes), 1e-3, dtype=np.float32); eps2[0] = eps0
        lp = cn.ListPlan(i_off, jb, jc, eps2)
        acc, _ = lp.run(d(pos_i), d(pool))
        status(name)
        a = acc.cpu().numpy(); e = 0.0
        for g in range(len(sizes)):
            lo, hi = i_off[g], i_off[g + 1]
            if hi == lo or jc[g] == 0: continue
            ref, _ = oracle.force(pos_i[lo:hi], pool[jb[g]:jb[g] + jc[g]], eps2[g], potential=False)
            e = max(e, oracle.e_max(a[lo:hi], ref))
        out["errors"][name] = e
        lp.close()

    # gathering lists: index arrays into particles and tree nodes (ragged
    # last j-tiles), default, dynamic and split-j shapes
    pg, ig, sg, xg, bg, cg = synth.interaction_lists_indexed(3000, 256, 700, seed=4)
    for name, tune in [("indexed", None),
                       ("indexed dynamic", {"i_per_thread": 2, "threads": 64, "j_tile": 128, "stages": 3,
                                            "chunk_units": 5}),
                       ("indexed splitj", {"i_per_thread": 8, "threads": 256, "j_tile": 256, "stages": 4,
                                           "j_lanes": 8})]:
        lp = cn.ListPlan(ig, bg, cg, 1e-3, tune=tune, j_index=xg)
        acc, _ = lp.run(d(pg), d(sg))
        status(name)
        a = acc.cpu().numpy(); e = 0.0
        for g in range(0, len(cg), 3):
            lo, hi = ig[g], ig[g + 1]
            ref, _ = oracle.force(pg[lo:hi], sg[xg[bg[g]:bg[g] + cg[g]]], 1e-3, potential=False)
            e = max(e, oracle.e_max(a[lo:hi], ref))
        out["errors"][name] = e
        lp.close()

    # single systems: split tiles with the FP64 merge, split-j, dynamic chunks
    p = synth.plummer(5000, 3); q = synth.plummer(3001, 4)
    ref, _ = oracle.force(p, q, 1e-3, potential=False)
    for name, tune in [("merge", {"i_per_thread": 8, "threads": 256, "j_tile": 128, "stages": 3}),
                       ("splitj", {"i_per_thread": 8, "threads": 256, "j_tile": 1024, "stages": 3, "j_lanes": 16}),
                       ("dynamic", {"i_per_thread": 2, "threads": 128, "j_tile": 64, "stages": 4, "chunk_units": 7})]:
        cn.cn_tune_set("f32", 5000, 3001, tune)
        acc, _ = cn.cn_force(d(p), d(q), 1e-3)
        cn.cn_tune_set("f32", 5000, 3001, None)
        status("force " + name)
        out["errors"]["force " + name] = oracle.e_max(acc.cpu().numpy(), ref)
    # default shapes with j-tiles fitted to the schedule (ragged last j-tile,
    # lane groups of 8 with the constant-stride loop), and a tiny j set
    for n_i, n_j in ((14000, 14000), (9000, 22000), (1000000, 50)):
        pi, pj = synth.plummer(n_i, n_i + 1), synth.plummer(n_j, n_j + 2)
        acc, _ = cn.cn_force(d(pi), d(pj), 1e-3)
        status("default %dx%d" % (n_i, n_j))
        rows = synth.sample_rows(n_i, 256, seed=n_i)
        ref_r, _ = oracle.force(pi, pj, 1e-3, rows=rows, potential=False)
        out["errors"]["default %dx%d" % (n_i, n_j)] = oracle.e_max(acc.cpu().numpy()[rows], ref_r)
    acc, _ = cn.cn_force_dd(d(p), d(q), 1e-3)
    status("compensated")
    out["errors"]["compensated"] = oracle.e_max(acc.cpu().numpy(), ref)
    w = synth.adjoint_weights(3001, 5)
    gp, gm = cn.cn_force_adjoint(d(q), 1e-3, d(w))
    status("adjoint")
    rp, _ = oracle.adjoint(q, 1e-3, w)
    out["errors"]["adjoint"] = oracle.e_max(gp.cpu().numpy().astype(np.float64), rp)
    v = synth.plummer_velocities(3001, 6)
    a, j, _ = cn.cn_force_jerk(d(q), d(v), d(q), d(v), 1e-3)
    status("jerk")
    ra, rj, _ = oracle.force_jerk(q, v, q, v, 1e-3, potential=False)
    out["errors"]["jerk"] = oracle.e_max(j.cpu().numpy(), rj)

    # symmetric form in bands of two tile rows
    h = synth.hernquist(5000, 9)
    cn.cn_tune_set("symmetric", 5000, 5000, {"i_per_thread": 2, "threads": 64, "j_tile": 64, "stages": 3,
                                             "chunk_units": 2})
    acc, _ = cn.cn_force_symmetric(d(h), 1e-4)
    cn.cn_tune_set("symmetric", 5000, 5000, None)
    status("symmetric bands")
    ref, _ = oracle.force(h, h, 1e-4, potential=False)
    out["errors"]["symmetric bands"] = oracle.e_max(acc.cpu().numpy(), ref)
    print(json.dumps(out))
""")


def test_debug_bounds_build_runs_clean():
    torch_cuda()
    from paper_astro_ph_0703100_gb300 import _build

    lib = _build.build(debug_bounds=True)
    env = dict(os.environ, CUNBODY_LIB=lib)
    res = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], env=env, capture_output=True, text=True, timeout=900)
    assert res.returncode == 0, res.stderr[-2000:]
    out = json.loads(res.stdout.strip().splitlines()[-1])
    for tag, st in out["status"]:
        assert st == 0, f"{tag}: device status {st}"
    tol = {"adjoint": 1.5e-5, "jerk": 2e-5}
    for name, e in out["errors"].items():
        assert e <= tol.get(name, 1e-5), f"{name}: E_max {e:.3e}"
