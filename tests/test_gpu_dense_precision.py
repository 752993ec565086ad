"""Precision split on dense frames: a 128-ring x 1,024-column LiDAR (131 k rays per
spin) on the urban loop, frames downsampled to 120,000 points, voxelmaps at 0.25 m.
Factors between neighbouring frames (i, i+1) and (i, i+2) are linearised by the
batched float32 path (plain and compensated transform) and the plain float64 path
and recomputed one by one by the FP64 oracle (with the oracle's own kNN
covariances).  Inlier counts are bit-exact; err(H), err(b), err(cost) stay within
1e-4 (float32 paths) and 1e-5 (float64); max / p99 / median go to
$VGICP_REPORT_DIR/precision_dense.json when that variable names a folder."""
import json
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import datagen as dg
import oracle
import paper_2109_07073_b300 as vg
from util import err_metric

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N_FRAMES = 6
RES = 0.25


def test_dense_frames_precision_split():
    cores = os.cpu_count() or 1
    g = dg.graph_workload(seed=dg.config_seed(4), n_frames=N_FRAMES, spacing=4.0, n_points=120000,
                          lidar=dg.Lidar(rings=128), resolution=RES, frame_ids=range(N_FRAMES),
                          workers=min(cores, N_FRAMES))
    pts = g.points
    assert min(p.shape[0] for p in pts) > 100000
    with ThreadPoolExecutor(max_workers=cores) as ex:
        covs = list(ex.map(oracle.covariances, pts))
    pairs = [(i, i + 1) for i in range(N_FRAMES - 1)] + [(i, i + 2) for i in range(N_FRAMES - 2)]
    tgt = np.array([t for t, _ in pairs])
    src = np.array([s for _, s in pairs])

    def ref(k):
        t, s = pairs[k]
        vm = oracle.voxelmap(pts[t], covs[t], RES)
        return oracle.linearize(vm, pts[s], covs[s], oracle.relative_pose(g.poses[t], g.poses[s]))

    with ThreadPoolExecutor(max_workers=cores) as ex:
        refs = list(ex.map(ref, range(len(pairs))))
    out = {}
    with vg.Context() as ctx:
        fr = np.array([ctx.add_frame(p, c) for p, c in zip(pts, covs)], np.int64)
        maps = ctx.build_voxelmaps(fr, RES)
        f = vg.make_factors(maps[tgt], fr[src], tgt, src)
        for name, prec in (("f32", vg.VGICP_PREC_F32), ("f32_comp", vg.VGICP_PREC_F32_COMP),
                           ("f64", vg.VGICP_PREC_F64)):
            ctx.set_options(precision=prec)
            out[name] = ctx.linearize(f, g.poses)
        ctx.set_options(precision=vg.VGICP_PREC_F32)
        for h in list(maps) + list(fr):
            ctx.release(int(h))
    tol = {"f32": 1e-4, "f32_comp": 1e-4, "f64": 1e-5}
    report = {"frames": N_FRAMES, "points_per_frame": [int(p.shape[0]) for p in pts], "resolution_m": RES,
              "factors": len(pairs)}
    for name, (H, b, cost, inl) in out.items():
        errs = {"H": [], "b": [], "cost": []}
        for k, L in enumerate(refs):
            assert inl[k] == L.inliers, (name, k)
            assert L.inliers > 1000
            e = (err_metric(H[k], L.H, L.SH), err_metric(b[k], L.b, L.Sb), abs(cost[k] - L.cost) / L.Scost)
            assert max(e) <= tol[name], (name, k, e)
            for nm, v in zip(("H", "b", "cost"), e):
                errs[nm].append(v)
        report[name] = {nm: {"max": float(np.max(v)), "p99": float(np.percentile(v, 99)),
                             "median": float(np.median(v))} for nm, v in errs.items()}
    d = os.environ.get("VGICP_REPORT_DIR", "")
    if os.path.isdir(d):
        with open(os.path.join(d, "precision_dense.json"), "w") as fh:
            json.dump(report, fh, indent=1)
