"""Parity at the benchmark's full size and launch configuration.

The paper-scale graph (500 frames x 20,000 points, 1 m voxels, all factors
with overlap >= 0.05) runs through the same calls bench.py times, with the
autotuned batched kernel; sampled outputs are recomputed one by one by the FP64
oracle: overlap-matrix rows (bit-exact), the factor set they imply, and
sampled factors' cost / H / b for both the batched float32 and the plain
float64 path.  The per-factor errors of both paths (the precision split) are
written to $VGICP_REPORT_DIR/precision_paper_scale.json when that variable names a folder.
"""
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

THRESH = 0.05
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def graph():
    g = dg.graph_workload()
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        covs = list(ex.map(oracle.covariances, g.points))
    return g, covs


def test_paper_scale_graph_sampled_parity(graph):
    import torch
    g, covs = graph
    n = len(g.points)
    stream = torch.cuda.Stream()
    with vg.Context(stream=stream) as ctx:
        frames = np.array([ctx.add_frame(p, c) for p, c in zip(g.points, covs)], np.int64)
        maps = ctx.build_voxelmaps(frames, 1.0)
        counts = ctx.overlap_matrix(frames, maps, g.poses, g.poses)
        rng = dg.Stream(2024)
        rows = rng.choose(n, 6)
        with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
            vms = list(ex.map(lambda i: oracle.voxelmap(g.points[i], covs[i], 1.0), range(n)))

            def row(s):
                return [oracle.overlap_count(vms[t], g.points[s], oracle.relative_pose(g.poses[t], g.poses[s]))
                        for t in range(n)]
            ref_rows = list(ex.map(row, rows))
        for s, ref in zip(rows, ref_rows):
            assert np.array_equal(counts[s], np.array(ref)), s
        frac = counts / np.array([p.shape[0] for p in g.points])[:, None]
        tgt, src = [], []
        for j in range(n):
            for i in range(j):
                if frac[j, i] >= THRESH:
                    tgt.append(i)
                    src.append(j)
        assert 3600 <= len(tgt) <= 8000
        factors = vg.make_factors(maps[tgt], frames[src], tgt, src)
        best, _ = ctx.autotune(factors, g.poses, reps=1)
        H, b, cost, inl = ctx.linearize(factors, g.poses)
        ctx.set_options(precision=vg.VGICP_PREC_F64)
        pick = rng.choose(len(tgt), 24)
        sub = factors[pick]
        H64, b64, c64, i64 = ctx.linearize(sub, g.poses)
        ctx.set_options(precision=vg.VGICP_PREC_F32_COMP)
        Hc, bc, cc, ic = ctx.linearize(sub, g.poses)
        ctx.set_options(precision=vg.VGICP_PREC_F32)
        report = {"factors": int(len(tgt)), "autotuned": {"variant": int(best.linearize_variant),
                                                         "chunk_points": int(best.chunk_points)},
                  "f32": {"H": [], "b": [], "cost": []}, "f64": {"H": [], "b": [], "cost": []},
                  "f32_comp": {"H": [], "b": [], "cost": []}}

        def ref(k):
            f = pick[k]
            return oracle.linearize(vms[tgt[f]], g.points[src[f]], covs[src[f]],
                                    oracle.relative_pose(g.poses[tgt[f]], g.poses[src[f]]))
        with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
            refs = list(ex.map(ref, range(len(pick))))
        for k, L in enumerate(refs):
            f = pick[k]
            assert inl[f] == L.inliers and i64[k] == L.inliers and ic[k] == L.inliers
            e32 = (err_metric(H[f], L.H, L.SH), err_metric(b[f], L.b, L.Sb), abs(cost[f] - L.cost) / L.Scost)
            e64 = (err_metric(H64[k], L.H, L.SH), err_metric(b64[k], L.b, L.Sb), abs(c64[k] - L.cost) / L.Scost)
            for name, v in zip(("H", "b", "cost"), e32):
                report["f32"][name].append(v)
            ec = (err_metric(Hc[k], L.H, L.SH), err_metric(bc[k], L.b, L.Sb), abs(cc[k] - L.cost) / L.Scost)
            for name, v in zip(("H", "b", "cost"), e64):
                report["f64"][name].append(v)
            for name, v in zip(("H", "b", "cost"), ec):
                report["f32_comp"][name].append(v)
            assert max(e32) <= 1e-4, (k, e32)
            assert max(e64) <= 1e-5, (k, e64)
            assert max(ec) <= 1e-4, (k, ec)
        for path in ("f32", "f64", "f32_comp"):
            for name in ("H", "b", "cost"):
                v = np.array(report[path][name])
                report[path][name] = {"max": float(v.max()), "p99": float(np.percentile(v, 99)),
                                      "median": float(np.median(v))}
        out = os.environ.get("VGICP_REPORT_DIR", "")
        if os.path.isdir(out):
            with open(os.path.join(out, "precision_paper_scale.json"), "w") as fh:
                json.dump(report, fh, indent=1)
        for h in list(frames) + list(maps):
            ctx.release(int(h))
