"""Two lanes of one context at work at once: the next batch of frames is registered
on lane 1 from page-locked host memory (a large copy, followed by enough further
frames to grow the shared descriptor tables) while lane 0 builds voxelmaps, computes
the overlap matrix and linearises the current batch.  Every batch's results equal
those of the same calls on one lane, bit for bit, and the overlap counts equal the
oracle's."""
import numpy as np
import pytest
import torch

import datagen as dg
import oracle
import paper_2109_07073_b300 as vg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch():
    ids = [40, 41, 42, 43, 44, 45]
    g = dg.graph_workload(frame_ids=ids)
    pts = [g.points[i] for i in ids]
    covs = [oracle.covariances(p) for p in pts]
    return g.poses[ids], pts, covs


def _pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()


def test_pipelined_lanes_match_one_lane(batch):
    poses, pts, covs = batch
    n = len(pts)
    P, C = _pinned(np.concatenate(pts)), _pinned(np.concatenate(covs))
    sizes = np.array([p.shape[0] for p in pts], np.int64)
    tgt = np.array([i for j in range(n) for i in range(j)])
    src = np.array([j for j in range(n) for i in range(j)])
    tiny_p = np.zeros((3, 3), np.float32)
    tiny_c = np.tile(np.array([1, 0, 0, 1, 0, 1e-3], np.float32), (3, 1))

    def finish(ctx, fr, mp):
        counts = ctx.overlap_matrix(fr, mp, poses, poses)
        out = ctx.linearize(vg.make_factors(mp[tgt], fr[src], tgt, src), poses)
        return counts, out

    with vg.Context() as ctx:
        fr = ctx.add_frames(P, C, sizes)
        ref_counts, ref = finish(ctx, fr, ctx.build_voxelmaps(fr, 1.0))
    for i in range(n):
        vm = oracle.voxelmap(pts[i], covs[i], 1.0)
        for j in (max(0, i - 1), min(n - 1, i + 1)):
            assert ref_counts[j, i] == oracle.overlap_count(vm, pts[j], oracle.relative_pose(poses[i], poses[j]))

    with vg.Context() as ctx:
        ctx.set_lane(1)
        nxt = ctx.add_frames(P, C, sizes)
        ctx.set_lane(0)
        extra = []
        for step in range(3):
            fr = nxt
            ctx.set_lane(1)
            ctx.synchronize()
            ctx.set_lane(0)
            mp = ctx.build_voxelmaps(fr, 1.0)
            ctx.set_lane(1)
            nxt = ctx.add_frames(P, C, sizes)
            # more frames than the tables hold: they grow while lane 1 still copies
            extra += [ctx.add_frame(tiny_p, tiny_c) for _ in range(150)]
            ctx.set_lane(0)
            counts, out = finish(ctx, fr, mp)
            assert np.array_equal(counts, ref_counts)
            for a, b in zip(out, ref):
                assert np.array_equal(a, b)
            ctx.release_many(np.concatenate([fr, mp]))
        ctx.set_lane(1)
        ctx.synchronize()
        ctx.release_many(np.concatenate([nxt, np.array(extra, np.int64)]))
        ctx.synchronize()
        ctx.set_lane(0)
