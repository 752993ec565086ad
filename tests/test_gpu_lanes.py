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


def test_released_index_reused_on_another_lane(batch):
    """A frame registered, built into a voxelmap and released on lane 1 while
    lane 1 is still busy with a long linearisation; lane 2 then registers a
    larger frame, which takes the released descriptor index at once, and builds
    its voxelmap.  Lane 2's writes to that index wait for lane 1's queued work,
    so both voxelmaps (and the larger frame's overlap) equal those made on one
    lane, bit for bit."""
    poses, pts, covs = batch
    small_p, small_c = pts[0][:5000], covs[0][:5000]
    big_p, big_c = pts[1], covs[1]
    with vg.Context() as ref:
        want_a = ref.export_voxelmap(ref.build_voxelmap(small_p, small_c, 1.0))
        hb = ref.add_frame(big_p, big_c)
        want_b = ref.export_voxelmap(ref.build_voxelmaps([hb], 1.0)[0])
        want_ov = ref.overlap_matrix([hb], ref.build_voxelmaps([ref.add_frame(pts[2], covs[2])], 1.0),
                                     poses[1:2], poses[2:3])
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    # device inputs are read by the lane's queued work: they stay alive until it is done
    d_small, d_big = (dev(small_p), dev(small_c)), (dev(big_p), dev(big_c))
    with vg.Context() as ctx:
        fr = ctx.add_frames(np.concatenate(pts), np.concatenate(covs), np.array([p.shape[0] for p in pts]))
        mp = ctx.build_voxelmaps(fr, 1.0)
        m2 = ctx.build_voxelmaps([ctx.add_frame(pts[2], covs[2])], 1.0)
        pairs = [(i, j) for j in range(len(pts)) for i in range(len(pts)) if i != j] * 100
        f = vg.make_factors(mp[[i for i, _ in pairs]], fr[[j for _, j in pairs]], [i for i, _ in pairs],
                            [j for _, j in pairs])
        nf = f.shape[0]
        out = (torch.empty((nf, 12, 12), dtype=torch.float64, device="cuda"),
               torch.empty((nf, 12), dtype=torch.float64, device="cuda"),
               torch.empty(nf, dtype=torch.float64, device="cuda"), torch.empty(nf, dtype=torch.int64, device="cuda"))
        torch.cuda.synchronize()
        for _ in range(3):
            ctx.set_lane(1)
            ctx.linearize(f, poses, out=out)                   # long work queued on lane 1
            ha = ctx.add_frame(*d_small)
            ma = ctx.build_voxelmaps([ha], 1.0)[0]
            ctx.release(ha)                                    # its index is free on the host at once
            ctx.set_lane(2)
            hb = ctx.add_frame(*d_big)                         # takes that index
            mb = ctx.build_voxelmaps([hb], 1.0)[0]
            ctx.synchronize()
            ctx.set_lane(1)
            ctx.synchronize()
            ctx.set_lane(0)
            for x, y in zip(ctx.export_voxelmap(int(ma)), want_a):
                assert np.array_equal(x, y)
            for x, y in zip(ctx.export_voxelmap(int(mb)), want_b):
                assert np.array_equal(x, y)
            assert np.array_equal(ctx.overlap_matrix([hb], m2, poses[1:2], poses[2:3]), want_ov)
            ctx.release_many([int(ma), int(mb), hb])
