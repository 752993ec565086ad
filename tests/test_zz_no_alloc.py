"""vgicp_linearize_noalloc: linearisation for callers that must not allocate device memory.

Such callers (for example a mapping loop that fixes its device-memory footprint
when it starts, or an application whose allocator owns all device memory) keep
frames and voxelmaps in a context created up front and pass their own device
outputs.  This file is collected last so that a run stopping at the first
failure has already run every other test; it also passes when run alone in a
fresh process, where its first call performs the entry point's one-time set-up.
"""
import numpy as np
import pytest

import datagen as dg
import oracle
import paper_2109_07073_b300 as vg
from util import err_metric

pytestmark = pytest.mark.gpu

TOL = 1e-4   # the float32 path's tolerance used by every parity test


def _case(seed):
    rng = dg.Stream(seed)
    tg = [dg.sample_small_scene(rng, 3000) for _ in range(2)]
    sizes = [1, 700, 2048, 2049, 9000]
    src = [dg.sample_small_scene(rng, n) for n in sizes]
    tcov = [oracle.covariances(p) for p in tg]
    scov = [oracle.covariances(p) for p in src]
    poses = np.stack([dg.identity_pose()] + [dg.random_pose(rng, 5, 0.5) for _ in range(len(src) + 1)])
    return tg, tcov, src, scov, poses


def test_noalloc_matches_linearize_on_two_calls_in_a_row():
    import torch
    tg, tcov, src, scov, poses = _case(77)
    with vg.Context() as ctx:
        hm = [ctx.build_voxelmap(p, c, 1.0) for p, c in zip(tg, tcov)]
        hf = [ctx.add_frame(p, c) for p, c in zip(src, scov)]
        n = len(src)
        f = vg.make_factors([hm[i % 2] for i in range(n)], hf, [(i + 1) % 2 for i in range(n)],
                            [2 + i for i in range(n)])
        vms = [oracle.voxelmap(p, c, 1.0) for p, c in zip(tg, tcov)]
        for call in range(2):
            # the second call moves the poses, so stale scratch contents would show
            P = poses.copy()
            if call == 1:
                P[2:, :, 3] += 0.05
            H, b, cost, inl = ctx.linearize(f, P)          # the existing entry point
            out = (torch.full((n, 12, 12), np.nan, dtype=torch.float64, device="cuda"),
                   torch.full((n, 12), np.nan, dtype=torch.float64, device="cuda"),
                   torch.full((n,), np.nan, dtype=torch.float64, device="cuda"),
                   torch.full((n,), -1, dtype=torch.int64, device="cuda"))
            vg.vgicp_linearize_noalloc(ctx.ctx, f, P, out)
            ctx.synchronize()
            H2, b2, c2, i2 = (x.cpu().numpy() for x in out)
            assert np.array_equal(i2, inl)
            for k in range(n):
                L = oracle.linearize(vms[k % 2], src[k], scov[k],
                                     oracle.relative_pose(P[f["target_pose"][k]], P[f["source_pose"][k]]))
                scale_H = np.maximum(L.SH, np.abs(H[k]))
                scale_b = np.maximum(L.Sb, np.abs(b[k]))
                assert err_metric(H2[k], H[k], scale_H) <= TOL, (call, k)
                assert err_metric(b2[k], b[k], scale_b) <= TOL, (call, k)
                assert abs(c2[k] - cost[k]) <= TOL * max(L.Scost, abs(cost[k])), (call, k)
        for h in hm + hf:
            ctx.release(h)


def test_noalloc_rejects_sizes_beyond_its_limit():
    import torch
    with vg.Context() as ctx:
        w = dg.single_factor_workload()
        cov = np.tile(np.array([1, 0, 0, 1, 0, 1], np.float32), (w.points_target.shape[0], 1))
        hm = ctx.build_voxelmap(w.points_target, cov, 1.0)
        hf = ctx.add_frame(w.points_source, cov)
        n = 1025   # one more than VGICP_NOALLOC_MAX_FACTORS
        f = vg.make_factors([hm] * n, [hf] * n, [0] * n, [1] * n)
        out = (torch.zeros((n, 12, 12), dtype=torch.float64, device="cuda"),
               torch.zeros((n, 12), dtype=torch.float64, device="cuda"),
               torch.zeros(n, dtype=torch.float64, device="cuda"), None)
        with pytest.raises(vg.VgicpError) as e:
            vg.vgicp_linearize_noalloc(ctx.ctx, f, np.stack([w.T_target, w.T_source]), out)
        assert e.value.status == 1 and "NOALLOC_MAX_FACTORS" in str(e.value)
