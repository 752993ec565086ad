"""Error evaluation and the Levenberg-Marquardt loop on the GPU.

- vgicp_evaluate's costs equal vgicp_linearize's cost output bit for bit (same
  chunks, order and kernel variant) and the FP64 oracle's within tolerance;
- one damped Gauss-Newton step from the GPU's factor blocks matches the step the
  oracle's dense solve takes from the oracle's own blocks;
- vgicp_optimize lowers the summed cost monotonically and brings the relative
  poses of a perturbed 16-frame stretch of the urban loop closer to the truth.
"""
import numpy as np
import pytest

import datagen as dg
import oracle
import paper_2109_07073_b300 as vg
from util import err_metric

pytestmark = pytest.mark.gpu

N_FRAMES = 16


@pytest.fixture(scope="module")
def stretch():
    g = dg.graph_workload(n_frames=500, n_points=8000, frame_ids=range(N_FRAMES))
    pts = g.points[:N_FRAMES]
    covs = [oracle.covariances(p) for p in pts]
    poses, gt = g.poses[:N_FRAMES].copy(), g.poses_gt[:N_FRAMES].copy()
    return pts, covs, poses, gt


def _setup(ctx, pts, covs, poses):
    fr = np.array([ctx.add_frame(p, c) for p, c in zip(pts, covs)], np.int64)
    maps = ctx.build_voxelmaps(fr, 1.0)
    counts = ctx.overlap_matrix(fr, maps, poses, poses)
    frac = counts / np.array([p.shape[0] for p in pts])[:, None]
    tgt, src = [], []
    for j in range(len(pts)):
        for i in range(j):
            if frac[j, i] >= 0.05:
                tgt.append(i)
                src.append(j)
    return fr, maps, vg.make_factors(maps[tgt], fr[src], tgt, src), np.array(tgt), np.array(src)


def _rel_errors(P, gt):
    rot, tr = [], []
    for i in range(len(P) - 1):
        def rel(T, k):
            A = np.vstack([T[k], [0, 0, 0, 1]])
            B = np.vstack([T[k + 1], [0, 0, 0, 1]])
            return np.linalg.inv(A) @ B
        E = np.linalg.inv(rel(gt, i)) @ rel(P, i)
        rot.append(np.degrees(np.arccos(np.clip((np.trace(E[:3, :3]) - 1) / 2, -1, 1))))
        tr.append(np.linalg.norm(E[:3, 3]))
    return float(np.mean(rot)), float(np.mean(tr))


@pytest.mark.parametrize("prec", [vg.VGICP_PREC_F32, vg.VGICP_PREC_F32_COMP])
@pytest.mark.parametrize("variant", [0, 2, 4, 6])
def test_evaluate_equals_linearize_cost(stretch, prec, variant):
    pts, covs, poses, _ = stretch
    with vg.Context(precision=prec, linearize_variant=variant) as ctx:
        fr, maps, f, tgt, src = _setup(ctx, pts, covs, poses)
        H, b, cost, inl = ctx.linearize(f, poses)
        c2, i2 = ctx.evaluate(f, poses)
        assert np.array_equal(cost, c2) and np.array_equal(inl, i2)
        if variant == 0:
            vms = {t: oracle.voxelmap(pts[t], covs[t], 1.0) for t in set(tgt.tolist())}
            for k in range(0, len(f), max(1, len(f) // 6)):
                L = oracle.linearize(vms[tgt[k]], pts[src[k]], covs[src[k]],
                                     oracle.relative_pose(poses[tgt[k]], poses[src[k]]))
                assert i2[k] == L.inliers
                assert abs(c2[k] - L.cost) <= 1e-4 * L.Scost


def test_first_step_matches_oracle(stretch):
    pts, covs, poses, _ = stretch
    with vg.Context() as ctx:
        fr, maps, f, tgt, src = _setup(ctx, pts, covs, poses)
        H, b, cost, inl = ctx.linearize(f, poses)
        pairs = np.stack([tgt, src], 1)
        vms = {t: oracle.voxelmap(pts[t], covs[t], 1.0) for t in set(tgt.tolist())}
        Ls = [oracle.linearize(vms[t], pts[s], covs[s], oracle.relative_pose(poses[t], poses[s]))
              for t, s in zip(tgt, src)]
        for k, L in enumerate(Ls):
            assert err_metric(H[k], L.H, L.SH) <= 1e-4
        d_ref, dec_ref = oracle.gn_step(pairs, np.stack([L.H for L in Ls]), np.stack([L.b for L in Ls]),
                                        N_FRAMES, anchor=0, lam=1e-4)
        d_got, dec_got = vg.vgicp_solve_step(pairs, H, b, N_FRAMES, 0, 1e-4)
        assert np.linalg.norm(d_got - d_ref) <= 1e-3 * np.linalg.norm(d_ref)
        assert dec_got == pytest.approx(dec_ref, rel=1e-3)
        assert dec_ref > 0


def test_optimize_reduces_cost_and_pose_error(stretch):
    pts, covs, poses, gt = stretch
    with vg.Context() as ctx:
        fr, maps, f, tgt, src = _setup(ctx, pts, covs, poses)
        out, rep = ctx.optimize(f, poses, max_iterations=15, anchor=0)
        hist = np.array(rep.history[:rep.n_history])
        assert rep.accepted >= 2 and np.all(np.diff(hist) < 0)
        assert rep.final_cost == hist[-1] and rep.initial_cost == hist[0]
        assert rep.final_cost < 0.9 * rep.initial_cost
        assert np.array_equal(out[0], poses[0])                     # the anchor stays
        assert float(np.sum(ctx.evaluate(f, out)[0])) == rep.final_cost
        r0, t0 = _rel_errors(poses, gt)
        r1, t1 = _rel_errors(out, gt)
        assert r1 < 0.5 * r0 and t1 < 0.5 * t0, (r0, t0, r1, t1)


def test_optimize_with_loop_factor(stretch):
    """A ground-truth loop measurement between the stretch's ends, under the shifted
    Tukey kernel, is honoured by the optimiser together with the matching cost factors."""
    pts, covs, poses, gt = stretch
    h = lambda T: np.vstack([T, [0, 0, 0, 1]])
    rel_gt = (np.linalg.inv(h(gt[0])) @ h(gt[N_FRAMES - 1]))[:3]
    loops = vg.make_loop_factors([0], [N_FRAMES - 1], rel_gt[None], 100.0 * np.eye(6), 25.0, 0.0)
    with vg.Context() as ctx:
        fr, maps, f, tgt, src = _setup(ctx, pts, covs, poses)
        out, rep = ctx.optimize_with_loops(f, loops, poses, max_iterations=15, anchor=0)
        hist = np.array(rep.history[:rep.n_history])
        assert rep.accepted >= 2 and np.all(np.diff(hist) < 0)
        _, _, lc0 = vg.vgicp_loop_linearize(loops, poses)
        _, _, lc1 = vg.vgicp_loop_linearize(loops, out)
        assert lc1[0] < lc0[0]
        c1, _ = ctx.evaluate(f, out)
        assert float(np.sum(c1)) + lc1[0] == pytest.approx(rep.final_cost, rel=1e-12)
        err0 = np.linalg.norm(oracle.loop_residual(poses[0], poses[N_FRAMES - 1], rel_gt))
        err1 = np.linalg.norm(oracle.loop_residual(out[0], out[N_FRAMES - 1], rel_gt))
        assert err1 < err0
