"""Gauss-Newton iteration plans (one CUDA graph per iteration).

A plan's run must equal, bit for bit, vgicp_linearize() on the same factors,
poses and options: over several iterations at new poses, after a voxelmap is
rebuilt in place, after the options change (the graph is captured again), after
the descriptor tables grow, and with device outputs.  One plan result is also
checked against the FP64 oracle.
"""
import numpy as np
import pytest

import datagen as dg
import oracle
import paper_2109_07073_b300 as vg
from test_gpu_parity import _ragged_case
from util import err_metric

pytestmark = pytest.mark.gpu


def _same(a, b):
    for x, y in zip(a, b):
        assert np.array_equal(np.asarray(x), np.asarray(y))


def _jitter(poses, rng, it):
    return np.stack([dg.compose(P, dg.random_pose(rng, 0.5 * it, 0.05 * it)) for P in poses])


def test_plan_runs_equal_linearize():
    tg, tcov, src, scov, poses, factors = _ragged_case(seed=47)
    rng = dg.Stream(4747)
    with vg.Context() as ctx:
        hm = [ctx.build_voxelmap(p, c, 1.0) for p, c in zip(tg, tcov)]
        hf = [ctx.add_frame(p, c) for p, c in zip(src, scov)]
        f = vg.make_factors([hm[t] for t, _, _, _ in factors], [hf[s] for _, s, _, _ in factors],
                            [a for _, _, a, _ in factors], [b for _, _, _, b in factors])
        plan = ctx.plan_create(f, len(poses))
        for it in range(3):
            P = _jitter(poses, rng, it)
            _same(ctx.plan_linearize(plan, P), ctx.linearize(f, P))
        assert ctx.plan_info(plan) == (3, 1)

        # oracle on the last iteration's first non-empty factor
        H, b, cost, inl = ctx.plan_linearize(plan, P)
        k = next(i for i in range(len(factors)) if inl[i] > 0)
        t, s, pt, ps = factors[k]
        L = oracle.linearize(oracle.voxelmap(tg[t], tcov[t], 1.0), src[s], scov[s],
                             oracle.relative_pose(P[pt], P[ps]))
        assert inl[k] == L.inliers and err_metric(H[k], L.H, L.SH) <= 1e-4

        # a voxelmap rebuilt in place between iterations is read at run time
        other = ctx.add_frame(src[7], scov[7])
        ctx.build_voxelmaps([other], 1.0, maps=np.array([hm[0]], np.int64))
        _same(ctx.plan_linearize(plan, P), ctx.linearize(f, P))
        assert ctx.plan_info(plan)[1] == 1

        # new options: captured again, still equal
        ctx.set_options(chunk_points=256, linearize_variant=2)
        _same(ctx.plan_linearize(plan, P), ctx.linearize(f, P))
        assert ctx.plan_info(plan)[1] == 2
        ctx.set_options(chunk_points=2048, linearize_variant=0)

        # descriptor tables grow (their device address changes): captured again
        extra = [ctx.add_frame(src[1], scov[1]) for _ in range(300)]
        _same(ctx.plan_linearize(plan, P), ctx.linearize(f, P))
        assert ctx.plan_info(plan)[1] == 3

        # a released handle makes the run fail cleanly
        ctx.release(hf[3])
        with pytest.raises(vg.VgicpError) as e:
            ctx.plan_linearize(plan, P)
        assert e.value.status == 3
        ctx.plan_destroy(plan)
        for h in hm + [h for i, h in enumerate(hf) if i != 3] + extra + [other]:
            ctx.release(h)


def test_plan_device_outputs():
    import torch
    tg, tcov, src, scov, poses, factors = _ragged_case(seed=48)
    stream = torch.cuda.Stream()
    with vg.Context(stream=stream) as ctx:
        hm = [ctx.build_voxelmap(p, c, 1.0) for p, c in zip(tg, tcov)]
        hf = [ctx.add_frame(p, c) for p, c in zip(src, scov)]
        f = vg.make_factors([hm[t] for t, _, _, _ in factors], [hf[s] for _, s, _, _ in factors],
                            [a for _, _, a, _ in factors], [b for _, _, _, b in factors])
        n = len(factors)
        out = (torch.zeros((n, 12, 12), dtype=torch.float64, device="cuda"),
               torch.zeros((n, 12), dtype=torch.float64, device="cuda"),
               torch.zeros(n, dtype=torch.float64, device="cuda"), torch.zeros(n, dtype=torch.int64, device="cuda"))
        plan = ctx.plan_create(f, len(poses))
        for _ in range(4):
            ctx.plan_linearize(plan, poses, out=out)
        stream.synchronize()
        _same([x.cpu().numpy() for x in out], ctx.linearize(f, poses))
        ctx.plan_destroy(plan)
        for h in hm + hf:
            ctx.release(h)


def test_plan_rejects_bad_arguments():
    with vg.Context() as ctx:
        with pytest.raises(vg.VgicpError):
            ctx.plan_create(vg.make_factors([0], [0], [0], [5]), 2)       # pose index out of range
        empty = ctx.plan_create(vg.make_factors([], [], [], []), 0)
        ctx.plan_linearize(empty, np.zeros((0, 3, 4)))
        ctx.plan_destroy(empty)
