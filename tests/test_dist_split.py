"""One batch split across ranks by target voxelmap, run as gloo ranks on the CPU.

Each rank owns the targets the partition gives it, computes the overlap-matrix
columns of those targets and the factors whose target it owns (here with the
FP64 oracle standing in for the per-rank GPU computation), and the gather puts
every result back in global order.  The gathered results must equal one
rank's computation of the whole batch bit for bit, also when a rank owns
nothing.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import datagen as dg


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _workload(n_frames, n_targets, seed):
    """n_frames small clouds at random poses; factors (target i, source j) for every
    target i < n_targets and source j != i."""
    rng = dg.Stream(seed)
    pts = [dg.sample_small_scene(rng, 300 + 150 * k) for k in range(n_frames)]
    poses = np.stack([dg.random_pose(rng, 10, 1.0) for _ in range(n_frames)])
    tgt = [i for i in range(n_targets) for j in range(n_frames) if j != i]
    src = [j for i in range(n_targets) for j in range(n_frames) if j != i]
    return pts, poses, np.array(tgt), np.array(src)


def _compute(pts, poses, tgt, src, my_targets, my_factors, n_targets):
    """Oracle results of the given targets' overlap columns and the given factors."""
    import oracle
    covs = [oracle.covariances(p) for p in pts]
    vms = {t: oracle.voxelmap(pts[t], covs[t], 1.0) for t in range(n_targets)}
    cols = np.zeros((len(pts), len(my_targets)), np.int64)
    for c, t in enumerate(my_targets):
        for s in range(len(pts)):
            cols[s, c] = oracle.overlap_count(vms[t], pts[s], oracle.relative_pose(poses[t], poses[s]))
    m = len(my_factors)
    H, b, cost, inl = np.zeros((m, 12, 12)), np.zeros((m, 12)), np.zeros(m), np.zeros(m, np.int64)
    for q, f in enumerate(my_factors):
        L = oracle.linearize(vms[tgt[f]], pts[src[f]], covs[src[f]], oracle.relative_pose(poses[tgt[f]], poses[src[f]]))
        H[q], b[q], cost[q], inl[q] = L.H, L.b, L.cost, L.inliers
    return cols, H, b, cost, inl


def _worker(rank, world, port, n_frames, n_targets, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    from paper_2109_07073_b300 import dist
    r, w = dist.init("gloo")
    pts, poses, tgt, src = _workload(n_frames, n_targets, 5)
    sizes = np.array([p.shape[0] for p in pts])
    work = dist.target_work(tgt, sizes[src], sizes, sizes, n_targets)
    owner = dist.partition_targets(work, w)
    mine = dist.shares(owner, w)[r]
    my_f = dist.factor_share(tgt, owner, r)
    cols, H, b, cost, inl = _compute(pts, poses, tgt, src, mine, my_f, n_targets)
    T = torch.from_numpy
    full_cols = dist.gather_columns(T(cols), mine, n_targets, w)
    gH, gb, gc, gi = dist.gather_factor_results(T(H), T(b), T(cost), T(inl), my_f, len(tgt), w)
    dist.barrier(w)
    import torch.distributed as tdist
    tdist.destroy_process_group()
    q.put((r, len(mine), len(my_f), full_cols.numpy(), gH.numpy(), gb.numpy(), gc.numpy(), gi.numpy()))


@pytest.mark.parametrize("world,n_frames,n_targets", [(2, 5, 5), (3, 4, 2)])
def test_split_batch_gathers_the_single_rank_result(world, n_frames, n_targets):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n_frames, n_targets, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in procs), key=lambda o: o[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    pts, poses, tgt, src = _workload(n_frames, n_targets, 5)
    ref = _compute(pts, poses, tgt, src, list(range(n_targets)), list(range(len(tgt))), n_targets)
    assert sum(o[1] for o in out) == n_targets and sum(o[2] for o in out) == len(tgt)
    if world > n_targets:
        assert any(o[1] == 0 and o[2] == 0 for o in out)      # a rank with an empty share
    for o in out:                                             # every rank holds the whole result
        assert np.array_equal(o[3], ref[0])
        for got, want in zip(o[4:], ref[1:]):
            assert np.array_equal(got, want)


def test_partition_is_balanced_and_deterministic():
    from paper_2109_07073_b300 import dist
    rng = np.random.default_rng(3)
    work = rng.uniform(1, 100, 500)
    o1, o2 = dist.partition_targets(work, 8), dist.partition_targets(work.copy(), 8)
    assert np.array_equal(o1, o2)
    loads = np.bincount(o1, weights=work, minlength=8)
    assert loads.max() - loads.min() <= work.max()            # LPT: within one item of each other
    assert sorted(np.concatenate(dist.shares(o1, 8)).tolist()) == list(range(500))
    # one rank: everything
    assert np.all(dist.partition_targets(work, 1) == 0)
    # factor shares cover each factor once
    ft = rng.integers(0, 500, 3000)
    got = np.concatenate([dist.factor_share(ft, o1, r) for r in range(8)])
    assert sorted(got.tolist()) == list(range(3000))


def test_pack_unpack_round_trip():
    import torch
    from paper_2109_07073_b300 import dist
    rng = np.random.default_rng(4)
    A = rng.normal(size=(6, 12, 12))
    H = torch.from_numpy(A + A.transpose(0, 2, 1))
    b, c = torch.from_numpy(rng.normal(size=(6, 12))), torch.from_numpy(rng.normal(size=6))
    i = torch.from_numpy(rng.integers(0, 2 ** 40, 6))
    rows = dist.pack_factor_results(H, b, c, i)
    assert rows.shape == (6, dist.ROW) and rows.shape[1] * 8 - 8 == 728
    H2, b2, c2, i2 = dist.unpack_factor_results(rows)
    assert torch.equal(H, H2) and torch.equal(b, b2) and torch.equal(c, c2) and torch.equal(i, i2)
