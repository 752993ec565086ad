"""Multi-process plumbing: one process per GPU, one workload split among them.

Factors, overlap pairs and voxelmaps are independent units (Sec. III-D: every
factor's cost evaluation is issued to the GPU on its own, and the optimiser
only collects the results).  One batch is split by target voxelmap: each rank
owns a set of targets, builds only their voxelmaps, computes the overlap-matrix
columns of those targets (every source against its targets) and linearises the
factors whose target it owns.  The sources are replicated on every rank (each
rank copies the frames it needs into its own HBM; no peer loads).  The one
exchange step is the gather of the results to rank 0, where the host solver
runs: per factor 91 float64 values (the 78 unique entries of the symmetric H,
b and the cost, 728 B) plus its inlier count, and per owned target one column
of overlap counts.

The partition depends only on the sizes of the work, so every rank computes the
same partition without communicating.
"""
from __future__ import annotations

import os

import numpy as np

# upper-triangle indices of a 12 x 12 matrix, row by row
_IU = np.triu_indices(12)
ROW = 78 + 12 + 1 + 1          # packed factor result: H upper, b, cost, inliers


def rank_world():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def init(backend: str = "nccl"):
    """Join the process group named by the launcher's environment (no-op for one rank)."""
    rank, world = rank_world()
    if world > 1:
        import torch.distributed as tdist
        if backend == "nccl":
            import torch
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        if not tdist.is_initialized():
            tdist.init_process_group(backend)
    return rank, world


def barrier(world: int):
    if world > 1:
        import torch.distributed as tdist
        tdist.barrier()


def max_over_ranks(x: float, world: int, device=None) -> float:
    """Largest value of x over all ranks (the slowest rank's step time)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as tdist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(units_per_rank: float, world: int, ms_per_step_max: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's step time."""
    return units_per_rank * world / (ms_per_step_max / 1e3)


# ------------------------------------------------------------- partition --

def partition_targets(target_work, world: int) -> np.ndarray:
    """Owner rank of every target: longest-processing-time assignment of the
    targets' work (largest first, ties by target index) to the least-loaded rank
    (ties to the lower rank).  Deterministic: the same on every rank."""
    w = np.asarray(target_work, dtype=np.float64)
    owner = np.zeros(w.shape[0], np.int64)
    load = np.zeros(max(1, world), np.float64)
    for t in sorted(range(w.shape[0]), key=lambda i: (-w[i], i)):
        r = int(np.argmin(load))
        owner[t] = r
        load[r] += w[t]
    return owner


def target_work(factor_targets, factor_points, target_points, source_points, n_targets: int):
    """Work of each target: its voxelmap build (its own points), the points of every
    factor that targets it (the linearisation) and one pass over all sources for
    its overlap-matrix column (an upper bound: culling removes most of it)."""
    work = np.asarray(target_points, np.float64).copy()[:n_targets]
    np.add.at(work, np.asarray(factor_targets, np.int64), np.asarray(factor_points, np.float64))
    return work + 0.05 * float(np.sum(source_points))


def shares(owner, world: int):
    """Target indices owned by each rank, in increasing order."""
    owner = np.asarray(owner)
    return [np.flatnonzero(owner == r) for r in range(world)]


def factor_share(factor_targets, owner, rank: int) -> np.ndarray:
    """Indices of the factors whose target the rank owns, in factor order."""
    return np.flatnonzero(np.asarray(owner)[np.asarray(factor_targets, np.int64)] == rank)


# ---------------------------------------------------------------- gather --

def pack_factor_results(H, b, cost, inliers):
    """(m, 92) float64 rows: H's upper triangle, b, cost, inliers (exact below 2^53)."""
    import torch
    m = H.shape[0]
    if m == 0:
        return torch.zeros((0, ROW), dtype=torch.float64, device=H.device)
    Hm = H.reshape(m, 12, 12)
    iu = torch.as_tensor(np.stack(_IU), device=H.device)
    return torch.cat([Hm[:, iu[0], iu[1]], b.reshape(m, 12), cost.reshape(m, 1),
                      inliers.reshape(m, 1).to(torch.float64)], dim=1)


def unpack_factor_results(rows):
    """Inverse of pack_factor_results: (H (m,12,12), b (m,12), cost (m,), inliers (m,))."""
    import torch
    m = rows.shape[0]
    H = torch.zeros((m, 12, 12), dtype=torch.float64, device=rows.device)
    iu = torch.as_tensor(np.stack(_IU), device=rows.device)
    H[:, iu[0], iu[1]] = rows[:, :78]
    H[:, iu[1], iu[0]] = rows[:, :78]
    return H, rows[:, 78:90].clone(), rows[:, 90].clone(), rows[:, 91].to(torch.int64)


def all_gather_rows(local, counts, world: int):
    """Rows of every rank in rank order: each rank's (counts[rank], k) tensor is
    padded to the largest share, gathered, and the padding dropped."""
    import torch
    import torch.distributed as tdist
    if world == 1:
        return local
    k = local.shape[1]
    mx = max(1, int(max(counts)))
    pad = torch.zeros((mx, k), dtype=local.dtype, device=local.device)
    pad[:local.shape[0]] = local
    bufs = [torch.empty_like(pad) for _ in range(world)]
    tdist.all_gather(bufs, pad)
    return torch.cat([bufs[r][:int(counts[r])] for r in range(world)], dim=0)


def gather_factor_results(H, b, cost, inliers, factor_ids, n_total: int, world: int):
    """Every rank's factor results (its factors factor_ids, in that order) gathered
    and put back in global factor order: (H, b, cost, inliers) of all n_total
    factors, the same on every rank."""
    import torch
    import torch.distributed as tdist
    ids = torch.as_tensor(np.asarray(factor_ids, np.int64), device=H.device)
    rows = pack_factor_results(H, b, cost, inliers)
    if world > 1:
        cnt = torch.tensor([ids.shape[0]], dtype=torch.int64, device=H.device)
        cnts = [torch.zeros_like(cnt) for _ in range(world)]
        tdist.all_gather(cnts, cnt)
        counts = [int(c.item()) for c in cnts]
        rows = all_gather_rows(rows, counts, world)
        ids = all_gather_rows(ids.reshape(-1, 1), counts, world).reshape(-1)
    full = torch.zeros((n_total, ROW), dtype=torch.float64, device=H.device)
    full[ids] = rows
    return unpack_factor_results(full)


def gather_columns(cols, col_ids, n_cols: int, world: int):
    """Column blocks of a matrix (n_rows x len(col_ids) on each rank) gathered into
    the full n_rows x n_cols matrix, the same on every rank."""
    import torch
    import torch.distributed as tdist
    ids = torch.as_tensor(np.asarray(col_ids, np.int64), device=cols.device)
    blk = cols.t().contiguous()            # one row per owned column
    if world > 1:
        cnt = torch.tensor([ids.shape[0]], dtype=torch.int64, device=cols.device)
        cnts = [torch.zeros_like(cnt) for _ in range(world)]
        tdist.all_gather(cnts, cnt)
        counts = [int(c.item()) for c in cnts]
        blk = all_gather_rows(blk, counts, world)
        ids = all_gather_rows(ids.reshape(-1, 1), counts, world).reshape(-1)
    full = torch.zeros((n_cols, cols.shape[0]), dtype=cols.dtype, device=cols.device)
    full[ids] = blk
    return full.t().contiguous()
