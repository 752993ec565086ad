"""Seeded synthetic inputs shared by the oracle tests and the CUDA path.

This module holds no arithmetic of the method itself (no voxelisation, no
correspondence search, no cost, no covariance estimation).  It only draws
random numbers, samples scene geometry, raycasts a simulated spinning LiDAR and
builds poses, so that both sides of every parity test see identical inputs.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used in its counter form:
value i of a stream with seed s is mix(s + (i + 1) * 0x9E3779B97F4A7C15).
Normal deviates use the Box-Muller transform (Box and Muller, 1958).

Workload shapes follow the paper's evaluation (Sec. IV and Fig. 1): factors of
roughly 20,000 points, more than 4,500 factors, urban scenes with planar
structure, 1 m voxels.  KITTI itself is not used; these scenes stand in for it.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

BASE_SEED = 2109070730


def config_seed(c: int) -> int:
    """Base seed of workload configuration c (1-based)."""
    return BASE_SEED + int(c)


def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


class Stream:
    """Counter-based SplitMix64 stream."""

    def __init__(self, seed: int):
        self.seed = np.uint64(int(seed) & 0xFFFFFFFFFFFFFFFF)
        self.counter = 0

    def bits(self, n: int) -> np.ndarray:
        idx = np.arange(self.counter + 1, self.counter + n + 1, dtype=np.uint64)
        self.counter += int(n)
        with np.errstate(over="ignore"):
            return _mix64(self.seed + idx * _GAMMA)

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.bits(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        return lo + (hi - lo) * u

    def normal(self, n: int, sigma: float = 1.0) -> np.ndarray:
        m = (n + 1) // 2
        u1 = 1.0 - self.uniform(m)          # (0, 1]
        u2 = self.uniform(m)
        rad = np.sqrt(-2.0 * np.log(u1))
        z = np.concatenate([rad * np.cos(2 * np.pi * u2), rad * np.sin(2 * np.pi * u2)])
        return sigma * z[:n]

    def unit_vectors(self, n: int) -> np.ndarray:
        v = self.normal(3 * n).reshape(n, 3)
        return v / np.linalg.norm(v, axis=1, keepdims=True)

    def permutation(self, n: int) -> np.ndarray:
        return np.argsort(self.uniform(n), kind="stable")

    def choose(self, n: int, k: int) -> np.ndarray:
        """k distinct indices of range(n), uniform without replacement, sorted."""
        if k >= n:
            return np.arange(n)
        return np.sort(self.permutation(n)[:k])


# --------------------------------------------------------------------------
# poses: 3x4 row-major world-from-frame, float64
# --------------------------------------------------------------------------

def hat(w) -> np.ndarray:
    return np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])


def so3_exp(w) -> np.ndarray:
    w = np.asarray(w, dtype=np.float64)
    th = float(np.linalg.norm(w))
    K = hat(w)
    if th < 1e-8:
        return np.eye(3) + K + 0.5 * K @ K
    return np.eye(3) + math.sin(th) / th * K + (1.0 - math.cos(th)) / (th * th) * K @ K


def se3_exp(xi) -> np.ndarray:
    """Exp of xi = (omega, v), rotation first; returns a 3x4 pose."""
    xi = np.asarray(xi, dtype=np.float64)
    w, v = xi[:3], xi[3:]
    th = float(np.linalg.norm(w))
    K = hat(w)
    if th < 1e-8:
        V = np.eye(3) + 0.5 * K + K @ K / 6.0
    else:
        V = (np.eye(3) + (1.0 - math.cos(th)) / th ** 2 * K
             + (th - math.sin(th)) / th ** 3 * K @ K)
    T = np.zeros((3, 4))
    T[:, :3] = so3_exp(w)
    T[:, 3] = V @ v
    return T


def compose(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    T = np.zeros((3, 4))
    T[:, :3] = A[:, :3] @ B[:, :3]
    T[:, 3] = A[:, :3] @ B[:, 3] + A[:, 3]
    return T


def identity_pose() -> np.ndarray:
    T = np.zeros((3, 4))
    T[:, :3] = np.eye(3)
    return T


def random_pose(rng: Stream, max_angle_deg: float, max_trans: float) -> np.ndarray:
    """Rotation of U[0, max] about a uniform axis; translation uniform direction, U[0, max] length."""
    axis = rng.unit_vectors(1)[0]
    ang = math.radians(rng.uniform(1, 0.0, max_angle_deg)[0])
    T = np.zeros((3, 4))
    T[:, :3] = so3_exp(axis * ang)
    T[:, 3] = rng.unit_vectors(1)[0] * rng.uniform(1, 0.0, max_trans)[0]
    return T


# --------------------------------------------------------------------------
# Workload 1: one factor between two 2,000-point frames of a small room-like scene
# --------------------------------------------------------------------------

# (fixed axis, fixed value, axis a, [a0, a1], axis b, [b0, b1])
_SMALL_SCENE = [
    (2, 0.0, 0, (-10.0, 10.0), 1, (-10.0, 10.0)),   # ground z = 0
    (0, 8.0, 1, (-10.0, 10.0), 2, (0.0, 4.0)),      # wall x = 8
    (1, 8.0, 0, (-10.0, 8.0), 2, (0.0, 4.0)),       # wall y = 8
    (1, -8.0, 0, (-10.0, 8.0), 2, (0.0, 4.0)),      # wall y = -8
]


def sample_small_scene(rng: Stream, n: int, noise: float = 0.02) -> np.ndarray:
    areas = np.array([(a1 - a0) * (b1 - b0) for (_, _, _, (a0, a1), _, (b0, b1)) in _SMALL_SCENE])
    cdf = np.cumsum(areas) / areas.sum()
    which = np.searchsorted(cdf, rng.uniform(n), side="right")
    ua, ub = rng.uniform(n), rng.uniform(n)
    pts = np.zeros((n, 3))
    for i, (fx, fv, ax, (a0, a1), bx, (b0, b1)) in enumerate(_SMALL_SCENE):
        m = which == i
        pts[m, fx] = fv
        pts[m, ax] = a0 + (a1 - a0) * ua[m]
        pts[m, bx] = b0 + (b1 - b0) * ub[m]
    pts += rng.normal(3 * n, noise).reshape(n, 3)
    return pts.astype(np.float32)


@dataclass
class SingleFactorWorkload:
    points_target: np.ndarray   # (n, 3) float32, frame B
    points_source: np.ndarray   # (n, 3) float32, frame A
    T_target: np.ndarray        # 3x4 world-from-B
    T_source: np.ndarray        # 3x4 world-from-A
    resolution: float = 1.0


def single_factor_workload(seed: int = None, n: int = 2000,
                           max_angle_deg: float = 5.0, max_trans: float = 0.5) -> SingleFactorWorkload:
    rng = Stream(config_seed(1) if seed is None else seed)
    pb = sample_small_scene(rng, n)
    pa = sample_small_scene(rng, n)
    return SingleFactorWorkload(pb, pa, identity_pose(), random_pose(rng, max_angle_deg, max_trans))


# --------------------------------------------------------------------------
# Urban loop scene: ground plane + axis-aligned boxes along a rounded-rectangle road
# --------------------------------------------------------------------------

@dataclass
class Road:
    half_x: float = 375.0
    half_y: float = 150.0
    radius: float = 50.0
    segs: list = field(default_factory=list)
    length: float = 0.0

    def __post_init__(self):
        hx, hy, r = self.half_x, self.half_y, self.radius
        # straight: ("L", start xy, direction); arc: ("A", centre, start angle), quarter turns CCW
        self.segs = [
            ("L", (-hx + r, -hy), (1.0, 0.0), 2 * (hx - r)),
            ("A", (hx - r, -hy + r), -math.pi / 2, math.pi / 2 * r),
            ("L", (hx, -hy + r), (0.0, 1.0), 2 * (hy - r)),
            ("A", (hx - r, hy - r), 0.0, math.pi / 2 * r),
            ("L", (hx - r, hy), (-1.0, 0.0), 2 * (hx - r)),
            ("A", (-hx + r, hy - r), math.pi / 2, math.pi / 2 * r),
            ("L", (-hx, hy - r), (0.0, -1.0), 2 * (hy - r)),
            ("A", (-hx + r, -hy + r), math.pi, math.pi / 2 * r),
        ]
        self.length = sum(s[3] for s in self.segs)

    def at(self, s: float):
        """(x, y, heading) at arc length s (wraps)."""
        s = s % self.length
        for kind, a, b, ln in self.segs:
            if s <= ln:
                if kind == "L":
                    return a[0] + b[0] * s, a[1] + b[1] * s, math.atan2(b[1], b[0])
                ang = b + s / self.radius
                return (a[0] + self.radius * math.cos(ang), a[1] + self.radius * math.sin(ang),
                        ang + math.pi / 2)
            s -= ln
        raise AssertionError


@dataclass
class Boxes:
    lo: np.ndarray   # (m, 3)
    hi: np.ndarray   # (m, 3)


def urban_scene(rng: Stream, road: Road, n_boxes: int = 400, band: float = 60.0,
                corridor: float = 6.0) -> Boxes:
    """Axis-aligned boxes (sides and height U[5, 30] m) within `band` of the road, outside its corridor."""
    s_dense = np.arange(0.0, road.length, 1.0)
    road_xy = np.array([road.at(s)[:2] for s in s_dense])
    lo, hi = [], []
    while len(lo) < n_boxes:
        s, side, off = rng.uniform(1, 0, road.length)[0], rng.uniform(1)[0], rng.uniform(1, corridor, corridor + band)[0]
        sx, sy, sz = rng.uniform(3, 5.0, 30.0)
        x, y, hd = road.at(s)
        sign = 1.0 if side < 0.5 else -1.0
        cx = x - sign * math.sin(hd) * (off + 0.5 * sx)
        cy = y + sign * math.cos(hd) * (off + 0.5 * sy)
        h = np.array([0.5 * sx, 0.5 * sy])
        d = np.maximum(np.abs(road_xy - np.array([cx, cy])) - h, 0.0)
        if np.min(np.hypot(d[:, 0], d[:, 1])) < corridor:
            continue
        lo.append([cx - h[0], cy - h[1], 0.0])
        hi.append([cx + h[0], cy + h[1], sz])
    return Boxes(np.array(lo), np.array(hi))


@dataclass
class Lidar:
    rings: int = 64
    cols: int = 1024
    el_lo_deg: float = -24.8
    el_hi_deg: float = 2.0
    max_range: float = 100.0
    height: float = 1.73
    noise: float = 0.02

    def directions(self) -> np.ndarray:
        el = np.radians(np.linspace(self.el_lo_deg, self.el_hi_deg, self.rings))
        az = 2 * np.pi * np.arange(self.cols) / self.cols
        E, A = np.meshgrid(el, az, indexing="ij")
        return np.stack([np.cos(E) * np.cos(A), np.cos(E) * np.sin(A), np.sin(E)], -1).reshape(-1, 3)


def raycast(boxes: Boxes, pose: np.ndarray, lidar: Lidar, rng: Stream) -> np.ndarray:
    """Sensor-frame hit points (float64) of one spin from world pose `pose` (sensor origin),
    in firing order (column by column, the rings of a column together)."""
    d_s = lidar.directions()
    R, o = pose[:, :3], pose[:, 3]
    d_w = d_s @ R.T
    t_best = np.full(d_s.shape[0], np.inf)
    down = d_w[:, 2] < 0
    t_best[down] = -o[2] / d_w[down, 2]
    # boxes within reach of this sensor (2D distance to the footprint)
    dd = np.maximum(np.maximum(boxes.lo[:, :2] - o[:2], o[:2] - boxes.hi[:, :2]), 0.0)
    near = np.nonzero(np.hypot(dd[:, 0], dd[:, 1]) < lidar.max_range)[0]
    # candidate (ray, box) pairs: only the columns whose world azimuth can meet the
    # box footprint (the sensor stands outside every box, so the span is < pi)
    az_ray = np.arctan2(d_w[:, 1], d_w[:, 0])
    step = 2 * np.pi / lidar.cols
    col_az = az_ray.reshape(lidar.rings, lidar.cols)[lidar.rings // 2]
    ray_ids, box_ids = [], []
    for b in near:
        cx = np.array([boxes.lo[b, 0], boxes.hi[b, 0], boxes.hi[b, 0], boxes.lo[b, 0]]) - o[0]
        cy = np.array([boxes.lo[b, 1], boxes.lo[b, 1], boxes.hi[b, 1], boxes.hi[b, 1]]) - o[1]
        ac = math.atan2(cy.mean(), cx.mean())
        rel = np.angle(np.exp(1j * (np.arctan2(cy, cx) - ac)))
        lo_a, hi_a = ac + rel.min() - 2 * step, ac + rel.max() + 2 * step
        dc = np.angle(np.exp(1j * (col_az - lo_a)))
        cols = np.nonzero((dc >= 0) & (dc <= hi_a - lo_a))[0]
        ids = (np.arange(lidar.rings)[:, None] * lidar.cols + cols[None, :]).ravel()
        ray_ids.append(ids)
        box_ids.append(np.full(ids.size, b))
    if ray_ids:
        ray_ids = np.concatenate(ray_ids)
        box_ids = np.concatenate(box_ids)
        with np.errstate(divide="ignore", invalid="ignore"):
            inv = 1.0 / d_w[ray_ids]
            t1 = (boxes.lo[box_ids] - o) * inv
            t2 = (boxes.hi[box_ids] - o) * inv
            tmin = np.nanmax(np.minimum(t1, t2), axis=1)
            tmax = np.nanmin(np.maximum(t1, t2), axis=1)
        hit = (tmax >= tmin) & (tmin > 0.0)
        np.minimum.at(t_best, ray_ids[hit], tmin[hit])
    # firing order of a spinning LiDAR: column by column, all rings of a column together
    cm = (np.arange(lidar.rings)[None, :] * lidar.cols + np.arange(lidar.cols)[:, None]).ravel()
    t_best, d_s = t_best[cm], d_s[cm]
    ok = t_best <= lidar.max_range
    t = t_best[ok] + rng.normal(int(ok.sum()), lidar.noise)
    return d_s[ok] * t[:, None]


@dataclass
class GraphWorkload:
    """Frames along a closed loop: sensor-frame points and perturbed world poses."""
    points: list            # list of (n_i, 3) float32
    poses: np.ndarray       # (F, 3, 4) perturbed world-from-sensor (the optimiser's estimate)
    poses_gt: np.ndarray    # (F, 3, 4) ground truth
    resolution: float
    boxes: Boxes = None


def _graph_frame_job(args):
    boxes, pose, lidar, seed, n_points = args
    frng = Stream(seed)
    p = raycast(boxes, pose, lidar, frng)
    sel = frng.choose(p.shape[0], n_points)
    return p[sel].astype(np.float32)


def graph_workload(seed: int = None, n_frames: int = 500, spacing: float = 4.0,
                   n_points: int = 20000, n_boxes: int = 400, lidar: Lidar = None,
                   resolution: float = 1.0, rot_sigma_deg: float = 1.0,
                   trans_sigma: float = 0.1, frame_ids=None, workers: int = 0) -> GraphWorkload:
    """Frames of a 2 km closed loop through the urban scene.

    frame_ids: optional subset of frame indices to raycast (the others are left
    as None); poses are always produced for every frame.  workers > 1 raycasts in a
    spawn process pool (same frames).
    """
    lidar = lidar or Lidar()
    rng = Stream(config_seed(2) if seed is None else seed)
    road = Road()
    boxes = urban_scene(rng, road, n_boxes)
    poses_gt = np.zeros((n_frames, 3, 4))
    poses = np.zeros((n_frames, 3, 4))
    for i in range(n_frames):
        x, y, hd = road.at(i * spacing)
        T = np.zeros((3, 4))
        T[:, :3] = so3_exp([0.0, 0.0, hd])
        T[:, 3] = [x, y, lidar.height]
        poses_gt[i] = T
        xi = np.concatenate([rng.normal(3, math.radians(rot_sigma_deg)), rng.normal(3, trans_sigma)])
        poses[i] = compose(T, se3_exp(xi))
    wanted = set(range(n_frames)) if frame_ids is None else set(int(f) for f in frame_ids)
    jobs = {i: (boxes, poses_gt[i], lidar, int(rng.seed) ^ (0x5851F42D4C957F2D * (i + 1) & 0xFFFFFFFFFFFFFFFF),
                n_points) for i in range(n_frames) if i in wanted}
    keys = sorted(jobs)
    if workers and workers > 1 and len(keys) > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as pool:
            done = dict(zip(keys, pool.map(_graph_frame_job, [jobs[k] for k in keys],
                                           chunksize=max(1, len(keys) // (4 * workers)))))
    else:
        done = {k: _graph_frame_job(jobs[k]) for k in keys}
    points = [done.get(i) for i in range(n_frames)]
    return GraphWorkload(points, poses, poses_gt, resolution, boxes)


def log_uniform_sizes(rng: Stream, n: int, lo: int = 2000, hi: int = 60000) -> np.ndarray:
    return np.floor(np.exp(rng.uniform(n, math.log(lo), math.log(hi)))).astype(np.int64)


def subsample(rng: Stream, points: np.ndarray, n: int) -> np.ndarray:
    return points[rng.choose(points.shape[0], n)]


@dataclass
class UnevenWorkload:
    """Batched factors of uneven size over a pool of target frames.

    frames[i]: full raycast of frame i (sensor frame, firing order); poses[i] its
    perturbed world pose.  Target t is frame target_frame[t], downsampled to
    target_idx[t] (indices into frames[...]), with resolution target_res[t].
    Factor f pairs target factor_target[f] with source frame factor_frame[f],
    subsampled to factor_idx[f] (indices into that frame's points).
    """
    frames: list
    poses: np.ndarray
    target_frame: np.ndarray
    target_idx: list
    target_res: np.ndarray
    factor_target: np.ndarray
    factor_frame: np.ndarray
    factor_idx: list


def _raycast_job(args):
    boxes, pose, lidar, seed = args
    return raycast(boxes, pose, lidar, Stream(seed)).astype(np.float32)


def raycast_many(boxes: Boxes, poses, lidar: Lidar, seeds, workers: int = 0) -> list:
    """Raycasts of many poses; workers > 1 uses a spawn process pool (safe next to CUDA)."""
    jobs = [(boxes, p, lidar, int(s)) for p, s in zip(poses, seeds)]
    if workers and workers > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as pool:
            return pool.map(_raycast_job, jobs, chunksize=max(1, len(jobs) // (4 * workers)))
    return [_raycast_job(j) for j in jobs]


def uneven_workload(seed: int = None, n_frames: int = 1000, spacing: float = 2.0, n_factors: int = 10000,
                    target_points: int = 20000, lo: int = 2000, hi: int = 60000, max_offset: float = 10.0,
                    resolutions=(0.5, 1.0, 2.0), n_boxes: int = 400, lidar: Lidar = None,
                    rot_sigma_deg: float = 1.0, trans_sigma: float = 0.1, workers: int = 0) -> UnevenWorkload:
    """Factors with source sizes floor(exp(U[ln lo, ln hi])), targets from a pool of
    n_frames frames (one per frame) at resolutions drawn from `resolutions`, each source a
    frame within max_offset metres (along the loop) of its target's frame, subsampled."""
    lidar = lidar or Lidar()
    rng = Stream(config_seed(3) if seed is None else seed)
    road = Road()
    boxes = urban_scene(rng, road, n_boxes)
    poses = np.zeros((n_frames, 3, 4))
    gt = np.zeros((n_frames, 3, 4))
    for i in range(n_frames):
        x, y, hd = road.at(i * spacing)
        T = np.zeros((3, 4))
        T[:, :3] = so3_exp([0.0, 0.0, hd])
        T[:, 3] = [x, y, lidar.height]
        gt[i] = T
        xi = np.concatenate([rng.normal(3, math.radians(rot_sigma_deg)), rng.normal(3, trans_sigma)])
        poses[i] = compose(T, se3_exp(xi))
    seeds = [int(rng.seed) ^ (0x5851F42D4C957F2D * (i + 1) & 0xFFFFFFFFFFFFFFFF) for i in range(n_frames)]
    frames = raycast_many(boxes, gt, lidar, seeds, workers)
    target_idx = [rng.choose(f.shape[0], target_points) for f in frames]
    target_res = np.array(resolutions)[np.floor(rng.uniform(n_frames, 0, len(resolutions))).astype(int)]
    k = int(max_offset // spacing)
    tgt = np.floor(rng.uniform(n_factors, 0, n_frames)).astype(np.int64)
    off = np.floor(rng.uniform(n_factors, 1, k + 1)).astype(np.int64) * np.where(rng.uniform(n_factors) < 0.5, -1, 1)
    src = (tgt + off) % n_frames
    sizes = log_uniform_sizes(rng, n_factors, lo, hi)
    idx = [rng.choose(frames[s].shape[0], int(n)) for s, n in zip(src, sizes)]
    return UnevenWorkload(frames, poses, np.arange(n_frames), target_idx, target_res, tgt, src, idx)
