"""The linearisation kernels' own voxel association, point by point, against the oracle.

Sec. III-A associates each transformed source point with the target voxel that
contains it; the voxel coordinate is the float64 floor of x / r (x = T_BA p by
the fixed fma chain).  The float32 linearisation decides that floor with its own
split-translation code and proven margins, the float32-pair path with its pair
transform, the float64 path with the literal definition, and the shared-memory
variant probes a compact table instead of the global hash.  Here every one of
those paths records the voxel coordinate and the hit of every point it visits
(vgicp_linearize_correspondences: the recording instantiation of the same
kernels), and the record must equal the oracle's correspondences bit for bit on
clouds whose points lie exactly on voxel faces and corners, under poses that
keep them there (identity, whole-voxel shifts, a 1,000-voxel shift) and under
rotations with large translations, at r = 1, 0.5 and 0.3.  The same calls'
H, b and cost must equal vgicp_linearize()'s bit for bit and the oracle's within
err(X) <= 1e-4 (float32 paths) / 1e-5 (float64 path), with identical inliers.
"""
import numpy as np
import pytest

import datagen as dg
import oracle
import paper_2109_07073_b300 as vg
from util import err_metric

pytestmark = pytest.mark.gpu

TOL = {vg.VGICP_PREC_F32: 1e-4, vg.VGICP_PREC_F64: 1e-5, vg.VGICP_PREC_F32_COMP: 1e-4}
I64_MIN = np.iinfo(np.int64).min

# (precision, kernel variant, exact culling): every float32 variant with and
# without culling, the pair transform on each kernel family, the float64 path
CONFIGS = ([(vg.VGICP_PREC_F32, v, c) for v in range(7) for c in (1, 0)] +
           [(vg.VGICP_PREC_F32_COMP, v, 1) for v in (0, 2, 4, 6)] + [(vg.VGICP_PREC_F64, 0, 1)])


def _face_cloud(seed, n, r):
    """Points on the half-voxel lattice (faces, edges and corners of voxels at
    identity), plus points out of the voxel-coordinate range and not finite."""
    rng = dg.Stream(seed)
    pts = (np.round(rng.uniform(3 * n, -20, 20)) * r * 0.5).reshape(-1, 3)
    odd = np.array([[2 ** 20 * r, 0, 0], [-(2 ** 20) * r - 1, 0, 0], [np.nan, 1, 1], [np.inf, 0, 0],
                    [0, 0, -np.inf], [(2 ** 20 - 1) * r, 2 * r, 0]])
    return np.concatenate([pts, odd]).astype(np.float32)


def _poses(r):
    rng = dg.Stream(31)
    out = [dg.identity_pose()]
    T = dg.identity_pose()
    T[:, 3] = [r * 3, -r * 2, r]                 # whole voxels: faces stay on faces
    out.append(T)
    T = dg.identity_pose()
    T[:, 3] = [r * 1000, -r * 2000, r * 777]     # large split translation, faces on faces
    out.append(T)
    out.append(dg.random_pose(rng, 60, 3.0))
    T = dg.random_pose(rng, 180, 1.0)
    T[:, 3] += [512.0, -300.25, 40.5]            # large translation with rotation
    out.append(T)
    T = dg.identity_pose()
    T[:, 3] = [0.5 * r, 0.25 * r, -1.5 * r]      # half-voxel shift: lattice points onto faces
    out.append(T)
    return out


@pytest.fixture(scope="module")
def case():
    w = dg.single_factor_workload()
    cb = oracle.covariances(w.points_target)
    ca = oracle.covariances(w.points_source)
    return w, cb, ca


def _batch(w, ca, r):
    """Factors (source cloud, pose) of one batch: the workload's source and a face
    cloud, each under every pose; pose 0 is the target's (identity), so the
    relative pose of factor i is exactly poses[i + 1]."""
    face = _face_cloud(5, 3000, r)
    unit = np.tile(np.array([1, 0, 0, 1, 0, 1], np.float32), (face.shape[0], 1))
    clouds = [(w.points_source, ca), (face, unit)]
    rows = [(c, T) for c in range(len(clouds)) for T in _poses(r)]
    return clouds, rows


def _run(prec, variant, cull, w, cb, clouds, rows, r, neighbors=1):
    with vg.Context(precision=prec, linearize_variant=variant, linearize_cull=cull, neighbors=neighbors) as ctx:
        hm = ctx.build_voxelmap(w.points_target, cb, r)
        hf = [ctx.add_frame(p, c) for p, c in clouds]
        poses = np.stack([dg.identity_pose()] + [T for _, T in rows])
        f = vg.make_factors([hm] * len(rows), [hf[c] for c, _ in rows], [0] * len(rows),
                            list(range(1, len(rows) + 1)))
        rec = ctx.linearize_correspondences(f, poses)
        plain = ctx.linearize(f, poses)
        return rec, plain


@pytest.mark.parametrize("r", [1.0, 0.5, 0.3])
def test_linearize_correspondences_bit_exact(case, r):
    w, cb, ca = case
    vm = oracle.voxelmap(w.points_target, cb, r)
    clouds, rows = _batch(w, ca, r)
    ref = [oracle.correspondences(vm, clouds[c][0], T) for c, T in rows]
    lin = [oracle.linearize(vm, clouds[c][0], clouds[c][1], T) for c, T in rows]
    for prec, variant, cull in CONFIGS:
        (H, b, cost, inl, keys, state), (H0, b0, c0, i0) = _run(prec, variant, cull, w, cb, clouds, rows, r)
        tag = (prec, variant, cull, r)
        # the recording run is the plain run
        assert np.array_equal(H, H0) and np.array_equal(b, b0) and np.array_equal(cost, c0), tag
        assert np.array_equal(inl, i0), tag
        off = 0
        for q, (c, T) in enumerate(rows):
            n = clouds[c][0].shape[0]
            k, s = keys[off:off + n], state[off:off + n]
            corr, rkeys = ref[q]
            off += n
            seen = s >= 0
            if not cull:
                assert seen.all(), tag
            # every visited point: the kernel's voxel coordinate and hit are the oracle's
            assert np.array_equal(k[seen], rkeys[seen]), (tag, q, np.flatnonzero((k != rkeys).any(1) & seen)[:5])
            assert np.array_equal(s[seen] == 1, corr[seen] >= 0), (tag, q)
            assert np.all(s[seen] <= 1), tag
            # a skipped point provably has no voxel
            assert np.all(corr[~seen] < 0) and np.all(k[~seen] == I64_MIN), (tag, q)
            assert inl[q] == int((corr >= 0).sum()) == lin[q].inliers, (tag, q)
            tol = TOL[prec]
            assert err_metric(H[q], lin[q].H, lin[q].SH) <= tol, (tag, q)
            assert err_metric(b[q], lin[q].b, lin[q].Sb) <= tol, (tag, q)
            assert err_metric([cost[q]], [lin[q].cost], [lin[q].Scost]) <= tol, (tag, q)
        assert off == keys.shape[0]


def _neighbour_offsets():
    """The documented neighbour order: own voxel, the six face neighbours
    (-x, +x, -y, +y, -z, +z), then the other 20 voxels of the 3x3x3 block in
    lexicographic (x, y, z) order."""
    face = [(0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
    rest = [(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1) if abs(a) + abs(b) + abs(c) > 1]
    return face + rest


@pytest.mark.parametrize("nb", [7, 27])
def test_linearize_neighbour_association_record(case, nb):
    """DIRECT7 / DIRECT27: the recorded bit o is set exactly when the oracle's
    voxelmap holds the voxel at neighbour offset o of the point's own voxel."""
    w, cb, ca = case
    r = 0.5
    vm = oracle.voxelmap(w.points_target, cb, r)
    have = {tuple(k) for k in vm.keys.tolist()}
    offs = _neighbour_offsets()[:nb]
    clouds, rows = _batch(w, ca, r)
    for prec in (vg.VGICP_PREC_F32, vg.VGICP_PREC_F64):
        (H, b, cost, inl, keys, state), _ = _run(prec, 0, 1, w, cb, clouds, rows, r, neighbors=nb)
        off = 0
        for q, (c, T) in enumerate(rows):
            n = clouds[c][0].shape[0]
            k, s = keys[off:off + n], state[off:off + n]
            off += n
            _, rkeys = oracle.correspondences(vm, clouds[c][0], T)
            valid = rkeys[:, 0] != I64_MIN
            assert np.all(s >= 0), (prec, q)       # neighbour association is never culled
            assert np.array_equal(k, rkeys), (prec, q)
            lim = 2 ** 20
            for i in np.flatnonzero(valid):
                bits = 0
                for o, d in enumerate(offs):
                    kk = (int(k[i, 0]) + d[0], int(k[i, 1]) + d[1], int(k[i, 2]) + d[2])
                    if all(-lim <= x < lim for x in kk) and kk in have:
                        bits |= 1 << o
                assert s[i] == bits, (prec, q, i)
            assert np.all(s[~valid] == 0)
            ref = oracle.linearize(vm, clouds[c][0], clouds[c][1], T, neighbors=nb)
            assert inl[q] == ref.inliers == sum(bin(int(x)).count("1") for x in s), (prec, q)
