"""Python face of the plain FP64 CPU oracle (``vgicp_oracle.c``).

TEST INFRASTRUCTURE ONLY: the parity tests, the smoke check and the benchmark's
CPU-baseline leg use it.  The CUDA library never imports or links it, and this
package imports nothing of the CUDA library.  Each routine follows one passage
of Koide et al. (RA-L 2021); the C source names the passage.

Parity status: every routine here is pinned by the CPU tests (hand-worked
closed forms, brute force, finite differences, invariances, null space,
eigen-solver identities).  End-to-end KITTI accuracy (Sec. IV) is parity
unpinned and out of scope.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vgicp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64 = C.c_int64
_f64 = C.c_double


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (gcc, contraction off)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    P = lambda name, args, res=None: (setattr(getattr(lib, name), "argtypes", args),
                                       setattr(getattr(lib, name), "restype", res))
    vp = C.c_void_p
    P("oracle_relative_pose", [_f64p, _f64p, _f64p])
    P("oracle_voxel_coords", [_f32p, _i64, vp, _f64, _i64p, _i32p])
    P("oracle_voxelmap_build", [_f32p, _f32p, _i64, _f64, _i64p, _i64p, _f64p, _f64p], _i64)
    P("oracle_voxelmap_build_bruteforce", [_f32p, _f32p, _i64, _f64, _i64p, _i64p, _f64p, _f64p], _i64)
    P("oracle_lookup", [_i64p, _i64, _i64p], _i64)
    P("oracle_lookup_bruteforce", [_i64p, _i64, _i64p], _i64)
    P("oracle_correspondences", [_i64p, _i64, _f64, _f32p, _i64, _f64p, _i64p, vp])
    P("oracle_overlap_count", [_i64p, _i64, _f64, _f32p, _i64, _f64p], _i64)
    P("oracle_linearize", [_i64p, _f64p, _f64p, _i64, _f64, _f32p, _f32p, _i64, _f64p,
                           _f64p, _f64p, _f64p, _i64p, vp, vp, vp, vp])
    P("oracle_linearize_ex", [_i64p, _f64p, _f64p, vp, _i64, _f64, C.c_int, _f32p, _f32p, _i64, _f64p,
                              _f64p, _f64p, _f64p, _i64p, vp, vp, vp, vp])
    P("oracle_residuals", [_f64p, _f64p, _f32p, _f32p, _i64, _f64p, _i64p, _f64p, vp, vp])
    P("oracle_knn_bruteforce", [_f32p, _i64, C.c_int, _i64p])
    P("oracle_knn_grid", [_f32p, _i64, C.c_int, _f64, _i64p])
    P("oracle_jacobi_eig3", [_f64p, _f64p, _f64p])
    P("oracle_covariances_from_neighbors", [_f32p, _i64, C.c_int, _i64p, _f64, _f32p])
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _pts(a):
    return np.ascontiguousarray(a, dtype=np.float32).reshape(-1, 3)


def _covs(a):
    return np.ascontiguousarray(a, dtype=np.float32).reshape(-1, 6)


def _pose(T):
    return np.ascontiguousarray(np.asarray(T, dtype=np.float64).reshape(12))


# ------------------------------------------------------------------ poses --

def relative_pose(T_target, T_source) -> np.ndarray:
    """T_BA = T_B^-1 T_A (Eq. 3) as a 3x4 float64 matrix."""
    out = np.zeros(12)
    _load().oracle_relative_pose(_pose(T_target), _pose(T_source), out)
    return out.reshape(3, 4)


def voxel_coords(points, resolution: float, T=None):
    """Voxel coordinates (n, 3) int64 and validity (n,) bool of points under T."""
    p = _pts(points)
    n = p.shape[0]
    k = np.zeros((n, 3), np.int64)
    v = np.zeros(n, np.int32)
    Tp = None if T is None else _pose(T)
    _load().oracle_voxel_coords(p, n, _ptr(Tp), float(resolution), k, v)
    return k, v.astype(bool)


# ---------------------------------------------------------------- voxelmap --

@dataclass
class Voxelmap:
    """Voxels sorted by (kx, ky, kz): keys (V, 3), counts (V,), mu (V, 3), cov (V, 6)."""
    keys: np.ndarray
    counts: np.ndarray
    mu: np.ndarray
    cov: np.ndarray
    resolution: float

    @property
    def n_voxels(self) -> int:
        return int(self.keys.shape[0])


def voxelmap(points, covs, resolution: float, brute_force: bool = False) -> Voxelmap:
    """Voxelmap of a cloud in its own frame (Sec. III-A); brute_force selects the linear-list builder."""
    p, c = _pts(points), _covs(covs)
    n = p.shape[0]
    keys = np.zeros((max(n, 1), 3), np.int64)
    counts = np.zeros(max(n, 1), np.int64)
    mu = np.zeros((max(n, 1), 3))
    cov = np.zeros((max(n, 1), 6))
    fn = _load().oracle_voxelmap_build_bruteforce if brute_force else _load().oracle_voxelmap_build
    nv = fn(p, c, n, float(resolution), keys, counts, mu, cov)
    return Voxelmap(keys[:nv].copy(), counts[:nv].copy(), mu[:nv].copy(), cov[:nv].copy(), float(resolution))


def lookup(vm: Voxelmap, key, brute_force: bool = False) -> int:
    k = np.ascontiguousarray(key, dtype=np.int64).reshape(3)
    keys = np.ascontiguousarray(vm.keys).reshape(-1, 3) if vm.n_voxels else np.zeros((1, 3), np.int64)
    fn = _load().oracle_lookup_bruteforce if brute_force else _load().oracle_lookup
    return int(fn(keys, vm.n_voxels, k))


def _keys_arg(vm):
    return vm.keys if vm.n_voxels else np.zeros((1, 3), np.int64)


def correspondences(vm: Voxelmap, source_points, T_target_source):
    """(corr (n,) voxel index or -1, keys (n, 3) with INT64_MIN rows for invalid points)."""
    p = _pts(source_points)
    n = p.shape[0]
    corr = np.zeros(max(n, 1), np.int64)
    keys = np.zeros((max(n, 1), 3), np.int64)
    _load().oracle_correspondences(_keys_arg(vm), vm.n_voxels, vm.resolution, p, n,
                                   _pose(T_target_source), corr, _ptr(keys))
    return corr[:n], keys[:n]


def overlap_count(vm: Voxelmap, source_points, T_target_source) -> int:
    """Numerator of Eq. 8: points of the source that fall in a voxel of the target."""
    p = _pts(source_points)
    return int(_load().oracle_overlap_count(_keys_arg(vm), vm.n_voxels, vm.resolution, p,
                                            p.shape[0], _pose(T_target_source)))


def overlap(vm: Voxelmap, source_points, T_target_source) -> float:
    """Eq. 8: fraction of source points that fall in a voxel of the target map."""
    n = _pts(source_points).shape[0]
    if n == 0:
        raise ValueError("overlap of an empty cloud is undefined")
    return overlap_count(vm, source_points, T_target_source) / n


# -------------------------------------------------------------- linearise --

@dataclass
class Linearization:
    H: np.ndarray        # (12, 12), order [xi_B ; xi_A], xi = (omega, v)
    b: np.ndarray        # (12,)
    cost: float
    inliers: int
    SH: np.ndarray       # sums of |per-point contributions| (error-metric scale)
    Sb: np.ndarray
    Scost: float
    corr: np.ndarray     # (n,) voxel index per source point or -1


def linearize(vm: Voxelmap, source_points, source_covs, T_target_source, neighbors: int = 1,
              count_weighted: bool = False) -> Linearization:
    """Eq. 3-6 for one factor, FP64, literal 3x12 Jacobians, naive sums in point order.
    neighbors 7 / 27: every face neighbour / every voxel of the 3x3x3 block around the
    containing voxel is a correspondence too; count_weighted: each correspondence
    weighted by its voxel's point count.  inliers counts correspondences."""
    if neighbors not in (1, 7, 27):
        raise ValueError("neighbors must be 1, 7 or 27")
    p, c = _pts(source_points), _covs(source_covs)
    n = p.shape[0]
    H, b, cost = np.zeros(144), np.zeros(12), np.zeros(1)
    SH, Sb, Sc = np.zeros(144), np.zeros(12), np.zeros(1)
    inl = np.zeros(1, np.int64)
    corr = np.zeros(max(n, 1), np.int64)
    mu = vm.mu if vm.n_voxels else np.zeros((1, 3))
    cov = vm.cov if vm.n_voxels else np.zeros((1, 6))
    counts = np.ascontiguousarray(vm.counts, dtype=np.int64) if (count_weighted and vm.n_voxels) else None
    _load().oracle_linearize_ex(_keys_arg(vm), np.ascontiguousarray(mu), np.ascontiguousarray(cov), _ptr(counts),
                                vm.n_voxels, vm.resolution, int(neighbors), p, c, n, _pose(T_target_source),
                                H, b, cost, inl, _ptr(SH), _ptr(Sb), _ptr(Sc), _ptr(corr))
    return Linearization(H.reshape(12, 12), b, float(cost[0]), int(inl[0]), SH.reshape(12, 12), Sb,
                         float(Sc[0]), corr[:n])


def residuals(vm: Voxelmap, source_points, source_covs, T_target_source, corr):
    """Per-point e (n, 3), J (n, 3, 12) and Omega (n, 3, 3) under frozen correspondences."""
    p, c = _pts(source_points), _covs(source_covs)
    n = p.shape[0]
    e = np.zeros((n, 3))
    J = np.zeros((n, 3, 12))
    Om = np.zeros((n, 3, 3))
    mu = vm.mu if vm.n_voxels else np.zeros((1, 3))
    cov = vm.cov if vm.n_voxels else np.zeros((1, 6))
    _load().oracle_residuals(np.ascontiguousarray(mu), np.ascontiguousarray(cov), p, c, n,
                             _pose(T_target_source), np.ascontiguousarray(corr, dtype=np.int64),
                             e, _ptr(J), _ptr(Om))
    return e, J, Om


# ------------------------------------------------------- kNN covariances --

def knn(points, k: int = 10, brute_force: bool = False, cell: float = 1.0) -> np.ndarray:
    """Indices (n, k) of the k nearest neighbours of every point (itself included)."""
    p = _pts(points)
    n = p.shape[0]
    out = np.zeros((max(n, 1), k), np.int64)
    if brute_force:
        _load().oracle_knn_bruteforce(p, n, k, out)
    else:
        _load().oracle_knn_grid(p, n, k, float(cell), out)
    return out[:n]


def jacobi_eig3(A):
    """Eigenvalues w (3,) and eigenvectors V (columns) of a symmetric 3x3."""
    w, V = np.zeros(3), np.zeros(9)
    _load().oracle_jacobi_eig3(np.ascontiguousarray(A, dtype=np.float64).reshape(9), w, V)
    return w, V.reshape(3, 3)


def covariances(points, k: int = 10, eps: float = 1e-3, nbr=None) -> np.ndarray:
    """Per-point covariances (n, 6) float32 from k neighbours, eigenvalues (1, 1, eps) (Sec. III)."""
    p = _pts(points)
    n = p.shape[0]
    if nbr is None:
        nbr = knn(p, k)
    out = np.zeros((max(n, 1), 6), np.float32)
    _load().oracle_covariances_from_neighbors(p, n, k, np.ascontiguousarray(nbr, dtype=np.int64),
                                              float(eps), out)
    return out[:n]


# --------------------------------------------------------------------------
# Gauss-Newton step of the global optimisation (Sec. III-D): the factors'
# blocks assembled into one dense system and solved plainly.
# --------------------------------------------------------------------------

def se3_exp(xi) -> np.ndarray:
    """Exp of a twist xi = (omega, v) as a 3x4 [R | t]: Rodrigues' formula for R and
    t = V v, V = I + (1 - cos th) / th^2 [w]x + (th - sin th) / th^3 [w]x^2."""
    xi = np.asarray(xi, dtype=np.float64)
    w, v = xi[:3], xi[3:]
    th = float(np.sqrt(w @ w))
    K = np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])
    if th < 1e-8:
        A, B, Cc = 1.0, 0.5, 1.0 / 6.0
    else:
        A, B, Cc = np.sin(th) / th, (1.0 - np.cos(th)) / th**2, (th - np.sin(th)) / th**3
    R = np.eye(3) + A * K + B * (K @ K)
    V = np.eye(3) + B * K + Cc * (K @ K)
    return np.hstack([R, (V @ v)[:, None]])


def retract(poses, delta) -> np.ndarray:
    """T_p Exp(delta_p) for every pose (right perturbation)."""
    out = []
    for T, d in zip(np.asarray(poses, dtype=np.float64).reshape(-1, 3, 4), np.asarray(delta).reshape(-1, 6)):
        E = se3_exp(d)
        out.append(np.hstack([T[:, :3] @ E[:, :3], (T[:, :3] @ E[:, 3] + T[:, 3])[:, None]]))
    return np.stack(out)


def assemble(pairs, H, b, n_poses):
    """Dense global H (6n x 6n) and b (6n) from factor blocks in [xi_target ; xi_source] order."""
    n = int(n_poses)
    Hg, bg = np.zeros((6 * n, 6 * n)), np.zeros(6 * n)
    for (t, s), Hf, bf in zip(np.asarray(pairs).reshape(-1, 2), np.asarray(H).reshape(-1, 12, 12),
                              np.asarray(b).reshape(-1, 12)):
        idx = np.r_[6 * t:6 * t + 6, 6 * s:6 * s + 6]
        for i in range(12):
            bg[idx[i]] += bf[i]
            for j in range(12):
                Hg[idx[i], idx[j]] += Hf[i, j]
    return Hg, bg


def gn_step(pairs, H, b, n_poses, anchor=0, lam=0.0):
    """Damped step (H + lam D) d = -b over every pose but the anchor (d = 0 there),
    D = diag(H) floored at 1e-12 of its mean over the free variables, plus that floor;
    returns d (n, 6) and the undamped model decrease -(2 b'd + d'H d)."""
    Hg, bg = assemble(pairs, H, b, n_poses)
    free = np.array([i for i in range(6 * int(n_poses)) if i // 6 != anchor])
    A = Hg[np.ix_(free, free)].copy()
    fl = 1e-12 * max(float(np.mean(np.diag(A))), 1e-300)
    dg = np.diag(A).copy()
    A[np.diag_indices_from(A)] = dg + lam * np.maximum(dg, fl) + fl
    d = np.zeros(6 * int(n_poses))
    d[free] = np.linalg.solve(A, -bg[free])
    return d.reshape(-1, 6), float(-(2.0 * bg @ d + d @ Hg @ d))


# --------------------------------------------------------------------------
# SE(3) loop constraint with the shifted Tukey kernel (Sec. III-D, Eq. 10-11)
# --------------------------------------------------------------------------

def se3_log(T) -> np.ndarray:
    """Twist (omega, v) of a rigid transform: the principal matrix logarithm of its 4x4 form."""
    import scipy.linalg
    M = np.vstack([np.asarray(T, dtype=np.float64).reshape(3, 4), [0.0, 0.0, 0.0, 1.0]])
    Lg = np.real(scipy.linalg.logm(M))
    return np.array([Lg[2, 1], Lg[0, 2], Lg[1, 0], Lg[0, 3], Lg[1, 3], Lg[2, 3]])


def tukey_weight(x, width, offset) -> float:
    """Shifted Tukey weight of a whitened error norm: (max(0, 1 - (x - offset)^2 / width))^2."""
    u = 1.0 - (x - offset) ** 2 / width
    return u * u if u > 0.0 else 0.0


def tukey_loss(x, width, offset) -> float:
    """rho(x^2) = int_0^x weight(u) 2u du (adaptive quadrature)."""
    import scipy.integrate
    if x <= 0.0:
        return 0.0
    return scipy.integrate.quad(lambda u: tukey_weight(u, width, offset) * 2.0 * u, 0.0, x,
                                points=[max(0.0, offset - np.sqrt(width)), offset, offset + np.sqrt(width)],
                                epsabs=0.0, epsrel=1e-13, limit=200)[0]


def _h(T):
    return np.vstack([np.asarray(T, dtype=np.float64).reshape(3, 4), [0.0, 0.0, 0.0, 1.0]])


def loop_residual(Ti, Tj, T_ij) -> np.ndarray:
    """r = Log(T_ij^-1 T_i^-1 T_j)."""
    return se3_log((np.linalg.inv(_h(T_ij)) @ np.linalg.inv(_h(Ti)) @ _h(Tj))[:3])


def loop_factor(Ti, Tj, T_ij, information, width, offset, h=1e-6):
    """Cost, H (12x12, [xi_i ; xi_j]) and b of one loop factor: Jacobian of r by central
    differences over right perturbations, weight frozen at the given poses."""
    Om = np.asarray(information, dtype=np.float64).reshape(6, 6)
    r = loop_residual(Ti, Tj, T_ij)
    x = float(np.sqrt(max(r @ Om @ r, 0.0)))
    J = np.zeros((6, 12))
    for k in range(12):
        d = np.zeros(12)
        d[k] = h
        rp = loop_residual(retract(Ti, d[:6])[0], retract(Tj, d[6:])[0], T_ij)
        rm = loop_residual(retract(Ti, -d[:6])[0], retract(Tj, -d[6:])[0], T_ij)
        J[:, k] = (rp - rm) / (2 * h)
    w = tukey_weight(x, width, offset)
    return tukey_loss(x, width, offset), w * J.T @ Om @ J, w * J.T @ Om @ r
