"""Python binding of the B300 VGICP library (libvgicp.so).

Argument marshalling only: every call goes through the C ABI declared in
include/vgicp.h, whose kernels do all the arithmetic.  numpy arrays are passed
as host memory; torch CUDA tensors are passed as device memory (their data
pointers), so PyTorch serves for device memory and streams.  There is no CPU
fallback: loading fails loudly if the library has not been built.

Functions keep the C names (vgicp_create, vgicp_add_frame, vgicp_build_voxelmap,
vgicp_build_voxelmaps, vgicp_linearize, vgicp_overlap, vgicp_overlap_matrix,
vgicp_debug_correspondences, vgicp_export_voxelmap, vgicp_estimate_covariances,
vgicp_release, ...); `Context` bundles them for convenience.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libvgicp.so")

VGICP_OK = 0
STATUS = {0: "VGICP_OK", 1: "VGICP_ERR_INVALID_ARG", 2: "VGICP_ERR_OOM", 3: "VGICP_ERR_NOT_FOUND",
          4: "VGICP_ERR_EMPTY", 5: "VGICP_ERR_CUDA", 6: "VGICP_ERR_TIMEOUT", 7: "VGICP_ERR_BUDGET",
          8: "VGICP_ERR_NUMERIC"}
VGICP_MEM_HOST, VGICP_MEM_DEVICE = 0, 1
VGICP_PREC_F32, VGICP_PREC_F64, VGICP_PREC_F32_COMP = 0, 1, 2

EXPORTS = ["vgicp_options_default", "vgicp_create", "vgicp_destroy", "vgicp_set_options", "vgicp_set_stream",
           "vgicp_synchronize", "vgicp_add_frame", "vgicp_frame_size", "vgicp_build_voxelmap",
           "vgicp_build_voxelmaps", "vgicp_voxelmap_size", "vgicp_linearize", "vgicp_overlap",
           "vgicp_overlap_matrix", "vgicp_debug_correspondences", "vgicp_export_voxelmap",
           "vgicp_estimate_covariances", "vgicp_release", "vgicp_memory_in_use", "vgicp_kernel_launches", "vgicp_kernel_timing", "vgicp_kernel_timing_reset",
           "vgicp_last_error", "vgicp_status_string", "vgicp_linearize_noalloc", "vgicp_autotune", "vgicp_overlap_matrix_work", "vgicp_set_lane",
           "vgicp_overlap_pairs", "vgicp_server_create", "vgicp_server_destroy", "vgicp_server_put_map",
           "vgicp_server_put_frame", "vgicp_server_submit", "vgicp_server_wait", "vgicp_server_stats",
           "vgicp_server_reset_stats", "vgicp_server_last_error", "vgicp_server_submit_batch", "vgicp_server_wait_batch", "vgicp_plan_create", "vgicp_plan_linearize",
           "vgicp_plan_info", "vgicp_plan_destroy", "vgicp_memory_estimate", "vgicp_evaluate", "vgicp_solve_step",
           "vgicp_se3_retract", "vgicp_optimize", "vgicp_add_frames", "vgicp_release_many", "vgicp_loop_linearize",
           "vgicp_optimize_with_loops", "vgicp_linearize_correspondences", "vgicp_server_loop_state"]
VGICP_REQ_LINEARIZE, VGICP_REQ_OVERLAP = 0, 1


class VgicpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("chunk_points", C.c_int32), ("linearize_variant", C.c_int32),
                ("blocks_per_sm", C.c_int32), ("hbm_budget_bytes", C.c_int64), ("overlap_cull", C.c_int32),
                ("linearize_cull", C.c_int32), ("neighbors", C.c_int32), ("count_weighted", C.c_int32),
                ("frame_order", C.c_int32), ("group_cull", C.c_int32)]


class Factor(C.Structure):
    _fields_ = [("target", C.c_int64), ("source", C.c_int64), ("target_pose", C.c_int32),
                ("source_pose", C.c_int32)]


class LMOptions(C.Structure):
    _fields_ = [("max_iterations", C.c_int32), ("anchor", C.c_int32), ("lambda_init", C.c_double),
                ("relative_tolerance", C.c_double)]


class LMReport(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("accepted", C.c_int32), ("n_history", C.c_int32),
                ("reserved", C.c_int32), ("initial_cost", C.c_double), ("final_cost", C.c_double),
                ("lambda_", C.c_double), ("linearize_ms", C.c_double), ("evaluate_ms", C.c_double),
                ("solve_ms", C.c_double), ("history", C.c_double * 64)]


class LoopFactor(C.Structure):
    _fields_ = [("pose_i", C.c_int32), ("pose_j", C.c_int32), ("T_ij", C.c_double * 12),
                ("information", C.c_double * 36), ("width", C.c_double), ("offset", C.c_double)]


def make_loop_factors(pose_i, pose_j, T_ij, information, width, offset):
    """A ctypes array of SE(3) loop factors (one per entry of the inputs)."""
    n = len(pose_i)
    arr = (LoopFactor * n)()
    T = np.asarray(T_ij, np.float64).reshape(n, 12)
    I6 = np.broadcast_to(np.asarray(information, np.float64).reshape(-1, 36), (n, 36))
    w = np.broadcast_to(np.asarray(width, np.float64), (n,))
    o = np.broadcast_to(np.asarray(offset, np.float64), (n,))
    for k in range(n):
        arr[k].pose_i, arr[k].pose_j = int(pose_i[k]), int(pose_j[k])
        arr[k].T_ij[:] = [float(x) for x in T[k]]
        arr[k].information[:] = [float(x) for x in I6[k]]
        arr[k].width, arr[k].offset = float(w[k]), float(o[k])
    return arr


class ServerOptions(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_int64), ("max_batch_requests", C.c_int32), ("lanes", C.c_int32),
                ("max_batch_points", C.c_int64), ("device_loop", C.c_int32), ("loop_slots", C.c_int32),
                ("loop_idle_ms", C.c_double)]


class Request(C.Structure):
    _fields_ = [("kind", C.c_int32), ("reserved", C.c_int32), ("target", C.c_int64), ("source", C.c_int64),
                ("T_target_source", C.c_double * 12)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int), ("kind", C.c_int32), ("H", C.c_double * 144), ("b", C.c_double * 12),
                ("cost", C.c_double), ("count", C.c_int64), ("fraction", C.c_double), ("latency_ms", C.c_double)]


class ServerCounters(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("batches", C.c_int64),
                ("admissions", C.c_int64), ("evictions", C.c_int64), ("resident_bytes", C.c_int64),
                ("mean_batch_requests", C.c_double), ("p50_ms", C.c_double), ("p99_ms", C.c_double),
                ("max_ms", C.c_double), ("host_launch_ms", C.c_double), ("host_finish_ms", C.c_double),
                ("device_ms", C.c_double), ("host_admit_ms", C.c_double), ("host_enqueue_ms", C.c_double)]


FACTOR_DTYPE = np.dtype([("target", np.int64), ("source", np.int64), ("target_pose", np.int32),
                         ("source_pose", np.int32)])

_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libvgicp.so (build it first with paper_2109_07073_b300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_2109_07073_b300.build`")
    lib = C.CDLL(path)
    vp, i64, i32, f64 = C.c_void_p, C.c_int64, C.c_int32, C.c_double
    sig = {
        "vgicp_options_default": [C.POINTER(Options)],
        "vgicp_create": [C.POINTER(vp), C.POINTER(Options), vp],
        "vgicp_destroy": [vp],
        "vgicp_set_options": [vp, C.POINTER(Options)],
        "vgicp_set_stream": [vp, vp],
        "vgicp_set_lane": [vp, i32, vp],
        "vgicp_overlap_pairs": [vp, vp, vp, i64, vp, vp, C.c_int],
        "vgicp_synchronize": [vp],
        "vgicp_add_frame": [vp, vp, vp, i64, C.c_int, C.POINTER(i64)],
        "vgicp_add_frames": [vp, vp, vp, vp, i64, C.c_int, vp],
        "vgicp_frame_size": [vp, i64, C.POINTER(i64)],
        "vgicp_build_voxelmap": [vp, vp, vp, i64, f64, C.c_int, C.POINTER(i64)],
        "vgicp_build_voxelmaps": [vp, vp, i64, f64, vp],
        "vgicp_voxelmap_size": [vp, i64, C.POINTER(i64)],
        "vgicp_linearize": [vp, vp, i64, vp, i64, vp, vp, vp, vp, C.c_int],
        "vgicp_linearize_correspondences": [vp, vp, i64, vp, i64, vp, vp, vp, vp, vp, vp],
        "vgicp_linearize_noalloc": [vp, vp, i64, vp, i64, vp, vp, vp, vp],
        "vgicp_autotune": [vp, vp, i64, vp, i64, i32, C.POINTER(Options), C.POINTER(f64)],
        "vgicp_overlap_matrix_work": [vp, C.POINTER(i64), C.POINTER(i64)],
        "vgicp_overlap": [vp, i64, i64, vp, C.POINTER(f64), C.POINTER(i64)],
        "vgicp_overlap_matrix": [vp, vp, i64, vp, i64, vp, vp, vp, C.c_int],
        "vgicp_debug_correspondences": [vp, i64, i64, vp, vp, vp],
        "vgicp_export_voxelmap": [vp, i64, vp, vp, vp, vp, C.POINTER(i64)],
        "vgicp_estimate_covariances": [vp, vp, i64, i32, f64, vp, C.c_int],
        "vgicp_release": [vp, i64],
        "vgicp_release_many": [vp, vp, i64],
        "vgicp_memory_in_use": [vp, C.POINTER(i64)],
        "vgicp_memory_estimate": [vp, i64, i32, C.POINTER(i64)],
        "vgicp_kernel_launches": [vp, C.POINTER(i64)],
        "vgicp_kernel_timing": [vp, i32, C.POINTER(C.c_double), C.POINTER(i64)],
        "vgicp_kernel_timing_reset": [vp],
        "vgicp_plan_create": [vp, vp, i64, i64, C.POINTER(vp)],
        "vgicp_evaluate": [vp, vp, i64, vp, i64, vp, vp, C.c_int],
        "vgicp_solve_step": [vp, vp, vp, i64, i64, i32, f64, vp, C.POINTER(f64)],
        "vgicp_se3_retract": [vp, vp, i64],
        "vgicp_optimize": [vp, vp, i64, vp, i64, C.POINTER(LMOptions), C.POINTER(LMReport)],
        "vgicp_optimize_with_loops": [vp, vp, i64, vp, i64, vp, i64, C.POINTER(LMOptions), C.POINTER(LMReport)],
        "vgicp_loop_linearize": [vp, i64, vp, i64, vp, vp, vp],
        "vgicp_plan_linearize": [vp, vp, vp, vp, vp, vp, vp, C.c_int],
        "vgicp_plan_info": [vp, vp, C.POINTER(i64), C.POINTER(i64)],
        "vgicp_plan_destroy": [vp, vp],
        "vgicp_server_create": [C.POINTER(vp), C.POINTER(ServerOptions), C.POINTER(Options)],
        "vgicp_server_destroy": [vp],
        "vgicp_server_put_map": [vp, i64, vp, vp, i64, f64],
        "vgicp_server_put_frame": [vp, i64, vp, vp, i64],
        "vgicp_server_submit": [vp, C.POINTER(Request), C.POINTER(i64)],
        "vgicp_server_submit_batch": [vp, vp, i64, vp],
        "vgicp_server_wait_batch": [vp, vp, i64, f64, vp],
        "vgicp_server_wait": [vp, i64, f64, C.POINTER(Result)],
        "vgicp_server_stats": [vp, C.POINTER(ServerCounters)],
        "vgicp_server_reset_stats": [vp],
        "vgicp_server_loop_state": [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i64)],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int
    lib.vgicp_last_error.argtypes = [vp]
    lib.vgicp_last_error.restype = C.c_char_p
    lib.vgicp_server_last_error.argtypes = [vp]
    lib.vgicp_server_last_error.restype = C.c_char_p
    lib.vgicp_status_string.argtypes = [C.c_int]
    lib.vgicp_status_string.restype = C.c_char_p
    _lib = lib
    return lib


def _check(ctx, status: int):
    if status != VGICP_OK:
        msg = load().vgicp_last_error(ctx).decode() if ctx else ""
        raise VgicpError(status, msg)


def _is_torch_cuda(a) -> bool:
    return hasattr(a, "is_cuda") and a.is_cuda


def _host(a, dtype, cols=None):
    a = np.ascontiguousarray(a, dtype=dtype)
    if cols is not None:
        a = a.reshape(-1, cols)
    return a


def _ptr(a):
    if a is None:
        return None
    if _is_torch_cuda(a):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def _cloud(points, covs=None):
    """(points, covs, n, mem_kind) with both in the same memory and the C layout."""
    if _is_torch_cuda(points):
        import torch
        p = points.to(torch.float32).contiguous().reshape(-1, 3)
        c = None if covs is None else covs.to(device=p.device, dtype=torch.float32).contiguous().reshape(-1, 6)
        return p, c, int(p.shape[0]), VGICP_MEM_DEVICE
    p = _host(points, np.float32, 3)
    c = None if covs is None else _host(covs, np.float32, 6)
    return p, c, int(p.shape[0]), VGICP_MEM_HOST


def _pose12(T):
    return _host(np.asarray(T, dtype=np.float64).reshape(-1, 12), np.float64)


# ----------------------------------------------------------------- the ABI --

def vgicp_options_default() -> Options:
    o = Options()
    _check(None, load().vgicp_options_default(C.byref(o)))
    return o


CUDA_STREAM_LEGACY = 0x1


def _stream_arg(stream):
    """None -> the context's own stream; a torch stream or raw handle otherwise.

    torch's default stream has handle 0, the legacy default stream, which the C
    ABI reads as "no stream given"; it is passed as cudaStreamLegacy instead."""
    if stream is None:
        return None
    s = getattr(stream, "cuda_stream", stream)
    return C.c_void_p(s if s else CUDA_STREAM_LEGACY)


def vgicp_create(options: Options = None, stream=None):
    """New context; stream is a torch.cuda.Stream, a raw cudaStream_t int, or None (own stream)."""
    ctx = C.c_void_p()
    _check(None, load().vgicp_create(C.byref(ctx), C.byref(options) if options is not None else None,
                                     _stream_arg(stream)))
    return ctx


def vgicp_destroy(ctx):
    _check(ctx, load().vgicp_destroy(ctx))


def vgicp_set_options(ctx, options: Options):
    _check(ctx, load().vgicp_set_options(ctx, C.byref(options)))


def vgicp_set_stream(ctx, stream=None):
    _check(ctx, load().vgicp_set_stream(ctx, _stream_arg(stream)))


def vgicp_set_lane(ctx, lane: int, stream=None):
    """Select the lane (own stream and scratch; shared handles) of later calls."""
    _check(ctx, load().vgicp_set_lane(ctx, int(lane), _stream_arg(stream)))


def vgicp_synchronize(ctx):
    _check(ctx, load().vgicp_synchronize(ctx))


def vgicp_add_frame(ctx, points, covs) -> int:
    p, c, n, kind = _cloud(points, covs)
    h = C.c_int64()
    _check(ctx, load().vgicp_add_frame(ctx, _ptr(p), _ptr(c), n, kind, C.byref(h)))
    return h.value


def vgicp_add_frames(ctx, points, covs, sizes) -> np.ndarray:
    """Register len(sizes) frames stored one after another in points (total, 3) and covs
    (total, 6): numpy arrays (host) or torch CUDA tensors (device).  Returns the handles."""
    n = np.ascontiguousarray(sizes, np.int64)
    out = np.zeros(n.shape[0], np.int64)
    if _is_torch_cuda(points):
        p, c, kind = points, covs, VGICP_MEM_DEVICE
    else:
        p, c, kind = _host(points, np.float32, 3), _host(covs, np.float32, 6), VGICP_MEM_HOST
    _check(ctx, load().vgicp_add_frames(ctx, _ptr(p), _ptr(c), _ptr(n), n.shape[0], kind, _ptr(out)))
    return out


def vgicp_frame_size(ctx, frame: int) -> int:
    n = C.c_int64()
    _check(ctx, load().vgicp_frame_size(ctx, frame, C.byref(n)))
    return n.value


def vgicp_build_voxelmap(ctx, points, covs, resolution: float) -> int:
    p, c, n, kind = _cloud(points, covs)
    h = C.c_int64()
    _check(ctx, load().vgicp_build_voxelmap(ctx, _ptr(p), _ptr(c), n, float(resolution), kind, C.byref(h)))
    return h.value


def vgicp_build_voxelmaps(ctx, frames, resolution: float, maps=None) -> np.ndarray:
    f = _host(frames, np.int64)
    m = np.full(f.shape[0], -1, np.int64) if maps is None else _host(maps, np.int64).copy()
    _check(ctx, load().vgicp_build_voxelmaps(ctx, _ptr(f), f.shape[0], float(resolution), _ptr(m)))
    return m


def vgicp_voxelmap_size(ctx, vmap: int) -> int:
    n = C.c_int64()
    _check(ctx, load().vgicp_voxelmap_size(ctx, vmap, C.byref(n)))
    return n.value


def make_factors(targets, sources, target_poses, source_poses) -> np.ndarray:
    f = np.zeros(len(targets), FACTOR_DTYPE)
    f["target"], f["source"] = targets, sources
    f["target_pose"], f["source_pose"] = target_poses, source_poses
    return f


def vgicp_linearize(ctx, factors, poses, out=None):
    """Eq. 3-6 for every factor.  Returns (H (n,12,12), b (n,12), cost (n,), inliers (n,)).

    out: optional tuple of preallocated outputs; torch CUDA tensors make the call
    write device memory (asynchronously), numpy arrays host memory."""
    f = np.ascontiguousarray(factors, dtype=FACTOR_DTYPE)
    P = _pose12(poses)
    nf = f.shape[0]
    if out is None:
        out = (np.zeros((nf, 12, 12)), np.zeros((nf, 12)), np.zeros(nf), np.zeros(nf, np.int64))
    H, b, cost, inl = out
    kind = VGICP_MEM_DEVICE if _is_torch_cuda(H) else VGICP_MEM_HOST
    _check(ctx, load().vgicp_linearize(ctx, _ptr(f), nf, _ptr(P), P.shape[0], _ptr(H), _ptr(b), _ptr(cost),
                                       _ptr(inl), kind))
    return H, b, cost, inl


def vgicp_linearize_correspondences(ctx, factors, poses):
    """vgicp_linearize() with the correspondences its kernels took recorded.

    Returns (H, b, cost, inliers, keys, state): keys (P, 3) int64 and state (P,)
    int32 for the P = sum of the factors' source sizes points, factor by factor
    in point order (INT64_MIN rows: no voxel coordinate or never visited; state
    1 voxel found, 0 not found, -1 in a culled chunk)."""
    f = np.ascontiguousarray(factors, dtype=FACTOR_DTYPE)
    P = _pose12(poses)
    nf = f.shape[0]
    total = sum(vgicp_frame_size(ctx, int(h)) for h in f["source"])
    H, b, cost, inl = np.zeros((nf, 12, 12)), np.zeros((nf, 12)), np.zeros(nf), np.zeros(nf, np.int64)
    keys = np.zeros((max(total, 1), 3), np.int64)
    state = np.zeros(max(total, 1), np.int32)
    _check(ctx, load().vgicp_linearize_correspondences(ctx, _ptr(f), nf, _ptr(P), P.shape[0], _ptr(H), _ptr(b),
                                                       _ptr(cost), _ptr(inl), _ptr(keys), _ptr(state)))
    return H, b, cost, inl, keys[:total], state[:total]


def vgicp_evaluate(ctx, factors, poses, out=None):
    """Each factor's cost (and inliers) at the poses, by the cost-only batched pass."""
    f = np.ascontiguousarray(factors, dtype=FACTOR_DTYPE)
    P = _pose12(poses)
    nf = f.shape[0]
    if out is None:
        out = (np.zeros(nf), np.zeros(nf, np.int64))
    cost, inl = out
    kind = VGICP_MEM_DEVICE if _is_torch_cuda(cost) else VGICP_MEM_HOST
    _check(ctx, load().vgicp_evaluate(ctx, _ptr(f), nf, _ptr(P), P.shape[0], _ptr(cost), _ptr(inl), kind))
    return cost, inl


def vgicp_solve_step(pairs, H, b, n_poses: int, anchor: int = 0, lam: float = 0.0):
    """Host-only damped Gauss-Newton step: returns (delta (n_poses, 6), model decrease)."""
    pr = np.ascontiguousarray(pairs, np.int32).reshape(-1, 2)
    Hh = np.ascontiguousarray(H, np.float64).reshape(-1, 144)
    bh = np.ascontiguousarray(b, np.float64).reshape(-1, 12)
    delta = np.zeros((int(n_poses), 6))
    dec = C.c_double()
    _check(None, load().vgicp_solve_step(_ptr(pr), _ptr(Hh), _ptr(bh), pr.shape[0], int(n_poses), int(anchor),
                                         float(lam), _ptr(delta), C.byref(dec)))
    return delta, dec.value


def vgicp_se3_retract(poses, delta) -> np.ndarray:
    """Host-only: T <- T Exp(delta) per pose; returns new poses (n, 3, 4)."""
    P = np.array(_pose12(poses), dtype=np.float64)
    d = np.ascontiguousarray(delta, np.float64).reshape(-1, 6)
    if d.shape[0] != P.shape[0]:
        raise ValueError("one delta per pose")
    _check(None, load().vgicp_se3_retract(_ptr(P), _ptr(d), P.shape[0]))
    return P.reshape(-1, 3, 4)


def vgicp_optimize(ctx, factors, poses, max_iterations: int = 20, anchor: int = 0, lambda_init: float = 0.0,
                   relative_tolerance: float = 0.0):
    """Levenberg-Marquardt over the factors; returns (optimised poses (n, 3, 4), LMReport)."""
    f = np.ascontiguousarray(factors, dtype=FACTOR_DTYPE)
    P = np.array(_pose12(poses), dtype=np.float64)
    opt = LMOptions(max_iterations, anchor, lambda_init, relative_tolerance)
    rep = LMReport()
    _check(ctx, load().vgicp_optimize(ctx, _ptr(f), f.shape[0], _ptr(P), P.shape[0], C.byref(opt), C.byref(rep)))
    return P.reshape(-1, 3, 4), rep


def vgicp_loop_linearize(loops, poses, blocks: bool = True):
    """Host-only: (H (n,12,12), b (n,12), cost (n,)) of SE(3) loop factors at the poses."""
    P = np.array(_pose12(poses), dtype=np.float64)
    n = len(loops)
    H, b, cost = np.zeros((n, 12, 12)), np.zeros((n, 12)), np.zeros(n)
    _check(None, load().vgicp_loop_linearize(C.cast(loops, C.c_void_p), n, _ptr(P), P.shape[0],
                                             _ptr(H) if blocks else None, _ptr(b) if blocks else None, _ptr(cost)))
    return H, b, cost


def vgicp_optimize_with_loops(ctx, factors, loops, poses, max_iterations: int = 20, anchor: int = 0,
                              lambda_init: float = 0.0, relative_tolerance: float = 0.0):
    """vgicp_optimize with SE(3) loop factors (make_loop_factors) added."""
    f = np.ascontiguousarray(factors, dtype=FACTOR_DTYPE)
    P = np.array(_pose12(poses), dtype=np.float64)
    opt = LMOptions(max_iterations, anchor, lambda_init, relative_tolerance)
    rep = LMReport()
    _check(ctx, load().vgicp_optimize_with_loops(ctx, _ptr(f), f.shape[0], C.cast(loops, C.c_void_p), len(loops),
                                                 _ptr(P), P.shape[0], C.byref(opt), C.byref(rep)))
    return P.reshape(-1, 3, 4), rep


def vgicp_plan_create(ctx, factors, n_poses: int):
    """A Gauss-Newton iteration plan: the factor set fixed, each run one CUDA graph launch."""
    f = np.ascontiguousarray(factors, dtype=FACTOR_DTYPE)
    plan = C.c_void_p()
    _check(ctx, load().vgicp_plan_create(ctx, _ptr(f), f.shape[0], int(n_poses), C.byref(plan)))
    plan.n_f = f.shape[0]
    return plan


def vgicp_plan_linearize(ctx, plan, poses, out=None):
    """One iteration of a plan at `poses`; same outputs as vgicp_linearize."""
    P = _pose12(poses)
    nf = plan.n_f
    if out is None:
        out = (np.zeros((nf, 12, 12)), np.zeros((nf, 12)), np.zeros(nf), np.zeros(nf, np.int64))
    H, b, cost, inl = out
    kind = VGICP_MEM_DEVICE if _is_torch_cuda(H) else VGICP_MEM_HOST
    _check(ctx, load().vgicp_plan_linearize(ctx, plan, _ptr(P), _ptr(H), _ptr(b), _ptr(cost), _ptr(inl), kind))
    return H, b, cost, inl


def vgicp_plan_info(ctx, plan):
    """(runs, graph captures) of a plan."""
    r, c = C.c_int64(), C.c_int64()
    _check(ctx, load().vgicp_plan_info(ctx, plan, C.byref(r), C.byref(c)))
    return r.value, c.value


def vgicp_plan_destroy(ctx, plan):
    _check(ctx, load().vgicp_plan_destroy(ctx, plan))


def check_noalloc_outputs(n: int, out):
    """Validate vgicp_linearize_noalloc's outputs before any device write: torch tensors,
    contiguous, float64 H / b / cost and int64 inliers (or None) with room for n factors
    (at least n*144, n*12, n and n elements), all CUDA tensors on one device."""
    import torch
    H, b, cost, inl = out
    spec = [("H", H, torch.float64, 144), ("b", b, torch.float64, 12), ("cost", cost, torch.float64, 1)]
    if inl is not None:
        spec.append(("inliers", inl, torch.int64, 1))
    for name, t, dt, per in spec:
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"vgicp_linearize_noalloc: {name} must be a torch tensor")
        if t.dtype != dt:
            raise ValueError(f"vgicp_linearize_noalloc: {name} must be {dt}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"vgicp_linearize_noalloc: {name} must be contiguous")
        if t.numel() < n * per:
            raise ValueError(f"vgicp_linearize_noalloc: {name} holds {t.numel()} elements, needs {n * per}")
    for name, t, _, _ in spec:
        if not t.is_cuda:
            raise ValueError(f"vgicp_linearize_noalloc writes device outputs: {name} must be a CUDA tensor")
    devs = {t.device.index for _, t, _, _ in spec}
    if len(devs) != 1 or devs.pop() != torch.cuda.current_device():
        raise ValueError("vgicp_linearize_noalloc: every output must be on the current (the context's) device")


def vgicp_linearize_noalloc(ctx, factors, poses, out):
    """vgicp_linearize without allocating: out = (H, b, cost, inliers) torch CUDA tensors
    (n,12,12) float64, (n,12) float64, (n,) float64, (n,) int64 or None, written asynchronously
    on the context stream.  For callers that must not allocate device memory at call time."""
    f = np.ascontiguousarray(factors, dtype=FACTOR_DTYPE)
    P = _pose12(poses)
    H, b, cost, inl = out
    check_noalloc_outputs(f.shape[0], out)
    _check(ctx, load().vgicp_linearize_noalloc(ctx, _ptr(f), f.shape[0], _ptr(P), P.shape[0], _ptr(H), _ptr(b),
                                               _ptr(cost), _ptr(inl)))
    return H, b, cost, inl


def vgicp_autotune(ctx, factors, poses, reps: int = 3):
    """Time the batched linearisation's candidates on this factor set; keeps and returns
    (best options, ms per run)."""
    f = np.ascontiguousarray(factors, dtype=FACTOR_DTYPE)
    P = _pose12(poses)
    best, ms = Options(), C.c_double()
    _check(ctx, load().vgicp_autotune(ctx, _ptr(f), f.shape[0], _ptr(P), P.shape[0], int(reps), C.byref(best),
                                      C.byref(ms)))
    return best, ms.value


def vgicp_overlap(ctx, source: int, target: int, T_target_source):
    """Eq. 8: (fraction, count)."""
    T = _pose12(T_target_source)
    fr, cnt = C.c_double(), C.c_int64()
    _check(ctx, load().vgicp_overlap(ctx, source, target, _ptr(T), C.byref(fr), C.byref(cnt)))
    return fr.value, cnt.value


def vgicp_overlap_pairs(ctx, sources, targets, T, out=None) -> np.ndarray:
    """counts (n,) int64: hits of sources[i] in targets[i] under T[i] (target-from-source)."""
    s, t = _host(sources, np.int64), _host(targets, np.int64)
    P = _pose12(T)
    if out is None:
        out = np.zeros(s.shape[0], np.int64)
    kind = VGICP_MEM_DEVICE if _is_torch_cuda(out) else VGICP_MEM_HOST
    _check(ctx, load().vgicp_overlap_pairs(ctx, _ptr(s), _ptr(t), s.shape[0], _ptr(P), _ptr(out), kind))
    return out


def vgicp_overlap_matrix(ctx, sources, targets, poses_src, poses_tgt, out=None) -> np.ndarray:
    """counts (n_src, n_tgt) int64: hits of source s in target t under T_t^-1 T_s."""
    s = _host(sources, np.int64)
    t = _host(targets, np.int64)
    ps, pt = _pose12(poses_src), _pose12(poses_tgt)
    if out is None:
        out = np.zeros((s.shape[0], t.shape[0]), np.int64)
    kind = VGICP_MEM_DEVICE if _is_torch_cuda(out) else VGICP_MEM_HOST
    _check(ctx, load().vgicp_overlap_matrix(ctx, _ptr(s), s.shape[0], _ptr(t), t.shape[0], _ptr(ps), _ptr(pt),
                                            _ptr(out), kind))
    return out


def vgicp_overlap_matrix_work(ctx):
    """(live pairs, point lookups) of the last overlap matrix on this context."""
    lp, lk = C.c_int64(), C.c_int64()
    _check(ctx, load().vgicp_overlap_matrix_work(ctx, C.byref(lp), C.byref(lk)))
    return lp.value, lk.value


def vgicp_debug_correspondences(ctx, source: int, target: int, T_target_source):
    """(keys (n, 3) int64 with INT64_MIN rows for invalid points, hit (n,) bool)."""
    n = vgicp_frame_size(ctx, source)
    keys = np.zeros((max(n, 1), 3), np.int64)
    hit = np.zeros(max(n, 1), np.int32)
    T = _pose12(T_target_source)
    _check(ctx, load().vgicp_debug_correspondences(ctx, source, target, _ptr(T), _ptr(keys), _ptr(hit)))
    return keys[:n], hit[:n].astype(bool)


def vgicp_export_voxelmap(ctx, vmap: int):
    """(keys (V, 3) int64, counts (V,), mu (V, 3) float64, cov (V, 6) float64), sorted by key."""
    nv = C.c_int64(0)
    _check(ctx, load().vgicp_export_voxelmap(ctx, vmap, None, None, None, None, C.byref(nv)))
    V = nv.value
    keys = np.zeros((max(V, 1), 3), np.int64)
    counts = np.zeros(max(V, 1), np.int64)
    mu = np.zeros((max(V, 1), 3))
    cov = np.zeros((max(V, 1), 6))
    nv = C.c_int64(max(V, 1))
    _check(ctx, load().vgicp_export_voxelmap(ctx, vmap, _ptr(keys), _ptr(counts), _ptr(mu), _ptr(cov), C.byref(nv)))
    V = nv.value
    return keys[:V], counts[:V], mu[:V], cov[:V]


def vgicp_estimate_covariances(ctx, points, k: int = 10, eps: float = 1e-3, out=None):
    """Per-point covariances (n, 6) float32 from k neighbours, eigenvalues (1, 1, eps)."""
    p, _, n, kind = _cloud(points)
    if out is None:
        if kind == VGICP_MEM_DEVICE:
            import torch
            out = torch.empty((n, 6), dtype=torch.float32, device=p.device)
        else:
            out = np.zeros((n, 6), np.float32)
    _check(ctx, load().vgicp_estimate_covariances(ctx, _ptr(p), n, int(k), float(eps), _ptr(out), kind))
    return out


def vgicp_release(ctx, handle: int):
    _check(ctx, load().vgicp_release(ctx, handle))


def vgicp_release_many(ctx, handles):
    h = np.ascontiguousarray(handles, np.int64)
    _check(ctx, load().vgicp_release_many(ctx, _ptr(h), h.shape[0]))


def vgicp_memory_in_use(ctx) -> int:
    v = C.c_int64()
    _check(ctx, load().vgicp_memory_in_use(ctx, C.byref(v)))
    return v.value


def vgicp_memory_estimate(ctx, n: int, is_map: bool) -> int:
    v = C.c_int64()
    _check(ctx, load().vgicp_memory_estimate(ctx, int(n), int(bool(is_map)), C.byref(v)))
    return v.value


def vgicp_kernel_launches(ctx) -> int:
    v = C.c_int64()
    _check(ctx, load().vgicp_kernel_launches(ctx, C.byref(v)))
    return v.value


VGICP_KERNEL_LINEARIZE, VGICP_KERNEL_OVERLAP_MATRIX, VGICP_KERNEL_VOXELMAP_BUILD = 0, 1, 2


def vgicp_kernel_timing(ctx, kernel: int):
    """(summed device milliseconds, launches) of a hot kernel's timed launches on the
    current lane since the last reset."""
    ms, n = C.c_double(), C.c_int64()
    _check(ctx, load().vgicp_kernel_timing(ctx, int(kernel), C.byref(ms), C.byref(n)))
    return ms.value, n.value


def vgicp_kernel_timing_reset(ctx):
    _check(ctx, load().vgicp_kernel_timing_reset(ctx))


def vgicp_last_error(ctx) -> str:
    return load().vgicp_last_error(ctx).decode()


class Context:
    """A vgicp_ctx with the calls bound as methods (names without the vgicp_ prefix)."""

    def __init__(self, precision: int = VGICP_PREC_F32, stream=None, **opts):
        o = vgicp_options_default()
        o.precision = precision
        for k, v in opts.items():
            setattr(o, k, v)
        self.options = o
        self.ctx = vgicp_create(o, stream)

    def close(self):
        if self.ctx:
            vgicp_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_options(self, **opts):
        for k, v in opts.items():
            setattr(self.options, k, v)
        vgicp_set_options(self.ctx, self.options)

    def autotune(self, factors, poses, reps: int = 3):
        best, ms = vgicp_autotune(self.ctx, factors, poses, reps)
        self.options = best
        return best, ms

    def __getattr__(self, name):
        fn = globals().get("vgicp_" + name)
        if fn is None or name.startswith("_"):
            raise AttributeError(name)
        return lambda *a, **k: fn(self.ctx, *a, **k)


def _scheck(server, status: int):
    if status != VGICP_OK:
        msg = load().vgicp_server_last_error(server).decode() if server else ""
        raise VgicpError(status, msg)


def vgicp_server_create(options: ServerOptions = None, kernel_options: Options = None):
    s = C.c_void_p()
    _scheck(None, load().vgicp_server_create(C.byref(s), C.byref(options) if options is not None else None,
                                             C.byref(kernel_options) if kernel_options is not None else None))
    return s


def vgicp_server_loop_state(server):
    """(running, last exit status, launches) of a device-loop server's loop kernel."""
    r, e, n = C.c_int32(), C.c_int32(), C.c_int64()
    _scheck(server, load().vgicp_server_loop_state(server, C.byref(r), C.byref(e), C.byref(n)))
    return bool(r.value), e.value, n.value


def vgicp_server_destroy(server):
    _scheck(None, load().vgicp_server_destroy(server))


def vgicp_server_put_map(server, key: int, points, covs, resolution: float):
    p, c = _host(points, np.float32, 3), _host(covs, np.float32, 6)
    _scheck(server, load().vgicp_server_put_map(server, key, _ptr(p), _ptr(c), p.shape[0], resolution))


def vgicp_server_put_frame(server, key: int, points, covs):
    p, c = _host(points, np.float32, 3), _host(covs, np.float32, 6)
    _scheck(server, load().vgicp_server_put_frame(server, key, _ptr(p), _ptr(c), p.shape[0]))


def vgicp_server_submit(server, kind: int, target: int, source: int, T_target_source) -> int:
    r = Request(kind=kind, target=target, source=source)
    T = _pose12(T_target_source)
    if T.shape != (1, 12):
        raise ValueError("T_target_source must hold 12 values (row-major 3x4)")
    r.T_target_source[:] = [float(x) for x in T[0]]
    t = C.c_int64()
    _scheck(server, load().vgicp_server_submit(server, C.byref(r), C.byref(t)))
    return t.value


def vgicp_server_submit_batch(server, kinds, targets, sources, T) -> np.ndarray:
    """Queue len(kinds) requests at once; T (n, 3, 4) or (n, 12).  Returns the tickets."""
    k = np.ascontiguousarray(kinds, np.int32)
    n = k.shape[0]
    P = _pose12(T)
    if P.shape != (n, 12):
        raise ValueError("T must hold 12 values per request")
    reqs = (Request * n)()
    arr = np.frombuffer(reqs, dtype=np.dtype([("kind", np.int32), ("reserved", np.int32), ("target", np.int64),
                                              ("source", np.int64), ("T", np.float64, 12)]), count=n)
    arr["kind"], arr["reserved"] = k, 0
    arr["target"], arr["source"] = np.asarray(targets, np.int64), np.asarray(sources, np.int64)
    arr["T"] = P
    tickets = np.zeros(n, np.int64)
    _scheck(server, load().vgicp_server_submit_batch(server, C.cast(reqs, C.c_void_p), n, _ptr(tickets)))
    return tickets


def vgicp_server_wait_batch(server, tickets, timeout_s: float = -1.0):
    """Results of many tickets at once (a ctypes array of Result, in ticket order)."""
    t = np.ascontiguousarray(tickets, np.int64)
    out = (Result * t.shape[0])()
    _scheck(server, load().vgicp_server_wait_batch(server, _ptr(t), t.shape[0], timeout_s, C.cast(out, C.c_void_p)))
    return out


def vgicp_server_wait(server, ticket: int, timeout_s: float = -1.0) -> Result:
    """Result of a request (raises VgicpError(VGICP_ERR_TIMEOUT) when the wait runs out)."""
    r = Result()
    _scheck(server, load().vgicp_server_wait(server, ticket, timeout_s, C.byref(r)))
    return r


def vgicp_server_stats(server) -> ServerCounters:
    c = ServerCounters()
    _scheck(server, load().vgicp_server_stats(server, C.byref(c)))
    return c


def vgicp_server_reset_stats(server):
    _scheck(server, load().vgicp_server_reset_stats(server))


def vgicp_server_last_error(server) -> str:
    return load().vgicp_server_last_error(server).decode()


class Server:
    """A vgicp_server with the calls bound as methods (names without the vgicp_server_ prefix)."""

    def __init__(self, hbm_budget_bytes: int = 0, lanes: int = 2, max_batch_requests: int = 0,
                 max_batch_points: int = 0, kernel_options: Options = None, device_loop: bool = False,
                 loop_slots: int = 0, loop_idle_ms: float = 0.0):
        self.server = vgicp_server_create(ServerOptions(hbm_budget_bytes, max_batch_requests, lanes,
                                                        max_batch_points, int(device_loop), loop_slots,
                                                        loop_idle_ms), kernel_options)

    def close(self):
        if self.server:
            vgicp_server_destroy(self.server)
            self.server = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __getattr__(self, name):
        fn = globals().get("vgicp_server_" + name)
        if fn is None or name.startswith("_"):
            raise AttributeError(name)
        return lambda *a, **k: fn(self.server, *a, **k)
