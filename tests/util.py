"""Helpers shared by the tests (error metric, small SE(3) algebra for finite differences)."""
import numpy as np


def err_metric(X, Xref, S):
    """max_i |X_i - Xref_i| / S_i, S_i = sum of |per-point contributions| of entry i.

    Entries whose scale is zero must match exactly (they are sums of zeros)."""
    X, Xref, S = (np.asarray(a, dtype=np.float64).ravel() for a in (X, Xref, S))
    d = np.abs(X - Xref)
    z = S == 0
    if np.any(d[z] != 0):
        return np.inf
    return float(np.max(d[~z] / S[~z])) if np.any(~z) else 0.0


def hat(w):
    return np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])


def se3_exp(xi):
    """Exp of xi = (omega, v) as a 4x4 matrix (Rodrigues, left Jacobian for v)."""
    w, v = np.asarray(xi[:3], float), np.asarray(xi[3:], float)
    th = np.linalg.norm(w)
    K = hat(w)
    if th < 1e-10:
        R = np.eye(3) + K + K @ K / 2
        V = np.eye(3) + K / 2 + K @ K / 6
    else:
        R = np.eye(3) + np.sin(th) / th * K + (1 - np.cos(th)) / th ** 2 * K @ K
        V = np.eye(3) + (1 - np.cos(th)) / th ** 2 * K + (th - np.sin(th)) / th ** 3 * K @ K
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = V @ v
    return T


def to44(T):
    T = np.asarray(T, float).reshape(3, 4)
    M = np.eye(4)
    M[:3] = T
    return M


def to34(M):
    return np.ascontiguousarray(M[:3])


def adjoint(T):
    """Ad(T) for xi = (omega, v): Exp(Ad xi) T = T Exp(xi)."""
    T = np.asarray(T, float).reshape(3, 4)
    R, t = T[:, :3], T[:, 3]
    A = np.zeros((6, 6))
    A[:3, :3] = R
    A[3:, 3:] = R
    A[3:, :3] = hat(t) @ R
    return A
