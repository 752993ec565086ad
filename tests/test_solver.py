"""Host-side Gauss-Newton pieces (no GPU): the library's sparse damped step and
SE(3) retraction against the oracle's dense solve and closed-form exponential,
and the oracle's own pins (scipy's matrix exponential, the normal equations'
residual, a hand-solved case)."""
import os

import numpy as np
import pytest
import scipy.linalg

import datagen as dg
import oracle
import paper_2109_07073_b300 as vg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _twist_matrix(xi):
    w, v = xi[:3], xi[3:]
    M = np.zeros((4, 4))
    M[:3, :3] = [[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]
    M[:3, 3] = v
    return M


def _random_system(rng, n_poses, n_loops=6, rank=12):
    """Factors along a ring (i, i+1), (i, i+2) plus random loop closures, each
    H_f = G'G with G rank x 12 random, b_f random."""
    pairs = [(i, (i + 1) % n_poses) for i in range(n_poses)] + [(i, (i + 2) % n_poses) for i in range(n_poses)]
    for _ in range(n_loops):
        a, c = (int(x) for x in np.floor(rng.uniform(2, 0, n_poses)))
        if a != c:
            pairs.append((a, c))
    H, b = [], []
    for _ in pairs:
        G = rng.normal(rank * 12).reshape(rank, 12)
        H.append(G.T @ G)
        b.append(rng.normal(12))
    return np.array(pairs), np.array(H), np.array(b)


def test_oracle_se3_exp_matches_matrix_exponential():
    rng = dg.Stream(5)
    for scale in (1e-9, 1e-3, 0.3, 2.5):
        xi = rng.normal(6) * scale
        E = scipy.linalg.expm(_twist_matrix(xi))
        assert np.allclose(oracle.se3_exp(xi), E[:3], rtol=0, atol=1e-12)


def test_retract_matches_oracle():
    rng = dg.Stream(6)
    poses = np.stack([dg.random_pose(rng, 30, 5.0) for _ in range(7)])
    delta = rng.normal(42).reshape(7, 6) * np.array([0.2, 0.2, 0.2, 1.0, 1.0, 1.0])
    delta[3] = 0.0
    delta[4] *= 1e-7                                    # the small-angle branch
    got = vg.vgicp_se3_retract(poses, delta)
    ref = oracle.retract(poses, delta)
    assert np.allclose(got, ref, rtol=0, atol=1e-12)
    assert np.array_equal(got[3], poses[3])


def test_oracle_gn_step_solves_the_damped_normal_equations():
    rng = dg.Stream(7)
    pairs, H, b = _random_system(rng, 6)
    d, dec = oracle.gn_step(pairs, H, b, 6, anchor=2, lam=0.3)
    Hg, bg = oracle.assemble(pairs, H, b, 6)
    free = [i for i in range(36) if i // 6 != 2]
    A = Hg[np.ix_(free, free)]
    fl = 1e-12 * np.mean(np.diag(A))
    D = np.diag(np.maximum(np.diag(A), fl)) * 0.3 + fl * np.eye(len(free))
    r = (A + D) @ d.reshape(-1)[free] + bg[free]
    assert np.max(np.abs(r)) <= 1e-10 * np.max(np.abs(bg))
    assert not d[2].any()
    dd = d.reshape(-1)
    assert dec == pytest.approx(-(2 * bg @ dd + dd @ Hg @ dd), rel=1e-12)


def test_oracle_gn_step_hand_case():
    # two poses, anchor 0, one factor with H = 2 I, b = (1, ..., 12): d_1 = -b_source / 2
    H = 2.0 * np.eye(12)[None]
    b = np.arange(1.0, 13.0)[None]
    d, dec = oracle.gn_step(np.array([[0, 1]]), H, b, 2, anchor=0, lam=0.0)
    assert np.allclose(d[1], -np.arange(7.0, 13.0) / 2, rtol=1e-10)
    assert not d[0].any()
    assert dec == pytest.approx(np.sum(np.arange(7.0, 13.0) ** 2) / 2, rel=1e-10)


@pytest.mark.parametrize("n_poses,anchor,lam", [(2, 0, 0.0), (9, 0, 0.0), (9, 4, 1e-3), (40, 17, 0.5), (40, 0, 10.0)])
def test_solve_step_matches_oracle(n_poses, anchor, lam):
    rng = dg.Stream(100 + n_poses + anchor)
    pairs, H, b = _random_system(rng, n_poses, n_loops=n_poses // 3)
    got, gdec = vg.vgicp_solve_step(pairs, H, b, n_poses, anchor, lam)
    ref, rdec = oracle.gn_step(pairs, H, b, n_poses, anchor, lam)
    assert np.allclose(got, ref, rtol=1e-7, atol=1e-9 * np.abs(ref).max())
    assert not got[anchor].any()
    assert gdec == pytest.approx(rdec, rel=1e-7)


def test_solve_step_rank_deficient_blocks_and_isolated_pose():
    # Gauss-Newton factor blocks have rank <= 6; a pose no factor touches gets d = 0
    rng = dg.Stream(11)
    pairs, H, b = _random_system(rng, 8, rank=6)
    pairs = np.where(pairs == 7, 6, pairs)          # pose 7 is now untouched
    got, _ = vg.vgicp_solve_step(pairs, H, b, 8, 0, 1e-2)
    ref, _ = oracle.gn_step(pairs, H, b, 8, 0, 1e-2)
    assert np.allclose(got, ref, rtol=1e-6, atol=1e-9 * np.abs(ref).max())
    assert not got[7].any()


def test_solve_step_errors():
    H = -np.eye(12)[None]
    b = np.ones((1, 12))
    with pytest.raises(vg.VgicpError) as e:
        vg.vgicp_solve_step(np.array([[0, 1]]), H, b, 2, 0, 0.0)
    assert e.value.status == 8                       # VGICP_ERR_NUMERIC
    with pytest.raises(vg.VgicpError):
        vg.vgicp_solve_step(np.array([[0, 5]]), np.eye(12)[None], b, 2, 0, 0.0)   # pose index out of range
    with pytest.raises(vg.VgicpError):
        vg.vgicp_solve_step(np.array([[0, 1]]), np.eye(12)[None], b, 2, 3, 0.0)   # anchor out of range


# ----------------------------------------------------- SE(3) loop factors --

def test_oracle_se3_log_inverts_exp():
    rng = dg.Stream(21)
    for scale in (1e-6, 0.1, 1.0, 2.5):
        xi = rng.normal(6) * scale
        if np.linalg.norm(xi[:3]) >= np.pi:
            continue
        assert np.allclose(oracle.se3_log(oracle.se3_exp(xi)), xi, rtol=0, atol=1e-10 * max(1.0, scale))


def test_oracle_tukey_loss_derivative_is_the_weight():
    # d rho / d(x^2) = weight(x); the weight peaks at the offset and vanishes outside the support
    for w, o in ((1.0, 0.0), (4.0, 1.5), (0.25, 3.0)):
        assert oracle.tukey_weight(o, w, o) == 1.0
        assert oracle.tukey_weight(o + np.sqrt(w) * 1.0001, w, o) == 0.0
        for x in (0.3, 1.0, 2.2, 3.4):
            h = 1e-5
            d = (oracle.tukey_loss(x + h, w, o) - oracle.tukey_loss(x - h, w, o)) / ((x + h) ** 2 - (x - h) ** 2)
            assert d == pytest.approx(oracle.tukey_weight(x, w, o), abs=1e-7)
        far = o + np.sqrt(w) + 1.0
        assert oracle.tukey_loss(far, w, o) == pytest.approx(oracle.tukey_loss(far + 5.0, w, o), rel=1e-12)


@pytest.mark.parametrize("offset,width", [(0.0, 4.0), (0.5, 2.0), (2.0, 9.0)])
def test_loop_factor_matches_oracle(offset, width):
    rng = dg.Stream(int(40 + 10 * offset))
    poses = np.stack([dg.random_pose(rng, 40, 20.0) for _ in range(4)])
    # measurements near the current relative poses: residuals of a few degrees / decimetres
    Tij = []
    pi, pj = [0, 1, 3], [2, 3, 0]
    for i, j in zip(pi, pj):
        rel = np.linalg.inv(oracle._h(poses[i])) @ oracle._h(poses[j])
        Tij.append(dg.compose(rel[:3], dg.random_pose(rng, 4, 0.2)))
    A = rng.normal(36).reshape(6, 6)
    info = A @ A.T + 6 * np.eye(6)
    loops = vg.make_loop_factors(pi, pj, np.stack(Tij), info, width, offset)
    H, b, cost = vg.vgicp_loop_linearize(loops, poses)
    for k, (i, j) in enumerate(zip(pi, pj)):
        c_ref, H_ref, b_ref = oracle.loop_factor(poses[i], poses[j], Tij[k], info, width, offset)
        assert cost[k] == pytest.approx(c_ref, rel=1e-9, abs=1e-12)
        assert np.allclose(H[k], H_ref, rtol=1e-4, atol=1e-6 * max(1.0, np.abs(H_ref).max()))
        assert np.allclose(b[k], b_ref, rtol=1e-4, atol=1e-6 * max(1.0, np.abs(b_ref).max()))


def _loop_graph(rng, n_poses, reach=12):
    """A pose graph shaped like the paper-scale loop: factors between poses up to
    `reach` apart and between the two ends (loop closure), rank-6 factor blocks."""
    pairs = [(i, j) for j in range(n_poses) for i in range(max(0, j - reach), j)]
    pairs += [(i, j) for j in range(n_poses - reach, n_poses) for i in range(reach)]
    H, b = [], []
    for _ in pairs:
        G = rng.normal(6 * 12).reshape(6, 12)
        H.append(G.T @ G)
        b.append(rng.normal(12))
    return np.array(pairs), np.array(H), np.array(b)


def test_solve_step_loop_graph_matches_oracle():
    # 160 poses: envelope rows of ~150 columns, so the blocked factorisation runs its
    # vector loops and their tails on every block pair
    rng = dg.Stream(909)
    pairs, H, b = _loop_graph(rng, 160)
    got, gdec = vg.vgicp_solve_step(pairs, H, b, 160, 0, 1e-3)
    ref, rdec = oracle.gn_step(pairs, H, b, 160, 0, 1e-3)
    assert np.allclose(got, ref, rtol=1e-7, atol=1e-9 * np.abs(ref).max())
    assert gdec == pytest.approx(rdec, rel=1e-7)


def test_solve_step_portable_factorisation_agrees():
    """The same solve with the host's vector instructions switched off (VGICP_HOST_SIMD=0,
    read once per process, so in a child process) gives the same step to rounding."""
    import json
    import subprocess
    import sys
    rng = dg.Stream(910)
    pairs, H, b = _loop_graph(rng, 60)
    got, _ = vg.vgicp_solve_step(pairs, H, b, 60, 0, 1e-3)
    code = ("import json, sys, numpy as np; sys.path.insert(0, %r); import paper_2109_07073_b300 as vg; "
            "d = json.load(sys.stdin); "
            "x, _ = vg.vgicp_solve_step(np.array(d['p']), np.array(d['H']), np.array(d['b']), 60, 0, 1e-3); "
            "print(json.dumps(x.tolist()))") % ROOT
    env = dict(os.environ, VGICP_HOST_SIMD="0")
    res = subprocess.run([sys.executable, "-c", code], input=json.dumps({"p": pairs.tolist(), "H": H.tolist(),
                                                                         "b": b.tolist()}),
                         capture_output=True, text=True, env=env, timeout=300)
    assert res.returncode == 0, res.stderr
    plain = np.array(json.loads(res.stdout))
    assert np.allclose(plain, got, rtol=1e-9, atol=1e-12 * np.abs(got).max())
