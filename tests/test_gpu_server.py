"""Serving loop: results are bit-identical to the same request run alone.

Client threads submit a mix of linearisation (Eq. 3-6) and overlap (Eq. 8)
requests of uneven size; each result must equal, bit for bit, a plain context
call on the same data (vgicp_linearize with T_target = I, T_source = T_BA;
vgicp_overlap), with and without a device-memory budget that forces evictions.
One request is also checked against the FP64 oracle.
"""
import threading

import numpy as np
import pytest

import datagen as dg
import oracle
import paper_2109_07073_b300 as vg
from util import err_metric

pytestmark = pytest.mark.gpu

IDENT = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)


@pytest.fixture(scope="module")
def data():
    ids = [0, 1, 2, 3, 5, 8, 13, 21]
    g = dg.graph_workload(n_frames=24, n_points=12000, frame_ids=ids)
    rng = dg.Stream(4242)
    sizes = dg.log_uniform_sizes(rng, len(ids), 500, 12000)
    frames = {}
    maps = {}
    with vg.Context() as ctx:
        for k, i in enumerate(ids):
            p = g.points[i]
            c = ctx.estimate_covariances(p, 10, 1e-3)
            maps[i] = (p, c, (1.0, 0.5, 2.0)[k % 3])
            sel = np.sort(rng.choose(p.shape[0], int(sizes[k])))
            frames[i] = (p[sel], c[sel])
    reqs = []
    for q in range(96):
        t = ids[int(rng.uniform(1, 0, len(ids))[0])]
        s = ids[int(rng.uniform(1, 0, len(ids))[0])]
        T = oracle.relative_pose(g.poses[t], g.poses[s])
        kind = vg.VGICP_REQ_OVERLAP if q % 3 == 0 else vg.VGICP_REQ_LINEARIZE
        reqs.append((kind, t, s, T))
    return maps, frames, reqs


def alone(maps, frames, reqs):
    out = []
    with vg.Context() as ctx:
        hm = {k: ctx.build_voxelmap(p, c, r) for k, (p, c, r) in maps.items()}
        hf = {k: ctx.add_frame(p, c) for k, (p, c) in frames.items()}
        for kind, t, s, T in reqs:
            if kind == vg.VGICP_REQ_LINEARIZE:
                f = vg.make_factors([hm[t]], [hf[s]], [0], [1])
                H, b, cost, inl = ctx.linearize(f, np.stack([IDENT, T]))
                out.append((H[0], b[0], cost[0], inl[0]))
            else:
                out.append(ctx.overlap_pairs([hf[s]], [hm[t]], T[None])[0])
    return out


def serve(maps, frames, reqs, clients=4, **opts):
    with vg.Server(**opts) as srv:
        for k, (p, c, r) in maps.items():
            srv.put_map(k, p, c, r)
        for k, (p, c) in frames.items():
            srv.put_frame(k, p, c)
        res = [None] * len(reqs)

        def client(j):
            mine = list(range(j, len(reqs), clients))
            if j % 2:      # odd clients queue all their requests in one call
                tickets = srv.submit_batch([reqs[i][0] for i in mine], [reqs[i][1] for i in mine],
                                           [reqs[i][2] for i in mine], np.stack([reqs[i][3] for i in mine]))
                tickets = [int(t) for t in tickets]
            else:
                tickets = [srv.submit(reqs[i][0], reqs[i][1], reqs[i][2], reqs[i][3]) for i in mine]
            for i, tk in zip(mine, tickets):
                res[i] = srv.wait(tk, 120.0)
        th = [threading.Thread(target=client, args=(j,)) for j in range(clients)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        return res, srv.stats()


def check_identical(reqs, res, ref):
    for i, ((kind, t, s, T), r, a) in enumerate(zip(reqs, res, ref)):
        assert r is not None and r.status == vg.VGICP_OK, (i, r.status if r else None)
        if kind == vg.VGICP_REQ_LINEARIZE:
            H, b, cost, inl = a
            assert np.array_equal(np.array(r.H).reshape(12, 12), H), i
            assert np.array_equal(np.array(r.b), b), i
            assert r.cost == cost and r.count == inl, i
        else:
            assert r.count == a, i


def test_server_mix_matches_alone(data):
    maps, frames, reqs = data
    ref = alone(maps, frames, reqs)
    res, st = serve(maps, frames, reqs)
    check_identical(reqs, res, ref)
    assert st.completed == len(reqs) and st.submitted == len(reqs)
    assert st.evictions == 0 and st.batches >= 1
    assert 0 < st.p50_ms <= st.p99_ms <= st.max_ms


def test_server_budget_evicts_and_matches(data):
    maps, frames, reqs = data
    ref = alone(maps, frames, reqs)
    _, st = serve(maps, frames, reqs, clients=1)
    full = st.resident_bytes
    res, st = serve(maps, frames, reqs, clients=3, hbm_budget_bytes=int(full * 0.4), lanes=2)
    check_identical(reqs, res, ref)
    assert st.evictions > 0 and st.resident_bytes <= int(full * 0.4)


@pytest.mark.parametrize("lanes", [2, 4])
def test_server_small_batches_across_lanes_under_eviction(data, lanes):
    """Batches of at most two requests on two or four lanes under a budget of a
    third of the working set: an object admitted (copied, built, its descriptor
    written) by one lane's batch is used, or evicted, by the next batch on
    another lane while that admission may still be in flight.  Every result
    equals the request run alone, bit for bit."""
    maps, frames, reqs = data
    reqs = reqs * 3
    ref = alone(maps, frames, reqs)
    _, st = serve(maps, frames, reqs[:len(reqs) // 3], clients=1)
    full = st.resident_bytes
    res, st = serve(maps, frames, reqs, clients=4, hbm_budget_bytes=int(full * 0.34), lanes=lanes,
                    max_batch_requests=2)
    check_identical(reqs, res, ref)
    assert st.evictions > 0 and st.batches >= len(reqs) // 2


def test_server_vs_oracle(data):
    maps, frames, reqs = data
    kind, t, s, T = next(r for r in reqs if r[0] == vg.VGICP_REQ_LINEARIZE)
    res, _ = serve(maps, frames, [(kind, t, s, T)], clients=1)
    p, c, r = maps[t]
    L = oracle.linearize(oracle.voxelmap(p, c, r), frames[s][0], frames[s][1], T)
    out = res[0]
    assert out.count == L.inliers
    assert err_metric(np.array(out.H).reshape(12, 12), L.H, L.SH) <= 1e-4
    assert err_metric(np.array(out.b), L.b, L.Sb) <= 1e-4
    assert abs(out.cost - L.cost) / L.Scost <= 1e-4


def test_server_errors(data):
    maps, frames, _ = data
    with vg.Server(hbm_budget_bytes=4096) as srv:
        p, c, r = maps[0]
        srv.put_map(0, p, c, r)
        srv.put_frame(0, *frames[0])
        srv.put_frame(1, np.zeros((0, 3), np.float32), np.zeros((0, 6), np.float32))
        with pytest.raises(vg.VgicpError):
            srv.put_map(0, p, c, r)                               # key taken
        with pytest.raises(vg.VgicpError):
            srv.submit(vg.VGICP_REQ_LINEARIZE, 7, 0, IDENT)       # unknown map
        with pytest.raises(vg.VgicpError):
            srv.submit(vg.VGICP_REQ_LINEARIZE, 0, 0, np.full((3, 4), np.nan))
        tk = srv.submit(vg.VGICP_REQ_LINEARIZE, 0, 0, IDENT)
        assert srv.wait(tk, 60.0).status == 7                    # VGICP_ERR_BUDGET: cannot fit
    with vg.Server() as srv:
        srv.put_map(0, p, c, r)
        srv.put_frame(1, np.zeros((0, 3), np.float32), np.zeros((0, 6), np.float32))
        r1 = srv.wait(srv.submit(vg.VGICP_REQ_OVERLAP, 0, 1, IDENT), 60.0)
        r2 = srv.wait(srv.submit(vg.VGICP_REQ_LINEARIZE, 0, 1, IDENT), 60.0)
        assert r1.status == 4 and r1.count == 0                  # VGICP_ERR_EMPTY (Eq. 8 undefined)
        assert r2.status == vg.VGICP_OK and r2.count == 0 and r2.cost == 0.0
        assert not np.any(np.array(r2.H))


def test_server_wait_timeout_keeps_the_ticket(data):
    """A wait that runs out returns VGICP_ERR_TIMEOUT and leaves the ticket valid: a
    later wait gets the same result as a request that was never timed out."""
    maps, frames, _ = data
    p, c, r = maps[0]
    with vg.Server() as srv:
        srv.put_map(0, p, c, r)
        srv.put_frame(0, *frames[0])
        first = srv.wait(srv.submit(vg.VGICP_REQ_LINEARIZE, 0, 0, IDENT), 60.0)
        timed_out = 0
        for _ in range(8):
            tk = srv.submit(vg.VGICP_REQ_LINEARIZE, 0, 0, IDENT)
            try:
                srv.wait(tk, 0.0)                                 # no time to run: runs out
            except vg.VgicpError as e:
                assert e.status == 6                              # VGICP_ERR_TIMEOUT
                timed_out += 1
                res = srv.wait(tk, 60.0)
                assert res.status == vg.VGICP_OK and res.cost == first.cost
                assert np.array_equal(np.array(res.H), np.array(first.H))
        assert timed_out > 0
        tks = [srv.submit(vg.VGICP_REQ_LINEARIZE, 0, 0, IDENT) for _ in range(4)]
        try:
            srv.wait_batch(tks, 0.0)
        except vg.VgicpError as e:
            assert e.status == 6
        for tk in tks:                                            # retired or still valid
            try:
                assert srv.wait(tk, 60.0).cost == first.cost
            except vg.VgicpError as e:
                assert e.status == 3                              # VGICP_ERR_NOT_FOUND: retired by the batch
