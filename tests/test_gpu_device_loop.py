"""Device-resident request loop (server option device_loop).

A persistent kernel takes requests from a ring of mapped host slots as the
server publishes them, while earlier requests are still running; each result
must equal, bit for bit, a plain context call on the same data
(vgicp_linearize with T_target = I, T_source = T_BA; vgicp_overlap_pairs),
whether the request ran alone or among others, with few or many slots, and
with a budget that forces evictions.  The loop's own wait is bounded: with no
request for loop_idle_ms the kernel ends with VGICP_ERR_TIMEOUT, and the next
request starts it again.
"""
import time

import numpy as np
import pytest

import oracle
import paper_2109_07073_b300 as vg
from test_gpu_server import IDENT, alone, check_identical, data, serve  # noqa: F401  (data: fixture)
from util import err_metric

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("slots", [0, 8])
def test_device_loop_mix_matches_alone(data, slots):
    maps, frames, reqs = data
    ref = alone(maps, frames, reqs)
    res, st = serve(maps, frames, reqs, device_loop=True, loop_slots=slots)
    check_identical(reqs, res, ref)
    assert st.completed == len(reqs) and st.submitted == len(reqs)
    assert st.evictions == 0 and st.batches >= 1           # batches: launches of the loop kernel
    assert 0 < st.p50_ms <= st.p99_ms <= st.max_ms


def test_device_loop_requests_one_at_a_time_match(data):
    """Each request alone in the loop (submitted only after the previous one finished)."""
    maps, frames, reqs = data
    ref = alone(maps, frames, reqs[:24])
    with vg.Server(device_loop=True) as srv:
        for k, (p, c, r) in maps.items():
            srv.put_map(k, p, c, r)
        for k, (p, c) in frames.items():
            srv.put_frame(k, p, c)
        res = [srv.wait(srv.submit(kind, t, s, T), 60.0) for kind, t, s, T in reqs[:24]]
    check_identical(reqs[:24], res, ref)


def test_device_loop_budget_evicts_and_matches(data):
    maps, frames, reqs = data
    ref = alone(maps, frames, reqs)
    _, st = serve(maps, frames, reqs, clients=1, device_loop=True)
    full = st.resident_bytes
    res, st = serve(maps, frames, reqs, clients=3, hbm_budget_bytes=int(full * 0.4), device_loop=True)
    check_identical(reqs, res, ref)
    assert st.evictions > 0 and st.resident_bytes <= int(full * 0.4)


def test_device_loop_vs_oracle(data):
    maps, frames, reqs = data
    kind, t, s, T = next(r for r in reqs if r[0] == vg.VGICP_REQ_LINEARIZE)
    res, _ = serve(maps, frames, [(kind, t, s, T)], clients=1, device_loop=True)
    p, c, r = maps[t]
    L = oracle.linearize(oracle.voxelmap(p, c, r), frames[s][0], frames[s][1], T)
    out = res[0]
    assert out.count == L.inliers
    assert err_metric(np.array(out.H).reshape(12, 12), L.H, L.SH) <= 1e-4
    assert err_metric(np.array(out.b), L.b, L.Sb) <= 1e-4
    assert abs(out.cost - L.cost) / L.Scost <= 1e-4


def test_device_loop_idle_limit_ends_the_kernel_with_timeout(data):
    """No request for longer than loop_idle_ms (nothing is written to the ring): the
    loop kernel ends by itself and reports VGICP_ERR_TIMEOUT; the next request
    launches it again and gets the same result."""
    maps, frames, _ = data
    p, c, r = maps[0]
    with vg.Server(device_loop=True, loop_idle_ms=2.0) as srv:
        srv.put_map(0, p, c, r)
        srv.put_frame(0, *frames[0])
        assert srv.loop_state() == (False, vg.VGICP_OK, 0)
        first = srv.wait(srv.submit(vg.VGICP_REQ_LINEARIZE, 0, 0, IDENT), 60.0)
        assert first.status == vg.VGICP_OK
        deadline = time.time() + 10.0
        while srv.loop_state()[0] and time.time() < deadline:
            time.sleep(0.01)
        running, last, launches = srv.loop_state()
        assert not running and last == 6 and launches == 1      # VGICP_ERR_TIMEOUT
        again = srv.wait(srv.submit(vg.VGICP_REQ_LINEARIZE, 0, 0, IDENT), 60.0)
        assert again.status == vg.VGICP_OK and again.cost == first.cost
        assert np.array_equal(np.array(again.H), np.array(first.H))
        assert srv.loop_state()[2] == 2


def test_device_loop_errors(data):
    maps, frames, _ = data
    p, c, r = maps[0]
    with vg.Server(device_loop=True, hbm_budget_bytes=4096) as srv:
        srv.put_map(0, p, c, r)
        srv.put_frame(0, *frames[0])
        tk = srv.submit(vg.VGICP_REQ_LINEARIZE, 0, 0, IDENT)
        assert srv.wait(tk, 60.0).status == 7                    # VGICP_ERR_BUDGET: cannot fit
    with vg.Server(device_loop=True) as srv:
        srv.put_map(0, p, c, r)
        srv.put_frame(1, np.zeros((0, 3), np.float32), np.zeros((0, 6), np.float32))
        r1 = srv.wait(srv.submit(vg.VGICP_REQ_OVERLAP, 0, 1, IDENT), 60.0)
        r2 = srv.wait(srv.submit(vg.VGICP_REQ_LINEARIZE, 0, 1, IDENT), 60.0)
        assert r1.status == 4 and r1.count == 0                  # VGICP_ERR_EMPTY (Eq. 8 undefined)
        assert r2.status == vg.VGICP_OK and r2.count == 0 and r2.cost == 0.0
    ko = vg.vgicp_options_default()
    ko.neighbors = 7
    with pytest.raises(vg.VgicpError):
        vg.Server(device_loop=True, kernel_options=ko)          # the loop runs the single-voxel association
    with pytest.raises(vg.VgicpError):
        vg.Server(device_loop=True, loop_slots=4096)
    with vg.Server() as srv:
        with pytest.raises(vg.VgicpError):
            srv.loop_state()                                     # not a device-loop server
