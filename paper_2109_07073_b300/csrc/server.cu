// Serving loop: an online mapper submits linearisation (Eq. 3-6) and overlap
// (Eq. 8) requests of uneven size; they run in continuous batches.
//
//   * Clients register target clouds (built into voxelmaps on the device when
//     needed) and source frames under their own keys; the server keeps host
//     copies and makes objects resident on demand, evicting the least recently
//     used idle objects when the device-memory budget would be exceeded.
//   * One scheduler thread owns the context.  Whenever a lane (a CUDA stream
//     with its own scratch) is free and requests are pending, it admits as many
//     pending requests as the batch limits and the budget allow and launches
//     them as one batched linearisation plus one batched overlap list; requests
//     that arrive meanwhile form the next batch on another lane, so their work
//     overlaps on the device with the batch in flight.  Requests that do not
//     fit the budget wait until objects of finished batches become evictable.
//   * A host callback on the lane's stream marks the batch done; the scheduler
//     copies each request's result out and wakes its waiter.
// A request's result does not depend on the batch it ran in: a factor's sums
// use fixed chunks and a fixed reduction order, and overlap counts are exact.
//
// Device-loop mode (options.device_loop): the scheduler thread admits each
// request (residency as above), writes it into a ring of page-locked,
// device-mapped request slots and keeps one persistent kernel running that
// takes requests from the ring as they are published (see the request loop in
// linearize.cu); finished results appear in the mapped result slots, where the
// scheduler reads them.  The loop kernel ends on its own after loop_idle_ms
// without a request and is launched again for the next one.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include <cuda_runtime.h>

#include "kernels.cuh"
#include "vgicp.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Resident {
    bool is_map = false;
    const float *pts = nullptr, *covs = nullptr;   // host copies (immutable once registered)
    std::vector<float> own;         // their storage when no page-locked slab could be had
    int64_t n = 0;
    double r = 0.0;
    int64_t handle = -1;            // device handle while resident
    uint64_t last_use = 0;
    int64_t key = 0;                // tagged key (position in the LRU order: (last_use, key))
    int pins = 0;                   // batches in flight that use it
    int64_t bytes = 0;              // device bytes it holds while resident
    cudaEvent_t ready = nullptr;    // recorded after the object's admission (on the admitting stream)
    bool ready_done = true;         // ... and seen complete
};

struct Pending {
    vgicp_request req;
    Clock::time_point t0;
    vgicp_result res;
    bool done = false;
};

struct LaneState {
    cudaStream_t stream = nullptr;
    bool busy = false;
    std::atomic<bool> finished{false};
    std::pair<vgicp_server *, int> cb;      // host-callback argument
    std::vector<int64_t> lin, ovl;          // tickets of the batch
    std::vector<int64_t> pinned;            // tagged keys pinned by the batch
    double *dH = nullptr, *db = nullptr, *dc = nullptr;
    int64_t *di = nullptr, *dcount = nullptr;
    double *hH = nullptr, *hb = nullptr, *hc = nullptr;
    int64_t *hi = nullptr, *hcount = nullptr;
    int64_t cap = 0;
    vgicp_status status = VGICP_OK;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;   // device time of the batch
};

}  // namespace

struct vgicp_server {
    vgicp_ctx *ctx = nullptr;
    vgicp_server_options opt{};
    std::thread thr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::unordered_map<int64_t, Resident> objs;   // tagged key -> object (references stay valid)
    std::set<std::pair<uint64_t, int64_t>> lru;   // resident objects by (last use, tagged key)
    std::deque<int64_t> pending;
    std::unordered_map<int64_t, Pending> reqs;
    int64_t next_ticket = 1;
    uint64_t clock = 0;
    int nl = 2;
    LaneState lanes[4];
    std::vector<double> lat_ms;
    int64_t resident_bytes = 0;
    double host_launch_ms = 0.0, host_finish_ms = 0.0, device_ms = 0.0, host_admit_ms = 0.0, host_enqueue_ms = 0.0;
    int64_t submitted = 0, completed = 0, batches = 0, admissions = 0, evictions = 0, batch_requests = 0;
    std::string err;
    // page-locked host copies of the registered objects, bump-allocated in slabs
    // that live as long as the server (re-admission copies them directly)
    std::vector<char *> slabs;
    size_t slab_cap = 0, slab_off = 0;
    // device-loop mode
    bool dloop = false;
    int chunk = 2048, cull = 1, num_sms = 148;
    int slots = 0;
    unsigned int qcap = 0;
    vg::LoopRequest *h_req = nullptr, *d_req = nullptr;      // mapped ring (host / device views)
    vg::LoopResult *h_res = nullptr, *d_res = nullptr;
    vg::LoopExit *h_exit = nullptr, *d_exit = nullptr;
    vg::LoopControl *d_ctl = nullptr, *h_ctl = nullptr;      // h_ctl: pinned staging of the control words
    vg::LoopSlotState *d_state = nullptr;
    double *d_partials = nullptr;
    long long *d_counts = nullptr;
    int2 *d_queue = nullptr;
    cudaStream_t loop_stream = nullptr;
    cudaEvent_t loop_ev0 = nullptr, loop_ev1 = nullptr;
    bool loop_running = false;
    int loop_last_exit = VGICP_OK;
    int64_t loop_launches = 0;
    unsigned long long n_pub = 0;                            // requests published so far
    double idle_ms = 20.0;
    std::vector<int64_t> slot_ticket;                        // ticket in each slot, -1 when free
    std::vector<unsigned long long> slot_seq;
    std::vector<std::pair<int64_t, int64_t>> slot_keys;      // tagged keys the slot's request pins
    std::vector<int> inflight;                               // slots with a request in flight
    std::vector<int64_t> waiting;                            // admitted, objects' copies / builds in flight
    std::deque<int64_t> ready_q;                             // objects ready, waiting for a ring slot
};

namespace {

inline int64_t tag(int64_t key, bool is_map) { return (int64_t)(((uint64_t)key << 1) | (is_map ? 1u : 0u)); }

void CUDART_CB lane_done(void *p)
{
    auto *a = static_cast<std::pair<vgicp_server *, int> *>(p);
    vgicp_server *s = a->first;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->lanes[a->second].finished.store(true);
    }
    s->cv_work.notify_all();
}

// An object's admission (copy, build, descriptor update) is enqueued on the
// context's current stream; its ready event marks where that work ends
// (scheduler thread).
vgicp_status mark_admitted(vgicp_server *s, Resident &o)
{
    vg::CtxView v;
    vg::ctx_view(s->ctx, &v);
    if (!o.ready && cudaEventCreateWithFlags(&o.ready, cudaEventDisableTiming) != cudaSuccess) return VGICP_ERR_CUDA;
    if (cudaEventRecord(o.ready, v.stream) != cudaSuccess) return VGICP_ERR_CUDA;
    o.ready_done = false;
    return VGICP_OK;
}

// Order the context's current stream after object o's admission, which may
// have been enqueued on another lane's stream: work that reads the object, or
// frees its memory and reuses its descriptor slot, must not overtake it
// (scheduler thread; nothing to do once the admission is seen complete).
vgicp_status after_admission(vgicp_server *s, Resident &o)
{
    if (o.ready_done || !o.ready) return VGICP_OK;
    const cudaError_t q = cudaEventQuery(o.ready);
    if (q == cudaSuccess) {
        o.ready_done = true;
        return VGICP_OK;
    }
    if (q != cudaErrorNotReady) return VGICP_ERR_CUDA;
    vg::CtxView v;
    vg::ctx_view(s->ctx, &v);
    return cudaStreamWaitEvent(v.stream, o.ready, 0) == cudaSuccess ? VGICP_OK : VGICP_ERR_CUDA;
}

// Release the least recently used idle resident object (scheduler thread).
bool evict_one(vgicp_server *s)
{
    Resident *best = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto it = s->lru.begin(); it != s->lru.end(); ++it) {   // pinned objects are few: skip them
            Resident &o = s->objs[it->second];
            if (o.pins == 0) {
                best = &o;
                s->lru.erase(it);
                break;
            }
        }
        if (!best) return false;
        ++s->evictions;
    }
    // the free and the reuse of the object's descriptor slot come after its admission
    if (after_admission(s, *best) != VGICP_OK) {
        vg::CtxView v;
        vg::ctx_view(s->ctx, &v);
        cudaStreamSynchronize(v.stream);
        if (best->ready) cudaEventSynchronize(best->ready);
    }
    vgicp_release(s->ctx, best->handle);
    best->handle = -1;
    return true;
}

// Device bytes an object holds once resident; for a map with the temporary
// frame it is built from, which is held until the build is queued.
int64_t object_bytes(vgicp_server *s, const Resident &o)
{
    int64_t b = 0, fb = 0;
    vgicp_memory_estimate(s->ctx, o.n, o.is_map ? 1 : 0, &b);
    if (o.is_map) vgicp_memory_estimate(s->ctx, o.n, 0, &fb);
    return b + fb;
}

// Make the distinct, non-resident objects `miss` resident in one batched pass
// on the context's current stream (scheduler thread; the caller has made room
// for them): one registration of every missing frame and of a temporary frame
// per missing map, one voxelmap build per resolution, the temporary frames
// released once their builds are queued, and each object's ready event
// recorded after all of it.  All or nothing.
vgicp_status admit_many(vgicp_server *s, const std::vector<Resident *> &miss)
{
    const size_t k = miss.size();
    if (k == 0) return VGICP_OK;
    std::vector<const float *> P(k), C(k);
    std::vector<int64_t> N(k), H(k, -1), MH(k, -1);
    for (size_t i = 0; i < k; ++i) {
        P[i] = miss[i]->pts;
        C[i] = miss[i]->covs;
        N[i] = miss[i]->n;
    }
    vgicp_status st = (vgicp_status)vg::ctx_add_frames_gather(s->ctx, P.data(), C.data(), N.data(), (int64_t)k,
                                                              H.data());
    if (st != VGICP_OK) return st;
    std::vector<size_t> maps;
    for (size_t i = 0; i < k; ++i)
        if (miss[i]->is_map) maps.push_back(i);
    std::vector<char> built(maps.size(), 0);
    for (size_t a = 0; a < maps.size() && st == VGICP_OK; ++a) {
        if (built[a]) continue;
        const double r = miss[maps[a]]->r;
        std::vector<int64_t> fr, out;
        std::vector<size_t> who;
        for (size_t b = a; b < maps.size(); ++b)
            if (!built[b] && miss[maps[b]]->r == r) {
                built[b] = 1;
                fr.push_back(H[maps[b]]);
                who.push_back(maps[b]);
            }
        out.assign(fr.size(), -1);
        st = vgicp_build_voxelmaps(s->ctx, fr.data(), (int64_t)fr.size(), r, out.data());
        if (st == VGICP_OK)
            for (size_t j = 0; j < who.size(); ++j) MH[who[j]] = out[j];
    }
    for (size_t i : maps) vgicp_release(s->ctx, H[i]);
    if (st != VGICP_OK) {
        for (size_t i = 0; i < k; ++i) {
            if (!miss[i]->is_map) vgicp_release(s->ctx, H[i]);
            else if (MH[i] >= 0) vgicp_release(s->ctx, MH[i]);
        }
        return st;
    }
    for (size_t i = 0; i < k; ++i) {
        Resident &o = *miss[i];
        o.handle = o.is_map ? MH[i] : H[i];
        vgicp_memory_estimate(s->ctx, o.n, o.is_map ? 1 : 0, &o.bytes);
        const vgicp_status ev = mark_admitted(s, o);
        std::lock_guard<std::mutex> lk(s->mu);
        o.last_use = ++s->clock;
        s->lru.insert({o.last_use, o.key});
        ++s->admissions;
        if (ev != VGICP_OK) st = ev;
    }
    return st;
}

// Requests admitted together at most (their missing objects in one pass).
constexpr size_t kAdmitGroup = 64;

// Make the objects of requests ts resident (scheduler thread, mutex not held).
// From the front, as many requests are taken as the budget can hold once the
// idle resident objects that those requests do not use are counted as free;
// least recently used idle objects are evicted to make exactly that room, the
// taken requests' missing objects are admitted together, and both objects of
// each taken request stay pinned until its result is read: those requests go
// to ok.  The rest go to deferred with nothing pinned (all of them when even
// the first does not fit).  When the admission fails other than for the
// budget, the taken requests go to failed and fail_status says why.
void prepare_group(vgicp_server *s, const std::vector<int64_t> &ts, std::vector<int64_t> &ok,
                   std::vector<int64_t> &deferred, std::vector<int64_t> &failed, vgicp_status &fail_status)
{
    const size_t nt = ts.size();
    std::vector<Resident *> m(nt), f(nt);
    // need[k]: bytes the missing objects of the first k requests take (each
    // once); kept[k]: bytes of the idle resident objects those requests use,
    // which cannot be evicted for them
    std::vector<int64_t> need(nt + 1, 0), kept(nt + 1, 0);
    std::vector<Resident *> order;                     // missing objects in first-use order
    std::vector<size_t> first_req;                     // the request that needs each first
    int64_t idle = 0;                                  // bytes held by evictable objects
    size_t take = nt;
    const auto ta = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        std::unordered_set<Resident *> seen;
        for (size_t i = 0; i < nt; ++i) {
            const vgicp_request &r = s->reqs[ts[i]].req;
            m[i] = &s->objs[tag(r.target, true)];
            f[i] = &s->objs[tag(r.source, false)];
            need[i + 1] = need[i];
            kept[i + 1] = kept[i];
            for (Resident *o : {m[i], f[i]}) {
                if (!seen.insert(o).second) continue;
                if (o->handle < 0) {
                    order.push_back(o);
                    first_req.push_back(i);
                    need[i + 1] += object_bytes(s, *o);
                } else if (o->pins == 0) {
                    kept[i + 1] += o->bytes;
                }
            }
        }
        int64_t used = 0;
        if (s->opt.hbm_budget_bytes > 0 && need[nt] > 0) vgicp_memory_in_use(s->ctx, &used);
        // only a group that does not fit as things stand walks the resident objects
        if (s->opt.hbm_budget_bytes > 0 && need[nt] > 0 && used + need[nt] > s->opt.hbm_budget_bytes) {
            for (const auto &e : s->lru) {
                const Resident &o = s->objs[e.second];
                if (o.pins == 0) idle += o.bytes;
            }
            const int64_t room = s->opt.hbm_budget_bytes - (used - idle);
            while (take > 0 && need[take] + kept[take] > room) --take;
        }
        for (size_t i = 0; i < take; ++i) {
            m[i]->pins++;
            f[i]->pins++;
        }
    }
    if (s->opt.hbm_budget_bytes > 0 && take > 0 && need[take] > 0) {
        int64_t used = 0;
        vgicp_memory_in_use(s->ctx, &used);
        while (used + need[take] > s->opt.hbm_budget_bytes && evict_one(s)) vgicp_memory_in_use(s->ctx, &used);
        // an estimate that fell short: fewer requests, down to none
        size_t k = take;
        while (k > 0 && used + need[k] > s->opt.hbm_budget_bytes) --k;
        std::lock_guard<std::mutex> lk(s->mu);
        for (size_t i = k; i < take; ++i) {
            m[i]->pins--;
            f[i]->pins--;
        }
        take = k;
    }
    std::vector<Resident *> miss;
    for (size_t j = 0; j < order.size() && first_req[j] < take; ++j) miss.push_back(order[j]);
    vgicp_status st = take ? admit_many(s, miss) : VGICP_OK;
    const double admit_ms = std::chrono::duration<double, std::milli>(Clock::now() - ta).count();
    std::lock_guard<std::mutex> lk(s->mu);
    s->host_admit_ms += admit_ms;
    if (st == VGICP_ERR_BUDGET) {                        // the allocation itself did not fit: later
        for (size_t i = 0; i < take; ++i) {
            m[i]->pins--;
            f[i]->pins--;
        }
        take = 0;
        st = VGICP_OK;
    }
    for (size_t i = 0; i < take; ++i) {
        if (st != VGICP_OK) {
            m[i]->pins--;
            f[i]->pins--;
            failed.push_back(ts[i]);
            continue;
        }
        for (Resident *o : {m[i], f[i]}) {
            s->lru.erase({o->last_use, o->key});
            o->last_use = ++s->clock;
            s->lru.insert({o->last_use, o->key});
        }
        ok.push_back(ts[i]);
    }
    fail_status = st;
    for (size_t i = take; i < nt; ++i) deferred.push_back(ts[i]);
}

vgicp_status ensure_lane_buffers(LaneState &L, int64_t n)
{
    if (n <= L.cap) return VGICP_OK;
    const int64_t cap = std::max<int64_t>(n, L.cap * 2);
    cudaFree(L.dH); cudaFree(L.db); cudaFree(L.dc); cudaFree(L.di); cudaFree(L.dcount);
    cudaFreeHost(L.hH); cudaFreeHost(L.hb); cudaFreeHost(L.hc); cudaFreeHost(L.hi); cudaFreeHost(L.hcount);
    L.dH = L.db = L.dc = L.hH = L.hb = L.hc = nullptr;
    L.di = L.dcount = L.hi = L.hcount = nullptr;
    L.cap = 0;
    if (cudaMalloc(&L.dH, cap * 144 * 8) || cudaMalloc(&L.db, cap * 12 * 8) || cudaMalloc(&L.dc, cap * 8) ||
        cudaMalloc(&L.di, cap * 8) || cudaMalloc(&L.dcount, cap * 8) || cudaMallocHost(&L.hH, cap * 144 * 8) ||
        cudaMallocHost(&L.hb, cap * 12 * 8) || cudaMallocHost(&L.hc, cap * 8) || cudaMallocHost(&L.hi, cap * 8) ||
        cudaMallocHost(&L.hcount, cap * 8))
        return VGICP_ERR_OOM;
    L.cap = cap;
    return VGICP_OK;
}

void complete(vgicp_server *s, int64_t t, vgicp_status st)   // mutex held
{
    Pending &p = s->reqs[t];
    p.res.status = st;
    p.res.kind = p.req.kind;
    p.res.latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - p.t0).count();
    p.done = true;
}

// Admit and launch one batch on lane li (scheduler thread, mutex not held).
// Returns the tickets deferred for lack of memory.
std::vector<int64_t> launch_batch(vgicp_server *s, int li, const std::vector<int64_t> &tickets)
{
    LaneState &L = s->lanes[li];
    L.lin.clear();
    L.ovl.clear();
    L.pinned.clear();
    std::vector<int64_t> deferred;
    std::vector<vgicp_factor> fac;
    std::vector<double> poses(12, 0.0);
    poses[0] = poses[5] = poses[10] = 1.0;               // pose 0: identity, so T_BA = T exactly
    std::vector<vgicp_frame_t> osrc;
    std::vector<vgicp_map_t> otgt;
    std::vector<double> oT;
    vgicp_set_lane(s->ctx, li, L.stream);
    std::vector<vgicp_request> rq(tickets.size());
    std::vector<Resident *> om(tickets.size()), of(tickets.size());
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (size_t k = 0; k < tickets.size(); ++k) {
            rq[k] = s->reqs[tickets[k]].req;
            om[k] = &s->objs[tag(rq[k].target, true)];
            of[k] = &s->objs[tag(rq[k].source, false)];
        }
    }
    fac.reserve(tickets.size());
    poses.reserve(12 * (tickets.size() + 1));
    // admission in groups; once a group leaves requests out for lack of room,
    // the rest of the batch waits with them (arrival order is kept)
    std::vector<char> admitted(tickets.size(), 0);
    size_t next = 0;
    while (next < tickets.size()) {
        const size_t end = std::min(tickets.size(), next + kAdmitGroup);
        const std::vector<int64_t> grp(tickets.begin() + (ptrdiff_t)next, tickets.begin() + (ptrdiff_t)end);
        std::vector<int64_t> ok, def, failed;
        vgicp_status fst = VGICP_OK;
        prepare_group(s, grp, ok, def, failed, fst);
        for (size_t k = next; k < next + ok.size(); ++k) admitted[k] = 1;   // ok is the group's front
        if (!failed.empty()) {
            std::lock_guard<std::mutex> lk(s->mu);
            for (int64_t t : failed) complete(s, t, fst);
        }
        if (!def.empty()) {
            deferred.assign(tickets.begin() + (ptrdiff_t)(next + ok.size() + failed.size()), tickets.end());
            break;
        }
        next = end;
    }
    for (size_t k = 0; k < tickets.size(); ++k) {
        if (!admitted[k]) continue;
        const int64_t t = tickets[k];
        const vgicp_request &r = rq[k];
        Resident *m = om[k], *f = of[k];
        // objects admitted by a batch on another lane may still be in transit:
        // this lane's work waits for their admission
        vgicp_status st = after_admission(s, *m);
        if (st == VGICP_OK) st = after_admission(s, *f);
        std::lock_guard<std::mutex> lk(s->mu);
        if (st != VGICP_OK) {
            m->pins--;
            f->pins--;
            complete(s, t, st);
            continue;
        }
        L.pinned.push_back(tag(r.target, true));           // pinned by the admission until finish
        L.pinned.push_back(tag(r.source, false));
        if (r.kind == VGICP_REQ_LINEARIZE) {
            vgicp_factor x;
            x.target = m->handle;
            x.source = f->handle;
            x.target_pose = 0;
            x.source_pose = (int32_t)(poses.size() / 12);
            poses.insert(poses.end(), r.T_target_source, r.T_target_source + 12);
            fac.push_back(x);
            L.lin.push_back(t);
        } else {
            osrc.push_back(f->handle);
            otgt.push_back(m->handle);
            oT.insert(oT.end(), r.T_target_source, r.T_target_source + 12);
            L.ovl.push_back(t);
        }
    }
    const size_t nf = fac.size(), no = osrc.size();
    const auto te = Clock::now();
    if (nf + no) cudaEventRecord(L.ev0, L.stream);
    vgicp_status st = ensure_lane_buffers(L, (int64_t)std::max<size_t>(std::max(nf, no), 1));
    if (st == VGICP_OK && nf)
        st = vgicp_linearize(s->ctx, fac.data(), (int64_t)nf, poses.data(), (int64_t)(poses.size() / 12), L.dH, L.db,
                             L.dc, L.di, VGICP_MEM_DEVICE);
    if (st == VGICP_OK && no)
        st = vgicp_overlap_pairs(s->ctx, osrc.data(), otgt.data(), (int64_t)no, oT.data(), L.dcount,
                                 VGICP_MEM_DEVICE);
    if (st == VGICP_OK && nf) {
        cudaMemcpyAsync(L.hH, L.dH, nf * 144 * 8, cudaMemcpyDeviceToHost, L.stream);
        cudaMemcpyAsync(L.hb, L.db, nf * 12 * 8, cudaMemcpyDeviceToHost, L.stream);
        cudaMemcpyAsync(L.hc, L.dc, nf * 8, cudaMemcpyDeviceToHost, L.stream);
        cudaMemcpyAsync(L.hi, L.di, nf * 8, cudaMemcpyDeviceToHost, L.stream);
    }
    if (st == VGICP_OK && no) cudaMemcpyAsync(L.hcount, L.dcount, no * 8, cudaMemcpyDeviceToHost, L.stream);
    L.status = st;
    if (nf + no) cudaEventRecord(L.ev1, L.stream);
    L.finished.store(false);
    if (nf + no && cudaLaunchHostFunc(L.stream, lane_done, &L.cb) != cudaSuccess) {
        cudaStreamSynchronize(L.stream);
        L.finished.store(true);
    }
    const double enq_ms = std::chrono::duration<double, std::milli>(Clock::now() - te).count();
    int64_t bytes = 0;
    vgicp_memory_in_use(s->ctx, &bytes);
    std::lock_guard<std::mutex> lk(s->mu);
    s->resident_bytes = bytes;
    s->host_enqueue_ms += enq_ms;
    return deferred;
}

void finish_batch(vgicp_server *s, int li)   // mutex held
{
    LaneState &L = s->lanes[li];
    const auto now = Clock::now();
    for (size_t i = 0; i < L.lin.size(); ++i) {
        Pending &p = s->reqs[L.lin[i]];
        p.res.status = L.status;
        p.res.kind = VGICP_REQ_LINEARIZE;
        if (L.status == VGICP_OK) {
            std::memcpy(p.res.H, L.hH + 144 * i, 144 * 8);
            std::memcpy(p.res.b, L.hb + 12 * i, 12 * 8);
            p.res.cost = L.hc[i];
            p.res.count = L.hi[i];
        }
        p.res.latency_ms = std::chrono::duration<double, std::milli>(now - p.t0).count();
        p.done = true;
        s->lat_ms.push_back(p.res.latency_ms);
    }
    for (size_t i = 0; i < L.ovl.size(); ++i) {
        Pending &p = s->reqs[L.ovl[i]];
        p.res.kind = VGICP_REQ_OVERLAP;
        p.res.status = L.status;
        if (L.status == VGICP_OK) {
            const int64_t n = s->objs[tag(p.req.source, false)].n;
            p.res.count = L.hcount[i];
            if (n == 0) p.res.status = VGICP_ERR_EMPTY;
            else p.res.fraction = (double)L.hcount[i] / (double)n;
        }
        p.res.latency_ms = std::chrono::duration<double, std::milli>(now - p.t0).count();
        p.done = true;
        s->lat_ms.push_back(p.res.latency_ms);
    }
    for (int64_t k : L.pinned) s->objs[k].pins--;
    float gms = 0.f;
    if (cudaEventElapsedTime(&gms, L.ev0, L.ev1) == cudaSuccess) s->device_ms += gms;
    s->completed += (int64_t)(L.lin.size() + L.ovl.size());
    ++s->batches;
    s->batch_requests += (int64_t)(L.lin.size() + L.ovl.size());
    L.busy = false;
}

void scheduler(vgicp_server *s)
{
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        // a failed context runs no host callbacks: a lane whose stream reports an
        // error is finished, with that status, so no waiter (nor the server's
        // destruction) waits for it forever
        for (int li = 0; li < s->nl; ++li) {
            LaneState &L = s->lanes[li];
            if (!L.busy || L.finished.load()) continue;
            const cudaError_t q = cudaStreamQuery(L.stream);
            if (q != cudaSuccess && q != cudaErrorNotReady) {
                s->err = cudaGetErrorString(q);
                L.status = VGICP_ERR_CUDA;
                L.finished.store(true);
            }
        }
        bool harvested = false;
        for (int li = 0; li < s->nl; ++li)
            if (s->lanes[li].busy && s->lanes[li].finished.load()) {
                const auto tf = Clock::now();
                finish_batch(s, li);
                s->host_finish_ms += std::chrono::duration<double, std::milli>(Clock::now() - tf).count();
                harvested = true;
            }
        if (harvested) s->cv_done.notify_all();
        bool any_busy = false;
        int free_lane = -1;
        for (int li = 0; li < s->nl; ++li) {
            any_busy = any_busy || s->lanes[li].busy;
            if (!s->lanes[li].busy && free_lane < 0) free_lane = li;
        }
        if (s->stop && !any_busy) return;
        if (!s->stop && free_lane >= 0 && !s->pending.empty()) {
            std::vector<int64_t> take;
            int64_t pts = 0;
            while (!s->pending.empty() && (int)take.size() < s->opt.max_batch_requests) {
                const int64_t t = s->pending.front();
                const int64_t n = s->objs[tag(s->reqs[t].req.source, false)].n;
                if (!take.empty() && pts + n > s->opt.max_batch_points) break;
                pts += n;
                take.push_back(t);
                s->pending.pop_front();
            }
            LaneState &L = s->lanes[free_lane];
            L.busy = true;
            lk.unlock();
            const auto tl = Clock::now();
            std::vector<int64_t> deferred = launch_batch(s, free_lane, take);
            const double dl = std::chrono::duration<double, std::milli>(Clock::now() - tl).count();
            lk.lock();
            s->host_launch_ms += dl;
            for (auto it = deferred.rbegin(); it != deferred.rend(); ++it) s->pending.push_front(*it);
            if (L.lin.empty() && L.ovl.empty()) {
                L.busy = false;
                bool other = false;
                for (int li = 0; li < s->nl; ++li) other = other || s->lanes[li].busy;
                if (!other && !deferred.empty()) {
                    // nothing in flight and still no room: the head request can never fit
                    const int64_t t = s->pending.front();
                    s->pending.pop_front();
                    complete(s, t, VGICP_ERR_BUDGET);
                    s->cv_done.notify_all();
                }
                if (other) s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
            }
            s->cv_done.notify_all();
            continue;
        }
        s->cv_work.wait_for(lk, std::chrono::milliseconds(20));
    }
}

// ------------------------------------------------------- device loop --

// Hand out every finished request of the ring (mutex held).
bool harvest_slots(vgicp_server *s)
{
    bool any = false;
    const auto now = Clock::now();
    for (size_t q = 0; q < s->inflight.size();) {
        const int slot = s->inflight[q];
        const vg::LoopResult &R = s->h_res[slot];
        if (__atomic_load_n(&R.done, __ATOMIC_ACQUIRE) != s->slot_seq[slot]) {
            ++q;
            continue;
        }
        Pending &p = s->reqs[s->slot_ticket[slot]];
        p.res.status = VGICP_OK;
        p.res.kind = p.req.kind;
        if (p.req.kind == VGICP_REQ_LINEARIZE) {
            std::memcpy(p.res.H, R.H, sizeof(p.res.H));
            std::memcpy(p.res.b, R.b, sizeof(p.res.b));
            p.res.cost = R.cost;
            p.res.count = R.count;
        } else {
            const int64_t n = s->objs[tag(p.req.source, false)].n;
            p.res.count = R.count;
            p.res.fraction = (double)R.count / (double)n;
        }
        p.res.latency_ms = std::chrono::duration<double, std::milli>(now - p.t0).count();
        p.done = true;
        s->lat_ms.push_back(p.res.latency_ms);
        s->objs[s->slot_keys[slot].first].pins--;
        s->objs[s->slot_keys[slot].second].pins--;
        s->slot_ticket[slot] = -1;
        ++s->completed;
        s->inflight[q] = s->inflight.back();
        s->inflight.pop_back();
        any = true;
    }
    return any;
}

// Launch the loop kernel, starting from the oldest request not yet answered (mutex held).
vgicp_status launch_loop(vgicp_server *s)
{
    unsigned long long first = s->n_pub;
    for (int slot : s->inflight) first = std::min(first, s->slot_seq[slot] - 1);
    *s->h_ctl = vg::LoopControl{0u, 0u, 0u, 0u, first};
    s->h_exit->status = VGICP_OK;
    s->h_exit->next_req = first;
    cudaEventRecord(s->loop_ev0, s->loop_stream);
    cudaMemcpyAsync(s->d_ctl, s->h_ctl, sizeof(vg::LoopControl), cudaMemcpyHostToDevice, s->loop_stream);
    vg::LoopArgs a{};
    a.req = s->d_req;
    a.res = s->d_res;
    a.exit = s->d_exit;
    a.ctl = s->d_ctl;
    a.state = s->d_state;
    a.partials = s->d_partials;
    a.counts = s->d_counts;
    a.queue = s->d_queue;
    a.slots = s->slots;
    a.qcap = s->qcap;
    a.idle_ns = (unsigned long long)(s->idle_ms * 1e6);
    a.worker_ns = a.idle_ns + 1000000000ull;       // the idle limit plus a second
    // an error left by an earlier call of this thread must not be taken for a
    // failed launch: the requests would be answered and their objects unpinned
    // while the kernel reads them
    cudaGetLastError();
    vg::launch_request_loop(a, s->num_sms, s->loop_stream);
    const cudaError_t e = cudaGetLastError();
    cudaEventRecord(s->loop_ev1, s->loop_stream);
    if (e != cudaSuccess) {
        s->err = cudaGetErrorString(e);
        return VGICP_ERR_CUDA;
    }
    s->loop_running = true;
    ++s->loop_launches;
    ++s->batches;
    return VGICP_OK;
}

// Whether an object's admission has completed on the device (mutex held).
bool object_ready(Resident &o)
{
    // an error (a failed context) counts as done: the loop launch then reports it
    if (!o.ready_done && cudaEventQuery(o.ready) != cudaErrorNotReady) o.ready_done = true;
    return o.ready_done;
}

// Unpin a prepared request's objects (mutex held).
void unpin(vgicp_server *s, int64_t t)
{
    const vgicp_request &r = s->reqs[t].req;
    s->objs[tag(r.target, true)].pins--;
    s->objs[tag(r.source, false)].pins--;
}

// Write prepared request t, whose objects are ready, into the next ring slot
// (mutex held; the slot is free).
void publish_slot(vgicp_server *s, int64_t t)
{
    const vgicp_request r = s->reqs[t].req;
    Resident &m = s->objs[tag(r.target, true)], &f = s->objs[tag(r.source, false)];
    vg::MapDesc md;
    vg::FrameDesc fd;
    int64_t n = 0;
    Pending &p = s->reqs[t];
    if (!vg::ctx_descs(s->ctx, m.handle, f.handle, &md, &fd, &n)) {
        unpin(s, t);
        complete(s, t, VGICP_ERR_NOT_FOUND);
        ++s->completed;
        return;
    }
    if (n == 0) {                      // nothing to run: an empty sum, or Eq. 8 undefined
        unpin(s, t);
        complete(s, t, r.kind == VGICP_REQ_OVERLAP ? VGICP_ERR_EMPTY : VGICP_OK);
        s->lat_ms.push_back(p.res.latency_ms);
        ++s->completed;
        return;
    }
    const int c = vg::item_chunk(n, s->chunk);
    const int64_t items = (n + c - 1) / c;
    if (items > vg::kLoopMaxItems) {
        unpin(s, t);
        s->err = "request larger than 128 chunks";
        complete(s, t, VGICP_ERR_INVALID_ARG);
        ++s->completed;
        return;
    }
    const int slot = (int)(s->n_pub % (unsigned long long)s->slots);
    const unsigned long long seq = ++s->n_pub;
    vg::LoopRequest &q = s->h_req[slot];
    q.map = md;
    q.frame = fd;
    std::memcpy(q.T, r.T_target_source, sizeof(q.T));
    q.kind = r.kind == VGICP_REQ_LINEARIZE ? vg::kLoopLinearize : vg::kLoopOverlap;
    q.n_items = (int32_t)items;
    q.chunk = c;
    q.cull = s->cull;
    __atomic_store_n(&s->h_res[slot].done, 0ull, __ATOMIC_RELAXED);
    __atomic_store_n(&q.seq, seq, __ATOMIC_RELEASE);      // the request is visible to the loop from here
    s->slot_ticket[slot] = t;
    s->slot_seq[slot] = seq;
    s->slot_keys[slot] = {tag(r.target, true), tag(r.source, false)};
    s->inflight.push_back(slot);
}

// Fail every request in flight (mutex held).
void fail_inflight(vgicp_server *s, vgicp_status st)
{
    for (int slot : s->inflight) {
        complete(s, s->slot_ticket[slot], st);
        s->objs[s->slot_keys[slot].first].pins--;
        s->objs[s->slot_keys[slot].second].pins--;
        s->slot_ticket[slot] = -1;
        ++s->completed;
    }
    s->inflight.clear();
    s->cv_done.notify_all();
}

void scheduler_device(vgicp_server *s)
{
    std::unique_lock<std::mutex> lk(s->mu);
    int idle_polls = 0, fruitless = 0;
    int64_t completed_at_launch = 0;
    for (;;) {
        if (harvest_slots(s)) {
            s->cv_done.notify_all();
            idle_polls = 0;
        }
        if (s->loop_running && cudaStreamQuery(s->loop_stream) != cudaErrorNotReady) {
            s->loop_running = false;
            s->loop_last_exit = s->h_exit->status;
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, s->loop_ev0, s->loop_ev1) == cudaSuccess) s->device_ms += ms;
            vg::LoopControl c{};
            if (cudaMemcpy(&c, s->d_ctl, sizeof(c), cudaMemcpyDeviceToHost) == cudaSuccess && c.status)
                s->err = "a worker of the request loop ran out of its wait limit";
            harvest_slots(s);
            // a loop that ended with requests in flight and answered none, several times
            // in a row, will not answer them: fail them instead of relaunching forever
            fruitless = (!s->inflight.empty() && s->completed == completed_at_launch) ? fruitless + 1 : 0;
            if (fruitless >= 8) {
                s->err = "the request loop ended repeatedly without answering the requests in flight";
                fail_inflight(s, VGICP_ERR_CUDA);
                fruitless = 0;
            }
            s->cv_done.notify_all();
        }
        if (s->stop) {
            // drop what is pending, ask the loop to end, answer what it finished, fail the rest
            for (int64_t t : s->pending) {
                complete(s, t, VGICP_ERR_CUDA);
                ++s->completed;
            }
            s->pending.clear();
            if (s->loop_running) {
                __atomic_store_n(&s->h_exit->stop, 1, __ATOMIC_RELEASE);
                lk.unlock();
                cudaStreamSynchronize(s->loop_stream);
                lk.lock();
                s->loop_running = false;
            }
            harvest_slots(s);
            fail_inflight(s, VGICP_ERR_CUDA);
            for (int64_t t : s->waiting) {
                unpin(s, t);
                complete(s, t, VGICP_ERR_CUDA);
                ++s->completed;
            }
            for (int64_t t : s->ready_q) {
                unpin(s, t);
                complete(s, t, VGICP_ERR_CUDA);
                ++s->completed;
            }
            s->waiting.clear();
            s->ready_q.clear();
            s->cv_done.notify_all();
            return;
        }
        const auto tl = Clock::now();
        bool published = false;
        // admit pending requests (asynchronously) in groups, at most a ring's worth
        // ahead of publishing
        while (!s->pending.empty() && s->waiting.size() + s->ready_q.size() < (size_t)s->slots) {
            const size_t room = (size_t)s->slots - s->waiting.size() - s->ready_q.size();
            std::vector<int64_t> grp;
            while (!s->pending.empty() && grp.size() < std::min(room, kAdmitGroup)) {
                grp.push_back(s->pending.front());
                s->pending.pop_front();
            }
            std::vector<int64_t> ok, def, failed;
            vgicp_status fst = VGICP_OK;
            lk.unlock();
            prepare_group(s, grp, ok, def, failed, fst);
            lk.lock();
            for (int64_t t : failed) {
                complete(s, t, fst);
                ++s->completed;
            }
            if (!failed.empty()) s->cv_done.notify_all();
            for (int64_t t : ok) s->waiting.push_back(t);
            if (def.empty()) continue;
            size_t d0 = 0;
            if (s->inflight.empty() && s->waiting.empty() && s->ready_q.empty()) {
                complete(s, def[0], VGICP_ERR_BUDGET);   // nothing to wait for: it can never fit
                ++s->completed;
                s->cv_done.notify_all();
                d0 = 1;
            }
            // the rest waits, in order, until other requests release objects
            for (size_t i = def.size(); i > d0; --i) s->pending.push_front(def[i - 1]);
            if (d0 == 0) break;
        }
        // requests whose objects' copies and builds are complete, in order
        for (size_t q = 0; q < s->waiting.size();) {
            const vgicp_request &r = s->reqs[s->waiting[q]].req;
            if (object_ready(s->objs[tag(r.target, true)]) && object_ready(s->objs[tag(r.source, false)])) {
                s->ready_q.push_back(s->waiting[q]);
                s->waiting.erase(s->waiting.begin() + (ptrdiff_t)q);
            } else {
                ++q;
            }
        }
        // into the ring while it has room in order
        while (!s->ready_q.empty() && s->slot_ticket[s->n_pub % (unsigned long long)s->slots] < 0) {
            publish_slot(s, s->ready_q.front());
            s->ready_q.pop_front();
            published = true;
        }
        if (published) {
            s->cv_done.notify_all();
            s->host_launch_ms += std::chrono::duration<double, std::milli>(Clock::now() - tl).count();
            int64_t bytes = 0;
            vgicp_memory_in_use(s->ctx, &bytes);
            s->resident_bytes = bytes;
        }
        if (!s->loop_running && !s->inflight.empty()) {
            completed_at_launch = s->completed;
            const vgicp_status st = launch_loop(s);
            if (st != VGICP_OK) fail_inflight(s, st);  // rather than wait forever
        }
        if (!s->inflight.empty() || !s->waiting.empty() || !s->ready_q.empty()) {
            // results arrive in host memory, admissions complete on the device: poll,
            // yielding the core, then sleep a little
            lk.unlock();
            if (++idle_polls < 2000) std::this_thread::yield();
            else std::this_thread::sleep_for(std::chrono::microseconds(50));
            lk.lock();
        } else {
            idle_polls = 0;
            s->cv_work.wait_for(lk, std::chrono::milliseconds(20));
        }
    }
}

vgicp_status loop_setup(vgicp_server *s, const vgicp_options &ko)
{
    s->dloop = true;
    s->slots = s->opt.loop_slots > 0 ? s->opt.loop_slots : 256;
    s->idle_ms = s->opt.loop_idle_ms > 0.0 ? s->opt.loop_idle_ms : 20.0;
    s->chunk = ko.chunk_points > 0 ? ko.chunk_points : 2048;
    s->cull = ko.linearize_cull ? (ko.group_cull ? 2 : 1) : 0;   // culling level (chunks, groups)
    unsigned int q = 1;
    while (q < (unsigned int)s->slots * (unsigned int)vg::kLoopMaxItems) q <<= 1;
    s->qcap = q;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t S = (size_t)s->slots;
    if (cudaHostAlloc((void **)&s->h_req, S * sizeof(vg::LoopRequest), cudaHostAllocMapped) ||
        cudaHostAlloc((void **)&s->h_res, S * sizeof(vg::LoopResult), cudaHostAllocMapped) ||
        cudaHostAlloc((void **)&s->h_exit, sizeof(vg::LoopExit), cudaHostAllocMapped) ||
        cudaHostAlloc((void **)&s->h_ctl, sizeof(vg::LoopControl), cudaHostAllocDefault) ||
        cudaHostGetDevicePointer((void **)&s->d_req, s->h_req, 0) ||
        cudaHostGetDevicePointer((void **)&s->d_res, s->h_res, 0) ||
        cudaHostGetDevicePointer((void **)&s->d_exit, s->h_exit, 0) ||
        cudaMalloc((void **)&s->d_ctl, sizeof(vg::LoopControl)) ||
        cudaMalloc((void **)&s->d_state, S * sizeof(vg::LoopSlotState)) ||
        cudaMalloc((void **)&s->d_partials, S * vg::kLoopMaxItems * 28 * sizeof(double)) ||
        cudaMalloc((void **)&s->d_counts, S * vg::kLoopMaxItems * sizeof(long long)) ||
        cudaMalloc((void **)&s->d_queue, (size_t)s->qcap * sizeof(int2)) ||
        cudaStreamCreateWithFlags(&s->loop_stream, cudaStreamNonBlocking) ||
        cudaEventCreate(&s->loop_ev0) || cudaEventCreate(&s->loop_ev1)) {
        cudaGetLastError();
        return VGICP_ERR_OOM;
    }
    std::memset(s->h_req, 0, S * sizeof(vg::LoopRequest));
    std::memset(s->h_res, 0, S * sizeof(vg::LoopResult));
    std::memset(s->h_exit, 0, sizeof(vg::LoopExit));
    s->slot_ticket.assign(S, -1);
    s->slot_seq.assign(S, 0ull);
    s->slot_keys.assign(S, {0, 0});
    return VGICP_OK;
}

void loop_free(vgicp_server *s)
{
    if (s->loop_stream) {
        if (s->h_exit) __atomic_store_n(&s->h_exit->stop, 1, __ATOMIC_RELEASE);
        cudaStreamSynchronize(s->loop_stream);
        cudaStreamDestroy(s->loop_stream);
    }
    if (s->loop_ev0) cudaEventDestroy(s->loop_ev0);
    if (s->loop_ev1) cudaEventDestroy(s->loop_ev1);
    cudaFreeHost(s->h_req);
    cudaFreeHost(s->h_res);
    cudaFreeHost(s->h_exit);
    cudaFreeHost(s->h_ctl);
    cudaFree(s->d_ctl);
    cudaFree(s->d_state);
    cudaFree(s->d_partials);
    cudaFree(s->d_counts);
    cudaFree(s->d_queue);
}

// Room for `bytes` in the page-locked slabs, or null when no page-locked memory
// can be had.  A new slab is pinned without the lock held (pinning 256 MB takes
// tens of milliseconds, which the scheduler thread must not wait for).
char *slab_alloc(vgicp_server *s, size_t bytes)
{
    bytes = (bytes + 255) & ~(size_t)255;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (!s->slabs.empty() && s->slab_off + bytes <= s->slab_cap) {
            char *r = s->slabs.back() + s->slab_off;
            s->slab_off += bytes;
            return r;
        }
    }
    const size_t cap = std::max(bytes, (size_t)256 << 20);
    char *p = nullptr;
    if (cudaMallocHost((void **)&p, cap) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->slabs.push_back(p);
    s->slab_cap = cap;
    s->slab_off = bytes;
    return p;
}

vgicp_status put(vgicp_server *s, int64_t key, bool is_map, const float *pts, const float *covs, int64_t n, double r)
{
    if (!s) return VGICP_ERR_INVALID_ARG;
    if (n < 0 || (n > 0 && (!pts || !covs)) || key < 0 || key >= ((int64_t)1 << 62)) return VGICP_ERR_INVALID_ARG;
    if (is_map && !(r > 0.0 && r < 1e30)) return VGICP_ERR_INVALID_ARG;
    const int64_t t = tag(key, is_map);
    Resident o;
    o.is_map = is_map;
    o.key = t;
    o.n = n;
    o.r = r;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->objs.count(t)) {
            s->err = "key already registered";
            return VGICP_ERR_INVALID_ARG;
        }
    }
    float *h = n > 0 ? (float *)slab_alloc(s, (size_t)n * 36) : nullptr;
    if (n > 0) {                                        // the copy runs without the lock
        if (!h) {
            o.own.resize((size_t)n * 9);
            h = o.own.data();
        }
        std::memcpy(h, pts, (size_t)n * 12);
        std::memcpy(h + 3 * n, covs, (size_t)n * 24);
        o.pts = h;
        o.covs = h + 3 * n;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->objs.count(t)) {
        s->err = "key already registered";
        return VGICP_ERR_INVALID_ARG;
    }
    s->objs.emplace(t, std::move(o));
    return VGICP_OK;
}

}  // namespace

extern "C" {

vgicp_status vgicp_server_create(vgicp_server **out, const vgicp_server_options *opt, const vgicp_options *kopt)
{
    if (!out) return VGICP_ERR_INVALID_ARG;
    *out = nullptr;
    vgicp_server *s = new vgicp_server();
    if (opt) s->opt = *opt;
    if (s->opt.max_batch_requests <= 0) s->opt.max_batch_requests = 4096;
    if (s->opt.max_batch_points <= 0) s->opt.max_batch_points = (int64_t)1 << 27;
    if (s->opt.lanes <= 0) s->opt.lanes = 2;
    if (s->opt.lanes > 4 || s->opt.hbm_budget_bytes < 0 || s->opt.device_loop < 0 || s->opt.device_loop > 1 ||
        s->opt.loop_slots < 0 || s->opt.loop_slots > 1024 || !(s->opt.loop_idle_ms >= 0.0) ||
        s->opt.loop_idle_ms > 60000.0) {
        delete s;
        return VGICP_ERR_INVALID_ARG;
    }
    s->nl = s->opt.lanes;
    vgicp_options ko;
    vgicp_options_default(&ko);
    if (kopt) ko = *kopt;
    ko.precision = VGICP_PREC_F32;
    ko.hbm_budget_bytes = s->opt.hbm_budget_bytes;
    if (s->opt.device_loop && (ko.neighbors > 1 || ko.count_weighted)) {
        delete s;
        return VGICP_ERR_INVALID_ARG;
    }
    vgicp_status st = vgicp_create(&s->ctx, &ko, nullptr);
    if (st != VGICP_OK) {
        delete s;
        return st;
    }
    if (s->opt.device_loop) {
        st = loop_setup(s, ko);
        if (st != VGICP_OK) {
            loop_free(s);
            vgicp_destroy(s->ctx);
            delete s;
            return st;
        }
        s->thr = std::thread(scheduler_device, s);
        *out = s;
        return VGICP_OK;
    }
    for (int li = 0; li < s->nl; ++li) {
        s->lanes[li].cb = {s, li};
        cudaEventCreate(&s->lanes[li].ev0);
        cudaEventCreate(&s->lanes[li].ev1);
        if (cudaStreamCreateWithFlags(&s->lanes[li].stream, cudaStreamNonBlocking) != cudaSuccess) {
            vgicp_destroy(s->ctx);
            delete s;
            return VGICP_ERR_CUDA;
        }
    }
    s->thr = std::thread(scheduler, s);
    *out = s;
    return VGICP_OK;
}

vgicp_status vgicp_server_destroy(vgicp_server *s)
{
    if (!s) return VGICP_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    s->thr.join();
    if (s->dloop) {
        loop_free(s);
        for (auto &kv : s->objs)
            if (kv.second.ready) cudaEventDestroy(kv.second.ready);
        vgicp_destroy(s->ctx);
        for (char *p : s->slabs) cudaFreeHost(p);
        delete s;
        return VGICP_OK;
    }
    for (int li = 0; li < s->nl; ++li) cudaStreamSynchronize(s->lanes[li].stream);
    vgicp_set_lane(s->ctx, 0, nullptr);
    for (auto &kv : s->objs)
        if (kv.second.ready) cudaEventDestroy(kv.second.ready);
    vgicp_destroy(s->ctx);
    for (int li = 0; li < s->nl; ++li) {
        LaneState &L = s->lanes[li];
        cudaFree(L.dH); cudaFree(L.db); cudaFree(L.dc); cudaFree(L.di); cudaFree(L.dcount);
        cudaFreeHost(L.hH); cudaFreeHost(L.hb); cudaFreeHost(L.hc); cudaFreeHost(L.hi); cudaFreeHost(L.hcount);
        cudaStreamDestroy(L.stream);
        cudaEventDestroy(L.ev0);
        cudaEventDestroy(L.ev1);
    }
    for (char *p : s->slabs) cudaFreeHost(p);
    delete s;
    return VGICP_OK;
}

vgicp_status vgicp_server_put_map(vgicp_server *s, int64_t key, const float *points, const float *covs, int64_t n,
                                  double resolution)
{
    return put(s, key, true, points, covs, n, resolution);
}

vgicp_status vgicp_server_put_frame(vgicp_server *s, int64_t key, const float *points, const float *covs, int64_t n)
{
    return put(s, key, false, points, covs, n, 0.0);
}

vgicp_status vgicp_server_submit(vgicp_server *s, const vgicp_request *req, int64_t *ticket)
{
    if (!s || !req || !ticket) return VGICP_ERR_INVALID_ARG;
    if (req->kind != VGICP_REQ_LINEARIZE && req->kind != VGICP_REQ_OVERLAP) return VGICP_ERR_INVALID_ARG;
    for (int i = 0; i < 12; ++i)
        if (!(req->T_target_source[i] - req->T_target_source[i] == 0.0)) return VGICP_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (!s->objs.count(tag(req->target, true)) || !s->objs.count(tag(req->source, false))) {
            s->err = "request names an unregistered key";
            return VGICP_ERR_NOT_FOUND;
        }
        const int64_t t = s->next_ticket++;
        Pending &p = s->reqs[t];
        p.req = *req;
        p.t0 = Clock::now();
        std::memset(&p.res, 0, sizeof(p.res));
        s->pending.push_back(t);
        ++s->submitted;
        *ticket = t;
    }
    s->cv_work.notify_all();
    return VGICP_OK;
}

vgicp_status vgicp_server_submit_batch(vgicp_server *s, const vgicp_request *reqs, int64_t n, int64_t *tickets)
{
    if (!s || n < 0 || (n > 0 && (!reqs || !tickets))) return VGICP_ERR_INVALID_ARG;
    for (int64_t k = 0; k < n; ++k) {
        const vgicp_request *req = reqs + k;
        if (req->kind != VGICP_REQ_LINEARIZE && req->kind != VGICP_REQ_OVERLAP) return VGICP_ERR_INVALID_ARG;
        for (int i = 0; i < 12; ++i)
            if (!(req->T_target_source[i] - req->T_target_source[i] == 0.0)) return VGICP_ERR_INVALID_ARG;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (int64_t k = 0; k < n; ++k)
            if (!s->objs.count(tag(reqs[k].target, true)) || !s->objs.count(tag(reqs[k].source, false))) {
                s->err = "request names an unregistered key";
                return VGICP_ERR_NOT_FOUND;
            }
        const auto now = Clock::now();
        for (int64_t k = 0; k < n; ++k) {
            const int64_t t = s->next_ticket++;
            Pending &p = s->reqs[t];
            p.req = reqs[k];
            p.t0 = now;
            std::memset(&p.res, 0, sizeof(p.res));
            s->pending.push_back(t);
            tickets[k] = t;
        }
        s->submitted += n;
    }
    s->cv_work.notify_all();
    return VGICP_OK;
}

vgicp_status vgicp_server_wait(vgicp_server *s, int64_t ticket, double timeout_s, vgicp_result *out)
{
    if (!s || !out) return VGICP_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return VGICP_ERR_NOT_FOUND;
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                             std::chrono::duration<double>(timeout_s < 0 ? 1e9 : timeout_s));
    while (!it->second.done) {
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !it->second.done)
            return VGICP_ERR_TIMEOUT;
        it = s->reqs.find(ticket);
    }
    *out = it->second.res;
    s->reqs.erase(it);
    return VGICP_OK;
}

vgicp_status vgicp_server_wait_batch(vgicp_server *s, const int64_t *tickets, int64_t n, double timeout_s,
                                     vgicp_result *out)
{
    if (!s || n < 0 || (n > 0 && (!tickets || !out))) return VGICP_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    for (int64_t k = 0; k < n; ++k)
        if (!s->reqs.count(tickets[k])) return VGICP_ERR_NOT_FOUND;
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                             std::chrono::duration<double>(timeout_s < 0 ? 1e9 : timeout_s));
    for (int64_t k = 0; k < n; ++k) {
        auto it = s->reqs.find(tickets[k]);
        while (!it->second.done) {
            if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !it->second.done)
                return VGICP_ERR_TIMEOUT;    // tickets before k are retired, k and later stay valid
            it = s->reqs.find(tickets[k]);
        }
        out[k] = it->second.res;
        s->reqs.erase(it);
    }
    return VGICP_OK;
}

vgicp_status vgicp_server_stats(vgicp_server *s, vgicp_server_counters *out)
{
    if (!s || !out) return VGICP_ERR_INVALID_ARG;
    std::vector<double> lat;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        std::memset(out, 0, sizeof(*out));
        out->submitted = s->submitted;
        out->completed = s->completed;
        out->batches = s->batches;
        out->admissions = s->admissions;
        out->evictions = s->evictions;
        out->mean_batch_requests = s->batches ? (double)s->batch_requests / (double)s->batches : 0.0;
        out->resident_bytes = s->resident_bytes;
        out->host_launch_ms = s->host_launch_ms;
        out->host_finish_ms = s->host_finish_ms;
        out->device_ms = s->device_ms;
        out->host_admit_ms = s->host_admit_ms;
        out->host_enqueue_ms = s->host_enqueue_ms;
        lat = s->lat_ms;
    }
    if (!lat.empty()) {
        std::sort(lat.begin(), lat.end());
        auto q = [&](double f) { return lat[std::min(lat.size() - 1, (size_t)(f * (double)(lat.size() - 1) + 0.5))]; };
        out->p50_ms = q(0.50);
        out->p99_ms = q(0.99);
        out->max_ms = lat.back();
    }
    return VGICP_OK;
}

vgicp_status vgicp_server_reset_stats(vgicp_server *s)
{
    if (!s) return VGICP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    s->lat_ms.clear();
    s->submitted = s->completed = s->batches = s->admissions = s->evictions = s->batch_requests = 0;
    s->host_launch_ms = s->host_finish_ms = s->device_ms = s->host_admit_ms = s->host_enqueue_ms = 0.0;
    return VGICP_OK;
}

const char *vgicp_server_last_error(const vgicp_server *s) { return s ? s->err.c_str() : "null server"; }

vgicp_status vgicp_server_loop_state(vgicp_server *s, int32_t *running, int32_t *last_exit, int64_t *launches)
{
    if (!s || !s->dloop) return VGICP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    bool run = s->loop_running;
    int last = s->loop_last_exit;
    if (run && cudaStreamQuery(s->loop_stream) != cudaErrorNotReady) {   // ended since the scheduler looked
        run = false;
        last = s->h_exit->status;
    }
    if (running) *running = run ? 1 : 0;
    if (last_exit) *last_exit = last;
    if (launches) *launches = s->loop_launches;
    return VGICP_OK;
}

}  // extern "C"
