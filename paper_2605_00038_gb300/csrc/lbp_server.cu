// lbp_server_*: a continuous-batching decode service on one device.
//
// Requests (host syndromes of any loaded code) enter a FIFO.  A scheduler
// thread admits the oldest waiting request as soon as an in-flight slot is
// free and the device arena has room for its buffers (syndromes, outputs and
// decode workspace): admission by memory, not by a fixed batch.  An admitted
// request gets its own stream: host-to-device copy, lbp_decode, device-to-host
// copies, then an event.  Requests therefore overlap on the device: a small
// request launches into the SMs a large one leaves idle, and work that
// arrives while others run starts without waiting for them to finish.  The
// scheduler frees a request's arena space when its event completes and
// records its latency (submission to completion, host clock).
//
// Each request's results depend only on its code, parameters (seed and
// shot_offset included) and syndromes, never on what else is in flight.
//
// Latency under load: the decode kernels are persistent (one CTA per SM
// loops over the shots), so a launch holds the SMs it got until it ends and
// work queued behind it waits that long.  Two rules bound the wait:
//  * a request larger than chunk_work edge-shots (shots x nnz(H)) runs as
//    consecutive launches of at most that much work on its stream, with
//    shot_offset advanced so every shot draws as it would in one launch;
//  * a request that fits one launch runs on a high-priority stream, so the
//    block scheduler starts it ahead of queued chunks of larger requests.
// lbp_server_configure sets both.
//
// Merged launches (lbp_server_set_batching): the scheduler takes the oldest
// waiting request and later ones that can share its launch (same message
// type, min-sum rule, codes of one degree bound) and decodes all of them with
// lbp_decode_batch, one BP launch over their shots on one stream, so many
// small requests of different codes fill the GPU together instead of each
// holding a launch of its own.
//
// The arena is one cudaMalloc made at creation; admission uses first-fit over
// it, so no allocation happens while serving.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

size_t al256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

struct Request {
    int64_t ticket;
    const lbp_code *code;
    lbp_params params;
    int64_t shots;
    const uint64_t *syn;
    uint64_t *err;
    uint8_t *conv, *osd;
    int32_t *iters;
    Clock::time_point submitted;
    int64_t fit_chunk = 0;              // shots per launch whose layout was checked against the arena
    // While in flight:
    int64_t chunk = 0;                  // shots per launch, fixed at admission
    int slot = -1;
    size_t arena_off = 0, arena_bytes = 0;
    int status = LBP_OK;
};

struct Slot {
    cudaStream_t stream = nullptr;      // normal priority
    cudaStream_t stream_hi = nullptr;   // highest priority
    cudaEvent_t done = nullptr;
    bool busy = false;
    Request req;                        // one request, or the first of a merged launch
    std::vector<Request> more;          // the other requests of a merged launch
};

// First-fit allocator over [0, size).
struct Arena {
    size_t size = 0;
    std::map<size_t, size_t> free_;  // offset -> bytes
    void init(size_t s) { size = s; free_.clear(); free_[0] = s; }
    bool alloc(size_t bytes, size_t *off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t noff = it->first + bytes;
                free_.erase(it);
                if (rest) free_[noff] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct Layout {
    size_t syn, err, conv, osd, iters, ws, ws_bytes, total;
};

// Shots per launch: chunk_work edge-shots, at least one shot; 0 = no limit.
int64_t chunk_shots(const lbp_code *c, int64_t chunk_work, int64_t B) {
    if (chunk_work <= 0) return B;
    const int64_t nnz = c->nnz > 0 ? c->nnz : 1;
    const int64_t k = chunk_work / nnz;
    return k < 1 ? 1 : (k < B ? k : B);
}

bool request_layout(const lbp_code *c, const lbp_params *p, int64_t B, int64_t chunk, Layout *L) {
    const size_t wsz = lbp_workspace_size(c, p, chunk < B ? chunk : B);
    if (wsz == 0) return false;
    const size_t wm = (c->m + 63) / 64, wn = (c->n + 63) / 64;
    size_t off = 0;
    L->syn = off;   off = al256(off + 8 * wm * B);
    L->err = off;   off = al256(off + 8 * wn * B);
    L->conv = off;  off = al256(off + B);
    L->osd = off;   off = al256(off + B);
    L->iters = off; off = al256(off + 4 * B);
    L->ws = off;    off = al256(off + wsz);
    L->ws_bytes = wsz;
    L->total = off;
    return true;
}

}  // namespace

struct lbp_server {
    int device = 0;
    uint8_t *arena_base = nullptr;
    Arena arena;
    std::vector<Slot> slots;
    std::deque<Request> waiting;
    std::map<int64_t, std::pair<int, double>> finished;   // ticket -> (status, latency s)
    std::map<int64_t, bool> known;                         // tickets not yet collected
    int64_t next_ticket = 1;
    int64_t chunk_work = int64_t(16) << 20;   // edge-shots per launch (0: one launch per request)
    bool priority = true;                      // single-launch requests on the high-priority stream
    int batch_items = 0;                       // merged launches of up to this many requests (0: off)
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::thread worker;
    // statistics
    int64_t completed = 0, shots_done = 0;
};

namespace {

void launch(lbp_server *s, int si) {
    Slot &sl = s->slots[si];
    Request &r = sl.req;
    const int64_t B = r.shots;
    const int64_t chunk = r.chunk;
    Layout L;
    request_layout(r.code, &r.params, B, chunk, &L);
    uint8_t *base = s->arena_base + r.arena_off;
    const size_t wm = (r.code->m + 63) / 64, wn = (r.code->n + 63) / 64;
    cudaStream_t st = (s->priority && chunk >= B) ? sl.stream_hi : sl.stream;
    // The latency layouts of small batches take whole SMs; only a request
    // that starts with nothing else in flight may use them.
    bool alone = true;
    for (size_t i = 0; i < s->slots.size(); ++i)
        if (static_cast<int>(i) != si && s->slots[i].busy) alone = false;
    int rc = LBP_OK;
    if (cudaMemcpyAsync(base + L.syn, r.syn, 8 * wm * B, cudaMemcpyHostToDevice, st) != cudaSuccess) rc = LBP_ECUDA;
    for (int64_t s0 = 0; rc == LBP_OK && s0 < B; s0 += chunk) {
        const int64_t nb = chunk < B - s0 ? chunk : B - s0;
        lbp_params p = r.params;
        p.shot_offset += static_cast<uint64_t>(s0);
        rc = lbp::decode_device(r.code, &p, nb, reinterpret_cast<const uint64_t *>(base + L.syn) + s0 * wm,
                                reinterpret_cast<uint64_t *>(base + L.err) + s0 * wn, base + L.conv + s0,
                                base + L.osd + s0, reinterpret_cast<int32_t *>(base + L.iters) + s0, nullptr,
                                base + L.ws, L.ws_bytes, st, alone);
    }
    if (rc == LBP_OK) {
        bool ok = cudaMemcpyAsync(r.err, base + L.err, 8 * wn * B, cudaMemcpyDeviceToHost, st) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(r.conv, base + L.conv, B, cudaMemcpyDeviceToHost, st) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(r.iters, base + L.iters, 4 * B, cudaMemcpyDeviceToHost, st) == cudaSuccess;
        if (r.osd) ok = ok && cudaMemcpyAsync(r.osd, base + L.osd, B, cudaMemcpyDeviceToHost, st) == cudaSuccess;
        if (!ok) rc = LBP_ECUDA;
    }
    if (rc != LBP_OK) cudaGetLastError();
    r.status = rc;
    cudaEventRecord(sl.done, st);
}

// Device buffers of one request of a merged launch (no workspace of its own).
struct BufLayout {
    size_t syn, err, conv, osd, iters, total;
};

BufLayout buf_layout(const lbp_code *c, int64_t B) {
    const size_t wm = (c->m + 63) / 64, wn = (c->n + 63) / 64;
    BufLayout L;
    size_t off = 0;
    L.syn = off;   off = al256(off + 8 * wm * B);
    L.err = off;   off = al256(off + 8 * wn * B);
    L.conv = off;  off = al256(off + B);
    L.osd = off;   off = al256(off + B);
    L.iters = off; off = al256(off + 4 * B);
    L.total = off;
    return L;
}

// Whether r can join a merged launch whose first request is f: the launch's
// conditions, and codes within a factor of two in size (a launch sizes every
// group's state and width for its largest code, which would idle most of a
// small code's threads).
bool mergeable(const Request &f, const Request &r) {
    const int64_t nf = f.code->n, nr = r.code->n;
    return r.params.msg == f.params.msg && r.params.rule == LBP_RULE_MIN_SUM && f.params.rule == LBP_RULE_MIN_SUM &&
           r.params.lottery_policy != LBP_LOTTERY_PROPOSED_CURRENT && r.code->d_ell && f.code->d_ell && r.code->ell.idx_bytes == 2 && f.code->ell.idx_bytes == 2 &&
           r.code->ell.DC == f.code->ell.DC && r.code->ell.DV == f.code->ell.DV && nr <= 2 * nf && nf <= 2 * nr;
}

// Arena bytes of a merged launch: the requests' buffers, then the batch
// workspace (0 if the requests cannot share a launch).
size_t merged_bytes(const std::vector<const Request *> &g, std::vector<size_t> *offs, size_t *ws_off) {
    std::vector<lbp_batch_item> items(g.size());
    size_t off = 0;
    offs->clear();
    for (size_t i = 0; i < g.size(); ++i) {
        offs->push_back(off);
        off += buf_layout(g[i]->code, g[i]->shots).total;
        lbp_batch_item &it = items[i];
        std::memset(&it, 0, sizeof(it));
        it.code = g[i]->code;
        it.params = g[i]->params;
        it.num_shots = g[i]->shots;
    }
    const size_t ws = lbp::batch_workspace_size(items.data(), static_cast<int>(items.size()));
    if (ws == 0) return 0;
    *ws_off = off;
    return off + ws;
}

void launch_merged(lbp_server *s, int si) {
    Slot &sl = s->slots[si];
    std::vector<Request *> rs;
    rs.push_back(&sl.req);
    for (auto &r : sl.more) rs.push_back(&r);
    std::vector<const Request *> g(rs.begin(), rs.end());
    std::vector<size_t> offs;
    size_t ws_off = 0;
    const size_t total = merged_bytes(g, &offs, &ws_off);
    uint8_t *base = s->arena_base + sl.req.arena_off;
    cudaStream_t st = sl.stream;
    int rc = total ? LBP_OK : LBP_ENOSYS;
    std::vector<lbp_batch_item> items(rs.size());
    for (size_t i = 0; rc == LBP_OK && i < rs.size(); ++i) {
        const Request &r = *rs[i];
        const BufLayout L = buf_layout(r.code, r.shots);
        uint8_t *b = base + offs[i];
        const size_t wm = (r.code->m + 63) / 64;
        if (cudaMemcpyAsync(b + L.syn, r.syn, 8 * wm * r.shots, cudaMemcpyHostToDevice, st) != cudaSuccess)
            rc = LBP_ECUDA;
        lbp_batch_item &it = items[i];
        it.code = r.code;
        it.params = r.params;
        it.num_shots = r.shots;
        it.syndromes = reinterpret_cast<const uint64_t *>(b + L.syn);
        it.err_out = reinterpret_cast<uint64_t *>(b + L.err);
        it.converged = b + L.conv;
        it.osd_out = b + L.osd;
        it.iters_out = reinterpret_cast<int32_t *>(b + L.iters);
    }
    if (rc == LBP_OK)
        rc = lbp_decode_batch(items.data(), static_cast<int32_t>(items.size()), base + ws_off, total - ws_off, st);
    for (size_t i = 0; rc == LBP_OK && i < rs.size(); ++i) {
        Request &r = *rs[i];
        const BufLayout L = buf_layout(r.code, r.shots);
        uint8_t *b = base + offs[i];
        const size_t wn = (r.code->n + 63) / 64;
        bool ok = cudaMemcpyAsync(r.err, b + L.err, 8 * wn * r.shots, cudaMemcpyDeviceToHost, st) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(r.conv, b + L.conv, r.shots, cudaMemcpyDeviceToHost, st) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(r.iters, b + L.iters, 4 * r.shots, cudaMemcpyDeviceToHost, st) == cudaSuccess;
        if (r.osd) ok = ok && cudaMemcpyAsync(r.osd, b + L.osd, r.shots, cudaMemcpyDeviceToHost, st) == cudaSuccess;
        if (!ok) rc = LBP_ECUDA;
    }
    if (rc != LBP_OK) cudaGetLastError();
    for (Request *r : rs) r->status = rc;
    cudaEventRecord(sl.done, st);
}

// Admit the oldest waiting request with the later requests that can share
// its launch (up to batch_items, oldest first, as long as the arena has room
// for all of them) into slot si.  Returns 1 when a group was admitted, 0 when
// the arena has no room for it yet, and -1 when the oldest request cannot
// take a merged launch even alone (lbp_decode_batch cannot plan it, or its
// merged layout, which holds every shot's workspace at once, exceeds the
// arena): it then runs as a single request.
int admit_merged(lbp_server *s, int si) {
    const Request &f = s->waiting.front();
    std::vector<size_t> pick{0};
    for (size_t i = 1; i < s->waiting.size() && static_cast<int>(pick.size()) < s->batch_items; ++i)
        if (mergeable(f, s->waiting[i])) pick.push_back(i);
    while (!pick.empty()) {
        std::vector<const Request *> g;
        for (size_t i : pick) g.push_back(&s->waiting[i]);
        std::vector<size_t> offs;
        size_t ws_off = 0;
        const size_t bytes = merged_bytes(g, &offs, &ws_off);
        if (pick.size() == 1 && (bytes == 0 || bytes > s->arena.size)) return -1;
        size_t off = 0;
        if (bytes && s->arena.alloc(bytes, &off)) {
            Slot &sl = s->slots[si];
            sl.req = s->waiting[pick[0]];
            sl.req.arena_off = off;
            sl.req.arena_bytes = bytes;
            sl.req.slot = si;
            sl.more.clear();
            for (size_t k = 1; k < pick.size(); ++k) sl.more.push_back(s->waiting[pick[k]]);
            for (size_t k = pick.size(); k-- > 0;) s->waiting.erase(s->waiting.begin() + static_cast<long>(pick[k]));
            sl.busy = true;
            launch_merged(s, si);
            return 1;
        }
        pick.pop_back();                     // smaller group, or wait for memory
    }
    return 0;
}

void run(lbp_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        // Retire finished requests.
        bool progressed = false;
        for (size_t i = 0; i < s->slots.size(); ++i) {
            Slot &sl = s->slots[i];
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) {
                cudaGetLastError();
                sl.req.status = LBP_ECUDA;
            }
            const auto now = Clock::now();
            const double lat = std::chrono::duration<double>(now - sl.req.submitted).count();
            s->finished[sl.req.ticket] = {sl.req.status, lat};
            s->arena.release(sl.req.arena_off, sl.req.arena_bytes);
            s->completed += 1;
            s->shots_done += sl.req.shots;
            for (const Request &r : sl.more) {
                const int st = q == cudaSuccess ? r.status : LBP_ECUDA;
                s->finished[r.ticket] = {st, std::chrono::duration<double>(now - r.submitted).count()};
                s->completed += 1;
                s->shots_done += r.shots;
            }
            sl.more.clear();
            sl.busy = false;
            progressed = true;
        }
        if (progressed) s->cv_done.notify_all();
        // Admit waiting requests, oldest first, while a slot and memory allow.
        while (!s->waiting.empty()) {
            int free_slot = -1;
            for (size_t i = 0; i < s->slots.size(); ++i)
                if (!s->slots[i].busy) { free_slot = static_cast<int>(i); break; }
            if (free_slot < 0) break;
            if (s->batch_items > 0 && s->waiting.front().params.rule == LBP_RULE_MIN_SUM &&
                s->waiting.front().code->d_ell && s->waiting.front().code->ell.idx_bytes == 2) {
                const int a = admit_merged(s, free_slot);
                if (a == 0) break;                                 // wait for memory to free up
                if (a > 0) {
                    progressed = true;
                    continue;
                }
            }
            Request &r = s->waiting.front();
            // The chunk size of the policy in force now; when lbp_server_configure
            // has grown it since submission past what the arena holds, the size
            // checked at submission.
            int64_t chunk = chunk_shots(r.code, s->chunk_work, r.shots);
            Layout L;
            request_layout(r.code, &r.params, r.shots, chunk, &L);
            if (L.total > s->arena.size) {
                chunk = r.fit_chunk;
                request_layout(r.code, &r.params, r.shots, chunk, &L);
            }
            size_t off = 0;
            if (!s->arena.alloc(L.total, &off)) break;           // wait for memory to free up
            Slot &sl = s->slots[free_slot];
            sl.req = r;
            sl.req.chunk = chunk;
            sl.req.arena_off = off;
            sl.req.arena_bytes = L.total;
            sl.req.slot = free_slot;
            sl.busy = true;
            s->waiting.pop_front();
            launch(s, free_slot);
            progressed = true;
        }
        bool any_busy = false;
        for (auto &sl : s->slots) any_busy = any_busy || sl.busy;
        if (s->stop && !any_busy && s->waiting.empty()) break;
        if (!any_busy && s->waiting.empty()) {
            s->cv_work.wait(lk, [&] { return s->stop || !s->waiting.empty(); });
        } else if (!progressed) {
            // Work is on the device: poll again shortly (bounded wait, no spin).
            s->cv_work.wait_for(lk, std::chrono::microseconds(20));
        }
    }
}

}  // namespace

extern "C" int lbp_server_create(size_t arena_bytes, int max_inflight, lbp_server **out) {
    if (!out) return LBP_EINVAL;
    *out = nullptr;
    if (arena_bytes < 4096 || max_inflight < 1 || max_inflight > 64) return LBP_EINVAL;
    lbp_server *s = new (std::nothrow) lbp_server();
    if (!s) return LBP_ENOMEM;
    if (cudaGetDevice(&s->device) != cudaSuccess) { delete s; return LBP_ECUDA; }
    if (cudaMalloc(reinterpret_cast<void **>(&s->arena_base), arena_bytes) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return LBP_ENOMEM;
    }
    s->arena.init(arena_bytes);
    s->slots.resize(max_inflight);
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
        cudaGetLastError();
        least = greatest = 0;
    }
    for (auto &sl : s->slots) {
        if (cudaStreamCreateWithPriority(&sl.stream, cudaStreamNonBlocking, least) != cudaSuccess ||
            cudaStreamCreateWithPriority(&sl.stream_hi, cudaStreamNonBlocking, greatest) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            for (auto &x : s->slots) {
                if (x.stream) cudaStreamDestroy(x.stream);
                if (x.stream_hi) cudaStreamDestroy(x.stream_hi);
                if (x.done) cudaEventDestroy(x.done);
            }
            cudaFree(s->arena_base);
            delete s;
            return LBP_ECUDA;
        }
    }
    s->worker = std::thread(run, s);
    *out = s;
    return LBP_OK;
}

extern "C" int lbp_server_configure(lbp_server *s, int64_t chunk_work, int priority) {
    if (!s || chunk_work < 0 || (priority != 0 && priority != 1)) return LBP_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    s->chunk_work = chunk_work;
    s->priority = priority != 0;
    return LBP_OK;
}

extern "C" int lbp_server_set_batching(lbp_server *s, int32_t max_items) {
    if (!s || max_items < 0 || max_items > 64) return LBP_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    s->batch_items = max_items;
    return LBP_OK;
}

extern "C" int lbp_server_submit(lbp_server *s, const lbp_code *code, const lbp_params *params,
                                 int64_t num_shots, const uint64_t *syndromes, uint64_t *err_out,
                                 uint8_t *converged, uint8_t *osd_out, int32_t *iters_out,
                                 int64_t *ticket) {
    if (!s || !code || !params || !ticket || num_shots < 1 || !syndromes || !err_out || !converged ||
        !iters_out)
        return LBP_EINVAL;
    if (code->device != s->device) return LBP_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    Layout L;
    const int64_t fit_chunk = chunk_shots(code, s->chunk_work, num_shots);
    if (!request_layout(code, params, num_shots, fit_chunk, &L))
        return LBP_EINVAL;
    if (L.total > s->arena.size) return LBP_E2BIG;            // can never be admitted
    if (s->stop) return LBP_EINVAL;
    Request r;
    r.ticket = s->next_ticket++;
    r.code = code;
    r.params = *params;
    r.shots = num_shots;
    r.syn = syndromes;
    r.err = err_out;
    r.conv = converged;
    r.osd = osd_out;
    r.iters = iters_out;
    r.submitted = Clock::now();
    r.fit_chunk = fit_chunk;
    s->waiting.push_back(r);
    s->known[r.ticket] = true;
    *ticket = r.ticket;
    s->cv_work.notify_one();
    return LBP_OK;
}

extern "C" int lbp_server_poll(lbp_server *s, int64_t ticket, int *done, double *latency_s) {
    if (!s || !done) return LBP_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->known.count(ticket)) return LBP_EINVAL;
    auto it = s->finished.find(ticket);
    if (it == s->finished.end()) { *done = 0; return LBP_OK; }
    *done = 1;
    if (latency_s) *latency_s = it->second.second;
    const int st = it->second.first;
    s->finished.erase(it);
    s->known.erase(ticket);
    s->cv_done.notify_all();                              // waiters on this ticket
    return st;
}

extern "C" int lbp_server_wait(lbp_server *s, int64_t ticket, double *latency_s) {
    if (!s) return LBP_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    if (!s->known.count(ticket)) return LBP_EINVAL;
    s->cv_done.wait(lk, [&] { return s->finished.count(ticket) > 0 || !s->known.count(ticket); });
    auto it = s->finished.find(ticket);
    if (it == s->finished.end()) return LBP_EINVAL;      // another caller collected it meanwhile
    if (latency_s) *latency_s = it->second.second;
    const int st = it->second.first;
    s->finished.erase(it);
    s->known.erase(ticket);
    s->cv_done.notify_all();                              // other waiters on this ticket
    return st;
}

extern "C" int lbp_server_destroy(lbp_server *s) {
    if (!s) return LBP_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto &sl : s->slots) {
        cudaStreamSynchronize(sl.stream);
        cudaStreamSynchronize(sl.stream_hi);
        cudaStreamDestroy(sl.stream);
        cudaStreamDestroy(sl.stream_hi);
        cudaEventDestroy(sl.done);
    }
    cudaFree(s->arena_base);
    delete s;
    return LBP_OK;
}
