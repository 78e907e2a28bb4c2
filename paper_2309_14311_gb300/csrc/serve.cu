// Serving: a request loop with continuous batching.
//
// Requests (one road each) queue in arrival order.  Every scheduling round
// (nasch_server_step) the server
//   1. retires requests whose last launches have finished: their per-step
//      statistics (and, if asked, final state) are copied back to the host
//      and their device memory returns to the budget;
//   2. admits queued requests, oldest first, while their state and
//      statistics fit the device-memory budget (a first-fit allocator over
//      one slab of that size) and a slot is free; new roads get their Floyd
//      start on the GPU, on a stream of their own, so that it overlaps the
//      running ticks; a road joins the ticks once the host has seen its
//      initialisation finish;
//   3. enqueues one tick: M launches of the super-step kernel over the items
//      of every resident road, each road continuing from its own super-step,
//      so a request admitted now runs in the same launches as requests
//      admitted earlier.  M is steps_per_tick, or more (up to
//      max_steps_per_tick) when the resident roads are too few to keep the
//      GPU busy for target_tick_ms: the tick's work is estimated from the
//      roads' cars and the rate the last finished ticks ran at.
// Up to ticks_in_flight ticks are queued at once; each has its own host
// staging buffers, reused only after that tick has finished, so planning
// the next tick overlaps the GPU running the earlier ones.  Every tick is
// timed by a pair of events (the GPU's busy time).  When a tick finishes,
// the steps it completed become readable: nasch_server_poll_series copies
// them from the device on a stream of its own (the kernels that wrote them
// have finished), or from the host copy once the request has retired.
// A request's result is identical to the same road run alone: its draws
// are keyed by its own seed and road id, never by its slot or by what else
// is resident.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "batch_internal.h"
#include "nasch.h"
#include "runtime_internal.h"

namespace nasch {
namespace {

// First-fit allocator over [0, size) with coalescing; offsets 256-aligned.
class SlabAllocator {
  public:
    void reset(size_t size)
    {
        free_.clear();
        if (size) free_[0] = size;
        used_ = 0;
    }
    bool alloc(size_t bytes, size_t *off)
    {
        bytes = (bytes + 255u) & ~(size_t)255u;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = (bytes + 255u) & ~(size_t)255u;
        used_ -= bytes;
        auto next = free_.lower_bound(off);
        size_t start = off, len = bytes;
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                start = prev->first;
                len += prev->second;
                free_.erase(prev);
            }
        }
        if (next != free_.end() && off + bytes == next->first) {
            len += next->second;
            free_.erase(next);
        }
        free_[start] = len;
    }
    size_t used() const { return used_; }

  private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0;
};

size_t align256(size_t x) { return (x + 255u) & ~(size_t)255u; }

struct Request {
    uint64_t id = 0;
    nasch_params prm{};
    int64_t T = 0;
    int layout = NASCH_LAYOUT_AGENT;
    BatchRoadDev rd{};
    int64_t n_items = 0, super = 0, done_super = 0;
    size_t off = 0, bytes = 0;
    size_t bm_off = 0, bm_bytes = 0;
    int slot = -1;
    int64_t last_tick = -1;   // sequence number of the last tick that ran it
    bool canceled = false;
    bool retired = false;     // results copied back, device memory released
    bool initialised = false; // its start state is on the device (initialisation observed finished)
    int status = NASCH_OK;
    double submit_t = 0, admit_t = 0, done_t = 0;
    std::vector<uint64_t> sum_v, crossings;
    std::vector<int32_t> x;
    std::vector<uint8_t> v;
    // streamed series: steps whose statistics are final (ticks finished),
    // steps already returned by nasch_server_poll_series, and the steps
    // completed by each tick still in flight, oldest first
    int64_t ready = 0, sent = 0;
    std::deque<std::pair<int64_t, int64_t>> marks;   // (tick sequence, steps done after it)
};

// Host staging of one tick in flight; reused only after that tick finished.
struct TickBuf {
    BatchRoadDev *h_slots = nullptr;     // pinned: slot descriptors
    BatchItem *h_items = nullptr;        // pinned: work-list
    BatchItem *d_items = nullptr;        // device work-list
    uint32_t *d_counters = nullptr;      // device work-list cursors, one per launch
};

struct Tick {
    int64_t seq = 0;
    int64_t vehicle_steps = 0;           // work of the tick (cars x steps)
    int32_t launches = 0;
    cudaEvent_t ev0 = nullptr, ev = nullptr;   // timing events around the tick's launches
};

constexpr int kMaxTicksInFlight = 4;

// One admission round's initialisation (Floyd start states), run on a
// stream of its own so that it overlaps the ticks of the roads already
// running; its staging buffers are reused only after its event completed.
struct InitRound {
    BatchRoadDev *h_new = nullptr, *d_new = nullptr;   // descriptors of the round's roads
    uint64_t **h_bm = nullptr, **d_bm = nullptr;       // their Floyd bit maps
    cudaEvent_t ev = nullptr;
    bool busy = false;
    std::vector<Request *> reqs;
};
constexpr int kInitRounds = 4;

}  // namespace
}  // namespace nasch

using namespace nasch;

struct nasch_server_s {
    nasch_server_config cfg{};
    int device = 0, sms = 1;
    cudaStream_t stream = nullptr;
    cudaStream_t copy_stream = nullptr;  // reads of finished series
    cudaStream_t init_stream = nullptr;  // start states of admitted roads
    bool own_stream = false;
    TuningSnapshot tuning;               // automatic choices in force when the server was made
    void *slab = nullptr;
    SlabAllocator alloc;
    int max_slots = 0;
    std::vector<int> free_slots;
    BatchRoadDev *d_slots = nullptr;
    InitRound init[kInitRounds];
    TickBuf bufs[kMaxTicksInFlight];
    int depth = 2;                       // ticks in flight
    int64_t items_cap = 0;
    uint32_t *h_cancel = nullptr, *d_cancel = nullptr;
    uint32_t padded = 0;
    int blocks = 1;
    std::deque<Request *> queue;
    std::vector<Request *> resident;
    std::deque<Tick> inflight;
    std::vector<Tick> spare_ticks;
    std::unordered_map<uint64_t, Request *> by_id;
    std::vector<Request *> completed;    // not yet polled
    std::vector<Request *> streaming;    // admitted, series not yet fully returned, in admission order
    int64_t tick_seq = 0, harvested_seq = -1;
    int64_t n_done = 0, vehicle_steps_done = 0;
    double gpu_busy = 0.0;
    double rate = 0.0;                   // vehicle-steps per GPU second of the last finished ticks
    int32_t last_launches = 0;
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;

    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

size_t request_bytes(const Request &r)
{
    size_t b = 0;
    const size_t n = std::max<uint32_t>(r.rd.N, 1);
    if (r.layout == NASCH_LAYOUT_AGENT)
        b += 2 * align256(n * 4) + 2 * align256(n);
    else
        b += 2 * align256((size_t)r.rd.L + 16);
    b += 2 * align256((size_t)std::max<int64_t>(r.T, 1) * 8);
    return b;
}

void free_tick_buf(TickBuf &b)
{
    cudaFree(b.d_items);
    cudaFree(b.d_counters);
    if (b.h_items) cudaFreeHost(b.h_items);
    if (b.h_slots) cudaFreeHost(b.h_slots);
    b = TickBuf{};
}

void destroy_server(nasch_server s)
{
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->copy_stream) cudaStreamSynchronize(s->copy_stream);
    if (s->init_stream) cudaStreamSynchronize(s->init_stream);
    for (auto &t : s->inflight) {
        cudaEventDestroy(t.ev0);
        cudaEventDestroy(t.ev);
    }
    for (auto &t : s->spare_ticks) {
        cudaEventDestroy(t.ev0);
        cudaEventDestroy(t.ev);
    }
    cudaFree(s->slab);
    cudaFree(s->d_slots);
    for (auto &ir : s->init) {
        if (ir.h_new) cudaFreeHost(ir.h_new);
        if (ir.h_bm) cudaFreeHost(ir.h_bm);
        cudaFree(ir.d_new);
        cudaFree(ir.d_bm);
        if (ir.ev) cudaEventDestroy(ir.ev);
    }
    for (auto &b : s->bufs) free_tick_buf(b);
    if (s->h_cancel) cudaFreeHost(s->h_cancel);
    // every request not yet released (queued, resident or finished) is in by_id
    for (auto &kv : s->by_id) delete kv.second;
    if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
    if (s->init_stream) cudaStreamDestroy(s->init_stream);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

// Copy the finished request's results back and return its memory and slot.
int retire(nasch_server s, Request *r)
{
    cudaError_t e = cudaSuccess;
    // a request that ran no tick (no steps, or no cars) retires in the round
    // that admitted it: its zeroed series and its start state were written by
    // initialisation work that may still be running
    if (r->super == 0 && !r->canceled) e = cudaStreamSynchronize(s->init_stream);
    if (e == cudaSuccess && !r->canceled && r->T > 0) {
        r->sum_v.resize((size_t)r->T);
        r->crossings.resize((size_t)r->T);
        e = cudaMemcpy(r->sum_v.data(), r->rd.sum_v, (size_t)r->T * 8, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            e = cudaMemcpy(r->crossings.data(), r->rd.crossings, (size_t)r->T * 8, cudaMemcpyDeviceToHost);
    }
    if (e == cudaSuccess && !r->canceled && s->cfg.keep_state && r->rd.N > 0) {
        const int par = (int)(r->super & 1);
        if (r->layout == NASCH_LAYOUT_AGENT) {
            r->x.resize(r->rd.N);
            r->v.resize(r->rd.N);
            e = cudaMemcpy(r->x.data(), r->rd.x[par], (size_t)r->rd.N * 4, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess) e = cudaMemcpy(r->v.data(), r->rd.v[par], r->rd.N, cudaMemcpyDeviceToHost);
        } else {
            std::vector<int8_t> cells(r->rd.L);
            e = cudaMemcpy(cells.data(), r->rd.cells[par], r->rd.L, cudaMemcpyDeviceToHost);
            r->x.clear();
            r->v.clear();
            for (uint32_t c = 0; c < r->rd.L && e == cudaSuccess; ++c)
                if (cells[c] >= 0) {
                    r->x.push_back((int32_t)c);
                    r->v.push_back((uint8_t)cells[c]);
                }
        }
    }
    if (e != cudaSuccess) return cuda_fail(e, "copy request results");
    if (r->bytes) s->alloc.release(r->off, r->bytes);
    if (r->slot >= 0) s->free_slots.push_back(r->slot);
    r->slot = -1;
    r->bytes = 0;
    r->retired = true;
    r->marks.clear();
    r->ready = r->canceled ? r->sent : r->T;   // the whole series is on the host now
    r->done_t = s->now();
    r->status = r->canceled ? NASCH_ECANCELED : NASCH_OK;
    if (!r->canceled) s->vehicle_steps_done += (int64_t)r->rd.N * r->T;
    s->completed.push_back(r);
    ++s->n_done;
    return NASCH_OK;
}

// Retire resident requests that are finished or cancelled, whose
// initialisation has finished and that no unfinished tick still runs.
int retire_ready(nasch_server s)
{
    std::vector<Request *> keep;
    keep.reserve(s->resident.size());
    int st = NASCH_OK;
    for (auto *r : s->resident) {
        const bool over = r->canceled || r->done_super >= r->super;
        if (over && r->initialised && r->last_tick <= s->harvested_seq && st == NASCH_OK)
            st = retire(s, r);
        else
            keep.push_back(r);
    }
    s->resident.swap(keep);
    return st;
}

// Steps whose statistics the ticks finished up to `seq` made final.
void advance_series(nasch_server s, int64_t seq)
{
    for (auto *r : s->resident)
        while (!r->marks.empty() && r->marks.front().first <= seq) {
            r->ready = std::max(r->ready, r->marks.front().second);
            r->marks.pop_front();
        }
}

// Observe finished ticks (blocking on the oldest if `block`).
int harvest(nasch_server s, bool block)
{
    while (!s->inflight.empty()) {
        Tick &t = s->inflight.front();
        cudaError_t q = block ? cudaEventSynchronize(t.ev) : cudaEventQuery(t.ev);
        if (q == cudaErrorNotReady) break;
        if (q != cudaSuccess) return cuda_fail(q, "tick completion");
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t.ev0, t.ev) == cudaSuccess && ms > 0.f) {
            s->gpu_busy += ms * 1e-3;
            const double r = (double)t.vehicle_steps / (ms * 1e-3);
            s->rate = s->rate > 0.0 ? 0.5 * (s->rate + r) : r;
        } else {
            cudaGetLastError();
        }
        s->harvested_seq = t.seq;
        advance_series(s, t.seq);
        s->spare_ticks.push_back(t);
        s->inflight.pop_front();
        block = false;
    }
    return retire_ready(s);
}

int ensure_items(nasch_server s, int64_t need)
{
    if (need <= s->items_cap) return NASCH_OK;
    // buffers may be in use by ticks in flight
    if (!s->inflight.empty()) {
        cudaError_t e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
        int st = harvest(s, false);
        if (st) return st;
    }
    const int64_t cap = std::max<int64_t>(need, 2 * s->items_cap);
    for (int i = 0; i < s->depth; ++i) {
        TickBuf &b = s->bufs[i];
        cudaFree(b.d_items);
        if (b.h_items) cudaFreeHost(b.h_items);
        b.d_items = nullptr;
        b.h_items = nullptr;
        cudaError_t e = cudaMalloc(&b.d_items, (size_t)cap * sizeof(BatchItem));
        if (e == cudaSuccess) e = cudaHostAlloc((void **)&b.h_items, (size_t)cap * sizeof(BatchItem), 0);
        if (e != cudaSuccess) return cuda_fail(e, "work-list buffers");
    }
    s->items_cap = cap;
    return NASCH_OK;
}

// Initialisation rounds whose work has finished: their roads may run.
int poll_init(nasch_server s)
{
    for (auto &ir : s->init) {
        if (!ir.busy) continue;
        const cudaError_t q = cudaEventQuery(ir.ev);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) return cuda_fail(q, "initialisation");
        for (auto *r : ir.reqs) r->initialised = true;
        ir.reqs.clear();
        ir.busy = false;
    }
    return NASCH_OK;
}

// Admit queued requests (oldest first) while memory and slots allow, and
// enqueue their initial state on the initialisation stream (one round; none
// while every round's staging is still in use).
int admit(nasch_server s)
{
    InitRound *round = nullptr;
    for (auto &ir : s->init)
        if (!ir.busy) {
            round = &ir;
            break;
        }
    if (!round) return NASCH_OK;
    std::vector<Request *> fresh;
    while (!s->queue.empty()) {
        Request *r = s->queue.front();
        if (r->canceled) {
            s->queue.pop_front();
            r->status = NASCH_ECANCELED;
            r->done_t = s->now();
            r->retired = true;
            s->completed.push_back(r);
            ++s->n_done;
            continue;
        }
        if (s->free_slots.empty() || (int64_t)fresh.size() >= s->max_slots) break;
        size_t off = 0;
        const size_t bytes = request_bytes(*r);
        if (!s->alloc.alloc(bytes, &off)) break;   // wait for memory (oldest first)
        size_t bm_off = 0;
        const size_t bm_bytes = ((size_t)r->rd.L + 63) / 64 * 8;
        if (r->rd.N > 0 && !s->alloc.alloc(bm_bytes, &bm_off)) {
            s->alloc.release(off, bytes);
            break;
        }
        s->queue.pop_front();
        r->off = off;
        r->bytes = bytes;
        r->bm_off = bm_off;
        r->bm_bytes = r->rd.N > 0 ? bm_bytes : 0;
        r->slot = s->free_slots.back();
        s->free_slots.pop_back();
        r->admit_t = s->now();
        char *base = static_cast<char *>(s->slab) + off;
        const size_t n = std::max<uint32_t>(r->rd.N, 1);
        size_t o = 0;
        if (r->layout == NASCH_LAYOUT_AGENT) {
            r->rd.x[0] = reinterpret_cast<int32_t *>(base + o);
            o += align256(n * 4);
            r->rd.x[1] = reinterpret_cast<int32_t *>(base + o);
            o += align256(n * 4);
            r->rd.v[0] = reinterpret_cast<uint8_t *>(base + o);
            o += align256(n);
            r->rd.v[1] = reinterpret_cast<uint8_t *>(base + o);
            o += align256(n);
        } else {
            r->rd.cells[0] = reinterpret_cast<int8_t *>(base + o);
            o += align256((size_t)r->rd.L + 16);
            r->rd.cells[1] = reinterpret_cast<int8_t *>(base + o);
            o += align256((size_t)r->rd.L + 16);
        }
        const size_t ss = align256((size_t)std::max<int64_t>(r->T, 1) * 8);
        r->rd.sum_v = reinterpret_cast<unsigned long long *>(base + o);
        r->rd.crossings = reinterpret_cast<unsigned long long *>(base + o + ss);
        const cudaStream_t is = s->init_stream;
        cudaError_t e = cudaMemsetAsync(base + o, 0, 2 * ss, is);
        if (e == cudaSuccess && r->layout == NASCH_LAYOUT_AGENT) e = cudaMemsetAsync(r->rd.v[0], 0, n, is);
        if (e == cudaSuccess && r->layout == NASCH_LAYOUT_GRID)
            e = cudaMemsetAsync(r->rd.cells[0], 0xFF, (size_t)r->rd.L, is);
        if (e == cudaSuccess && r->rd.N > 0)
            e = cudaMemsetAsync(static_cast<char *>(s->slab) + bm_off, 0, bm_bytes, is);
        if (e != cudaSuccess) return cuda_fail(e, "admit request");
        s->resident.push_back(r);
        s->streaming.push_back(r);
        if (r->rd.N > 0)
            fresh.push_back(r);
        else
            r->initialised = true;   // nothing to place (and nothing to run)
        if (r->super == 0) r->last_tick = s->harvested_seq;   // nothing to run (no steps or no cars): retire at once
    }
    if (!fresh.empty()) {
        InitRound &ir = *round;
        for (size_t i = 0; i < fresh.size(); ++i) {
            ir.h_new[i] = fresh[i]->rd;
            ir.h_bm[i] = reinterpret_cast<uint64_t *>(static_cast<char *>(s->slab) + fresh[i]->bm_off);
        }
        const cudaStream_t is = s->init_stream;
        cudaError_t e = cudaMemcpyAsync(ir.d_new, ir.h_new, fresh.size() * sizeof(BatchRoadDev), cudaMemcpyHostToDevice, is);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ir.d_bm, ir.h_bm, fresh.size() * sizeof(uint64_t *), cudaMemcpyHostToDevice, is);
        if (e == cudaSuccess) e = launch_batch_floyd(ir.d_new, (uint32_t)fresh.size(), ir.d_bm, s->sms, is);
        if (e == cudaSuccess) e = cudaEventRecord(ir.ev, is);
        if (e != cudaSuccess) return cuda_fail(e, "initialise admitted roads");
        ir.reqs = fresh;
        ir.busy = true;
        // the bit maps were only needed by the initialisation; memory given
        // out again is first touched by later work on the same stream
        // (admission clears it there), or by ticks of roads whose own
        // initialisation the host has seen finish
        for (auto *r : fresh) {
            s->alloc.release(r->bm_off, r->bm_bytes);
            r->bm_bytes = 0;
        }
    }
    return retire_ready(s);
}

// Launches of the next tick: steps_per_tick, or more while the resident
// work per launch is too small to keep the GPU busy for target_tick_ms.
int64_t tick_launches(nasch_server s, const std::vector<Request *> &act)
{
    const int64_t longest = act.front()->super - act.front()->done_super;
    int64_t M = s->cfg.steps_per_tick;
    if (s->cfg.target_tick_ms > 0.0 && s->rate > 0.0) {
        double per_launch = 0.0;   // cars x steps of one launch over every active road
        for (auto *r : act) per_launch += (double)r->rd.N * (double)r->rd.k;
        const double want = s->cfg.target_tick_ms * 1e-3 * s->rate / std::max(per_launch, 1.0);
        if (want > (double)M) M = (int64_t)std::min<double>(want, (double)s->cfg.max_steps_per_tick);
    }
    return std::min<int64_t>(M, longest);
}

// Plan and enqueue one tick over the resident roads.
int enqueue_tick(nasch_server s, TickBuf &buf)
{
    std::vector<Request *> act;
    for (auto *r : s->resident)
        if (!r->canceled && r->initialised && r->done_super < r->super) act.push_back(r);
    if (act.empty()) return NASCH_OK;
    std::stable_sort(act.begin(), act.end(), [](const Request *a, const Request *b) {
        return a->super - a->done_super > b->super - b->done_super;
    });
    const int64_t M = tick_launches(s, act);
    int64_t total = 0;
    for (auto *r : act) total += r->n_items;
    int st = ensure_items(s, total);
    if (st) return st;
    // work-list (roads by remaining super-steps, longest first) and prefix counts
    std::vector<uint32_t> active((size_t)M, 0);
    int64_t k = 0, work = 0;
    for (auto *r : act) {
        for (int64_t t = 0; t < r->n_items; ++t) buf.h_items[k++] = BatchItem{(uint32_t)r->slot, (uint32_t)t};
        const int64_t runs = std::min<int64_t>(M, r->super - r->done_super);
        for (int64_t j = 0; j < runs; ++j) active[(size_t)j] = (uint32_t)k;
        r->rd.sbase = (uint32_t)r->done_super;
        const int64_t steps_before = std::min<int64_t>(r->T, r->done_super * (int64_t)r->rd.k);
        const int64_t steps_after = std::min<int64_t>(r->T, (r->done_super + runs) * (int64_t)r->rd.k);
        work += (int64_t)r->rd.N * (steps_after - steps_before);
    }
    // every resident road's descriptor, in one copy of the slots up to the
    // highest in use (the others are never listed); the staging copy must stay
    // unchanged until this asynchronous copy has run, so each tick in flight
    // has its own staging buffers
    int top = 0;
    for (auto *r : s->resident) {
        buf.h_slots[r->slot] = r->rd;
        top = std::max(top, r->slot + 1);
    }
    Tick t;
    cudaError_t e = cudaSuccess;
    if (!s->spare_ticks.empty()) {
        t = s->spare_ticks.back();
        s->spare_ticks.pop_back();
    } else {
        e = cudaEventCreate(&t.ev0);
        if (e == cudaSuccess) e = cudaEventCreate(&t.ev);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(buf.d_items, buf.h_items, (size_t)total * sizeof(BatchItem), cudaMemcpyHostToDevice,
                            s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->d_slots, buf.h_slots, (size_t)top * sizeof(BatchRoadDev), cudaMemcpyHostToDevice,
                            s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(buf.d_counters, 0, sizeof(uint32_t) * (size_t)M, s->stream);
    if (e == cudaSuccess) e = cudaEventRecord(t.ev0, s->stream);
    for (int64_t j = 0; j < M && e == cudaSuccess; ++j) {
        BatchLaunch bl;
        bl.roads = s->d_slots;
        bl.items = buf.d_items;
        bl.n_items = active[(size_t)j];
        bl.super_step = (uint32_t)j;
        bl.counter = buf.d_counters + j;
        bl.cancel = s->d_cancel;
        bl.padded = s->padded;
        e = launch_batch_super_step(bl, (int)std::min<int64_t>(s->blocks, std::max<uint32_t>(bl.n_items, 1u)), s->stream);
    }
    t.seq = s->tick_seq++;
    t.vehicle_steps = work;
    t.launches = (int32_t)M;
    if (e == cudaSuccess) e = cudaEventRecord(t.ev, s->stream);
    if (e != cudaSuccess) {
        if (t.ev0) cudaEventDestroy(t.ev0);
        if (t.ev) cudaEventDestroy(t.ev);
        return cuda_fail(e, "enqueue tick");
    }
    s->inflight.push_back(t);
    s->last_launches = (int32_t)M;
    for (auto *r : act) {
        r->done_super += std::min<int64_t>(M, r->super - r->done_super);
        r->last_tick = t.seq;
        r->marks.emplace_back(t.seq, std::min<int64_t>(r->T, r->done_super * (int64_t)r->rd.k));
    }
    return NASCH_OK;
}

int alloc_tick_buf(nasch_server s, TickBuf &b)
{
    const size_t n = (size_t)s->max_slots;
    cudaError_t e = cudaHostAlloc((void **)&b.h_slots, sizeof(BatchRoadDev) * n, 0);
    if (e == cudaSuccess)
        e = cudaMalloc(&b.d_counters, sizeof(uint32_t) * (size_t)std::max(s->cfg.max_steps_per_tick, s->cfg.steps_per_tick));
    return e == cudaSuccess ? NASCH_OK : cuda_fail(e, "tick staging buffers");
}

int alloc_init_round(nasch_server s, InitRound &ir)
{
    const size_t n = (size_t)s->max_slots;
    cudaError_t e = cudaHostAlloc((void **)&ir.h_new, sizeof(BatchRoadDev) * n, 0);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&ir.h_bm, sizeof(uint64_t *) * n, 0);
    if (e == cudaSuccess) e = cudaMalloc(&ir.d_new, sizeof(BatchRoadDev) * n);
    if (e == cudaSuccess) e = cudaMalloc(&ir.d_bm, sizeof(uint64_t *) * n);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ir.ev, cudaEventDisableTiming);
    return e == cudaSuccess ? NASCH_OK : cuda_fail(e, "initialisation staging buffers");
}

}  // namespace

extern "C" {

void nasch_server_config_init(nasch_server_config *cfg)
{
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->memory_budget = int64_t(40) << 30;
    cfg->steps_per_tick = 8;
    cfg->max_resident = 4096;
    cfg->max_steps_per_tick = 256;
    cfg->ticks_in_flight = 3;
    cfg->target_tick_ms = 4.0;
}

int nasch_server_create(const nasch_server_config *cfg, nasch_server *out)
{
    clear_error();
    if (!cfg || !out) return fail(NASCH_EINVAL, "NULL argument");
    *out = nullptr;
    if (cfg->memory_budget < (1 << 20)) return fail(NASCH_EINVAL, "memory budget below 1 MiB");
    if (cfg->steps_per_tick < 1 || cfg->steps_per_tick > 4096) return fail(NASCH_EINVAL, "steps_per_tick outside 1..4096");
    if (cfg->max_steps_per_tick < 0 || cfg->max_steps_per_tick > 4096)
        return fail(NASCH_EINVAL, "max_steps_per_tick outside 0..4096");
    if (cfg->max_resident < 1 || cfg->max_resident > (1 << 20)) return fail(NASCH_EINVAL, "max_resident outside 1..2^20");
    if (cfg->ticks_in_flight < 0 || cfg->ticks_in_flight > kMaxTicksInFlight)
        return fail(NASCH_EINVAL, "ticks_in_flight outside 1..%d", kMaxTicksInFlight);
    if (!(cfg->target_tick_ms >= 0.0 && cfg->target_tick_ms <= 1e4))
        return fail(NASCH_EINVAL, "target_tick_ms outside 0..10000");
    nasch_server s = new (std::nothrow) nasch_server_s();
    if (!s) return fail(NASCH_ENOMEM, "host allocation");
    s->cfg = *cfg;
    if (s->cfg.max_steps_per_tick < s->cfg.steps_per_tick) s->cfg.max_steps_per_tick = s->cfg.steps_per_tick;
    s->depth = s->cfg.ticks_in_flight > 0 ? s->cfg.ticks_in_flight : 3;
    s->t0 = std::chrono::steady_clock::now();
    s->tuning = tuning_snapshot();
    int st = device_info(&s->device, &s->sms);
    if (st) {
        delete s;
        return st;
    }
    cudaError_t e;
    if (cfg->stream) {
        s->stream = (cudaStream_t)cfg->stream;
    } else {
        e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete s;
            return cuda_fail(e, "cudaStreamCreate");
        }
        s->own_stream = true;
    }
    s->max_slots = cfg->max_resident;
    s->padded = (uint32_t)kGridSpan;
    e = cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->init_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&s->slab, (size_t)cfg->memory_budget);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_slots, sizeof(BatchRoadDev) * (size_t)s->max_slots);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&s->h_cancel, sizeof(uint32_t), cudaHostAllocMapped);
    if (e == cudaSuccess) {
        *s->h_cancel = 0;
        e = cudaHostGetDevicePointer((void **)&s->d_cancel, s->h_cancel, 0);
    }
    if (e != cudaSuccess) {
        destroy_server(s);
        return e == cudaErrorMemoryAllocation ? fail(NASCH_ENOMEM, "server memory (budget %lld bytes)",
                                                     (long long)cfg->memory_budget)
                                              : cuda_fail(e, "server allocation");
    }
    for (int i = 0; i < s->depth; ++i)
        if ((st = alloc_tick_buf(s, s->bufs[i]))) {
            destroy_server(s);
            return st;
        }
    for (auto &ir : s->init)
        if ((st = alloc_init_round(s, ir))) {
            destroy_server(s);
            return st;
        }
    s->alloc.reset((size_t)cfg->memory_budget);
    for (int i = s->max_slots - 1; i >= 0; --i) s->free_slots.push_back(i);
    s->blocks = s->sms * batch_blocks_per_sm(s->padded);
    st = ensure_items(s, 4096);
    if (st) {
        destroy_server(s);
        return st;
    }
    *out = s;
    return NASCH_OK;
}

int nasch_server_submit(nasch_server s, const nasch_params *road, int64_t steps, uint64_t request_id)
{
    clear_error();
    if (!s || !road) return fail(NASCH_EINVAL, "NULL argument");
    int st = validate_params(road);
    if (st) return st;
    if (steps < 0 || steps > (int64_t)0xFFFFFFFF) return fail(NASCH_EINVAL, "steps=%lld outside 0..2^32-1", (long long)steps);
    std::lock_guard<std::mutex> g(s->mu);
    if (s->by_id.count(request_id)) return fail(NASCH_EINVAL, "request id %llu in use", (unsigned long long)request_id);
    Request *r = new (std::nothrow) Request();
    if (!r) return fail(NASCH_ENOMEM, "host allocation");
    r->id = request_id;
    r->prm = *road;
    r->prm.stream = nullptr;
    r->T = steps;
    plan_road(r->prm, steps, s->tuning, false, &r->rd, &r->layout, &r->n_items, &r->super);
    const size_t need = request_bytes(*r) + ((size_t)r->rd.L + 63) / 64 * 8 + 512;
    if (need > (size_t)s->cfg.memory_budget) {
        delete r;
        return fail(NASCH_ENOMEM, "request needs %zu bytes, more than the whole budget", need);
    }
    r->submit_t = s->now();
    s->queue.push_back(r);
    s->by_id[request_id] = r;
    return NASCH_OK;
}

int nasch_server_step(nasch_server s, int64_t *pending)
{
    clear_error();
    TraceRange trace("nasch_server_step");
    if (!s) return fail(NASCH_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> g(s->mu);
    int st = harvest(s, false);
    if (st) return st;
    if ((int)s->inflight.size() >= s->depth) {
        st = harvest(s, true);
        if (st) return st;
    }
    TickBuf &buf = s->bufs[s->tick_seq % s->depth];
    st = poll_init(s);
    if (st == NASCH_OK) st = retire_ready(s);   // roads with nothing to run, now initialised
    if (st) return st;
    st = admit(s);
    if (st) return st;
    st = enqueue_tick(s, buf);
    if (st) return st;
    if (s->inflight.empty() && !s->resident.empty()) st = retire_ready(s);
    if (pending) *pending = (int64_t)(s->queue.size() + s->resident.size());
    return st;
}

int nasch_server_drain(nasch_server s, int64_t timeout_ms)
{
    clear_error();
    if (!s) return fail(NASCH_EINVAL, "server is NULL");
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        int64_t pending = 0;
        int st = nasch_server_step(s, &pending);
        if (st) return st;
        {
            std::lock_guard<std::mutex> g(s->mu);
            if (pending == 0 && s->inflight.empty()) return NASCH_OK;
            if (s->resident.empty() && !s->queue.empty() && s->inflight.empty())
                return fail(NASCH_ENOMEM, "the oldest queued request does not fit the free budget");
        }
        if (timeout_ms >= 0 &&
            std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count() >=
                timeout_ms)
            return fail(NASCH_ETIMEOUT, "requests still pending after %lld ms", (long long)timeout_ms);
    }
}

int nasch_server_poll(nasch_server s, nasch_request_result *out, int64_t cap, int64_t *n_out)
{
    clear_error();
    if (!s || !n_out || (cap > 0 && !out)) return fail(NASCH_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> g(s->mu);
    const int64_t n = std::min<int64_t>(cap, (int64_t)s->completed.size());
    for (int64_t i = 0; i < n; ++i) {
        const Request *r = s->completed[(size_t)i];
        nasch_request_result &o = out[i];
        o.request_id = r->id;
        o.status = r->status;
        o.layout = r->layout;
        o.steps = r->T;
        o.vehicles = r->rd.N;
        o.submit_time = r->submit_t;
        o.admit_time = r->admit_t;
        o.done_time = r->done_t;
    }
    s->completed.erase(s->completed.begin(), s->completed.begin() + n);
    *n_out = n;
    return NASCH_OK;
}

int nasch_server_poll_series(nasch_server s, nasch_series_chunk *chunks, int64_t cap_chunks, uint64_t *sum_v_host,
                             uint64_t *crossings_host, int64_t cap_steps, int64_t *n_chunks)
{
    clear_error();
    if (!s || !n_chunks || (cap_chunks > 0 && !chunks) || cap_chunks < 0 || cap_steps < 0)
        return fail(NASCH_EINVAL, "NULL or negative argument");
    std::lock_guard<std::mutex> g(s->mu);
    int st = harvest(s, false);   // make the ticks that have finished count
    if (st) return st;
    int64_t n = 0, used = 0;
    cudaError_t e = cudaSuccess;
    std::vector<Request *> keep;
    keep.reserve(s->streaming.size());
    for (auto *r : s->streaming) {
        const int64_t avail = r->ready - r->sent;
        if (avail > 0 && n < cap_chunks && used < cap_steps && e == cudaSuccess) {
            const int64_t cnt = std::min<int64_t>(avail, cap_steps - used);
            const int64_t first = r->sent;
            if (r->retired) {   // the series is on the host
                if (sum_v_host) std::copy(r->sum_v.begin() + first, r->sum_v.begin() + first + cnt, sum_v_host + used);
                if (crossings_host)
                    std::copy(r->crossings.begin() + first, r->crossings.begin() + first + cnt, crossings_host + used);
            } else {            // steps written by finished ticks: read them from the device
                if (sum_v_host)
                    e = cudaMemcpyAsync(sum_v_host + used, r->rd.sum_v + first, (size_t)cnt * 8, cudaMemcpyDeviceToHost,
                                        s->copy_stream);
                if (e == cudaSuccess && crossings_host)
                    e = cudaMemcpyAsync(crossings_host + used, r->rd.crossings + first, (size_t)cnt * 8,
                                        cudaMemcpyDeviceToHost, s->copy_stream);
            }
            if (e == cudaSuccess) {
                chunks[n++] = nasch_series_chunk{r->id, first, cnt, used};
                used += cnt;
                r->sent += cnt;
            }
        }
        // a request leaves the list once all of its series has been returned
        // (or it was cancelled and retired)
        if (!(r->retired && (r->sent >= r->T || r->canceled))) keep.push_back(r);
    }
    s->streaming.swap(keep);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->copy_stream);
    *n_chunks = n;
    return e == cudaSuccess ? NASCH_OK : cuda_fail(e, "copy streamed series");
}

int nasch_server_result(nasch_server s, uint64_t request_id, uint64_t *sum_v_host, uint64_t *crossings_host,
                        int64_t cap_steps, int32_t *x_host, uint8_t *v_host, int64_t cap_cars)
{
    clear_error();
    if (!s) return fail(NASCH_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->by_id.find(request_id);
    if (it == s->by_id.end()) return fail(NASCH_EINVAL, "no request %llu", (unsigned long long)request_id);
    Request *r = it->second;
    if (r->done_t == 0) return fail(NASCH_EBUSY, "request %llu has not finished", (unsigned long long)request_id);
    if (r->status != NASCH_OK) return fail(r->status, "request %llu was cancelled", (unsigned long long)request_id);
    if ((sum_v_host || crossings_host) && cap_steps < r->T) return fail(NASCH_EINVAL, "cap_steps < steps");
    if (sum_v_host) std::copy(r->sum_v.begin(), r->sum_v.end(), sum_v_host);
    if (crossings_host) std::copy(r->crossings.begin(), r->crossings.end(), crossings_host);
    if (x_host || v_host) {
        if (!s->cfg.keep_state) return fail(NASCH_EINVAL, "the server was created without keep_state");
        if (cap_cars < (int64_t)r->x.size()) return fail(NASCH_EINVAL, "cap_cars < N");
        if (x_host) std::copy(r->x.begin(), r->x.end(), x_host);
        if (v_host) std::copy(r->v.begin(), r->v.end(), v_host);
    }
    return NASCH_OK;
}

int nasch_server_release(nasch_server s, uint64_t request_id)
{
    clear_error();
    if (!s) return fail(NASCH_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->by_id.find(request_id);
    if (it == s->by_id.end()) return fail(NASCH_EINVAL, "no request %llu", (unsigned long long)request_id);
    Request *r = it->second;
    if (r->done_t == 0) return fail(NASCH_EBUSY, "request %llu has not finished", (unsigned long long)request_id);
    for (auto *c : s->completed)
        if (c == r) return fail(NASCH_EBUSY, "request %llu has not been polled", (unsigned long long)request_id);
    // a series not yet streamed is dropped with the request
    s->streaming.erase(std::remove(s->streaming.begin(), s->streaming.end(), r), s->streaming.end());
    s->by_id.erase(it);
    delete r;
    return NASCH_OK;
}

int nasch_server_cancel(nasch_server s, uint64_t request_id)
{
    clear_error();
    if (!s) return fail(NASCH_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->by_id.find(request_id);
    if (it == s->by_id.end()) return fail(NASCH_EINVAL, "no request %llu", (unsigned long long)request_id);
    if (it->second->done_t != 0) return fail(NASCH_EINVAL, "request %llu already finished", (unsigned long long)request_id);
    it->second->canceled = true;
    return NASCH_OK;
}

int nasch_server_get_info(nasch_server s, nasch_server_info *info)
{
    clear_error();
    if (!s || !info) return fail(NASCH_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> g(s->mu);
    std::memset(info, 0, sizeof(*info));
    info->queued = (int64_t)s->queue.size();
    info->resident = (int64_t)s->resident.size();
    info->completed = s->n_done;
    info->bytes_in_use = (int64_t)s->alloc.used();
    info->ticks = s->tick_seq;
    info->vehicle_steps_done = s->vehicle_steps_done;
    info->blocks = s->blocks;
    info->now = s->now();
    info->gpu_busy_seconds = s->gpu_busy;
    info->last_tick_super_steps = s->last_launches;
    return NASCH_OK;
}

void nasch_server_destroy(nasch_server s) { destroy_server(s); }

}  // extern "C"
