// Batched runs: planning, memory, initialisation, CUDA-graph capture of the
// super-step launches, and the C ABI of nasch_submit / nasch_batch_*.
//
// Plan.  Road i gets a layout (AUTO: agent below the density rho_star, grid
// above), a kind of item (tiles, or one whole-ring item for small roads), a
// fusion depth k_i and S_i = ceil(T_i / k_i) super-steps.  Roads are sorted
// by S_i, longest first, and their items listed in that order, so the items
// still active at super-step s are a prefix of the list whose length the
// host knows in advance; every launch gets its own work-list cursor, so the
// whole sequence is captured once into CUDA graphs and replayed without
// host work.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <mutex>
#include <new>
#include <numeric>
#include <thread>
#include <vector>

#include "nasch.h"
#include "batch_internal.h"
#include "runtime_internal.h"

namespace nasch {

namespace {

std::mutex g_tuning_mu;
// AUTO picks the agent layout below this density.  With fused steps both
// layouts are bound by the step's arithmetic, not by HBM, and the agent step
// is the cheaper one at every density measured, so the default is 1;
// auto_rho_star falls back to kBytesRhoStar when memory is short.
double g_rho_star = 1.0;
constexpr double kBytesRhoStar = 0.2;   // state bytes equal: agent 10 per car, grid 2 per cell
constexpr double kMemoryShare = 0.85;   // a batch may plan for this share of the free device memory
int g_k_agent = 8;
int g_k_grid = 8;
std::vector<nasch_tuning_entry> g_table;   // per-road tuning, first match wins
constexpr int kRingK = 8;   // steps per item of whole-ring roads
constexpr int64_t kGraphChunk = 2048;   // super-steps per captured graph

uint32_t round_up(uint32_t a, uint32_t m) { return (a + m - 1u) / m * m; }

}  // namespace

double auto_rho_star(const nasch_params *roads, int64_t n)
{
    double rho;
    {
        std::lock_guard<std::mutex> g(g_tuning_mu);
        rho = g_rho_star;
    }
    if (rho <= kBytesRhoStar) return rho;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return kBytesRhoStar;
    }
    double bytes = 0.0;   // state of the AUTO roads at rho (two buffers each)
    for (int64_t i = 0; i < n; ++i) {
        if (roads[i].layout != NASCH_LAYOUT_AUTO) continue;
        bytes += (double)roads[i].N < rho * (double)roads[i].L ? 10.0 * (double)roads[i].N : 2.0 * (double)roads[i].L;
    }
    return bytes <= 0.5 * (double)free_b ? rho : kBytesRhoStar;
}

TuningSnapshot tuning_snapshot()
{
    std::lock_guard<std::mutex> g(g_tuning_mu);
    TuningSnapshot ts;
    ts.rho_star = g_rho_star;
    ts.k_agent = g_k_agent;
    ts.k_grid = g_k_grid;
    ts.table = g_table;
    return ts;
}

namespace {

// rule-3 draw mode of a road as the table keys it: 0 never, 1 draws, 2 always
int draw_key(double p)
{
    const uint64_t thr = slow_threshold(p);
    return thr == 0 ? 0 : (thr > 0xFFFFFFFFull ? 2 : 1);
}

const nasch_tuning_entry *match_entry(const TuningSnapshot &ts, const nasch_params &p)
{
    if (ts.table.empty()) return nullptr;
    const double rho = (double)p.N / (double)p.L;
    const int dk = draw_key(p.p);
    for (const auto &e : ts.table)
        if (p.L >= e.L_min && p.L < e.L_max && rho >= e.rho_min && rho < e.rho_max && p.vmax >= e.vmax_min &&
            p.vmax <= e.vmax_max && (e.draw < 0 || e.draw == dk))
            return &e;
    return nullptr;
}

int resolve_layout(const nasch_params &p, const TuningSnapshot &ts, bool memory_short, const nasch_tuning_entry *e)
{
    if (p.layout != NASCH_LAYOUT_AUTO) return p.layout;
    if (!memory_short && e && e->layout != NASCH_LAYOUT_AUTO) return e->layout;
    const double rho_star = memory_short ? kBytesRhoStar : ts.rho_star;
    return (double)p.N < rho_star * (double)p.L ? NASCH_LAYOUT_AGENT : NASCH_LAYOUT_GRID;
}

}  // namespace

bool auto_memory_short(const nasch_params *roads, int64_t n, const int64_t *steps, const TuningSnapshot &ts)
{
    // the batch's device memory with its AUTO roads laid out as chosen: two
    // state buffers, the statistics and (while the start states are built)
    // the bit maps; explicit layouts count at what they are
    double state = 0.0, other = 0.0, auto_state = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const int lay = resolve_layout(roads[i], ts, false, match_entry(ts, roads[i]));
        const double b = lay == NASCH_LAYOUT_AGENT ? 10.0 * (double)roads[i].N : 2.0 * (double)roads[i].L;
        state += b;
        if (roads[i].layout == NASCH_LAYOUT_AUTO) auto_state += b;
        other += 16.0 * (double)(steps ? std::max<int64_t>(steps[i], 1) : 1) + (double)roads[i].L / 8.0;
    }
    if (auto_state == 0.0) return false;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return state + other > kMemoryShare * (double)free_b;
}

void plan_road(const nasch_params &p, int64_t T, const TuningSnapshot &ts, bool memory_short, BatchRoadDev *out,
               int *layout_out, int64_t *n_items, int64_t *super)
{
    BatchRoadDev &rd = *out;
    std::memset(&rd, 0, sizeof(rd));
    const nasch_tuning_entry *e = match_entry(ts, p);
    const int layout = resolve_layout(p, ts, memory_short, e);
    *layout_out = layout;
    const int k_tuned = e && e->k > 0 ? e->k : 0;
    rd.L = (uint32_t)p.L;
    rd.N = (uint32_t)p.N;
    rd.vmax = (uint32_t)p.vmax;
    rd.thr = slow_threshold(p.p);
    rd.key0 = (uint32_t)p.seed;
    rd.key1 = (uint32_t)(p.seed >> 32);
    rd.road_id = p.road_id;
    rd.T = (uint32_t)T;
    int k;
    if (layout == NASCH_LAYOUT_AGENT) {
        if (p.N <= (int64_t)kBatchRingCars) {
            rd.type = kBatchAgentRing;
            k = p.k ? p.k : (k_tuned ? k_tuned : kRingK);
            *n_items = 1;
        } else {
            rd.type = kBatchAgentTile;
            k = p.k ? p.k : (k_tuned ? k_tuned : ts.k_agent);
            rd.halo = round_up((uint32_t)k, (uint32_t)kBatchAgentTileR);
            rd.tile = kBatchAgentSpan - rd.halo;
            const int64_t per_item = (int64_t)rd.tile * (kBatchThreads / 32) * kBatchWarpTilesPerWarp;
            *n_items = (p.N + per_item - 1) / per_item;
        }
    } else {
        if (p.L <= (int64_t)kBatchRingCells) {
            rd.type = kBatchGridRing;
            k = p.k ? p.k : (k_tuned ? k_tuned : kRingK);
            *n_items = 1;
        } else {
            k = p.k ? p.k : (k_tuned ? k_tuned : ts.k_grid);
            const int kfit = p.vmax > 0 ? std::max(1, (kGridSpan / 2 - 16) / p.vmax) : kMaxFusedSteps;
            k = std::min(k, kfit);
            rd.halo = grid_halo(k, (uint32_t)p.vmax);
            // tile: the road's own (8192 = block-wide spans), else the table's
            const int tile = p.tile ? p.tile : (e ? e->tile : 0);
            if (rd.halo <= kKwMaxHalo && tile != kGridTileCells) {   // warp-tiles of the list method
                rd.type = kBatchGridWarp;
                rd.tile = kKwSpan - 2u * rd.halo;
                const int64_t per_item = (int64_t)rd.tile * (kBatchThreads / 32);
                *n_items = (p.L + per_item - 1) / per_item;
            } else {                       // one block-wide span per item
                rd.type = kBatchGridTile;
                rd.tile = (uint32_t)kGridSpan - 2u * rd.halo;
                *n_items = (p.L + rd.tile - 1) / rd.tile;
            }
        }
    }
    rd.k = (uint32_t)k;
    *super = rd.T == 0 ? 0 : (rd.T + rd.k - 1) / rd.k;
    if (rd.N == 0) {
        *super = 0;
        *n_items = 0;
    }
}

}  // namespace nasch

using namespace nasch;

struct nasch_batch_s {
    int device = 0, sms = 1;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int64_t n = 0;
    std::vector<BatchRoadDev> roads;   // host copy with device pointers
    std::vector<int32_t> layout;       // NASCH_LAYOUT_* per road
    std::vector<int64_t> super;        // S_i
    void *pool = nullptr;
    size_t pool_bytes = 0;
    BatchRoadDev *d_roads = nullptr;
    BatchItem *d_items = nullptr;
    uint32_t *d_counters = nullptr;
    uint32_t *h_cancel = nullptr;      // pinned, mapped
    uint32_t *d_cancel = nullptr;
    int64_t n_super = 0, first_items = 0, vehicle_steps = 0, cell_steps = 0;
    int blocks = 1;
    uint32_t padded = 0;
    std::vector<cudaGraphExec_t> execs;
    std::vector<cudaGraph_t> graphs;
    cudaEvent_t done = nullptr;
    cudaEvent_t started = nullptr;     // recorded after initialisation, before the first launch
    bool canceled = false;
    bool finished = false;
};

namespace {

void free_batch(nasch_batch b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (auto e : b->execs) cudaGraphExecDestroy(e);
    for (auto g : b->graphs) cudaGraphDestroy(g);
    if (b->done) cudaEventDestroy(b->done);
    if (b->started) cudaEventDestroy(b->started);
    cudaFree(b->pool);
    cudaFree(b->d_roads);
    cudaFree(b->d_items);
    cudaFree(b->d_counters);
    if (b->h_cancel) cudaFreeHost(b->h_cancel);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

int check_road_index(nasch_batch b, int64_t i)
{
    if (!b) return fail(NASCH_EINVAL, "batch is NULL");
    if (i < 0 || i >= b->n) return fail(NASCH_EINVAL, "road %lld outside 0..%lld", (long long)i, (long long)(b->n - 1));
    return NASCH_OK;
}

// Wait for the batch; returns OK, ETIMEOUT or ECANCELED.
int wait_batch(nasch_batch b, int64_t timeout_ms)
{
    if (!b->finished) {
        const auto t0 = std::chrono::steady_clock::now();
        for (;;) {
            const cudaError_t q = cudaEventQuery(b->done);
            if (q == cudaSuccess) break;
            if (q != cudaErrorNotReady) return cuda_fail(q, "batch completion event");
            if (timeout_ms >= 0 &&
                std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count() >=
                    timeout_ms)
                return fail(NASCH_ETIMEOUT, "batch still running after %lld ms", (long long)timeout_ms);
            std::this_thread::sleep_for(std::chrono::microseconds(50));
        }
        b->finished = true;
#ifdef NASCH_DEBUG
        if (const unsigned int w = debug_word_batch() | debug_word_agent() | debug_word_grid())
            return fail(NASCH_EINVAL, "debug check failed in the batch kernels (sites 0x%x)", w);
#endif
    }
    if (b->canceled) return fail(NASCH_ECANCELED, "batch was cancelled");
    return NASCH_OK;
}

}  // namespace

extern "C" {

int nasch_set_tuning(double rho_star, int32_t k_agent, int32_t k_grid)
{
    clear_error();
    if (!(rho_star >= 0.0 && rho_star <= 1.0)) return fail(NASCH_EINVAL, "rho_star=%g outside [0, 1]", rho_star);
    if (k_agent < 0 || k_agent > kMaxFusedSteps || k_grid < 0 || k_grid > kMaxFusedSteps)
        return fail(NASCH_EINVAL, "k outside 0..%d", kMaxFusedSteps);
    std::lock_guard<std::mutex> g(g_tuning_mu);
    g_rho_star = rho_star;
    if (k_agent) g_k_agent = k_agent;
    if (k_grid) g_k_grid = k_grid;
    return NASCH_OK;
}

int nasch_set_tuning_table(const nasch_tuning_entry *entries, int64_t n)
{
    clear_error();
    if (n < 0 || (n > 0 && !entries)) return fail(NASCH_EINVAL, "bad table");
    if (n > (1 << 20)) return fail(NASCH_EINVAL, "table of %lld entries too long", (long long)n);
    for (int64_t i = 0; i < n; ++i) {
        const nasch_tuning_entry &e = entries[i];
        if (!(e.L_min < e.L_max) || !(e.rho_min < e.rho_max) || e.vmax_min > e.vmax_max || e.draw < -1 ||
            e.draw > 2)
            return fail(NASCH_EINVAL, "entry %lld: empty or unknown bucket", (long long)i);
        if (e.layout < NASCH_LAYOUT_AUTO || e.layout > NASCH_LAYOUT_GRID)
            return fail(NASCH_EINVAL, "entry %lld: layout=%d unknown", (long long)i, e.layout);
        if (e.k < 0 || e.k > kMaxFusedSteps) return fail(NASCH_EINVAL, "entry %lld: k=%d outside 0..%d", (long long)i, e.k, kMaxFusedSteps);
        if (e.tile != 0 && e.tile != (int32_t)kKwSpan && e.tile != kGridTileCells)
            return fail(NASCH_EINVAL, "entry %lld: tile=%d not 0, %u or %d", (long long)i, e.tile, kKwSpan, kGridTileCells);
    }
    std::lock_guard<std::mutex> g(g_tuning_mu);
    g_table.assign(entries, entries + n);
    return NASCH_OK;
}

int nasch_get_tuning_table(nasch_tuning_entry *out, int64_t cap, int64_t *n)
{
    clear_error();
    if (!n || cap < 0 || (cap > 0 && !out)) return fail(NASCH_EINVAL, "bad arguments");
    std::lock_guard<std::mutex> g(g_tuning_mu);
    *n = (int64_t)g_table.size();
    for (int64_t i = 0; i < std::min<int64_t>(cap, *n); ++i) out[i] = g_table[(size_t)i];
    return NASCH_OK;
}

int nasch_tuned_choice(const nasch_params *road, int32_t *layout, int32_t *k, int32_t *tile)
{
    clear_error();
    int st = validate_params(road);
    if (st) return st;
    BatchRoadDev rd;
    int lay = 0;
    int64_t items = 0, super = 0;
    plan_road(*road, 1, tuning_snapshot(), false, &rd, &lay, &items, &super);
    if (layout) *layout = lay;
    if (k) *k = (int32_t)rd.k;
    if (tile) {
        switch (rd.type) {
        case kBatchGridWarp: *tile = (int32_t)kKwSpan; break;
        case kBatchGridTile: *tile = kGridTileCells; break;
        case kBatchAgentTile: *tile = (int32_t)kBatchAgentSpan; break;
        default: *tile = 0; break;
        }
    }
    return NASCH_OK;
}

int nasch_get_tuning(double *rho_star, int32_t *k_agent, int32_t *k_grid)
{
    clear_error();
    std::lock_guard<std::mutex> g(g_tuning_mu);
    if (rho_star) *rho_star = g_rho_star;
    if (k_agent) *k_agent = g_k_agent;
    if (k_grid) *k_grid = g_k_grid;
    return NASCH_OK;
}

int nasch_submit(const nasch_params *roads, int64_t n_roads, const int64_t *steps, nasch_batch *out)
{
    clear_error();
    TraceRange trace("nasch_submit");
    if (!out) return fail(NASCH_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_roads <= 0 || !roads || !steps) return fail(NASCH_EINVAL, "no roads");
    if (n_roads > (int64_t)0x7FFFFFFF) return fail(NASCH_EINVAL, "too many roads");
    for (int64_t i = 0; i < n_roads; ++i) {
        int st = validate_params(&roads[i]);
        if (st) return fail(st, "road %lld: %s", (long long)i, nasch_last_error());
        if (steps[i] < 0 || steps[i] > (int64_t)0xFFFFFFFF)
            return fail(NASCH_EINVAL, "road %lld: steps=%lld outside 0..2^32-1", (long long)i, (long long)steps[i]);
    }
    nasch_batch b = new (std::nothrow) nasch_batch_s();
    if (!b) return fail(NASCH_ENOMEM, "host allocation");
    b->n = n_roads;
    int st = device_info(&b->device, &b->sms);
    if (st) {
        delete b;
        return st;
    }
    cudaError_t e;
    if (roads[0].stream) {
        b->stream = (cudaStream_t)roads[0].stream;
    } else {
        e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete b;
            return cuda_fail(e, "cudaStreamCreate");
        }
        b->own_stream = true;
    }

    // ---------------------------------------------------------------- plan
    const TuningSnapshot ts = tuning_snapshot();
    const bool memory_short = auto_memory_short(roads, n_roads, steps, ts);
    b->roads.resize((size_t)n_roads);
    b->layout.resize((size_t)n_roads);
    b->super.resize((size_t)n_roads);
    std::vector<int64_t> n_items((size_t)n_roads);
    uint32_t max_vmax_grid = 0;
    for (int64_t i = 0; i < n_roads; ++i) {
        int layout = 0;
        plan_road(roads[i], steps[i], ts, memory_short, &b->roads[(size_t)i], &layout, &n_items[(size_t)i],
                  &b->super[(size_t)i]);
        b->layout[(size_t)i] = layout;
        if (layout == NASCH_LAYOUT_GRID) max_vmax_grid = std::max(max_vmax_grid, (uint32_t)roads[i].vmax);
        b->vehicle_steps += (int64_t)roads[i].N * steps[i];
        b->cell_steps += roads[i].L * steps[i];
    }
    b->padded = (uint32_t)kGridSpan;   // ring buffers; grid tiles use the span-list method
    std::vector<int64_t> order((size_t)n_roads);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int64_t a, int64_t c) { return b->super[(size_t)a] > b->super[(size_t)c]; });
    std::vector<BatchItem> items;
    std::vector<int64_t> prefix((size_t)n_roads + 1, 0);   // items of the first j roads in order
    int64_t total_items = 0;
    for (int64_t j = 0; j < n_roads; ++j) {
        total_items += n_items[(size_t)order[(size_t)j]];
        prefix[(size_t)j + 1] = total_items;
    }
    if (total_items > (int64_t)0xFFFFFFF0) {
        free_batch(b);
        return fail(NASCH_EINVAL, "too many work items (%lld)", (long long)total_items);
    }
    try {
        items.reserve((size_t)total_items);
    } catch (const std::bad_alloc &) {
        free_batch(b);
        return fail(NASCH_ENOMEM, "host work-list");
    }
    for (int64_t j = 0; j < n_roads; ++j) {
        const int64_t r = order[(size_t)j];
        for (int64_t t = 0; t < n_items[(size_t)r]; ++t) items.push_back(BatchItem{(uint32_t)r, (uint32_t)t});
    }
    b->n_super = n_roads > 0 ? b->super[(size_t)order[0]] : 0;
    b->first_items = total_items;

    // ---------------------------------------------------------------- memory
    auto align = [](size_t x) { return (x + 255u) & ~(size_t)255u; };
    size_t bytes = 0;
    std::vector<size_t> off_state((size_t)n_roads), off_stats((size_t)n_roads);
    size_t cells_begin = 0, cells_end = 0, v_begin = 0, v_end = 0;
    // agent x buffers, then v buffers, then grid cells, then statistics: each kind contiguous
    for (int64_t i = 0; i < n_roads; ++i)
        if (b->layout[(size_t)i] == NASCH_LAYOUT_AGENT) {
            off_state[(size_t)i] = bytes;
            bytes += 2 * align((size_t)std::max<uint32_t>(b->roads[(size_t)i].N, 1) * 4);
        }
    v_begin = bytes;
    std::vector<size_t> off_v((size_t)n_roads, 0);
    for (int64_t i = 0; i < n_roads; ++i)
        if (b->layout[(size_t)i] == NASCH_LAYOUT_AGENT) {
            off_v[(size_t)i] = bytes;
            bytes += 2 * align((size_t)std::max<uint32_t>(b->roads[(size_t)i].N, 1));
        }
    v_end = bytes;
    cells_begin = bytes;
    for (int64_t i = 0; i < n_roads; ++i)
        if (b->layout[(size_t)i] == NASCH_LAYOUT_GRID) {
            off_state[(size_t)i] = bytes;
            bytes += 2 * align((size_t)b->roads[(size_t)i].L + 16);
        }
    cells_end = bytes;
    const size_t stats_begin = bytes;
    for (int64_t i = 0; i < n_roads; ++i) {
        off_stats[(size_t)i] = bytes;
        bytes += 2 * align((size_t)std::max<uint32_t>(b->roads[(size_t)i].T, 1) * 8);
    }
    const size_t stats_end = bytes;
    b->pool_bytes = bytes;
    e = cudaMalloc(&b->pool, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_roads, sizeof(BatchRoadDev) * (size_t)n_roads);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_items, sizeof(BatchItem) * (size_t)std::max<int64_t>(total_items, 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counters, sizeof(uint32_t) * (size_t)std::max<int64_t>(b->n_super, 1));
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&b->h_cancel, sizeof(uint32_t), cudaHostAllocMapped);
    if (e == cudaSuccess) {
        *b->h_cancel = 0;
        e = cudaHostGetDevicePointer((void **)&b->d_cancel, b->h_cancel, 0);
    }
    if (e != cudaSuccess) {
        free_batch(b);
        return e == cudaErrorMemoryAllocation ? fail(NASCH_ENOMEM, "batch needs %.2f GB of device memory", bytes / 1e9)
                                              : cuda_fail(e, "batch allocation");
    }
    char *base = static_cast<char *>(b->pool);
    for (int64_t i = 0; i < n_roads; ++i) {
        BatchRoadDev &rd = b->roads[(size_t)i];
        if (b->layout[(size_t)i] == NASCH_LAYOUT_AGENT) {
            const size_t xs = align((size_t)std::max<uint32_t>(rd.N, 1) * 4), vs = align((size_t)std::max<uint32_t>(rd.N, 1));
            rd.x[0] = reinterpret_cast<int32_t *>(base + off_state[(size_t)i]);
            rd.x[1] = reinterpret_cast<int32_t *>(base + off_state[(size_t)i] + xs);
            rd.v[0] = reinterpret_cast<uint8_t *>(base + off_v[(size_t)i]);
            rd.v[1] = reinterpret_cast<uint8_t *>(base + off_v[(size_t)i] + vs);
        } else {
            const size_t cs = align((size_t)rd.L + 16);
            rd.cells[0] = reinterpret_cast<int8_t *>(base + off_state[(size_t)i]);
            rd.cells[1] = reinterpret_cast<int8_t *>(base + off_state[(size_t)i] + cs);
        }
        const size_t ss = align((size_t)std::max<uint32_t>(rd.T, 1) * 8);
        rd.sum_v = reinterpret_cast<unsigned long long *>(base + off_stats[(size_t)i]);
        rd.crossings = reinterpret_cast<unsigned long long *>(base + off_stats[(size_t)i] + ss);
    }

    // ---------------------------------------------------------------- initial state (Floyd on the GPU)
    e = cudaMemcpyAsync(b->d_roads, b->roads.data(), sizeof(BatchRoadDev) * (size_t)n_roads, cudaMemcpyHostToDevice,
                        b->stream);
    if (e == cudaSuccess && total_items)
        e = cudaMemcpyAsync(b->d_items, items.data(), sizeof(BatchItem) * (size_t)total_items, cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess && v_end > v_begin) e = cudaMemsetAsync(base + v_begin, 0, v_end - v_begin, b->stream);
    if (e == cudaSuccess && cells_end > cells_begin)
        e = cudaMemsetAsync(base + cells_begin, 0xFF, cells_end - cells_begin, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + stats_begin, 0, stats_end - stats_begin, b->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(b->d_counters, 0, sizeof(uint32_t) * (size_t)std::max<int64_t>(b->n_super, 1), b->stream);
    // bit maps of the Floyd sets: scratch for the initialisation only
    size_t bm_words = 0;
    std::vector<size_t> bm_off((size_t)n_roads);
    for (int64_t i = 0; i < n_roads; ++i) {
        bm_off[(size_t)i] = bm_words;
        bm_words += ((size_t)b->roads[(size_t)i].L + 63) / 64;
    }
    uint64_t *d_bm = nullptr;
    uint64_t **d_bm_ptrs = nullptr;
    if (e == cudaSuccess) e = cudaMallocAsync(&d_bm, bm_words * 8, b->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_bm_ptrs, sizeof(uint64_t *) * (size_t)n_roads, b->stream);
    std::vector<uint64_t *> bm_ptrs((size_t)n_roads);
    if (e == cudaSuccess) {
        for (int64_t i = 0; i < n_roads; ++i) bm_ptrs[(size_t)i] = d_bm + bm_off[(size_t)i];
        e = cudaMemsetAsync(d_bm, 0, bm_words * 8, b->stream);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_bm_ptrs, bm_ptrs.data(), sizeof(uint64_t *) * (size_t)n_roads, cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess) e = launch_batch_floyd(b->d_roads, (uint32_t)n_roads, d_bm_ptrs, b->sms, b->stream);
    if (d_bm) cudaFreeAsync(d_bm, b->stream);
    if (d_bm_ptrs) cudaFreeAsync(d_bm_ptrs, b->stream);
    // host copies above read pageable vectors; wait before they go out of scope
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        free_batch(b);
        return cuda_fail(e, "batch initialisation");
    }

    // ---------------------------------------------------------------- launches, captured in graphs
    b->blocks = b->sms * batch_blocks_per_sm(b->padded);
    e = cudaEventCreate(&b->done);
    if (e == cudaSuccess) e = cudaEventCreate(&b->started);
    std::vector<uint32_t> active((size_t)std::max<int64_t>(b->n_super, 1));
    {
        // roads with S > s are a prefix of `order`; its length only falls as s grows
        int64_t cnt = n_roads;
        for (int64_t s = 0; s < b->n_super; ++s) {
            while (cnt > 0 && b->super[(size_t)order[(size_t)cnt - 1]] <= s) --cnt;
            active[(size_t)s] = (uint32_t)prefix[(size_t)cnt];
        }
    }
    for (int64_t c0 = 0; e == cudaSuccess && c0 < b->n_super; c0 += kGraphChunk) {
        const int64_t c1 = std::min<int64_t>(b->n_super, c0 + kGraphChunk);
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) break;
        cudaError_t le = cudaSuccess;
        for (int64_t s = c0; s < c1 && le == cudaSuccess; ++s) {
            BatchLaunch bl;
            bl.roads = b->d_roads;
            bl.items = b->d_items;
            bl.n_items = active[(size_t)s];
            bl.super_step = (uint32_t)s;
            bl.counter = b->d_counters + s;
            bl.cancel = b->d_cancel;
            bl.padded = b->padded;
            const int blocks = (int)std::min<int64_t>(b->blocks, std::max<uint32_t>(bl.n_items, 1u));
            le = launch_batch_super_step(bl, blocks, b->stream);
        }
        e = cudaStreamEndCapture(b->stream, &g);
        if (le != cudaSuccess) e = le;
        if (e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            break;
        }
        b->graphs.push_back(g);
        cudaGraphExec_t x = nullptr;
        e = cudaGraphInstantiate(&x, g, 0);
        if (e == cudaSuccess) b->execs.push_back(x);
    }
    if (e == cudaSuccess) e = cudaEventRecord(b->started, b->stream);
    for (size_t gi = 0; e == cudaSuccess && gi < b->execs.size(); ++gi) e = cudaGraphLaunch(b->execs[gi], b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(b->done, b->stream);
    if (e != cudaSuccess) {
        free_batch(b);
        return cuda_fail(e, "batch launch");
    }
    *out = b;
    return NASCH_OK;
}

int nasch_batch_wait(nasch_batch b, int64_t timeout_ms)
{
    clear_error();
    if (!b) return fail(NASCH_EINVAL, "batch is NULL");
    return wait_batch(b, timeout_ms);
}

int nasch_batch_cancel(nasch_batch b)
{
    clear_error();
    if (!b) return fail(NASCH_EINVAL, "batch is NULL");
    *(volatile uint32_t *)b->h_cancel = 1u;
    b->canceled = true;
    return NASCH_OK;
}

int nasch_batch_read_state(nasch_batch b, int64_t i, int32_t *x_host, uint8_t *v_host, int64_t cap)
{
    clear_error();
    int st = check_road_index(b, i);
    if (st) return st;
    if ((st = wait_batch(b, -1))) return st;
    const BatchRoadDev &rd = b->roads[(size_t)i];
    if (cap < (int64_t)rd.N) return fail(NASCH_EINVAL, "cap=%lld < N=%u", (long long)cap, rd.N);
    if (rd.N == 0) return NASCH_OK;
    if (!x_host || !v_host) return fail(NASCH_EINVAL, "NULL output array");
    const int par = (int)(b->super[(size_t)i] & 1);
    cudaError_t e;
    if (b->layout[(size_t)i] == NASCH_LAYOUT_AGENT) {
        e = cudaMemcpy(x_host, rd.x[par], (size_t)rd.N * 4, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(v_host, rd.v[par], (size_t)rd.N, cudaMemcpyDeviceToHost);
        return e == cudaSuccess ? NASCH_OK : cuda_fail(e, "read batch state");
    }
    std::vector<int8_t> cells((size_t)rd.L);
    e = cudaMemcpy(cells.data(), rd.cells[par], (size_t)rd.L, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read batch grid");
    int64_t n = 0;
    for (uint32_t c = 0; c < rd.L; ++c)
        if (cells[c] >= 0) {
            if (n >= (int64_t)rd.N) return fail(NASCH_EINVAL, "grid holds more than N cars");
            x_host[n] = (int32_t)c;
            v_host[n] = (uint8_t)cells[c];
            ++n;
        }
    return n == (int64_t)rd.N ? NASCH_OK : fail(NASCH_EINVAL, "grid holds %lld cars, expected %u", (long long)n, rd.N);
}

int nasch_batch_read_grid(nasch_batch b, int64_t i, int8_t *cells_host, int64_t cap)
{
    clear_error();
    int st = check_road_index(b, i);
    if (st) return st;
    if ((st = wait_batch(b, -1))) return st;
    const BatchRoadDev &rd = b->roads[(size_t)i];
    if (cap < (int64_t)rd.L || !cells_host) return fail(NASCH_EINVAL, "cap=%lld < L=%u", (long long)cap, rd.L);
    const int par = (int)(b->super[(size_t)i] & 1);
    if (b->layout[(size_t)i] == NASCH_LAYOUT_GRID) {
        cudaError_t e = cudaMemcpy(cells_host, rd.cells[par], (size_t)rd.L, cudaMemcpyDeviceToHost);
        return e == cudaSuccess ? NASCH_OK : cuda_fail(e, "read batch grid");
    }
    std::vector<int32_t> x((size_t)std::max<uint32_t>(rd.N, 1));
    std::vector<uint8_t> v((size_t)std::max<uint32_t>(rd.N, 1));
    if ((st = nasch_batch_read_state(b, i, x.data(), v.data(), (int64_t)x.size()))) return st;
    std::memset(cells_host, 0xFF, (size_t)rd.L);
    for (uint32_t k = 0; k < rd.N; ++k) cells_host[x[k]] = (int8_t)v[k];
    return NASCH_OK;
}

int nasch_batch_stats(nasch_batch b, int64_t i, uint64_t first_step, int64_t count, uint64_t *sum_v_host,
                      uint64_t *crossings_host)
{
    clear_error();
    int st = check_road_index(b, i);
    if (st) return st;
    if ((st = wait_batch(b, -1))) return st;
    const BatchRoadDev &rd = b->roads[(size_t)i];
    if (count < 0 || first_step + (uint64_t)count > rd.T)
        return fail(NASCH_EINVAL, "steps [%llu, %llu) outside [0, %u)", (unsigned long long)first_step,
                    (unsigned long long)(first_step + (uint64_t)count), rd.T);
    cudaError_t e = cudaSuccess;
    if (count && sum_v_host) e = cudaMemcpy(sum_v_host, rd.sum_v + first_step, (size_t)count * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && count && crossings_host)
        e = cudaMemcpy(crossings_host, rd.crossings + first_step, (size_t)count * 8, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? NASCH_OK : cuda_fail(e, "read batch statistics");
}

int nasch_batch_stats_sum(nasch_batch b, int64_t i, uint64_t first_step, int64_t count, uint64_t *sum_v_total,
                          uint64_t *crossings_total)
{
    clear_error();
    std::vector<uint64_t> sv((size_t)std::max<int64_t>(count, 1)), cr((size_t)std::max<int64_t>(count, 1));
    int st = nasch_batch_stats(b, i, first_step, count, sv.data(), cr.data());
    if (st) return st;
    uint64_t a = 0, c = 0;
    for (int64_t k = 0; k < count; ++k) {
        a += sv[(size_t)k];
        c += cr[(size_t)k];
    }
    if (sum_v_total) *sum_v_total = a;
    if (crossings_total) *crossings_total = c;
    return NASCH_OK;
}

int nasch_batch_get_info(nasch_batch b, nasch_batch_info *info)
{
    clear_error();
    if (!b || !info) return fail(NASCH_EINVAL, "NULL argument");
    info->n_roads = b->n;
    info->super_steps = b->n_super;
    info->items = b->first_items;
    info->device_bytes = (int64_t)b->pool_bytes;
    info->vehicle_steps = b->vehicle_steps;
    info->cell_steps = b->cell_steps;
    info->blocks = b->blocks;
    info->graphs = (int32_t)b->execs.size();
    info->run_seconds = 0.0;
    if (b->finished || cudaEventQuery(b->done) == cudaSuccess) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, b->started, b->done) == cudaSuccess) info->run_seconds = ms * 1e-3;
    }
    return NASCH_OK;
}

int nasch_batch_road_layout(nasch_batch b, int64_t i, int32_t *layout)
{
    clear_error();
    int st = check_road_index(b, i);
    if (st) return st;
    if (!layout) return fail(NASCH_EINVAL, "layout is NULL");
    *layout = b->layout[(size_t)i];
    return NASCH_OK;
}

void nasch_batch_destroy(nasch_batch b)
{
    if (!b) return;
    if (b->done) cudaEventSynchronize(b->done);
    free_batch(b);
}

}  // extern "C"
