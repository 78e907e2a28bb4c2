// C-ABI runtime of the NaSch library: road handles, argument validation,
// device memory, the per-step statistics series, launch planning (layout,
// fusion depth, whole-ring vs tiled kernel) and the host-side Floyd
// initialisation.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "nasch.h"
#include "kernels.h"
#include "road_output.h"
#include "runtime_internal.h"
#include "state_check.h"

namespace nasch {

static thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(NASCH_ECUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

void clear_error() { g_last_error.clear(); }

uint64_t slow_threshold(double p)
{
    // r = u * 2^-32 < p  <=>  u < ceil(p * 2^32); the scaling by 2^32 is exact.
    if (!(p > 0.0)) return 0;
    if (p >= 1.0) return 1ull << 32;
    return (uint64_t)std::ceil(std::ldexp(p, 32));
}

int validate_params(const nasch_params *prm)
{
    if (!prm) return fail(NASCH_EINVAL, "params is NULL");
    if (prm->L < 1 || prm->L > (int64_t(1) << 31))
        return fail(NASCH_EINVAL, "L=%lld outside 1..2^31", (long long)prm->L);
    if (prm->N < 0 || prm->N > prm->L)
        return fail(NASCH_EINVAL, "N=%lld outside 0..L=%lld", (long long)prm->N, (long long)prm->L);
    if (prm->vmax < 0 || prm->vmax > 127) return fail(NASCH_EINVAL, "vmax=%d outside 0..127", prm->vmax);
    if (!(prm->p >= 0.0 && prm->p <= 1.0)) return fail(NASCH_EINVAL, "p=%g outside [0, 1]", prm->p);
    if (prm->layout < NASCH_LAYOUT_AUTO || prm->layout > NASCH_LAYOUT_GRID)
        return fail(NASCH_EINVAL, "layout=%d unknown", prm->layout);
    if (prm->k < 0 || prm->k > kMaxFusedSteps)
        return fail(NASCH_EINVAL, "k=%d outside 0..%d", prm->k, kMaxFusedSteps);
    if (prm->tile != 0 && prm->tile != kAgentTileSpan && prm->tile != kAgentTileSpanSmall &&
        prm->tile != kGridTileCells)
        return fail(NASCH_EINVAL, "tile=%d not supported (0, %d, %d or %d)", prm->tile, kAgentTileSpanSmall,
                    kAgentTileSpan, kGridTileCells);
    return NASCH_OK;
}

// Floyd's sampling algorithm (Bentley & Floyd, CACM 1987): for m = 0..N-1
// with j = L-N+m, draw t uniform on 0..j (Lemire's multiply-shift of the
// 64-bit Philox word pair of counter (m, 0, road, 1)) and take t, or j if t
// is already taken.  A bitmap over the ring holds the set, so a scan of it
// yields the positions sorted.
int floyd_init_host(int64_t L, int64_t N, uint64_t seed, uint32_t road, int32_t *x)
{
    if (L < 1 || L > (int64_t(1) << 31) || N < 0 || N > L) return fail(NASCH_EINVAL, "floyd: bad L/N");
    if (N == 0) return NASCH_OK;
    std::vector<uint64_t> taken;
    try {
        taken.assign((size_t)((L + 63) / 64), 0ull);
    } catch (const std::bad_alloc &) {
        return fail(NASCH_ENOMEM, "floyd: host bitmap of %lld bits", (long long)L);
    }
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    // The draws do not depend on the set, so they are made a batch ahead and
    // the bitmap words they will test are prefetched (the bitmap is far
    // larger than the caches for long roads); the set updates stay in order.
    constexpr int kBatch = 64;
    uint64_t draws[kBatch];
    for (int64_t m0 = 0; m0 < N; m0 += kBatch) {
        const int nb = (int)std::min<int64_t>(kBatch, N - m0);
        for (int b = 0; b < nb; ++b) {
            const int64_t m = m0 + b;
            const uint64_t j = (uint64_t)(L - N + m);
            const Words4 w = philox4x32_10((uint32_t)m, 0u, road, kTagInit, k0, k1);
            const uint64_t r = ((uint64_t)w.w1 << 32) | w.w0;
            draws[b] = (uint64_t)(((unsigned __int128)r * (j + 1)) >> 64);
            __builtin_prefetch(&taken[draws[b] >> 6], 1);
        }
        for (int b = 0; b < nb; ++b) {
            const uint64_t j = (uint64_t)(L - N + m0 + b);
            const uint64_t t = draws[b];
            const uint64_t pick = (taken[t >> 6] >> (t & 63)) & 1ull ? j : t;
            taken[pick >> 6] |= 1ull << (pick & 63);
        }
    }
    int64_t n = 0;
    for (size_t wi = 0; wi < taken.size(); ++wi) {
        uint64_t word = taken[wi];
        while (word) {
            const int b = __builtin_ctzll(word);
            word &= word - 1;
            x[n++] = (int32_t)(wi * 64 + (size_t)b);
        }
    }
    return n == N ? NASCH_OK : fail(NASCH_EINVAL, "floyd: internal count mismatch");
}

int device_info(int *device, int *sms)
{
    cudaError_t e = cudaGetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    e = cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, *device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute(SM count)");
    return NASCH_OK;
}

}  // namespace nasch

using namespace nasch;

struct nasch_road {
    int64_t L = 0, N = 0;
    int vmax = 0;
    double p = 0;
    uint64_t thr = 0, seed = 0;
    uint32_t road = 0;
    int layout = NASCH_LAYOUT_AGENT;
    int k = 1;
    int device = 0, sms = 1;
    bool ring = false;
    int blocks = 1;
    int tile = 0;                       // agent warp-tile span or grid tile cells
    unsigned int *d_status = nullptr;   // kernels set bits here when a bounded wait runs out
    unsigned long long *d_check = nullptr;   // nasch_set_state's device checks (3 words), made on first use
    uint8_t *d_list = nullptr;          // the fused grid kernel's car lists of dense spans (GridStep::list_scratch)
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int32_t *x[2] = {nullptr, nullptr};
    uint8_t *v[2] = {nullptr, nullptr};
    int8_t *cells[2] = {nullptr, nullptr};
    int cur = 0;
    uint64_t step = 0;
    uint64_t stats_first = 0;
    unsigned long long *d_sum = nullptr, *d_cross = nullptr;
    int64_t stats_cap = 0;
    // slots [stats_dirty, stats_cap) of both series are zero; lower ones may
    // hold the statistics of steps before a reset of stats_first
    int64_t stats_dirty = 0;
    // open road (nasch_create_open): grid layout, one step per launch
    bool open = false;
    uint64_t thr_entry = 0, thr_exit = 0;
    // output (nasch_run_output), made on first use: two staging copies of
    // the cells, a copy stream and the events that order them
    int8_t *stage[2] = {nullptr, nullptr};
    cudaStream_t io_stream = nullptr;
    cudaEvent_t ev_ready[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
};

namespace {

// Wait for the handle's stream, then report a kernel that gave up a bounded
// wait (the status word is cleared for the next launch).
int sync_and_check(nasch_road *h)
{
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    unsigned int status = 0;
    e = cudaMemcpy(&status, h->d_status, sizeof(status), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read status word");
    if (status) {
        cudaMemset(h->d_status, 0, sizeof(status));
        return fail(NASCH_ETIMEOUT, "a kernel's bounded wait on an asynchronous copy ran out (status 0x%x); "
                    "the state of this road is undefined", status);
    }
    return NASCH_OK;
}

RoadConst road_const(const nasch_road *h)
{
    RoadConst rc;
    rc.L = (uint32_t)h->L;
    rc.vmax = (uint32_t)h->vmax;
    rc.thr = h->thr;
    rc.key0 = (uint32_t)h->seed;
    rc.key1 = (uint32_t)(h->seed >> 32);
    rc.road = h->road;
    return rc;
}

void free_road(nasch_road *h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (int i = 0; i < 2; ++i) {
        cudaFree(h->x[i]);
        cudaFree(h->v[i]);
        cudaFree(h->cells[i]);
    }
    cudaFree(h->d_sum);
    cudaFree(h->d_cross);
    cudaFree(h->d_status);
    cudaFree(h->d_check);
    cudaFree(h->d_list);
    if (h->io_stream) cudaStreamSynchronize(h->io_stream);
    for (int i = 0; i < 2; ++i) {
        cudaFree(h->stage[i]);
        if (h->ev_ready[i]) cudaEventDestroy(h->ev_ready[i]);
        if (h->ev_free[i]) cudaEventDestroy(h->ev_free[i]);
    }
    if (h->io_stream) cudaStreamDestroy(h->io_stream);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

// Grow the device statistics series so that steps [stats_first, upto) fit.
int ensure_stats(nasch_road *h, int64_t needed)
{
    if (needed <= h->stats_cap) return NASCH_OK;
    int64_t cap = std::max<int64_t>(needed, std::max<int64_t>(1024, 2 * h->stats_cap));
    unsigned long long *ns = nullptr, *nc = nullptr;
    cudaError_t e = cudaMalloc(&ns, (size_t)cap * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&nc, (size_t)cap * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(ns, 0, (size_t)cap * sizeof(unsigned long long), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(nc, 0, (size_t)cap * sizeof(unsigned long long), h->stream);
    if (e != cudaSuccess) {
        cudaFree(ns);
        cudaFree(nc);
        return cuda_fail(e, "cudaMalloc(statistics)");
    }
    const int64_t used = (int64_t)(h->step - h->stats_first);
    if (used > 0 && h->d_sum) {
        e = cudaMemcpyAsync(ns, h->d_sum, (size_t)used * 8, cudaMemcpyDeviceToDevice, h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(nc, h->d_cross, (size_t)used * 8, cudaMemcpyDeviceToDevice, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) {
            cudaFree(ns);
            cudaFree(nc);
            return cuda_fail(e, "copy statistics");
        }
    }
    cudaFree(h->d_sum);
    cudaFree(h->d_cross);
    h->d_sum = ns;
    h->d_cross = nc;
    h->stats_cap = cap;
    h->stats_dirty = std::max<int64_t>(used, 0);
    return NASCH_OK;
}

// Upload agent state (host arrays) into the handle's current buffers.
int upload_state(nasch_road *h, const int32_t *x, const uint8_t *v)
{
    const int64_t N = h->N;
    cudaError_t e = cudaSuccess;
    if (h->layout == NASCH_LAYOUT_AGENT) {
        if (N > 0) {
            e = cudaMemcpyAsync(h->x[h->cur], x, (size_t)N * 4, cudaMemcpyHostToDevice, h->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(h->v[h->cur], v, (size_t)N, cudaMemcpyHostToDevice, h->stream);
        }
    } else {
        int32_t *dx = nullptr;
        uint8_t *dv = nullptr;
        e = cudaMemsetAsync(h->cells[h->cur], 0xFF, (size_t)h->L, h->stream);
        if (e == cudaSuccess && N > 0) {
            e = cudaMallocAsync(&dx, (size_t)N * 4, h->stream);
            if (e == cudaSuccess) e = cudaMallocAsync(&dv, (size_t)N, h->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(dx, x, (size_t)N * 4, cudaMemcpyHostToDevice, h->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(dv, v, (size_t)N, cudaMemcpyHostToDevice, h->stream);
            if (e == cudaSuccess) e = launch_scatter_agent_to_grid(dx, dv, (uint32_t)N, h->cells[h->cur], h->stream);
            if (dx) cudaFreeAsync(dx, h->stream);
            if (dv) cudaFreeAsync(dv, h->stream);
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "upload state");
    return NASCH_OK;
}

// The message for car i, which the device check found bad (a cell outside
// the road, a velocity above vmax, or the next car's cell, in that order).
int bad_car(int64_t L, int64_t N, int vmax, const int32_t *x, const uint8_t *v, int64_t i)
{
    if (x[i] < 0 || x[i] >= L) return fail(NASCH_EINVAL, "x[%lld]=%d outside [0, L)", (long long)i, x[i]);
    if (v[i] > vmax) return fail(NASCH_EINVAL, "v[%lld]=%d above vmax=%d", (long long)i, v[i], vmax);
    (void)N;
    return fail(NASCH_EINVAL, "two cars on cell %d", x[i]);
}

// nasch_set_state's upload: the state goes into the buffers the next launch
// would write, is checked there on the device, and becomes the road's state
// only if it is valid, so a rejected state leaves the road as it was.
// Agent roads: positions inside the road, velocities up to vmax, no car on
// the next car's cell, and one descent round the ring (cyclic order).  Grid
// roads: the same per car, then the cars are scattered and the occupied
// cells counted (a shared cell leaves fewer than N).  The caller has
// synchronised the stream.
int upload_checked(nasch_road *h, int64_t N, const int32_t *x, const uint8_t *v)
{
    const int nxt = h->cur ^ 1;
    cudaError_t e = cudaSuccess;
    if (!h->d_check) e = cudaMalloc(&h->d_check, 3 * sizeof(unsigned long long));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(check words)");
    unsigned long long res[3] = {~0ull, 0ull, 0ull};   // first bad car, descents, occupied cells
    e = cudaMemcpyAsync(h->d_check, res, sizeof(res), cudaMemcpyHostToDevice, h->stream);
    int32_t *dx = nullptr;
    uint8_t *dv = nullptr;
    if (h->layout == NASCH_LAYOUT_AGENT) {
        dx = h->x[nxt];
        dv = h->v[nxt];
    } else if (N > 0) {
        if (e == cudaSuccess) e = cudaMallocAsync(&dx, (size_t)N * 4, h->stream);
        if (e == cudaSuccess) e = cudaMallocAsync(&dv, (size_t)N, h->stream);
    }
    if (e == cudaSuccess && N > 0) e = cudaMemcpyAsync(dx, x, (size_t)N * 4, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && N > 0) e = cudaMemcpyAsync(dv, v, (size_t)N, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = launch_check_cars(dx, dv, (uint32_t)N, (uint32_t)h->L, (uint32_t)h->vmax, h->d_check, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(res, h->d_check, sizeof(res), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    int st = NASCH_OK;
    if (e != cudaSuccess) {
        st = cuda_fail(e, "upload and check state");
    } else if (res[0] < (unsigned long long)N) {
        st = bad_car(h->L, N, h->vmax, x, v, (int64_t)res[0]);
    } else if (h->layout == NASCH_LAYOUT_AGENT) {
        if (N >= 2 && res[1] != 1)
            st = fail(NASCH_EINVAL, "positions are not in cyclic order (%llu descents)", res[1]);
    } else {
        // every car is on the road: scatter them and count the occupied cells
        e = cudaMemsetAsync(h->cells[nxt], 0xFF, (size_t)h->L, h->stream);
        if (e == cudaSuccess) e = launch_scatter_agent_to_grid(dx, dv, (uint32_t)N, h->cells[nxt], h->stream);
        if (e == cudaSuccess) e = launch_count_cars(h->cells[nxt], (uint32_t)h->L, h->d_check + 2, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&res[2], h->d_check + 2, 8, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) {
            st = cuda_fail(e, "scatter and count state");
        } else if (res[2] != (unsigned long long)N) {   // a shared cell: name it
            std::vector<int32_t> sorted(x, x + N);
            std::sort(sorted.begin(), sorted.end());
            int32_t cell = sorted[0];
            for (int64_t i = 1; i < N; ++i)
                if (sorted[i] == sorted[i - 1]) {
                    cell = sorted[i];
                    break;
                }
            st = fail(NASCH_EINVAL, "two cars on cell %d", cell);
        }
    }
    if (h->layout != NASCH_LAYOUT_AGENT) {
        if (dx) cudaFreeAsync(dx, h->stream);
        if (dv) cudaFreeAsync(dv, h->stream);
        if (st == NASCH_OK) {
            e = cudaStreamSynchronize(h->stream);
            if (e != cudaSuccess) st = cuda_fail(e, "upload state");
        }
    }
    if (st == NASCH_OK) h->cur = nxt;
    return st;
}

#ifdef NASCH_DEBUG
// Debug builds, after every nasch_run: wait for the steps, read the kernels'
// debug words, and check the state now current on the device (agent roads:
// every car inside the road, no faster than vmax, not on the next car's
// cell, one descent round the ring; closed grid roads: N occupied cells).
int debug_after_run(nasch_road *h)
{
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "debug: steps");
    const unsigned int w = debug_word_agent() | debug_word_grid() | debug_word_open();
    if (w) return fail(NASCH_EINVAL, "debug check failed before step %llu (sites 0x%x)", (unsigned long long)h->step, w);
    if (h->N == 0) return NASCH_OK;
    if (!h->d_check) e = cudaMalloc(&h->d_check, 3 * sizeof(unsigned long long));
    unsigned long long res[3] = {~0ull, 0ull, 0ull};
    if (e == cudaSuccess) e = cudaMemcpy(h->d_check, res, sizeof(res), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        if (h->layout == NASCH_LAYOUT_AGENT)
            e = launch_check_cars(h->x[h->cur], h->v[h->cur], (uint32_t)h->N, (uint32_t)h->L, (uint32_t)h->vmax,
                                  h->d_check, h->stream);
        else if (!h->open)
            e = launch_count_cars(h->cells[h->cur], (uint32_t)h->L, h->d_check + 2, h->stream);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(res, h->d_check, sizeof(res), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "debug: state check");
    if (h->layout == NASCH_LAYOUT_AGENT) {
        if (res[0] < (unsigned long long)h->N)
            return fail(NASCH_EINVAL, "debug: car %llu breaks a rule before step %llu", res[0],
                        (unsigned long long)h->step);
        if (h->N >= 2 && res[1] != 1)
            return fail(NASCH_EINVAL, "debug: cyclic order lost before step %llu (%llu descents)",
                        (unsigned long long)h->step, res[1]);
    } else if (!h->open && res[2] != (unsigned long long)h->N) {
        return fail(NASCH_EINVAL, "debug: %llu occupied cells for %lld cars before step %llu", res[2],
                    (long long)h->N, (unsigned long long)h->step);
    }
    return NASCH_OK;
}
#endif

int choose_layout(const nasch_params *prm)
{
    if (prm->layout != NASCH_LAYOUT_AUTO) return prm->layout;
    // the agent layout below the tuned density (see auto_rho_star)
    return (double)prm->N < auto_rho_star(prm, 1) * (double)prm->L ? NASCH_LAYOUT_AGENT : NASCH_LAYOUT_GRID;
}

// Enqueue `steps` steps on the handle's stream (validated by the caller).
int run_steps(nasch_road *h, int64_t steps)
{
    if (steps == 0) return NASCH_OK;
    const int64_t used = (int64_t)(h->step - h->stats_first);
    int st = ensure_stats(h, used + steps);
    if (st) return st;
    unsigned long long *sum = h->d_sum + used;
    unsigned long long *cross = h->d_cross + used;
    cudaError_t e = cudaSuccess;
    if (used < h->stats_dirty) {   // slots written before a reset of stats_first: clear them
        const size_t n = (size_t)(std::min<int64_t>(h->stats_dirty, used + steps) - used) * 8;
        e = cudaMemsetAsync(sum, 0, n, h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(cross, 0, n, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(statistics)");
    }
    h->stats_dirty = std::max<int64_t>(h->stats_dirty, used + steps);
    const RoadConst rc = road_const(h);

    if (h->layout == NASCH_LAYOUT_AGENT) {
        AgentStep a;
        a.status = h->d_status;
        a.N = (uint32_t)h->N;
        a.rc = rc;
        if (h->N == 0) {
            h->step += (uint64_t)steps;
            return NASCH_OK;
        }
        if (h->ring) {
            // the whole run in launches of up to 2^20 steps
            for (int64_t done = 0; done < steps;) {
                const int64_t kk = std::min<int64_t>(steps - done, 1 << 20);
                a.x_in = h->x[h->cur];
                a.v_in = h->v[h->cur];
                a.x_out = h->x[h->cur ^ 1];
                a.v_out = h->v[h->cur ^ 1];
                a.step0 = (uint32_t)(h->step + (uint64_t)done);
                a.ksteps = (int)kk;
                a.sum_v = sum + done;
                a.crossings = cross + done;
                e = launch_agent_ring(a, h->stream);
                if (e != cudaSuccess) return cuda_fail(e, "agent ring kernel");
                h->cur ^= 1;
                done += kk;
            }
        } else {
            for (int64_t done = 0; done < steps;) {
                const int kk = (int)std::min<int64_t>(steps - done, h->k);
                a.x_in = h->x[h->cur];
                a.v_in = h->v[h->cur];
                a.x_out = h->x[h->cur ^ 1];
                a.v_out = h->v[h->cur ^ 1];
                a.step0 = (uint32_t)(h->step + (uint64_t)done);
                a.ksteps = kk;
                a.sum_v = sum + done;
                a.crossings = cross + done;
                e = launch_agent_tiled(a, h->tile, h->sms, h->stream);
                if (e != cudaSuccess) return cuda_fail(e, "agent tiled kernel");
                h->cur ^= 1;
                done += kk;
            }
        }
    } else if (h->open) {
        GridStep g;
        g.status = h->d_status;
        g.rc = rc;
        for (int64_t done = 0; done < steps; ++done) {
            const uint32_t step = (uint32_t)(h->step + (uint64_t)done);
            const uint32_t k0 = (uint32_t)h->seed, k1 = (uint32_t)(h->seed >> 32);
            // the step's exit and entry draws (counter words 3: tags 2 and 3)
            const bool exit_open = (uint64_t)philox4x32_10(0u, step, h->road, 2u, k0, k1).w0 < h->thr_exit;
            const bool entry = (uint64_t)philox4x32_10(0u, step, h->road, 3u, k0, k1).w0 < h->thr_entry;
            g.c_in = h->cells[h->cur];
            g.c_out = h->cells[h->cur ^ 1];
            g.step0 = step;
            g.ksteps = 1;
            g.sum_v = sum + done;
            g.crossings = cross + done;
            e = launch_grid_open(g, exit_open, entry, h->stream);
            if (e != cudaSuccess) return cuda_fail(e, "open road kernel");
            h->cur ^= 1;
        }
    } else {
        GridStep g;
        g.status = h->d_status;
        g.rc = rc;
        g.list_scratch = h->d_list;
        for (int64_t done = 0; done < steps;) {
            const int kk = h->ring ? (int)std::min<int64_t>(steps - done, 1 << 20)
                                   : (int)std::min<int64_t>(steps - done, h->k);
            g.c_in = h->cells[h->cur];
            g.c_out = h->cells[h->cur ^ 1];
            g.step0 = (uint32_t)(h->step + (uint64_t)done);
            g.ksteps = kk;
            g.sum_v = sum + done;
            g.crossings = cross + done;
            e = h->ring ? launch_grid_ring(g, h->stream) : launch_grid_tiled(g, h->blocks, h->stream);
            if (e != cudaSuccess) return cuda_fail(e, h->ring ? "grid ring kernel" : "grid tiled kernel");
            h->cur ^= 1;
            done += kk;
        }
    }
    h->step += (uint64_t)steps;
    return NASCH_OK;
}

int create_road(const nasch_params *prm, bool open, uint64_t thr_entry, uint64_t thr_exit, nasch_handle *out)
{
    if (!out) return fail(NASCH_EINVAL, "out is NULL");
    *out = nullptr;
    int st = validate_params(prm);
    if (st) return st;
    nasch_road *h = new (std::nothrow) nasch_road();
    if (!h) return fail(NASCH_ENOMEM, "host allocation");
    h->L = prm->L;
    h->N = prm->N;
    h->vmax = prm->vmax;
    h->p = prm->p;
    h->thr = slow_threshold(prm->p);
    h->seed = prm->seed;
    h->road = prm->road_id;
    h->layout = choose_layout(prm);
    h->open = open;
    h->thr_entry = thr_entry;
    h->thr_exit = thr_exit;
    st = device_info(&h->device, &h->sms);
    if (st) {
        delete h;
        return st;
    }
    cudaError_t e;
    if (prm->stream) {
        h->stream = (cudaStream_t)prm->stream;
    } else {
        e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete h;
            return cuda_fail(e, "cudaStreamCreate");
        }
        h->own_stream = true;
    }
    // tile == 0: the whole-ring kernel when the ring fits one block; an
    // explicit tile always selects the tiled kernel.
    if (h->layout == NASCH_LAYOUT_AGENT) {
        if (prm->tile != 0 && prm->tile != kAgentTileSpan && prm->tile != kAgentTileSpanSmall) {
            free_road(h);
            return fail(NASCH_EINVAL, "agent tile must be %d or %d", kAgentTileSpanSmall, kAgentTileSpan);
        }
        h->ring = prm->tile == 0 && h->N <= kAgentRingMaxCars;
        h->tile = prm->tile ? prm->tile : kAgentTileSpan;
        h->k = prm->k ? prm->k : 16;   // fastest on the large road (the Philox multiplies bound every k >= 8)
        h->blocks = h->sms * agent_tiled_blocks_per_sm(h->k);
        const size_t n = (size_t)std::max<int64_t>(h->N, 1);
        e = cudaSuccess;
        for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
            e = cudaMalloc(&h->x[i], n * 4);
            if (e == cudaSuccess) e = cudaMalloc(&h->v[i], n);
        }
    } else {
        if (prm->tile != 0 && prm->tile != kGridTileCells) {
            free_road(h);
            return fail(NASCH_EINVAL, "grid tile must be %d", kGridTileCells);
        }
        h->ring = !open && prm->tile == 0 && h->L <= kGridRingMaxCells;
        h->tile = kGridTileCells;
        h->k = open ? 1 : (prm->k ? prm->k : 8);
        // the halo round_up(k * vmax, 16) on each side must leave the tile cells
        // of its own: clamp k so that 2 * halo < the staged span
        const int kfit = h->vmax > 0 ? std::max(1, ((kGridSpan / 2 - 16) / h->vmax)) : kMaxFusedSteps;
        h->k = std::min(h->k, kfit);
        if (!open && !h->ring && h->L < (int64_t)kGridSpan) {
            free_road(h);
            return fail(NASCH_EINVAL, "L=%lld too short for the tiled grid kernel (needs L >= %d)",
                        (long long)h->L, kGridSpan);
        }
        h->blocks = h->sms * grid_tiled_blocks_per_sm();
        e = cudaSuccess;
        for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaMalloc(&h->cells[i], (size_t)h->L + 16);
        // the fused warp kernel keeps the lists of dense spans here; any
        // launch of fewer than the road's k steps may take it (a halo of k
        // steps above kKwMaxHalo shrinks for a shorter last launch), so every
        // road that is not stepped one step at a time by the one-step kernel
        // gets it
        if (e == cudaSuccess && !open && !h->ring && (h->k >= 2 || h->vmax > 16)) {
            const size_t bytes = grid_list_scratch_bytes();
            e = bytes ? cudaMalloc(&h->d_list, bytes) : cudaErrorInvalidValue;
        }
    }
    if (e == cudaSuccess) e = cudaMalloc(&h->d_status, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(h->d_status, 0, sizeof(unsigned int));
    if (e != cudaSuccess) {
        free_road(h);
        return e == cudaErrorMemoryAllocation ? fail(NASCH_ENOMEM, "device state: %s", cudaGetErrorString(e))
                                              : cuda_fail(e, "cudaMalloc(state)");
    }
    // Floyd start, v = 0, step 0
    std::vector<int32_t> x;
    std::vector<uint8_t> v;
    try {
        x.resize((size_t)h->N);
        v.assign((size_t)h->N, 0);
    } catch (const std::bad_alloc &) {
        free_road(h);
        return fail(NASCH_ENOMEM, "host staging");
    }
    st = floyd_init_host(h->L, h->N, h->seed, h->road, x.data());
    if (!st) st = upload_state(h, x.data(), v.data());
    if (!st) st = ensure_stats(h, 1024);
    if (st) {
        free_road(h);
        return st;
    }
    *out = h;
    return NASCH_OK;
}

}  // namespace

extern "C" {

void nasch_params_init(nasch_params *prm)
{
    if (!prm) return;
    std::memset(prm, 0, sizeof(*prm));
    prm->vmax = 5;
    prm->layout = NASCH_LAYOUT_AUTO;
}

const char *nasch_last_error(void) { return g_last_error.c_str(); }

uint64_t nasch_slow_threshold(double p) { return slow_threshold(p); }

int nasch_floyd_init(int64_t L, int64_t N, uint64_t seed, uint32_t road_id, int32_t *x_host)
{
    clear_error();
    if (!x_host && N > 0) return fail(NASCH_EINVAL, "x_host is NULL");
    return floyd_init_host(L, N, seed, road_id, x_host);
}

int nasch_create_ex(const nasch_params *prm, nasch_handle *out)
{
    clear_error();
    TraceRange trace("nasch_create");
    return create_road(prm, false, 0, 0, out);
}

int nasch_create_open(const nasch_params *prm, double alpha, double beta, nasch_handle *out)
{
    clear_error();
    TraceRange trace("nasch_create_open");
    if (!prm) return fail(NASCH_EINVAL, "params is NULL");
    if (!(alpha >= 0.0 && alpha <= 1.0) || !(beta >= 0.0 && beta <= 1.0))
        return fail(NASCH_EINVAL, "alpha=%g and beta=%g must lie in [0, 1]", alpha, beta);
    if (prm->layout == NASCH_LAYOUT_AGENT) return fail(NASCH_EINVAL, "an open road uses the grid layout");
    nasch_params q = *prm;
    q.layout = NASCH_LAYOUT_GRID;
    q.k = 1;
    q.tile = 0;
    return create_road(&q, true, slow_threshold(alpha), slow_threshold(beta), out);
}

int nasch_create(int64_t L, int64_t N, int vmax, double p, uint64_t seed, nasch_handle *out)
{
    nasch_params prm;
    nasch_params_init(&prm);
    prm.L = L;
    prm.N = N;
    prm.vmax = vmax;
    prm.p = p;
    prm.seed = seed;
    return nasch_create_ex(&prm, out);
}

int nasch_set_state(nasch_handle h, const int32_t *x_host, const uint8_t *v_host, int64_t N, uint64_t step)
{
    clear_error();
    if (!h) return fail(NASCH_EINVAL, "handle is NULL");
    if (h->open ? (N < 0 || N > h->L) : N != h->N)
        return fail(NASCH_EINVAL, "N=%lld: must equal the handle's N=%lld (a ring) or lie in 0..L (an open road)",
                    (long long)N, (long long)h->N);
    if (N > 0 && (!x_host || !v_host)) return fail(NASCH_EINVAL, "NULL state array");
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    const int st = upload_checked(h, N, x_host, v_host);
    if (st) return st;
    h->N = N;
    h->step = step;
    h->stats_first = step;
    return NASCH_OK;
}

int nasch_run(nasch_handle h, int64_t steps)
{
    clear_error();
    TraceRange trace("nasch_run");
    if (!h) return fail(NASCH_EINVAL, "handle is NULL");
    if (steps < 0) return fail(NASCH_EINVAL, "steps=%lld < 0", (long long)steps);
    const int st = run_steps(h, steps);
#ifdef NASCH_DEBUG
    if (st == NASCH_OK) return debug_after_run(h);
#endif
    return st;
}

int nasch_run_output(nasch_handle h, int64_t steps, int64_t per, int8_t *snap_host, int64_t snap_cap,
                     uint8_t *raster_host, int32_t raster_width, int64_t raster_cap)
{
    clear_error();
    TraceRange trace("nasch_run_output");
    if (!h) return fail(NASCH_EINVAL, "handle is NULL");
    if (steps < 0 || per < 0) return fail(NASCH_EINVAL, "steps=%lld, per=%lld: negative", (long long)steps, (long long)per);
    const bool snap = snap_host != nullptr, raster = raster_host != nullptr;
    if (snap && snap_cap < 1) return fail(NASCH_EINVAL, "snap_cap=%lld < 1", (long long)snap_cap);
    if (raster && (raster_cap < 1 || raster_width < 1 || (int64_t)raster_width > h->L))
        return fail(NASCH_EINVAL, "raster_width=%d outside 1..L=%lld or raster_cap=%lld < 1", raster_width,
                    (long long)h->L, (long long)raster_cap);
    if (per == 0 || (!snap && !raster)) {   // output off
        int st = run_steps(h, steps);
        return st ? st : sync_and_check(h);
    }
    const size_t L = (size_t)h->L;
    cudaError_t e = cudaSuccess;
    // staging: snapshots leave from a copy of the cells, so the copy to the
    // host overlaps the next steps; an agent road is scattered into one
    const bool staged = snap || h->layout == NASCH_LAYOUT_AGENT;
    for (int i = 0; i < 2 && staged && e == cudaSuccess; ++i) {
        if (!h->stage[i]) e = cudaMalloc(&h->stage[i], L);
        if (e == cudaSuccess && !h->ev_ready[i]) e = cudaEventCreateWithFlags(&h->ev_ready[i], cudaEventDisableTiming);
        if (e == cudaSuccess && !h->ev_free[i]) e = cudaEventCreateWithFlags(&h->ev_free[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess && snap && !h->io_stream) e = cudaStreamCreateWithFlags(&h->io_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "output buffers");
    uint8_t *d_rows = nullptr;
    const size_t row_bytes = raster ? (size_t)raster_width : 0;
    if (raster) {
        e = cudaMallocAsync(&d_rows, (size_t)raster_cap * row_bytes, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "raster rows");
    }
    int64_t j = 0;   // snapshots taken
    int st = NASCH_OK;
    for (int64_t done = 0; done < steps && st == NASCH_OK;) {
        const int64_t chunk = std::min(per, steps - done);
        st = run_steps(h, chunk);
        if (st) break;
        done += chunk;
        if (chunk < per) break;   // a partial last chunk takes no snapshot
        const int b = (int)(j & 1);
        const int8_t *src = h->cells[h->cur];
        if (staged) {
            // staging buffer b: its copy to the host two snapshots ago must be done
            if (j >= 2 && snap) e = cudaStreamWaitEvent(h->stream, h->ev_free[b], 0);
            if (e == cudaSuccess) {
                if (h->layout == NASCH_LAYOUT_GRID) {
                    e = cudaMemcpyAsync(h->stage[b], h->cells[h->cur], L, cudaMemcpyDeviceToDevice, h->stream);
                } else {
                    e = cudaMemsetAsync(h->stage[b], 0xFF, L, h->stream);
                    if (e == cudaSuccess && h->N > 0)
                        e = launch_scatter_agent_to_grid(h->x[h->cur], h->v[h->cur], (uint32_t)h->N, h->stage[b],
                                                         h->stream);
                }
            }
            src = h->stage[b];
        }
        if (e == cudaSuccess && raster)
            e = launch_raster_row(src, (uint32_t)h->L, (uint32_t)raster_width,
                                  d_rows + (size_t)(j % raster_cap) * row_bytes, h->sms, h->stream);
        if (e == cudaSuccess && snap) {
            e = cudaEventRecord(h->ev_ready[b], h->stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(h->io_stream, h->ev_ready[b], 0);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(snap_host + (size_t)(j % snap_cap) * L, h->stage[b], L, cudaMemcpyDeviceToHost,
                                    h->io_stream);
            if (e == cudaSuccess) e = cudaEventRecord(h->ev_free[b], h->io_stream);
        }
        if (e != cudaSuccess) st = cuda_fail(e, "snapshot");
        ++j;
    }
    if (st == NASCH_OK && raster && j > 0) {
        const int64_t rows = std::min(j, raster_cap);
        e = cudaMemcpyAsync(raster_host, d_rows, (size_t)rows * row_bytes, cudaMemcpyDeviceToHost, h->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "raster rows to host");
    }
    if (d_rows) cudaFreeAsync(d_rows, h->stream);
    if (h->io_stream) {
        e = cudaStreamSynchronize(h->io_stream);
        if (e != cudaSuccess && st == NASCH_OK) st = cuda_fail(e, "snapshot copies");
    }
    const int st2 = sync_and_check(h);
    return st ? st : st2;
}

int nasch_read_state(nasch_handle h, int32_t *x_host, uint8_t *v_host, int64_t cap)
{
    clear_error();
    if (!h) return fail(NASCH_EINVAL, "handle is NULL");
    if (h->open) return fail(NASCH_EINVAL, "an open road's car count changes: read its cells with nasch_read_grid");
    if (cap < h->N) return fail(NASCH_EINVAL, "cap=%lld < N=%lld", (long long)cap, (long long)h->N);
    if (h->N > 0 && (!x_host || !v_host)) return fail(NASCH_EINVAL, "NULL output array");
    int st = sync_and_check(h);
    if (st) return st;
    cudaError_t e = cudaSuccess;
    if (h->N == 0) return NASCH_OK;
    if (h->layout == NASCH_LAYOUT_AGENT) {
        e = cudaMemcpyAsync(x_host, h->x[h->cur], (size_t)h->N * 4, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(v_host, h->v[h->cur], (size_t)h->N, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "read state");
        return NASCH_OK;
    }
    std::vector<int8_t> cells;
    try {
        cells.resize((size_t)h->L);
    } catch (const std::bad_alloc &) {
        return fail(NASCH_ENOMEM, "host grid staging");
    }
    e = cudaMemcpy(cells.data(), h->cells[h->cur], (size_t)h->L, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read grid");
    int64_t n = 0;
    for (int64_t c = 0; c < h->L; ++c) {
        if (cells[(size_t)c] >= 0) {
            if (n >= h->N) return fail(NASCH_EINVAL, "grid holds more than N cars");
            x_host[n] = (int32_t)c;
            v_host[n] = (uint8_t)cells[(size_t)c];
            ++n;
        }
    }
    if (n != h->N) return fail(NASCH_EINVAL, "grid holds %lld cars, expected %lld", (long long)n, (long long)h->N);
    return NASCH_OK;
}

int nasch_read_grid(nasch_handle h, int8_t *cells_host, int64_t cap)
{
    clear_error();
    if (!h) return fail(NASCH_EINVAL, "handle is NULL");
    if (cap < h->L || !cells_host) return fail(NASCH_EINVAL, "cap=%lld < L=%lld", (long long)cap, (long long)h->L);
    int st = sync_and_check(h);
    if (st) return st;
    cudaError_t e = cudaSuccess;
    if (h->layout == NASCH_LAYOUT_GRID) {
        e = cudaMemcpy(cells_host, h->cells[h->cur], (size_t)h->L, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "read grid");
        return NASCH_OK;
    }
    int8_t *d = nullptr;
    e = cudaMallocAsync(&d, (size_t)h->L, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d, 0xFF, (size_t)h->L, h->stream);
    if (e == cudaSuccess) e = launch_scatter_agent_to_grid(h->x[h->cur], h->v[h->cur], (uint32_t)h->N, d, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cells_host, d, (size_t)h->L, cudaMemcpyDeviceToHost, h->stream);
    if (d) cudaFreeAsync(d, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "agent to grid");
    return NASCH_OK;
}

int nasch_stats(nasch_handle h, uint64_t first_step, int64_t count, uint64_t *sum_v_host, uint64_t *crossings_host)
{
    clear_error();
    if (!h) return fail(NASCH_EINVAL, "handle is NULL");
    if (count < 0 || first_step < h->stats_first || first_step + (uint64_t)count > h->step)
        return fail(NASCH_EINVAL, "steps [%llu, %llu) outside the kept range [%llu, %llu)",
                    (unsigned long long)first_step, (unsigned long long)(first_step + (uint64_t)count),
                    (unsigned long long)h->stats_first, (unsigned long long)h->step);
    if (count == 0) return NASCH_OK;
    const size_t off = (size_t)(first_step - h->stats_first);
    int st = sync_and_check(h);
    if (st) return st;
    cudaError_t e = cudaSuccess;
    if (sum_v_host)
        e = cudaMemcpy(sum_v_host, h->d_sum + off, (size_t)count * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && crossings_host)
        e = cudaMemcpy(crossings_host, h->d_cross + off, (size_t)count * 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read statistics");
    return NASCH_OK;
}

int nasch_get_info(nasch_handle h, nasch_info *info)
{
    clear_error();
    if (!h || !info) return fail(NASCH_EINVAL, "NULL argument");
    info->L = h->L;
    info->N = h->N;
    info->vmax = h->vmax;
    info->layout = h->layout;
    info->k = h->k;
    info->tile = h->tile;
    info->step = h->step;
    info->stats_first = h->stats_first;
    info->threshold = h->thr;
    info->ring_kernel = h->ring ? 1 : 0;
    info->blocks = h->blocks;
    return NASCH_OK;
}

int nasch_synchronize(nasch_handle h)
{
    clear_error();
    if (!h) return fail(NASCH_EINVAL, "handle is NULL");
    return sync_and_check(h);
}

void nasch_destroy(nasch_handle h) { free_road(h); }

int nasch_philox_device(int64_t n, const uint32_t *ctr_host, uint64_t seed, uint32_t *out_host)
{
    clear_error();
    if (n < 0 || (n > 0 && (!ctr_host || !out_host))) return fail(NASCH_EINVAL, "bad arguments");
    if (n == 0) return NASCH_OK;
    uint32_t *dc = nullptr, *dout = nullptr;
    cudaError_t e = cudaMalloc(&dc, (size_t)n * 16);
    if (e == cudaSuccess) e = cudaMalloc(&dout, (size_t)n * 16);
    if (e == cudaSuccess) e = cudaMemcpy(dc, ctr_host, (size_t)n * 16, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_philox_test(dc, (uint32_t)seed, (uint32_t)(seed >> 32), dout, n, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(out_host, dout, (size_t)n * 16, cudaMemcpyDeviceToHost);
    cudaFree(dc);
    cudaFree(dout);
    return e == cudaSuccess ? NASCH_OK : cuda_fail(e, "philox test kernel");
}

}  // extern "C"
