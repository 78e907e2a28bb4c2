// Grid NaSch step kernels: one int8 per cell, -1 empty, else the velocity of
// the car on it ("Concepts Covered": the grid representation; Handout,
// model section rules 1-4).
//
// Tiled kernel.  A tile is kGridTileCells cells staged in shared memory with
// a halo of H = round_up(k * vmax, 16) cells on each side: after one step a
// cell depends on the cells within vmax of it (a car arriving from behind,
// the gap of that car ahead), so after k fused steps the middle tile is
// exact.  Persistent blocks walk the tiles; each tile (with its halos)
// arrives by one bulk (TMA) copy issued while the previous tile computes,
// completion counted on an mbarrier, and leaves by one bulk store.  Per step
// a warp turns 16-cell chunks into occupancy bit masks (one bit per cell),
// finds each car's gap with find-first-set on the mask of the cells ahead,
// compacts the cars into a list so the draws are spread evenly over the
// lanes, applies rules 1-3 and scatters each car into the next buffer,
// which was cleared to -1 one step earlier (rotating buffers, one barrier
// per step).  Rule 2 makes the scatter collision-free.  Statistics of the
// cars that start the step in the tile's own cells are reduced per warp,
// per block, and added to the per-step series once per block.  The first
// and last tiles take their halo across the ring boundary (modular cell
// index, plain loads).
//
// Ring kernel.  For L <= kGridRingMaxCells one block holds the whole ring
// in shared memory and runs any number of steps in one launch.
#include "kernels.h"

namespace nasch {
namespace {

// Occupancy bits of four cells packed in a 32-bit word (bit b = byte b has
// its sign bit clear, i.e. holds a car).
__device__ __forceinline__ uint32_t occupancy4(uint32_t w)
{
    const uint32_t m = (~w >> 7) & 0x01010101u;
    return (m * 0x10204080u) >> 28;
}

__device__ __forceinline__ uint32_t occupancy16(const uint4 q)
{
    return occupancy4(q.x) | (occupancy4(q.y) << 4) | (occupancy4(q.z) << 8) | (occupancy4(q.w) << 12);
}

__device__ __forceinline__ uint32_t byte_of(const uint4 q, uint32_t j)
{
    const uint32_t w = j < 8u ? (j < 4u ? q.x : q.y) : (j < 12u ? q.z : q.w);
    return (w >> (8u * (j & 3u))) & 0xFFu;
}

enum class Draw { kNever, kAlways, kPhilox };

constexpr uint4 kEmpty4 = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu};
constexpr int kGridWarps = kGridThreads / 32;
constexpr uint32_t kRowCells = 32u * 16u;           // cells one warp scans per pass
constexpr uint64_t kWaitLimitNs = 1000000000ull;    // bounded wait on an async copy: 1 s

// ---- PTX wrappers: shared-memory mbarriers and 1-D bulk (TMA) copies ----
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Orders this thread's generic-proxy shared-memory accesses before later
// async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for the phase of `bar` with the given parity, for at most 1 s.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > kWaitLimitNs) return false;
    return true;
}

// global -> shared, completion counted in bytes on `bar`
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// shared -> global, tracked by bulk groups
__device__ __forceinline__ void bulk_store(void *dst, const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

struct GridTileGeom {
    uint32_t halo;      // H, multiple of 16
    uint32_t width;     // W = tile + 2H cells processed per step
    uint32_t padded;    // W + pad: buffer length (multiple of 16)
    uint32_t n_tiles;
    uint32_t lookahead; // chunks read beyond a car's own chunk for its gap
    uint32_t nwork;     // rotating output buffers: 2 for k = 1, else 3
};

// One synchronous step over a staged buffer: read `cur`, scatter every car
// into `nxt` (already all -1), and clear `clr` for the step after.  Each warp
// scans rows of 512 cells; the cars of a row are compacted into the warp's
// list (cell index, gap, velocity) so that every lane then applies rules 1-4
// to the same number of cars (a lane's own cells hold 0..16 cars, which would
// leave most lanes idle through the draws).
template <Draw D>
__device__ __forceinline__ void grid_step(const RoadConst &rc, const int8_t *__restrict__ cur, int8_t *nxt,
                                          int8_t *clr, const GridTileGeom &geo, uint32_t own_cells, uint32_t base,
                                          uint32_t step, uint32_t *list, uint32_t &tsum, uint32_t &tcross)
{
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t chunks = geo.width / 16u;
    const uint32_t H = geo.halo;
    const uint32_t L = rc.L;
    const uint4 *cur4 = reinterpret_cast<const uint4 *>(cur);
    uint4 *clr4 = reinterpret_cast<uint4 *>(clr);
    for (uint32_t c = threadIdx.x; c < geo.padded / 16u; c += kGridThreads) clr4[c] = kEmpty4;

    for (uint32_t row = warp; row * 32u < chunks; row += kGridWarps) {
        const uint32_t c = row * 32u + lane;
        const uint4 q = c < chunks ? cur4[c] : kEmpty4;
        uint32_t m = occupancy16(q);
        uint32_t m_next = __shfl_down_sync(0xFFFFFFFFu, m, 1);
        if (lane == 31 && c < chunks) m_next = occupancy16(cur4[c + 1]);
        const uint32_t n = __popc(m);
        uint32_t incl = n;
#pragma unroll
        for (uint32_t d = 1; d < 32; d <<= 1) {
            const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
            if (lane >= d) incl += t;
        }
        const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
        if (total == 0) continue;
        uint32_t pos = incl - n;
        const uint32_t window = m | (m_next << 16);
        while (m) {
            const uint32_t j = (uint32_t)(__ffs(m) - 1);
            m &= m - 1u;
            const uint32_t after = window >> (j + 1u);
            uint32_t gap = after ? (uint32_t)(__ffs(after) - 1) : 31u - j;
            if (after == 0u && gap < rc.vmax) {
                // vmax > 16: keep scanning whole chunks ahead
                uint32_t cc = c + 2u;
                for (uint32_t k = 1; k < geo.lookahead && gap < rc.vmax; ++k, ++cc) {
                    const uint32_t m2 = occupancy16(cur4[cc]);
                    if (m2) {
                        gap += (uint32_t)(__ffs(m2) - 1);
                        break;
                    }
                    gap += 16u;
                }
            }
            list[pos++] = ((c * 16u + j) << 16) | (min(gap, 255u) << 8) | byte_of(q, j);
        }
        __syncwarp();
        for (uint32_t i = lane; i < total; i += 32u) {
            const uint32_t e = list[i];
            const uint32_t idx = e >> 16;
            uint32_t cell = base + idx;
            if (cell >= L) cell -= L;
            uint32_t vel = min(min((e & 0xFFu) + 1u, rc.vmax), (e >> 8) & 0xFFu);   // rules 1, 2
            if (D == Draw::kAlways) {
                vel -= vel > 0u ? 1u : 0u;                                          // rule 3, p = 1
            } else if (D == Draw::kPhilox) {
                const uint32_t u = philox_word0(cell, step, rc.road, kTagSlowdown, rc.key0, rc.key1);
                vel -= (vel > 0u && u < (uint32_t)rc.thr) ? 1u : 0u;                // rule 3
            }
            nxt[idx + vel] = (int8_t)vel;                                           // rule 4
            if (idx - H < own_cells) {
                tsum += vel;
                tcross += (cell + vel >= L) ? 1u : 0u;
            }
        }
        __syncwarp();
    }
}

template <Draw D>
__global__ void __launch_bounds__(kGridThreads) grid_tiled_kernel(const GridStep g, const GridTileGeom geo)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t s_full[2];
    __shared__ unsigned long long s_sum[kMaxFusedSteps];
    __shared__ unsigned long long s_cross[kMaxFusedSteps];
    __shared__ uint32_t s_list[kGridWarps][kRowCells];

    const RoadConst rc = g.rc;
    const uint32_t L = rc.L;
    const uint32_t H = geo.halo;
    const uint32_t W = geo.width;
    const uint32_t WP = geo.padded;
    const uint32_t C = (uint32_t)kGridTileCells;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    int8_t *const pool = reinterpret_cast<int8_t *>(smem);
    // buffers: stage 0, stage 1 (bulk-load targets), then nwork output buffers
    auto stage = [&](uint32_t b) { return pool + b * WP; };
    auto work = [&](uint32_t b) { return pool + (2u + b) * WP; };

    for (int i = tid; i < g.ksteps; i += kGridThreads) {
        s_sum[i] = 0ull;
        s_cross[i] = 0ull;
    }
    if (tid == 0) {
        mbar_init(&s_full[0], 1);
        mbar_init(&s_full[1], 1);
        fence_mbar_init();
    }
    // stage padding (never written by the loads) and the output buffers start empty
    for (uint32_t c = W / 16u + tid; c < WP / 16u; c += kGridThreads) {
        reinterpret_cast<uint4 *>(stage(0))[c] = kEmpty4;
        reinterpret_cast<uint4 *>(stage(1))[c] = kEmpty4;
    }
    for (uint32_t c = tid; c < geo.nwork * WP / 16u; c += kGridThreads) reinterpret_cast<uint4 *>(work(0))[c] = kEmpty4;
    __syncthreads();

    auto bulk_ok = [&](uint32_t tile) {
        const uint32_t t0 = tile * C;
        return t0 >= H && t0 + C + H <= L;
    };
    uint32_t parity = 0;   // bit b: phase parity of s_full[b]
    uint32_t wa = 0;       // output buffer of the next tile's first step (already empty)
    uint32_t tile = blockIdx.x;
    if (tid == 0 && tile < geo.n_tiles && bulk_ok(tile)) {
        fence_proxy_async();
        mbar_expect_tx(&s_full[0], W);
        bulk_load(stage(0), g.c_in + (tile * C - H), W, &s_full[0]);
    }
    for (uint32_t it = 0; tile < geo.n_tiles; tile += gridDim.x, ++it) {
        const uint32_t sb = it & 1u;
        const uint32_t t0 = tile * C;
        const uint32_t own_cells = min(C, L - t0);
        const uint32_t base = t0 >= H ? t0 - H : t0 + L - H;   // road cell of buffer index 0
        const uint32_t next = tile + gridDim.x;
        if (tid == 0) {
            // earlier bulk stores must have read their source before buffers are reused
            bulk_wait_read_all();
            if (next < geo.n_tiles && bulk_ok(next)) {
                fence_proxy_async();
                mbar_expect_tx(&s_full[sb ^ 1u], W);
                bulk_load(stage(sb ^ 1u), g.c_in + (next * C - H), W, &s_full[sb ^ 1u]);
            }
        }
        int8_t *in = stage(sb);
        bool ok = true;
        if (bulk_ok(tile)) {
            ok = mbar_wait_bounded(&s_full[sb], (parity >> sb) & 1u);
            parity ^= 1u << sb;
        } else {
            for (uint32_t i = tid; i < W; i += kGridThreads) {
                uint32_t cell = base + i;
                if (cell >= L) cell -= L;
                in[i] = g.c_in[cell];
            }
        }
        if (!__syncthreads_and(ok)) {
            if (tid == 0) {
                atomicOr(g.status, kStatusTimeout);
                if (next < geo.n_tiles && bulk_ok(next)) mbar_wait_bounded(&s_full[sb ^ 1u], (parity >> (sb ^ 1u)) & 1u);
                bulk_wait_all();
            }
            return;
        }

        const int8_t *cur = in;
        for (int s = 0; s < g.ksteps; ++s) {
            int8_t *nxt = work((wa + (uint32_t)s) % geo.nwork);
            int8_t *clr = work((wa + (uint32_t)s + 1u) % geo.nwork);
            uint32_t tsum = 0, tcross = 0;
            grid_step<D>(rc, cur, nxt, clr, geo, own_cells, base, g.step0 + (uint32_t)s, s_list[warp], tsum, tcross);
            tsum = __reduce_add_sync(0xFFFFFFFFu, tsum);
            tcross = __reduce_add_sync(0xFFFFFFFFu, tcross);
            if (lane == 0 && (tsum | tcross)) {
                atomicAdd(&s_sum[s], (unsigned long long)tsum);
                atomicAdd(&s_cross[s], (unsigned long long)tcross);
            }
            if (s + 1 == g.ksteps) fence_proxy_async();   // the result may leave by bulk store
            __syncthreads();
            cur = nxt;
        }
        const int8_t *fin = cur;
        wa = (wa + (uint32_t)g.ksteps) % geo.nwork;

        if (own_cells == C) {
            if (tid == 0) {
                bulk_store(g.c_out + t0, fin + H, C);
                bulk_commit();
            }
        } else {
            for (uint32_t i = tid; i < own_cells; i += kGridThreads) g.c_out[t0 + i] = fin[H + i];
        }
    }
    if (tid == 0) bulk_wait_all();
    __syncthreads();
    for (int i = tid; i < g.ksteps; i += kGridThreads) {
        if (s_sum[i]) atomicAdd(&g.sum_v[i], s_sum[i]);
        if (s_cross[i]) atomicAdd(&g.crossings[i], s_cross[i]);
    }
}

// Whole ring in one block.  Cells [0, L) plus the successor grid in shared
// memory; gaps and moves wrap modulo L.
__global__ void __launch_bounds__(1024) grid_ring_kernel(const GridStep g)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint32_t s_psum[32];
    __shared__ uint32_t s_pcross[32];
    const RoadConst rc = g.rc;
    const uint32_t L = rc.L;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t nwarps = blockDim.x >> 5;
    int8_t *cur = reinterpret_cast<int8_t *>(smem);
    int8_t *nxt = cur + ((L + 15u) / 16u) * 16u;

    for (uint32_t i = tid; i < L; i += blockDim.x) cur[i] = g.c_in[i];
    for (int s = 0; s < g.ksteps; ++s) {
        const uint32_t step = g.step0 + (uint32_t)s;
        for (uint32_t i = tid; i < L; i += blockDim.x) nxt[i] = -1;
        __syncthreads();
        uint32_t tsum = 0, tcross = 0;
        for (uint32_t i = tid; i < L; i += blockDim.x) {
            const int8_t here = cur[i];
            if (here < 0) continue;
            const uint32_t limit = min((uint32_t)here + 1u, rc.vmax);
            uint32_t gap = 0;
            uint32_t ahead = i + 1u == L ? 0u : i + 1u;
            while (gap < limit && cur[ahead] < 0) {   // reaches the car itself after L-1 cells
                ++gap;
                ahead = ahead + 1u == L ? 0u : ahead + 1u;
            }
            const uint32_t vel = new_velocity(rc, (uint32_t)here, gap, i, step);
            uint32_t dest = i + vel;
            const bool wrap = dest >= L;
            if (wrap) dest -= L;
            nxt[dest] = (int8_t)vel;
            tsum += vel;
            tcross += wrap ? 1u : 0u;
        }
        tsum = __reduce_add_sync(0xFFFFFFFFu, tsum);
        tcross = __reduce_add_sync(0xFFFFFFFFu, tcross);
        if (lane == 0) {
            s_psum[warp] = tsum;
            s_pcross[warp] = tcross;
        }
        __syncthreads();
        if (tid == 0) {
            unsigned long long sv = 0, cr = 0;
            for (uint32_t w = 0; w < nwarps; ++w) {
                sv += s_psum[w];
                cr += s_pcross[w];
            }
            g.sum_v[s] = sv;
            g.crossings[s] = cr;
        }
        int8_t *t = cur;
        cur = nxt;
        nxt = t;
        // the next step's clear of nxt (the old cur) must wait for this step's
        // reads, and thread 0's reads of s_psum for the next step's writes
        __syncthreads();
    }
    for (uint32_t i = tid; i < L; i += blockDim.x) g.c_out[i] = cur[i];
}

GridTileGeom make_geom(int ksteps, uint32_t vmax, uint32_t L)
{
    GridTileGeom geo;
    geo.halo = grid_halo(ksteps, vmax);
    geo.width = (uint32_t)kGridTileCells + 2u * geo.halo;
    geo.lookahead = (vmax + 15u) / 16u + 1u;
    geo.padded = geo.width + 16u * (geo.lookahead + 1u);
    geo.n_tiles = (L + (uint32_t)kGridTileCells - 1u) / (uint32_t)kGridTileCells;
    geo.nwork = ksteps == 1 ? 2u : 3u;
    return geo;
}

size_t grid_tiled_smem(const GridTileGeom &geo) { return (2u + geo.nwork) * (size_t)geo.padded; }

// Static plus dynamic shared memory exceeds the default 48 KB, so the
// dynamic size is allowed explicitly (a per-device function attribute).
template <Draw D>
cudaError_t prepare_grid_kernel(size_t smem)
{
    return cudaFuncSetAttribute(grid_tiled_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

}  // namespace

int grid_tiled_blocks_per_sm()
{
    // the common case: k = 1, vmax = 5
    const GridTileGeom geo = make_geom(1, 5, 1u << 20);
    const size_t smem = grid_tiled_smem(geo);
    if (prepare_grid_kernel<Draw::kPhilox>(smem) != cudaSuccess) return 1;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, grid_tiled_kernel<Draw::kPhilox>, kGridThreads, smem) !=
        cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

cudaError_t launch_grid_tiled(const GridStep &g, int blocks, cudaStream_t s)
{
    if (g.ksteps <= 0) return cudaSuccess;
    if (g.ksteps > kMaxFusedSteps) return cudaErrorInvalidValue;
    const GridTileGeom geo = make_geom(g.ksteps, g.rc.vmax, g.rc.L);
    if (g.rc.L < geo.width) return cudaErrorInvalidValue;   // the buffer must not wrap the ring twice
    const size_t smem = grid_tiled_smem(geo);
    const int grid = (int)((uint32_t)blocks < geo.n_tiles ? (uint32_t)blocks : geo.n_tiles);
    cudaError_t e;
    if (g.rc.thr == 0) {
        if ((e = prepare_grid_kernel<Draw::kNever>(smem)) != cudaSuccess) return e;
        grid_tiled_kernel<Draw::kNever><<<grid, kGridThreads, smem, s>>>(g, geo);
    } else if (g.rc.thr > 0xFFFFFFFFull) {
        if ((e = prepare_grid_kernel<Draw::kAlways>(smem)) != cudaSuccess) return e;
        grid_tiled_kernel<Draw::kAlways><<<grid, kGridThreads, smem, s>>>(g, geo);
    } else {
        if ((e = prepare_grid_kernel<Draw::kPhilox>(smem)) != cudaSuccess) return e;
        grid_tiled_kernel<Draw::kPhilox><<<grid, kGridThreads, smem, s>>>(g, geo);
    }
    return cudaGetLastError();
}

cudaError_t launch_grid_ring(const GridStep &g, cudaStream_t s)
{
    if (g.ksteps <= 0) return cudaSuccess;
    if (g.rc.L == 0 || g.rc.L > (uint32_t)kGridRingMaxCells) return cudaErrorInvalidValue;
    const size_t smem = 2u * (((size_t)g.rc.L + 15u) / 16u * 16u);
    if (smem > 48u * 1024u) {
        cudaError_t e = cudaFuncSetAttribute(grid_ring_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    uint32_t threads = (g.rc.L + 31u) / 32u * 32u;
    if (threads > 1024u) threads = 1024u;
    grid_ring_kernel<<<1, threads, smem, s>>>(g);
    return cudaGetLastError();
}

}  // namespace nasch
