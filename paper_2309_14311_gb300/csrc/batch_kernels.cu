// Batched NaSch: many independent roads advanced together (the paper's
// "Variations": a parameter study as embarrassingly parallel work).
//
// One launch per super-step.  A persistent grid of 256-thread blocks pulls
// items from the super-step's work-list with an atomic cursor; an item is a
// piece of one road and runs that road's k fused steps:
//   agent tile: 16 warp-tiles of 256 consecutive cars, two per warp (32 lanes
//               x 8 cars in registers, leader by warp shuffle, halo of
//               round_up(k, 8));
//   grid warp:  8 warp-tiles, one per warp, of 2048 staged cells (tile + halos
//               of round_up(k*vmax,16) <= 512), each stepped by its warp alone
//               as a list of its cars (the list method of the single-road
//               fused kernel);
//   grid tile:  one staged 8192-cell span for larger halos, stepped as a list
//               of its cars by the whole block (the span-list method);
//   agent ring: a whole ring of N <= 2048 cars in one block;
//   grid ring:  a whole ring of L <= 8192 cells in shared memory.
// The step code is the single-road kernels' (tile_device.cuh), so a road in
// a batch computes exactly what it computes alone.  Per-step statistics are
// reduced per block and added to the road's series.  A host-mapped flag lets
// the host cancel: items pulled after it is set do nothing.
//
// Initial positions come from Floyd's algorithm run on the GPU, one block
// per road, into a bit map of the road's cells (sorted positions are then
// the set bits in order).
#include "batch_internal.h"
#include "floyd_device.cuh"
#include "tile_device.cuh"

namespace nasch {
namespace {

template <Draw D>
__device__ __forceinline__ void batch_agent_tile(const BatchRoadDev &rd, const RoadConst &rc, uint32_t item_tile,
                                                 uint32_t par, uint32_t step0, int kk, unsigned long long *s_sum,
                                                 unsigned long long *s_cross)
{
    const uint32_t warp = threadIdx.x >> 5;
    const uint32_t owned = rd.tile;
    AgentStep a;
    a.status = nullptr;
    // select by branch, not by index, so the descriptor stays in registers
    a.x_in = par ? rd.x[1] : rd.x[0];
    a.v_in = par ? rd.v[1] : rd.v[0];
    a.x_out = par ? rd.x[0] : rd.x[1];
    a.v_out = par ? rd.v[0] : rd.v[1];
    a.N = rd.N;
    a.rc = rc;
    a.step0 = step0;
    a.ksteps = kk;
    a.sum_v = nullptr;
    a.crossings = nullptr;
    // this warp's consecutive warp-tiles of the item
    for (uint32_t w2 = 0; w2 < kBatchWarpTilesPerWarp; ++w2) {
        const uint32_t t0 = ((item_tile * (uint32_t)(kBatchThreads / 32) + warp) * kBatchWarpTilesPerWarp + w2) * owned;
        if (t0 >= rd.N) return;
        if (t0 + kBatchAgentSpan <= rd.N)
            agent_warp_tile<kBatchAgentTileR, D, true, true>(a, t0, owned, s_sum, s_cross);
        else
            agent_warp_tile<kBatchAgentTileR, D, false, true>(a, t0, owned, s_sum, s_cross);
    }
}

template <Draw D>
__device__ __forceinline__ void batch_grid_tile(const BatchRoadDev &rd, const RoadConst &rc, uint32_t item_tile,
                                                uint32_t par, uint32_t step0, int kk, int8_t *pool, uint32_t *s_first,
                                                uint32_t *s_count, unsigned long long *s_sum,
                                                unsigned long long *s_cross)
{
    const uint32_t tid = threadIdx.x;
    const uint32_t L = rd.L, H = rd.halo, C = rd.tile;
    const uint32_t W = (uint32_t)kGridSpan;
    int8_t *stage = pool;
    int8_t *out = pool + W;
    uint16_t *s_pos = reinterpret_cast<uint16_t *>(pool + 2u * W);
    uint8_t *s_vel = reinterpret_cast<uint8_t *>(s_pos + W);
    const int8_t *c_in = par ? rd.cells[1] : rd.cells[0];
    int8_t *c_out = par ? rd.cells[0] : rd.cells[1];
    const uint32_t t0 = item_tile * C;
    const uint32_t own_cells = min(C, L - t0);
    const uint32_t base = t0 >= H ? t0 - H : t0 + L - H;

    if (t0 >= H && t0 + C + H <= L) {
        const uint4 *src = reinterpret_cast<const uint4 *>(c_in + (t0 - H));
        for (uint32_t c = tid; c < W / 16u; c += kBatchThreads) reinterpret_cast<uint4 *>(stage)[c] = __ldg(src + c);
    } else {
        for (uint32_t i = tid; i < W; i += kBatchThreads) {
            uint32_t cell = base + i;
            if (cell >= L) cell -= L;
            stage[i] = c_in[cell];
        }
    }
    __syncthreads();
    grid_span_steps<D>(rc, stage, out, H, own_cells, base, step0, kk, s_pos, s_vel, W, s_first, s_count, s_sum,
                       s_cross);
    __syncthreads();
    if (own_cells == C) {
        const uint4 *f4 = reinterpret_cast<const uint4 *>(out + H);
        uint4 *dst = reinterpret_cast<uint4 *>(c_out + t0);
        for (uint32_t c = tid; c < C / 16u; c += kBatchThreads) dst[c] = f4[c];
    } else {
        for (uint32_t i = tid; i < own_cells; i += kBatchThreads) c_out[t0 + i] = out[H + i];
    }
}

// Per warp: its staged span, and the list of the span's cars.
struct BatchWarpSmem {
    int8_t span[kKwBuf];
    uint16_t pos[kKwList];
    uint8_t vel[kKwList];
};

template <Draw D>
__device__ __forceinline__ void batch_grid_warp(const BatchRoadDev &rd, const RoadConst &rc, uint32_t item_tile,
                                                uint32_t par, uint32_t step0, int kk, int8_t *pool,
                                                unsigned long long *s_sum, unsigned long long *s_cross)
{
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    BatchWarpSmem &w = reinterpret_cast<BatchWarpSmem *>(pool)[warp];
    const uint32_t L = rd.L, H = rd.halo, C = rd.tile;
    const int8_t *c_in = par ? rd.cells[1] : rd.cells[0];
    int8_t *c_out = par ? rd.cells[0] : rd.cells[1];
    const uint32_t t0 = (item_tile * (uint32_t)(kBatchThreads / 32) + warp) * C;
    if (t0 >= L) return;
    const uint32_t own = min(C, L - t0);
    const uint32_t base = t0 >= H ? t0 - H : t0 + L - H;
    if (t0 >= H && t0 + C + H <= L) {
        const uint4 *src = reinterpret_cast<const uint4 *>(c_in + (t0 - H));
#pragma unroll
        for (uint32_t k = 0; k < kKwSpan / 512u; ++k)
            reinterpret_cast<uint4 *>(w.span)[lane + 32u * k] = __ldg(src + lane + 32u * k);
    } else {
        for (uint32_t i = lane; i < kKwSpan; i += 32u) {
            uint32_t c = base + i;
            if (c >= L) c -= L;
            w.span[i] = c_in[c];
        }
    }
    __syncwarp();
    grid_warp_steps<D>(rc, PlainDraws{rc, 0}, w.span, WarpList{w.pos, w.vel, kKwList, nullptr, nullptr}, H, own, base, step0,
                       kk, []() {},
                       [&](int s, uint32_t sum, uint32_t cross) {
                           if (sum) atomicAdd(&s_sum[s], (unsigned long long)sum);
                           if (cross) atomicAdd(&s_cross[s], (unsigned long long)cross);
                       });
    if (own == C) {
        const uint4 *f4 = reinterpret_cast<const uint4 *>(w.span + H);
        uint4 *dst = reinterpret_cast<uint4 *>(c_out + t0);
        for (uint32_t c = lane; c < C / 16u; c += 32u) dst[c] = f4[c];
    } else {
        for (uint32_t i = lane; i < own; i += 32u) c_out[t0 + i] = w.span[H + i];
    }
}

template <Draw D>
__device__ __forceinline__ void batch_item(const BatchRoadDev &rd, const RoadConst &rc, uint32_t item_tile,
                                           uint32_t par, uint32_t step0, int kk, uint32_t padded, int8_t *pool,
                                           uint32_t *s_first, uint32_t *s_count, uint32_t *s_psum, uint32_t *s_pcross,
                                           unsigned long long *s_sum, unsigned long long *s_cross)
{
    switch (rd.type) {
    case kBatchAgentTile:
        batch_agent_tile<D>(rd, rc, item_tile, par, step0, kk, s_sum, s_cross);
        break;
    case kBatchGridWarp:
        batch_grid_warp<D>(rd, rc, item_tile, par, step0, kk, pool, s_sum, s_cross);
        break;
    case kBatchGridTile:
        batch_grid_tile<D>(rd, rc, item_tile, par, step0, kk, pool, s_first, s_count, s_sum, s_cross);
        break;
    case kBatchAgentRing:
        agent_ring_steps<kBatchAgentR>(par ? rd.x[1] : rd.x[0], par ? rd.v[1] : rd.v[0], par ? rd.x[0] : rd.x[1],
                                       par ? rd.v[0] : rd.v[1], rd.N, rc, step0, kk, s_sum, s_cross, s_first, s_psum,
                                       s_pcross);
        break;
    default:
        grid_ring_steps(par ? rd.cells[1] : rd.cells[0], par ? rd.cells[0] : rd.cells[1], rc, step0, kk, pool,
                        pool + padded, s_sum, s_cross, s_psum, s_pcross);
        break;
    }
}

__global__ void __launch_bounds__(kBatchThreads, kBatchMinBlocks) batch_kernel(const BatchLaunch bl)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint32_t s_first[2 * kBatchThreads];
    __shared__ uint32_t s_count[kBatchThreads / 32 + 1];
    __shared__ uint32_t s_psum[2 * 32];
    __shared__ uint32_t s_pcross[2 * 32];
    __shared__ unsigned long long s_sum[kMaxFusedSteps];
    __shared__ unsigned long long s_cross[kMaxFusedSteps];
    __shared__ uint32_t s_item;
    int8_t *const pool = reinterpret_cast<int8_t *>(smem);
    const uint32_t tid = threadIdx.x;

    for (;;) {
        if (tid == 0) {
            uint32_t i = atomicAdd(bl.counter, 1u);
            if (*bl.cancel) i = 0xFFFFFFFFu;
            s_item = i;
        }
        __syncthreads();
        const uint32_t i = s_item;
        if (i >= bl.n_items) break;
        const BatchItem it = bl.items[i];
        const BatchRoadDev rd = bl.roads[it.road];
        const uint32_t sst = rd.sbase + bl.super_step;   // this road's super-step
        const uint32_t s0 = sst * rd.k;
        // an item past the road's last step has nothing to do (the host never
        // lists one; this keeps a stale list from writing past the series)
        const int kk = s0 < rd.T ? (int)min(rd.k, rd.T - s0) : 0;
        const uint32_t par = sst & 1u;
        const uint32_t step0 = rd.step0 + s0;
        RoadConst rc;
        rc.L = rd.L;
        rc.vmax = rd.vmax;
        rc.thr = rd.thr;
        rc.key0 = rd.key0;
        rc.key1 = rd.key1;
        rc.road = rd.road_id;
        for (int j = tid; j < kk; j += kBatchThreads) {
            s_sum[j] = 0ull;
            s_cross[j] = 0ull;
        }
        __syncthreads();
        if (kk == 0) continue;   // uniform across the block; the loop head synchronises again
        switch (draw_mode(rd.thr)) {
        case Draw::kNever:
            batch_item<Draw::kNever>(rd, rc, it.tile, par, step0, kk, bl.padded, pool, s_first, s_count, s_psum,
                                     s_pcross, s_sum, s_cross);
            break;
        case Draw::kAlways:
            batch_item<Draw::kAlways>(rd, rc, it.tile, par, step0, kk, bl.padded, pool, s_first, s_count, s_psum,
                                      s_pcross, s_sum, s_cross);
            break;
        default:
            batch_item<Draw::kPhilox>(rd, rc, it.tile, par, step0, kk, bl.padded, pool, s_first, s_count, s_psum,
                                      s_pcross, s_sum, s_cross);
            break;
        }
        __syncthreads();
        for (int j = tid; j < kk; j += kBatchThreads) {
            if (s_sum[j]) atomicAdd(&rd.sum_v[s0 + j], s_sum[j]);
            if (s_cross[j]) atomicAdd(&rd.crossings[s0 + j], s_cross[j]);
        }
    }
}

// Floyd's algorithm (Bentley & Floyd, CACM 1987), one block per road, 1024
// draws at a time (floyd_road_bits): the road's chosen cells become set bits
// of its bit map.
__global__ void __launch_bounds__(kFloydBlock) batch_floyd_bits_kernel(const BatchRoadDev *roads, uint32_t n,
                                                                       uint64_t *const *bitmaps)
{
    __shared__ FloydSmem sm;
    for (uint32_t r = blockIdx.x; r < n; r += gridDim.x) {
        const BatchRoadDev rd = roads[r];
        floyd_road_bits(rd.L, rd.N, rd.road_id, rd.key0, rd.key1,
                        reinterpret_cast<unsigned long long *>(bitmaps[r]), sm);
    }
}

// Bit map -> state, one block per road: agent roads get their sorted
// positions (a block-wide prefix sum over the words' bit counts), grid roads
// a 0 (a car at rest) on every chosen cell.
__global__ void __launch_bounds__(256) batch_floyd_expand_kernel(const BatchRoadDev *roads, uint32_t n,
                                                                 uint64_t *const *bitmaps)
{
    __shared__ uint32_t s_warp[8];
    __shared__ uint32_t s_total;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    for (uint32_t r = blockIdx.x; r < n; r += gridDim.x) {
        const BatchRoadDev rd = roads[r];
        const uint64_t *bm = bitmaps[r];
        const uint32_t words = (rd.L + 63u) / 64u;
        const bool grid = rd.type == kBatchGridTile || rd.type == kBatchGridRing || rd.type == kBatchGridWarp;
        if (grid) {
            for (uint32_t w = tid; w < words; w += 256u)
                for (uint64_t bits = bm[w]; bits; bits &= bits - 1) rd.cells[0][64u * w + (uint32_t)__ffsll(bits) - 1u] = 0;
            continue;
        }
        uint32_t running = 0;
        for (uint32_t base = 0; base < words; base += 256u) {
            const uint32_t w = base + tid;
            const uint64_t bits = w < words ? bm[w] : 0ull;
            const uint32_t c = (uint32_t)__popcll(bits);
            uint32_t incl = c;
#pragma unroll
            for (uint32_t d = 1; d < 32; d <<= 1) {
                const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
                if (lane >= d) incl += t;
            }
            if (lane == 31) s_warp[warp] = incl;
            __syncthreads();
            if (tid == 0) {
                uint32_t acc = 0;
                for (int k = 0; k < 8; ++k) {
                    const uint32_t t = s_warp[k];
                    s_warp[k] = acc;
                    acc += t;
                }
                s_total = acc;
            }
            __syncthreads();
            uint32_t pos = running + s_warp[warp] + incl - c;
            for (uint64_t b2 = bits; b2; b2 &= b2 - 1) rd.x[0][pos++] = (int32_t)(64u * w + (uint32_t)__ffsll(b2) - 1u);
            running += s_total;
            __syncthreads();
        }
    }
}

}  // namespace

// grid tiles: staged span, output span, car list (uint16 position + uint8
// velocity per cell of the span); grid rings: two ring buffers of <= 8192
size_t batch_smem_bytes(uint32_t padded)
{
    (void)padded;
    // the larger of: a block-wide span (stage, out, and its list) and the
    // eight warp-tiles of the list method
    const size_t span = 5u * (size_t)kGridSpan;
    const size_t warps = (size_t)(kBatchThreads / 32) * sizeof(BatchWarpSmem);
    return span > warps ? span : warps;
}

int batch_blocks_per_sm(uint32_t padded)
{
    const size_t smem = batch_smem_bytes(padded);
    if (cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 1;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel, kBatchThreads, smem) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

cudaError_t launch_batch_super_step(const BatchLaunch &bl, int blocks, cudaStream_t s)
{
    const size_t smem = batch_smem_bytes(bl.padded);
    cudaError_t e = cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    batch_kernel<<<blocks, kBatchThreads, smem, s>>>(bl);
    return cudaGetLastError();
}

cudaError_t launch_batch_floyd(const BatchRoadDev *roads, uint32_t n, uint64_t *const *bitmaps, int sms, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    batch_floyd_bits_kernel<<<n < (uint32_t)sms * 2u ? n : (uint32_t)sms * 2u, kFloydBlock, 0, s>>>(roads, n, bitmaps);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const uint32_t blocks = n < (uint32_t)sms * 8u ? n : (uint32_t)sms * 8u;
    batch_floyd_expand_kernel<<<blocks, 256, 0, s>>>(roads, n, bitmaps);
    return cudaGetLastError();
}

// This unit's debug word (zero in release builds).
NASCH_DEBUG_READER(debug_word_batch)

}  // namespace nasch
