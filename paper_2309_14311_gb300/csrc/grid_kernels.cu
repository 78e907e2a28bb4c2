// Grid NaSch step kernels: one int8 per cell, -1 empty, else the velocity of
// the car on it ("Concepts Covered": the grid representation; Handout,
// model section rules 1-4).
//
// Tiled kernel.  A tile is kGridTileCells cells staged in shared memory with
// a halo of H = round_up(k * vmax, 16) cells on each side: after one step a
// cell depends on the cells within vmax of it (a car arriving from behind,
// the gap of that car ahead), so after k fused steps the middle tile is
// exact.  Per step every thread takes 16-cell chunks, turns them into an
// occupancy bit mask (one bit per cell), finds each car's gap with
// find-first-set on the mask of the cells ahead, applies rules 1-3 and
// scatters the car into the next buffer, which was cleared to -1 one step
// earlier (three rotating buffers, one barrier per step).  Rule 2 makes the
// scatter collision-free.  Statistics of the cars that start the step in
// the tile's own cells are reduced per warp, per block, and added to the
// per-step series once per block.  The first and last tiles take their halo
// across the ring boundary (modular cell index).
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

struct GridTileGeom {
    uint32_t halo;      // H, multiple of 16
    uint32_t width;     // W = tile + 2H cells processed per step
    uint32_t padded;    // W + pad: buffer length (multiple of 16)
    uint32_t n_tiles;
    uint32_t lookahead; // chunks read beyond a car's own chunk for its gap
};

constexpr uint4 kEmpty4 = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu};

template <int NT>
__global__ void __launch_bounds__(NT) grid_tiled_kernel(const GridStep g, const GridTileGeom geo)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long s_sum[kMaxFusedSteps];
    __shared__ unsigned long long s_cross[kMaxFusedSteps];

    for (int i = threadIdx.x; i < g.ksteps; i += NT) {
        s_sum[i] = 0ull;
        s_cross[i] = 0ull;
    }

    const RoadConst rc = g.rc;
    const uint32_t L = rc.L;
    const uint32_t H = geo.halo;
    const uint32_t W = geo.width;
    const uint32_t WP = geo.padded;
    const uint32_t chunks = W / 16u;
    const uint32_t chunks_padded = WP / 16u;
    const uint32_t lane = threadIdx.x & 31u;
    int8_t *const pool = reinterpret_cast<int8_t *>(smem);
    // rotating roles of the three buffers, as byte offsets into the pool
    uint32_t ia = 0, ib = WP, ic = 2u * WP;

    for (uint32_t tile = blockIdx.x; tile < geo.n_tiles; tile += gridDim.x) {
        const uint32_t t0 = tile * (uint32_t)kGridTileCells;
        const uint32_t own_cells = min((uint32_t)kGridTileCells, L - t0);
        // road cell of buffer index 0, i.e. t0 - H on the ring (L > H here)
        const uint32_t base = t0 >= H ? t0 - H : t0 + L - H;

        // stage the tile and its halos; pad with empty cells
        uint4 *a4 = reinterpret_cast<uint4 *>(pool + ia);
        if (t0 >= H && t0 + (uint32_t)kGridTileCells + H <= L) {
            const uint4 *src = reinterpret_cast<const uint4 *>(g.c_in + (t0 - H));
            for (uint32_t c = threadIdx.x; c < chunks; c += NT) a4[c] = __ldg(src + c);
        } else {
            for (uint32_t i = threadIdx.x; i < W; i += NT) {
                uint32_t cell = base + i;
                if (cell >= L) cell -= L;
                if (cell >= L) cell -= L;
                pool[ia + i] = g.c_in[cell];
            }
        }
        for (uint32_t c = chunks + threadIdx.x; c < chunks_padded; c += NT) a4[c] = kEmpty4;
        uint4 *b4 = reinterpret_cast<uint4 *>(pool + ib);
        for (uint32_t c = threadIdx.x; c < chunks_padded; c += NT) b4[c] = kEmpty4;
        __syncthreads();

        for (int s = 0; s < g.ksteps; ++s) {
            const uint32_t step = g.step0 + (uint32_t)s;
            const int8_t *cur = pool + ia;
            int8_t *nxt = pool + ib;
            const uint4 *cur4 = reinterpret_cast<const uint4 *>(cur);
            uint32_t tsum = 0, tcross = 0;
            for (uint32_t c = threadIdx.x; c < chunks; c += NT) {
                const uint4 q = cur4[c];
                uint32_t mask = occupancy16(q);
                if (mask == 0u) continue;
                // occupancy of the following 16 cells, for gaps that cross the chunk end
                const uint32_t ahead = occupancy16(cur4[c + 1]);
                const uint32_t window = mask | (ahead << 16);
                while (mask) {
                    const uint32_t j = (uint32_t)(__ffs(mask) - 1);
                    mask &= mask - 1u;
                    const uint32_t i = c * 16u + j;   // buffer index of the car
                    const uint32_t vel0 = byte_of(q, j);
                    const uint32_t after = window >> (j + 1u);
                    uint32_t gap = after ? (uint32_t)(__ffs(after) - 1) : 31u - j;
                    if (after == 0u && gap < rc.vmax) {
                        // vmax > 16: keep scanning whole chunks ahead
                        uint32_t cc = c + 2u;
                        for (uint32_t n = 1; n < geo.lookahead && gap < rc.vmax; ++n, ++cc) {
                            const uint32_t m2 = occupancy16(cur4[cc]);
                            if (m2) {
                                gap += (uint32_t)(__ffs(m2) - 1);
                                break;
                            }
                            gap += 16u;
                        }
                    }
                    uint32_t cell = base + i;
                    if (cell >= L) cell -= L;
                    if (cell >= L) cell -= L;
                    const uint32_t vel = new_velocity(rc, vel0, gap, cell, step);
                    nxt[i + vel] = (int8_t)vel;
                    if (i >= H && i - H < own_cells) {
                        tsum += vel;
                        tcross += (cell + vel >= L) ? 1u : 0u;
                    }
                }
            }
            // clear the buffer that the next step scatters into
            uint4 *c4 = reinterpret_cast<uint4 *>(pool + ic);
            for (uint32_t c = threadIdx.x; c < chunks_padded; c += NT) c4[c] = kEmpty4;

            tsum = __reduce_add_sync(0xFFFFFFFFu, tsum);
            tcross = __reduce_add_sync(0xFFFFFFFFu, tcross);
            if (lane == 0 && (tsum | tcross)) {
                atomicAdd(&s_sum[s], (unsigned long long)tsum);
                atomicAdd(&s_cross[s], (unsigned long long)tcross);
            }
            __syncthreads();
            const uint32_t old_a = ia;
            ia = ib;
            ib = ic;
            ic = old_a;
        }

        // write back the tile's own cells
        const int8_t *fin = pool + ia;
        if (own_cells == (uint32_t)kGridTileCells) {
            const uint4 *f4 = reinterpret_cast<const uint4 *>(fin + H);
            uint4 *dst = reinterpret_cast<uint4 *>(g.c_out + t0);
            for (uint32_t c = threadIdx.x; c < (uint32_t)kGridTileCells / 16u; c += NT) dst[c] = f4[c];
        } else {
            for (uint32_t i = threadIdx.x; i < own_cells; i += NT) g.c_out[t0 + i] = fin[H + i];
        }
        __syncthreads();
    }

    __syncthreads();
    for (int i = threadIdx.x; i < g.ksteps; i += NT) {
        if (s_sum[i]) atomicAdd(&g.sum_v[i], s_sum[i]);
        if (s_cross[i]) atomicAdd(&g.crossings[i], s_cross[i]);
    }
}

// Whole ring in one block.  Cells [0, L) plus the successor grid in shared
// memory; gaps and moves wrap modulo L.
__global__ void __launch_bounds__(1024) grid_ring_kernel(const GridStep g)
{
    extern __shared__ __align__(16) unsigned char smem[];
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

GridTileGeom make_geom(const GridStep &g)
{
    GridTileGeom geo;
    geo.halo = grid_halo(g.ksteps, g.rc.vmax);
    geo.width = (uint32_t)kGridTileCells + 2u * geo.halo;
    geo.lookahead = (g.rc.vmax + 15u) / 16u + 1u;
    geo.padded = geo.width + 16u * (geo.lookahead + 1u);
    geo.n_tiles = (g.rc.L + (uint32_t)kGridTileCells - 1u) / (uint32_t)kGridTileCells;
    return geo;
}

size_t grid_tiled_smem(const GridTileGeom &geo) { return 3u * (size_t)geo.padded; }

}  // namespace

int grid_tiled_blocks_per_sm()
{
    // the common case: k = 8, vmax = 5
    GridStep g{};
    g.ksteps = 8;
    g.rc.vmax = 5;
    g.rc.L = 1u << 20;
    const size_t smem = grid_tiled_smem(make_geom(g));
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, grid_tiled_kernel<kGridThreads>, kGridThreads,
                                                      smem) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

cudaError_t launch_grid_tiled(const GridStep &g, int blocks, cudaStream_t s)
{
    if (g.ksteps <= 0) return cudaSuccess;
    if (g.ksteps > kMaxFusedSteps || g.rc.L <= (uint32_t)kGridRingMaxCells) return cudaErrorInvalidValue;
    const GridTileGeom geo = make_geom(g);
    const size_t smem = grid_tiled_smem(geo);
    if (smem > 48u * 1024u) {
        cudaError_t e = cudaFuncSetAttribute(grid_tiled_kernel<kGridThreads>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int grid = (int)((uint32_t)blocks < geo.n_tiles ? (uint32_t)blocks : geo.n_tiles);
    grid_tiled_kernel<kGridThreads><<<grid, kGridThreads, smem, s>>>(g, geo);
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
