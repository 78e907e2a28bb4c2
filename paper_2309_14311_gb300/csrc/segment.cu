// One rank's share of a ring road split into contiguous cell ranges: the
// grid layout's 1-D domain decomposition (the paper's "Variations":
// distributed memory).  A rank owns cells [a, b) of the ring and holds them
// with a halo of H >= k * vmax cells on each side, refreshed from its ring
// neighbours before every launch; the launch runs k steps on the buffer and
// writes the owned cells.  Cell j at step t+1 depends on cells j - vmax ..
// j + vmax at step t (a car arriving from behind, the gap ahead), so after k
// steps the owned cells depend on the buffer alone.
//
// The kernel is the list method of the fused grid kernels (grid_warp_steps):
// independent warps take 2048-cell spans of the buffer (an owned tile of
// 2048 - 2H cells with H cells each side), list the span's cars in cell
// order, run the k steps on the list and write back the cars that end in
// the tile's own cells.  The rule-3 draw of a car uses its ring cell, so a
// decomposed road draws exactly what the whole road draws.  Statistics
// count the cars whose cell at the start of a step is owned, so the ranks'
// series add up to the whole road's.
#include <cuda_runtime.h>

#include "nasch.h"
#include "runtime_internal.h"
#include "tile_device.cuh"

namespace nasch {
namespace {

constexpr int kSegWarps = 4;

struct SegmentStep {
    const int8_t *in;      // buffer: cells first - H .. first + owned + H - 1 (mod L)
    int8_t *out;           // same layout; owned part written
    RoadConst rc;
    uint32_t H;            // halo cells per side
    uint32_t owned;        // owned cells
    uint32_t first;        // ring cell of the first owned cell
    uint32_t step0;
    int ksteps;
    uint32_t n_tiles;
    unsigned long long *sum_v;
    unsigned long long *crossings;
};

struct __align__(16) SegWarpSmem {
    int8_t span[kKwBuf];
    uint16_t pos[kKwList];
    uint8_t vel[kKwList];
};

template <Draw D>
__global__ void __launch_bounds__(32 * kSegWarps) grid_segment_kernel(const SegmentStep g)
{
    __shared__ SegWarpSmem s_w[kSegWarps];
    __shared__ unsigned long long s_sum[kMaxFusedSteps];
    __shared__ unsigned long long s_cross[kMaxFusedSteps];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    SegWarpSmem &w = s_w[warp];
    for (int i = threadIdx.x; i < g.ksteps; i += blockDim.x) {
        s_sum[i] = 0ull;
        s_cross[i] = 0ull;
    }
    __syncthreads();
    const uint32_t L = g.rc.L, H = g.H;
    const uint32_t C = kKwSpan - 2u * H;                    // owned cells per tile
    const uint32_t W = g.owned + 2u * H;                    // buffer length
    const uint32_t nw = gridDim.x * (uint32_t)kSegWarps;
    for (uint32_t tile = blockIdx.x * (uint32_t)kSegWarps + warp; tile < g.n_tiles; tile += nw) {
        const uint32_t t0 = tile * C;                       // buffer index of the span's first cell
        const uint32_t own = min(C, g.owned - t0);
        // ring cell of span index 0: first - H + t0 (mod L)
        const uint32_t base = (uint32_t)(((uint64_t)g.first + (uint64_t)L - (uint64_t)(H % L) + (uint64_t)t0) % L);
        // stage the span: 16-byte loads inside the buffer, empty cells past its end
        for (uint32_t c = lane; c < kKwSpan / 16u; c += 32u) {
            const uint32_t i = t0 + 16u * c;
            uint4 q = kEmpty4;
            if (i + 16u <= W) {
                q = *reinterpret_cast<const uint4 *>(g.in + i);
            } else if (i < W) {
                int8_t b[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) b[j] = i + (uint32_t)j < W ? g.in[i + (uint32_t)j] : (int8_t)-1;
                memcpy(&q, b, 16);
            }
            reinterpret_cast<uint4 *>(w.span)[c] = q;
        }
        __syncwarp();
        grid_warp_steps<D>(g.rc, PlainDraws{g.rc, 0}, w.span, WarpList{w.pos, w.vel, kKwList, nullptr, nullptr}, H, own, base,
                           g.step0, g.ksteps, []() {},
                           [&](int s, uint32_t sum, uint32_t cross) {
                               if (sum) atomicAdd(&s_sum[s], (unsigned long long)sum);
                               if (cross) atomicAdd(&s_cross[s], (unsigned long long)cross);
                           });
        for (uint32_t i = lane; i < own; i += 32u)
            if (NASCH_DCHECK(H + t0 + i < W, kDbgSegmentWrite)) g.out[H + t0 + i] = w.span[H + i];
        __syncwarp();
    }
    __syncthreads();
    for (int i = threadIdx.x; i < g.ksteps; i += blockDim.x) {
        if (s_sum[i]) atomicAdd(&g.sum_v[i], s_sum[i]);
        if (s_cross[i]) atomicAdd(&g.crossings[i], s_cross[i]);
    }
}

}  // namespace

// This unit's debug word (zero in release builds).
NASCH_DEBUG_READER(debug_word_segment)

}  // namespace nasch

using namespace nasch;

extern "C" int nasch_segment_run(const int8_t *seg_in_dev, int8_t *seg_out_dev, int64_t owned, int32_t halo,
                                 int64_t first_cell, int64_t L, int32_t vmax, double p, uint64_t seed,
                                 uint32_t road_id, uint64_t step0, int32_t k, uint64_t *sum_v_dev,
                                 uint64_t *crossings_dev, void *stream)
{
    clear_error();
    if (L < 1 || L > (int64_t(1) << 31)) return fail(NASCH_EINVAL, "L=%lld outside 1..2^31", (long long)L);
    if (vmax < 0 || vmax > 127) return fail(NASCH_EINVAL, "vmax=%d outside 0..127", vmax);
    if (!(p >= 0.0 && p <= 1.0)) return fail(NASCH_EINVAL, "p=%g outside [0, 1]", p);
    if (k < 1 || k > kMaxFusedSteps) return fail(NASCH_EINVAL, "k=%d outside 1..%d", k, kMaxFusedSteps);
    if (owned < 1 || owned > L) return fail(NASCH_EINVAL, "owned=%lld outside 1..L", (long long)owned);
    if (first_cell < 0 || first_cell >= L) return fail(NASCH_EINVAL, "first_cell=%lld outside 0..L-1", (long long)first_cell);
    if (halo < 0 || halo % 16 != 0 || halo > (int32_t)kKwMaxHalo || (int64_t)halo < (int64_t)k * vmax)
        return fail(NASCH_EINVAL, "halo=%d must be a multiple of 16 with k*vmax=%d <= halo <= %u", halo, k * vmax,
                    kKwMaxHalo);
    if (owned + 2 * (int64_t)halo > (int64_t(1) << 31))
        return fail(NASCH_EINVAL, "buffer of %lld cells too long", (long long)(owned + 2 * (int64_t)halo));
    if (!seg_in_dev || !seg_out_dev || !sum_v_dev || !crossings_dev) return fail(NASCH_EINVAL, "NULL buffer");
    if ((reinterpret_cast<uintptr_t>(seg_in_dev) | reinterpret_cast<uintptr_t>(seg_out_dev)) % 16 != 0)
        return fail(NASCH_EINVAL, "segment buffers must be 16-byte aligned");
    const char *ib = reinterpret_cast<const char *>(seg_in_dev), *ob = reinterpret_cast<const char *>(seg_out_dev);
    const int64_t len = owned + 2 * (int64_t)halo;
    if (ib < ob + len && ob < ib + len) return fail(NASCH_EINVAL, "input and output buffers overlap");
    SegmentStep g;
    g.in = seg_in_dev;
    g.out = seg_out_dev;
    g.rc.L = (uint32_t)L;
    g.rc.vmax = (uint32_t)vmax;
    g.rc.thr = slow_threshold(p);
    g.rc.key0 = (uint32_t)seed;
    g.rc.key1 = (uint32_t)(seed >> 32);
    g.rc.road = road_id;
    g.H = (uint32_t)halo;
    g.owned = (uint32_t)owned;
    g.first = (uint32_t)first_cell;
    g.step0 = (uint32_t)step0;
    g.ksteps = k;
    const uint32_t C = kKwSpan - 2u * (uint32_t)halo;
    g.n_tiles = (uint32_t)((owned + C - 1) / C);
    g.sum_v = reinterpret_cast<unsigned long long *>(sum_v_dev);
    g.crossings = reinterpret_cast<unsigned long long *>(crossings_dev);
    int device = 0, sms = 1;
    int st = device_info(&device, &sms);
    if (st) return st;
    const uint32_t need = (g.n_tiles + kSegWarps - 1) / kSegWarps;
    const uint32_t grid = need < (uint32_t)sms * 8u ? need : (uint32_t)sms * 8u;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    switch (draw_mode(g.rc.thr)) {
    case Draw::kNever: grid_segment_kernel<Draw::kNever><<<grid, 32 * kSegWarps, 0, s>>>(g); break;
    case Draw::kAlways: grid_segment_kernel<Draw::kAlways><<<grid, 32 * kSegWarps, 0, s>>>(g); break;
    default: grid_segment_kernel<Draw::kPhilox><<<grid, 32 * kSegWarps, 0, s>>>(g); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "segment kernel");
#ifdef NASCH_DEBUG
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "segment kernel");
    if (const unsigned int w = debug_word_segment())
        return fail(NASCH_EINVAL, "debug check failed in the segment kernel (sites 0x%x)", w);
#endif
    return NASCH_OK;
}
