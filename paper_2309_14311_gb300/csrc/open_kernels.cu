// Open road (the handout's "Variations": other boundary conditions): cells
// 0..L-1 with an entry before cell 0 and an exit after cell L-1, no ring.
// The reading, the same as the oracle's:
//   - the exit is open at step t with probability beta; the leading car then
//     sees an unbounded road, else the road's end; a car whose move passes
//     cell L-1 leaves the road (counted in crossings);
//   - rules 1-4 otherwise as on the ring, from start-of-step positions;
//   - after the moves, if cell 0 is empty, a car enters there at rest with
//     probability alpha.
// The exit and entry draws of a step are decided on the host (Philox tags 2
// and 3); the kernel gets the two outcomes.
//
// One step per launch.  For vmax <= 16 the ring's one-step kernel runs the
// open road (grid_k1_kernel in its open form: bulk copies, stepped in
// place).  For larger vmax this kernel does: every warp works alone on
// tiles of kKwSpan - 2H cells, H = round_up(vmax, 16); it stages the tile
// with H cells on each side (cells off the road read as empty; a closed
// exit as a car standing on cell L), steps the span by the list method
// (grid_warp_steps, as the ring's fused kernels), lets a car enter on cell
// 0, and writes the tile.
#include <atomic>

#include "road_output.h"
#include "tile_device.cuh"

namespace nasch {
namespace {

constexpr int kOpenWarps = 4;   // warps per block
constexpr int kMaxDevices = 64;

struct __align__(16) OpenWarpSmem {
    int8_t span[kKwBuf];
    uint16_t pos[kKwList];
    uint8_t vel[kKwList];
};

template <Draw D>
__global__ void __launch_bounds__(32 * kOpenWarps) grid_open_kernel(const GridStep g, const uint32_t H,
                                                                    const uint32_t n_tiles, const int exit_open,
                                                                    const int entry)
{
    __shared__ OpenWarpSmem s_w[kOpenWarps];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    OpenWarpSmem &w = s_w[warp];
    const uint32_t L = g.rc.L;
    const uint32_t C = kKwSpan - 2u * H;
    uint32_t tsum = 0, tcross = 0;
    for (uint32_t tile = blockIdx.x * (uint32_t)kOpenWarps + warp; tile < n_tiles;
         tile += gridDim.x * (uint32_t)kOpenWarps) {
        const uint32_t t0 = tile * C;
        const uint32_t own = min(C, L - t0);
        const int64_t first = (int64_t)t0 - (int64_t)H;   // road cell of span index 0 (negative: before the road)
        const uint32_t base = (uint32_t)first;             // the same modulo 2^32, as the step code takes it
        if (first >= 0 && first + (int64_t)kKwSpan <= (int64_t)L) {
            const uint4 *src = reinterpret_cast<const uint4 *>(g.c_in + first);
#pragma unroll
            for (uint32_t k = 0; k < kKwSpan / 512u; ++k)
                reinterpret_cast<uint4 *>(w.span)[lane + 32u * k] = src[lane + 32u * k];
        } else {
            for (uint32_t i = lane; i < kKwSpan; i += 32u) {
                const int64_t c = first + (int64_t)i;
                w.span[i] = (c >= 0 && c < (int64_t)L) ? g.c_in[c] : (int8_t)-1;
            }
        }
        __syncwarp();
        // a closed exit: a car standing on cell L, seen by the car behind it
        const int64_t end = (int64_t)L - first;
        if (!exit_open && lane == 0 && end >= 0 && end < (int64_t)kKwSpan) w.span[end] = 0;
        __syncwarp();
        grid_warp_steps<D>(g.rc, PlainDraws{g.rc, 0}, w.span, WarpList{w.pos, w.vel, kKwList, nullptr, nullptr}, H, own,
                           base, g.step0, 1, []() {},
                           [&](int, uint32_t sum, uint32_t cross) {
                               tsum += sum;
                               tcross += cross;
                           });
        if (tile == 0 && lane == 0 && entry && w.span[H] < 0) w.span[H] = 0;   // a car enters at rest
        __syncwarp();
        if (own == C) {
            const uint4 *f4 = reinterpret_cast<const uint4 *>(w.span + H);
            uint4 *dst = reinterpret_cast<uint4 *>(g.c_out + t0);
            for (uint32_t c = lane; c < C / 16u; c += 32u) dst[c] = f4[c];
        } else {
            for (uint32_t i = lane; i < own; i += 32u) g.c_out[t0 + i] = w.span[H + i];
        }
        __syncwarp();
    }
    if (lane == 0) {
        if (tsum) atomicAdd(&g.sum_v[0], (unsigned long long)tsum);
        if (tcross) atomicAdd(&g.crossings[0], (unsigned long long)tcross);
    }
}

template <Draw D>
cudaError_t launch_open_variant(const GridStep &g, uint32_t H, uint32_t n_tiles, bool exit_open, bool entry,
                                cudaStream_t s)
{
    static std::atomic<int> per_sm[kMaxDevices];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    int n = per_sm[dev].load();
    if (n == 0) {
        int sms = 0, b = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, grid_open_kernel<D>, 32 * kOpenWarps, 0);
        if (e != cudaSuccess) return e;
        n = sms * (b > 0 ? b : 1);
        per_sm[dev].store(n);
    }
    const uint32_t need = (n_tiles + (uint32_t)kOpenWarps - 1u) / (uint32_t)kOpenWarps;
    const int grid = (int)((uint32_t)n < need ? (uint32_t)n : need);
    grid_open_kernel<D><<<grid, 32 * kOpenWarps, 0, s>>>(g, H, n_tiles, exit_open ? 1 : 0, entry ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_grid_open(const GridStep &g, bool exit_open, bool entry, cudaStream_t s)
{
    if (g.ksteps != 1 || g.rc.vmax > 127u || g.rc.L == 0) return cudaErrorInvalidValue;
    if (g.rc.vmax <= 16u) return launch_grid_k1_open(g, exit_open, entry, s);   // bulk copies, stepped in place
    const uint32_t H = grid_halo(1, g.rc.vmax) < 16u ? 16u : grid_halo(1, g.rc.vmax);
    const uint32_t C = kKwSpan - 2u * H;
    const uint32_t n_tiles = (g.rc.L + C - 1u) / C;
    if (g.rc.thr == 0) return launch_open_variant<Draw::kNever>(g, H, n_tiles, exit_open, entry, s);
    if (g.rc.thr > 0xFFFFFFFFull) return launch_open_variant<Draw::kAlways>(g, H, n_tiles, exit_open, entry, s);
    return launch_open_variant<Draw::kPhilox>(g, H, n_tiles, exit_open, entry, s);
}

// This unit's debug word (zero in release builds).
NASCH_DEBUG_READER(debug_word_open)

}  // namespace nasch
