// Agent-based NaSch step kernels: positions int32 x[N], velocities uint8 v[N],
// cars in cyclic order ("Concepts Covered": the agent-based representation;
// Handout, model section rules 1-4).
//
// Tiled kernel.  A warp-tile is 512 consecutive cars held in registers, 16
// per lane, and every warp works alone (no block barrier in the step loop).
// Car i's next state depends on car i+1's position only, so after k fused
// steps the first 512 - round_up(k, 16) cars of the tile are exact and the
// rest (the look-ahead halo) is discarded; warp-tiles overlap by the halo.
// The leader of a lane's last car comes from the next lane by a warp
// shuffle.  The last tile's halo wraps to cars 0, 1, ... and the gap is
// taken modulo L, so the ring needs no special case.  The rule-3 draw is
// computed for every car without a branch, so the 16 Philox chains of a
// lane interleave; p = 0 and p = 1 launch variants without draws.
// Statistics of the owned cars are reduced per warp, then per block in
// shared memory, and added to the per-step series once per block at the end
// (a persistent grid of a few blocks per SM).
//
// Ring kernel.  For N <= 8192 one block holds the whole ring and runs any
// number of steps in one launch, with the exact ring neighbour and no halo.
#include "kernels.h"

namespace nasch {
namespace {

// R consecutive cars starting at car g (g a multiple of 8): x by 16-byte
// loads, v by 8-byte loads.
template <int R>
__device__ __forceinline__ void load_cars_vec(const int32_t *__restrict__ x_in,
                                              const uint8_t *__restrict__ v_in, uint32_t g,
                                              uint32_t (&x)[R], uint32_t (&v)[R])
{
    static_assert(R % 8 == 0, "vector path loads 8 cars at a time");
#pragma unroll
    for (int q = 0; q < R / 4; ++q) {
        const int4 xq = __ldg(reinterpret_cast<const int4 *>(x_in + g) + q);
        x[4 * q] = (uint32_t)xq.x;
        x[4 * q + 1] = (uint32_t)xq.y;
        x[4 * q + 2] = (uint32_t)xq.z;
        x[4 * q + 3] = (uint32_t)xq.w;
    }
#pragma unroll
    for (int q = 0; q < R / 8; ++q) {
        const uint2 vv = __ldg(reinterpret_cast<const uint2 *>(v_in + g) + q);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            v[8 * q + r] = (vv.x >> (8 * r)) & 0xFFu;
            v[8 * q + r + 4] = (vv.y >> (8 * r)) & 0xFFu;
        }
    }
}

template <int R>
__device__ __forceinline__ void store_cars_vec(int32_t *__restrict__ x_out,
                                               uint8_t *__restrict__ v_out, uint32_t g,
                                               const uint32_t (&x)[R], const uint32_t (&v)[R])
{
    static_assert(R % 8 == 0, "vector path stores 8 cars at a time");
#pragma unroll
    for (int q = 0; q < R / 4; ++q)
        reinterpret_cast<int4 *>(x_out + g)[q] =
            make_int4((int)x[4 * q], (int)x[4 * q + 1], (int)x[4 * q + 2], (int)x[4 * q + 3]);
#pragma unroll
    for (int q = 0; q < R / 8; ++q) {
        uint2 vv;
        vv.x = v[8 * q] | (v[8 * q + 1] << 8) | (v[8 * q + 2] << 16) | (v[8 * q + 3] << 24);
        vv.y = v[8 * q + 4] | (v[8 * q + 5] << 8) | (v[8 * q + 6] << 16) | (v[8 * q + 7] << 24);
        reinterpret_cast<uint2 *>(v_out + g)[q] = vv;
    }
}

// How rule 3 is decided for a whole launch: p = 0 never slows down, p = 1
// always does (no draw needed), anything else draws.
enum class Draw { kNever, kAlways, kPhilox };

// One warp-tile: 32 lanes x R consecutive cars in registers.  kFull: the
// tile lies inside [0, N) and every owned car of a lane is owned (lanes are
// either all-owned or all-halo), so no per-car ownership test is needed.
template <int R, Draw D, bool kFull>
__device__ __forceinline__ void agent_warp_tile(const AgentStep &a, uint32_t t0, uint32_t owned,
                                                unsigned long long *s_sum, unsigned long long *s_cross)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t e0 = lane * R;
    const uint32_t N = a.N;
    const uint32_t L = a.rc.L;
    const uint32_t Lm1 = L - 1u;
    const uint32_t vmax = a.rc.vmax;
    const uint32_t thr = (uint32_t)a.rc.thr;
    uint32_t x[R], v[R];
    if (kFull) {
        load_cars_vec<R>(a.x_in, a.v_in, t0 + e0, x, v);
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint32_t g = (t0 + e0 + (uint32_t)r) % N;   // halo wraps round the ring
            x[r] = (uint32_t)a.x_in[g];
            v[r] = a.v_in[g];
        }
    }
    // cars of this lane that the tile owns (statistics and write-back)
    const uint32_t own_end = min(owned, N - t0);
    const uint32_t n_own = e0 >= own_end ? 0u : min((uint32_t)R, own_end - e0);

    for (int s = 0; s < a.ksteps; ++s) {
        const uint32_t step = a.step0 + (uint32_t)s;
        // leader of the lane's last car: the next lane's first car (start-of-step)
        const uint32_t lead_last = __shfl_down_sync(0xFFFFFFFFu, x[0], 1);
        uint32_t tsum = 0, tcross = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint32_t xi = x[r];
            const uint32_t lead = (r + 1 < R) ? x[r + 1] : lead_last;
            // empty cells ahead on the ring: (lead - x - 1) mod L, or L - 1 if
            // the car is its own leader; as the smaller of two unsigned values
            const uint32_t d = lead - xi;
            const uint32_t gap = min(d - 1u, d + Lm1);
            uint32_t vel = min(min(v[r] + 1u, vmax), gap);            // rules 1, 2
            if (D == Draw::kAlways) {
                vel -= vel > 0u ? 1u : 0u;                              // rule 3, p = 1
            } else if (D == Draw::kPhilox) {
                const uint32_t u = philox_word0(xi, step, a.rc.road, kTagSlowdown, a.rc.key0, a.rc.key1);
                vel -= (vel > 0u && u < thr) ? 1u : 0u;                 // rule 3
            }
            uint32_t nx = xi + vel;                                     // rule 4
            const bool wrap = nx >= L;
            nx = wrap ? nx - L : nx;
            x[r] = nx;
            v[r] = vel;
            if (kFull || (uint32_t)r < n_own) {
                tsum += vel;
                tcross += wrap ? 1u : 0u;
            }
        }
        if (kFull && n_own == 0u) tsum = tcross = 0u;   // halo lanes
        tsum = __reduce_add_sync(0xFFFFFFFFu, tsum);
        tcross = __reduce_add_sync(0xFFFFFFFFu, tcross);
        if (lane == 0 && (tsum | tcross)) {
            atomicAdd(&s_sum[s], (unsigned long long)tsum);
            atomicAdd(&s_cross[s], (unsigned long long)tcross);
        }
    }

    if (n_own == (uint32_t)R) {
        store_cars_vec<R>(a.x_out, a.v_out, t0 + e0, x, v);
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if ((uint32_t)r < n_own) {
                a.x_out[t0 + e0 + r] = (int32_t)x[r];
                a.v_out[t0 + e0 + r] = (uint8_t)v[r];
            }
        }
    }
}

// Persistent grid of independent warps; warp w takes warp-tiles w, w + W, ...
template <int R, Draw D>
__global__ void __launch_bounds__(kAgentThreads) agent_tiled_kernel(const AgentStep a, const uint32_t owned,
                                                                    const uint32_t n_tiles)
{
    __shared__ unsigned long long s_sum[kMaxFusedSteps];
    __shared__ unsigned long long s_cross[kMaxFusedSteps];
    for (int i = threadIdx.x; i < a.ksteps; i += blockDim.x) {
        s_sum[i] = 0ull;
        s_cross[i] = 0ull;
    }
    __syncthreads();
    constexpr uint32_t kSpan = 32u * R;
    const uint32_t warps_per_block = blockDim.x >> 5;
    const uint32_t n_warps = gridDim.x * warps_per_block;
    for (uint32_t tile = blockIdx.x * warps_per_block + (threadIdx.x >> 5); tile < n_tiles; tile += n_warps) {
        const uint32_t t0 = tile * owned;
        if (t0 + kSpan <= a.N)
            agent_warp_tile<R, D, true>(a, t0, owned, s_sum, s_cross);
        else
            agent_warp_tile<R, D, false>(a, t0, owned, s_sum, s_cross);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < a.ksteps; i += blockDim.x) {
        if (s_sum[i]) atomicAdd(&a.sum_v[i], s_sum[i]);
        if (s_cross[i]) atomicAdd(&a.crossings[i], s_cross[i]);
    }
}

// Whole ring in one block: thread t holds cars [t*R, t*R + R) of the N cars;
// the car after thread t's last car is thread t+1's first, or car 0.
template <int R>
__global__ void __launch_bounds__(1024) agent_ring_kernel(const AgentStep a)
{
    __shared__ uint32_t s_first[2][1024];
    __shared__ uint32_t s_psum[2][32];
    __shared__ uint32_t s_pcross[2][32];

    const uint32_t N = a.N;
    const uint32_t tid = threadIdx.x;
    const uint32_t lane = tid & 31u, warp = tid >> 5;
    const uint32_t nwarps = blockDim.x >> 5;
    const uint32_t e0 = tid * R;
    const int cnt = e0 < N ? (int)min((uint32_t)R, N - e0) : 0;
    const uint32_t next_owner = (e0 + R < N) ? tid + 1 : 0u;
    const RoadConst rc = a.rc;

    uint32_t x[R], v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        x[r] = r < cnt ? (uint32_t)a.x_in[e0 + r] : 0u;
        v[r] = r < cnt ? (uint32_t)a.v_in[e0 + r] : 0u;
    }

    for (int s = 0; s < a.ksteps; ++s) {
        const uint32_t ph = (uint32_t)s & 1u;
        const uint32_t step = a.step0 + (uint32_t)s;
        if (cnt > 0) s_first[ph][tid] = x[0];
        __syncthreads();
        if (tid == 0 && s > 0) {
            unsigned long long sv = 0, cr = 0;
            for (uint32_t w = 0; w < nwarps; ++w) {
                sv += s_psum[ph ^ 1u][w];
                cr += s_pcross[ph ^ 1u][w];
            }
            a.sum_v[s - 1] = sv;
            a.crossings[s - 1] = cr;
        }
        const uint32_t lead_last = s_first[ph][next_owner];
        uint32_t tsum = 0, tcross = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (r < cnt) {
                const uint32_t xi = x[r];
                const uint32_t lead = (r + 1 < cnt) ? x[r + 1] : lead_last;
                const uint32_t vel = new_velocity(rc, v[r], agent_gap(xi, lead, rc.L), xi, step);
                uint32_t nx = xi + vel;
                const bool wrap = nx >= rc.L;
                if (wrap) nx -= rc.L;
                x[r] = nx;
                v[r] = vel;
                tsum += vel;
                tcross += wrap ? 1u : 0u;
            }
        }
        tsum = __reduce_add_sync(0xFFFFFFFFu, tsum);
        tcross = __reduce_add_sync(0xFFFFFFFFu, tcross);
        if (lane == 0) {
            s_psum[ph][warp] = tsum;
            s_pcross[ph][warp] = tcross;
        }
    }
    __syncthreads();
    if (tid == 0 && a.ksteps > 0) {
        const uint32_t ph = (uint32_t)(a.ksteps - 1) & 1u;
        unsigned long long sv = 0, cr = 0;
        for (uint32_t w = 0; w < nwarps; ++w) {
            sv += s_psum[ph][w];
            cr += s_pcross[ph][w];
        }
        a.sum_v[a.ksteps - 1] = sv;
        a.crossings[a.ksteps - 1] = cr;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (r < cnt) {
            a.x_out[e0 + r] = (int32_t)x[r];
            a.v_out[e0 + r] = (uint8_t)v[r];
        }
    }
}

__global__ void scatter_agent_to_grid_kernel(const int32_t *__restrict__ x,
                                             const uint8_t *__restrict__ v, uint32_t N,
                                             int8_t *__restrict__ cells)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        cells[x[i]] = (int8_t)v[i];
}

__global__ void philox_test_kernel(const uint32_t *__restrict__ ctr, uint32_t k0, uint32_t k1,
                                   uint32_t *__restrict__ out, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const Words4 w = philox4x32_10(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3], k0, k1);
        out[4 * i] = w.w0;
        out[4 * i + 1] = w.w1;
        out[4 * i + 2] = w.w2;
        out[4 * i + 3] = w.w3;
    }
}

}  // namespace

int agent_tiled_blocks_per_sm()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &n, agent_tiled_kernel<kAgentCarsPerThread, Draw::kPhilox>, kAgentThreads, 0) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

template <int R>
static void launch_agent_r(const AgentStep &a, uint32_t owned, uint32_t n_tiles, int grid, cudaStream_t s)
{
    if (a.rc.thr == 0)
        agent_tiled_kernel<R, Draw::kNever><<<grid, kAgentThreads, 0, s>>>(a, owned, n_tiles);
    else if (a.rc.thr > 0xFFFFFFFFull)
        agent_tiled_kernel<R, Draw::kAlways><<<grid, kAgentThreads, 0, s>>>(a, owned, n_tiles);
    else
        agent_tiled_kernel<R, Draw::kPhilox><<<grid, kAgentThreads, 0, s>>>(a, owned, n_tiles);
}

cudaError_t launch_agent_tiled(const AgentStep &a, int span, int blocks, cudaStream_t s)
{
    if (a.N == 0 || a.ksteps <= 0) return cudaSuccess;
    if (a.ksteps > kMaxFusedSteps) return cudaErrorInvalidValue;
    if (span != kAgentTileSpan && span != kAgentTileSpanSmall) return cudaErrorInvalidValue;
    const uint32_t owned = agent_tile_owned(a.ksteps, span);
    const uint32_t n_tiles = (a.N + owned - 1) / owned;
    const uint32_t warps_per_block = kAgentThreads / 32;
    const uint32_t need = (n_tiles + warps_per_block - 1) / warps_per_block;
    const int grid = (int)((uint32_t)blocks < need ? (uint32_t)blocks : need);
    if (span == kAgentTileSpan)
        launch_agent_r<kAgentCarsPerThread>(a, owned, n_tiles, grid, s);
    else
        launch_agent_r<8>(a, owned, n_tiles, grid, s);
    return cudaGetLastError();
}

cudaError_t launch_agent_ring(const AgentStep &a, cudaStream_t s)
{
    if (a.ksteps <= 0) return cudaSuccess;
    if (a.N == 0 || a.N > (uint32_t)kAgentRingMaxCars) return cudaErrorInvalidValue;
    // Fewest cars per thread that fit in 1024 threads, so the step's dependency
    // chain per thread stays short.
    int R = 1;
    while ((uint32_t)R * 1024u < a.N) R *= 2;
    const uint32_t threads_needed = (a.N + R - 1) / R;
    const int threads = (int)((threads_needed + 31u) / 32u * 32u);
    switch (R) {
    case 1: agent_ring_kernel<1><<<1, threads, 0, s>>>(a); break;
    case 2: agent_ring_kernel<2><<<1, threads, 0, s>>>(a); break;
    case 4: agent_ring_kernel<4><<<1, threads, 0, s>>>(a); break;
    default: agent_ring_kernel<8><<<1, threads, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_scatter_agent_to_grid(const int32_t *x, const uint8_t *v, uint32_t N, int8_t *cells,
                                         cudaStream_t s)
{
    if (N == 0) return cudaSuccess;
    const uint32_t threads = 256;
    uint32_t blocks = (N + threads - 1) / threads;
    if (blocks > 65535u * 8u) blocks = 65535u * 8u;
    scatter_agent_to_grid_kernel<<<blocks, threads, 0, s>>>(x, v, N, cells);
    return cudaGetLastError();
}

cudaError_t launch_philox_test(const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out, int64_t n,
                               cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    philox_test_kernel<<<(int)blocks, 256, 0, s>>>(ctr, k0, k1, out, n);
    return cudaGetLastError();
}

}  // namespace nasch
