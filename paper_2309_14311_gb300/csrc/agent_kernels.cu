// Agent-based NaSch step kernels: positions int32 x[N], velocities uint8 v[N],
// cars in cyclic order ("Concepts Covered": the agent-based representation;
// Handout, model section rules 1-4).
//
// Tiled kernel.  A tile is 2048 consecutive cars held in registers, 8 per
// thread.  Car i's next state depends on car i+1's position only, so after
// k fused steps the first 2048 - round_up(k, 8) cars of the tile are exact
// and the rest (the look-ahead halo) is discarded; tiles overlap by the halo.
// The leader of a thread's last car comes from the next lane by a warp
// shuffle, or across warps through shared memory.  The last tile's halo
// wraps to cars 0, 1, ... and the gap is taken modulo L, so the ring needs
// no special case.  Statistics of the owned cars are reduced per warp, then
// per block in shared memory, and added to the per-step series once per
// block at the end (a persistent grid of a few blocks per SM).
//
// Ring kernel.  For N <= 8192 one block holds the whole ring and runs any
// number of steps in one launch, with the exact ring neighbour and no halo.
#include "kernels.h"

namespace nasch {
namespace {

template <int R>
__device__ __forceinline__ void load_cars_vec(const int32_t *__restrict__ x_in,
                                              const uint8_t *__restrict__ v_in, uint32_t g,
                                              uint32_t (&x)[R], uint32_t (&v)[R])
{
    static_assert(R == 8, "vector path assumes 8 cars per thread");
    const int4 xa = __ldg(reinterpret_cast<const int4 *>(x_in + g));
    const int4 xb = __ldg(reinterpret_cast<const int4 *>(x_in + g + 4));
    const uint2 vv = __ldg(reinterpret_cast<const uint2 *>(v_in + g));
    x[0] = (uint32_t)xa.x; x[1] = (uint32_t)xa.y; x[2] = (uint32_t)xa.z; x[3] = (uint32_t)xa.w;
    x[4] = (uint32_t)xb.x; x[5] = (uint32_t)xb.y; x[6] = (uint32_t)xb.z; x[7] = (uint32_t)xb.w;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        v[r] = (vv.x >> (8 * r)) & 0xFFu;
        v[r + 4] = (vv.y >> (8 * r)) & 0xFFu;
    }
}

template <int R>
__device__ __forceinline__ void store_cars_vec(int32_t *__restrict__ x_out,
                                               uint8_t *__restrict__ v_out, uint32_t g,
                                               const uint32_t (&x)[R], const uint32_t (&v)[R])
{
    static_assert(R == 8, "vector path assumes 8 cars per thread");
    reinterpret_cast<int4 *>(x_out + g)[0] = make_int4((int)x[0], (int)x[1], (int)x[2], (int)x[3]);
    reinterpret_cast<int4 *>(x_out + g)[1] = make_int4((int)x[4], (int)x[5], (int)x[6], (int)x[7]);
    uint2 vv;
    vv.x = v[0] | (v[1] << 8) | (v[2] << 16) | (v[3] << 24);
    vv.y = v[4] | (v[5] << 8) | (v[6] << 16) | (v[7] << 24);
    *reinterpret_cast<uint2 *>(v_out + g) = vv;
}

template <int R, int NT>
__global__ void __launch_bounds__(NT) agent_tiled_kernel(const AgentStep a, const uint32_t owned,
                                                         const uint32_t n_tiles)
{
    constexpr int kWarps = NT / 32;
    constexpr uint32_t kSpan = (uint32_t)NT * R;
    __shared__ uint32_t s_first[2][kWarps];
    __shared__ unsigned long long s_sum[kMaxFusedSteps];
    __shared__ unsigned long long s_cross[kMaxFusedSteps];

    for (int i = threadIdx.x; i < a.ksteps; i += NT) {
        s_sum[i] = 0ull;
        s_cross[i] = 0ull;
    }
    __syncthreads();

    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = threadIdx.x >> 5;
    const uint32_t e0 = threadIdx.x * R;   // first car of this thread within the tile
    const uint32_t N = a.N;
    const RoadConst rc = a.rc;
    uint32_t phase = 0;

    for (uint32_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const uint32_t t0 = tile * owned;
        uint32_t x[R], v[R];
        if (t0 + kSpan <= N) {
            load_cars_vec<R>(a.x_in, a.v_in, t0 + e0, x, v);
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const uint32_t g = (t0 + e0 + (uint32_t)r) % N;   // halo wraps round the ring
                x[r] = (uint32_t)a.x_in[g];
                v[r] = a.v_in[g];
            }
        }

        for (int s = 0; s < a.ksteps; ++s, ++phase) {
            const uint32_t step = a.step0 + (uint32_t)s;
            const uint32_t ph = phase & 1u;
            if (lane == 0) s_first[ph][warp] = x[0];
            __syncthreads();
            uint32_t lead_last = __shfl_down_sync(0xFFFFFFFFu, x[0], 1);
            if (lane == 31) lead_last = (warp + 1 < (uint32_t)kWarps) ? s_first[ph][warp + 1] : x[R - 1];

            uint32_t tsum = 0, tcross = 0;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const uint32_t xi = x[r];
                const uint32_t lead = (r + 1 < R) ? x[r + 1] : lead_last;   // start-of-step position
                const uint32_t vel = new_velocity(rc, v[r], agent_gap(xi, lead, rc.L), xi, step);
                uint32_t nx = xi + vel;
                const bool wrap = nx >= rc.L;
                if (wrap) nx -= rc.L;
                x[r] = nx;
                v[r] = vel;
                const bool own = (e0 + (uint32_t)r < owned) && (t0 + e0 + (uint32_t)r < N);
                tsum += own ? vel : 0u;
                tcross += (own && wrap) ? 1u : 0u;
            }
            tsum = __reduce_add_sync(0xFFFFFFFFu, tsum);
            tcross = __reduce_add_sync(0xFFFFFFFFu, tcross);
            if (lane == 0 && (tsum | tcross)) {
                atomicAdd(&s_sum[s], (unsigned long long)tsum);
                atomicAdd(&s_cross[s], (unsigned long long)tcross);
            }
        }

        const uint32_t own_end = min(t0 + owned, N);
        if (e0 < owned) {
            if (t0 + e0 + R <= own_end) {
                store_cars_vec<R>(a.x_out, a.v_out, t0 + e0, x, v);
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const uint32_t g = t0 + e0 + (uint32_t)r;
                    if (g < own_end) {
                        a.x_out[g] = (int32_t)x[r];
                        a.v_out[g] = (uint8_t)v[r];
                    }
                }
            }
        }
    }

    __syncthreads();
    for (int i = threadIdx.x; i < a.ksteps; i += NT) {
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
            &n, agent_tiled_kernel<kAgentCarsPerThread, kAgentThreads>, kAgentThreads, 0) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

cudaError_t launch_agent_tiled(const AgentStep &a, int blocks, cudaStream_t s)
{
    if (a.N == 0 || a.ksteps <= 0) return cudaSuccess;
    if (a.ksteps > kMaxFusedSteps) return cudaErrorInvalidValue;
    const uint32_t owned = agent_tile_owned(a.ksteps);
    const uint32_t n_tiles = (a.N + owned - 1) / owned;
    const int grid = (int)((uint32_t)blocks < n_tiles ? (uint32_t)blocks : n_tiles);
    agent_tiled_kernel<kAgentCarsPerThread, kAgentThreads><<<grid, kAgentThreads, 0, s>>>(a, owned, n_tiles);
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
