// Agent-based NaSch step kernels: positions int32 x[N], velocities uint8 v[N],
// cars in cyclic order ("Concepts Covered": the agent-based representation;
// Handout, model section rules 1-4).
//
// Tiled kernel.  A warp-tile is 512 consecutive cars held in registers, 16
// per lane, and every warp works alone (no block barrier in the step loop).
// A tile that cannot reach cell L-1 within the launch (all but the few
// near the ring's wrap point) steps without modular cell arithmetic.
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
#include "tile_device.cuh"

namespace nasch {
namespace {

// Persistent grid of independent warps; warp w takes warp-tiles w, w + W, ...
// Launches of at least kAgentDeepSteps steps (kMinBlocks = kAgentBlocksPerSm)
// step interior tiles in the carried form, shallower ones in plain cell order.
template <int R, Draw D, int kMinBlocks>
__global__ void __launch_bounds__(kAgentThreads, kMinBlocks) agent_tiled_kernel(const AgentStep a,
                                                                                const uint32_t owned,
                                                                                const uint32_t n_tiles)
{
    constexpr bool kCarry = kMinBlocks == kAgentBlocksPerSm;
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
            agent_warp_tile<R, D, true, kCarry>(a, t0, owned, s_sum, s_cross);
        else
            agent_warp_tile<R, D, false, kCarry>(a, t0, owned, s_sum, s_cross);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < a.ksteps; i += blockDim.x) {
        if (s_sum[i]) atomicAdd(&a.sum_v[i], s_sum[i]);
        if (s_cross[i]) atomicAdd(&a.crossings[i], s_cross[i]);
    }
}

// Whole ring in one block (N <= 1024 * R).
template <int R>
__global__ void __launch_bounds__(1024) agent_ring_kernel(const AgentStep a)
{
    __shared__ uint32_t s_first[2 * 1024];
    __shared__ uint32_t s_psum[2 * 32];
    __shared__ uint32_t s_pcross[2 * 32];
    agent_ring_steps<R>(a.x_in, a.v_in, a.x_out, a.v_out, a.N, a.rc, a.step0, a.ksteps, a.sum_v, a.crossings,
                        s_first, s_psum, s_pcross);
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

template <int kMinBlocks>
static int occupancy_of()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &n, agent_tiled_kernel<kAgentCarsPerThread, Draw::kPhilox, kMinBlocks>, kAgentThreads, 0) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

int agent_tiled_blocks_per_sm(int ksteps)
{
    static const int deep = occupancy_of<kAgentBlocksPerSm>();
    static const int shallow = occupancy_of<kAgentBlocksPerSmShallow>();
    return ksteps >= kAgentDeepSteps ? deep : shallow;
}

template <int R, int kMinBlocks>
static void launch_agent_r(const AgentStep &a, uint32_t owned, uint32_t n_tiles, int grid, cudaStream_t s)
{
    if (a.rc.thr == 0)
        agent_tiled_kernel<R, Draw::kNever, kMinBlocks><<<grid, kAgentThreads, 0, s>>>(a, owned, n_tiles);
    else if (a.rc.thr > 0xFFFFFFFFull)
        agent_tiled_kernel<R, Draw::kAlways, kMinBlocks><<<grid, kAgentThreads, 0, s>>>(a, owned, n_tiles);
    else
        agent_tiled_kernel<R, Draw::kPhilox, kMinBlocks><<<grid, kAgentThreads, 0, s>>>(a, owned, n_tiles);
}

cudaError_t launch_agent_tiled(const AgentStep &a, int span, int sms, cudaStream_t s)
{
    if (a.N == 0 || a.ksteps <= 0) return cudaSuccess;
    if (a.ksteps > kMaxFusedSteps) return cudaErrorInvalidValue;
    if (span != kAgentTileSpan && span != kAgentTileSpanSmall) return cudaErrorInvalidValue;
    const uint32_t owned = agent_tile_owned(a.ksteps, span);
    const uint32_t n_tiles = (a.N + owned - 1) / owned;
    const uint32_t warps_per_block = kAgentThreads / 32;
    const uint32_t need = (n_tiles + warps_per_block - 1) / warps_per_block;
    const uint32_t blocks = (uint32_t)sms * (uint32_t)agent_tiled_blocks_per_sm(a.ksteps);
    const int grid = (int)(blocks < need ? blocks : need);
    const bool deep = a.ksteps >= kAgentDeepSteps;
    if (span == kAgentTileSpan) {
        if (deep) launch_agent_r<kAgentCarsPerThread, kAgentBlocksPerSm>(a, owned, n_tiles, grid, s);
        else launch_agent_r<kAgentCarsPerThread, kAgentBlocksPerSmShallow>(a, owned, n_tiles, grid, s);
    } else {
        if (deep) launch_agent_r<8, kAgentBlocksPerSm>(a, owned, n_tiles, grid, s);
        else launch_agent_r<8, kAgentBlocksPerSmShallow>(a, owned, n_tiles, grid, s);
    }
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

// This unit's debug word (zero in release builds).
NASCH_DEBUG_READER(debug_word_agent)

}  // namespace nasch
