// Launchers of the NaSch step kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nasch_device.cuh"

namespace nasch {

// Fusion depth limit of the tiled kernels (per-step statistics live in
// shared memory for the whole launch).
constexpr int kMaxFusedSteps = 64;

// Agent tiled kernel geometry: each warp holds a tile of 32 lanes x R cars
// (R = 16: 512 cars, the default; R = 8: 256 cars), of which the last
// round_up(k, R) are look-ahead halo; blocks of 128 threads (4 independent
// warps).
constexpr int kAgentThreads = 128;
// Register budget by fusion depth: launches of at least kAgentDeepSteps
// steps are bound by the Philox multiplies and run fastest at 3 blocks of
// 128 threads per SM (up to 168 registers); shallower launches move more
// bytes per car-step and gain from the fourth block's warps (127 registers).
constexpr int kAgentDeepSteps = 8;
constexpr int kAgentBlocksPerSm = 3;          // ksteps >= kAgentDeepSteps
constexpr int kAgentBlocksPerSmShallow = 4;   // ksteps < kAgentDeepSteps
static_assert(kAgentBlocksPerSm != kAgentBlocksPerSmShallow, "the budget names the launch's form");
constexpr int kAgentCarsPerThread = 16;
constexpr int kAgentTileSpan = 32 * kAgentCarsPerThread;
constexpr int kAgentTileSpanSmall = 32 * 8;

// Whole-ring agent kernel: one block of up to 1024 threads x 8 cars.
constexpr int kAgentRingMaxCars = 1024 * 8;

// Grid tiled kernel (k >= 2): a span of kGridSpan cells staged per tile =
// the tile's own kGridSpan - 2H cells plus a halo of H = round_up(k * vmax,
// 16) cells on each side; 256 threads, 32 cells each.  (The one-step kernel
// has tiles of its own.)
constexpr int kGridThreads = 256;
constexpr int kGridSpan = 8192;
constexpr int kGridTileCells = kGridSpan;   // the `tile` parameter value that selects the tiled kernel

// Warp-tiles of the list method (fused grid steps by one warp): staged cells
// per warp-tile and the largest halo (the tile keeps at least half the span).
constexpr uint32_t kKwSpan = 2048;
constexpr uint32_t kKwBuf = kKwSpan + 32u;              // + padding
constexpr uint32_t kKwList = kKwSpan + 64u;             // every cell a car, + dummies and one leader
constexpr uint32_t kKwMaxHalo = 512;
constexpr uint32_t kKwDummy = 0xF000u;                  // position of the dummy cars: beyond any move

// Status word bits set by kernels (read by the host after a launch).
constexpr unsigned int kStatusTimeout = 1u;   // a bounded wait on an async copy ran out

// Whole-ring grid kernel: the ring (and its successor) in shared memory.
constexpr int kGridRingMaxCells = 32768;

struct AgentStep {
    unsigned int *status;        // device status word (nonzero: a bounded wait ran out)
    const int32_t *x_in;
    const uint8_t *v_in;
    int32_t *x_out;
    uint8_t *v_out;
    uint32_t N;
    RoadConst rc;
    uint32_t step0;              // global step of the first fused step (mod 2^32)
    int ksteps;                  // steps in this launch
    unsigned long long *sum_v;   // [ksteps], accumulated (must start at 0 for the tiled kernel)
    unsigned long long *crossings;
};

struct GridStep {
    unsigned int *status;
    const int8_t *c_in;
    int8_t *c_out;
    RoadConst rc;
    uint32_t step0;
    int ksteps;
    unsigned long long *sum_v;
    unsigned long long *crossings;
    // the fused grid kernel's car lists of spans too dense for its shared
    // list, kKwList entries (3 bytes each) per warp of the launch
    // (grid_list_scratch_bytes()); null for the other kernels
    uint8_t *list_scratch = nullptr;
};

// Owned cars per warp-tile of `span` cars (32 lanes x span/32) for fusion depth k.
inline uint32_t agent_tile_owned(int k, int span)
{
    const int r = span / 32;
    return (uint32_t)(span - ((k + r - 1) / r) * r);
}
// Shared-memory list entries per warp of the fused grid kernel (a span with
// more cars uses its warp's part of GridStep::list_scratch).
constexpr uint32_t kKwListSmem = 1024;

// Halo cells per side for the grid tile.
inline uint32_t grid_halo(int k, uint32_t vmax) { return ((uint32_t)k * vmax + 15u) / 16u * 16u; }

// Debug words of the kernels' translation units (read and cleared; always
// zero in release builds): bits of the DebugSite checks that failed.
unsigned int debug_word_agent();
unsigned int debug_word_grid();
unsigned int debug_word_open();
unsigned int debug_word_batch();
unsigned int debug_word_segment();

// Resident blocks per SM of the agent tiled kernel for launches of `ksteps` steps.
int agent_tiled_blocks_per_sm(int ksteps);
int grid_tiled_blocks_per_sm();
// Bytes of GridStep::list_scratch a launch of the fused grid kernel needs on
// the current device (0 if the occupancy query fails).
size_t grid_list_scratch_bytes();

// A persistent grid of sms x agent_tiled_blocks_per_sm(a.ksteps) blocks at most.
cudaError_t launch_agent_tiled(const AgentStep &a, int span, int sms, cudaStream_t s);
cudaError_t launch_agent_ring(const AgentStep &a, cudaStream_t s);
cudaError_t launch_grid_tiled(const GridStep &g, int blocks, cudaStream_t s);
cudaError_t launch_grid_ring(const GridStep &g, cudaStream_t s);

// cells[x[i]] = v[i] for i < N into a grid already filled with -1.
cudaError_t launch_scatter_agent_to_grid(const int32_t *x, const uint8_t *v, uint32_t N,
                                         int8_t *cells, cudaStream_t s);
// Philox of n counters (testing).
cudaError_t launch_philox_test(const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out,
                               int64_t n, cudaStream_t s);

}  // namespace nasch
