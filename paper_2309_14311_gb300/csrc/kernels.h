// Launchers of the NaSch step kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nasch_device.cuh"

namespace nasch {

// Fusion depth limit of the tiled kernels (per-step statistics live in
// shared memory for the whole launch).
constexpr int kMaxFusedSteps = 64;

// Agent tiled kernel geometry: 256 threads x 8 cars = 2048 cars per tile,
// of which the last round_up(k, 8) are look-ahead halo.
constexpr int kAgentThreads = 256;
constexpr int kAgentCarsPerThread = 8;
constexpr int kAgentTileSpan = kAgentThreads * kAgentCarsPerThread;

// Whole-ring agent kernel: one block of up to 1024 threads x 8 cars.
constexpr int kAgentRingMaxCars = 1024 * 8;

// Grid tiled kernel: tile of kGridTileCells cells plus a halo of
// round_up(k * vmax, 16) cells on each side.
constexpr int kGridThreads = 256;
constexpr int kGridTileCells = 8192;

// Whole-ring grid kernel: the ring (and its successor) in shared memory.
constexpr int kGridRingMaxCells = 32768;

struct AgentStep {
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
    const int8_t *c_in;
    int8_t *c_out;
    RoadConst rc;
    uint32_t step0;
    int ksteps;
    unsigned long long *sum_v;
    unsigned long long *crossings;
};

// Owned cars per tile for fusion depth k.
inline uint32_t agent_tile_owned(int k) { return (uint32_t)(kAgentTileSpan - ((k + 7) / 8) * 8); }
// Halo cells per side for the grid tile.
inline uint32_t grid_halo(int k, uint32_t vmax) { return ((uint32_t)k * vmax + 15u) / 16u * 16u; }

int agent_tiled_blocks_per_sm();
int grid_tiled_blocks_per_sm();

cudaError_t launch_agent_tiled(const AgentStep &a, int blocks, cudaStream_t s);
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
