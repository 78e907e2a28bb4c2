// Device-side structures of batched runs (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "kernels.h"
#include "nasch.h"

namespace nasch {

// How one road of a batch is stepped.
enum BatchType : uint32_t {
    kBatchAgentTile = 0,   // agent layout, warp-tiles of 256 cars, 16 per item (2 per warp)
    kBatchGridTile = 1,    // grid layout, one staged 8192-cell span per item
    kBatchAgentRing = 2,   // agent layout, N <= 2048: the whole ring in one item
    kBatchGridRing = 3,    // grid layout, L <= 8192: the whole ring in one item
    kBatchGridWarp = 4,    // grid layout, H <= 512: 8 warp-tiles of 2048 staged cells per item (list method)
};

constexpr int kBatchThreads = 256;
constexpr int kBatchMinBlocks = 3;                                    // launch bound: blocks per SM
constexpr int kBatchAgentR = 8;                                       // cars per thread of a whole-ring item
constexpr int kBatchAgentTileR = 8;                                   // cars per lane of an agent warp-tile
constexpr uint32_t kBatchAgentSpan = 32u * kBatchAgentTileR;          // cars per warp-tile
constexpr uint32_t kBatchRingCars = kBatchThreads * kBatchAgentR;     // 2048
constexpr uint32_t kBatchRingCells = (uint32_t)kGridSpan;             // 8192
constexpr uint32_t kBatchWarpTilesPerWarp = 2;                        // agent warp-tiles per warp per item

struct BatchRoadDev {
    uint32_t L, N, vmax, type;
    uint64_t thr;
    uint32_t key0, key1, road_id, k;   // k: steps per super-step
    uint32_t T;                        // steps to run
    uint32_t step0;                    // global index of the first step
    uint32_t sbase;                    // the road's super-step at launch super_step 0 (serving; 0 in batches)
    uint32_t pad0;
    uint32_t halo;                     // grid: H cells per side; agent: halo cars per warp-tile
    uint32_t tile;                     // grid: owned cells per item (per warp-tile for kBatchGridWarp);
                                       // agent: owned cars per warp-tile
    int32_t *x[2];
    uint8_t *v[2];
    int8_t *cells[2];
    unsigned long long *sum_v;         // [T]
    unsigned long long *crossings;     // [T]
};

struct BatchItem {
    uint32_t road;
    uint32_t tile;
};

struct BatchLaunch {
    const BatchRoadDev *roads;
    const BatchItem *items;
    uint32_t n_items;                  // active items this super-step (a prefix of the list)
    uint32_t super_step;               // launch index; road r runs its super-step sbase_r + super_step
    uint32_t *counter;                 // work-list cursor of this super-step (starts at 0)
    const volatile uint32_t *cancel;   // host-mapped; nonzero: skip remaining work
    uint32_t padded;                   // grid buffer length (max over the batch's grid roads)
};

// The automatic choices in force when a batch or a server is made: the
// global tuning and the per-road table (nasch_set_tuning_table).
struct TuningSnapshot {
    double rho_star = 1.0;
    int k_agent = 8, k_grid = 8;
    std::vector<nasch_tuning_entry> table;
};
TuningSnapshot tuning_snapshot();
// True when a batch with its AUTO roads laid out as the snapshot chooses
// (state, statistics of steps[i] steps, start-state bit maps) would need more
// than 85 % of the free device memory: the batch then uses the state-byte
// crossover density and ignores the table's layouts.
bool auto_memory_short(const nasch_params *roads, int64_t n, const int64_t *steps, const TuningSnapshot &ts);

// Per-road plan shared by batches and the server: layout (AUTO: the table,
// else by density), item kind, fusion depth, halo/tile geometry, items per
// super-step and the number of super-steps.  Pointers and sbase are left
// zero.
void plan_road(const nasch_params &p, int64_t T, const TuningSnapshot &ts, bool memory_short, BatchRoadDev *rd,
               int *layout, int64_t *n_items, int64_t *super);

size_t batch_smem_bytes(uint32_t padded);
int batch_blocks_per_sm(uint32_t padded);
cudaError_t launch_batch_super_step(const BatchLaunch &bl, int blocks, cudaStream_t s);
// Floyd initial positions for every road: bit maps, then x[0] (agent) or
// cells[0] (grid; cells must already hold -1).
cudaError_t launch_batch_floyd(const BatchRoadDev *roads, uint32_t n, uint64_t *const *bitmaps, int sms,
                               cudaStream_t s);

}  // namespace nasch
