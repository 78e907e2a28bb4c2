// Helpers shared by the runtime translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

#include "nasch.h"

namespace nasch {

// Names a host phase in profiler timelines (NVTX range; free when no tool
// is attached).
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

// Record a message for nasch_last_error() and return `code`.
int fail(int code, const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);
void clear_error();

uint64_t slow_threshold(double p);
int validate_params(const nasch_params *prm);
int floyd_init_host(int64_t L, int64_t N, uint64_t seed, uint32_t road, int32_t *x);
int device_info(int *device, int *sms);
// The density below which the AUTO roads of a job (one road, or a batch)
// take the agent layout: the tuned value, or the state-byte crossover 0.2
// when those roads would need more than half of the free device memory at
// the tuned value.
double auto_rho_star(const nasch_params *roads, int64_t n);

}  // namespace nasch
