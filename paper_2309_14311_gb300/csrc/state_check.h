// Checks of a state uploaded by nasch_set_state, run on the device.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nasch {

// out[0]: the lowest index i of a car outside [0, L), faster than vmax, or
// (N >= 2) on the same cell as the next car in the array (the last car's
// next is car 0); out[1]: the number of descents x[next] < x[i] over all
// cars (N >= 2).  out[0] must hold UINT64_MAX and out[1] zero before the
// launch.
cudaError_t launch_check_cars(const int32_t *x, const uint8_t *v, uint32_t N, uint32_t L, uint32_t vmax,
                              unsigned long long *out, cudaStream_t s);

// *out += the number of occupied cells (value >= 0) of cells[0, L).
cudaError_t launch_count_cars(const int8_t *cells, uint32_t L, unsigned long long *out, cudaStream_t s);

}  // namespace nasch
