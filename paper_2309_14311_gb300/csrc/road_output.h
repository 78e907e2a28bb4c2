// Launchers of the open-road step and of the output kernels (internal to
// the library).
#pragma once

#include "kernels.h"

namespace nasch {

// One step of an open road (grid layout; see open_kernels.cu): the exit's
// and the entry's outcomes for the step are decided by the caller.
cudaError_t launch_grid_open(const GridStep &g, bool exit_open, bool entry, cudaStream_t s);
// The same by the one-step kernel (grid_kernels.cu), for vmax <= 16.
cudaError_t launch_grid_k1_open(const GridStep &g, bool exit_open, bool entry, cudaStream_t s);

// One row of the space-time raster from a road's cells (see output_kernels.cu).
cudaError_t launch_raster_row(const int8_t *cells, uint32_t L, uint32_t W, uint8_t *row, int sms, cudaStream_t s);

}  // namespace nasch
