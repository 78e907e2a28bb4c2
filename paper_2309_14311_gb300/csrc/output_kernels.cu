// Output of a running road: one row of the space-time diagram (the
// handout's density picture of the road over time, Fig. 1) per snapshot.
//
// Pixel i of a row of W pixels covers the cells c with floor(c * W / L) = i,
// that is [ceil(i L / W), ceil((i + 1) L / W)), and holds
// floor(255 * cars / cells) of that range: 0 empty, 255 full.
#include "road_output.h"

namespace nasch {
namespace {

constexpr int kRasterThreads = 256;

// ceil(i * L / W) without overflow (i <= W <= 2^31, L <= 2^31)
__device__ __forceinline__ uint64_t pixel_start(uint64_t i, uint64_t L, uint64_t W) { return (i * L + W - 1) / W; }

// One block per pixel (grid-stride over pixels): count the occupied cells of
// its range with coalesced byte loads, reduce, write the pixel.
__global__ void __launch_bounds__(kRasterThreads) raster_row_kernel(const int8_t *__restrict__ cells, uint32_t L,
                                                                    uint32_t W, uint8_t *__restrict__ row)
{
    __shared__ uint32_t s_warp[kRasterThreads / 32];
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    for (uint32_t i = blockIdx.x; i < W; i += gridDim.x) {
        const uint64_t c0 = pixel_start(i, L, W), c1 = pixel_start(i + 1u, L, W);
        uint32_t n = 0;
        for (uint64_t c = c0 + tid; c < c1; c += kRasterThreads) n += cells[c] >= 0 ? 1u : 0u;
        n = __reduce_add_sync(0xFFFFFFFFu, n);
        if (lane == 0) s_warp[warp] = n;
        __syncthreads();
        if (tid == 0) {
            uint32_t cars = 0;
            for (int w = 0; w < kRasterThreads / 32; ++w) cars += s_warp[w];
            const uint64_t cellsn = c1 - c0;
            row[i] = cellsn ? (uint8_t)((255ull * cars) / cellsn) : 0u;
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_raster_row(const int8_t *cells, uint32_t L, uint32_t W, uint8_t *row, int sms, cudaStream_t s)
{
    if (L == 0 || W == 0 || W > L) return cudaErrorInvalidValue;
    const uint32_t blocks = W < (uint32_t)sms * 8u ? W : (uint32_t)sms * 8u;
    raster_row_kernel<<<blocks, kRasterThreads, 0, s>>>(cells, L, W, row);
    return cudaGetLastError();
}

}  // namespace nasch
