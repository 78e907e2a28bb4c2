// Calibration kernel: the rate at which this GPU evaluates the rule-3 draw
// (word 0 of Philox4x32-10) with nothing else to do.  Every car-step of the
// NaSch step needs one such draw, so this rate is the integer-pipe ceiling
// of the step; the benchmark reports the step kernels against it.
#include <cuda_runtime.h>

#include "nasch.h"
#include "runtime_internal.h"
#include "tile_device.cuh"

namespace nasch {
namespace {

constexpr int kChains = 8;   // independent draws in flight per thread

// Draws keyed as in a step: within one step (i) the counter's cell word
// varies from draw to draw and the step word does not, so the parts of the
// rounds that depend only on the step are shared by the kChains draws, as
// they are by the cars of one step in the kernels.
__global__ void __launch_bounds__(256) philox_rate_kernel(uint32_t k0, uint32_t k1, uint32_t iters,
                                                          uint32_t *sink)
{
    const uint32_t cell = (blockIdx.x * blockDim.x + threadIdx.x) * (uint32_t)kChains;
    uint32_t acc = 0;
    for (uint32_t i = 0; i < iters; i += kChains) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) acc ^= philox_word0(cell + (uint32_t)j, i, 7u, kTagSlowdown, k0, k1);
    }
    if (acc == 0x9E3779B9u) sink[0] = acc;   // keeps the draws live; practically never taken
}

// A bounded wait that runs out on purpose: the mbarrier expects 16 bytes
// that no copy will deliver, so every thread's wait gives up after limit_ns,
// the kernel records the timeout in the status word and returns.  No copy
// is in flight, so nothing outlives the kernel.
__global__ void bounded_wait_selftest_kernel(uint64_t limit_ns, unsigned int *status)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_expect_tx(&bar, 16);
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0u, limit_ns);
    if (!__syncthreads_and(ok) && threadIdx.x == 0) atomicOr(status, kStatusTimeout);
}

}  // namespace
}  // namespace nasch

using namespace nasch;

extern "C" int nasch_selftest_bounded_wait(int64_t limit_ms, uint32_t *status_out)
{
    clear_error();
    if (limit_ms < 1 || limit_ms > 5000) return fail(NASCH_EINVAL, "limit_ms outside 1..5000");
    unsigned int *d = nullptr;
    unsigned int h = 0;
    cudaError_t e = cudaMalloc(&d, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(d, 0, sizeof(unsigned int));
    if (e == cudaSuccess) {
        bounded_wait_selftest_kernel<<<1, 64>>>((uint64_t)limit_ms * 1000000ull, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "bounded-wait self-test");
    if (status_out) *status_out = h;
    return h ? fail(NASCH_ETIMEOUT, "the kernel's bounded wait ran out (status 0x%x), as the self-test intends", h)
             : NASCH_OK;
}

extern "C" int nasch_calibrate_philox(int64_t draws_per_thread, double *draws_per_second, double *seconds)
{
    clear_error();
    if (!draws_per_second || draws_per_thread <= 0 || draws_per_thread > (int64_t(1) << 30))
        return fail(NASCH_EINVAL, "bad arguments");
    int dev = 0, sms = 1;
    int st = device_info(&dev, &sms);
    if (st) return st;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, philox_rate_kernel, 256, 0);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy");
    const int blocks = sms * (per_sm > 0 ? per_sm : 1);
    const uint32_t iters = (uint32_t)((draws_per_thread + kChains - 1) / kChains * kChains);
    uint32_t *sink = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    e = cudaMalloc(&sink, 4);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaSuccess) {
        philox_rate_kernel<<<blocks, 256>>>(1u, 2u, iters, sink);   // warm-up
        e = cudaEventRecord(a);
    }
    if (e == cudaSuccess) {
        philox_rate_kernel<<<blocks, 256>>>(3u, 4u, iters, sink);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(b);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(sink);
    if (e != cudaSuccess) return cuda_fail(e, "philox calibration");
    const double s = ms * 1e-3;
    *draws_per_second = (double)blocks * 256.0 * (double)iters / s;
    if (seconds) *seconds = s;
    return NASCH_OK;
}
