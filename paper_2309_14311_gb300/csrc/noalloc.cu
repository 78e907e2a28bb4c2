// Start positions of one road computed on the GPU without allocating any
// device memory: Floyd's sampling (the same draws and the same bit-map method
// as the batched initialisation) with its bit map in a fixed, file-scope
// device array instead of a buffer obtained from the allocator.
//
// For callers that cannot allocate device memory themselves or through this
// library: a process whose device memory is entirely owned by another
// allocator (a framework's caching pool, a fixed arena set up at start), or
// a host that forbids allocation after start-up.  They pass the output
// buffer; the scratch comes from the array below, which every GPU that loads
// the library holds until the process exits.
#include <cuda_runtime.h>

#include "nasch.h"
#include "floyd_device.cuh"
#include "nasch_device.cuh"
#include "runtime_internal.h"

namespace nasch {
namespace {

constexpr int64_t kNoAllocMaxCells = int64_t(1) << 24;                // longest road: 16 Mi cells
constexpr size_t kNoAllocWords = (size_t)(kNoAllocMaxCells / 64);     // 2 MiB of bit map

// One bit per cell of the road being initialised.  Shared by every call.
static __device__ __align__(256) unsigned long long g_floyd_scratch[kNoAllocWords];

// Host code cannot use the array's name as a device address; look the
// address up with the calling thread's device current.  This is done on
// every call rather than cached: a context that is torn down and made again
// (cudaDeviceReset, or a framework resetting the device) reloads the
// library's device code, and a cached address would then be stale.
int scratch_address(unsigned long long **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_floyd_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(Floyd scratch)");
    *out = static_cast<unsigned long long *>(p);
    return NASCH_OK;
}

// Floyd's algorithm (Bentley & Floyd, CACM 1987) for the road by one block,
// 1024 draws at a time (floyd_road_bits: the same draws and result as the
// sequential algorithm), into the scratch bit map.
__global__ void __launch_bounds__(kFloydBlock) floyd_bits_single_kernel(uint64_t L, uint64_t N, uint32_t k0,
                                                                        uint32_t k1, uint32_t road,
                                                                        unsigned long long *bm)
{
    __shared__ FloydSmem sm;
    floyd_road_bits(L, N, road, k0, k1, bm, sm);
}

// Set bits in order -> sorted positions, one block of 256 threads: a
// block-wide prefix sum over the words' bit counts gives each word's first
// output slot.
__global__ void __launch_bounds__(256) floyd_expand_single_kernel(const unsigned long long *bm, uint32_t words,
                                                                  int32_t *x)
{
    __shared__ uint32_t s_warp[8];
    __shared__ uint32_t s_total;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    uint32_t running = 0;
    for (uint32_t base = 0; base < words; base += 256u) {
        const uint32_t w = base + tid;
        const unsigned long long bits = w < words ? bm[w] : 0ull;
        const uint32_t c = (uint32_t)__popcll(bits);
        uint32_t incl = c;
#pragma unroll
        for (uint32_t d = 1; d < 32; d <<= 1) {
            const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
            if (lane >= d) incl += t;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        if (tid == 0) {
            uint32_t acc = 0;
            for (int k = 0; k < 8; ++k) {
                const uint32_t t = s_warp[k];
                s_warp[k] = acc;
                acc += t;
            }
            s_total = acc;
        }
        __syncthreads();
        uint32_t pos = running + s_warp[warp] + incl - c;
        for (unsigned long long b2 = bits; b2; b2 &= b2 - 1) x[pos++] = (int32_t)(64u * w + (uint32_t)__ffsll(b2) - 1u);
        running += s_total;
        __syncthreads();
    }
}

}  // namespace
}  // namespace nasch

using namespace nasch;

extern "C" int nasch_floyd_init_device_noalloc(int64_t L, int64_t N, uint64_t seed, uint32_t road_id,
                                               int32_t *x_dev, void *stream)
{
    clear_error();
    if (L < 1 || L > kNoAllocMaxCells)
        return fail(NASCH_EINVAL, "L=%lld outside 1..%lld: the fixed scratch bit map holds %lld cells", (long long)L,
                    (long long)kNoAllocMaxCells, (long long)kNoAllocMaxCells);
    if (N < 0 || N > L) return fail(NASCH_EINVAL, "N=%lld outside 0..L=%lld", (long long)N, (long long)L);
    if (N > 0 && !x_dev) return fail(NASCH_EINVAL, "x_dev is NULL");
    if (N == 0) return NASCH_OK;
    unsigned long long *bm = nullptr;
    int st = scratch_address(&bm);
    if (st) return st;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint32_t words = (uint32_t)((L + 63) / 64);
    // the array keeps the previous call's bits: clear the part this road uses
    cudaError_t e = cudaMemsetAsync(bm, 0, (size_t)words * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "clear Floyd scratch");
    floyd_bits_single_kernel<<<1, kFloydBlock, 0, s>>>((uint64_t)L, (uint64_t)N, (uint32_t)seed, (uint32_t)(seed >> 32), road_id,
                                             bm);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "Floyd bit-map kernel");
    floyd_expand_single_kernel<<<1, 256, 0, s>>>(bm, words, x_dev);
    e = cudaGetLastError();
    return e == cudaSuccess ? NASCH_OK : cuda_fail(e, "Floyd expand kernel");
}
