// Device checks of a state handed to nasch_set_state: one pass over the
// cars (cells inside the road, velocities up to vmax, no car on the next
// car's cell, the descents that tell the cyclic order) and a count of the
// occupied cells after the cars are scattered into a grid (a shared cell
// leaves fewer occupied cells than cars).
#include "state_check.h"

namespace nasch {
namespace {

constexpr int kCheckThreads = 256;

__global__ void __launch_bounds__(kCheckThreads) check_cars_kernel(const int32_t *__restrict__ x,
                                                                   const uint8_t *__restrict__ v, uint32_t N,
                                                                   uint32_t L, uint32_t vmax,
                                                                   unsigned long long *out)
{
    __shared__ unsigned long long s_desc;
    if (threadIdx.x == 0) s_desc = 0;
    __syncthreads();
    const uint32_t stride = gridDim.x * blockDim.x;
    uint32_t desc = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        const int32_t xi = x[i];
        const int32_t nx = i + 1u < N ? x[i + 1u] : x[0];
        const bool bad = xi < 0 || (uint32_t)xi >= L || v[i] > vmax || (N >= 2u && nx == xi);
        if (bad) {   // this thread's later cars have larger indices
            atomicMin(&out[0], (unsigned long long)i);
            break;
        }
        desc += (N >= 2u && nx < xi) ? 1u : 0u;
    }
    desc = __reduce_add_sync(0xFFFFFFFFu, desc);
    if ((threadIdx.x & 31u) == 0 && desc) atomicAdd(&s_desc, (unsigned long long)desc);
    __syncthreads();
    if (threadIdx.x == 0 && s_desc) atomicAdd(&out[1], s_desc);
}

__global__ void __launch_bounds__(kCheckThreads) count_cars_kernel(const int8_t *__restrict__ cells, uint32_t L,
                                                                   unsigned long long *out)
{
    __shared__ unsigned long long s_n;
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t n4 = L / 16u;   // whole 16-cell vectors (the buffer is 256-byte aligned)
    const uint4 *c4 = reinterpret_cast<const uint4 *>(cells);
    uint32_t n = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        const uint4 q = c4[i];
        // a cell holds a car when its sign bit is clear
        n += __popc(~q.x & 0x80808080u) + __popc(~q.y & 0x80808080u) + __popc(~q.z & 0x80808080u) +
             __popc(~q.w & 0x80808080u);
    }
    for (uint32_t i = 16u * n4 + blockIdx.x * blockDim.x + threadIdx.x; i < L; i += stride)
        n += cells[i] >= 0 ? 1u : 0u;
    n = __reduce_add_sync(0xFFFFFFFFu, n);
    if ((threadIdx.x & 31u) == 0 && n) atomicAdd(&s_n, (unsigned long long)n);
    __syncthreads();
    if (threadIdx.x == 0 && s_n) atomicAdd(out, s_n);
}

int check_blocks(uint32_t work)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
        sms = 1;
    const uint32_t need = (work + kCheckThreads - 1u) / kCheckThreads;
    const uint32_t most = 8u * (uint32_t)(sms > 0 ? sms : 1);
    return (int)(need < most ? (need > 0 ? need : 1u) : most);
}

}  // namespace

cudaError_t launch_check_cars(const int32_t *x, const uint8_t *v, uint32_t N, uint32_t L, uint32_t vmax,
                              unsigned long long *out, cudaStream_t s)
{
    if (N == 0) return cudaSuccess;
    check_cars_kernel<<<check_blocks(N), kCheckThreads, 0, s>>>(x, v, N, L, vmax, out);
    return cudaGetLastError();
}

cudaError_t launch_count_cars(const int8_t *cells, uint32_t L, unsigned long long *out, cudaStream_t s)
{
    if (L == 0) return cudaSuccess;
    count_cars_kernel<<<check_blocks(L / 16u + 16u), kCheckThreads, 0, s>>>(cells, L, out);
    return cudaGetLastError();
}

}  // namespace nasch
