// Block- and warp-level helpers shared by the kernels of libbitruss.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace bt {
namespace dev {

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Exclusive scan of one value per thread over a block of <= 1024 threads;
// the block total is returned through *total.  Contains __syncthreads().
template <typename T>
__device__ T block_excl_scan(T x, T *total) {
    __shared__ T s_warp[32];
    __shared__ T s_total;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    T inc = warp_incl_scan(x);
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T v = lane < nwarps ? s_warp[lane] : T(0);
        T vi = warp_incl_scan(v);
        if (lane < nwarps) s_warp[lane] = vi - v;
        if (lane == nwarps - 1) s_total = vi;
    }
    __syncthreads();
    T res = inc - x + s_warp[warp];
    *total = s_total;
    __syncthreads();
    return res;
}

// Sum over the block (result valid in every thread).  Contains __syncthreads().
template <typename T>
__device__ T block_sum(T x) {
    __shared__ T s_part[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    x = warp_sum(x);
    if (lane == 0) s_part[warp] = x;
    __syncthreads();
    T t = 0;
    for (int i = 0; i < nwarps; ++i) t += s_part[i];
    __syncthreads();
    return t;
}

__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t *a, uint32_t len, uint32_t key) {
    uint32_t lo = 0, hi = len;
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Largest index i in [0, len) with a[i] <= key (a sorted ascending, a[0] <= key).
__device__ __forceinline__ uint32_t last_le_u32(const uint32_t *a, uint32_t len, uint32_t key) {
    uint32_t lo = 0, hi = len;  // answer in [lo, hi)
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (a[mid] <= key) lo = mid; else hi = mid;
    }
    return lo;
}

}  // namespace dev
}  // namespace bt
