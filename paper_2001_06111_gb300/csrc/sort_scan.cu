// Device-wide exclusive scan and stable LSD radix sort used by the CSR build
// and the BE-Index layout (prefix sums over per-vertex / per-edge counts).
#include "bt_internal.cuh"
#include "bt_device.cuh"

namespace bt {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanChunk = kScanThreads * kScanItems;

using dev::block_excl_scan;

template <typename T>
__global__ void k_scan_reduce(const T *in, size_t n, T *sums) {
    size_t base = (size_t)blockIdx.x * kScanChunk;
    T acc = 0;
    for (int i = 0; i < kScanItems; ++i) {
        size_t idx = base + (size_t)i * kScanThreads + threadIdx.x;
        if (idx < n) acc += in[idx];
    }
    // block reduce
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ T s[kScanThreads / 32];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        T t = 0;
        for (int i = 0; i < kScanThreads / 32; ++i) t += s[i];
        sums[blockIdx.x] = t;
    }
}

// One block scans the block sums (any count) with a running carry.
template <typename T>
__global__ void k_scan_top(T *sums, size_t nb, T *total) {
    T carry = 0;
    for (size_t base = 0; base < nb; base += kScanThreads) {
        size_t idx = base + threadIdx.x;
        T x = idx < nb ? sums[idx] : T(0);
        T tot;
        T ex = block_excl_scan(x, &tot);
        if (idx < nb) sums[idx] = ex + carry;
        carry += tot;
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

template <typename T>
__global__ void k_scan_down(const T *in, T *out, size_t n, const T *sums) {
    __shared__ T s[kScanChunk];
    size_t base = (size_t)blockIdx.x * kScanChunk;
    for (int i = 0; i < kScanItems; ++i) {
        int li = i * kScanThreads + threadIdx.x;
        size_t idx = base + li;
        s[li] = idx < n ? in[idx] : T(0);
    }
    __syncthreads();
    T v[kScanItems];
    T acc = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = s[threadIdx.x * kScanItems + i];
        acc += v[i];
    }
    T tot;
    T ex = block_excl_scan(acc, &tot) + sums[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        s[threadIdx.x * kScanItems + i] = ex;
        ex += v[i];
    }
    __syncthreads();
    for (int i = 0; i < kScanItems; ++i) {
        int li = i * kScanThreads + threadIdx.x;
        size_t idx = base + li;
        if (idx < n) out[idx] = s[li];
    }
}

template <typename T>
cudaError_t scan_impl(const T *in, T *out, size_t n, T *total, Alloc &al) {
    if (n == 0) {
        if (total) BT_CUDA(cudaMemsetAsync(total, 0, sizeof(T), al.stream));
        return cudaSuccess;
    }
    size_t nb = (n + kScanChunk - 1) / kScanChunk;
    T *sums = al.get<T>(nb);
    if (!sums) return al.err;
    k_scan_reduce<T><<<(unsigned)nb, kScanThreads, 0, al.stream>>>(in, n, sums);
    al.launches++;
    k_scan_top<T><<<1, kScanThreads, 0, al.stream>>>(sums, nb, total);
    al.launches++;
    k_scan_down<T><<<(unsigned)nb, kScanThreads, 0, al.stream>>>(in, out, n, sums);
    al.launches++;
    al.put(sums);
    return cudaGetLastError();
}

// ------------------------------------------------------------- radix sort
constexpr int kSortThreads = 256;
constexpr int kSortRounds = 16;
constexpr int kSortTile = kSortThreads * kSortRounds;

template <typename K>
__global__ void k_radix_hist(const K *keys, size_t n, int shift, uint32_t *hist, uint32_t ntiles) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    size_t base = (size_t)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortRounds; ++r) {
        size_t idx = base + (size_t)r * kSortThreads + threadIdx.x;
        if (idx < n) atomicAdd(&h[(uint32_t)(keys[idx] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: items of a tile keep their input order within a digit.
template <typename K>
__global__ void k_radix_scatter(const K *kin, const uint32_t *vin, K *kout, uint32_t *vout,
                                size_t n, int shift, const uint32_t *offs, uint32_t ntiles) {
    __shared__ uint32_t s_base[256];
    __shared__ uint32_t s_wcnt[kSortThreads / 32][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    s_base[tid] = offs[(size_t)tid * ntiles + blockIdx.x];
    for (int w = 0; w < kSortThreads / 32; ++w) s_wcnt[w][tid] = 0;
    __syncthreads();
    const uint32_t lt_mask = (1u << lane) - 1u;
    size_t base = (size_t)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortRounds; ++r) {
        size_t idx = base + (size_t)r * kSortThreads + tid;
        bool valid = idx < n;
        K key = valid ? kin[idx] : K(0);
        uint32_t val = valid ? vin[idx] : 0u;
        uint32_t d = valid ? ((uint32_t)(key >> shift) & 255u) : 256u;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t lrank = __popc(peers & lt_mask);
        if (valid && lrank == 0) s_wcnt[warp][d] = __popc(peers);
        __syncthreads();
        uint32_t run = 0;
        for (int w = 0; w < kSortThreads / 32; ++w) {
            uint32_t c = s_wcnt[w][tid];
            s_wcnt[w][tid] = run;
            run += c;
        }
        __syncthreads();
        if (valid) {
            uint32_t pos = s_base[d] + s_wcnt[warp][d] + lrank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        s_base[tid] += run;
        for (int w = 0; w < kSortThreads / 32; ++w) s_wcnt[w][tid] = 0;
        __syncthreads();
    }
}

template <typename K>
cudaError_t radix_impl(K *keys, uint32_t *vals, K *tk, uint32_t *tv, size_t n, int bits,
                       Alloc &al) {
    if (n <= 1 || bits <= 0) return cudaSuccess;
    uint32_t ntiles = (uint32_t)((n + kSortTile - 1) / kSortTile);
    uint32_t *hist = al.get<uint32_t>((size_t)256 * ntiles);
    if (!hist) return al.err;
    K *ka = keys, *kb = tk;
    uint32_t *va = vals, *vb = tv;
    int passes = (bits + 7) / 8;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        k_radix_hist<K><<<ntiles, kSortThreads, 0, al.stream>>>(ka, n, shift, hist, ntiles);
        al.launches++;
        cudaError_t e = scan_impl<uint32_t>(hist, hist, (size_t)256 * ntiles, nullptr, al);
        if (e != cudaSuccess) return e;
        k_radix_scatter<K><<<ntiles, kSortThreads, 0, al.stream>>>(ka, va, kb, vb, n, shift, hist,
                                                                    ntiles);
        al.launches++;
        K *t = ka; ka = kb; kb = t;
        uint32_t *u = va; va = vb; vb = u;
    }
    if (ka != keys) {
        BT_CUDA(cudaMemcpyAsync(keys, ka, n * sizeof(K), cudaMemcpyDeviceToDevice, al.stream));
        BT_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, al.stream));
    }
    al.put(hist);
    return cudaGetLastError();
}

__global__ void k_widen(const uint32_t *in, uint64_t *out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        out[i] = in[i];
}

}  // namespace

cudaError_t widen_u32(const uint32_t *in, uint64_t *out, size_t n, Alloc &al) {
    if (n == 0) return cudaSuccess;
    size_t g = (n + 255) / 256;
    if (g > 152 * 64) g = 152 * 64;
    k_widen<<<(unsigned)g, 256, 0, al.stream>>>(in, out, n);
    al.launches++;
    return cudaGetLastError();
}

cudaError_t exclusive_scan_u32(const uint32_t *in, uint32_t *out, size_t n, uint32_t *total,
                               Alloc &al) {
    return scan_impl<uint32_t>(in, out, n, total, al);
}
cudaError_t exclusive_scan_u64(const uint64_t *in, uint64_t *out, size_t n, uint64_t *total,
                               Alloc &al) {
    return scan_impl<uint64_t>(in, out, n, total, al);
}
cudaError_t radix_sort_u32(uint32_t *keys, uint32_t *vals, uint32_t *tk, uint32_t *tv, size_t n,
                           int bits, Alloc &al) {
    return radix_impl<uint32_t>(keys, vals, tk, tv, n, bits, al);
}
cudaError_t radix_sort_u64(uint64_t *keys, uint32_t *vals, uint64_t *tk, uint32_t *tv, size_t n,
                           int bits, Alloc &al) {
    return radix_impl<uint64_t>(keys, vals, tk, tv, n, bits, al);
}

}  // namespace bt
