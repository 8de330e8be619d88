// Bitruss hierarchy from the bitruss numbers (Defs. 4-5, Section II).
//
// The k-bitrusses are nested (H_{k+1} satisfies the support bound of H_k, and
// H_k is the unique maximal subgraph that does), and an edge lies in H_k
// exactly when phi_e >= k.  So one stable sort of the edges by phi, largest
// first, lists every H_k as a prefix, and H_k alone is a stream compaction of
// the edges with phi_e >= k.
#include "bt_device.cuh"
#include "bt_internal.cuh"

namespace bt {
namespace {

// keys sort ascending, so the complement of phi puts the largest phi first;
// the stable radix sort keeps equal phi in input order
__global__ void k_hier_keys(const uint32_t *phi, uint64_t m, uint32_t *keys, uint32_t *vals) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m;
         i += (uint64_t)gridDim.x * blockDim.x) {
        keys[i] = ~phi[i];
        vals[i] = (uint32_t)i;
    }
}

__global__ void k_hier_phi(const uint32_t *keys, uint64_t m, uint32_t *phi_sorted) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m;
         i += (uint64_t)gridDim.x * blockDim.x)
        phi_sorted[i] = ~keys[i];
}

__global__ void k_flag_ge(const uint32_t *phi, uint64_t m, uint32_t k, uint32_t *flag) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m;
         i += (uint64_t)gridDim.x * blockDim.x)
        flag[i] = phi[i] >= k ? 1u : 0u;
}

__global__ void k_compact(const uint32_t *phi, const uint32_t *pos, uint64_t m, uint32_t k, uint32_t *out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m;
         i += (uint64_t)gridDim.x * blockDim.x)
        if (phi[i] >= k) out[pos[i]] = (uint32_t)i;
}

inline unsigned grid_for(uint64_t items, int threads) {
    uint64_t g = (items + threads - 1) / threads;
    if (g == 0) g = 1;
    return (unsigned)(g < 152 * 32 ? g : 152 * 32);
}

}  // namespace

cudaError_t hierarchy_order(const uint32_t *phi, uint64_t m, uint32_t *order, uint32_t *phi_sorted, Alloc &al) {
    if (m == 0) return cudaSuccess;
    uint32_t *keys = al.get<uint32_t>(m);
    uint32_t *tk = al.get<uint32_t>(m);
    uint32_t *tv = al.get<uint32_t>(m);
    if (al.err != cudaSuccess) return al.err;
    k_hier_keys<<<grid_for(m, 256), 256, 0, al.stream>>>(phi, m, keys, order);
    al.launches++;
    BT_CUDA(radix_sort_u32(keys, order, tk, tv, m, 32, al));
    if (phi_sorted) {
        k_hier_phi<<<grid_for(m, 256), 256, 0, al.stream>>>(keys, m, phi_sorted);
        al.launches++;
    }
    al.put(keys);
    al.put(tk);
    al.put(tv);
    return cudaGetLastError();
}

cudaError_t select_ge(const uint32_t *phi, uint64_t m, uint32_t k, uint32_t *out, uint32_t *d_count,
                      Alloc &al) {
    if (m == 0) return cudaMemsetAsync(d_count, 0, sizeof(uint32_t), al.stream);
    uint32_t *flag = al.get<uint32_t>(m);
    uint32_t *pos = al.get<uint32_t>(m);
    if (al.err != cudaSuccess) return al.err;
    k_flag_ge<<<grid_for(m, 256), 256, 0, al.stream>>>(phi, m, k, flag);
    al.launches++;
    BT_CUDA(exclusive_scan_u32(flag, pos, m, d_count, al));
    k_compact<<<grid_for(m, 256), 256, 0, al.stream>>>(phi, pos, m, k, out);
    al.launches++;
    al.put(flag);
    al.put(pos);
    return cudaGetLastError();
}

}  // namespace bt
