// Kernels of progressive compression (BiT-PC, Section V-C, Alg. 6-7):
// k_max from the supports, extraction of the candidate subgraph G_{>=eps},
// and the hand-back of the bitruss numbers a pass has settled.
#include "bt_device.cuh"
#include "bt_internal.cuh"

namespace bt {
namespace {

inline unsigned grid_for(uint64_t items, int threads, unsigned cap = 152 * 32) {
    uint64_t g = (items + threads - 1) / threads;
    if (g == 0) g = 1;
    return (unsigned)(g < cap ? g : cap);
}

// hist[min(support, m)] += 1
__global__ void k_support_hist(const uint64_t *sup, uint64_t m, uint32_t *hist) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t s = sup[i];
        atomicAdd(&hist[s < m ? s : m], 1u);
    }
}

// Edges with support >= eps (Lemma 10: the eps-bitruss lies inside them),
// compacted with their global ids and assigned flags.
__global__ void k_select(const int32_t *edges, const uint64_t *sup, uint64_t m, uint64_t eps,
                         const uint8_t *assigned, int32_t *cand, uint32_t *cmap, uint8_t *cassigned,
                         unsigned long long *counts) {
    const int lane = threadIdx.x & 31;
    for (uint64_t i0 = blockIdx.x * (uint64_t)blockDim.x; i0 < m; i0 += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = i0 + threadIdx.x;
        const bool keep = i < m && sup[i] >= eps;
        const bool un = keep && !assigned[i];
        const unsigned mask = __ballot_sync(0xffffffffu, keep);
        const unsigned umask = __ballot_sync(0xffffffffu, un);
        if (!mask) continue;
        unsigned long long base = 0;
        if (lane == 0) {
            base = atomicAdd(&counts[0], (unsigned long long)__popc(mask));
            if (umask) atomicAdd(&counts[1], (unsigned long long)__popc(umask));
        }
        base = __shfl_sync(0xffffffffu, base, 0);
        if (keep) {
            const uint64_t j = base + __popc(mask & ((1u << lane) - 1u));
            reinterpret_cast<int2 *>(cand)[j] = reinterpret_cast<const int2 *>(edges)[i];
            cmap[j] = (uint32_t)i;
            cassigned[j] = assigned[i];
        }
    }
}

// Bitruss numbers settled by a pass (written, i.e. not the 0xFFFFFFFF fill)
// go back to the global arrays and their edges become assigned.
__global__ void k_settle(const uint32_t *cmap, uint64_t n, const uint8_t *cassigned,
                         const uint32_t *phi_local, uint32_t *phi, uint8_t *assigned) {
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < n;
         j += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t v = phi_local[j];
        if (!cassigned[j] && v != 0xFFFFFFFFu) {
            phi[cmap[j]] = v;
            assigned[cmap[j]] = 1;
        }
    }
}

}  // namespace

cudaError_t support_hist(const uint64_t *sup, uint64_t m, uint32_t *hist, Alloc &al) {
    BT_CUDA(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * (m + 1), al.stream));
    k_support_hist<<<grid_for(m, 256), 256, 0, al.stream>>>(sup, m, hist);
    al.launches++;
    return cudaGetLastError();
}

cudaError_t select_candidates(const int32_t *edges, const uint64_t *sup, uint64_t m, uint64_t eps,
                              const uint8_t *assigned, int32_t *cand, uint32_t *cmap,
                              uint8_t *cassigned, unsigned long long *counts, Alloc &al) {
    BT_CUDA(cudaMemsetAsync(counts, 0, 2 * sizeof(unsigned long long), al.stream));
    k_select<<<grid_for(m, 256), 256, 0, al.stream>>>(edges, sup, m, eps, assigned, cand, cmap,
                                                      cassigned, counts);
    al.launches++;
    return cudaGetLastError();
}

cudaError_t settle(const uint32_t *cmap, uint64_t n, const uint8_t *cassigned,
                   const uint32_t *phi_local, uint32_t *phi, uint8_t *assigned, Alloc &al) {
    if (n == 0) return cudaSuccess;
    k_settle<<<grid_for(n, 256), 256, 0, al.stream>>>(cmap, n, cassigned, phi_local, phi, assigned);
    al.launches++;
    return cudaGetLastError();
}

}  // namespace bt
