// Internal declarations shared by the CUDA translation units of libbitruss.
// Nothing here is part of the public ABI (include/bitruss.h).
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/bitruss.h"

namespace bt {

constexpr uint32_t kAlive = 0xFFFFFFFFu;  // edge state: unassigned, not queued

// Device error word bits (written with atomicOr, read back by the host).
enum : uint32_t {
    kErrRange = 1u << 0,
    kErrDup = 1u << 1,
    kErrOverflow = 1u << 2,
};

// Optional per-phase CUDA-event timing (bt_profile_enable).
enum Phase { kPhCsr = 0, kPhCount = 1, kPhEmit = 2, kPhPeel = 3, kPhTotal = 4, kNumPhases = 5 };
struct Prof {
    bool on = false;
    cudaEvent_t ev[2 * kNumPhases] = {};
    bool used[kNumPhases] = {};
};

// Stream-ordered scratch allocation from the handle's memory pool, plus the
// call's launch counter and profiler.
struct Alloc {
    cudaStream_t stream;
    cudaMemPool_t pool;
    cudaError_t err = cudaSuccess;
    uint64_t launches = 0;
    Prof *prof = nullptr;
    // Optional fixed arena (set only by the allocation-free entry point):
    // get() then bump-allocates inside it and put() does nothing.
    unsigned char *arena = nullptr;
    size_t arena_size = 0, arena_used = 0;
    // Limits and host-side fault injection of the handle (bt_set_limits), or
    // null.  fail_alloc_at = n > 0 makes allocation number n of this call fail.
    const bt_limits *limits = nullptr;
    uint64_t n_allocs = 0;
    // NVTX push/pop ranges of the phases, nested call > csr, count, emit,
    // peel (host-side issue order; no-ops unless a profiler is attached).
    // Ranges an early error return left open are popped when the call's
    // allocator goes away, so the thread's range stack stays balanced.
    struct NvtxStack {
        int open = 0;
        NvtxStack() = default;
        NvtxStack(const NvtxStack &) = delete;
        NvtxStack(NvtxStack &&o) noexcept : open(o.open) { o.open = 0; }
        ~NvtxStack() {
            for (; open > 0; --open) nvtxRangePop();
        }
    } nvtx;
    void mark(int phase, bool end) {
        static const char *const kNames[kNumPhases] = {"bitruss: csr", "bitruss: count", "bitruss: emit",
                                                       "bitruss: peel", "bitruss: call"};
        if (!end) {
            nvtxRangePushA(kNames[phase]);
            ++nvtx.open;
        } else if (nvtx.open > 0) {
            nvtxRangePop();
            --nvtx.open;
        }
        if (prof && prof->on) {
            cudaEventRecord(prof->ev[2 * phase + (end ? 1 : 0)], stream);
            prof->used[phase] = true;
        }
    }
    template <typename T>
    T *get(size_t count) {
        if (err != cudaSuccess) return nullptr;
        if (limits && limits->fail_alloc_at && ++n_allocs == limits->fail_alloc_at) {
            err = cudaErrorMemoryAllocation;
            return nullptr;
        }
        void *p = nullptr;
        size_t bytes = count * sizeof(T);
        if (bytes == 0) bytes = 16;
        if (arena) {
            size_t off = (arena_used + 255) & ~size_t(255);
            if (off + bytes > arena_size) {
                err = cudaErrorMemoryAllocation;
                return nullptr;
            }
            arena_used = off + bytes;
            return reinterpret_cast<T *>(arena + off);
        }
        err = cudaMallocFromPoolAsync(&p, bytes, pool, stream);
        return err == cudaSuccess ? static_cast<T *>(p) : nullptr;
    }
    void put(void *p) {
        if (p && !arena) cudaFreeAsync(p, stream);
    }
};

// ---------------------------------------------------------------- scan/sort
// Exclusive prefix sum of n values (in-place allowed).  Writes the grand total
// to *total (device pointer) when total != nullptr.
cudaError_t exclusive_scan_u32(const uint32_t *in, uint32_t *out, size_t n, uint32_t *total,
                               Alloc &al);
cudaError_t exclusive_scan_u64(const uint64_t *in, uint64_t *out, size_t n, uint64_t *total,
                               Alloc &al);
// out[i] = in[i] widened to 64 bits.
cudaError_t widen_u32(const uint32_t *in, uint64_t *out, size_t n, Alloc &al);
// Stable LSD radix sort of (key, value) pairs on the low `bits` bits of the
// keys.  Result ends in (keys, vals); (tk, tv) are scratch of the same size.
cudaError_t radix_sort_u32(uint32_t *keys, uint32_t *vals, uint32_t *tk, uint32_t *tv, size_t n,
                           int bits, Alloc &al);
cudaError_t radix_sort_u64(uint64_t *keys, uint32_t *vals, uint64_t *tk, uint32_t *tv, size_t n,
                           int bits, Alloc &al);

// ---------------------------------------------------------------- graph
// Rank-ordered CSR over one id space of n = nU + nL vertices.  Vertex r is
// the vertex of rank r (priority order of Def. 7: degree, then global id);
// adjacency lists hold neighbour ranks sorted ascending, eid the edge ids.
struct Csr {
    uint32_t n = 0;
    uint64_t m = 0;
    uint64_t *off = nullptr;  // [n+1]
    uint32_t *adj = nullptr;  // [2m]
    uint32_t *eid = nullptr;  // [2m]
    uint32_t *hv = nullptr;   // [n] #neighbours of lower rank (a prefix of the list)
    uint32_t *pl = nullptr;   // [2m] for arc (u->v), v<u: #w in N(v) with w<u; else 0
    uint64_t *wv = nullptr;   // [n] priority-obeyed wedges started at each vertex
    // Internal edge ids: an edge is numbered by its position in the lower-rank
    // prefix of its higher-ranked endpoint, so the edges of one vertex are
    // contiguous (blooms anchored there touch neighbouring words).  eid holds
    // internal ids; newid maps input id -> internal id.
    uint32_t *newid = nullptr;  // [m]
    // A disjoint union of graphs is ranked graph by graph (each graph's own
    // degree-then-id order, graph after graph), so the wedges of a start
    // vertex stay inside its graph: vbase[r] is the first rank of r's graph,
    // and the counting kernels index their per-block counters by w - vbase[u],
    // cnt_n entries each (the largest graph) instead of n.
    uint32_t *vbase = nullptr;  // [n], or null for one graph
    uint32_t cnt_n = 0;
};

// The graphs of a disjoint union (bt_decompose_batch): offU/offL (device,
// ng entries) are each graph's first upper / lower id in the union; max_n
// the largest nU + nL.
struct GraphSplit {
    uint32_t ng = 0;
    const uint32_t *offU = nullptr, *offL = nullptr;
    uint32_t max_n = 0;
};

// Builds the CSR (and wedge prefix lengths) from a device edge list.
// err_word: device u32 receiving kErr* bits.  Returns a CUDA error.
cudaError_t build_csr(const int32_t *d_edges, uint64_t m, uint32_t nU, uint32_t nL, uint32_t flags,
                      Csr &g, uint32_t *err_word, Alloc &al, const GraphSplit *split = nullptr);
void free_csr(Csr &g, Alloc &al);
// out[e] = in[newid[e]]: a per-edge array in internal order back to input order.
cudaError_t gather_u64(const uint64_t *in, const uint32_t *newid, uint64_t *out, uint64_t m, Alloc &al);
cudaError_t gather_u32(const uint32_t *in, const uint32_t *newid, uint32_t *out, uint64_t m, Alloc &al);
// out[newid[e]] = in[e]: a per-edge byte array in input order to internal order.
cudaError_t scatter_u8(const uint8_t *in, const uint32_t *newid, uint8_t *out, uint64_t m, Alloc &al);
// In-place relabelling of ng concatenated edge lists (graph g owns edges
// [goff[g], goff[g+1])) into one disjoint union; range errors set kErrRange
// and the lowest failing graph index in *bad_graph.
cudaError_t union_edges(int32_t *d_edges, uint64_t m_total, const uint64_t *d_goff, uint32_t ng,
                        const uint32_t *d_offU, const uint32_t *d_offL, const uint32_t *d_nU,
                        const uint32_t *d_nL, uint32_t *err_word, uint32_t *bad_graph, Alloc &al);

// ---------------------------------------------------------------- counting
struct CountOut {
    uint64_t *support = nullptr;  // [m] (caller-provided, zeroed by count)
    uint32_t *inc_cnt = nullptr;  // [m] links per edge (index mode) or nullptr
    uint64_t *w2v = nullptr;      // [n] bloom wedges per start vertex (index mode)
    uint64_t *nbv = nullptr;      // [n] blooms per start vertex (index mode)
    unsigned long long *butterflies_dev = nullptr;  // [1] set by count_wedges; caller frees
    // [m] or nullptr: edges whose bitruss number is already known (progressive
    // compression); they get no links and are flagged in bit 31 inside pairs
    const uint8_t *assigned = nullptr;
};
// nt: count block size (256, 512 or 1024; anything else means 512).  Only
// start vertices of rank in [lo, hi) are enumerated: the supports are then
// those of the blooms started there (a counting shard).
cudaError_t count_wedges(const Csr &g, CountOut &o, int num_sms, Alloc &al, int nt = 512, uint32_t lo = 0,
                         uint32_t hi = 0xFFFFFFFFu);
// out[0], out[1]: the first rank r with pre[r] >= t0, resp. >= t1 (pre is a
// non-decreasing array of n values; n when no such rank).
cudaError_t rank_bounds(const uint64_t *pre, uint32_t n, uint64_t t0, uint64_t t1, uint32_t *out, Alloc &al);

// Device-resident BE-Index (Section IV-A).
struct Index {
    uint64_t m = 0;
    uint64_t nb = 0;             // blooms
    uint64_t w2 = 0;             // twin pairs (= links / 2)
    uint64_t w = 0;              // priority-obeyed wedges
    uint64_t butterflies = 0;
    uint64_t links = 0;          // edge-bloom links stored (2 w2, fewer in a compressed index)
    uint32_t *bloom_k = nullptr;     // [nb] bloom numbers
    uint32_t *bloom_off = nullptr;   // [nb+1] first pair of each bloom
    uint2 *pairs = nullptr;          // [w2] (e_uv, e_vw) twin edge ids
    uint64_t *inc_off = nullptr;     // [m+1]
    // [links] per edge: (pair id, bloom id | side << 31), side 0 when the
    // edge is the pair's first member (e_uv), 1 when it is the second
    uint2 *inc = nullptr;
    uint32_t *newid = nullptr;       // [m] input edge id -> internal id (ids above are internal)
    size_t bytes() const {
        return nb * 8 + 4 + w2 * 8 + (m + 1) * 8 + links * 8;
    }
};
cudaError_t emit_index(const Csr &g, const CountOut &c, Index &ix, int num_sms, Alloc &al,
                       cudaStream_t stream, int nt = 512);
void free_index(Index &ix, Alloc &al);

// ---------------------------------------------------------------- peeling
struct PeelResult {
    uint64_t rounds = 0, levels = 0, updates = 0, kmax = 0, windows = 0, slots = 0, scanned = 0;
    uint64_t inc_phases = 0;  // rounds that ran a separate incidence phase
    int status = BT_OK;
};
// support: [m] initial supports (device, preserved); phi_out: [m] device.
// Progressive compression (Alg. 6-7): edges with assigned[e] set keep their
// phi and are never peeled; the m_active others are peeled starting at level
// k_init, and phi is written only for edges leaving at a level >= assign_from.
struct PeelOpts {
    const uint8_t *assigned = nullptr;
    uint64_t m_active = 0;
    long long k_init = 0;
    long long assign_from = 0;
};
// seg: peel work-item size (32 or 64 entries; anything else means 32)
cudaError_t peel(const Index &ix, const uint64_t *support, uint32_t *phi_out, PeelResult &res,
                 int num_sms, Alloc &al, int seg = 32, const PeelOpts *opts = nullptr);

// ---------------------------------------------------------------- serving
// The peel of handle h spans 1/ways of the SMs (server workers share the GPU).
void share_peel_sms(bt_handle *h, int ways);

// ---------------------------------------------------------------- hierarchy
// order[i]: edge ids by phi descending, equal phi in ascending id (stable);
// phi_sorted (nullable) receives phi[order[i]].  m < 2^32.
cudaError_t hierarchy_order(const uint32_t *phi, uint64_t m, uint32_t *order, uint32_t *phi_sorted, Alloc &al);
// out[0 .. *d_count): ids of the edges with phi >= k, ascending (d_count: device).
cudaError_t select_ge(const uint32_t *phi, uint64_t m, uint32_t k, uint32_t *out, uint32_t *d_count,
                      Alloc &al);

// ---------------------------------------------------------------- progressive compression
// hist[min(sup, m)] counts over all edges (m + 1 bins, zeroed here).
cudaError_t support_hist(const uint64_t *sup, uint64_t m, uint32_t *hist, Alloc &al);
// Candidate subgraph G_{>=eps}: edges with support >= eps, compacted (cand
// int32 pairs, cmap = global edge id, cassigned = assigned flag);
// counts[0] = candidates, counts[1] = unassigned candidates.
cudaError_t select_candidates(const int32_t *edges, const uint64_t *sup, uint64_t m, uint64_t eps,
                              const uint8_t *assigned, int32_t *cand, uint32_t *cmap,
                              uint8_t *cassigned, unsigned long long *counts, Alloc &al);
// Copies the phi a pass settled (phi_local != 0xFFFFFFFF, edge not yet
// assigned) to the global arrays and marks those edges assigned.
cudaError_t settle(const uint32_t *cmap, uint64_t n, const uint8_t *cassigned,
                   const uint32_t *phi_local, uint32_t *phi, uint8_t *assigned, Alloc &al);

// ---------------------------------------------------------------- helpers
__host__ __device__ inline int bits_for(uint64_t maxval) {
    int b = 0;
    while (b < 64 && (maxval >> b) != 0) ++b;
    return b;
}

}  // namespace bt

#define BT_CUDA(x)                          \
    do {                                    \
        cudaError_t e_ = (x);               \
        if (e_ != cudaSuccess) return e_;   \
    } while (0)
