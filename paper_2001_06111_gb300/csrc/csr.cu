// Degree, priority rank and rank-ordered CSR (the preprocessing of Alg. 3:
// "compute p(u) for each u", Def. 7), plus the per-arc wedge prefix lengths
// that bound the priority-obeyed wedge loops (Def. 10, Lemma 6).
#include "bt_internal.cuh"

namespace bt {
namespace {

// Global id of each endpoint.  Section II assumes every upper id exceeds
// every lower id: lower v -> v, upper u -> nL + u.  BT_TIE_LOWER_FIRST swaps
// the layers (upper u -> u, lower v -> nU + v).
__device__ __forceinline__ void gids(int32_t u, int32_t v, uint32_t nU, uint32_t nL, uint32_t flags,
                                     uint32_t &gu, uint32_t &gv) {
    if (flags & BT_TIE_LOWER_FIRST) {
        gu = (uint32_t)u;
        gv = nU + (uint32_t)v;
    } else {
        gu = nL + (uint32_t)u;
        gv = (uint32_t)v;
    }
}

__global__ void k_degree(const int32_t *edges, uint64_t m, uint32_t nU, uint32_t nL, uint32_t flags,
                         uint32_t *deg, uint32_t *err) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m;
         i += (uint64_t)gridDim.x * blockDim.x) {
        int2 e = reinterpret_cast<const int2 *>(edges)[i];
        if (e.x < 0 || e.y < 0 || (uint32_t)e.x >= nU || (uint32_t)e.y >= nL) {
            atomicOr(err, kErrRange);
            continue;
        }
        uint32_t gu, gv;
        gids(e.x, e.y, nU, nL, flags, gu, gv);
        atomicAdd(&deg[gu], 1u);
        atomicAdd(&deg[gv], 1u);
    }
}

__global__ void k_iota(uint32_t *a, uint32_t n) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        a[i] = i;
}

// order[r] = global id of rank r (sorted by degree, stable on id => ties by
// id); deg_sorted[r] = its degree.
__global__ void k_rank(const uint32_t *order, const uint32_t *deg_sorted, uint32_t n,
                       uint32_t *rank, uint64_t *degr) {
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        rank[order[r]] = r;
        degr[r] = deg_sorted[r];
    }
}

// Union ranking key of every vertex id: its graph, then its degree (the sort
// is stable, so ties stay in id order, as for the graph alone).
__global__ void k_graph_keys(const uint32_t *deg, uint32_t n, uint32_t nU, uint32_t nL, uint32_t flags,
                             uint32_t ng, const uint32_t *offU, const uint32_t *offL, int dbits,
                             uint32_t *keys) {
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        // the layer and layer-local id of x (see gids)
        bool upper;
        uint32_t loc;
        if (flags & BT_TIE_LOWER_FIRST) {
            upper = x < nU;
            loc = upper ? x : x - nU;
        } else {
            upper = x >= nL;
            loc = upper ? x - nL : x;
        }
        const uint32_t *off = upper ? offU : offL;
        uint32_t lo = 0, hi = ng;  // largest g with off[g] <= loc
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (off[mid] <= loc) lo = mid; else hi = mid;
        }
        keys[x] = lo << dbits | deg[x];
    }
}

// After the union sort: rank r's degree and the first rank of its graph.
__global__ void k_graph_rank(const uint32_t *keys_sorted, uint32_t n, int dbits, const uint32_t *offU,
                             const uint32_t *offL, uint32_t *deg_sorted, uint32_t *vbase) {
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const uint32_t k = keys_sorted[r];
        const uint32_t gi = k >> dbits;
        deg_sorted[r] = k & ((1u << dbits) - 1u);
        vbase[r] = offU[gi] + offL[gi];  // vertices of the graphs before it
    }
}

__global__ void k_arcs(const int32_t *edges, uint64_t m, uint32_t nU, uint32_t nL, uint32_t flags,
                       const uint32_t *rank, uint32_t n, uint64_t *keys, uint32_t *vals) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m;
         i += (uint64_t)gridDim.x * blockDim.x) {
        int2 e = reinterpret_cast<const int2 *>(edges)[i];
        if (e.x < 0 || e.y < 0 || (uint32_t)e.x >= nU || (uint32_t)e.y >= nL) {
            keys[2 * i] = keys[2 * i + 1] = 0;  // flagged by k_degree; call fails
            vals[2 * i] = vals[2 * i + 1] = (uint32_t)i;
            continue;
        }
        uint32_t gu, gv;
        gids(e.x, e.y, nU, nL, flags, gu, gv);
        uint64_t ru = rank[gu], rv = rank[gv];
        keys[2 * i] = ru * n + rv;
        vals[2 * i] = (uint32_t)i;
        keys[2 * i + 1] = rv * n + ru;
        vals[2 * i + 1] = (uint32_t)i;
    }
}

__global__ void k_csr_fill(const uint64_t *keys, const uint32_t *vals, uint64_t na, uint32_t n,
                           uint32_t *adj, uint32_t *eid, uint32_t *err) {
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < na;
         j += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t k = keys[j];
        adj[j] = (uint32_t)(k % n);
        eid[j] = vals[j];
        if (j > 0 && keys[j - 1] == k) atomicOr(err, kErrDup);
    }
}

__device__ __forceinline__ uint32_t lower_bound(const uint32_t *a, uint32_t len, uint32_t key) {
    uint32_t lo = 0, hi = len;
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Warp per vertex u: hv[u] = |{v in N(u): v < u}|; for those arcs
// pl = |{w in N(v): w < u}|; wv[u] = sum of pl (wedges started at u).
__global__ void k_wedge_prefix(const uint64_t *off, const uint32_t *adj, uint32_t n, uint32_t *hv,
                               uint32_t *pl, uint64_t *wv) {
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t u = warp; u < n; u += nwarps) {
        uint64_t a = off[u];
        uint32_t d = (uint32_t)(off[u + 1] - a);
        uint32_t h = lower_bound(adj + a, d, u);
        uint64_t acc = 0;
        for (uint32_t i = lane; i < d; i += 32) {
            uint32_t p = 0;
            if (i < h) {
                uint32_t v = adj[a + i];
                uint64_t b = off[v];
                p = lower_bound(adj + b, (uint32_t)(off[v + 1] - b), u);
            }
            pl[a + i] = p;
            acc += p;
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            hv[u] = h;
            wv[u] = acc;
        }
    }
}

// Warp per vertex u: its lower-rank prefix edges get internal ids
// hoff[u] .. hoff[u] + hv[u] - 1.
__global__ void k_newid(const uint64_t *off, const uint32_t *eid, const uint32_t *hv,
                        const uint32_t *hoff, uint32_t n, uint32_t *newid) {
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t u = warp; u < n; u += nwarps) {
        const uint64_t a = off[u];
        const uint32_t h = hv[u], base = hoff[u];
        for (uint32_t i = lane; i < h; i += 32) newid[eid[a + i]] = base + i;
    }
}

__global__ void k_relabel(uint32_t *eid, uint64_t na, const uint32_t *newid) {
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < na;
         j += (uint64_t)gridDim.x * blockDim.x)
        eid[j] = newid[eid[j]];
}

template <typename T>
__global__ void k_gather(const T *in, const uint32_t *newid, T *out, uint64_t m) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < m;
         e += (uint64_t)gridDim.x * blockDim.x)
        out[e] = in[newid[e]];
}

__global__ void k_scatter_u8(const uint8_t *in, const uint32_t *newid, uint8_t *out, uint64_t m) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < m;
         e += (uint64_t)gridDim.x * blockDim.x)
        out[newid[e]] = in[e];
}

inline unsigned grid_for(uint64_t items, int threads, unsigned cap = 152 * 32) {
    uint64_t g = (items + threads - 1) / threads;
    if (g == 0) g = 1;
    return (unsigned)(g < cap ? g : cap);
}

// Relabels a concatenation of independent graphs into one disjoint union:
// edge i of graph g gets its upper id shifted by offU[g] and its lower id by
// offL[g].  Ids are checked against the graph's own layer sizes first; the
// lowest failing graph index is kept in *bad_graph.
__global__ void k_union(int32_t *edges, uint64_t m_total, const uint64_t *goff, uint32_t ng,
                        const uint32_t *offU, const uint32_t *offL, const uint32_t *gnU,
                        const uint32_t *gnL, uint32_t *err, uint32_t *bad_graph) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m_total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t lo = 0, hi = ng;  // largest g with goff[g] <= i
        while (hi - lo > 1) {
            uint32_t mid = (lo + hi) >> 1;
            if (goff[mid] <= i) lo = mid; else hi = mid;
        }
        const uint32_t g = lo;
        int2 e = reinterpret_cast<int2 *>(edges)[i];
        if (e.x < 0 || e.y < 0 || (uint32_t)e.x >= gnU[g] || (uint32_t)e.y >= gnL[g]) {
            atomicOr(err, kErrRange);
            atomicMin(bad_graph, g);
            continue;
        }
        e.x += (int32_t)offU[g];
        e.y += (int32_t)offL[g];
        reinterpret_cast<int2 *>(edges)[i] = e;
    }
}

}  // namespace

cudaError_t union_edges(int32_t *d_edges, uint64_t m_total, const uint64_t *d_goff, uint32_t ng,
                        const uint32_t *d_offU, const uint32_t *d_offL, const uint32_t *d_nU,
                        const uint32_t *d_nL, uint32_t *err_word, uint32_t *bad_graph, Alloc &al) {
    if (m_total == 0) return cudaSuccess;
    k_union<<<grid_for(m_total, 256), 256, 0, al.stream>>>(d_edges, m_total, d_goff, ng, d_offU,
                                                           d_offL, d_nU, d_nL, err_word, bad_graph);
    al.launches++;
    return cudaGetLastError();
}

cudaError_t build_csr(const int32_t *d_edges, uint64_t m, uint32_t nU, uint32_t nL, uint32_t flags,
                      Csr &g, uint32_t *err_word, Alloc &al, const GraphSplit *split) {
    const uint32_t n = nU + nL;
    g.n = n;
    g.m = m;
    g.cnt_n = n;
    // graph-by-graph ranking when graph and degree fit one 32-bit key
    const int dbits = split ? bits_for(split->max_n) : 0;
    const int gbits = split ? bits_for(split->ng > 0 ? split->ng - 1 : 0) : 0;
    const bool by_graph = split && split->ng > 1 && dbits + gbits <= 32 && dbits < 32;
    uint32_t *deg = al.get<uint32_t>(n);
    uint32_t *order = al.get<uint32_t>(n);
    uint32_t *tk = al.get<uint32_t>(n);
    uint32_t *tv = al.get<uint32_t>(n);
    uint32_t *rank = al.get<uint32_t>(n);
    uint64_t *degr = al.get<uint64_t>((size_t)n + 1);
    g.off = al.get<uint64_t>((size_t)n + 1);
    if (al.err != cudaSuccess) return al.err;
    al.mark(kPhCsr, false);
    BT_CUDA(cudaMemsetAsync(deg, 0, sizeof(uint32_t) * n, al.stream));
    k_degree<<<grid_for(m, 256), 256, 0, al.stream>>>(d_edges, m, nU, nL, flags, deg, err_word);
    al.launches++;
    k_iota<<<grid_for(n, 256), 256, 0, al.stream>>>(order, n);
    al.launches++;
    if (by_graph) {
        uint32_t *gkey = al.get<uint32_t>(n);
        g.vbase = al.get<uint32_t>(n);
        if (al.err != cudaSuccess) return al.err;
        k_graph_keys<<<grid_for(n, 256), 256, 0, al.stream>>>(deg, n, nU, nL, flags, split->ng, split->offU,
                                                              split->offL, dbits, gkey);
        al.launches++;
        BT_CUDA(radix_sort_u32(gkey, order, tk, tv, n, dbits + gbits, al));
        k_graph_rank<<<grid_for(n, 256), 256, 0, al.stream>>>(gkey, n, dbits, split->offU, split->offL, deg,
                                                              g.vbase);
        al.launches++;
        al.put(gkey);
        g.cnt_n = split->max_n;
    } else {
        // degrees are <= max(nU, nL); a stable sort on degree keeps ties in id order
        BT_CUDA(radix_sort_u32(deg, order, tk, tv, n, bits_for(nU > nL ? nU : nL), al));
    }
    // deg now holds the degrees in rank order
    BT_CUDA(cudaMemsetAsync(degr, 0, sizeof(uint64_t) * ((size_t)n + 1), al.stream));
    k_rank<<<grid_for(n, 256), 256, 0, al.stream>>>(order, deg, n, rank, degr);
    al.launches++;
    BT_CUDA(cudaGetLastError());
    al.put(tk);
    al.put(tv);
    // off = exclusive scan of degree by rank
    BT_CUDA(exclusive_scan_u64(degr, g.off, (size_t)n + 1, nullptr, al));

    const uint64_t na = 2 * m;
    uint64_t *keys = al.get<uint64_t>(na);
    uint32_t *vals = al.get<uint32_t>(na);
    uint64_t *k2 = al.get<uint64_t>(na);
    uint32_t *v2 = al.get<uint32_t>(na);
    if (al.err != cudaSuccess) return al.err;
    k_arcs<<<grid_for(m, 256), 256, 0, al.stream>>>(d_edges, m, nU, nL, flags, rank, n, keys, vals);
    al.launches++;
    BT_CUDA(radix_sort_u64(keys, vals, k2, v2, na, bits_for((uint64_t)n * n - 1), al));
    al.put(k2);
    al.put(v2);
    g.adj = al.get<uint32_t>(na);
    g.eid = al.get<uint32_t>(na);
    g.pl = al.get<uint32_t>(na);
    g.hv = al.get<uint32_t>(n);
    g.wv = al.get<uint64_t>(n);
    if (al.err != cudaSuccess) return al.err;
    k_csr_fill<<<grid_for(na, 256), 256, 0, al.stream>>>(keys, vals, na, n, g.adj, g.eid, err_word);
    al.launches++;
    al.put(keys);
    al.put(vals);
    k_wedge_prefix<<<grid_for((uint64_t)n * 32, 256), 256, 0, al.stream>>>(g.off, g.adj, n, g.hv,
                                                                           g.pl, g.wv);
    al.launches++;
    // internal edge ids grouped by the higher-ranked endpoint
    {
        uint32_t *hoff = al.get<uint32_t>(n);
        g.newid = al.get<uint32_t>(m);
        if (al.err != cudaSuccess) return al.err;
        BT_CUDA(exclusive_scan_u32(g.hv, hoff, n, nullptr, al));
        k_newid<<<grid_for((uint64_t)n * 32, 256), 256, 0, al.stream>>>(g.off, g.eid, g.hv, hoff, n,
                                                                         g.newid);
        al.launches++;
        k_relabel<<<grid_for(na, 256), 256, 0, al.stream>>>(g.eid, na, g.newid);
        al.launches++;
        al.put(hoff);
    }
    al.mark(kPhCsr, true);
    al.put(deg);
    al.put(order);
    al.put(rank);
    al.put(degr);
    return cudaGetLastError();
}

cudaError_t gather_u64(const uint64_t *in, const uint32_t *newid, uint64_t *out, uint64_t m, Alloc &al) {
    if (m == 0) return cudaSuccess;
    k_gather<uint64_t><<<grid_for(m, 256), 256, 0, al.stream>>>(in, newid, out, m);
    al.launches++;
    return cudaGetLastError();
}

cudaError_t gather_u32(const uint32_t *in, const uint32_t *newid, uint32_t *out, uint64_t m, Alloc &al) {
    if (m == 0) return cudaSuccess;
    k_gather<uint32_t><<<grid_for(m, 256), 256, 0, al.stream>>>(in, newid, out, m);
    al.launches++;
    return cudaGetLastError();
}

cudaError_t scatter_u8(const uint8_t *in, const uint32_t *newid, uint8_t *out, uint64_t m, Alloc &al) {
    if (m == 0) return cudaSuccess;
    k_scatter_u8<<<grid_for(m, 256), 256, 0, al.stream>>>(in, newid, out, m);
    al.launches++;
    return cudaGetLastError();
}

// Frees the CSR (and newid unless a caller took it over).
void free_csr(Csr &g, Alloc &al) {
    al.put(g.newid);
    al.put(g.vbase);
    al.put(g.off);
    al.put(g.adj);
    al.put(g.eid);
    al.put(g.pl);
    al.put(g.hv);
    al.put(g.wv);
    g = Csr{};
}

}  // namespace bt
