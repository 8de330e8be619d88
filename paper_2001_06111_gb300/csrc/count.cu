// Butterfly support counting and BE-Index construction by priority-obeyed
// wedge enumeration (Section IV-B, Alg. 3; Defs. 7, 8, 10).
//
// For a start vertex u (processed in rank space, so p(x) < p(u) <=> x < u):
//   pass A  for v in N(u), v < u; for w in N(v), w < u:  cnt[w] += 1
//           -> cnt[w] = |N(u) ∩ N(w) ∩ {x < u}|  (Alg. 3, the first wedge loop)
//   pass B  every wedge (u,v,w) with c = cnt[w] >= 2 lies in the maximal
//           priority-obeyed bloom anchored by (u,w), a c-bloom (Lemma 7); each
//           of its two edges is in c-1 of the bloom's butterflies (Lemma 2)
//           and every butterfly lies in exactly one such bloom (Lemma 3), so
//           support(u,v) += c-1 and support(v,w) += c-1 sums to the support.
//   emit    the bloom gets bloom number c, and the wedge becomes one twin
//           pair ((u,v),(v,w)) linked to it (Alg. 3, the second wedge loop).
//
// Work layout: persistent blocks pull start vertices from a global queue in
// decreasing rank (heaviest first).  A block enumerates the wedges of its
// vertex in chunks of NT middle vertices (NT = block size, picked by the
// batch autotuner from 256, 512, 1024): a block scan of the per-arc
// prefix lengths flattens the chunk's wedges, so every thread handles whole
// wedges regardless of the degree skew.  Counters are a dense per-block
// array indexed by rank, kept at zero between vertices: when u has fewer
// than 2^16 lower-ranked neighbours and the arrays are small, a counter's
// word also counts its readers in pass B and the last reader clears it;
// otherwise a third walk (pass C) clears the counters.  Emit keeps one 64-bit word per counter (count and
// claimed bloom) so each wedge touches one memory sector per walk.
#include "bt_device.cuh"
#include "bt_internal.cuh"

namespace bt {
namespace {

template <int NT>
struct Chunk {
    uint32_t off[NT + 1];  // exclusive prefix of wedge counts; off[NT] = total
    uint32_t v[NT];        // middle vertex (rank)
    uint32_t e[NT];        // edge id of (u, v)
};

// Loads middle vertices [c0, c0 + NT) of start vertex u.  Returns the
// number of wedges in the chunk.  Contains __syncthreads().
template <int NT>
__device__ __forceinline__ uint32_t load_chunk(Chunk<NT> &ch, const uint32_t *adj, const uint32_t *eid,
                                               const uint32_t *pl, uint64_t a, uint32_t h,
                                               uint32_t c0) {
    uint32_t i = c0 + threadIdx.x;
    uint32_t p = 0, v = 0, e = 0;
    if (i < h) {
        p = pl[a + i];
        v = adj[a + i];
        e = eid[a + i];
    }
    uint32_t tot;
    uint32_t ex = dev::block_excl_scan<uint32_t>(p, &tot);
    ch.off[threadIdx.x] = ex;
    ch.v[threadIdx.x] = v;
    ch.e[threadIdx.x] = e;
    if (threadIdx.x == 0) ch.off[NT] = tot;
    __syncthreads();
    return tot;
}

// Wedge t of the chunk -> (chunk slot vi, arc index of (v, w) in the CSR).
template <int NT>
__device__ __forceinline__ uint64_t wedge_arc(const Chunk<NT> &ch, const uint64_t *off, uint32_t t,
                                              uint32_t &vi) {
    vi = dev::last_le_u32(ch.off, NT, t);
    return off[ch.v[vi]] + (t - ch.off[vi]);
}

// Next start vertex of the rank range [lo, hi), highest rank first.
__device__ __forceinline__ uint32_t next_vertex(uint32_t *queue, uint32_t lo, uint32_t hi, uint32_t *s_q) {
    if (threadIdx.x == 0) *s_q = atomicAdd(queue, 1u);
    __syncthreads();
    uint32_t qi = *s_q;
    __syncthreads();
    return qi < hi - lo ? hi - 1 - qi : 0xFFFFFFFFu;
}

__device__ __forceinline__ uint32_t ld_cg(const uint32_t *p) { return __ldcg(p); }

// Pass A over all chunks of u.
template <int NT>
__device__ void pass_count(Chunk<NT> &ch, const uint64_t *off, const uint32_t *adj,
                           const uint32_t *eid, const uint32_t *pl, uint64_t a, uint32_t h,
                           uint32_t *cnt, uint32_t vb) {
    for (uint32_t c0 = 0; c0 < h; c0 += NT) {
        uint32_t T = load_chunk(ch, adj, eid, pl, a, h, c0);
        for (uint32_t t = threadIdx.x; t < T; t += NT) {
            uint32_t vi;
            uint64_t arc = wedge_arc(ch, off, t, vi);
            atomicAdd(&cnt[adj[arc] - vb], 1u);
        }
        __syncthreads();
    }
}

// Pass A on emit's packed words (count in the low 32 bits).
template <int NT>
__device__ void pass_count64(Chunk<NT> &ch, const uint64_t *off, const uint32_t *adj,
                             const uint32_t *eid, const uint32_t *pl, uint64_t a, uint32_t h,
                             unsigned long long *cw, uint32_t vb) {
    for (uint32_t c0 = 0; c0 < h; c0 += NT) {
        uint32_t T = load_chunk(ch, adj, eid, pl, a, h, c0);
        for (uint32_t t = threadIdx.x; t < T; t += NT) {
            uint32_t vi;
            uint64_t arc = wedge_arc(ch, off, t, vi);
            atomicAdd(&cw[adj[arc] - vb], 1ull);
        }
        __syncthreads();
    }
}

template <bool kIndex, int NT>
__global__ void __launch_bounds__(NT) k_count(
    const uint64_t *__restrict__ off, const uint32_t *__restrict__ adj,
    const uint32_t *__restrict__ eid, const uint32_t *__restrict__ hv,
    const uint32_t *__restrict__ pl, const uint64_t *__restrict__ wv, uint32_t lo, uint32_t hi,
    const uint32_t *__restrict__ vbase, uint32_t cn,
    uint32_t *cnt_all, unsigned long long *support, uint32_t *inc_cnt, uint64_t *w2v,
    uint64_t *nbv, unsigned long long *totals, uint32_t *queue, const uint8_t *__restrict__ assigned,
    bool pack) {
    __shared__ Chunk<NT> ch;
    __shared__ unsigned long long s_acc[NT];
    __shared__ uint32_t s_inc[NT];
    __shared__ uint32_t s_q;
    // this block's counters: the w of a start vertex u lie in u's graph, at
    // w - vbase[u] (vbase null: one graph)
    uint32_t *cnt = cnt_all + (size_t)blockIdx.x * cn;
    s_acc[threadIdx.x] = 0;
    s_inc[threadIdx.x] = 0;
    unsigned long long bf_total = 0;
    for (;;) {
        uint32_t u = next_vertex(queue, lo, hi, &s_q);
        if (u == 0xFFFFFFFFu) break;
        if (wv[u] == 0) {
            if (kIndex && threadIdx.x == 0) {
                w2v[u] = 0;
                nbv[u] = 0;
            }
            continue;
        }
        const uint64_t a = off[u];
        const uint32_t h = hv[u];
        const uint32_t vb = vbase ? vbase[u] : 0u;
        pass_count(ch, off, adj, eid, pl, a, h, cnt, vb);
        // a counter never exceeds h (one per middle vertex): when h < 2^16 the
        // count keeps the low half of its word and pass B counts its readers
        // in the high half, so the last reader clears the word (no pass C).
        // Only while the counter arrays are small (pack): when they live in
        // DRAM the returning atomic lengthens pass B more than pass C costs.
        const bool packed = pack && h < 0x10000u;
        unsigned long long nb_local = 0;
        // pass B: attribute c-1 to both edges of every wedge in a bloom
        unsigned long long w2_local = 0;
        for (uint32_t c0 = 0; c0 < h; c0 += NT) {
            uint32_t T = load_chunk(ch, adj, eid, pl, a, h, c0);
            for (uint32_t t = threadIdx.x; t < T; t += NT) {
                uint32_t vi;
                uint64_t arc = wedge_arc(ch, off, t, vi);
                uint32_t *cp = &cnt[adj[arc] - vb];
                uint32_t c;
                if (packed) {
                    const uint32_t old = atomicAdd(cp, 1u << 16);
                    c = old & 0xFFFFu;
                    if ((old >> 16) + 1u == c) {
                        // the last of the c wedges: the bloom is counted once
                        *cp = 0u;
                        if (c >= 2) {
                            ++nb_local;
                            bf_total += (unsigned long long)c * (c - 1) / 2;
                        }
                    }
                } else {
                    c = ld_cg(cp);
                }
                if (c >= 2) {
                    uint32_t evw = eid[arc];
                    atomicAdd(&support[evw], (unsigned long long)(c - 1));
                    atomicAdd(&s_acc[vi], (unsigned long long)(c - 1));
                    if (kIndex) {
                        // edges already assigned (progressive compression) get no links
                        if (!assigned || !assigned[evw]) atomicAdd(&inc_cnt[evw], 1u);
                        if (!assigned || !assigned[ch.e[vi]]) atomicAdd(&s_inc[vi], 1u);
                        ++w2_local;
                    }
                }
            }
            __syncthreads();
            if (s_acc[threadIdx.x]) {
                atomicAdd(&support[ch.e[threadIdx.x]], s_acc[threadIdx.x]);
                s_acc[threadIdx.x] = 0;
            }
            if (kIndex && s_inc[threadIdx.x]) {
                atomicAdd(&inc_cnt[ch.e[threadIdx.x]], s_inc[threadIdx.x]);
                s_inc[threadIdx.x] = 0;
            }
            __syncthreads();
        }
        // pass C: reset counters; the first thread to clear a bloom counts it
        for (uint32_t c0 = 0; c0 < (packed ? 0u : h); c0 += NT) {
            uint32_t T = load_chunk(ch, adj, eid, pl, a, h, c0);
            for (uint32_t t = threadIdx.x; t < T; t += NT) {
                uint32_t vi;
                uint64_t arc = wedge_arc(ch, off, t, vi);
                uint32_t old = atomicExch(&cnt[adj[arc] - vb], 0u);
                if (old >= 2) {
                    ++nb_local;
                    bf_total += (unsigned long long)old * (old - 1) / 2;
                }
            }
            __syncthreads();
        }
        if (kIndex) {
            unsigned long long w2s = dev::block_sum(w2_local);
            unsigned long long nbs = dev::block_sum(nb_local);
            if (threadIdx.x == 0) {
                w2v[u] = w2s;
                nbv[u] = nbs;
            }
        }
    }
    bf_total = dev::block_sum(bf_total);
    if (threadIdx.x == 0 && bf_total) atomicAdd(&totals[0], bf_total);
}

// Emit the index: blooms (bloom number, first pair), twin pairs and the
// per-edge link lists.  The dense per-block array holds one 64-bit word per
// end vertex: the wedge count in the low half and, once the bloom is claimed,
// 2 + its index among the vertex's blooms in the high half, so a wedge reads
// and updates one word (one memory sector) in every pass.
template <int NT>
__global__ void __launch_bounds__(NT) k_emit(
    const uint64_t *__restrict__ off, const uint32_t *__restrict__ adj,
    const uint32_t *__restrict__ eid, const uint32_t *__restrict__ hv,
    const uint32_t *__restrict__ pl, const uint64_t *__restrict__ wv, uint32_t n,
    const uint32_t *__restrict__ vbase, uint32_t cn,
    unsigned long long *cw_all, const uint64_t *__restrict__ bloom_base,
    const uint64_t *__restrict__ pair_base, const uint64_t *__restrict__ inc_off,
    uint32_t *inc_fill, uint32_t *bloom_k, uint32_t *bloom_off, uint2 *pairs,
    uint2 *inc, uint32_t *queue, const uint8_t *__restrict__ assigned) {
    __shared__ Chunk<NT> ch;
    __shared__ uint32_t s_q;
    // bloom count (high 32 bits) and pair count (low 32 bits) of the vertex,
    // advanced by one atomic so that pair ranges follow bloom ids
    __shared__ unsigned long long s_alloc;
    unsigned long long *cw = cw_all + (size_t)blockIdx.x * cn;
    for (;;) {
        uint32_t u = next_vertex(queue, 0u, n, &s_q);
        if (u == 0xFFFFFFFFu) break;
        if (wv[u] == 0) continue;
        const uint64_t a = off[u];
        const uint32_t h = hv[u];
        const uint64_t bb = bloom_base[u];
        const uint64_t pb = pair_base[u];
        const uint32_t vb = vbase ? vbase[u] : 0u;
        if (threadIdx.x == 0) s_alloc = 0;
        pass_count64(ch, off, adj, eid, pl, a, h, cw, vb);
        // claim: one thread per bloom allocates its id and pair range
        for (uint32_t c0 = 0; c0 < h; c0 += NT) {
            uint32_t T = load_chunk(ch, adj, eid, pl, a, h, c0);
            for (uint32_t t = threadIdx.x; t < T; t += NT) {
                uint32_t vi;
                uint64_t arc = wedge_arc(ch, off, t, vi);
                const uint32_t w = adj[arc] - vb;  // counter index
                const unsigned long long x = __ldcg(&cw[w]);
                const uint32_t c = (uint32_t)x;
                // a single wedge is the only reader of its word: clear it now
                if (c == 1u) cw[w] = 0ull;
                if (c >= 2 && atomicCAS(&cw[w], (unsigned long long)c, 1ull << 32 | c) == (unsigned long long)c) {
                    unsigned long long old = atomicAdd(&s_alloc, (1ull << 32) | c);
                    uint32_t j = (uint32_t)(old >> 32);
                    uint32_t p = (uint32_t)old;
                    uint64_t B = bb + j;
                    bloom_k[B] = c;
                    bloom_off[B] = (uint32_t)(pb + p);
                    atomicExch(&cw[w], (unsigned long long)(j + 2u) << 32 | c);
                }
            }
            __syncthreads();
        }
        // place each bloom wedge as a twin pair and link both edges to it
        for (uint32_t c0 = 0; c0 < h; c0 += NT) {
            uint32_t T = load_chunk(ch, adj, eid, pl, a, h, c0);
            for (uint32_t t = threadIdx.x; t < T; t += NT) {
                uint32_t vi;
                uint64_t arc = wedge_arc(ch, off, t, vi);
                const uint32_t w = adj[arc] - vb;  // counter index
                const uint32_t x = (uint32_t)(__ldcg(&cw[w]) >> 32);
                if (x >= 2) {
                    uint64_t B = bb + (x - 2);
                    // the low half counts down the bloom's wedges still to place
                    uint32_t pos = (uint32_t)atomicAdd(&cw[w], ~0ull) - 1u;
                    // the last wedge of the bloom comes after every read of the
                    // word (each precedes its own decrement): clear it
                    if (pos == 0u) cw[w] = 0ull;
                    uint32_t slot = ld_cg(&bloom_off[B]) + pos;
                    uint32_t euv = ch.e[vi], evw = eid[arc];
                    const bool fu = assigned && assigned[euv], fw = assigned && assigned[evw];
                    // an assigned edge is flagged in bit 31 and gets no link
                    pairs[slot] = make_uint2(euv | (fu ? 0x80000000u : 0u), evw | (fw ? 0x80000000u : 0u));
                    // each link carries its bloom and which member of the pair the edge is
                    if (!fu) {
                        uint32_t q1 = atomicAdd(&inc_fill[euv], 1u);
                        inc[inc_off[euv] + q1] = make_uint2(slot, (uint32_t)B);
                    }
                    if (!fw) {
                        uint32_t q2 = atomicAdd(&inc_fill[evw], 1u);
                        inc[inc_off[evw] + q2] = make_uint2(slot, (uint32_t)B | 0x80000000u);
                    }
                }
            }
            __syncthreads();
        }
    }
}

template <int NT>
int blocks_per_sm_count() {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_count<true, NT>, NT, 0);
    return b > 0 ? b : 1;
}

int blocks_per_sm_for(int nt) {
    return nt == 256 ? blocks_per_sm_count<256>()
                     : nt == 1024 ? blocks_per_sm_count<1024>() : blocks_per_sm_count<512>();
}

template <int NT>
void launch_count(bool index, unsigned blocks, const Csr &g, uint32_t lo, uint32_t hi, uint32_t *cnt,
                  unsigned long long *sup, CountOut &o, unsigned long long *totals, uint32_t *queue,
                  cudaStream_t st) {
    // two walks per vertex while all blocks' counter arrays total at most
    // 1 GiB (2M-edge graph, 0.34 GB: 6.98 -> 6.47 ms); three above it
    // (30M-edge graph, 3 GB: 267-274 against 305-318 ms with two)
    const bool pack = (uint64_t)blocks * g.cnt_n * sizeof(uint32_t) <= (1ull << 30);
    if (index)
        k_count<true, NT><<<blocks, NT, 0, st>>>(g.off, g.adj, g.eid, g.hv, g.pl, g.wv, lo, hi, g.vbase, g.cnt_n, cnt,
                                                  sup, o.inc_cnt, o.w2v, o.nbv, totals, queue, o.assigned, pack);
    else
        k_count<false, NT><<<blocks, NT, 0, st>>>(g.off, g.adj, g.eid, g.hv, g.pl, g.wv, lo, hi, g.vbase, g.cnt_n, cnt,
                                                   sup, nullptr, nullptr, nullptr, totals, queue, nullptr, pack);
}

}  // namespace

cudaError_t count_wedges(const Csr &g, CountOut &o, int num_sms, Alloc &al, int nt, uint32_t lo, uint32_t hi) {
    const bool index = o.inc_cnt != nullptr;
    if (hi > g.n) hi = g.n;
    if (lo > hi) lo = hi;
    if (nt != 256 && nt != 1024) nt = 512;
    int bps = blocks_per_sm_for(nt);
    unsigned blocks = (unsigned)(num_sms * bps);
    uint32_t *cnt = al.get<uint32_t>((size_t)blocks * g.cnt_n);
    uint32_t *queue = al.get<uint32_t>(1);
    unsigned long long *totals = al.get<unsigned long long>(1);
    if (al.err != cudaSuccess) return al.err;
    BT_CUDA(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * (size_t)blocks * g.cnt_n, al.stream));
    BT_CUDA(cudaMemsetAsync(queue, 0, sizeof(uint32_t), al.stream));
    BT_CUDA(cudaMemsetAsync(totals, 0, sizeof(unsigned long long), al.stream));
    BT_CUDA(cudaMemsetAsync(o.support, 0, sizeof(uint64_t) * g.m, al.stream));
    if (index) BT_CUDA(cudaMemsetAsync(o.inc_cnt, 0, sizeof(uint32_t) * g.m, al.stream));
    auto *sup = reinterpret_cast<unsigned long long *>(o.support);
    al.mark(kPhCount, false);
    if (nt == 256) launch_count<256>(index, blocks, g, lo, hi, cnt, sup, o, totals, queue, al.stream);
    else if (nt == 1024) launch_count<1024>(index, blocks, g, lo, hi, cnt, sup, o, totals, queue, al.stream);
    else launch_count<512>(index, blocks, g, lo, hi, cnt, sup, o, totals, queue, al.stream);
    al.launches++;
    al.mark(kPhCount, true);
    BT_CUDA(cudaGetLastError());
    o.butterflies_dev = totals;
    al.put(cnt);
    al.put(queue);
    return cudaSuccess;
}

cudaError_t emit_index(const Csr &g, const CountOut &c, Index &ix, int num_sms, Alloc &al,
                       cudaStream_t stream, int nt) {
    if (nt != 256 && nt != 1024) nt = 512;
    const uint32_t n = g.n;
    const uint64_t m = g.m;
    ix.m = m;
    // layout prefix sums
    uint64_t *bloom_base = al.get<uint64_t>(n);
    uint64_t *pair_base = al.get<uint64_t>(n);
    uint64_t *tot = al.get<uint64_t>(3);
    uint64_t *incc64 = al.get<uint64_t>(m + 1);
    ix.inc_off = al.get<uint64_t>(m + 1);
    if (al.err != cudaSuccess) return al.err;
    BT_CUDA(exclusive_scan_u64(c.nbv, bloom_base, n, tot + 0, al));
    BT_CUDA(exclusive_scan_u64(c.w2v, pair_base, n, tot + 1, al));
    BT_CUDA(widen_u32(c.inc_cnt, incc64, m, al));
    BT_CUDA(cudaMemsetAsync(incc64 + m, 0, sizeof(uint64_t), al.stream));
    BT_CUDA(exclusive_scan_u64(incc64, ix.inc_off, m + 1, tot + 2, al));
    al.put(incc64);
    uint64_t h_tot[3];
    BT_CUDA(cudaMemcpyAsync(h_tot, tot, sizeof(h_tot), cudaMemcpyDeviceToHost, stream));
    BT_CUDA(cudaStreamSynchronize(stream));
    ix.nb = h_tot[0];
    ix.w2 = h_tot[1];
    ix.links = h_tot[2];  // 2 w2, less the links of assigned edges in a compressed index
    // pair ids are u32; bloom ids keep bit 31 free for the link's side
    if (ix.w2 >= 0xFFFFFFFFull || ix.nb >= 0x80000000ull) {
        al.put(bloom_base);
        al.put(pair_base);
        al.put(tot);
        return cudaErrorInvalidValue;  // reported as overflow by the caller
    }
    ix.bloom_k = al.get<uint32_t>(ix.nb);
    ix.bloom_off = al.get<uint32_t>(ix.nb + 1);
    ix.pairs = al.get<uint2>(ix.w2);
    ix.inc = al.get<uint2>(ix.links);
    uint32_t *inc_fill = al.get<uint32_t>(m);
    // 1024-thread emit blocks: one per SM, so that half as many pairs of
    // dense per-block arrays compete for L2 (measured 5-20 % faster than two
    // per SM; the count kernel keeps two per SM, where one measured slower)
    int bps = nt == 1024 ? 1 : blocks_per_sm_for(nt);
    unsigned blocks = (unsigned)(num_sms * bps);
    unsigned long long *cw = al.get<unsigned long long>((size_t)blocks * g.cnt_n);
    uint32_t *queue = al.get<uint32_t>(1);
    if (al.err != cudaSuccess) return al.err;
    uint32_t w2_32 = (uint32_t)ix.w2;
    BT_CUDA(cudaMemcpyAsync(ix.bloom_off + ix.nb, &w2_32, sizeof(uint32_t), cudaMemcpyHostToDevice,
                            stream));
    BT_CUDA(cudaMemsetAsync(inc_fill, 0, sizeof(uint32_t) * m, al.stream));
    BT_CUDA(cudaMemsetAsync(cw, 0, sizeof(unsigned long long) * (size_t)blocks * g.cnt_n, al.stream));
    BT_CUDA(cudaMemsetAsync(queue, 0, sizeof(uint32_t), al.stream));
    al.mark(kPhEmit, false);
#define BT_EMIT_ARGS                                                                         \
    g.off, g.adj, g.eid, g.hv, g.pl, g.wv, n, g.vbase, g.cnt_n, cw, bloom_base, pair_base, ix.inc_off,  \
        inc_fill, ix.bloom_k, ix.bloom_off, ix.pairs, ix.inc, queue, c.assigned
    if (nt == 256) k_emit<256><<<blocks, 256, 0, al.stream>>>(BT_EMIT_ARGS);
    else if (nt == 1024) k_emit<1024><<<blocks, 1024, 0, al.stream>>>(BT_EMIT_ARGS);
    else k_emit<512><<<blocks, 512, 0, al.stream>>>(BT_EMIT_ARGS);
#undef BT_EMIT_ARGS
    al.launches++;
    al.mark(kPhEmit, true);
    BT_CUDA(cudaGetLastError());
    // the host copy of w2_32 must outlive the async copy
    BT_CUDA(cudaStreamSynchronize(stream));
    al.put(cw);
    al.put(queue);
    al.put(inc_fill);
    al.put(bloom_base);
    al.put(pair_base);
    al.put(tot);
    return cudaSuccess;
}

namespace {
__device__ __forceinline__ uint32_t first_at_least(const uint64_t *pre, uint32_t n, uint64_t t) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = lo + (hi - lo) / 2;
        if (pre[mid] < t) lo = mid + 1; else hi = mid;
    }
    return lo;
}
__global__ void k_rank_bounds(const uint64_t *pre, uint32_t n, uint64_t t0, uint64_t t1, uint32_t *out) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        out[0] = first_at_least(pre, n, t0);
        out[1] = first_at_least(pre, n, t1);
    }
}
}  // namespace

cudaError_t rank_bounds(const uint64_t *pre, uint32_t n, uint64_t t0, uint64_t t1, uint32_t *out, Alloc &al) {
    k_rank_bounds<<<1, 32, 0, al.stream>>>(pre, n, t0, t1, out);
    al.launches++;
    return cudaGetLastError();
}

void free_index(Index &ix, Alloc &al) {
    al.put(ix.newid);
    al.put(ix.bloom_k);
    al.put(ix.bloom_off);
    al.put(ix.pairs);
    al.put(ix.inc_off);
    al.put(ix.inc);
    ix = Index{};
}

}  // namespace bt
