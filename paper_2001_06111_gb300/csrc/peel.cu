// Level-synchronous batch peeling through the BE-Index (Section V-B,
// Alg. 5, BiT-BU++; the <= k frontier rule of Alg. 4).
//
// One round removes the batch S = {unassigned e : support(e) <= k} at once:
//   incidence phase (Alg. 5, the loop over e in S and B in N_I(e)):
//     every live twin pair of a bloom B that holds an edge of S dies once;
//     C(B) counts the dead pairs.  When both twins are in S the one with the
//     smaller edge id owns the pair, so a pair is counted once (the example of
//     Section V-B: three twin pairs of B0 drop its bloom number to 0).  A twin
//     outside S loses all k_B - 1 butterflies it had in B (Lemma 2).
//   bloom phase (Alg. 5, the loop over blooms with C(B) > 0):
//     every edge of a surviving pair of B loses C(B) butterflies (one per
//     dead pair); then k_B -= C(B), so the bloom keeps C(k_B - C, 2)
//     butterflies (Lemma 1).
//   phi(e) = k for e in S.
// k only grows: when no unassigned edge has support <= k, k jumps to the
// minimum remaining support (the batch-edge rule of Lemma 9).  Supports are
// decremented without the max(MBS, .) clamp of Alg. 5; an edge that drops to
// or below k is taken by the next round with the same k, which gives the same
// phi.  An edge joins the next batch exactly when one decrement carries its
// support from above k to <= k, so rounds inside a level never rescan edges.
//
// The whole loop runs in one persistent cooperative kernel (one block per SM
// slot the occupancy allows).  Phases are separated by a grid barrier whose
// wait is bounded by a timer; on timeout the kernel raises an error word and
// every block returns.  Work is split into items of at most kSeg entries: an
// edge of S with a long link list becomes several incidence items, and a
// touched bloom with many pairs several bloom items, so no warp straggles on
// a hub.  A twin pair carries the round it died in; the edges of S race to
// stamp it with atomicCAS, so exactly one of them counts it in C(B) (the
// twin rule above, without reading the twin's state), and the twin
// decrements are applied by the bloom phase, which sees which pairs died in
// this round.  Counters and work lists are double- or triple-buffered by
// round, which leaves two barriers per round.  Data written by other blocks
// during the kernel is read with L2 (.cg) loads.
#include "bt_device.cuh"
#include "bt_internal.cuh"

namespace bt {
namespace {

constexpr int kPeelThreads = 1024;
// entries per work item: SEG = 32 or 64 (template parameter picked by the
// batch autotuner); each lane handles SEG / 32 entries with their loads and
// atomics issued together.
// items with at most kSmall entries are processed by one lane each, larger
// ones by the whole warp.  Lane l of warp w takes item w + l * nwarps (plus
// multiples of 32 * nwarps): a round with fewer items than warps still gives
// every item its own warp, and a large round fills all lanes.
constexpr uint32_t kSmall = 2;
constexpr unsigned long long kBarrierTimeoutNs = 20ull * 1000 * 1000 * 1000;  // 20 s
constexpr uint32_t kErrBarrier = 1u;
constexpr uint32_t kErrRounds = 2u;
constexpr uint32_t kErrPeelOverflow = 4u;

struct Ctl {
    unsigned long long bar_count;  // barrier arrivals (monotonic within a launch)
    unsigned int err;
    unsigned int pad0;
    unsigned int n_items[2];  // incidence items per round parity
    unsigned int n_edges[2];  // frontier edges per round parity
    unsigned int n_bseg[3];   // bloom items per round mod 3
    unsigned int n_alive[2];  // alive list sizes (ping-pong)
    unsigned int n_near[2];   // near-window list sizes (ping-pong)
    unsigned int pad1;
    unsigned long long minsup;   // level-jump minimum over the near window
    unsigned long long minsup2;  // minimum over all alive edges (window rebuild)
    unsigned long long updates;
    unsigned long long slots;  // bloom pair slots visited by the bloom phase
    unsigned long long rounds;
    unsigned long long levels;
    unsigned long long windows;
    unsigned long long kfinal;
};

struct PeelArgs {
    uint64_t m;
    const uint64_t *inc_off;
    const uint32_t *inc;
    const uint2 *pairs;
    const uint32_t *pair_bloom;
    const uint32_t *bloom_off;
    long long *sup;
    uint32_t *state;
    uint32_t *phi;
    uint32_t *died;    // round a twin pair died in (kAlive while alive)
    uint32_t *bk;
    uint32_t *Cb[3];
    uint4 *items[2];   // (edge, first link lo, first link hi, count | head flag << 31)
    uint4 *bseg[3];    // (bloom, first pair, count | head flag << 31, bloom number at round start)
    uint32_t *alive[2];
    uint32_t *near[2];
    uint64_t item_cap;
    Ctl *ctl;
    uint64_t round_limit;
    // progressive compression: peel only the m_active unassigned edges, start
    // at level k_init, and record phi only for levels >= assign_from
    uint64_t m_active;
    long long k_init;
    long long assign_from;
};

// Loop state every thread keeps identically (derived from values read after
// grid barriers).
struct Lvl {
    long long k;    // current level
    long long khi;  // top of the near window: alive edges with support < khi are listed
    uint32_t nq;    // current near list
};

__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ldcg_u32(const uint32_t *p) { return __ldcg(p); }
__device__ __forceinline__ unsigned int ldcg_ui(const unsigned int *p) { return __ldcg(p); }
__device__ __forceinline__ long long ldcg_ll(const long long *p) { return __ldcg(p); }

// Grid-wide barrier over all blocks of a cooperative launch.  Arrivals go
// to one monotonic counter (release); barrier number b completes when the
// counter reaches (b + 1) * gridDim.x, which every block polls (acquire).
// Returns false when the wait timed out or another block raised an error.
__device__ __forceinline__ void arrive_release(unsigned long long *p) {
    asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(p) : "memory");
}
__device__ __forceinline__ unsigned long long load_acquire(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ bool grid_barrier(Ctl *ctl, unsigned long long &bar_no) {
    __syncthreads();
    __shared__ int s_ok;
    const unsigned long long target = (bar_no + 1) * gridDim.x;
    ++bar_no;
    if (threadIdx.x == 0) {
        int ok = 1;
        arrive_release(&ctl->bar_count);
        if (load_acquire(&ctl->bar_count) < target) {
            const unsigned long long t0 = now_ns();
            unsigned int spins = 0;
            while (load_acquire(&ctl->bar_count) < target) {
                if (((++spins) & 63u) == 0) {
                    if (*(volatile unsigned int *)&ctl->err) {
                        ok = 0;
                        break;
                    }
                    if (now_ns() - t0 > kBarrierTimeoutNs) {
                        atomicOr(&ctl->err, kErrBarrier);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Queue edge e (links [ib, ie)) for the round `next_round`: one incidence
// item per kSeg links, each carrying its link range.
template <uint32_t kSeg>
__device__ __forceinline__ void push_edge(const PeelArgs &a, uint32_t e, uint32_t dst,
                                          uint32_t next_round, uint64_t ib, uint64_t ie, long long k) {
    a.state[e] = next_round;
    if (k >= a.assign_from) a.phi[e] = (uint32_t)k;  // e leaves in a batch of this level
    const uint64_t d = ie - ib;
    const uint32_t nseg = d == 0 ? 1u : (uint32_t)((d + kSeg - 1) / kSeg);
    const uint32_t base = atomicAdd(&a.ctl->n_items[dst], nseg);
    for (uint32_t s = 0; s < nseg; ++s) {
        const uint64_t j = ib + (uint64_t)s * kSeg;
        const uint64_t left = d - (uint64_t)s * kSeg;
        const uint32_t cnt = (uint32_t)(left < kSeg ? left : kSeg);
        a.items[dst][base + s] =
            make_uint4(e, (uint32_t)j, (uint32_t)(j >> 32), cnt | (s == 0 ? 0x80000000u : 0u));
    }
    atomicAdd(&a.ctl->n_edges[dst], 1u);
}

__device__ __forceinline__ void push_near(const PeelArgs &a, uint32_t e, uint32_t nq) {
    a.near[nq][atomicAdd(&a.ctl->n_near[nq], 1u)] = e;
}

// Subtract dec from support(e).  Queue e for the next round when this takes
// it from > k to <= k, and list it in the near window when it falls below khi.
template <uint32_t kSeg>
__device__ __forceinline__ void decrement(const PeelArgs &a, uint32_t e, long long dec, const Lvl &L,
                                          uint32_t dst, uint32_t next_round, bool have_range,
                                          uint64_t ib, uint64_t ie) {
    const long long old = (long long)atomicAdd(reinterpret_cast<unsigned long long *>(&a.sup[e]),
                                               (unsigned long long)(-dec));
    const long long now = old - dec;
    if (old > L.k && now <= L.k) {
        if (!have_range) {
            ib = a.inc_off[e];
            ie = a.inc_off[e + 1];
        }
        push_edge<kSeg>(a, e, dst, next_round, ib, ie, L.k);
    }
    if (old >= L.khi && now < L.khi) push_near(a, e, L.nq);
}

// Window above the current minimum: narrow enough that a level jump scans few
// edges at high levels (dense cores hold many edges in a support range), wide
// enough that rebuilds from the full alive list stay rare.
__device__ __forceinline__ long long window_top(long long kmin) {
    long long w = kmin / 64;
    return kmin + (w < 8 ? 8 : w);
}

// Incidence phase, one killed pair of bloom B: count it in C(B) and, for the
// first kill of B this round, queue B's pairs as bloom items (each records the
// bloom number k_B at round start).
template <uint32_t kSeg>
__device__ __forceinline__ void count_kill(const PeelArgs &a, uint32_t *C, uint32_t B, uint32_t c3) {
    const uint32_t bkB = __ldcg(&a.bk[B]);
    const uint32_t bo0 = a.bloom_off[B], bo1 = a.bloom_off[B + 1];
    if (atomicAdd(&C[B], 1u) == 0u) {
        const uint32_t span = bo1 - bo0;
        const uint32_t nseg = (span + kSeg - 1) / kSeg;
        const uint32_t base = atomicAdd(&a.ctl->n_bseg[c3], nseg);
        for (uint32_t s = 0; s < nseg; ++s) {
            const uint32_t left = span - s * kSeg;
            a.bseg[c3][base + s] =
                make_uint4(B, bo0 + s * kSeg, (left < kSeg ? left : kSeg) | (s == 0 ? 0x80000000u : 0u), bkB);
        }
    }
}

// Bloom phase, one pair slot (died stamp d, members pr) of a bloom with c
// pairs killed this round and bloom number kB at round start.
template <uint32_t kSeg>
__device__ __forceinline__ void apply_slot(const PeelArgs &a, uint32_t d, uint2 pr, uint32_t c, uint32_t kB,
                                           const Lvl &L, uint32_t np, uint32_t round,
                                           unsigned long long &upd) {
    // bit 31 flags an edge whose bitruss number is already known: it is never
    // peeled again, so it needs no decrement
    const bool fx = pr.x >> 31, fy = pr.y >> 31;
    const uint32_t ex = pr.x & 0x7FFFFFFFu, ey = pr.y & 0x7FFFFFFFu;
    if (d == kAlive) {
        // a surviving pair: one butterfly lost per dead pair
        if (!fx) decrement<kSeg>(a, ex, c, L, np, round + 1, false, 0, 0);
        if (!fy) decrement<kSeg>(a, ey, c, L, np, round + 1, false, 0, 0);
        upd += (fx ? 0 : 1) + (fy ? 0 : 1);
    } else if (d == round && kB > 1u) {
        // died now: a member outside S loses its k_B - 1 butterflies
        const uint32_t sx = fx ? round : __ldcg(&a.state[ex]);
        const uint32_t sy = fy ? round : __ldcg(&a.state[ey]);
        if (sx != round) {
            decrement<kSeg>(a, ex, (long long)kB - 1, L, np, round + 1, false, 0, 0);
            ++upd;
        }
        if (sy != round) {
            decrement<kSeg>(a, ey, (long long)kB - 1, L, np, round + 1, false, 0, 0);
            ++upd;
        }
    }
}

template <uint32_t kSeg>
__global__ void __launch_bounds__(kPeelThreads, 1) k_peel(PeelArgs a) {
    constexpr uint32_t R = kSeg / 32;  // entries per lane
    const int lane = threadIdx.x & 31;
    const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t nthreads = gridDim.x * blockDim.x;
    Ctl *ctl = a.ctl;
    uint64_t remaining = a.m_active;
    uint32_t round = 0;
    Lvl L{a.k_init, 0, 0};
    uint32_t ap = 0;  // current alive list
    bool level_jump = true;
    unsigned long long upd = 0, slots = 0;
    unsigned long long bar_no = 0;  // barriers passed (identical in every block)

    while (remaining > 0) {
        const uint32_t par = round & 1u, np = par ^ 1u;
        const uint32_t c3 = round % 3u;
        if (round > a.round_limit) {
            if (gtid == 0) atomicOr(&ctl->err, kErrRounds);
            break;
        }
        if (level_jump) {
            // L1: minimum over the near window, compacting it
            {
                const uint32_t nn = ldcg_ui(&ctl->n_near[L.nq]);
                unsigned long long best = ~0ull;
                for (uint32_t i0 = blockIdx.x * blockDim.x; i0 < nn; i0 += nthreads) {
                    const uint32_t i = i0 + threadIdx.x;
                    bool keep = false;
                    uint32_t e = 0;
                    if (i < nn) {
                        e = ldcg_u32(&a.near[L.nq][i]);
                        if (ldcg_u32(&a.state[e]) == kAlive) {
                            keep = true;
                            const unsigned long long sv = (unsigned long long)ldcg_ll(&a.sup[e]);
                            best = sv < best ? sv : best;
                        }
                    }
                    const unsigned int mask = __ballot_sync(0xffffffffu, keep);
                    if (mask) {
                        unsigned int base = 0;
                        if (lane == 0) base = atomicAdd(&ctl->n_near[L.nq ^ 1u], (unsigned)__popc(mask));
                        base = __shfl_sync(0xffffffffu, base, 0);
                        if (keep) a.near[L.nq ^ 1u][base + __popc(mask & ((1u << lane) - 1u))] = e;
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const unsigned long long y = __shfl_xor_sync(0xffffffffu, best, o);
                    best = y < best ? y : best;
                }
                if (lane == 0 && best != ~0ull) atomicMin(&ctl->minsup, best);
            }
            if (!grid_barrier(ctl, bar_no)) break;
            unsigned long long mn = __ldcg(&ctl->minsup);
            L.nq ^= 1u;
            if (gtid == 0) ctl->n_near[L.nq ^ 1u] = 0;
            if (mn == ~0ull) {
                // the window holds no alive edge: rebuild it from all alive edges.
                // W1: overall minimum, compacting the alive list
                const uint32_t na = ldcg_ui(&ctl->n_alive[ap]);
                unsigned long long best = ~0ull;
                for (uint32_t i0 = blockIdx.x * blockDim.x; i0 < na; i0 += nthreads) {
                    const uint32_t i = i0 + threadIdx.x;
                    bool keep = false;
                    uint32_t e = 0;
                    if (i < na) {
                        e = ldcg_u32(&a.alive[ap][i]);
                        if (ldcg_u32(&a.state[e]) == kAlive) {
                            keep = true;
                            const unsigned long long sv = (unsigned long long)ldcg_ll(&a.sup[e]);
                            best = sv < best ? sv : best;
                        }
                    }
                    const unsigned int mask = __ballot_sync(0xffffffffu, keep);
                    if (mask) {
                        unsigned int base = 0;
                        if (lane == 0) base = atomicAdd(&ctl->n_alive[ap ^ 1u], (unsigned)__popc(mask));
                        base = __shfl_sync(0xffffffffu, base, 0);
                        if (keep) a.alive[ap ^ 1u][base + __popc(mask & ((1u << lane) - 1u))] = e;
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const unsigned long long y = __shfl_xor_sync(0xffffffffu, best, o);
                    best = y < best ? y : best;
                }
                if (lane == 0 && best != ~0ull) atomicMin(&ctl->minsup2, best);
                if (!grid_barrier(ctl, bar_no)) break;
                mn = __ldcg(&ctl->minsup2);
                if (mn == ~0ull) break;  // no alive edge: cannot happen while remaining > 0
                L.khi = window_top((long long)mn);
                ap ^= 1u;
                if (gtid == 0) ctl->n_alive[ap ^ 1u] = 0;
                // W2: list every alive edge below the new window top
                const uint32_t na2 = ldcg_ui(&ctl->n_alive[ap]);
                for (uint32_t i = gtid; i < na2; i += nthreads) {
                    const uint32_t e = ldcg_u32(&a.alive[ap][i]);
                    if (ldcg_ll(&a.sup[e]) < L.khi) push_near(a, e, L.nq);
                }
                if (gtid == 0) atomicAdd(&ctl->windows, 1ull);
                if (!grid_barrier(ctl, bar_no)) break;
                if (gtid == 0) ctl->minsup2 = ~0ull;
            }
            if ((long long)mn > L.k) L.k = (long long)mn;
            if ((unsigned long long)L.k > 0xFFFFFFFFull) {
                if (gtid == 0) atomicOr(&ctl->err, kErrPeelOverflow);
                break;
            }
            // L2: the batch is every window edge with support <= k
            const uint32_t nn2 = ldcg_ui(&ctl->n_near[L.nq]);
            for (uint32_t i = gtid; i < nn2; i += nthreads) {
                const uint32_t e = ldcg_u32(&a.near[L.nq][i]);
                if (ldcg_u32(&a.state[e]) == kAlive && ldcg_ll(&a.sup[e]) <= L.k)
                    push_edge<kSeg>(a, e, par, round, a.inc_off[e], a.inc_off[e + 1], L.k);
            }
            if (gtid == 0) atomicAdd(&ctl->levels, 1ull);
            if (!grid_barrier(ctl, bar_no)) break;
            if (gtid == 0) ctl->minsup = ~0ull;
        }

        // ---------------- incidence phase
        uint32_t *C = a.Cb[c3];
        // read before the barrier below: block 0 clears it in the bloom phase
        const uint32_t n_edges = ldcg_ui(&ctl->n_edges[par]);
        {
            const uint32_t n_items = ldcg_ui(&ctl->n_items[par]);
            if (gtid == 0) ctl->n_bseg[(c3 + 1u) % 3u] = 0;
            for (uint32_t base = gwarp; base < n_items; base += nwarps * 32u) {
                const uint32_t i = base + lane * nwarps;
                const uint4 it = i < n_items ? __ldcg(&a.items[par][i]) : make_uint4(0, 0, 0, 0);
                const uint32_t cnt = it.w & 0x7FFFFFFFu;
                if (cnt <= kSmall) {
                    // this lane's own item: its links' loads and stamps go out together
                    const uint64_t j0 = (uint64_t)it.z << 32 | it.y;
                    uint32_t p[kSmall], B[kSmall];
                    bool won[kSmall];
#pragma unroll
                    for (uint32_t r = 0; r < kSmall; ++r) {
                        won[r] = r < cnt;
                        p[r] = won[r] ? a.inc[j0 + r] : 0u;
                    }
#pragma unroll
                    for (uint32_t r = 0; r < kSmall; ++r)
                        if (won[r]) B[r] = a.pair_bloom[p[r]];
                    // the first edge of S to stamp a pair kills it (once)
#pragma unroll
                    for (uint32_t r = 0; r < kSmall; ++r)
                        if (won[r]) won[r] = atomicCAS(&a.died[p[r]], kAlive, round) == kAlive;
#pragma unroll
                    for (uint32_t r = 0; r < kSmall; ++r)
                        if (won[r]) count_kill<kSeg>(a, C, B[r], c3);
                }
                // items with many links: the whole warp, one item at a time
                unsigned big = __ballot_sync(0xffffffffu, cnt > kSmall);
                while (big) {
                    const int src = __ffs(big) - 1;
                    big &= big - 1u;
                    const uint32_t bcnt = __shfl_sync(0xffffffffu, cnt, src);
                    const uint32_t jlo = __shfl_sync(0xffffffffu, it.y, src);
                    const uint32_t jhi = __shfl_sync(0xffffffffu, it.z, src);
                    const uint64_t j0 = ((uint64_t)jhi << 32 | jlo) + lane;
                    uint32_t p[R], B[R];
                    bool won[R];
#pragma unroll
                    for (uint32_t r = 0; r < R; ++r) {
                        won[r] = lane + 32u * r < bcnt;
                        p[r] = won[r] ? a.inc[j0 + 32u * r] : 0u;
                    }
#pragma unroll
                    for (uint32_t r = 0; r < R; ++r)
                        if (won[r]) B[r] = a.pair_bloom[p[r]];
#pragma unroll
                    for (uint32_t r = 0; r < R; ++r)
                        if (won[r]) won[r] = atomicCAS(&a.died[p[r]], kAlive, round) == kAlive;
#pragma unroll
                    for (uint32_t r = 0; r < R; ++r)
                        if (won[r]) count_kill<kSeg>(a, C, B[r], c3);
                }
            }
        }
        if (!grid_barrier(ctl, bar_no)) break;

        // ---------------- bloom phase
        if (gtid == 0) {
            ctl->n_items[par] = 0;
            ctl->n_edges[par] = 0;
        }
        {
            const uint32_t n_bseg = ldcg_ui(&ctl->n_bseg[c3]);
            for (uint32_t base = gwarp; base < n_bseg; base += nwarps * 32u) {
                const uint32_t i = base + lane * nwarps;
                const uint4 it = i < n_bseg ? __ldcg(&a.bseg[c3][i]) : make_uint4(0, 0, 0, 0);
                const uint32_t cnt = it.z & 0x7FFFFFFFu;
                const uint32_t c = cnt ? __ldcg(&C[it.x]) : 0u;
                if (cnt && (it.z >> 31)) a.bk[it.x] = it.w - c;
                slots += cnt;
                if (cnt <= kSmall) {
                    uint32_t d[kSmall];
                    uint2 pr[kSmall];
#pragma unroll
                    for (uint32_t r = 0; r < kSmall; ++r) {
                        const bool act = r < cnt;
                        d[r] = act ? __ldcg(&a.died[it.y + r]) : round + 1u;  // inactive: no case applies
                        pr[r] = act ? a.pairs[it.y + r] : make_uint2(0, 0);
                    }
#pragma unroll
                    for (uint32_t r = 0; r < kSmall; ++r) apply_slot<kSeg>(a, d[r], pr[r], c, it.w, L, np, round, upd);
                }
                unsigned big = __ballot_sync(0xffffffffu, cnt > kSmall);
                while (big) {
                    const int src = __ffs(big) - 1;
                    big &= big - 1u;
                    const uint32_t bcnt = __shfl_sync(0xffffffffu, cnt, src);
                    const uint32_t p0 = __shfl_sync(0xffffffffu, it.y, src) + lane;
                    const uint32_t kB = __shfl_sync(0xffffffffu, it.w, src);
                    const uint32_t bc = __shfl_sync(0xffffffffu, c, src);
                    uint32_t d[R];
                    uint2 pr[R];
#pragma unroll
                    for (uint32_t r = 0; r < R; ++r) {
                        const bool act = lane + 32u * r < bcnt;
                        d[r] = act ? __ldcg(&a.died[p0 + 32u * r]) : round + 1u;
                        pr[r] = act ? a.pairs[p0 + 32u * r] : make_uint2(0, 0);
                    }
#pragma unroll
                    for (uint32_t r = 0; r < R; ++r) apply_slot<kSeg>(a, d[r], pr[r], bc, kB, L, np, round, upd);
                }
            }
            // clear C of the blooms the previous round touched (threads from
            // the top of the grid, away from the bloom items above)
            const uint32_t cp = (c3 + 2u) % 3u;
            const uint32_t nprev = ldcg_ui(&ctl->n_bseg[cp]);
            for (uint32_t i = nthreads - 1u - gtid; i < nprev; i += nthreads) {
                const uint4 it = __ldcg(&a.bseg[cp][i]);
                if (it.w) a.Cb[cp][it.x] = 0;
            }
        }
        if (!grid_barrier(ctl, bar_no)) break;
        remaining -= n_edges;
        ++round;
        level_jump = remaining > 0 && ldcg_ui(&ctl->n_items[np]) == 0;
    }
    upd = dev::warp_sum(upd);
    if (lane == 0 && upd) atomicAdd(&ctl->updates, upd);
    slots = dev::warp_sum(slots);
    if (lane == 0 && slots) atomicAdd(&ctl->slots, slots);
    if (gtid == 0) {
        ctl->rounds = round;
        ctl->kfinal = (unsigned long long)L.k;
    }
}

// Edges already assigned (mask set) start in the permanent state: never alive,
// never queued.
constexpr uint32_t kPerm = 0xFFFFFFFEu;
__global__ void k_peel_init(const uint64_t *support, uint64_t m, long long *sup, uint32_t *state,
                            const uint8_t *assigned,
                            uint32_t *alive) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m;
         i += (uint64_t)gridDim.x * blockDim.x) {
        sup[i] = (long long)support[i];
        state[i] = (assigned && assigned[i]) ? kPerm : kAlive;
        alive[i] = (uint32_t)i;
    }
}

inline unsigned grid_for(uint64_t items, int threads, unsigned cap) {
    uint64_t g = (items + threads - 1) / threads;
    if (g == 0) g = 1;
    return (unsigned)(g < cap ? g : cap);
}

}  // namespace

cudaError_t peel(const Index &ix, const uint64_t *support, uint32_t *phi_out, PeelResult &res,
                 int num_sms, Alloc &al, int seg, const PeelOpts *opts) {
    const uint32_t kSeg = seg == 64 ? 64u : 32u;
    const uint64_t m = ix.m;
    res = PeelResult{};
    if (m == 0 || (opts && opts->assigned && opts->m_active == 0)) return cudaSuccess;
    const uint64_t item_cap = m + (2 * ix.w2) / kSeg + 2;
    const uint64_t bseg_cap = ix.nb + ix.w2 / kSeg + 2;
    PeelArgs a{};
    a.m = m;
    a.inc_off = ix.inc_off;
    a.inc = ix.inc;
    a.pairs = ix.pairs;
    a.pair_bloom = ix.pair_bloom;
    a.bloom_off = ix.bloom_off;
    a.phi = phi_out;
    a.sup = al.get<long long>(m);
    a.state = al.get<uint32_t>(m);
    a.died = al.get<uint32_t>(ix.w2);
    a.bk = al.get<uint32_t>(ix.nb);
    for (int i = 0; i < 3; ++i) {
        a.Cb[i] = al.get<uint32_t>(ix.nb);
        a.bseg[i] = al.get<uint4>(bseg_cap);
    }
    for (int i = 0; i < 2; ++i) {
        a.items[i] = al.get<uint4>(item_cap);
        a.alive[i] = al.get<uint32_t>(m);
        a.near[i] = al.get<uint32_t>(m);
    }
    a.item_cap = item_cap;
    a.ctl = al.get<Ctl>(1);
    a.round_limit = m + 1;
    a.m_active = (opts && opts->assigned) ? opts->m_active : m;
    a.k_init = opts ? opts->k_init : 0;
    a.assign_from = opts ? opts->assign_from : 0;
    if (al.err != cudaSuccess) return al.err;
    cudaStream_t st = al.stream;
    al.mark(kPhPeel, false);
    k_peel_init<<<grid_for(m, 256, (unsigned)num_sms * 16), 256, 0, st>>>(
        support, m, a.sup, a.state, opts ? opts->assigned : nullptr, a.alive[0]);
    al.launches++;
    BT_CUDA(cudaMemsetAsync(a.died, 0xFF, sizeof(uint32_t) * (ix.w2 ? ix.w2 : 1), st));
    if (ix.nb) {
        BT_CUDA(cudaMemcpyAsync(a.bk, ix.bloom_k, sizeof(uint32_t) * ix.nb, cudaMemcpyDeviceToDevice, st));
        for (int i = 0; i < 3; ++i)
            BT_CUDA(cudaMemsetAsync(a.Cb[i], 0, sizeof(uint32_t) * ix.nb, st));
    }
    Ctl h{};
    h.n_alive[0] = (unsigned int)m;
    h.minsup = ~0ull;
    h.minsup2 = ~0ull;
    BT_CUDA(cudaMemcpyAsync(a.ctl, &h, sizeof(Ctl), cudaMemcpyHostToDevice, st));
    int bps = 0;
    void *kfn = kSeg == 64 ? (void *)k_peel<64> : (void *)k_peel<32>;
    BT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kfn, kPeelThreads, 0));
    if (bps < 1) return cudaErrorCooperativeLaunchTooLarge;
    dim3 grid((unsigned)(num_sms * bps)), block(kPeelThreads);
    void *kargs[] = {&a};
    BT_CUDA(cudaLaunchCooperativeKernel(kfn, grid, block, kargs, 0, st));
    al.launches++;
    BT_CUDA(cudaMemcpyAsync(&h, a.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    BT_CUDA(cudaStreamSynchronize(st));
    al.mark(kPhPeel, true);
    if (h.err & kErrBarrier) res.status = BT_ERR_CUDA;
    else if (h.err & kErrPeelOverflow) res.status = BT_ERR_OVERFLOW;
    else if (h.err & kErrRounds) res.status = BT_ERR_NOCONVERGE;
    res.rounds = h.rounds;
    res.levels = h.levels;
    res.windows = h.windows;
    res.updates = h.updates;
    res.slots = h.slots;
    res.kmax = h.kfinal;
    al.put(a.sup);
    al.put(a.state);
    al.put(a.died);
    al.put(a.bk);
    for (int i = 0; i < 3; ++i) {
        al.put(a.Cb[i]);
        al.put(a.bseg[i]);
    }
    for (int i = 0; i < 2; ++i) {
        al.put(a.items[i]);
        al.put(a.alive[i]);
        al.put(a.near[i]);
    }
    al.put(a.ctl);
    return cudaSuccess;
}

}  // namespace bt
