// Level-synchronous batch peeling through the BE-Index (Section V-B,
// Alg. 5, BiT-BU++; the <= k frontier rule of Alg. 4).
//
// One round removes the batch S = {unassigned e : support(e) <= k} at once:
//   kills (Alg. 5, the loop over e in S and B in N_I(e)):
//     every live twin pair of a bloom B that holds an edge of S dies once;
//     C(B) counts the dead pairs.  When both twins are in S the pair is
//     counted once (the example of Section V-B: three twin pairs of B0 drop
//     its bloom number to 0).  A twin outside S loses all k_B - 1
//     butterflies it had in B (Lemma 2).
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
// Scheduling.  The whole loop runs in one persistent cooperative kernel (one
// block per SM slot the occupancy allows); phases are separated by a grid
// barrier whose wait is bounded by a timer (on timeout the kernel raises an
// error word and every block returns).  The kills of round r + 1 need only
// C_r, which is final once the bloom phase of round r starts, so they are
// made inside that bloom phase: the warp whose decrement carries an edge
// into the batch of round r + 1 kills the edge's twin pairs at once when the
// edge has few links, and queues the links as incidence items otherwise.  A
// round therefore costs one barrier, plus a separate incidence phase (and a
// second barrier) only when such items exist or a level jump selected the
// batch.  Pairs killed early carry stamp r + 1 and still count as alive in
// the bloom phase of round r.  The bloom number at the start of round q is
// the value recorded after the last round that touched the bloom, less
// C_{q-1} when round q - 1 touched it and its bloom phase has not recorded
// the new value yet.  Work is split into items of at most kSeg entries, so no
// warp straggles on a hub edge or bloom.  A twin pair carries the round it
// died in; the edges of a batch race to stamp it with atomicCAS, so exactly
// one of them counts it in C(B); the stamp also records which members of the
// pair are in the batch (the killer's side bit, and the other member's bit
// when it stamps the same round), so the bloom phase knows which member
// loses k_B - 1 without reading edge states.  Counters and work lists rotate by round
// (C by 3, bloom items by 4, batch sizes by 3, incidence items by 2) so each
// is reset a barrier after its last reader.  Data written by other blocks
// during the kernel is read with L2 (.cg) loads.
#include "bt_device.cuh"
#include "bt_internal.cuh"

namespace bt {
namespace {

// entries per work item: SEG = 32, 64 or 128 (template parameter: 32 or 64
// picked by the batch autotuner, 128 for indexes of over 2^30 twin pairs);
// each lane handles SEG / 32 entries with their loads and atomics issued
// together.  Threads a block: 640 (96 registers, no spills) for 32- and
// 64-entry items, 512 (128 registers) for 128-entry items, whose four slots
// a lane need the registers.
__host__ __device__ constexpr int peel_threads(uint32_t seg) { return seg == 128 ? 512 : 640; }
// items with at most kSmall entries are processed by one lane each, larger
// ones by the whole warp.  Lane l of warp w takes item w + l * nwarps (plus
// multiples of 32 * nwarps): a round with fewer items than warps still gives
// every item its own warp, and a large round fills all lanes.
constexpr uint32_t kSmall = 2;
// edges that join the next batch in a bloom phase are listed per block (up to
// one per thread); the block kills their twin pairs at the end of the phase,
// two links per thread, for the edges whose links fit in the first two per
// thread
constexpr unsigned long long kBarrierTimeoutNs = 20ull * 1000 * 1000 * 1000;  // 20 s (default)
// pair death stamps: round << 2 | (first member in the batch) | (second << 1);
// kAlive (all ones) is never a stamp while rounds stay below kMaxRounds
constexpr uint32_t kMaxRounds = (1u << 30) - 4u;
constexpr uint32_t kErrBarrier = 1u;
constexpr uint32_t kErrRounds = 2u;
constexpr uint32_t kErrPeelOverflow = 4u;
constexpr unsigned kFull = 0xffffffffu;
// level-jump windows above this size queue their batch with warp-aggregated atomics
constexpr uint32_t kWarpSlotsMin = 1u << 16;

struct Ctl {
    unsigned long long bar_count;  // barrier arrivals (monotonic within a launch)
    unsigned int err;
    unsigned int pad0;
    unsigned int n_items[2];  // incidence items, by round parity
    unsigned int n_edges[3];  // batch sizes, by round mod 3
    unsigned int n_bseg[4];   // bloom items, by round mod 4
    unsigned int n_alive[2];  // alive list sizes (ping-pong)
    unsigned int n_near[2];   // near-window list sizes (ping-pong)
    unsigned int pad1;
    unsigned long long minsup;   // level-jump minimum over the near window
    unsigned long long minsup2;  // minimum over all alive edges (window rebuild)
    unsigned long long updates;
    unsigned long long slots;  // bloom pair slots visited by the bloom phase
    unsigned long long scanned;  // edge-list entries scanned by level jumps
    unsigned long long rounds;
    unsigned long long levels;
    unsigned long long windows;
    unsigned long long kfinal;
    unsigned long long inc_phases;  // rounds that ran a separate incidence phase
};

struct PeelArgs {
    uint64_t m;
    const uint64_t *inc_off;
    const uint2 *inc;  // (pair, bloom | side << 31)
    const uint2 *pairs;
    const uint32_t *bloom_off;
    long long *sup;
    uint32_t *state;
    uint32_t *phi;
    uint32_t *died;           // death stamp of a twin pair (kAlive while alive)
    unsigned long long *bw;   // per bloom: last round that touched it << 32 | k_B after it
    uint32_t *Cb[3];          // C_r by round mod 3
    uint4 *items[2];          // (edge, first link lo, first link hi, count | head flag << 31)
    uint4 *bseg[4];           // (bloom, first pair, count | head flag << 31, k_B at round start)
    uint32_t *alive[2];
    uint32_t *near[2];
    uint64_t item_cap;
    uint64_t bseg_cap;
    Ctl *ctl;
    uint64_t round_limit;
    unsigned long long barrier_timeout_ns;
    unsigned long long hold_barrier;  // 0, or n: block 0 skips its arrival at barrier n (from 1)
    uint32_t join_cap;     // edges a block lists in a bloom phase (<= threads a block)
    uint32_t block_links;  // links of the listed edges the block stage kills itself (<= 2 a thread)
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

// Counters the next phase needs.  Thread 0 of each block reads them once
// after the barrier and hands them to its block through shared memory, so a
// counter that every thread needs costs one L2 request per block instead of
// one per warp (same-address requests queue up at one L2 slice).
struct Snap {
    const unsigned int *u[5];
    const unsigned long long *w;
};
struct SnapVals {
    unsigned int u[5];
    unsigned long long w;
};

__device__ bool grid_barrier(const PeelArgs &a, unsigned long long &bar_no, const Snap &sn, SnapVals *s_v) {
    Ctl *ctl = a.ctl;
    __syncthreads();
    __shared__ int s_ok;
    const unsigned long long target = (bar_no + 1) * gridDim.x;
    ++bar_no;
    if (threadIdx.x == 0) {
        int ok = 1;
        // a held barrier (fault injection) never completes: every block's
        // wait below runs out and raises the error word
        if (!(blockIdx.x == 0 && bar_no == a.hold_barrier)) arrive_release(&ctl->bar_count);
        if (load_acquire(&ctl->bar_count) < target) {
            const unsigned long long t0 = now_ns();
            unsigned int spins = 0;
            while (load_acquire(&ctl->bar_count) < target) {
                if (((++spins) & 63u) == 0) {
                    if (*(volatile unsigned int *)&ctl->err) {
                        ok = 0;
                        break;
                    }
                    if (now_ns() - t0 > a.barrier_timeout_ns) {
                        atomicOr(&ctl->err, kErrBarrier);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        if (ok) {
            unsigned int v[5];
#pragma unroll
            for (int i = 0; i < 5; ++i) v[i] = sn.u[i] ? __ldcg(sn.u[i]) : 0u;
            const unsigned long long w = sn.w ? __ldcg(sn.w) : 0ull;
#pragma unroll
            for (int i = 0; i < 5; ++i) s_v->u[i] = v[i];
            s_v->w = w;
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Queue the links [ib, ie) of edge e as incidence items of list dst, one item
// per kSeg links, each carrying its link range.
template <uint32_t kSeg>
__device__ __forceinline__ void push_items(const PeelArgs &a, uint32_t e, uint32_t dst, uint64_t ib,
                                           uint64_t ie) {
    const uint64_t d = ie - ib;
    if (d == 0) return;
    const uint32_t nseg = (uint32_t)((d + kSeg - 1) / kSeg);
    const uint32_t base = atomicAdd(&a.ctl->n_items[dst], nseg);
    for (uint32_t s = 0; s < nseg; ++s) {
        const uint64_t j = ib + (uint64_t)s * kSeg;
        const uint64_t left = d - (uint64_t)s * kSeg;
        const uint32_t cnt = (uint32_t)(left < kSeg ? left : kSeg);
        a.items[dst][base + s] =
            make_uint4(e, (uint32_t)j, (uint32_t)(j >> 32), cnt | (s == 0 ? 0x80000000u : 0u));
    }
}

// Edge e joins the batch of round q at level k.
__device__ __forceinline__ void join_batch(const PeelArgs &a, uint32_t e, uint32_t q, long long k) {
    a.state[e] = q;
    if (k >= a.assign_from) a.phi[e] = (uint32_t)k;  // e leaves in a batch of this level
}

__device__ __forceinline__ void push_near(const PeelArgs &a, uint32_t e, uint32_t nq) {
    a.near[nq][atomicAdd(&a.ctl->n_near[nq], 1u)] = e;
}

// Window above the current minimum: narrow enough that a level jump scans few
// edges at high levels (dense cores hold many edges in a support range), wide
// enough that rebuilds from the full alive list stay rare.
__device__ __forceinline__ long long window_top(long long kmin) {
    long long w = kmin / 64;
    return kmin + (w < 8 ? 8 : w);
}

// One kill of a pair of bloom B for round q: count it in C_q(B).  Returns
// true for the first kill of B in round q, with B's first pair, pair count
// and k_B at the start of round q (its bloom items are then queued).
__device__ __forceinline__ bool count_kill(const PeelArgs &a, uint32_t B, uint32_t q, uint32_t &bo0,
                                           uint32_t &span, uint32_t &kB) {
    bo0 = a.bloom_off[B];
    const uint32_t bo1 = a.bloom_off[B + 1];
    const unsigned long long w = __ldcg(&a.bw[B]);
    const uint32_t cprev = __ldcg(&a.Cb[(q + 2u) % 3u][B]);  // C_{q-1}(B)
    span = bo1 - bo0;
    kB = (uint32_t)(w >> 32) == q - 1u ? (uint32_t)w : (uint32_t)w - cprev;
    return atomicAdd(&a.Cb[q % 3u][B], 1u) == 0u;
}

// Edges of the batch of round q kill the pairs of up to N links (won[r] set
// on entry for the valid ones; link l[r] names the pair and which member the
// edge is, 0 first, 1 second).  The first edge to stamp a pair counts it
// (won[r] stays true); a twin of the same batch adds its side bit to the
// stamp.  A lane's stamps go out together before any result is examined.
template <uint32_t N>
__device__ __forceinline__ void kill_pairs(const PeelArgs &a, const uint2 (&l)[N], bool (&won)[N], uint32_t q) {
    uint32_t old[N];
#pragma unroll
    for (uint32_t r = 0; r < N; ++r)
        old[r] = won[r] ? atomicCAS(&a.died[l[r].x], kAlive, (q << 2) | (1u << (l[r].y >> 31))) : 0u;
#pragma unroll
    for (uint32_t r = 0; r < N; ++r) {
        if (!won[r]) continue;
        won[r] = old[r] == kAlive;
        if (!won[r] && (old[r] >> 2) == q) atomicOr(&a.died[l[r].x], 1u << (l[r].y >> 31));
    }
}

// Whole warp (converged): each lane's pairs killed for round q (won[r], bloom
// B[r]) are counted, and the blooms killed for the first time in round q get
// their bloom items (one per kSeg pairs, each with k_B at the start of round
// q).  The warp takes all its item slots with one atomic: in large rounds
// millions of first kills would otherwise queue on the one counter.
template <uint32_t kSeg, uint32_t N>
__device__ __forceinline__ void warp_kills(const PeelArgs &a, uint32_t q, const uint32_t (&B)[N],
                                           const bool (&won)[N], int lane) {
    uint32_t bo0[N], span[N], kB[N], nseg[N];
    uint32_t mine = 0;
    if constexpr (N >= 4) {
        // four kills a lane: their bloom loads, then their count atomics, go
        // out together
        uint32_t prev[N];
#pragma unroll
        for (uint32_t r = 0; r < N; ++r) {
            if (won[r]) {
                bo0[r] = a.bloom_off[B[r]];
                span[r] = a.bloom_off[B[r] + 1] - bo0[r];
                const unsigned long long w = __ldcg(&a.bw[B[r]]);
                const uint32_t cprev = __ldcg(&a.Cb[(q + 2u) % 3u][B[r]]);  // C_{q-1}(B)
                kB[r] = (uint32_t)(w >> 32) == q - 1u ? (uint32_t)w : (uint32_t)w - cprev;
            }
        }
#pragma unroll
        for (uint32_t r = 0; r < N; ++r) prev[r] = won[r] ? atomicAdd(&a.Cb[q % 3u][B[r]], 1u) : 1u;
#pragma unroll
        for (uint32_t r = 0; r < N; ++r) {
            nseg[r] = prev[r] == 0u ? (span[r] + kSeg - 1) / kSeg : 0u;
            mine += nseg[r];
        }
    } else {
#pragma unroll
        for (uint32_t r = 0; r < N; ++r) {
            nseg[r] = 0;
            if (won[r] && count_kill(a, B[r], q, bo0[r], span[r], kB[r])) nseg[r] = (span[r] + kSeg - 1) / kSeg;
            mine += nseg[r];
        }
    }
    const uint32_t incl = dev::warp_incl_scan(mine);
    const uint32_t all = __shfl_sync(kFull, incl, 31);
    if (all == 0) return;
    const uint32_t qb = q & 3u;
    uint32_t base = 0;
    if (lane == 31) base = atomicAdd(&a.ctl->n_bseg[qb], all);
    uint32_t slot = __shfl_sync(kFull, base, 31) + incl - mine;
#pragma unroll
    for (uint32_t r = 0; r < N; ++r)
        for (uint32_t s = 0; s < nseg[r]; ++s, ++slot) {
            const uint32_t left = span[r] - s * kSeg;
            a.bseg[qb][slot] =
                make_uint4(B[r], bo0[r] + s * kSeg, (left < kSeg ? left : kSeg) | (s == 0 ? 0x80000000u : 0u), kB[r]);
        }
}

// Edge e joins the batch of round q in a bloom phase: it goes to the block's
// list, or, when that is full, the lane queues its links itself.
template <uint32_t kSeg>
__device__ __forceinline__ void join_next(const PeelArgs &a, uint32_t e, uint32_t q, long long k,
                                          uint32_t *s_je, uint32_t *s_jn) {
    const uint32_t slot = atomicAdd(s_jn, 1u);
    if (slot < a.join_cap) {
        s_je[slot] = e;
    } else {
        join_batch(a, e, q, k);
        push_items<kSeg>(a, e, q & 1u, a.inc_off[e], a.inc_off[e + 1]);
        atomicAdd(&a.ctl->n_edges[q % 3u], 1u);
    }
}

// Bloom phase of round r, N pair slots (died stamps d, members pr) of a bloom
// with c pairs killed this round and bloom number kB at round start.  All the
// slots' support decrements are issued before any result is examined, so they
// travel together.
template <uint32_t kSeg, uint32_t N>
__device__ __forceinline__ void apply_slots(const PeelArgs &a, const uint32_t (&d)[N], const uint2 (&pr)[N],
                                            uint32_t c, uint32_t kB, const Lvl &L, uint32_t round,
                                            unsigned long long &upd, uint32_t *s_je, uint32_t *s_jn) {
    const uint32_t q = round + 1u;
    uint32_t e[2 * N];
    long long dec[2 * N];
#pragma unroll
    for (uint32_t r = 0; r < N; ++r) {
        // bit 31 flags an edge whose bitruss number is already known: it is
        // never peeled again, so it needs no decrement
        const bool fx = pr[r].x >> 31, fy = pr[r].y >> 31;
        e[2 * r] = pr[r].x & 0x7FFFFFFFu;
        e[2 * r + 1] = pr[r].y & 0x7FFFFFFFu;
        dec[2 * r] = 0;
        dec[2 * r + 1] = 0;
        const uint32_t dr = d[r] >> 2;  // round of death (kAlive: 0x3FFFFFFF, no round)
        if (d[r] == kAlive || dr == q) {
            // alive during this round (a pair killed for the next round still
            // is): one butterfly lost per dead pair
            if (!fx) dec[2 * r] = c;
            if (!fy) dec[2 * r + 1] = c;
        } else if (dr == round && kB > 1u) {
            // died now: a member outside S (its bit not stamped) loses its
            // k_B - 1 butterflies
            if (!(fx || (d[r] & 1u))) dec[2 * r] = (long long)kB - 1;
            if (!(fy || (d[r] & 2u))) dec[2 * r + 1] = (long long)kB - 1;
        }
    }
    long long old[2 * N];
#pragma unroll
    for (uint32_t i = 0; i < 2 * N; ++i)
        old[i] = dec[i] ? (long long)atomicAdd(reinterpret_cast<unsigned long long *>(&a.sup[e[i]]),
                                               (unsigned long long)(-dec[i]))
                        : 0;
#pragma unroll
    for (uint32_t i = 0; i < 2 * N; ++i) {
        if (!dec[i]) continue;
        ++upd;
        const long long now = old[i] - dec[i];
        if (old[i] >= L.khi && now < L.khi) push_near(a, e[i], L.nq);
        // exactly one decrement takes the edge from > k to <= k: it joins the
        // next batch
        if (old[i] > L.k && now <= L.k) join_next<kSeg>(a, e[i], q, L.k, s_je, s_jn);
    }
}

template <uint32_t kSeg>
__global__ void __launch_bounds__(peel_threads(kSeg), 1) k_peel(PeelArgs a) {
    constexpr uint32_t R = kSeg / 32;  // entries per lane
    constexpr uint32_t kT = peel_threads(kSeg);
    constexpr uint32_t kJoinCap = kT;
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
    // edges this block's bloom items carried into the next batch
    __shared__ uint32_t s_je[kJoinCap], s_joff[kJoinCap], s_jd[kJoinCap];
    __shared__ unsigned long long s_jib[kJoinCap];
    __shared__ uint32_t s_jn;
    __shared__ SnapVals s_v;
    if (threadIdx.x == 0) s_jn = 0;
    __syncthreads();
    // list sizes, kept identically by every thread from the barrier snapshots
    uint32_t v_near = 0;                      // near list L.nq
    uint32_t v_alive = (uint32_t)a.m;         // alive list ap
    uint32_t n_batch = 0, n_items = 0;        // this round's batch and incidence items
    uint32_t nb_cur = 0, nb_prev = 0;         // bloom items of this round and of the last

    while (remaining > 0) {
        const uint32_t par = round & 1u;
        const uint32_t c3 = round % 3u;
        const uint32_t b4 = round & 3u;
        const uint32_t bp = (round + 3u) & 3u;  // previous round's bloom items
        if (round > a.round_limit) {
            if (gtid == 0) atomicOr(&ctl->err, kErrRounds);
            break;
        }
        if (level_jump) {
            if (gtid == 0) atomicAdd(&ctl->scanned, (unsigned long long)v_near);
            // L1: minimum over the near window, compacting it
            {
                unsigned long long best = ~0ull;
                for (uint32_t i0 = blockIdx.x * blockDim.x; i0 < v_near; i0 += nthreads) {
                    const uint32_t i = i0 + threadIdx.x;
                    bool keep = false;
                    uint32_t e = 0;
                    if (i < v_near) {
                        e = ldcg_u32(&a.near[L.nq][i]);
                        // state and support requested together
                        const uint32_t stv = ldcg_u32(&a.state[e]);
                        const unsigned long long sv = (unsigned long long)ldcg_ll(&a.sup[e]);
                        if (stv == kAlive) {
                            keep = true;
                            best = sv < best ? sv : best;
                        }
                    }
                    const unsigned int mask = __ballot_sync(kFull, keep);
                    if (mask) {
                        unsigned int base = 0;
                        if (lane == 0) base = atomicAdd(&ctl->n_near[L.nq ^ 1u], (unsigned)__popc(mask));
                        base = __shfl_sync(kFull, base, 0);
                        if (keep) a.near[L.nq ^ 1u][base + __popc(mask & ((1u << lane) - 1u))] = e;
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const unsigned long long y = __shfl_xor_sync(kFull, best, o);
                    best = y < best ? y : best;
                }
                if (lane == 0 && best != ~0ull) atomicMin(&ctl->minsup, best);
            }
            {
                const Snap sn{{nullptr, nullptr, nullptr, nullptr, &ctl->n_near[L.nq ^ 1u]}, &ctl->minsup};
                if (!grid_barrier(a, bar_no, sn, &s_v)) break;
            }
            unsigned long long mn = s_v.w;
            v_near = s_v.u[4];
            L.nq ^= 1u;
            if (gtid == 0) ctl->n_near[L.nq ^ 1u] = 0;
            if (mn == ~0ull) {
                // the window holds no alive edge: rebuild it from all alive edges.
                // W1: overall minimum, compacting the alive list
                if (gtid == 0) atomicAdd(&ctl->scanned, (unsigned long long)v_alive);
                unsigned long long best = ~0ull;
                for (uint32_t i0 = blockIdx.x * blockDim.x; i0 < v_alive; i0 += nthreads) {
                    const uint32_t i = i0 + threadIdx.x;
                    bool keep = false;
                    uint32_t e = 0;
                    if (i < v_alive) {
                        e = ldcg_u32(&a.alive[ap][i]);
                        const uint32_t stv = ldcg_u32(&a.state[e]);
                        const unsigned long long sv = (unsigned long long)ldcg_ll(&a.sup[e]);
                        if (stv == kAlive) {
                            keep = true;
                            best = sv < best ? sv : best;
                        }
                    }
                    const unsigned int mask = __ballot_sync(kFull, keep);
                    if (mask) {
                        unsigned int base = 0;
                        if (lane == 0) base = atomicAdd(&ctl->n_alive[ap ^ 1u], (unsigned)__popc(mask));
                        base = __shfl_sync(kFull, base, 0);
                        if (keep) a.alive[ap ^ 1u][base + __popc(mask & ((1u << lane) - 1u))] = e;
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const unsigned long long y = __shfl_xor_sync(kFull, best, o);
                    best = y < best ? y : best;
                }
                if (lane == 0 && best != ~0ull) atomicMin(&ctl->minsup2, best);
                {
                    const Snap sn{{nullptr, nullptr, nullptr, nullptr, &ctl->n_alive[ap ^ 1u]}, &ctl->minsup2};
                    if (!grid_barrier(a, bar_no, sn, &s_v)) break;
                }
                mn = s_v.w;
                if (mn == ~0ull) break;  // no alive edge: cannot happen while remaining > 0
                v_alive = s_v.u[4];
                L.khi = window_top((long long)mn);
                ap ^= 1u;
                if (gtid == 0) ctl->n_alive[ap ^ 1u] = 0;
                // W2: list every alive edge below the new window top (one
                // counter atomic per warp: the list can take most edges)
                if (gtid == 0) atomicAdd(&ctl->scanned, (unsigned long long)v_alive);
                for (uint32_t i0 = gwarp * 32u; i0 < v_alive; i0 += nthreads) {
                    const uint32_t i = i0 + lane;
                    uint32_t e = 0;
                    bool keep = false;
                    if (i < v_alive) {
                        e = ldcg_u32(&a.alive[ap][i]);
                        keep = ldcg_ll(&a.sup[e]) < L.khi;
                    }
                    const unsigned int mask = __ballot_sync(kFull, keep);
                    if (mask) {
                        unsigned int base = 0;
                        if (lane == 0) base = atomicAdd(&ctl->n_near[L.nq], (unsigned)__popc(mask));
                        base = __shfl_sync(kFull, base, 0);
                        if (keep) a.near[L.nq][base + __popc(mask & ((1u << lane) - 1u))] = e;
                    }
                }
                if (gtid == 0) atomicAdd(&ctl->windows, 1ull);
                {
                    const Snap sn{{nullptr, nullptr, nullptr, nullptr, &ctl->n_near[L.nq]}, nullptr};
                    if (!grid_barrier(a, bar_no, sn, &s_v)) break;
                }
                v_near = s_v.u[4];
                if (gtid == 0) ctl->minsup2 = ~0ull;
            }
            if ((long long)mn > L.k) L.k = (long long)mn;
            if ((unsigned long long)L.k > 0xFFFFFFFFull) {
                if (gtid == 0) atomicOr(&ctl->err, kErrPeelOverflow);
                break;
            }
            // L2: the batch is every window edge with support <= k; their
            // links become incidence items of this round.  A large window
            // (a level can select millions of edges) takes its item slots
            // with one atomic per warp; a small one per edge, which is faster
            // when only a few edges are selected.
            uint32_t sel = 0;
            if (gtid == 0) atomicAdd(&ctl->scanned, (unsigned long long)v_near);
            if (v_near > kWarpSlotsMin) {
                for (uint32_t i0 = gwarp * 32u; i0 < v_near; i0 += nthreads) {
                    const uint32_t i = i0 + lane;
                    uint32_t e = 0, nseg = 0;
                    uint64_t ib = 0, ie = 0;
                    if (i < v_near) {
                        e = ldcg_u32(&a.near[L.nq][i]);
                        // state, support and link range requested together
                        const uint32_t stv = ldcg_u32(&a.state[e]);
                        const long long sv = ldcg_ll(&a.sup[e]);
                        const uint64_t b0 = a.inc_off[e], b1 = a.inc_off[e + 1];
                        if (stv == kAlive && sv <= L.k) {
                            join_batch(a, e, round, L.k);
                            ++sel;
                            ib = b0;
                            ie = b1;
                            nseg = (uint32_t)((ie - ib + kSeg - 1) / kSeg);
                        }
                    }
                    const uint32_t incl = dev::warp_incl_scan(nseg);
                    const uint32_t all = __shfl_sync(kFull, incl, 31);
                    if (all) {
                        uint32_t base = 0;
                        if (lane == 31) base = atomicAdd(&ctl->n_items[par], all);
                        uint32_t slot = __shfl_sync(kFull, base, 31) + incl - nseg;
                        for (uint32_t s2 = 0; s2 < nseg; ++s2, ++slot) {
                            const uint64_t j = ib + (uint64_t)s2 * kSeg;
                            const uint64_t left = ie - j;
                            const uint32_t cnt = (uint32_t)(left < kSeg ? left : kSeg);
                            a.items[par][slot] =
                                make_uint4(e, (uint32_t)j, (uint32_t)(j >> 32), cnt | (s2 == 0 ? 0x80000000u : 0u));
                        }
                    }
                }
            } else {
                for (uint32_t i = gtid; i < v_near; i += nthreads) {
                    const uint32_t e = ldcg_u32(&a.near[L.nq][i]);
                    const uint32_t stv = ldcg_u32(&a.state[e]);
                    const long long sv = ldcg_ll(&a.sup[e]);
                    const uint64_t b0 = a.inc_off[e], b1 = a.inc_off[e + 1];
                    if (stv == kAlive && sv <= L.k) {
                        join_batch(a, e, round, L.k);
                        push_items<kSeg>(a, e, par, b0, b1);
                        ++sel;
                    }
                }
            }
            sel = dev::warp_sum(sel);
            if (lane == 0 && sel) atomicAdd(&ctl->n_edges[c3], sel);
            if (gtid == 0) atomicAdd(&ctl->levels, 1ull);
            {
                const Snap sn{{&ctl->n_edges[c3], &ctl->n_items[par], &ctl->n_bseg[b4], &ctl->n_bseg[bp],
                               &ctl->n_near[L.nq]},
                              nullptr};
                if (!grid_barrier(a, bar_no, sn, &s_v)) break;
            }
            n_batch = s_v.u[0];
            n_items = s_v.u[1];
            nb_cur = s_v.u[2];
            nb_prev = s_v.u[3];
            v_near = s_v.u[4];
            if (gtid == 0) ctl->minsup = ~0ull;
        }

        if (gtid == 0) {
            ctl->n_edges[(round + 2u) % 3u] = 0;  // batch of round - 1: read before the last barrier
            ctl->n_bseg[(round + 2u) & 3u] = 0;   // bloom items of round - 2: C cleared in round - 1
        }

        // ---------------- incidence phase (only for queued link lists)
        if (n_items > 0) {
            if (gtid == 0) atomicAdd(&ctl->inc_phases, 1ull);
            for (uint32_t base = gwarp; base < n_items; base += nwarps * 32u) {
                const uint32_t i = base + lane * nwarps;
                const uint4 it = i < n_items ? __ldcg(&a.items[par][i]) : make_uint4(0, 0, 0, 0);
                const uint32_t cnt = it.w & 0x7FFFFFFFu;
                {
                    // a small item is this lane's own: its links' loads and
                    // stamps go out together
                    const uint64_t j0 = (uint64_t)it.z << 32 | it.y;
                    uint2 l[kSmall];
                    uint32_t B[kSmall];
                    bool won[kSmall];
#pragma unroll
                    for (uint32_t r = 0; r < kSmall; ++r) {
                        won[r] = cnt <= kSmall && r < cnt;
                        l[r] = won[r] ? a.inc[j0 + r] : make_uint2(0u, 0u);
                        B[r] = l[r].y & 0x7FFFFFFFu;
                    }
                    // the first edge of the batch to stamp a pair kills it (once)
                    kill_pairs<kSmall>(a, l, won, round);
                    warp_kills<kSeg, kSmall>(a, round, B, won, lane);
                }
                // items with many links: the whole warp, one item at a time
                unsigned big = __ballot_sync(kFull, cnt > kSmall);
                while (big) {
                    const int src = __ffs(big) - 1;
                    big &= big - 1u;
                    const uint32_t bcnt = __shfl_sync(kFull, cnt, src);
                    const uint32_t jlo = __shfl_sync(kFull, it.y, src);
                    const uint32_t jhi = __shfl_sync(kFull, it.z, src);
                    const uint64_t j0 = ((uint64_t)jhi << 32 | jlo) + lane;
                    uint2 l[R];
                    uint32_t B[R];
                    bool won[R];
#pragma unroll
                    for (uint32_t r = 0; r < R; ++r) {
                        won[r] = lane + 32u * r < bcnt;
                        l[r] = won[r] ? a.inc[j0 + 32u * r] : make_uint2(0u, 0u);
                        B[r] = l[r].y & 0x7FFFFFFFu;
                    }
                    kill_pairs<R>(a, l, won, round);
                    warp_kills<kSeg, R>(a, round, B, won, lane);
                }
            }
            {
                const Snap sn{{nullptr, nullptr, &ctl->n_bseg[b4], nullptr, nullptr}, nullptr};
                if (!grid_barrier(a, bar_no, sn, &s_v)) break;
            }
            nb_cur = s_v.u[2];
        }

        // ---------------- bloom phase of this round, kills of the next
        if (gtid == 0) ctl->n_items[par] = 0;
        {
            const uint32_t q = round + 1u;
            const uint32_t *C = a.Cb[c3];
            for (uint32_t base = gwarp; base < nb_cur; base += nwarps * 32u) {
                const uint32_t i = base + lane * nwarps;
                const uint4 it = i < nb_cur ? __ldcg(&a.bseg[b4][i]) : make_uint4(0, 0, 0, 0);
                const uint32_t cnt = it.z & 0x7FFFFFFFu;
                const uint32_t c = cnt ? __ldcg(&C[it.x]) : 0u;
                if (cnt && (it.z >> 31))
                    a.bw[it.x] = (unsigned long long)round << 32 | (uint32_t)(it.w - c);
                slots += cnt;
                if (cnt <= kSmall) {
                    uint32_t d[kSmall];
                    uint2 pr[kSmall];
#pragma unroll
                    for (uint32_t r = 0; r < kSmall; ++r) {
                        const bool act = r < cnt;
                        d[r] = act ? __ldcg(&a.died[it.y + r]) : (round + 2u) << 2;  // inactive: no case applies
                        pr[r] = act ? a.pairs[it.y + r] : make_uint2(0, 0);
                    }
                    apply_slots<kSeg, kSmall>(a, d, pr, c, it.w, L, round, upd, s_je, &s_jn);
                }
                // items with many slots: the whole warp, one item at a time.
                // With one slot a lane the next item's pair words are
                // requested before this item's decrements go out (2M-edge
                // graph 467 -> 460 ms, a C3-shaped 3M-edge graph 1534 ->
                // 1481 ms); with two the extra registers spill and the
                // 30M-edge graph measured 1 % slower, so items go one by one.
                unsigned big = __ballot_sync(kFull, cnt > kSmall);
                uint32_t d[R], kB = 0, bc = 0;
                uint2 pr[R];
                if constexpr (R == 1) {
                    if (big) {
                        const int src = __ffs(big) - 1;
                        big &= big - 1u;
                        const uint32_t bcnt = __shfl_sync(kFull, cnt, src);
                        const uint32_t p0 = __shfl_sync(kFull, it.y, src) + lane;
                        kB = __shfl_sync(kFull, it.w, src);
                        bc = __shfl_sync(kFull, c, src);
                        const bool act = lane < bcnt;
                        d[0] = act ? __ldcg(&a.died[p0]) : (round + 2u) << 2;
                        pr[0] = act ? a.pairs[p0] : make_uint2(0, 0);
                        for (;;) {
                            const bool more = big != 0u;
                            uint32_t dn = 0, kBn = 0, bcn = 0;
                            uint2 prn = make_uint2(0, 0);
                            if (more) {
                                const int s2 = __ffs(big) - 1;
                                big &= big - 1u;
                                const uint32_t ncnt = __shfl_sync(kFull, cnt, s2);
                                const uint32_t np0 = __shfl_sync(kFull, it.y, s2) + lane;
                                kBn = __shfl_sync(kFull, it.w, s2);
                                bcn = __shfl_sync(kFull, c, s2);
                                const bool nact = lane < ncnt;
                                dn = nact ? __ldcg(&a.died[np0]) : (round + 2u) << 2;
                                prn = nact ? a.pairs[np0] : make_uint2(0, 0);
                            }
                            apply_slots<kSeg, R>(a, d, pr, bc, kB, L, round, upd, s_je, &s_jn);
                            if (!more) break;
                            d[0] = dn;
                            pr[0] = prn;
                            kB = kBn;
                            bc = bcn;
                        }
                    }
                } else {
                    while (big) {
                        const int src = __ffs(big) - 1;
                        big &= big - 1u;
                        const uint32_t bcnt = __shfl_sync(kFull, cnt, src);
                        const uint32_t p0 = __shfl_sync(kFull, it.y, src) + lane;
                        kB = __shfl_sync(kFull, it.w, src);
                        bc = __shfl_sync(kFull, c, src);
#pragma unroll
                        for (uint32_t r = 0; r < R; ++r) {
                            const bool act = lane + 32u * r < bcnt;
                            d[r] = act ? __ldcg(&a.died[p0 + 32u * r]) : (round + 2u) << 2;
                            pr[r] = act ? a.pairs[p0 + 32u * r] : make_uint2(0, 0);
                        }
                        apply_slots<kSeg, R>(a, d, pr, bc, kB, L, round, upd, s_je, &s_jn);
                    }
                }
            }
            // clear C of the blooms the previous round touched (threads from
            // the top of the grid, away from the bloom items above)
            uint32_t *Cp = a.Cb[(round + 2u) % 3u];
            for (uint32_t i = nthreads - 1u - gtid; i < nb_prev; i += nthreads) {
                const uint4 it = __ldcg(&a.bseg[bp][i]);
                if (it.z >> 31) Cp[it.x] = 0;
            }

            // the block kills the twin pairs of the edges it listed
            __syncthreads();
            const uint32_t njr = s_jn;
            const uint32_t nj = njr < a.join_cap ? njr : a.join_cap;
            if (nj > 0) {
                uint32_t e = 0, d = 0;
                uint64_t ib = 0;
                if (threadIdx.x < nj) {
                    e = s_je[threadIdx.x];
                    join_batch(a, e, q, L.k);
                    ib = a.inc_off[e];
                    const uint64_t dl = a.inc_off[e + 1] - ib;
                    d = dl > a.block_links ? a.block_links + 1u : (uint32_t)dl;  // longer lists are queued
                }
                uint32_t total = 0;
                const uint32_t off = dev::block_excl_scan<uint32_t>(d, &total);
                if (threadIdx.x < nj) {
                    s_joff[threadIdx.x] = off;
                    s_jd[threadIdx.x] = d;
                    s_jib[threadIdx.x] = ib;
                    if (off + d > a.block_links) push_items<kSeg>(a, e, q & 1u, ib, a.inc_off[e + 1]);
                }
                if (threadIdx.x == 0) atomicAdd(&ctl->n_edges[q % 3u], nj);
                __syncthreads();
                const uint32_t lim = total < a.block_links ? total : a.block_links;
                uint2 l[2];
                uint32_t B[2];
                bool won[2];
#pragma unroll
                for (uint32_t r = 0; r < 2; ++r) {
                    const uint32_t x = threadIdx.x + r * kT;
                    won[r] = false;
                    l[r] = make_uint2(0u, 0u);
                    if (x < lim) {
                        const uint32_t j = dev::last_le_u32(s_joff, nj, x);
                        if (s_joff[j] + s_jd[j] <= a.block_links) {
                            won[r] = true;
                            l[r] = a.inc[s_jib[j] + (x - s_joff[j])];
                        }
                    }
                    B[r] = l[r].y & 0x7FFFFFFFu;
                }
                // the first edge of the batch to stamp a pair kills it (once)
                kill_pairs<2>(a, l, won, q);
                warp_kills<kSeg, 2>(a, q, B, won, lane);
                if (threadIdx.x == 0) s_jn = 0;
            }
        }
        {
            // next round: its batch, incidence items, bloom items, this
            // round's bloom items (C to clear) and the near list size
            const uint32_t q = round + 1u;
            const Snap sn{{&ctl->n_edges[q % 3u], &ctl->n_items[q & 1u], &ctl->n_bseg[q & 3u], &ctl->n_bseg[b4],
                           &ctl->n_near[L.nq]},
                          nullptr};
            if (!grid_barrier(a, bar_no, sn, &s_v)) break;
        }
        remaining -= n_batch;
        ++round;
        n_batch = s_v.u[0];
        n_items = s_v.u[1];
        nb_cur = s_v.u[2];
        nb_prev = s_v.u[3];
        v_near = s_v.u[4];
        level_jump = remaining > 0 && n_batch == 0;
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
                            const uint8_t *assigned, uint32_t *alive) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m;
         i += (uint64_t)gridDim.x * blockDim.x) {
        sup[i] = (long long)support[i];
        state[i] = (assigned && assigned[i]) ? kPerm : kAlive;
        alive[i] = (uint32_t)i;
    }
}

// Bloom words: no round has touched the bloom yet, k_B from the index.
__global__ void k_bw_init(const uint32_t *bloom_k, uint64_t nb, unsigned long long *bw) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nb;
         i += (uint64_t)gridDim.x * blockDim.x)
        bw[i] = 0xFFFFFFFFull << 32 | bloom_k[i];
}

inline unsigned grid_for(uint64_t items, int threads, unsigned cap) {
    uint64_t g = (items + threads - 1) / threads;
    if (g == 0) g = 1;
    return (unsigned)(g < cap ? g : cap);
}

}  // namespace

cudaError_t peel(const Index &ix, const uint64_t *support, uint32_t *phi_out, PeelResult &res,
                 int num_sms, Alloc &al, int seg, const PeelOpts *opts) {
    const uint32_t kSeg = seg == 128 ? 128u : seg == 64 ? 64u : 32u;
    const uint32_t kT = (uint32_t)peel_threads(kSeg);
    const uint32_t kJoinCap = kT, kBlockLinks = 2 * kT;
    const uint64_t m = ix.m;
    res = PeelResult{};
    if (m == 0 || (opts && opts->assigned && opts->m_active == 0)) return cudaSuccess;
    // one round queues each edge and each bloom at most once
    const uint64_t item_cap = m + (2 * ix.w2) / kSeg + 2;
    const uint64_t bseg_cap = ix.nb + ix.w2 / kSeg + 2;
    PeelArgs a{};
    a.m = m;
    a.inc_off = ix.inc_off;
    a.inc = ix.inc;
    a.pairs = ix.pairs;
    a.bloom_off = ix.bloom_off;
    a.phi = phi_out;
    a.sup = al.get<long long>(m);
    a.state = al.get<uint32_t>(m);
    a.died = al.get<uint32_t>(ix.w2);
    a.bw = al.get<unsigned long long>(ix.nb);
    for (int i = 0; i < 3; ++i) a.Cb[i] = al.get<uint32_t>(ix.nb);
    for (int i = 0; i < 4; ++i) a.bseg[i] = al.get<uint4>(bseg_cap);
    for (int i = 0; i < 2; ++i) {
        a.items[i] = al.get<uint4>(item_cap);
        a.alive[i] = al.get<uint32_t>(m);
        a.near[i] = al.get<uint32_t>(m);
    }
    a.item_cap = item_cap;
    a.bseg_cap = bseg_cap;
    a.ctl = al.get<Ctl>(1);
    {
        const bt_limits *lim = al.limits;
        uint64_t rl = m + 1 < kMaxRounds ? m + 1 : kMaxRounds;
        if (lim && lim->peel_round_limit && lim->peel_round_limit < rl) rl = lim->peel_round_limit;
        a.round_limit = rl;
        a.barrier_timeout_ns = (lim && lim->barrier_timeout_ns) ? lim->barrier_timeout_ns : kBarrierTimeoutNs;
        a.hold_barrier = lim ? lim->hold_barrier : 0;
        a.join_cap = (lim && lim->join_cap && lim->join_cap < kJoinCap) ? lim->join_cap : kJoinCap;
        a.block_links = (lim && lim->block_links && lim->block_links < kBlockLinks) ? lim->block_links : kBlockLinks;
    }
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
        k_bw_init<<<grid_for(ix.nb, 256, (unsigned)num_sms * 16), 256, 0, st>>>(ix.bloom_k, ix.nb, a.bw);
        al.launches++;
        for (int i = 0; i < 3; ++i)
            BT_CUDA(cudaMemsetAsync(a.Cb[i], 0, sizeof(uint32_t) * ix.nb, st));
    }
    Ctl h{};
    h.n_alive[0] = (unsigned int)m;
    h.minsup = ~0ull;
    h.minsup2 = ~0ull;
    BT_CUDA(cudaMemcpyAsync(a.ctl, &h, sizeof(Ctl), cudaMemcpyHostToDevice, st));
    int bps = 0;
    void *kfn = kSeg == 128 ? (void *)k_peel<128> : kSeg == 64 ? (void *)k_peel<64> : (void *)k_peel<32>;
    BT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kfn, (int)kT, 0));
    if (bps < 1) return cudaErrorCooperativeLaunchTooLarge;
    dim3 grid((unsigned)(num_sms * bps)), block(kT);
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
    res.scanned = h.scanned;
    res.kmax = h.kfinal;
    res.inc_phases = h.inc_phases;
    al.put(a.sup);
    al.put(a.state);
    al.put(a.died);
    al.put(a.bw);
    for (int i = 0; i < 3; ++i) al.put(a.Cb[i]);
    for (int i = 0; i < 4; ++i) al.put(a.bseg[i]);
    for (int i = 0; i < 2; ++i) {
        al.put(a.items[i]);
        al.put(a.alive[i]);
        al.put(a.near[i]);
    }
    al.put(a.ctl);
    return cudaSuccess;
}

}  // namespace bt
