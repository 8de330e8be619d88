// Level-synchronous batch peeling through the BE-Index (Section V-B,
// Alg. 5, BiT-BU++; the <= k frontier rule of Alg. 4).
//
// One round removes the batch S = {unassigned e : support(e) <= k} at once:
//   incidence pass (Alg. 5, the loop over e in S and B in N_I(e)):
//     every live twin pair of a bloom B that holds an edge of S dies once;
//     C(B) counts the dead pairs.  When both twins are in S the one with the
//     smaller edge id owns the pair, so a pair is counted once (the example of
//     Section V-B: three twin pairs of B0 drop its bloom number to 0).  A twin
//     outside S loses all k_B - 1 butterflies it had in B (Lemma 2).
//   bloom pass (Alg. 5, the loop over blooms with C(B) > 0):
//     every edge of a surviving pair of B loses C(B) butterflies (one per
//     dead pair); then k_B -= C(B), so the bloom keeps C(k_B - C, 2)
//     butterflies (Lemma 1).
//   phi(e) = k for e in S.
// k only grows: when no unassigned edge has support <= k, k jumps to the
// minimum remaining support (the batch-edge rule of Lemma 9).  Supports are
// decremented without the max(MBS, .) clamp of Alg. 5; an edge that drops to
// or below k is simply taken by the next round with the same k, which gives
// the same phi.  An edge joins the next batch exactly when one decrement
// carries its support from above k to <= k, so rounds inside a level never
// rescan all edges.
#include "bt_device.cuh"
#include "bt_internal.cuh"

namespace bt {
namespace {

struct Ctrl {
    unsigned long long minsup;
    unsigned long long updates;
    uint32_t n_next;
    uint32_t n_touched;
    uint32_t n_collect;
    uint32_t pad;
};

__global__ void k_peel_init(const uint64_t *support, uint64_t m, long long *sup, uint32_t *state) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m;
         i += (uint64_t)gridDim.x * blockDim.x) {
        sup[i] = (long long)support[i];
        state[i] = kAlive;
    }
}

__global__ void k_min_alive(const uint32_t *state, const long long *sup, uint64_t m, Ctrl *ctrl) {
    unsigned long long best = ~0ull;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m;
         i += (uint64_t)gridDim.x * blockDim.x)
        if (state[i] == kAlive) {
            unsigned long long s = (unsigned long long)sup[i];
            best = s < best ? s : best;
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long y = __shfl_xor_sync(0xffffffffu, best, o);
        best = y < best ? y : best;
    }
    if ((threadIdx.x & 31) == 0 && best != ~0ull) atomicMin(&ctrl->minsup, best);
}

__global__ void k_collect(uint32_t *state, const long long *sup, uint64_t m, long long k,
                          uint32_t round, uint32_t *S, Ctrl *ctrl) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m;
         i += (uint64_t)gridDim.x * blockDim.x)
        if (state[i] == kAlive && sup[i] <= k) {
            state[i] = round;
            S[atomicAdd(&ctrl->n_collect, 1u)] = (uint32_t)i;
        }
}

// Subtract dec from the support of e; queue e for the next round when this
// decrement takes it from above k to <= k.
__device__ __forceinline__ void decrement(long long *sup, uint32_t *state, uint32_t *S_next,
                                          Ctrl *ctrl, uint32_t e, long long dec, long long k,
                                          uint32_t round) {
    long long old = (long long)atomicAdd(reinterpret_cast<unsigned long long *>(&sup[e]),
                                         (unsigned long long)(-dec));
    if (old > k && old - dec <= k) {
        state[e] = round + 1;
        S_next[atomicAdd(&ctrl->n_next, 1u)] = e;
    }
}

// Warp per edge of S.
__global__ void k_incidence(const uint32_t *__restrict__ S, uint32_t nS, uint32_t round,
                            long long k, const uint64_t *__restrict__ inc_off,
                            const uint32_t *__restrict__ inc, const uint2 *__restrict__ pairs,
                            const uint32_t *__restrict__ pair_bloom, uint8_t *pair_alive,
                            const uint32_t *__restrict__ bk, uint32_t *C, uint32_t *touched,
                            long long *sup, uint32_t *state, uint32_t *S_next, uint32_t *phi,
                            Ctrl *ctrl) {
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    unsigned long long upd = 0;
    for (uint32_t i = warp; i < nS; i += nwarps) {
        const uint32_t e = S[i];
        if (lane == 0) phi[e] = (uint32_t)k;
        const uint64_t b = inc_off[e], end = inc_off[e + 1];
        for (uint64_t j = b + lane; j < end; j += 32) {
            const uint32_t p = inc[j];
            if (!pair_alive[p]) continue;
            const uint2 pr = pairs[p];
            const uint32_t t = pr.x == e ? pr.y : pr.x;
            const uint32_t st = state[t];
            if (st == round && t < e) continue;  // twin in S with smaller id owns the pair
            pair_alive[p] = 0;
            const uint32_t B = pair_bloom[p];
            if (atomicAdd(&C[B], 1u) == 0u) touched[atomicAdd(&ctrl->n_touched, 1u)] = B;
            if (st != round) {
                const long long dec = (long long)bk[B] - 1;
                if (dec > 0) {
                    decrement(sup, state, S_next, ctrl, t, dec, k, round);
                    ++upd;
                }
            }
        }
    }
    upd = dev::warp_sum(upd);
    if (lane == 0 && upd) atomicAdd(&ctrl->updates, upd);
}

// Warp per touched bloom.
__global__ void k_bloom(const uint32_t *__restrict__ touched, const uint32_t *__restrict__ bloom_off, const uint2 *__restrict__ pairs,
                        const uint8_t *__restrict__ pair_alive, uint32_t *bk, uint32_t *C,
                        long long *sup, uint32_t *state, uint32_t *S_next, uint32_t round,
                        long long k, Ctrl *ctrl) {
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t nt = *(volatile uint32_t *)&ctrl->n_touched;
    unsigned long long upd = 0;
    for (uint32_t i = warp; i < nt; i += nwarps) {
        const uint32_t B = touched[i];
        const uint32_t c = C[B];
        const uint32_t b = bloom_off[B], end = bloom_off[B + 1];
        for (uint32_t p = b + lane; p < end; p += 32) {
            if (!pair_alive[p]) continue;
            const uint2 pr = pairs[p];
            decrement(sup, state, S_next, ctrl, pr.x, c, k, round);
            decrement(sup, state, S_next, ctrl, pr.y, c, k, round);
            upd += 2;
        }
        if (lane == 0) {
            bk[B] -= c;
            C[B] = 0;
        }
    }
    upd = dev::warp_sum(upd);
    if (lane == 0 && upd) atomicAdd(&ctrl->updates, upd);
}

inline unsigned grid_for(uint64_t items, int threads, unsigned cap) {
    uint64_t g = (items + threads - 1) / threads;
    if (g == 0) g = 1;
    return (unsigned)(g < cap ? g : cap);
}

}  // namespace

cudaError_t peel(const Index &ix, const uint64_t *support, uint32_t *phi_out, PeelResult &res,
                 int num_sms, Alloc &al) {
    const uint64_t m = ix.m;
    res = PeelResult{};
    if (m == 0) return cudaSuccess;
    long long *sup = al.get<long long>(m);
    uint32_t *state = al.get<uint32_t>(m);
    uint32_t *S = al.get<uint32_t>(m);
    uint32_t *S_next = al.get<uint32_t>(m);
    uint8_t *pair_alive = al.get<uint8_t>(ix.w2);
    uint32_t *bk = al.get<uint32_t>(ix.nb);
    uint32_t *C = al.get<uint32_t>(ix.nb);
    uint32_t *touched = al.get<uint32_t>(ix.nb);
    Ctrl *ctrl = al.get<Ctrl>(1);
    if (al.err != cudaSuccess) return al.err;
    cudaStream_t st = al.stream;
    al.mark(kPhPeel, false);
    const unsigned cap = (unsigned)num_sms * 16;
    k_peel_init<<<grid_for(m, 256, cap), 256, 0, st>>>(support, m, sup, state);
    al.launches++;
    BT_CUDA(cudaMemsetAsync(pair_alive, 1, ix.w2 ? ix.w2 : 1, st));
    if (ix.nb) {
        BT_CUDA(cudaMemcpyAsync(bk, ix.bloom_k, sizeof(uint32_t) * ix.nb, cudaMemcpyDeviceToDevice, st));
        BT_CUDA(cudaMemsetAsync(C, 0, sizeof(uint32_t) * ix.nb, st));
    }
    BT_CUDA(cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st));
    Ctrl h{};
    uint64_t remaining = m;
    uint32_t nS = 0;
    long long k = 0;
    uint32_t round = 0;
    const uint64_t round_limit = m + 1;
    while (remaining > 0) {
        if (nS == 0) {
            unsigned long long init = ~0ull;
            BT_CUDA(cudaMemcpyAsync(&ctrl->minsup, &init, sizeof(init), cudaMemcpyHostToDevice, st));
            BT_CUDA(cudaMemsetAsync(&ctrl->n_collect, 0, sizeof(uint32_t), st));
            k_min_alive<<<grid_for(m, 256, cap), 256, 0, st>>>(state, sup, m, ctrl);
            al.launches++;
            BT_CUDA(cudaMemcpyAsync(&h, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
            BT_CUDA(cudaStreamSynchronize(st));
            if (h.minsup == ~0ull) break;  // no alive edge left (cannot happen while remaining > 0)
            long long mn = (long long)h.minsup;
            if (mn > k) k = mn;
            if ((unsigned long long)k > 0xFFFFFFFFull) {
                res.status = BT_ERR_OVERFLOW;
                break;
            }
            k_collect<<<grid_for(m, 256, cap), 256, 0, st>>>(state, sup, m, k, round, S, ctrl);
            al.launches++;
            BT_CUDA(cudaMemcpyAsync(&h, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
            BT_CUDA(cudaStreamSynchronize(st));
            nS = h.n_collect;
            ++res.levels;
            if (nS == 0) {
                res.status = BT_ERR_NOCONVERGE;
                break;
            }
        }
        BT_CUDA(cudaMemsetAsync(&ctrl->n_next, 0, 2 * sizeof(uint32_t), st));  // n_next, n_touched
        k_incidence<<<grid_for((uint64_t)nS * 32, 256, cap), 256, 0, st>>>(
            S, nS, round, k, ix.inc_off, ix.inc, ix.pairs, ix.pair_bloom, pair_alive, bk, C,
            touched, sup, state, S_next, phi_out, ctrl);
        al.launches++;
        k_bloom<<<cap, 256, 0, st>>>(touched, ix.bloom_off, ix.pairs, pair_alive, bk, C, sup,
                                     state, S_next, round, k, ctrl);
        al.launches++;
        BT_CUDA(cudaGetLastError());
        BT_CUDA(cudaMemcpyAsync(&h, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
        BT_CUDA(cudaStreamSynchronize(st));
        remaining -= nS;
        uint32_t *t = S;
        S = S_next;
        S_next = t;
        nS = h.n_next;
        ++round;
        if (round > round_limit) {
            res.status = BT_ERR_NOCONVERGE;
            break;
        }
    }
    al.mark(kPhPeel, true);
    res.rounds = round;
    res.updates = h.updates;
    res.kmax = (uint64_t)k;
    al.put(sup);
    al.put(state);
    al.put(S);
    al.put(S_next);
    al.put(pair_alive);
    al.put(bk);
    al.put(C);
    al.put(touched);
    al.put(ctrl);
    return cudaSuccess;
}

}  // namespace bt
