/*
 * CPU oracle for bitruss decomposition -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this library.  The product path (the CUDA library) shares no code,
 * header, helper or table with it, and neither side includes the other.
 *
 * What it computes (Section II, "Problem Definition"):
 *   support(e)  = number of butterflies ((2,2)-bicliques, Def. 2) containing e
 *   phi(e)      = the largest k such that some k-bitruss (Def. 4) contains e
 *                 (the bitruss number, Def. 5); 0 when e is in no butterfly.
 *
 * Both are computed "the slow, obvious way" that the paper describes as the
 * prior art (Section III, Alg. 1, BiT-BS):
 *   - support by direct enumeration: for e=(u,v),
 *       support(e) = sum over w in N(v)\{u} of ( |N(u) ∩ N(w)| - 1 ),
 *     i.e. every pair (w, x) with x in N(u) ∩ N(w) \ {v} closes a butterfly
 *     [u, v, w, x];
 *   - phi by one-edge-at-a-time bottom-up peeling: repeatedly take an
 *     unassigned edge e of minimum current support, set phi(e) = support(e),
 *     enumerate every butterfly [u, v, w, x] through e in the current graph
 *     and decrement the support of each of its other three edges whose
 *     support is larger than support(e) (Alg. 1), then delete e.
 * No priority ordering, no blooms and no batching are used here: the oracle
 * is independent of the method it checks (BE-Index, Section IV; BiT-BU++,
 * Alg. 5).
 *
 * A fourth routine splits the supports by the anchor of each butterfly: the
 * butterfly's vertex of highest priority (Def. 7: degree, then global id).
 * Lemma 3 puts every butterfly in exactly one maximal priority-obeyed bloom,
 * the one started at that vertex, so the supports contributed by the
 * butterflies anchored in disjoint rank ranges sum to the supports.  It is
 * the definition a counting shard over start-vertex ranges must reproduce.
 *
 * A third routine evaluates, for sampled edges, the local fixpoint property
 * that any correct phi satisfies (follows from Defs. 4-5): phi(e) equals the
 * largest j such that at least j butterflies through e have all their other
 * three edges with phi >= j.  It serves as a full-size check where the full
 * peeling is too slow.
 *
 * Edge input: int32 pairs (u, v), u in [0, nU) upper layer, v in [0, nL)
 * lower layer, m distinct edges.  Returns 0 on success, negative on error
 * (-1 allocation, -2 id out of range, -3 duplicate edge).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    uint32_t nU, nL;
    uint64_t m;
    /* upper vertices: neighbours (lower ids) sorted ascending, with edge ids */
    uint64_t *offU; uint32_t *adjU; uint32_t *eidU;
    /* lower vertices: neighbours (upper ids) sorted ascending, with edge ids */
    uint64_t *offL; uint32_t *adjL; uint32_t *eidL;
} og_t;

static void og_free(og_t *g) {
    free(g->offU); free(g->adjU); free(g->eidU);
    free(g->offL); free(g->adjL); free(g->eidL);
}

/* sort (key, val) pairs of one adjacency list by key: insertion sort for short
 * lists, heap sort otherwise (plain, no tricks). */
static void sort_pairs(uint32_t *k, uint32_t *v, uint64_t n) {
    if (n < 32) {
        for (uint64_t i = 1; i < n; ++i) {
            uint32_t kk = k[i], vv = v[i];
            uint64_t j = i;
            while (j > 0 && k[j - 1] > kk) { k[j] = k[j - 1]; v[j] = v[j - 1]; --j; }
            k[j] = kk; v[j] = vv;
        }
        return;
    }
    /* heap sort */
    for (uint64_t s = n / 2; s-- > 0;) {
        uint64_t r = s;
        for (;;) {
            uint64_t c = 2 * r + 1;
            if (c >= n) break;
            if (c + 1 < n && k[c + 1] > k[c]) ++c;
            if (k[r] >= k[c]) break;
            uint32_t t = k[r]; k[r] = k[c]; k[c] = t;
            t = v[r]; v[r] = v[c]; v[c] = t;
            r = c;
        }
    }
    for (uint64_t end = n - 1; end > 0; --end) {
        uint32_t t = k[0]; k[0] = k[end]; k[end] = t;
        t = v[0]; v[0] = v[end]; v[end] = t;
        uint64_t r = 0;
        for (;;) {
            uint64_t c = 2 * r + 1;
            if (c >= end) break;
            if (c + 1 < end && k[c + 1] > k[c]) ++c;
            if (k[r] >= k[c]) break;
            t = k[r]; k[r] = k[c]; k[c] = t;
            t = v[r]; v[r] = v[c]; v[c] = t;
            r = c;
        }
    }
}

static int og_build(og_t *g, const int32_t *edges, uint64_t m, uint32_t nU, uint32_t nL) {
    memset(g, 0, sizeof(*g));
    g->nU = nU; g->nL = nL; g->m = m;
    g->offU = (uint64_t *)calloc((uint64_t)nU + 1, sizeof(uint64_t));
    g->offL = (uint64_t *)calloc((uint64_t)nL + 1, sizeof(uint64_t));
    g->adjU = (uint32_t *)malloc(sizeof(uint32_t) * (m ? m : 1));
    g->eidU = (uint32_t *)malloc(sizeof(uint32_t) * (m ? m : 1));
    g->adjL = (uint32_t *)malloc(sizeof(uint32_t) * (m ? m : 1));
    g->eidL = (uint32_t *)malloc(sizeof(uint32_t) * (m ? m : 1));
    if (!g->offU || !g->offL || !g->adjU || !g->eidU || !g->adjL || !g->eidL) { og_free(g); return -1; }
    for (uint64_t i = 0; i < m; ++i) {
        int32_t u = edges[2 * i], v = edges[2 * i + 1];
        if (u < 0 || v < 0 || (uint32_t)u >= nU || (uint32_t)v >= nL) { og_free(g); return -2; }
        g->offU[u + 1]++;
        g->offL[v + 1]++;
    }
    for (uint32_t i = 0; i < nU; ++i) g->offU[i + 1] += g->offU[i];
    for (uint32_t i = 0; i < nL; ++i) g->offL[i + 1] += g->offL[i];
    uint64_t *fu = (uint64_t *)malloc(sizeof(uint64_t) * ((uint64_t)nU + 1));
    uint64_t *fl = (uint64_t *)malloc(sizeof(uint64_t) * ((uint64_t)nL + 1));
    if (!fu || !fl) { free(fu); free(fl); og_free(g); return -1; }
    memcpy(fu, g->offU, sizeof(uint64_t) * ((uint64_t)nU + 1));
    memcpy(fl, g->offL, sizeof(uint64_t) * ((uint64_t)nL + 1));
    for (uint64_t i = 0; i < m; ++i) {
        uint32_t u = (uint32_t)edges[2 * i], v = (uint32_t)edges[2 * i + 1];
        g->adjU[fu[u]] = v; g->eidU[fu[u]++] = (uint32_t)i;
        g->adjL[fl[v]] = u; g->eidL[fl[v]++] = (uint32_t)i;
    }
    free(fu); free(fl);
    for (uint32_t u = 0; u < nU; ++u) {
        uint64_t a = g->offU[u], b = g->offU[u + 1];
        sort_pairs(g->adjU + a, g->eidU + a, b - a);
        for (uint64_t j = a + 1; j < b; ++j)
            if (g->adjU[j] == g->adjU[j - 1]) { og_free(g); return -3; }
    }
    for (uint32_t v = 0; v < nL; ++v) {
        uint64_t a = g->offL[v], b = g->offL[v + 1];
        sort_pairs(g->adjL + a, g->eidL + a, b - a);
    }
    return 0;
}

/* position of key in sorted list, or -1 */
static int64_t find_sorted(const uint32_t *a, uint64_t n, uint32_t key) {
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return (lo < n && a[lo] == key) ? (int64_t)lo : -1;
}

/* |N(u) ∩ N(w)| for two upper vertices: walk the shorter list, search the longer */
static uint64_t common_lower(const og_t *g, uint32_t u, uint32_t w) {
    const uint32_t *a = g->adjU + g->offU[u], *b = g->adjU + g->offU[w];
    uint64_t na = g->offU[u + 1] - g->offU[u], nb = g->offU[w + 1] - g->offU[w];
    if (na > nb) { const uint32_t *t = a; a = b; b = t; uint64_t tn = na; na = nb; nb = tn; }
    uint64_t c = 0;
    for (uint64_t i = 0; i < na; ++i) c += find_sorted(b, nb, a[i]) >= 0;
    return c;
}

static uint64_t support_of(const og_t *g, uint64_t e, const int32_t *edges) {
    uint32_t u = (uint32_t)edges[2 * e], v = (uint32_t)edges[2 * e + 1];
    uint64_t s = 0;
    for (uint64_t j = g->offL[v]; j < g->offL[v + 1]; ++j) {
        uint32_t w = g->adjL[j];
        if (w == u) continue;
        s += common_lower(g, u, w) - 1; /* v itself is always common */
    }
    return s;
}

int oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* support of every edge (OpenMP over edges, read-only graph) */
int oracle_support(const int32_t *edges, uint64_t m, uint32_t nU, uint32_t nL, uint64_t *sup) {
    og_t g;
    int rc = og_build(&g, edges, m, nU, nL);
    if (rc) return rc;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t e = 0; e < (int64_t)m; ++e) sup[e] = support_of(&g, (uint64_t)e, edges);
    og_free(&g);
    return 0;
}

/* support of the queried edges only */
int oracle_support_sampled(const int32_t *edges, uint64_t m, uint32_t nU, uint32_t nL,
                           const uint64_t *which, uint64_t nq, uint64_t *sup) {
    og_t g;
    int rc = og_build(&g, edges, m, nU, nL);
    if (rc) return rc;
    for (uint64_t i = 0; i < nq; ++i) if (which[i] >= m) { og_free(&g); return -2; }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < (int64_t)nq; ++i) sup[i] = support_of(&g, which[i], edges);
    og_free(&g);
    return 0;
}

/* ---- indexed binary min-heap on (support, edge id) with decrease-key ---- */
typedef struct { uint32_t *h; uint32_t *pos; const uint64_t *key; uint64_t n; } heap_t;

static inline int hless(const heap_t *H, uint32_t a, uint32_t b) {
    return H->key[a] < H->key[b] || (H->key[a] == H->key[b] && a < b);
}
static void hswap(heap_t *H, uint64_t i, uint64_t j) {
    uint32_t t = H->h[i]; H->h[i] = H->h[j]; H->h[j] = t;
    H->pos[H->h[i]] = (uint32_t)i; H->pos[H->h[j]] = (uint32_t)j;
}
static void hup(heap_t *H, uint64_t i) {
    while (i > 0) {
        uint64_t p = (i - 1) / 2;
        if (!hless(H, H->h[i], H->h[p])) break;
        hswap(H, i, p); i = p;
    }
}
static void hdown(heap_t *H, uint64_t i) {
    for (;;) {
        uint64_t l = 2 * i + 1, r = l + 1, s = i;
        if (l < H->n && hless(H, H->h[l], H->h[s])) s = l;
        if (r < H->n && hless(H, H->h[r], H->h[s])) s = r;
        if (s == i) break;
        hswap(H, i, s); i = s;
    }
}
static uint32_t hpop(heap_t *H) {
    uint32_t top = H->h[0];
    hswap(H, 0, H->n - 1);
    H->n--;
    if (H->n) hdown(H, 0);
    return top;
}

/*
 * Support (initial) and bitruss number of every edge by Alg. 1 (BiT-BS).
 * sup_out receives the initial supports; phi_out the bitruss numbers (u64).
 */
int oracle_bitruss(const int32_t *edges, uint64_t m, uint32_t nU, uint32_t nL,
                   uint64_t *sup_out, uint64_t *phi_out) {
    og_t g;
    int rc = og_build(&g, edges, m, nU, nL);
    if (rc) return rc;
    uint64_t *s = (uint64_t *)malloc(sizeof(uint64_t) * (m ? m : 1));
    uint8_t *alive = (uint8_t *)malloc(m ? m : 1);
    heap_t H;
    H.h = (uint32_t *)malloc(sizeof(uint32_t) * (m ? m : 1));
    H.pos = (uint32_t *)malloc(sizeof(uint32_t) * (m ? m : 1));
    if (!s || !alive || !H.h || !H.pos) { og_free(&g); return -1; }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t e = 0; e < (int64_t)m; ++e) s[e] = support_of(&g, (uint64_t)e, edges);
    memcpy(sup_out, s, sizeof(uint64_t) * m);
    H.key = s; H.n = m;
    for (uint64_t e = 0; e < m; ++e) { H.h[e] = (uint32_t)e; H.pos[e] = (uint32_t)e; alive[e] = 1; }
    for (uint64_t i = m / 2; i-- > 0;) hdown(&H, i);

    while (H.n) {
        uint32_t e = hpop(&H);
        uint64_t se = s[e];
        phi_out[e] = se;
        uint32_t u = (uint32_t)edges[2 * (uint64_t)e], v = (uint32_t)edges[2 * (uint64_t)e + 1];
        /* every butterfly [u, v, w, x] of the current graph through e */
        for (uint64_t j = g.offL[v]; j < g.offL[v + 1]; ++j) {
            uint32_t w = g.adjL[j], ewv = g.eidL[j];
            if (w == u || !alive[ewv]) continue;
            const uint32_t *nu = g.adjU + g.offU[u], *nw = g.adjU + g.offU[w];
            const uint32_t *iu = g.eidU + g.offU[u], *iw = g.eidU + g.offU[w];
            uint64_t du = g.offU[u + 1] - g.offU[u], dw = g.offU[w + 1] - g.offU[w];
            int walk_u = du <= dw;
            uint64_t nwalk = walk_u ? du : dw;
            for (uint64_t t = 0; t < nwalk; ++t) {
                uint32_t x = walk_u ? nu[t] : nw[t];
                if (x == v) continue;
                int64_t p = walk_u ? find_sorted(nw, dw, x) : find_sorted(nu, du, x);
                if (p < 0) continue;
                uint32_t eux = walk_u ? iu[t] : iu[p];
                uint32_t ewx = walk_u ? iw[p] : iw[t];
                if (!alive[eux] || !alive[ewx]) continue;
                uint32_t other[3] = {eux, ewv, ewx};
                for (int q = 0; q < 3; ++q) {
                    uint32_t f = other[q];
                    if (s[f] > se) { s[f] -= 1; hup(&H, H.pos[f]); }
                }
            }
        }
        alive[e] = 0;
    }
    free(s); free(alive); free(H.h); free(H.pos);
    og_free(&g);
    return 0;
}

/*
 * For each queried edge e: the number of butterflies through e whose other
 * three edges all have phi >= phi(e) (cnt_at_phi), and the local h-value
 * h(e) = max j such that >= j butterflies through e have min phi of their
 * other three edges >= j.  A correct phi has h(e) == phi(e) and
 * cnt_at_phi >= phi(e) for every e.
 */
int oracle_local_check(const int32_t *edges, uint64_t m, uint32_t nU, uint32_t nL,
                       const uint32_t *phi, const uint64_t *which, uint64_t nq,
                       uint64_t *cnt_at_phi, uint64_t *hval) {
    og_t g;
    int rc = og_build(&g, edges, m, nU, nL);
    if (rc) return rc;
    for (uint64_t i = 0; i < nq; ++i) if (which[i] >= m) { og_free(&g); return -2; }
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t qi = 0; qi < (int64_t)nq; ++qi) {
        uint64_t e = which[qi];
        uint32_t u = (uint32_t)edges[2 * e], v = (uint32_t)edges[2 * e + 1];
        uint64_t pe = phi[e];
        /* strengths of all butterflies through e */
        uint64_t cap = 1024, n = 0;
        uint32_t *str = (uint32_t *)malloc(sizeof(uint32_t) * cap);
        if (!str) { bad = 1; continue; }
        for (uint64_t j = g.offL[v]; j < g.offL[v + 1]; ++j) {
            uint32_t w = g.adjL[j], ewv = g.eidL[j];
            if (w == u) continue;
            const uint32_t *nu = g.adjU + g.offU[u], *nw = g.adjU + g.offU[w];
            const uint32_t *iu = g.eidU + g.offU[u], *iw = g.eidU + g.offU[w];
            uint64_t du = g.offU[u + 1] - g.offU[u], dw = g.offU[w + 1] - g.offU[w];
            for (uint64_t t = 0; t < du; ++t) {
                uint32_t x = nu[t];
                if (x == v) continue;
                int64_t p = find_sorted(nw, dw, x);
                if (p < 0) continue;
                uint32_t a = phi[iu[t]], b = phi[ewv], c = phi[iw[p]];
                uint32_t mn = a < b ? a : b;
                mn = mn < c ? mn : c;
                if (n == cap) {
                    cap *= 2;
                    uint32_t *ns = (uint32_t *)realloc(str, sizeof(uint32_t) * cap);
                    if (!ns) { bad = 1; break; }
                    str = ns;
                }
                str[n++] = mn;
            }
        }
        uint64_t c_at = 0;
        for (uint64_t i = 0; i < n; ++i) c_at += str[i] >= pe;
        /* h-index: sort descending by counting on capped values */
        uint64_t *hist = (uint64_t *)calloc(n + 2, sizeof(uint64_t));
        if (!hist) { bad = 1; free(str); continue; }
        for (uint64_t i = 0; i < n; ++i) hist[str[i] > n ? n : str[i]]++;
        uint64_t h = 0, acc = 0;
        for (uint64_t j = n + 1; j-- > 0;) {
            acc += hist[j];
            if (acc >= j) { h = j; break; }
        }
        cnt_at_phi[qi] = c_at;
        hval[qi] = h;
        free(hist);
        free(str);
    }
    og_free(&g);
    return bad ? -1 : 0;
}

/*
 * Supports counting only the butterflies whose anchor -- the butterfly's
 * vertex of highest priority, Def. 7: larger degree, ties broken by the
 * larger global id -- has a priority rank in [rank_lo, rank_hi) (rank 0 is
 * the lowest priority).  Global ids follow Section II (lower v -> v, upper
 * u -> nL + u), or with lower_first the reading of Fig. 6 (upper u -> u,
 * lower v -> nU + v).  Butterflies through e = (u, v) are enumerated as in
 * support_of: w in N(v) \ {u}, x in N(u) ∩ N(w) \ {v}.
 */
int oracle_support_anchored(const int32_t *edges, uint64_t m, uint32_t nU, uint32_t nL, int lower_first,
                            uint64_t rank_lo, uint64_t rank_hi, uint64_t *sup) {
    og_t g;
    int rc = og_build(&g, edges, m, nU, nL);
    if (rc) return rc;
    const uint64_t n = (uint64_t)nU + nL;
    /* rank of every vertex: upper u at index u, lower v at index nU + v */
    uint64_t *key = (uint64_t *)malloc(sizeof(uint64_t) * (n ? n : 1));
    uint32_t *idx = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    uint32_t *rank = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    if (!key || !idx || !rank) { free(key); free(idx); free(rank); og_free(&g); return -1; }
    for (uint64_t x = 0; x < n; ++x) {
        int upper = x < nU;
        uint64_t deg = upper ? g.offU[x + 1] - g.offU[x] : g.offL[x - nU + 1] - g.offL[x - nU];
        uint64_t gid = upper ? (lower_first ? x : (uint64_t)nL + x) : (lower_first ? x : x - nU);
        key[x] = deg << 32 | gid; /* degrees and ids < 2^32 */
        idx[x] = (uint32_t)x;
    }
    /* sort vertex indices by key ascending (heap sort on (key, idx)) */
    for (uint64_t s0 = n / 2; s0-- > 0;) {
        uint64_t r = s0;
        for (;;) {
            uint64_t c = 2 * r + 1;
            if (c >= n) break;
            if (c + 1 < n && key[idx[c + 1]] > key[idx[c]]) ++c;
            if (key[idx[r]] >= key[idx[c]]) break;
            uint32_t t = idx[r]; idx[r] = idx[c]; idx[c] = t;
            r = c;
        }
    }
    for (uint64_t end = n; end-- > 1;) {
        uint32_t t = idx[0]; idx[0] = idx[end]; idx[end] = t;
        uint64_t r = 0;
        for (;;) {
            uint64_t c = 2 * r + 1;
            if (c >= end) break;
            if (c + 1 < end && key[idx[c + 1]] > key[idx[c]]) ++c;
            if (key[idx[r]] >= key[idx[c]]) break;
            t = idx[r]; idx[r] = idx[c]; idx[c] = t;
            r = c;
        }
    }
    for (uint64_t r = 0; r < n; ++r) rank[idx[r]] = (uint32_t)r;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t e = 0; e < (int64_t)m; ++e) {
        uint32_t u = (uint32_t)edges[2 * e], v = (uint32_t)edges[2 * e + 1];
        uint64_t s = 0;
        for (uint64_t j = g.offL[v]; j < g.offL[v + 1]; ++j) {
            uint32_t w = g.adjL[j];
            if (w == u) continue;
            const uint32_t *nu = g.adjU + g.offU[u], *nw = g.adjU + g.offU[w];
            uint64_t du = g.offU[u + 1] - g.offU[u], dw = g.offU[w + 1] - g.offU[w];
            for (uint64_t t = 0; t < du; ++t) {
                uint32_t x = nu[t];
                if (x == v || find_sorted(nw, dw, x) < 0) continue;
                /* butterfly {u, w} x {v, x}: its anchor's rank */
                uint32_t top = rank[u];
                if (rank[w] > top) top = rank[w];
                if (rank[nU + v] > top) top = rank[nU + v];
                if (rank[nU + x] > top) top = rank[nU + x];
                s += top >= rank_lo && top < rank_hi;
            }
        }
        sup[e] = s;
    }
    free(key); free(idx); free(rank);
    og_free(&g);
    return 0;
}
