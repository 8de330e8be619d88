/*
 * Seeded synthetic bipartite graphs (Chung-Lu model with power-law expected
 * degrees, optional degree cap and optional planted dense bicliques).
 *
 * This file is input generation only: it holds none of the bitruss method's
 * arithmetic (no butterfly, bloom or peeling logic).  Both the CPU oracle
 * harness and the GPU harness call it to obtain identical inputs.
 *
 * Random numbers: xoshiro256** (Blackman & Vigna, 2018) seeded through
 * SplitMix64 (Steele, Lea & Flood, 2014), both written from their published
 * definitions.  Vertex sampling uses Vose's alias method.
 *
 * Model (stand-in for the paper's skewed real-world graphs, Table 3):
 *   w_i ∝ (i+1)^(-1/(gamma-1)) on each side, scaled so that sum_i w_i = m,
 *   then capped at min(cap, size of the other side).  Edges are drawn as
 *   (u ~ w^U, v ~ w^L) independently; duplicates and draws that would push a
 *   vertex over the cap are rejected until m distinct edges exist.  Vertex ids
 *   on both sides and the edge order are then shuffled.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64_next(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t rng_next(rng_t *r) {
    uint64_t *s = r->s;
    uint64_t out = rotl64(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return out;
}

static void rng_seed(rng_t *r, uint64_t seed) {
    uint64_t x = seed;
    for (int i = 0; i < 4; ++i) r->s[i] = splitmix64_next(&x);
}

/* uniform double in [0,1) from the top 53 bits */
static inline double rng_unit(rng_t *r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }

/* uniform integer in [0,n) by 128-bit multiply (bias < n / 2^64, negligible) */
static inline uint64_t rng_below(rng_t *r, uint64_t n) {
    return (uint64_t)(((unsigned __int128)rng_next(r) * (unsigned __int128)n) >> 64);
}

/* SplitMix64 of a single value: used to derive per-graph seeds. */
uint64_t synth_splitmix(uint64_t x) { return splitmix64_next(&x); }

/* ---- alias table (Vose) ---- */
typedef struct { double *prob; uint32_t *alias; uint32_t n; } alias_t;

static int alias_build(alias_t *a, const double *w, uint32_t n) {
    a->n = n;
    a->prob = (double *)malloc(sizeof(double) * (n ? n : 1));
    a->alias = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    uint32_t *small = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    uint32_t *large = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    double *p = (double *)malloc(sizeof(double) * (n ? n : 1));
    if (!a->prob || !a->alias || !small || !large || !p) return -1;
    double tot = 0;
    for (uint32_t i = 0; i < n; ++i) tot += w[i];
    uint32_t ns = 0, nl = 0;
    for (uint32_t i = 0; i < n; ++i) {
        p[i] = w[i] * (double)n / tot;
        if (p[i] < 1.0) small[ns++] = i; else large[nl++] = i;
    }
    while (ns && nl) {
        uint32_t s = small[--ns], l = large[--nl];
        a->prob[s] = p[s];
        a->alias[s] = l;
        p[l] = (p[l] + p[s]) - 1.0;
        if (p[l] < 1.0) small[ns++] = l; else large[nl++] = l;
    }
    while (nl) { uint32_t l = large[--nl]; a->prob[l] = 1.0; a->alias[l] = l; }
    while (ns) { uint32_t s = small[--ns]; a->prob[s] = 1.0; a->alias[s] = s; }
    free(small); free(large); free(p);
    return 0;
}

static inline uint32_t alias_draw(const alias_t *a, rng_t *r) {
    uint32_t i = (uint32_t)rng_below(r, a->n);
    return rng_unit(r) < a->prob[i] ? i : a->alias[i];
}

static void alias_free(alias_t *a) { free(a->prob); free(a->alias); }

/* ---- open-addressing set of u64 keys (key 0 reserved as empty) ---- */
typedef struct { uint64_t *k; uint64_t mask; } set_t;

static int set_init(set_t *s, uint64_t want) {
    uint64_t cap = 16;
    while (cap < 2 * want + 16) cap <<= 1;
    s->k = (uint64_t *)calloc(cap, sizeof(uint64_t));
    s->mask = cap - 1;
    return s->k ? 0 : -1;
}

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* returns 1 if inserted, 0 if already present */
static int set_insert(set_t *s, uint64_t key) {
    uint64_t h = mix64(key) & s->mask;
    for (;;) {
        if (s->k[h] == 0) { s->k[h] = key; return 1; }
        if (s->k[h] == key) return 0;
        h = (h + 1) & s->mask;
    }
}

static void power_weights(double *w, uint32_t n, double gamma, double total, double capw) {
    double ex = -1.0 / (gamma - 1.0), s = 0;
    for (uint32_t i = 0; i < n; ++i) { w[i] = pow((double)(i + 1), ex); s += w[i]; }
    for (uint32_t i = 0; i < n; ++i) { w[i] *= total / s; if (w[i] > capw) w[i] = capw; }
}

static void shuffle_u32(uint32_t *a, uint64_t n, rng_t *r) {
    for (uint64_t i = n; i > 1; --i) {
        uint64_t j = rng_below(r, i);
        uint32_t t = a[i - 1]; a[i - 1] = a[j]; a[j] = t;
    }
}

/*
 * Generate a graph into edges_out (int32 pairs, length 2*m, caller-allocated).
 *   nplant bicliques: sides a,b ~ U[plant_lo, plant_hi], random vertex
 *   subsets, each edge kept with probability plant_p; they are placed first
 *   (counted toward m).  cap == 0 means no degree cap.
 * Returns 0 on success, -1 on allocation failure, -2 if m distinct edges
 * could not be drawn within the attempt budget, -3 on bad arguments.
 */
int synth_chunglu(uint32_t nU, uint32_t nL, uint64_t m, double gammaU, double gammaL,
                  uint32_t cap, uint32_t nplant, uint32_t plant_lo, uint32_t plant_hi,
                  double plant_p, uint64_t seed, int32_t *edges_out) {
    if (nU == 0 || nL == 0 || (double)m > (double)nU * (double)nL || gammaU <= 1.0 || gammaL <= 1.0)
        return m == 0 ? 0 : -3;
    rng_t r;
    rng_seed(&r, seed);
    uint32_t *du = (uint32_t *)calloc(nU, sizeof(uint32_t));
    uint32_t *dl = (uint32_t *)calloc(nL, sizeof(uint32_t));
    double *wu = (double *)malloc(sizeof(double) * nU);
    double *wl = (double *)malloc(sizeof(double) * nL);
    uint32_t *eu = (uint32_t *)malloc(sizeof(uint32_t) * (m ? m : 1));
    uint32_t *ev = (uint32_t *)malloc(sizeof(uint32_t) * (m ? m : 1));
    set_t set;
    if (!du || !dl || !wu || !wl || !eu || !ev || set_init(&set, m)) return -1;
    double capu = (double)nL, capl = (double)nU;
    if (cap) { if (capu > cap) capu = cap; if (capl > cap) capl = cap; }
    uint32_t hard_u = cap ? cap : nL, hard_l = cap ? cap : nU;
    power_weights(wu, nU, gammaU, (double)m, capu);
    power_weights(wl, nL, gammaL, (double)m, capl);
    uint64_t cnt = 0;

    /* planted bicliques */
    if (nplant) {
        uint32_t *pu = (uint32_t *)malloc(sizeof(uint32_t) * nU);
        uint32_t *pl = (uint32_t *)malloc(sizeof(uint32_t) * nL);
        if (!pu || !pl) return -1;
        for (uint32_t i = 0; i < nU; ++i) pu[i] = i;
        for (uint32_t i = 0; i < nL; ++i) pl[i] = i;
        for (uint32_t b = 0; b < nplant && cnt < m; ++b) {
            uint32_t a = plant_lo + (uint32_t)rng_below(&r, plant_hi - plant_lo + 1);
            uint32_t c = plant_lo + (uint32_t)rng_below(&r, plant_hi - plant_lo + 1);
            if (a > nU) a = nU;
            if (c > nL) c = nL;
            /* partial Fisher-Yates: first a (resp. c) entries become the subset */
            for (uint32_t i = 0; i < a; ++i) {
                uint32_t j = i + (uint32_t)rng_below(&r, nU - i);
                uint32_t t = pu[i]; pu[i] = pu[j]; pu[j] = t;
            }
            for (uint32_t i = 0; i < c; ++i) {
                uint32_t j = i + (uint32_t)rng_below(&r, nL - i);
                uint32_t t = pl[i]; pl[i] = pl[j]; pl[j] = t;
            }
            for (uint32_t i = 0; i < a && cnt < m; ++i)
                for (uint32_t j = 0; j < c && cnt < m; ++j) {
                    if (rng_unit(&r) >= plant_p) continue;
                    uint32_t u = pu[i], v = pl[j];
                    if (set_insert(&set, (uint64_t)u * nL + v + 1)) {
                        eu[cnt] = u; ev[cnt] = v; ++cnt; ++du[u]; ++dl[v];
                    }
                }
        }
        free(pu); free(pl);
    }

    alias_t au, al;
    if (alias_build(&au, wu, nU) || alias_build(&al, wl, nL)) return -1;
    uint64_t tries = 0, budget = 200 * (m + 1000);
    while (cnt < m) {
        if (++tries > budget) { cnt = UINT64_MAX; break; }
        uint32_t u = alias_draw(&au, &r), v = alias_draw(&al, &r);
        if (du[u] >= hard_u || dl[v] >= hard_l) continue;
        if (!set_insert(&set, (uint64_t)u * nL + v + 1)) continue;
        eu[cnt] = u; ev[cnt] = v; ++cnt; ++du[u]; ++dl[v];
    }
    alias_free(&au); alias_free(&al);
    int rc = 0;
    if (cnt == UINT64_MAX) {
        rc = -2;
    } else {
        /* relabel both sides and shuffle edge order */
        uint32_t *perm_u = (uint32_t *)malloc(sizeof(uint32_t) * nU);
        uint32_t *perm_l = (uint32_t *)malloc(sizeof(uint32_t) * nL);
        uint32_t *order = (uint32_t *)malloc(sizeof(uint32_t) * (m ? m : 1));
        if (!perm_u || !perm_l || !order) return -1;
        for (uint32_t i = 0; i < nU; ++i) perm_u[i] = i;
        for (uint32_t i = 0; i < nL; ++i) perm_l[i] = i;
        for (uint64_t i = 0; i < m; ++i) order[i] = (uint32_t)i;
        shuffle_u32(perm_u, nU, &r);
        shuffle_u32(perm_l, nL, &r);
        shuffle_u32(order, m, &r);
        for (uint64_t i = 0; i < m; ++i) {
            uint32_t j = order[i];
            edges_out[2 * i] = (int32_t)perm_u[eu[j]];
            edges_out[2 * i + 1] = (int32_t)perm_l[ev[j]];
        }
        free(perm_u); free(perm_l); free(order);
    }
    free(du); free(dl); free(wu); free(wl); free(eu); free(ev); free(set.k);
    return rc;
}

/* Uniform draws for harness use (graph-size / exponent sampling). */
double synth_unit_from(uint64_t seed, uint32_t index) {
    rng_t r;
    rng_seed(&r, seed);
    double x = 0;
    for (uint32_t i = 0; i <= index; ++i) x = rng_unit(&r);
    return x;
}
