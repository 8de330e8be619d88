/*
 * bitruss.h -- C ABI of the GB300 (sm_103a) bitruss decomposition library
 * (libbitruss.so).
 *
 * Method: "Efficient Bitruss Decomposition for Large-scale Bipartite Graphs"
 * (arXiv 2001.06111).  The library computes, for a bipartite graph
 * G(U, L, E) given as an edge list,
 *   support(e) -- the butterfly support of every edge (Section II, Defs. 2-3),
 *                 counted by priority-obeyed wedge enumeration (Def. 10, Section IV-B,
 *                 Alg. 3; vertex priority of Def. 7);
 *   the BE-Index -- maximal priority-obeyed blooms with their bloom numbers,
 *                 edge-bloom links and twin edges (Section IV-A, Defs. 8-9,
 *                 built as in Alg. 3);
 *   phi(e)     -- the bitruss number of every edge (Defs. 4-5), by
 *                 level-synchronous batch peeling through the BE-Index
 *                 (Section V-B, Alg. 5 with the <= k rule of Alg. 4).
 *
 * Conventions shared by all calls
 *   - Edges: int32 pairs (u, v), row-major, 2*m values; u in [0, nU) names an
 *     upper-layer vertex, v in [0, nL) a lower-layer vertex.  Edges must be
 *     distinct.  Outputs are indexed like the input edges.
 *   - Pointers are host pointers unless flags contain BT_DEVICE_PTRS, in which
 *     case every edge/output pointer of that call is a device pointer on the
 *     handle's device.  The caller owns all input and output memory; the
 *     library never frees it and never keeps it past the call.
 *   - Vertex ids: the paper orders equal-degree vertices by a global id with
 *     every upper id above every lower id (Section II).  BT_TIE_LOWER_FIRST
 *     puts the lower layer above instead (the reading under which the paper's
 *     Fig. 6 index is reproduced).  Supports and bitruss numbers do not
 *     depend on this choice; only the BE-Index layout does.
 *   - Every call returns a bt_status.  On failure bt_last_error() describes
 *     it; outputs are then unspecified.  No call throws or aborts.
 *   - Calls on one handle are serialised by the caller (a handle is not
 *     thread-safe); different handles may be used from different threads.
 *   - All device work is issued on the handle's stream.  A call returns after
 *     its results are in the caller's buffers (it synchronises that stream).
 */
#ifndef BITRUSS_H
#define BITRUSS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BT_OK = 0,
    BT_ERR_ARG = 1,         /* null pointer, bad size or flag */
    BT_ERR_RANGE = 2,       /* a vertex id outside [0,nU) / [0,nL) */
    BT_ERR_DUP = 3,         /* the same edge appears twice */
    BT_ERR_NOMEM = 4,       /* device allocation failed */
    BT_ERR_OVERFLOW = 5,    /* a count exceeds its storage type (e.g. phi > 2^32-1) */
    BT_ERR_NOCONVERGE = 6,  /* peeling exceeded its round limit */
    BT_ERR_CUDA = 7,        /* a CUDA runtime call failed */
    BT_ERR_STATE = 8,       /* call needs state the handle does not hold */
    BT_ERR_TOO_LARGE = 9,   /* graph exceeds bt_count_support_static's fixed capacity */
    BT_ERR_CANCELLED = 10   /* a queued serving request was cancelled (bt_server_cancel_queued) */
} bt_status;

/* flags */
#define BT_DEVICE_PTRS 0x1u      /* edge/output pointers are device pointers */
#define BT_TIE_LOWER_FIRST 0x2u  /* lower-layer global ids above upper-layer ids */
#define BT_PC_RECOUNT 0x4u       /* bt_decompose_progressive: Alg. 7's candidate extraction */

typedef struct bt_handle bt_handle;

/* Sizes of a BE-Index (Section IV-A) and of the wedge work that built it. */
typedef struct {
    uint64_t n_wedges;        /* priority-obeyed wedges (Def. 10), W */
    uint64_t n_bloom_wedges;  /* wedges inside a bloom (end pair count >= 2), W2 = links/2 */
    uint64_t n_blooms;        /* maximal priority-obeyed blooms, |U(I)| */
    uint64_t n_butterflies;   /* sum over blooms of C(k,2) = butterflies of G (Lemmas 1, 3) */
    uint64_t index_bytes;     /* device bytes held by the index */
} bt_index_stats;

/* One bloom of the index copied out for inspection (bt_index_export). */
typedef struct {
    uint32_t k;               /* bloom number */
    uint32_t first_pair;      /* index of its first twin pair in pairs_out */
} bt_bloom_rec;

/* Per-call peel statistics (filled by bt_decompose when stats != NULL). */
typedef struct {
    uint64_t rounds;          /* peeling rounds (batches S, Alg. 5 line 4) */
    uint64_t levels;          /* distinct k values at which a batch was peeled */
    uint64_t support_updates; /* edge-support decrements applied (Fig. 10's count) */
    uint32_t phi_max;         /* largest bitruss number */
    uint32_t reserved;
} bt_peel_stats;

/* Per-call profile (bt_profile_read): CUDA-event times of the phases of the
 * last call on the handle, recorded on the handle's stream, and its kernel
 * launch count.  A phase that did not run reads 0. */
typedef struct {
    float csr_ms;      /* degree, rank and rank-ordered CSR build */
    float count_ms;    /* the wedge-count kernel (support attribution) */
    float emit_ms;     /* the BE-Index emit kernel */
    float peel_ms;     /* the whole peeling loop */
    float total_ms;    /* the whole call, host staging included */
    uint32_t reserved;
    uint64_t launches; /* kernels this call launched */
    uint64_t n_edges, n_vertices, n_wedges, n_bloom_wedges, n_blooms;
    uint64_t rounds, levels, support_updates;
    uint64_t pair_slots;   /* bloom pair slots the peel's bloom phase visited */
    uint64_t link_visits;  /* edge-bloom links the peel's incidence phase visited */
    uint64_t scanned;      /* edge-list entries the peel's level jumps scanned (the
                              near window, and the alive list when it is rebuilt) */
} bt_profile;

/*
 * Create a handle on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * to issue work on, or NULL to let the handle create and own one.
 * Errors: BT_ERR_ARG (h NULL), BT_ERR_CUDA (device unusable).
 */
int bt_create(bt_handle **h, int device, void *cuda_stream);

/* Release the handle, its stream (if owned) and all device memory it holds. */
int bt_destroy(bt_handle *h);

/* Last error message of the handle ("" if none); valid until the next call. */
const char *bt_last_error(const bt_handle *h);

/*
 * Butterfly support of every edge (Defs. 2-3; counted by priority-obeyed
 * wedges as in Alg. 3, with Lemmas 2-3).
 *   support_out: uint64[m], caller-allocated (host, or device with
 *   BT_DEVICE_PTRS).
 * Errors: BT_ERR_ARG, BT_ERR_RANGE, BT_ERR_DUP, BT_ERR_NOMEM, BT_ERR_CUDA.
 * m == 0 returns BT_OK.
 */
int bt_count_support(bt_handle *h, const int32_t *edges, uint64_t m, uint32_t nU, uint32_t nL,
                     uint64_t *support_out, uint32_t flags);

/*
 * Build the BE-Index (Section IV, Alg. 3) and keep it resident on the device
 * inside the handle (replacing any earlier index).  stats_out may be NULL.
 * Errors: as bt_count_support, plus BT_ERR_OVERFLOW when the index has
 * 2^32 or more twin pairs.
 */
int bt_build_index(bt_handle *h, const int32_t *edges, uint64_t m, uint32_t nU, uint32_t nL,
                   bt_index_stats *stats_out, uint32_t flags);

/*
 * Copy the resident index to host memory for inspection.  Any of the output
 * pointers may be NULL to skip it; sizes come from bt_index_stats.
 *   blooms_out:   bt_bloom_rec[n_blooms]  (blooms in index order)
 *   pairs_out:    uint32[2 * n_bloom_wedges]: twin pair i is the edge ids
 *                 (pairs_out[2i], pairs_out[2i+1]) = ((u,v), (v,w)) of one
 *                 priority-obeyed wedge (u,v,w) of its bloom; the two edges
 *                 are each other's twin (Def. 9).  Pairs of one bloom are
 *                 contiguous, starting at first_pair.
 *   edge_deg_out: uint32[m]: number of links of each edge, |N_I(e)|.
 * Errors: BT_ERR_STATE (no index), BT_ERR_CUDA.
 */
int bt_index_export(bt_handle *h, bt_bloom_rec *blooms_out, uint32_t *pairs_out,
                    uint32_t *edge_deg_out);

/*
 * One part of a counting shard over start vertices (Section IV-B: every
 * priority-obeyed wedge is enumerated from its start vertex, the vertex of
 * highest priority, and by Lemma 3 every butterfly lies in exactly one bloom,
 * the one started at its vertex of highest priority).  The vertices are
 * ranked by priority (Def. 7) and cut into nparts contiguous rank ranges
 * holding about equal numbers of priority-obeyed wedges; this call counts
 * part `part`: support_out receives, per edge, the butterflies anchored at a
 * vertex of that range.  The parts of one graph add up to bt_count_support's
 * result, so processes that each count one part and sum the arrays (one
 * reduction) obtain the supports.
 *   part, nparts:   0 <= part < nparts.
 *   support_out:    uint64[m] (host, or device with BT_DEVICE_PTRS), input order.
 *   rank_lo_out, rank_hi_out: nullable; the rank range [lo, hi) counted
 *                   (rank 0 is the lowest priority).
 * Errors: as bt_count_support, plus BT_ERR_ARG for part >= nparts.
 */
int bt_count_support_part(bt_handle *h, const int32_t *edges, uint64_t m, uint32_t nU, uint32_t nL,
                          uint32_t part, uint32_t nparts, uint64_t *support_out, uint32_t *rank_lo_out,
                          uint32_t *rank_hi_out, uint32_t flags);

/*
 * Bitruss number of every edge (Defs. 4-5): counting, BE-Index build, then
 * level-synchronous batch peeling (Alg. 5; every unassigned edge with
 * support <= k is peeled in one batch, k = max(k, minimum support)).
 *   support_out: uint64[m] or NULL -- the initial supports.
 *   phi_out:     uint32[m].
 *   stats:       may be NULL.
 * Errors: as bt_build_index, plus BT_ERR_OVERFLOW (phi > 2^32-1),
 * BT_ERR_NOCONVERGE (round limit, by default m + 1 rounds; see bt_set_limits)
 * and BT_ERR_CUDA (also when a grid-barrier wait of the peel kernel ran out).
 */
int bt_decompose(bt_handle *h, const int32_t *edges, uint64_t m, uint32_t nU, uint32_t nL,
                 uint64_t *support_out, uint32_t *phi_out, bt_peel_stats *stats, uint32_t flags);

/*
 * Turn per-phase event timing on (on != 0) or off for later calls on h.
 * Timing adds one event record per phase boundary and a final wait.
 * Errors: BT_ERR_ARG, BT_ERR_CUDA.
 */
int bt_profile_enable(bt_handle *h, int on);

/* Profile of the last bt_count_support / bt_build_index / bt_decompose call
 * on h (zeros for phases it did not run, and times only when profiling was
 * enabled).  Errors: BT_ERR_ARG. */
int bt_profile_read(const bt_handle *h, bt_profile *out);

/*
 * Limits of the device peel loop and host-side fault injection, for
 * diagnostics and for tests of the failure paths.  The paper has no
 * counterpart (its algorithms are sequential CPU code without failure modes).
 * Every field left 0 keeps the default; the settings apply to later calls on
 * h until changed.  None of them faults, traps or hangs the GPU: each makes a
 * bounded device wait give up, or a host step fail, and the call returns an
 * error with the handle still usable.
 *   peel_round_limit:   stop peeling after this many rounds and return
 *                       BT_ERR_NOCONVERGE (default: m + 1 rounds, capped at
 *                       2^30 - 4, more than any decomposition needs).
 *   barrier_timeout_ns: longest wait of one block of the persistent peel
 *                       kernel at a grid barrier; when it runs out the kernel
 *                       raises its error word, every block returns, and the
 *                       call returns BT_ERR_CUDA (default 20 s).
 *   hold_barrier:       n > 0: block 0 of the peel kernel does not arrive at
 *                       its n-th grid barrier (counted from 1), so that wait
 *                       runs out in every block (use with a short
 *                       barrier_timeout_ns).
 *   fail_alloc_at:      n > 0: inside each call, device allocation number n
 *                       (counted from 1) fails as if the device were out of
 *                       memory; the call returns BT_ERR_NOMEM.
 *   join_cap:           n > 0: a peel block lists at most n (instead of its
 *                       thread count: 640, or 512 with 128-entry items)
 *                       of the edges that join the next batch during its
 *                       bloom phase; the others queue their own links.
 *   block_links:        n > 0: a peel block's kill stage handles at most n
 *                       (instead of two a thread) links itself; longer lists become
 *                       incidence items.  (These two change no result; they
 *                       make small graphs take the paths large ones take.)
 * limits == NULL restores every default.  Errors: BT_ERR_ARG (h NULL).
 */
typedef struct {
    uint64_t peel_round_limit;
    uint64_t barrier_timeout_ns;
    uint64_t hold_barrier;
    uint64_t fail_alloc_at;
    uint32_t join_cap;
    uint32_t block_links;
} bt_limits;
int bt_set_limits(bt_handle *h, const bt_limits *limits);

/*
 * Allocation-free variant of bt_count_support.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory
 * around a library call -- hosts that own all GPU memory through their own
 * pool and accounting (often under a hard cap), and latency-critical loops
 * that must not trigger the device-wide synchronisation cudaMalloc/cudaFree
 * may cause.  It runs the same CSR-build and wedge-count kernels, taking all
 * scratch from one fixed 48 MiB device array inside the library; it calls no
 * cudaMalloc, cudaFree or allocating library routine.
 *   d_edges:        device pointer, int32 pairs as for bt_count_support.
 *   d_support_out:  device pointer, uint64[m].
 *   flags:          0 or BT_TIE_LOWER_FIRST (pointers are always device).
 *   cuda_stream:    cudaStream_t to run on (NULL = legacy default stream);
 *                   the call synchronises it before returning.
 * Capacity: m <= 262,144 edges and nU + nL <= 131,072 vertices; larger
 * graphs return BT_ERR_TOO_LARGE.  Runs on the current CUDA device.  The
 * array lives in every GPU that loads the library until the process exits;
 * the first call on a device looks up its address and keeps it for the
 * process (make that first call before any stream capture); after a
 * cudaDeviceReset of that device the kept address is stale, so the entry
 * point must not be used again in that process.  All calls share the array and it keeps the last call's
 * contents (the call clears what must start at zero); calls whose GPU work
 * overlaps race on it and must be ordered by the caller.
 * Errors: BT_ERR_ARG, BT_ERR_RANGE, BT_ERR_DUP, BT_ERR_TOO_LARGE, BT_ERR_CUDA
 * (no handle, so no message).  m == 0 returns BT_OK.
 */
int bt_count_support_static(const int32_t *d_edges, uint64_t m, uint32_t nU, uint32_t nL,
                            uint64_t *d_support_out, uint32_t flags, void *cuda_stream);

/* One graph of a batch (bt_decompose_batch).  Pointers are host pointers,
 * or device pointers when the batch call passes BT_DEVICE_PTRS. */
typedef struct {
    const int32_t *edges;   /* int32 pairs (u, v), 2*m values, as for bt_decompose */
    uint64_t m;
    uint32_t nU, nL;
    uint64_t *support_out;  /* uint64[m] or NULL */
    uint32_t *phi_out;      /* uint32[m] */
} bt_graph;

/* Batch schedule.  Zero fields are chosen by the library: the autotuner
 * times candidate schedules on a sample of the batch (about 8M edges of its
 * graphs) and caches the winner in the handle per batch signature (log4 of
 * the total edges and of the largest graph). */
typedef struct {
    uint64_t max_edges_per_launch;  /* graphs are packed into unions of at most this many edges */
    uint32_t count_threads;         /* wedge-count / index block size: 256, 512 or 1024 */
    uint32_t peel_item;             /* peel work item: 32, 64 or 128 links / pair slots per warp */
    uint32_t reserved[2];
} bt_tune;

typedef struct {
    uint64_t graphs;           /* graphs decomposed */
    uint64_t launches;         /* union graphs (device pipelines) used */
    uint64_t edges;            /* total edges */
    uint64_t wedges;           /* total priority-obeyed wedges */
    uint64_t rounds, levels;   /* peeling rounds and levels, summed over unions */
    uint64_t support_updates;
    uint32_t count_threads;    /* schedule used */
    uint32_t peel_item;
    uint32_t tuned;            /* 1 if this call ran the autotuner, 2 if it used a cached choice */
    uint32_t reserved;
} bt_batch_stats;

/*
 * Bitruss decomposition of n independent graphs.  Butterflies never span two
 * graphs, so the decomposition of their disjoint union is the union of their
 * decompositions (Defs. 4-5): the graphs are relabelled on the device into
 * one union (upper and lower ids shifted per graph, keeping every graph's own
 * priority order, Def. 7) and decomposed by one pipeline -- one count, one
 * index emit and one persistent peeling launch -- so the peel's rounds are
 * shared by all graphs instead of paid per graph.  Results are exactly those
 * of bt_decompose on each graph alone.  Graphs are packed into unions of at
 * most tune->max_edges_per_launch edges (0: as many as device memory allows;
 * a union that does not fit is split in two and retried).
 * stats may be NULL; tune may be NULL.
 * Errors: as bt_decompose; BT_ERR_RANGE names the first graph with a bad id.
 */
int bt_decompose_batch(bt_handle *h, const bt_graph *graphs, uint32_t n, const bt_tune *tune,
                       bt_batch_stats *stats, uint32_t flags);

/* Statistics of a progressive-compression decomposition. */
typedef struct {
    uint64_t passes;           /* candidate subgraphs peeled (eps values with unassigned edges) */
    uint64_t rounds, levels;   /* peeling rounds and levels, summed over passes */
    uint64_t support_updates;  /* support decrements applied, summed over passes */
    uint64_t candidate_edges;  /* edges of the candidate subgraphs, summed */
    uint64_t wedges;           /* priority-obeyed wedges of the candidate subgraphs, summed */
    uint64_t k_max;            /* largest k with >= k edges of support >= k */
    uint64_t alpha;            /* eps step, ceil(k_max * tau) */
    uint64_t index_bytes_max;  /* largest compressed BE-Index of a pass (bytes, as bt_index_stats) */
    uint64_t links;            /* edge-bloom links stored, summed over passes (assigned edges get none) */
    uint64_t dropped_edges;    /* with BT_PC_RECOUNT: candidates whose support recounted on
                                  G_{>=eps} fell below eps, summed over passes */
} bt_pc_stats;

/*
 * Bitruss numbers by progressive compression (BiT-PC, Section V-C, Alg. 7):
 * after counting, eps runs from k_max down to 0 in steps of
 * alpha = ceil(k_max * tau).  For each eps the candidate subgraph G_{>=eps}
 * (edges of support >= eps, which holds every k-bitruss with k >= eps,
 * Lemma 10) gets a compressed BE-Index (Alg. 6: blooms keep all their twin
 * pairs, edges already assigned get no links and receive no updates) and is
 * peeled in batches; edges leaving at a level >= eps are assigned, the others
 * wait for a smaller eps.  Two readings of the extraction step:
 *   default        every edge below eps is taken in one batch level eps - 1
 *                  of the pass's peel, so a pass spends one level on them;
 *   BT_PC_RECOUNT  as Alg. 7 writes it: the supports are recounted on
 *                  G_{>=eps}, candidates whose recounted support is below
 *                  eps are dropped before the compressed index is built, and
 *                  the pass peels from the candidates' minimum support.
 * Both give the results of bt_decompose (Thm. 3); they differ in the support
 * updates and index sizes they report (Figs. 10-11).
 *   tau in (0, 1] (the paper uses 0.02 by default and suggests 0.05-0.2).
 *   flags: BT_DEVICE_PTRS, BT_TIE_LOWER_FIRST, BT_PC_RECOUNT.
 *   support_out may be NULL; stats may be NULL.
 * Errors: as bt_decompose, plus BT_ERR_ARG for tau outside (0, 1].
 */
int bt_decompose_progressive(bt_handle *h, const int32_t *edges, uint64_t m, uint32_t nU, uint32_t nL,
                             double tau, uint64_t *support_out, uint32_t *phi_out, bt_pc_stats *stats,
                             uint32_t flags);

/* ---------------------------------------------------------------- hierarchy
 * The k-bitruss H_k (Def. 4, Section II) is the maximal subgraph in which every
 * edge lies in at least k butterflies of that subgraph; the bitruss number
 * phi(e) is the largest k with e in H_k (Def. 5).  The k-bitrusses are nested,
 * so H_k = {e : phi(e) >= k}: given the phi of bt_decompose (same edge order),
 * these calls return the hierarchy that the applications of Section I
 * consume (nested groups, communities at several levels).
 */

/*
 * Order the edges by bitruss number, largest first, edges of equal phi in
 * ascending input index.  Every k-bitruss is then a prefix: H_k is
 * order_out[0 .. n_k), n_k = number of edges with phi >= k.
 *   phi            -- u32[m] bitruss numbers, indexed like the input edges
 *   order_out      -- u32[m] edge indices (caller-allocated)
 *   phi_sorted_out -- u32[m] or NULL: phi of order_out[i] (non-increasing),
 *                     for finding n_k by binary search
 * flags: BT_DEVICE_PTRS only (phi, order_out and phi_sorted_out are then
 * device pointers).  m must be below 2^32.  Errors: BT_ERR_ARG (NULL pointer,
 * unknown flag, m too large), BT_ERR_NOMEM, BT_ERR_CUDA.
 */
int bt_hierarchy(bt_handle *h, const uint32_t *phi, uint64_t m, uint32_t *order_out,
                 uint32_t *phi_sorted_out, uint32_t flags);

/*
 * The edges of one k-bitruss H_k: the indices of the edges with phi >= k, in
 * ascending order, written to edges_out[0 .. *count_out) (edges_out has room
 * for m entries; count_out is always a host pointer).  H_0 is every edge.
 * flags, limits and errors as bt_hierarchy.
 */
int bt_k_bitruss(bt_handle *h, const uint32_t *phi, uint64_t m, uint32_t k, uint32_t *edges_out,
                 uint64_t *count_out, uint32_t flags);

/* ---------------------------------------------------------------- serving
 * A request loop with continuous batching.  Each submitted request is one
 * graph (host pointers, as in bt_graph; the caller keeps edges and outputs
 * alive until the request completes).  Worker threads, each owning a handle
 * (stream, memory pool, device-resident BE-Index), take all waiting requests
 * that fit the memory budget whenever they become free and decompose them as
 * one batch (bt_decompose_batch); requests that arrive meanwhile join the next
 * batch, and with several workers batches overlap on the device.  Admission
 * uses an O(m) upper bound on a request's device bytes from its degrees
 * (priority-obeyed wedges <= sum over edges of min(d(u), d(v)), Lemma 6).
 * Large requests (config large_edges) are never batched with small ones
 * (several waiting large ones may share a batch, config large_batch), and
 * with several workers one of them serves the small requests first (passing
 * waiting large ones), so a large graph does not hold back the small requests
 * that arrive behind it; the other workers take the oldest large request
 * first.  Each worker falls back to the other kind when its own has none
 * waiting (the small-first worker only when two or more large requests
 * wait), so neither kind starves; within a kind, first come, first served.
 * Results are exactly those of bt_decompose on the graph alone. */
typedef struct bt_server bt_server;

typedef struct {
    uint64_t memory_budget_bytes;  /* admission budget; 0 = 120 GiB */
    uint32_t workers;              /* concurrent batches; 0 = 2 */
    uint32_t max_batch_graphs;     /* 0 = unlimited; 1 = one request at a time (plain serial) */
    uint32_t flags;                /* 0 or BT_TIE_LOWER_FIRST */
    uint32_t large_edges;          /* a request with at least this many edges runs in a batch of its
                                      own; with several workers the last one serves small requests
                                      first and the others large ones first; 0 = 2^20,
                                      UINT32_MAX = no request counts as large */
    uint32_t large_batch;          /* up to this many waiting large requests share one batch
                                      (their peels then share rounds); 0 = 2, 1 = each alone */
} bt_server_config;

typedef struct {
    int done;                /* 1 when the request completed */
    int status;              /* its bt_status once done */
    double queue_seconds;    /* submit -> batch start (so far, if not started) */
    double latency_seconds;  /* submit -> completion (so far, if not done) */
    uint64_t admitted_bytes; /* the admission bound used */
} bt_request_info;

typedef struct {
    uint64_t submitted, completed, rejected, batches, queued;
    uint64_t max_batch_graphs;
    uint64_t in_flight_bytes, peak_in_flight_bytes;
    uint64_t edges;
    double busy_seconds;     /* summed over workers */
} bt_server_stats;

/* Start a server on `device`.  cfg may be NULL (defaults).
 * Errors: BT_ERR_ARG, BT_ERR_NOMEM, BT_ERR_CUDA. */
int bt_server_create(bt_server **s, int device, const bt_server_config *cfg);
/* Finish every queued request, then stop the workers and free the server. */
int bt_server_destroy(bt_server *s);
/* Complete every request still waiting in the queue (not yet in a batch)
 * with status BT_ERR_CANCELLED; batches already on the GPU finish normally.
 * *cancelled_out (nullable) receives how many were cancelled.  Used to end a
 * measurement window on an overloaded server.  Errors: BT_ERR_ARG. */
int bt_server_cancel_queued(bt_server *s, uint64_t *cancelled_out);
/* Queue one graph; returns its id.  Errors: BT_ERR_ARG, BT_ERR_NOMEM. */
int bt_server_submit(bt_server *s, const bt_graph *g, uint64_t *request_id);
/* State of a request (wait != 0 blocks until it completes).  Once a done
 * request has been reported its id is released.  Errors: BT_ERR_ARG,
 * BT_ERR_STATE (unknown or released id). */
int bt_server_poll(bt_server *s, uint64_t request_id, int wait, bt_request_info *info);
int bt_server_stats_read(bt_server *s, bt_server_stats *out);

/*
 * Device bytes a bt_decompose of this graph needs (host computation, O(m)
 * time; edges are host pointers).  It counts priority-obeyed wedges exactly,
 * so the estimate for the BE-Index is an upper bound (every wedge assumed to
 * lie in a bloom).
 * Errors: BT_ERR_ARG, BT_ERR_RANGE.
 */
int bt_estimate_bytes(const int32_t *edges, uint64_t m, uint32_t nU, uint32_t nL, uint32_t flags,
                      uint64_t *bytes_out, uint64_t *wedges_out);

#ifdef __cplusplus
}
#endif
#endif /* BITRUSS_H */
