// C ABI of libbitruss (declared in include/bitruss.h): argument checks,
// host/device staging, the handle's stream and memory pool, and the call
// sequences CSR build -> wedge count -> BE-Index emit -> batch peel.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "bt_internal.cuh"

struct bt_handle {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaMemPool_t pool = nullptr;
    int num_sms = 0;
    uint32_t *err_word = nullptr;  // device
    bt::Index index;
    bool has_index = false;
    std::string err;
    bt::Prof prof;
    bt_profile last{};
    int count_nt = 1024;  // schedule used by the next pipeline run (1024: fewest per-block counter arrays)
    int peel_seg = 32;
    int peel_sms = 0;     // SMs the peel kernel spans (0: all); a server worker takes its share
    const bt::GraphSplit *split = nullptr;  // graphs of the batch union being prepared, if any
    std::map<uint64_t, std::pair<int, int>> tuned;  // batch signature -> (count_nt, peel_seg)
    unsigned char *pinned = nullptr;  // page-locked staging for batch copies
    size_t pinned_bytes = 0;
    bt_limits limits{};  // bt_set_limits (all zero: defaults)
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int d) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != d) cudaSetDevice(d);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int fail(bt_handle *h, int code, const char *fmt, ...) {
    if (h) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        h->err = buf;
    }
    return code;
}

int cuda_fail(bt_handle *h, cudaError_t e, const char *where) {
    if (e == cudaErrorMemoryAllocation)
        return fail(h, BT_ERR_NOMEM, "%s: device allocation failed (%s)", where, cudaGetErrorString(e));
    return fail(h, BT_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

int peel_sms(const bt_handle *h) { return h->peel_sms > 0 ? h->peel_sms : h->num_sms; }

bt::Alloc make_alloc(bt_handle *h) {
    bt::Alloc al;
    al.stream = h->stream;
    al.pool = h->pool;
    al.prof = &h->prof;
    al.limits = &h->limits;
    return al;
}

// Starts a profiled call: clears the last profile and marks the call start.
void call_begin(bt_handle *h, bt::Alloc &al, uint64_t m, uint32_t n) {
    h->last = bt_profile{};
    h->last.n_edges = m;
    h->last.n_vertices = n;
    for (bool &u : h->prof.used) u = false;
    al.mark(bt::kPhTotal, false);
}

// Ends a profiled call: reads back the phase times.
void call_end(bt_handle *h, bt::Alloc &al) {
    al.mark(bt::kPhTotal, true);
    h->last.launches = al.launches;
    if (!h->prof.on) return;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return;
    float *dst[bt::kNumPhases] = {&h->last.csr_ms, &h->last.count_ms, &h->last.emit_ms,
                                  &h->last.peel_ms, &h->last.total_ms};
    for (int p = 0; p < bt::kNumPhases; ++p) {
        float ms = 0.f;
        if (h->prof.used[p] &&
            cudaEventElapsedTime(&ms, h->prof.ev[2 * p], h->prof.ev[2 * p + 1]) != cudaSuccess)
            ms = 0.f;
        *dst[p] = h->prof.used[p] ? ms : 0.f;
    }
}

int check_args(bt_handle *h, const int32_t *edges, uint64_t m, uint32_t nU, uint32_t nL,
               uint32_t flags) {
    if (!h) return BT_ERR_ARG;
    if (flags & ~(BT_DEVICE_PTRS | BT_TIE_LOWER_FIRST))
        return fail(h, BT_ERR_ARG, "unknown flag bits 0x%x", flags);
    if (m > 0 && !edges) return fail(h, BT_ERR_ARG, "edges is NULL");
    if ((uint64_t)nU + nL >= 0xFFFFFFFFull)
        return fail(h, BT_ERR_ARG, "nU + nL = %llu exceeds 2^32 - 2",
                    (unsigned long long)nU + nL);
    if (m >= (1ull << 31)) return fail(h, BT_ERR_ARG, "m = %llu exceeds 2^31 - 1", (unsigned long long)m);
    if (m > (uint64_t)nU * nL) return fail(h, BT_ERR_DUP, "m exceeds nU * nL: edges cannot be distinct");
    return BT_OK;
}

// Stages the edge list on the device and builds the rank-ordered CSR.
struct Prepared {
    const int32_t *d_edges = nullptr;
    int32_t *owned = nullptr;
    bt::Csr g;
};

int prepare(bt_handle *h, const int32_t *edges, uint64_t m, uint32_t nU, uint32_t nL,
            uint32_t flags, Prepared &P, bt::Alloc &al) {
    if (flags & BT_DEVICE_PTRS) {
        P.d_edges = edges;
    } else {
        P.owned = al.get<int32_t>(2 * m);
        if (!P.owned) return cuda_fail(h, al.err, "staging edges");
        cudaError_t e = cudaMemcpyAsync(P.owned, edges, sizeof(int32_t) * 2 * m,
                                        cudaMemcpyHostToDevice, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "copying edges to the device");
        P.d_edges = P.owned;
    }
    cudaError_t e = cudaMemsetAsync(h->err_word, 0, sizeof(uint32_t), h->stream);
    if (e == cudaSuccess) e = bt::build_csr(P.d_edges, m, nU, nL, flags, P.g, h->err_word, al, h->split);
    if (e != cudaSuccess) return cuda_fail(h, e, "building the CSR");
    uint32_t hw = 0;
    e = cudaMemcpyAsync(&hw, h->err_word, sizeof(uint32_t), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "building the CSR");
    if (hw & bt::kErrRange) return fail(h, BT_ERR_RANGE, "a vertex id is outside [0,nU) x [0,nL)");
    if (hw & bt::kErrDup) return fail(h, BT_ERR_DUP, "duplicate edge in the input");
    return BT_OK;
}

void release(Prepared &P, bt::Alloc &al) {
    bt::free_csr(P.g, al);
    al.put(P.owned);
    P.owned = nullptr;
}

// Copies a device result of `bytes` to the caller's buffer (host or device).
cudaError_t deliver(bt_handle *h, void *dst, const void *src, size_t bytes, uint32_t flags) {
    if (dst == src || bytes == 0) return cudaSuccess;
    return cudaMemcpyAsync(dst, src, bytes,
                           (flags & BT_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                           h->stream);
}

// Count (+ optional index).  d_support receives supports (device) indexed by
// internal edge id (P.g.newid maps input ids to them; with an index, the map
// moves to ix.newid).
int count_and_index(bt_handle *h, Prepared &P, uint64_t *d_support, bool want_index,
                    bt::Index &ix, uint64_t &butterflies, bt::Alloc &al,
                    const uint8_t *assigned = nullptr) {
    bt::CountOut co;
    co.support = d_support;
    co.assigned = assigned;
    uint64_t W = 0;
    if (want_index) {
        co.inc_cnt = al.get<uint32_t>(P.g.m);
        co.w2v = al.get<uint64_t>(P.g.n);
        co.nbv = al.get<uint64_t>(P.g.n);
        if (al.err != cudaSuccess) return cuda_fail(h, al.err, "allocating count buffers");
    }
    cudaError_t e = bt::count_wedges(P.g, co, h->num_sms, al, h->count_nt);
    if (e != cudaSuccess) return cuda_fail(h, e, "counting wedges");
    unsigned long long bf = 0;
    e = cudaMemcpyAsync(&bf, co.butterflies_dev, sizeof(bf), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    al.put(co.butterflies_dev);
    if (e != cudaSuccess) return cuda_fail(h, e, "counting wedges");
    butterflies = bf;
    if (want_index) {
        // W for the statistics: sum of wedges per start vertex
        uint64_t *tot = al.get<uint64_t>(1);
        uint64_t *scratch = al.get<uint64_t>(P.g.n);
        if (al.err != cudaSuccess) return cuda_fail(h, al.err, "allocating");
        e = bt::exclusive_scan_u64(P.g.wv, scratch, P.g.n, tot, al);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&W, tot, sizeof(W), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        al.put(tot);
        al.put(scratch);
        if (e != cudaSuccess) return cuda_fail(h, e, "summing wedges");
        e = bt::emit_index(P.g, co, ix, h->num_sms, al, h->stream, h->count_nt);
        al.put(co.inc_cnt);
        al.put(co.w2v);
        al.put(co.nbv);
        if (e == cudaErrorInvalidValue)
            return fail(h, BT_ERR_OVERFLOW, "BE-Index has >= 2^32 twin pairs or blooms");
        if (e != cudaSuccess) return cuda_fail(h, e, "emitting the BE-Index");
        ix.w = W;
        ix.butterflies = bf;
        ix.newid = P.g.newid;  // the index speaks internal edge ids
        P.g.newid = nullptr;
    }
    return BT_OK;
}

}  // namespace

extern "C" {

int bt_create(bt_handle **out, int device, void *cuda_stream) {
    if (!out) return BT_ERR_ARG;
    *out = nullptr;
    bt_handle *h = new (std::nothrow) bt_handle();
    if (!h) return BT_ERR_NOMEM;
    h->device = device;
    DeviceGuard dg(device);
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) {
        if (cuda_stream) {
            h->stream = static_cast<cudaStream_t>(cuda_stream);
        } else {
            e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
            h->own_stream = true;
        }
    }
    if (e == cudaSuccess) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        e = cudaMemPoolCreate(&h->pool, &props);
    }
    if (e == cudaSuccess) {
        uint64_t thr = ~0ull;  // keep freed blocks cached for the next call
        e = cudaMemPoolSetAttribute(h->pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    if (e == cudaSuccess) e = cudaMalloc(&h->err_word, sizeof(uint32_t));
    if (e != cudaSuccess) {
        if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
        if (h->pool) cudaMemPoolDestroy(h->pool);
        delete h;
        return e == cudaErrorMemoryAllocation ? BT_ERR_NOMEM : BT_ERR_CUDA;
    }
    *out = h;
    return BT_OK;
}

int bt_destroy(bt_handle *h) {
    if (!h) return BT_ERR_ARG;
    DeviceGuard dg(h->device);
    if (h->has_index) {
        bt::Alloc al = make_alloc(h);
        bt::free_index(h->index, al);
    }
    cudaStreamSynchronize(h->stream);
    for (auto &ev : h->prof.ev)
        if (ev) cudaEventDestroy(ev);
    cudaFree(h->err_word);
    if (h->pinned) cudaFreeHost(h->pinned);
    if (h->pool) cudaMemPoolDestroy(h->pool);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return BT_OK;
}

const char *bt_last_error(const bt_handle *h) { return h ? h->err.c_str() : "null handle"; }

int bt_count_support(bt_handle *h, const int32_t *edges, uint64_t m, uint32_t nU, uint32_t nL,
                     uint64_t *support_out, uint32_t flags) {
    int rc = check_args(h, edges, m, nU, nL, flags);
    if (rc) return rc;
    h->err.clear();
    if (m == 0) return BT_OK;
    if (!support_out) return fail(h, BT_ERR_ARG, "support_out is NULL");
    DeviceGuard dg(h->device);
    bt::Alloc al = make_alloc(h);
    call_begin(h, al, m, nU + nL);
    Prepared P;
    rc = prepare(h, edges, m, nU, nL, flags, P, al);
    uint64_t *d_sup = nullptr, *d_int = nullptr;
    if (rc == BT_OK) {
        d_int = al.get<uint64_t>(m);
        d_sup = (flags & BT_DEVICE_PTRS) ? support_out : al.get<uint64_t>(m);
        if (al.err != cudaSuccess) rc = cuda_fail(h, al.err, "allocating supports");
    }
    bt::Index unused;
    uint64_t bf = 0;
    if (rc == BT_OK) rc = count_and_index(h, P, d_int, false, unused, bf, al);
    if (rc == BT_OK) {
        cudaError_t e = bt::gather_u64(d_int, P.g.newid, d_sup, m, al);  // back to input order
        if (e == cudaSuccess) e = deliver(h, support_out, d_sup, sizeof(uint64_t) * m, flags);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) rc = cuda_fail(h, e, "returning supports");
    }
    al.put(d_int);
    if (!(flags & BT_DEVICE_PTRS)) al.put(d_sup);
    release(P, al);
    call_end(h, al);
    cudaStreamSynchronize(h->stream);
    return rc;
}

int bt_count_support_part(bt_handle *h, const int32_t *edges, uint64_t m, uint32_t nU, uint32_t nL,
                          uint32_t part, uint32_t nparts, uint64_t *support_out, uint32_t *rank_lo_out,
                          uint32_t *rank_hi_out, uint32_t flags) {
    int rc = check_args(h, edges, m, nU, nL, flags);
    if (rc) return rc;
    h->err.clear();
    if (nparts == 0 || part >= nparts) return fail(h, BT_ERR_ARG, "part %u of %u parts", part, nparts);
    if (rank_lo_out) *rank_lo_out = 0;
    if (rank_hi_out) *rank_hi_out = 0;
    if (m == 0) return BT_OK;
    if (!support_out) return fail(h, BT_ERR_ARG, "support_out is NULL");
    DeviceGuard dg(h->device);
    bt::Alloc al = make_alloc(h);
    call_begin(h, al, m, nU + nL);
    Prepared P;
    rc = prepare(h, edges, m, nU, nL, flags, P, al);
    uint64_t *d_sup = nullptr, *d_int = nullptr, *pre = nullptr, *tot = nullptr;
    uint32_t *bounds = nullptr;
    if (rc == BT_OK) {
        d_int = al.get<uint64_t>(m);
        d_sup = (flags & BT_DEVICE_PTRS) ? support_out : al.get<uint64_t>(m);
        pre = al.get<uint64_t>(P.g.n);
        tot = al.get<uint64_t>(1);
        bounds = al.get<uint32_t>(2);
        if (al.err != cudaSuccess) rc = cuda_fail(h, al.err, "allocating supports");
    }
    uint32_t hb[2] = {0, 0};
    if (rc == BT_OK) {
        // W-balanced contiguous rank ranges: part p starts at the first rank
        // whose preceding start vertices hold at least p W / nparts wedges
        uint64_t W = 0;
        cudaError_t e = bt::exclusive_scan_u64(P.g.wv, pre, P.g.n, tot, al);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&W, tot, sizeof(W), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        const uint64_t t0 = (uint64_t)((unsigned __int128)W * part / nparts);
        const uint64_t t1 = (uint64_t)((unsigned __int128)W * (part + 1) / nparts);
        if (e == cudaSuccess) e = bt::rank_bounds(pre, P.g.n, t0, t1, bounds, al);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hb, bounds, sizeof(hb), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) rc = cuda_fail(h, e, "splitting the start vertices");
        if (part == 0) hb[0] = 0;
        if (part + 1 == nparts) hb[1] = P.g.n;
    }
    if (rc == BT_OK) {
        bt::CountOut co;
        co.support = d_int;
        cudaError_t e = bt::count_wedges(P.g, co, h->num_sms, al, h->count_nt, hb[0], hb[1]);
        if (e == cudaSuccess) {
            al.put(co.butterflies_dev);
            e = bt::gather_u64(d_int, P.g.newid, d_sup, m, al);  // back to input order
        }
        if (e == cudaSuccess) e = deliver(h, support_out, d_sup, sizeof(uint64_t) * m, flags);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) rc = cuda_fail(h, e, "counting a part");
    }
    if (rc == BT_OK) {
        if (rank_lo_out) *rank_lo_out = hb[0];
        if (rank_hi_out) *rank_hi_out = hb[1];
    }
    al.put(d_int);
    if (!(flags & BT_DEVICE_PTRS)) al.put(d_sup);
    al.put(pre);
    al.put(tot);
    al.put(bounds);
    release(P, al);
    call_end(h, al);
    cudaStreamSynchronize(h->stream);
    return rc;
}

// Stages a u32[m] array on the device (or uses it in place with BT_DEVICE_PTRS).
static int stage_u32(bt_handle *h, const uint32_t *src, uint64_t m, uint32_t flags, bt::Alloc &al,
                     const uint32_t **d_out, uint32_t **owned) {
    *owned = nullptr;
    if (flags & BT_DEVICE_PTRS) {
        *d_out = src;
        return BT_OK;
    }
    *owned = al.get<uint32_t>(m);
    if (!*owned) return cuda_fail(h, al.err, "staging phi");
    cudaError_t e = cudaMemcpyAsync(*owned, src, sizeof(uint32_t) * m, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "copying phi to the device");
    *d_out = *owned;
    return BT_OK;
}

static int check_phi_args(bt_handle *h, const uint32_t *phi, uint64_t m, const void *out, uint32_t flags) {
    if (!h) return BT_ERR_ARG;
    if (flags & ~(uint32_t)BT_DEVICE_PTRS) return fail(h, BT_ERR_ARG, "unknown flag bits 0x%x", flags);
    if (m >= (1ull << 32)) return fail(h, BT_ERR_ARG, "m = %llu exceeds 2^32 - 1", (unsigned long long)m);
    if (m > 0 && (!phi || !out)) return fail(h, BT_ERR_ARG, "phi or the output is NULL");
    return BT_OK;
}

extern "C" int bt_hierarchy(bt_handle *h, const uint32_t *phi, uint64_t m, uint32_t *order_out,
                            uint32_t *phi_sorted_out, uint32_t flags) {
    int rc = check_phi_args(h, phi, m, order_out, flags);
    if (rc) return rc;
    h->err.clear();
    if (m == 0) return BT_OK;
    DeviceGuard dg(h->device);
    bt::Alloc al = make_alloc(h);
    const bool dev = flags & BT_DEVICE_PTRS;
    const uint32_t *d_phi = nullptr;
    uint32_t *owned = nullptr;
    rc = stage_u32(h, phi, m, flags, al, &d_phi, &owned);
    uint32_t *d_order = nullptr, *d_ps = nullptr;
    if (rc == BT_OK) {
        d_order = dev ? order_out : al.get<uint32_t>(m);
        if (phi_sorted_out) d_ps = dev ? phi_sorted_out : al.get<uint32_t>(m);
        if (al.err != cudaSuccess) rc = cuda_fail(h, al.err, "allocating the order");
    }
    if (rc == BT_OK) {
        cudaError_t e = bt::hierarchy_order(d_phi, m, d_order, d_ps, al);
        if (e == cudaSuccess) e = deliver(h, order_out, d_order, sizeof(uint32_t) * m, flags);
        if (e == cudaSuccess && phi_sorted_out)
            e = deliver(h, phi_sorted_out, d_ps, sizeof(uint32_t) * m, flags);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) rc = cuda_fail(h, e, "ordering the edges by phi");
    }
    if (!dev) {
        al.put(d_order);
        al.put(d_ps);
    }
    al.put(owned);
    h->last = bt_profile{};
    h->last.n_edges = m;
    h->last.launches = al.launches;
    cudaStreamSynchronize(h->stream);
    return rc;
}

extern "C" int bt_k_bitruss(bt_handle *h, const uint32_t *phi, uint64_t m, uint32_t k, uint32_t *edges_out,
                            uint64_t *count_out, uint32_t flags) {
    int rc = check_phi_args(h, phi, m, edges_out, flags);
    if (rc) return rc;
    if (!count_out) return fail(h, BT_ERR_ARG, "count_out is NULL");
    h->err.clear();
    *count_out = 0;
    if (m == 0) return BT_OK;
    DeviceGuard dg(h->device);
    bt::Alloc al = make_alloc(h);
    const bool dev = flags & BT_DEVICE_PTRS;
    const uint32_t *d_phi = nullptr;
    uint32_t *owned = nullptr;
    rc = stage_u32(h, phi, m, flags, al, &d_phi, &owned);
    uint32_t *d_out = nullptr;
    if (rc == BT_OK) {
        d_out = dev ? edges_out : al.get<uint32_t>(m);
        if (al.err != cudaSuccess) rc = cuda_fail(h, al.err, "allocating the edge list");
    }
    if (rc == BT_OK) {
        uint32_t n = 0;
        cudaError_t e = bt::select_ge(d_phi, m, k, d_out, h->err_word, al);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&n, h->err_word, sizeof(uint32_t), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e == cudaSuccess && !dev && n)
            e = cudaMemcpyAsync(edges_out, d_out, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) rc = cuda_fail(h, e, "selecting the k-bitruss");
        else *count_out = n;
    }
    if (!dev) al.put(d_out);
    al.put(owned);
    h->last = bt_profile{};
    h->last.n_edges = m;
    h->last.launches = al.launches;
    cudaStreamSynchronize(h->stream);
    return rc;
}

static int build_index_impl(bt_handle *h, const int32_t *edges, uint64_t m, uint32_t nU,
                            uint32_t nL, uint32_t flags, uint64_t *d_sup, bt::Alloc &al) {
    Prepared P;
    int rc = prepare(h, edges, m, nU, nL, flags, P, al);
    if (h->has_index) {
        bt::free_index(h->index, al);
        h->has_index = false;
    }
    bt::Index ix;
    uint64_t bf = 0;
    if (rc == BT_OK) rc = count_and_index(h, P, d_sup, true, ix, bf, al);
    release(P, al);
    if (rc == BT_OK) {
        h->index = ix;
        h->has_index = true;
    } else {
        bt::free_index(ix, al);
    }
    return rc;
}

int bt_build_index(bt_handle *h, const int32_t *edges, uint64_t m, uint32_t nU, uint32_t nL,
                   bt_index_stats *stats_out, uint32_t flags) {
    int rc = check_args(h, edges, m, nU, nL, flags);
    if (rc) return rc;
    h->err.clear();
    DeviceGuard dg(h->device);
    bt::Alloc al = make_alloc(h);
    call_begin(h, al, m, nU + nL);
    uint64_t *d_sup = al.get<uint64_t>(m);
    if (!d_sup) return cuda_fail(h, al.err, "allocating supports");
    if (m == 0) {
        if (h->has_index) bt::free_index(h->index, al);
        h->index = bt::Index{};
        h->has_index = true;
        rc = BT_OK;
    } else {
        rc = build_index_impl(h, edges, m, nU, nL, flags, d_sup, al);
    }
    al.put(d_sup);
    call_end(h, al);
    if (rc == BT_OK) {
        h->last.n_wedges = h->index.w;
        h->last.n_bloom_wedges = h->index.w2;
        h->last.n_blooms = h->index.nb;
    }
    cudaStreamSynchronize(h->stream);
    if (rc == BT_OK && stats_out) {
        stats_out->n_wedges = h->index.w;
        stats_out->n_bloom_wedges = h->index.w2;
        stats_out->n_blooms = h->index.nb;
        stats_out->n_butterflies = h->index.butterflies;
        stats_out->index_bytes = h->index.bytes();
    }
    return rc;
}

int bt_index_export(bt_handle *h, bt_bloom_rec *blooms_out, uint32_t *pairs_out,
                    uint32_t *edge_deg_out) {
    if (!h) return BT_ERR_ARG;
    if (!h->has_index) return fail(h, BT_ERR_STATE, "no BE-Index has been built on this handle");
    DeviceGuard dg(h->device);
    const bt::Index &ix = h->index;
    cudaError_t e = cudaSuccess;
    if (blooms_out && ix.nb) {
        std::vector<uint32_t> k(ix.nb), off(ix.nb);
        e = cudaMemcpyAsync(k.data(), ix.bloom_k, 4 * ix.nb, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(off.data(), ix.bloom_off, 4 * ix.nb, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e == cudaSuccess)
            for (uint64_t i = 0; i < ix.nb; ++i) blooms_out[i] = bt_bloom_rec{k[i], off[i]};
    }
    // the index holds internal edge ids: map them back to input ids
    std::vector<uint32_t> newid(ix.m), orig(ix.m);
    if (e == cudaSuccess && ix.m && (pairs_out || edge_deg_out)) {
        e = cudaMemcpyAsync(newid.data(), ix.newid, 4 * ix.m, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        for (uint64_t i = 0; i < ix.m; ++i) orig[newid[i]] = (uint32_t)i;
    }
    if (e == cudaSuccess && pairs_out && ix.w2) {
        e = cudaMemcpyAsync(pairs_out, ix.pairs, 8 * ix.w2, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e == cudaSuccess)
            for (uint64_t i = 0; i < 2 * ix.w2; ++i) pairs_out[i] = orig[pairs_out[i] & 0x7FFFFFFFu];
    }
    if (e == cudaSuccess && edge_deg_out && ix.m) {
        std::vector<uint64_t> off(ix.m + 1);
        e = cudaMemcpyAsync(off.data(), ix.inc_off, 8 * (ix.m + 1), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e == cudaSuccess)
            for (uint64_t i = 0; i < ix.m; ++i)
                edge_deg_out[i] = (uint32_t)(off[newid[i] + 1] - off[newid[i]]);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "exporting the index");
    return BT_OK;
}

int bt_decompose(bt_handle *h, const int32_t *edges, uint64_t m, uint32_t nU, uint32_t nL,
                 uint64_t *support_out, uint32_t *phi_out, bt_peel_stats *stats, uint32_t flags) {
    int rc = check_args(h, edges, m, nU, nL, flags);
    if (rc) return rc;
    h->err.clear();
    if (stats) memset(stats, 0, sizeof(*stats));
    if (m == 0) return BT_OK;
    if (!phi_out) return fail(h, BT_ERR_ARG, "phi_out is NULL");
    DeviceGuard dg(h->device);
    bt::Alloc al = make_alloc(h);
    call_begin(h, al, m, nU + nL);
    const bool dev = flags & BT_DEVICE_PTRS;
    uint64_t *d_sup = (dev && support_out) ? support_out : al.get<uint64_t>(m);
    uint32_t *d_phi = dev ? phi_out : al.get<uint32_t>(m);
    uint64_t *s_int = al.get<uint64_t>(m);  // internal edge order
    uint32_t *p_int = al.get<uint32_t>(m);
    if (al.err != cudaSuccess) return cuda_fail(h, al.err, "allocating outputs");
    rc = build_index_impl(h, edges, m, nU, nL, flags, s_int, al);
    bt::PeelResult pr;
    if (rc == BT_OK) {
        // larger work items pay off when rounds are heavy: on the 30M-edge
        // planted graph (3.1e9 twin pairs) the peel took 18.1 s with 128
        // pair slots an item (four a lane, 512-thread blocks), 18.6 s with 64
        // and 21.9 s with 32; on graphs with up to 2e8 pairs 32 measured
        // 3-8 % faster than 64
        const int seg = h->index.w2 > (1ull << 30) ? 128 : h->peel_seg;
        cudaError_t e = bt::peel(h->index, s_int, p_int, pr, peel_sms(h), al, seg);
        if (e == cudaSuccess) e = bt::gather_u64(s_int, h->index.newid, d_sup, m, al);
        if (e == cudaSuccess) e = bt::gather_u32(p_int, h->index.newid, d_phi, m, al);
        if (e != cudaSuccess) rc = cuda_fail(h, e, "peeling");
        else if (pr.status == BT_ERR_OVERFLOW)
            rc = fail(h, BT_ERR_OVERFLOW, "a bitruss number exceeds 2^32 - 1");
        else if (pr.status == BT_ERR_CUDA)
            rc = fail(h, BT_ERR_CUDA, "peeling stopped: a grid-barrier wait of the peel kernel ran out");
        else if (pr.status != BT_OK)
            rc = fail(h, pr.status, "peeling did not converge within its round limit");
    }
    if (rc == BT_OK) {
        cudaError_t e = cudaSuccess;
        if (support_out) e = deliver(h, support_out, d_sup, sizeof(uint64_t) * m, flags);
        if (e == cudaSuccess) e = deliver(h, phi_out, d_phi, sizeof(uint32_t) * m, flags);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) rc = cuda_fail(h, e, "returning results");
    }
    if (stats && rc == BT_OK) {
        stats->rounds = pr.rounds;
        stats->levels = pr.levels;
        stats->support_updates = pr.updates;
        stats->phi_max = (uint32_t)pr.kmax;
    }
    if (!(dev && support_out)) al.put(d_sup);
    if (!dev) al.put(d_phi);
    al.put(s_int);
    al.put(p_int);
    call_end(h, al);
    if (rc == BT_OK) {
        h->last.n_wedges = h->index.w;
        h->last.n_bloom_wedges = h->index.w2;
        h->last.n_blooms = h->index.nb;
        h->last.rounds = pr.rounds;
        h->last.levels = pr.levels;
        h->last.support_updates = pr.updates;
        h->last.pair_slots = pr.slots;
        h->last.scanned = pr.scanned;
        h->last.link_visits = h->index.links;
    }
    cudaStreamSynchronize(h->stream);
    return rc;
}

int bt_set_limits(bt_handle *h, const bt_limits *limits) {
    if (!h) return BT_ERR_ARG;
    h->limits = limits ? *limits : bt_limits{};
    return BT_OK;
}

int bt_profile_enable(bt_handle *h, int on) {
    if (!h) return BT_ERR_ARG;
    DeviceGuard dg(h->device);
    if (on && !h->prof.ev[0]) {
        for (auto &ev : h->prof.ev) {
            cudaError_t e = cudaEventCreate(&ev);
            if (e != cudaSuccess) return cuda_fail(h, e, "creating profiling events");
        }
    }
    h->prof.on = on != 0;
    return BT_OK;
}

int bt_profile_read(const bt_handle *h, bt_profile *out) {
    if (!h || !out) return BT_ERR_ARG;
    *out = h->last;
    return BT_OK;
}

// Page-locked staging buffer of at least `bytes` (grown on demand), or null.
static unsigned char *pinned_buffer(bt_handle *h, size_t bytes) {
    if (h->pinned_bytes >= bytes) return h->pinned;
    if (h->pinned) cudaFreeHost(h->pinned);
    h->pinned = nullptr;
    h->pinned_bytes = 0;
    void *p = nullptr;
    if (cudaMallocHost(&p, bytes) != cudaSuccess) return nullptr;
    h->pinned = static_cast<unsigned char *>(p);
    h->pinned_bytes = bytes;
    return h->pinned;
}

// Runs fn(g) for g in [0, n) on up to 8 host threads.
extern "C++" {
template <typename F>
static void parallel_for(uint32_t n, uint64_t total_bytes, F fn) {
    unsigned nt = total_bytes > (64ull << 20) ? std::min(8u, std::max(1u, std::thread::hardware_concurrency())) : 1u;
    if (nt <= 1 || n < 2) {
        for (uint32_t g = 0; g < n; ++g) fn(g);
        return;
    }
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t)
        th.emplace_back([&, t] {
            for (uint32_t g = t; g < n; g += nt) fn(g);
        });
    for (auto &x : th) x.join();
}
}  // extern "C++"

// Decomposes graphs[0..n) as one disjoint union (see bt_decompose_batch).
static int decompose_union(bt_handle *h, const bt_graph *graphs, uint32_t n, uint32_t flags,
                           bt_batch_stats *acc, bt::Alloc &al) {
    const bool dev = flags & BT_DEVICE_PTRS;
    std::vector<uint64_t> goff(n + 1, 0);
    std::vector<uint32_t> offU(n), offL(n), gnU(n), gnL(n);
    uint64_t NU = 0, NL = 0;
    for (uint32_t g = 0; g < n; ++g) {
        goff[g + 1] = goff[g] + graphs[g].m;
        offU[g] = (uint32_t)NU;
        offL[g] = (uint32_t)NL;
        gnU[g] = graphs[g].nU;
        gnL[g] = graphs[g].nL;
        NU += graphs[g].nU;
        NL += graphs[g].nL;
    }
    const uint64_t M = goff[n];
    if (NU + NL >= 0xFFFFFFFFull || M >= (1ull << 31))
        return fail(h, BT_ERR_ARG, "union of %u graphs exceeds 2^31 edges or 2^32 vertices", n);
    al.err = cudaSuccess;
    int rc = BT_OK;
    int32_t *d_edges = al.get<int32_t>(2 * M);
    uint64_t *d_goff = al.get<uint64_t>(n + 1);
    uint32_t *d_tab = al.get<uint32_t>(4 * (size_t)n + 1);
    uint64_t *d_sup = al.get<uint64_t>(M);
    uint32_t *d_phi = al.get<uint32_t>(M);
    if (al.err != cudaSuccess) rc = cuda_fail(h, al.err, "allocating the batch union");
    cudaError_t e = cudaSuccess;
    if (rc == BT_OK) {
        std::vector<uint32_t> tab(4 * (size_t)n + 1);
        std::copy(offU.begin(), offU.end(), tab.begin());
        std::copy(offL.begin(), offL.end(), tab.begin() + n);
        std::copy(gnU.begin(), gnU.end(), tab.begin() + 2 * (size_t)n);
        std::copy(gnL.begin(), gnL.end(), tab.begin() + 3 * (size_t)n);
        tab[4 * (size_t)n] = 0xFFFFFFFFu;  // lowest failing graph
        e = cudaMemcpyAsync(d_goff, goff.data(), 8 * (n + 1), cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_tab, tab.data(), 4 * tab.size(), cudaMemcpyHostToDevice, h->stream);
        unsigned char *stage = dev ? nullptr : pinned_buffer(h, 12 * M + 16);
        if (stage) {
            // gather all host edge lists into page-locked memory, one DMA
            parallel_for(n, 8 * M, [&](uint32_t g) {
                if (graphs[g].m) memcpy(stage + 8 * goff[g], graphs[g].edges, 8 * graphs[g].m);
            });
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(d_edges, stage, 8 * M, cudaMemcpyHostToDevice, h->stream);
        } else {
            for (uint32_t g = 0; g < n && e == cudaSuccess; ++g)
                if (graphs[g].m)
                    e = cudaMemcpyAsync(d_edges + 2 * goff[g], graphs[g].edges, 8 * graphs[g].m,
                                        dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream);
        }
        if (e == cudaSuccess) e = cudaMemsetAsync(h->err_word, 0, sizeof(uint32_t), h->stream);
        uint32_t *bad = d_tab + 4 * (size_t)n;
        if (e == cudaSuccess)
            e = bt::union_edges(d_edges, M, d_goff, n, d_tab, d_tab + n, d_tab + 2 * (size_t)n,
                                d_tab + 3 * (size_t)n, h->err_word, bad, al);
        uint32_t hw[2] = {0, 0};
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&hw[0], h->err_word, 4, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hw[1], bad, 4, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) rc = cuda_fail(h, e, "staging the batch");
        else if (hw[0] & bt::kErrRange)
            rc = fail(h, BT_ERR_RANGE, "graph %u of the batch has a vertex id outside its layers", hw[1]);
    }
    if (rc == BT_OK && M > 0) {
        // rank the union graph by graph: the counting kernels then size their
        // per-block counters by the largest graph instead of the union
        bt::GraphSplit split;
        split.ng = n;
        split.offU = d_tab;
        split.offL = d_tab + n;
        for (uint32_t g = 0; g < n; ++g) split.max_n = std::max(split.max_n, gnU[g] + gnL[g]);
        h->split = &split;
        rc = build_index_impl(h, d_edges, M, (uint32_t)NU, (uint32_t)NL,
                              (flags & BT_TIE_LOWER_FIRST) | BT_DEVICE_PTRS, d_sup, al);
        h->split = nullptr;
    }
    bt::PeelResult pr;
    if (rc == BT_OK && M > 0) {
        e = bt::peel(h->index, d_sup, d_phi, pr, peel_sms(h), al, h->peel_seg);
        // results back to input order (the edge array is free by now: reuse it)
        uint64_t *g_sup = reinterpret_cast<uint64_t *>(d_edges);
        uint32_t *g_phi = al.get<uint32_t>(M);
        if (e == cudaSuccess && !g_phi) e = al.err;
        if (e == cudaSuccess) e = bt::gather_u64(d_sup, h->index.newid, g_sup, M, al);
        if (e == cudaSuccess) e = bt::gather_u32(d_phi, h->index.newid, g_phi, M, al);
        if (e == cudaSuccess) {
            d_edges = reinterpret_cast<int32_t *>(d_sup);  // freed below under its old name
            d_sup = g_sup;
            al.put(d_phi);
            d_phi = g_phi;
        } else {
            al.put(g_phi);
        }
        if (e != cudaSuccess) rc = cuda_fail(h, e, "peeling");
        else if (pr.status == BT_ERR_OVERFLOW)
            rc = fail(h, BT_ERR_OVERFLOW, "a bitruss number exceeds 2^32 - 1");
        else if (pr.status != BT_OK)
            rc = fail(h, pr.status, "peeling stopped: device barrier timeout or round limit");
    }
    if (rc == BT_OK) {
        unsigned char *stage = (dev || M == 0) ? nullptr : pinned_buffer(h, 12 * M + 16);
        if (stage) {
            // one DMA of all results into page-locked memory, then scatter
            e = cudaMemcpyAsync(stage, d_sup, 8 * M, cudaMemcpyDeviceToHost, h->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(stage + 8 * M, d_phi, 4 * M, cudaMemcpyDeviceToHost, h->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
            if (e == cudaSuccess)
                parallel_for(n, 12 * M, [&](uint32_t g) {
                    if (!graphs[g].m) return;
                    if (graphs[g].support_out)
                        memcpy(graphs[g].support_out, stage + 8 * goff[g], 8 * graphs[g].m);
                    memcpy(graphs[g].phi_out, stage + 8 * M + 4 * goff[g], 4 * graphs[g].m);
                });
        } else {
            for (uint32_t g = 0; g < n && e == cudaSuccess; ++g) {
                if (!graphs[g].m) continue;
                if (graphs[g].support_out)
                    e = deliver(h, graphs[g].support_out, d_sup + goff[g], 8 * graphs[g].m, flags);
                if (e == cudaSuccess)
                    e = deliver(h, graphs[g].phi_out, d_phi + goff[g], 4 * graphs[g].m, flags);
            }
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) rc = cuda_fail(h, e, "returning batch results");
    }
    if (rc == BT_OK && acc) {
        acc->graphs += n;
        acc->launches += 1;
        acc->edges += M;
        acc->wedges += h->index.w;
        acc->rounds += pr.rounds;
        acc->levels += pr.levels;
        acc->support_updates += pr.updates;
    }
    al.put(d_edges);
    al.put(d_goff);
    al.put(d_tab);
    al.put(d_sup);
    al.put(d_phi);
    cudaStreamSynchronize(h->stream);
    return rc;
}

// Packs graphs into unions of at most `cap` edges; a union that runs out of
// device memory is split in two and retried.
static int decompose_packed(bt_handle *h, const bt_graph *graphs, uint32_t n, uint64_t cap,
                            uint32_t flags, bt_batch_stats *acc, bt::Alloc &al) {
    uint32_t g0 = 0;
    while (g0 < n) {
        uint32_t g1 = g0;
        uint64_t edges = 0, verts = 0;
        while (g1 < n && (g1 == g0 || (edges + graphs[g1].m <= cap &&
                                      verts + graphs[g1].nU + graphs[g1].nL < 0xF0000000ull))) {
            edges += graphs[g1].m;
            verts += (uint64_t)graphs[g1].nU + graphs[g1].nL;
            ++g1;
        }
        int rc = decompose_union(h, graphs + g0, g1 - g0, flags, acc, al);
        if (rc == BT_ERR_NOMEM && g1 - g0 > 1) {
            uint32_t half = (g1 - g0) / 2;
            rc = decompose_packed(h, graphs + g0, half, cap, flags, acc, al);
            if (rc == BT_OK)
                rc = decompose_packed(h, graphs + g0 + half, g1 - g0 - half, cap, flags, acc, al);
        }
        if (rc != BT_OK) return rc;
        g0 = g1;
    }
    return BT_OK;
}

// Elapsed ms between the profiler events of a phase (0 if not recorded).
static float phase_ms(bt_handle *h, int phase) {
    float ms = 0.f;
    if (!h->prof.used[phase] ||
        cudaEventElapsedTime(&ms, h->prof.ev[2 * phase], h->prof.ev[2 * phase + 1]) != cudaSuccess)
        return 0.f;
    return ms;
}

// Picks the count block size and the peel item size for this batch: looks up
// the handle's cache by signature, else times three candidate schedules on a
// sample of the graphs (writing the sample graphs' outputs, which the real
// run overwrites with the same values) and caches the fastest parts.
static int autotune(bt_handle *h, const bt_graph *graphs, uint32_t n, uint32_t flags, bt::Alloc &al,
                    uint32_t *tuned) {
    uint64_t total = 0, mx = 0;
    for (uint32_t g = 0; g < n; ++g) {
        total += graphs[g].m;
        mx = std::max<uint64_t>(mx, graphs[g].m);
    }
    // coarse buckets (powers of 4) so that similar batches share a choice
    const uint64_t sig = ((uint64_t)(bt::bits_for(total) / 2) << 8) | (uint64_t)(bt::bits_for(mx) / 2);
    auto it = h->tuned.find(sig);
    if (it != h->tuned.end()) {
        h->count_nt = it->second.first;
        h->peel_seg = it->second.second;
        *tuned = 2;
        return BT_OK;
    }
    if (total == 0) return BT_OK;
    // sample: every stride-th graph, about 8M edges
    const uint64_t target = 8ull << 20;
    const uint32_t stride = (uint32_t)std::max<uint64_t>(1, (total + target - 1) / target);
    std::vector<bt_graph> sample;
    for (uint32_t g = 0; g < n; g += stride) sample.push_back(graphs[g]);
    const bool prof_was_on = h->prof.on;
    if (!h->prof.ev[0]) {
        for (auto &ev : h->prof.ev)
            if (cudaEventCreate(&ev) != cudaSuccess) return cuda_fail(h, cudaErrorUnknown, "creating events");
    }
    h->prof.on = true;
    const int cand[3][2] = {{512, 32}, {256, 64}, {1024, 32}};
    float t_build[3] = {0, 0, 0}, t_peel[3] = {0, 0, 0};
    int rc = BT_OK;
    for (int c = 0; c < 3 && rc == BT_OK; ++c) {
        h->count_nt = cand[c][0];
        h->peel_seg = cand[c][1];
        for (bool &u : h->prof.used) u = false;
        rc = decompose_union(h, sample.data(), (uint32_t)sample.size(), flags, nullptr, al);
        t_build[c] = phase_ms(h, bt::kPhCount) + phase_ms(h, bt::kPhEmit);
        t_peel[c] = phase_ms(h, bt::kPhPeel);
    }
    h->prof.on = prof_was_on;
    if (rc != BT_OK) return rc;
    int best = 0;
    for (int c = 1; c < 3; ++c)
        if (t_build[c] < t_build[best]) best = c;
    const float peel32 = 0.5f * (t_peel[0] + t_peel[2]);
    h->count_nt = cand[best][0];
    h->peel_seg = t_peel[1] < peel32 ? 64 : 32;
    h->tuned[sig] = {h->count_nt, h->peel_seg};
    *tuned = 1;
    return BT_OK;
}

int bt_decompose_batch(bt_handle *h, const bt_graph *graphs, uint32_t n, const bt_tune *tune,
                       bt_batch_stats *stats, uint32_t flags) {
    if (!h) return BT_ERR_ARG;
    h->err.clear();
    if (stats) memset(stats, 0, sizeof(*stats));
    if (flags & ~(BT_DEVICE_PTRS | BT_TIE_LOWER_FIRST))
        return fail(h, BT_ERR_ARG, "unknown flag bits 0x%x", flags);
    if (n && !graphs) return fail(h, BT_ERR_ARG, "graphs is NULL");
    for (uint32_t g = 0; g < n; ++g) {
        const bt_graph &G = graphs[g];
        if (G.m && (!G.edges || !G.phi_out)) return fail(h, BT_ERR_ARG, "graph %u: NULL edges or phi_out", g);
        if (G.m >= (1ull << 31)) return fail(h, BT_ERR_ARG, "graph %u: m exceeds 2^31 - 1", g);
        if (G.m > (uint64_t)G.nU * G.nL)
            return fail(h, BT_ERR_DUP, "graph %u: m exceeds nU * nL", g);
    }
    uint64_t cap = (tune && tune->max_edges_per_launch) ? tune->max_edges_per_launch : (1ull << 31) - 1;
    DeviceGuard dg(h->device);
    bt::Alloc al = make_alloc(h);
    call_begin(h, al, 0, 0);
    bt_batch_stats acc{};
    const int saved_nt = h->count_nt, saved_seg = h->peel_seg;
    uint32_t tuned = 0;
    int rc = BT_OK;
    if (tune && tune->count_threads && tune->peel_item) {
        h->count_nt = tune->count_threads;
        h->peel_seg = tune->peel_item;
    } else {
        rc = autotune(h, graphs, n, flags, al, &tuned);
        if (tune && tune->count_threads) h->count_nt = tune->count_threads;
        if (tune && tune->peel_item) h->peel_seg = tune->peel_item;
    }
    if (rc == BT_OK) rc = decompose_packed(h, graphs, n, cap, flags, &acc, al);
    acc.count_threads = (uint32_t)h->count_nt;
    acc.peel_item = (uint32_t)h->peel_seg;
    acc.tuned = tuned;
    h->count_nt = saved_nt;
    h->peel_seg = saved_seg;
    call_end(h, al);
    if (rc == BT_OK) {
        h->last.n_edges = acc.edges;
        h->last.n_wedges = acc.wedges;
        h->last.rounds = acc.rounds;
        h->last.levels = acc.levels;
        h->last.support_updates = acc.support_updates;
    }
    if (stats && rc == BT_OK) *stats = acc;
    return rc;
}

int bt_decompose_progressive(bt_handle *h, const int32_t *edges, uint64_t m, uint32_t nU, uint32_t nL,
                             double tau, uint64_t *support_out, uint32_t *phi_out, bt_pc_stats *stats,
                             uint32_t flags) {
    const bool recount = flags & BT_PC_RECOUNT;
    flags &= ~(uint32_t)BT_PC_RECOUNT;
    int rc = check_args(h, edges, m, nU, nL, flags);
    if (rc) return rc;
    h->err.clear();
    if (stats) memset(stats, 0, sizeof(*stats));
    if (!(tau > 0.0 && tau <= 1.0)) return fail(h, BT_ERR_ARG, "tau must be in (0, 1]");
    if (m == 0) return BT_OK;
    if (!phi_out) return fail(h, BT_ERR_ARG, "phi_out is NULL");
    DeviceGuard dg(h->device);
    bt::Alloc al = make_alloc(h);
    call_begin(h, al, m, nU + nL);
    const bool dev = flags & BT_DEVICE_PTRS;
    bt_pc_stats st{};
    Prepared P;
    rc = prepare(h, edges, m, nU, nL, flags, P, al);
    uint64_t *d_sup0 = (dev && support_out) ? support_out : al.get<uint64_t>(m);
    uint32_t *d_phi = dev ? phi_out : al.get<uint32_t>(m);
    uint8_t *d_asg = al.get<uint8_t>(m);
    int32_t *cand = al.get<int32_t>(2 * m);
    uint32_t *cmap = al.get<uint32_t>(m);
    uint8_t *cass = al.get<uint8_t>(m);
    uint32_t *phi_local = al.get<uint32_t>(m);
    uint64_t *sup_c = al.get<uint64_t>(m);
    uint32_t *hist = al.get<uint32_t>(m + 1);
    unsigned long long *counts = al.get<unsigned long long>(2);
    uint8_t *cass_int = al.get<uint8_t>(m);   // candidate flags in internal edge order
    uint32_t *phi_c = al.get<uint32_t>(m);    // candidate phi in candidate input order
    // Alg. 7's extraction: supports recounted on the candidates, and the
    // candidates kept (edges, map to candidate index, map to global id, flags)
    uint64_t *sup_r = nullptr;
    int32_t *cand2 = nullptr;
    uint32_t *cmap2 = nullptr, *cmapg2 = nullptr;
    uint8_t *cass2 = nullptr;
    if (recount) {
        sup_r = al.get<uint64_t>(m);
        cand2 = al.get<int32_t>(2 * m);
        cmap2 = al.get<uint32_t>(m);
        cmapg2 = al.get<uint32_t>(m);
        cass2 = al.get<uint8_t>(m);
    }
    if (rc == BT_OK && al.err != cudaSuccess) rc = cuda_fail(h, al.err, "allocating");
    uint64_t bf = 0;
    bt::Index unused;
    // supports of G (the counting process of Alg. 7)
    if (rc == BT_OK) rc = count_and_index(h, P, sup_c, false, unused, bf, al);
    if (rc == BT_OK) {
        cudaError_t eg = bt::gather_u64(sup_c, P.g.newid, d_sup0, m, al);  // input order
        if (eg != cudaSuccess) rc = cuda_fail(h, eg, "counting");
    }
    bt::free_csr(P.g, al);
    // k_max: the largest k with at least k edges of support >= k (Section V-C)
    uint64_t kmax = 0;
    cudaError_t e = cudaSuccess;
    if (rc == BT_OK) {
        std::vector<uint32_t> hh(m + 1);
        e = bt::support_hist(d_sup0, m, hist, al);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hh.data(), hist, 4 * (m + 1), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_asg, 0, m, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) rc = cuda_fail(h, e, "computing k_max");
        uint64_t acc = 0;
        for (uint64_t k = m + 1; k-- > 0;) {
            acc += hh[k];
            if (acc >= k) {
                kmax = k;
                break;
            }
        }
    }
    const uint64_t alpha = std::max<uint64_t>(1, (uint64_t)std::ceil((double)kmax * tau));
    st.k_max = kmax;
    st.alpha = alpha;
    uint64_t eps = kmax;
    while (rc == BT_OK) {
        // candidate subgraph G_{>=eps} (Alg. 7, extraction step)
        unsigned long long hc[2] = {0, 0};
        e = bt::select_candidates(P.d_edges, d_sup0, m, eps, d_asg, cand, cmap, cass, counts, al);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hc, counts, sizeof(hc), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) {
            rc = cuda_fail(h, e, "extracting a candidate subgraph");
            break;
        }
        // the candidate graph the pass indexes and peels
        const int32_t *pc_edges = cand;
        const uint32_t *pc_map = cmap;
        const uint8_t *pc_ass = cass;
        uint64_t pc_n = hc[0];
        if (hc[1] > 0 && recount) {
            // Alg. 7, extraction: recount the supports on G_{>=eps} and drop
            // the candidates below eps (an assigned edge never is: its
            // phi-bitruss lies inside G_{>=eps}, so it keeps >= phi butterflies)
            Prepared R;
            rc = prepare(h, cand, hc[0], nU, nL, (flags & BT_TIE_LOWER_FIRST) | BT_DEVICE_PTRS, R, al);
            if (rc == BT_OK) rc = count_and_index(h, R, sup_c, false, unused, bf, al);
            if (rc == BT_OK) {
                unsigned long long h2[2] = {0, 0};
                e = bt::gather_u64(sup_c, R.g.newid, sup_r, hc[0], al);  // candidate order
                if (e == cudaSuccess)
                    e = bt::select_candidates(cand, sup_r, hc[0], eps, cass, cand2, cmap2, cass2, counts, al);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(h2, counts, sizeof(h2), cudaMemcpyDeviceToHost, h->stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
                // global ids of the kept candidates (only the h2[0] entries written)
                if (e == cudaSuccess && h2[0]) e = bt::gather_u32(cmap, cmap2, cmapg2, h2[0], al);
                if (e != cudaSuccess) rc = cuda_fail(h, e, "recounting a candidate subgraph");
                st.dropped_edges += hc[0] - h2[0];
                pc_edges = cand2;
                pc_map = cmapg2;
                pc_ass = cass2;
                pc_n = h2[0];
                hc[1] = h2[1];
            }
            bt::free_csr(R.g, al);
            if (rc != BT_OK) break;
        }
        if (hc[1] > 0) {
            // compressed BE-Index of the candidate graph (Alg. 6), then a batch
            // peel that settles every edge leaving at a level >= eps
            Prepared Q;
            rc = prepare(h, pc_edges, pc_n, nU, nL, (flags & BT_TIE_LOWER_FIRST) | BT_DEVICE_PTRS, Q, al);
            bt::Index ix;
            if (rc == BT_OK) {
                cudaError_t es = bt::scatter_u8(pc_ass, Q.g.newid, cass_int, pc_n, al);
                if (es != cudaSuccess) rc = cuda_fail(h, es, "extracting a candidate subgraph");
            }
            if (rc == BT_OK) rc = count_and_index(h, Q, sup_c, true, ix, bf, al, cass_int);
            bt::free_csr(Q.g, al);
            bt::PeelResult pr;
            if (rc == BT_OK) {
                bt::PeelOpts o;
                o.assigned = cass_int;
                o.m_active = hc[1];
                // default reading: every edge below eps leaves at level eps - 1;
                // Alg. 7's: the peel starts at the minimum support
                o.k_init = (!recount && eps > 0) ? (long long)eps - 1 : 0;
                o.assign_from = (long long)eps;
                e = cudaMemsetAsync(phi_local, 0xFF, 4 * pc_n, h->stream);
                if (e == cudaSuccess) e = bt::peel(ix, sup_c, phi_local, pr, peel_sms(h), al, h->peel_seg, &o);
                if (e == cudaSuccess) e = bt::gather_u32(phi_local, ix.newid, phi_c, pc_n, al);
                if (e == cudaSuccess) e = bt::settle(pc_map, pc_n, pc_ass, phi_c, d_phi, d_asg, al);
                if (e != cudaSuccess) rc = cuda_fail(h, e, "peeling a candidate subgraph");
                else if (pr.status == BT_ERR_OVERFLOW) rc = fail(h, BT_ERR_OVERFLOW, "a bitruss number exceeds 2^32 - 1");
                else if (pr.status != BT_OK) rc = fail(h, pr.status, "peeling stopped: device barrier timeout or round limit");
            }
            st.wedges += ix.w;
            st.links += ix.links;
            if (ix.bytes() > st.index_bytes_max) st.index_bytes_max = ix.bytes();
            bt::free_index(ix, al);
            st.passes++;
            st.rounds += pr.rounds;
            st.levels += pr.levels;
            st.support_updates += pr.updates;
            st.candidate_edges += pc_n;
        }
        if (eps == 0) break;
        eps = eps > alpha ? eps - alpha : 0;
    }
    if (rc == BT_OK) {
        e = cudaSuccess;
        if (support_out) e = deliver(h, support_out, d_sup0, sizeof(uint64_t) * m, flags);
        if (e == cudaSuccess) e = deliver(h, phi_out, d_phi, sizeof(uint32_t) * m, flags);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) rc = cuda_fail(h, e, "returning results");
    }
    al.put(P.owned);
    if (!(dev && support_out)) al.put(d_sup0);
    if (!dev) al.put(d_phi);
    al.put(d_asg);
    al.put(cand);
    al.put(cmap);
    al.put(cass);
    al.put(phi_local);
    al.put(sup_c);
    al.put(hist);
    al.put(counts);
    al.put(cass_int);
    al.put(phi_c);
    al.put(sup_r);
    al.put(cand2);
    al.put(cmap2);
    al.put(cmapg2);
    al.put(cass2);
    call_end(h, al);
    if (rc == BT_OK) {
        h->last.rounds = st.rounds;
        h->last.levels = st.levels;
        h->last.support_updates = st.support_updates;
        if (stats) *stats = st;
    }
    cudaStreamSynchronize(h->stream);
    return rc;
}

int bt_estimate_bytes(const int32_t *edges, uint64_t m, uint32_t nU, uint32_t nL, uint32_t flags,
                      uint64_t *bytes_out, uint64_t *wedges_out) {
    if (!bytes_out || (m && !edges)) return BT_ERR_ARG;
    if ((uint64_t)nU + nL >= 0xFFFFFFFFull || m >= (1ull << 31)) return BT_ERR_ARG;
    const uint64_t n = (uint64_t)nU + nL;
    std::vector<uint32_t> deg(n, 0);
    auto gid_u = [&](uint32_t u) { return (flags & BT_TIE_LOWER_FIRST) ? u : nL + u; };
    auto gid_v = [&](uint32_t v) { return (flags & BT_TIE_LOWER_FIRST) ? nU + v : v; };
    for (uint64_t i = 0; i < m; ++i) {
        int32_t u = edges[2 * i], v = edges[2 * i + 1];
        if (u < 0 || v < 0 || (uint32_t)u >= nU || (uint32_t)v >= nL) return BT_ERR_RANGE;
        deg[gid_u(u)]++;
        deg[gid_v(v)]++;
    }
    // rank by (degree, id)
    std::vector<uint32_t> order(n), rank(n);
    for (uint64_t i = 0; i < n; ++i) order[i] = (uint32_t)i;
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return deg[a] < deg[b]; });
    for (uint64_t r = 0; r < n; ++r) rank[order[r]] = (uint32_t)r;
    std::vector<uint64_t> off(n + 1, 0);
    for (uint64_t x = 0; x < n; ++x) off[rank[x] + 1] = deg[x];
    for (uint64_t r = 0; r < n; ++r) off[r + 1] += off[r];
    std::vector<uint32_t> adj(2 * m);
    std::vector<uint64_t> fill(off.begin(), off.end() - 1);
    for (uint64_t i = 0; i < m; ++i) {
        uint32_t a = rank[gid_u(edges[2 * i])], b = rank[gid_v(edges[2 * i + 1])];
        adj[fill[a]++] = b;
        adj[fill[b]++] = a;
    }
    for (uint64_t r = 0; r < n; ++r) std::sort(adj.begin() + off[r], adj.begin() + off[r + 1]);
    uint64_t W = 0;
    for (uint64_t u = 0; u < n; ++u)
        for (uint64_t j = off[u]; j < off[u + 1]; ++j) {
            uint32_t v = adj[j];
            if (v >= u) break;
            W += (uint64_t)(std::lower_bound(adj.begin() + off[v], adj.begin() + off[v + 1], (uint32_t)u) -
                            (adj.begin() + off[v]));
        }
    if (wedges_out) *wedges_out = W;
    // CSR + sort scratch + counters (peak), supports/phi/peel state, and an
    // index bound of 16 bytes per wedge plus per-bloom records (<= W/2 blooms)
    uint64_t csr = (n + 1) * 8 + 2 * m * (4 + 4 + 4) + n * 12;
    uint64_t sort_scratch = 2 * m * 24;
    // two u32 counters per vertex for every resident count block (at most
    // SMs x resident threads per SM / 256-thread blocks, read from the
    // current device; a GB300's 152 x 2048 when no device answers)
    uint64_t resident = 152ull * 2048 / 256;
    {
        int dev = 0, sms = 0, tpm = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&tpm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) == cudaSuccess &&
            sms > 0 && tpm > 0)
            resident = (uint64_t)sms * (uint64_t)tpm / 256;
    }
    uint64_t counters = 2ull * 4 * n * resident;
    uint64_t edges_b = m * (8 + 8 + 4 + 4 + 4 + 4 + 8 + 8 + 4);
    uint64_t index_b = W * (8 + 4 + 8 + 1) + (W / 2 + 1) * 16;
    *bytes_out = csr + std::max(sort_scratch, counters) + edges_b + index_b + (1ull << 20);
    return BT_OK;
}

}  // extern "C"

namespace bt {
// Let the handle's peel kernel span 1/ways of the SMs, so that the peels of
// `ways` handles (server workers) can be resident at once; the kernel is
// latency-bound, so half the SMs cost the 2M-edge peel about 6 %.
void share_peel_sms(bt_handle *h, int ways) {
    if (h && ways > 1) h->peel_sms = h->num_sms / ways > 0 ? h->num_sms / ways : 1;
}
}  // namespace bt
