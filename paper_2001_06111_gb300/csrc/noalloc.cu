// Allocation-free butterfly support count (bt_count_support_static).
//
// Some callers cannot allocate device memory around a library call: hosts
// that own every byte of the GPU through their own pool (and account for it
// themselves, often under a hard cap), and latency-critical loops that must
// not trigger the device-wide synchronisation cudaMalloc/cudaFree may cause.
// This entry point runs the same CSR build and wedge-count kernels as
// bt_count_support, but every scratch buffer comes from one fixed device
// array declared below instead of from an allocator.  The caller passes only
// device inputs and outputs.
//
// The array is a file-scope __device__ variable, so every GPU that loads the
// library holds it (kStaticBytes) until the process exits.  Host code cannot
// use the symbol itself as a device address: on the first call on each
// device (with that device current) the address is fetched once with
// cudaGetSymbolAddress and cached.  That first call should therefore come
// before any stream capture.  The cached address belongs to the device's
// primary context: after a cudaDeviceReset of that device it is stale, and
// the entry point must not be called again in that process.  Every call
// synchronises the caller's stream twice (input validation and the end of
// the count).  All calls share the array and it keeps the
// contents of the last call; everything that must start at zero is cleared
// by the call itself.  Two calls whose GPU work overlaps (different streams,
// or different host threads) race on the array and give wrong results: the
// caller must order them.
#include <mutex>

#include "bt_internal.cuh"

namespace {

constexpr size_t kStaticBytes = 48ull << 20;   // 48 MiB per device
constexpr uint64_t kMaxEdges = 1ull << 18;      // 262,144 edges
constexpr uint64_t kMaxVertices = 1ull << 17;   // nU + nL <= 131,072
constexpr int kStaticSms = 8;                   // count kernel: 8 x (blocks per SM) blocks
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

std::mutex g_mu;
unsigned char *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set-up once).
cudaError_t scratch_address(int device, unsigned char **out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[device] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_ptr[device];
    return cudaSuccess;
}

}  // namespace

extern "C" int bt_count_support_static(const int32_t *d_edges, uint64_t m, uint32_t nU, uint32_t nL,
                                       uint64_t *d_support_out, uint32_t flags, void *cuda_stream) {
    if (flags & ~(uint32_t)BT_TIE_LOWER_FIRST) return BT_ERR_ARG;
    if (m == 0) return BT_OK;
    if (!d_edges || !d_support_out) return BT_ERR_ARG;
    if (m > kMaxEdges || (uint64_t)nU + nL > kMaxVertices) return BT_ERR_TOO_LARGE;
    if (m > (uint64_t)nU * nL) return BT_ERR_DUP;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices)
        return BT_ERR_CUDA;
    unsigned char *scratch = nullptr;
    if (scratch_address(device, &scratch) != cudaSuccess) return BT_ERR_CUDA;
    int num_sms = 0;
    if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return BT_ERR_CUDA;

    bt::Alloc al;
    al.stream = static_cast<cudaStream_t>(cuda_stream);
    al.pool = nullptr;
    al.arena = scratch;
    al.arena_size = kStaticBytes;
    uint32_t *err_word = al.get<uint32_t>(1);
    if (!err_word) return BT_ERR_TOO_LARGE;
    cudaError_t e = cudaMemsetAsync(err_word, 0, sizeof(uint32_t), al.stream);
    bt::Csr g;
    if (e == cudaSuccess) e = bt::build_csr(d_edges, m, nU, nL, flags, g, err_word, al);
    if (e == cudaErrorMemoryAllocation) return BT_ERR_TOO_LARGE;
    if (e != cudaSuccess) return BT_ERR_CUDA;
    uint32_t hw = 0;
    e = cudaMemcpyAsync(&hw, err_word, sizeof(uint32_t), cudaMemcpyDeviceToHost, al.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(al.stream);
    if (e != cudaSuccess) return BT_ERR_CUDA;
    if (hw & bt::kErrRange) return BT_ERR_RANGE;
    if (hw & bt::kErrDup) return BT_ERR_DUP;
    bt::CountOut co;
    co.support = al.get<uint64_t>(m);  // internal edge order, gathered below
    if (!co.support) return BT_ERR_TOO_LARGE;
    e = bt::count_wedges(g, co, kStaticSms < num_sms ? kStaticSms : num_sms, al);
    if (e == cudaErrorMemoryAllocation) return BT_ERR_TOO_LARGE;
    if (e == cudaSuccess) e = bt::gather_u64(co.support, g.newid, d_support_out, m, al);
    if (e == cudaSuccess) e = cudaStreamSynchronize(al.stream);
    return e == cudaSuccess ? BT_OK : BT_ERR_CUDA;
}
