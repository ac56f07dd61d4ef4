// noalloc.cu — dbscan_run_noalloc: clustering without any device allocation.
//
// Some callers cannot call cudaMalloc.  Examples:
//   - a serving process that reserved every device byte for its own pool at
//     start-up and may not grow;
//   - code that must not take the allocator's locks while other work runs;
//   - a host with a fixed memory budget.
// dbscan_run_noalloc serves them.  It runs the all-pairs CUDA-core path (the
// same kernels dbscan_run uses for d > 3), taking its scratch from one
// fixed-size array that is part of this library's device image.  Every GPU
// that loads the library holds that array (about 1.3 MiB) until the process
// exits.
//
// The array's name, used in host code, is a host-side stand-in, not a device
// address.  So the first call on a device (with that device current) asks the
// runtime for the real address with cudaGetSymbolAddress, checks the result
// and caches it for that device, keyed by the id of the current CUDA context:
// if the context changes (cudaDeviceReset, a new primary context), the next
// call looks the address up again.  The first call on a device, and the first
// after such a change, should therefore come before any stream capture.  All
// calls share the one array and it keeps the last call's contents: everything
// that must start at zero is cleared on the stream at the start of each call,
// and two calls whose work overlaps on the GPU race on the array.  No cudaMalloc, cudaFree or allocating library routine
// is called.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "internal.cuh"

namespace {

constexpr int64_t kMaxN = DBSCAN_NOALLOC_MAX_N;
constexpr int kMaxD = DBSCAN_NOALLOC_MAX_D;

constexpr size_t al(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kBytesP = al(sizeof(float) * (size_t)kMaxN * kMaxD);   // packed rows, stride <= 16
constexpr size_t kBytesI = al(sizeof(int32_t) * (size_t)kMaxN);         // count / parent / border
constexpr size_t kBytesCore = al((size_t)kMaxN);                         // core flags
constexpr size_t kBytesScan = al(sizeof(int32_t) * ((size_t)kMaxN + 1));
constexpr int64_t kPartCap = kMaxN / 2048 + 4;
constexpr size_t kBytesPart = al(sizeof(int32_t) * (size_t)kPartCap);
constexpr size_t kBytesStatus = 256, kBytesCtr = 256;
constexpr size_t kScratchBytes =
    kBytesP + 3 * kBytesI + kBytesCore + kBytesScan + kBytesPart + kBytesStatus + kBytesCtr;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct ScratchEntry {
    unsigned char *addr = nullptr;
    unsigned long long ctx_id = 0;  // context the address belongs to (0: unknown)
};
ScratchEntry g_entry[kMaxDevices];

// Unique id of the calling thread's current CUDA context (0 if there is none
// or the driver does not say).  The driver's entry points are looked up through
// the runtime, so the library needs no link to the driver library.
unsigned long long current_context_id() {
    using GetCurrent = int (*)(void **);
    using GetId = int (*)(void *, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
        cudaGetLastError();
    });
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&ctx) == 0 && ctx && get_id(ctx, &id) == 0) return id;
    return 0;
}

// Device address of g_scratch in the calling thread's current device and
// context.  Looked up once per device and cached with the context's id; a new
// context on that device (after cudaDeviceReset, say) triggers a new lookup.
int scratch_address(unsigned char **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DBSCAN_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    ScratchEntry &e = g_entry[dev];
    const unsigned long long ctx = current_context_id();
    if (!e.addr || (ctx != 0 && ctx != e.ctx_id)) {
        void *p = nullptr;
        const cudaError_t err = cudaGetSymbolAddress(&p, g_scratch);
        if (err != cudaSuccess || !p) {
            cudaGetLastError();
            e.addr = nullptr;
            return DBSCAN_ERR_CUDA;
        }
        e.addr = static_cast<unsigned char *>(p);
        e.ctx_id = current_context_id();  // the lookup may have created the context
    }
    *out = e.addr;
    return DBSCAN_OK;
}

}  // namespace

extern "C" int dbscan_run_noalloc(const float *points, int64_t n, int32_t d, float eps, int32_t min_pts,
                                  int32_t label_mode, int32_t *labels_out, void *stream) {
    if (n < 0 || n > kMaxN || d < 1 || d > kMaxD || !(eps > 0.0f) || eps != eps || eps > 3.0e38f || min_pts < 1 ||
        (label_mode != DBSCAN_LABEL_ROOT_INDEX && label_mode != DBSCAN_LABEL_COMPACT))
        return DBSCAN_ERR_ARG;
    if (n > 0 && (!points || !labels_out)) return DBSCAN_ERR_ARG;
    if (n == 0) return DBSCAN_OK;

    unsigned char *base = nullptr;
    int s = scratch_address(&base);
    if (s) return s;

    // Carve the fixed array exactly as sized above.
    DbWork w{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        unsigned char *p = base + off;
        off += bytes;
        return p;
    };
    w.cap_n = kMaxN;
    w.cap_d = kMaxD;
    w.dp_cap = kMaxD;
    w.P = reinterpret_cast<float *>(take(kBytesP));
    w.count = reinterpret_cast<int32_t *>(take(kBytesI));
    w.parent = reinterpret_cast<int32_t *>(take(kBytesI));
    w.border = reinterpret_cast<int32_t *>(take(kBytesI));
    w.core = take(kBytesCore);
    w.scan = reinterpret_cast<int32_t *>(take(kBytesScan));
    w.scan_part = reinterpret_cast<int32_t *>(take(kBytesPart));
    w.scan_part_cap = kPartCap;
    w.status = reinterpret_cast<unsigned *>(take(kBytesStatus));
    w.ctr = reinterpret_cast<unsigned long long *>(take(kBytesCtr));
    PhaseMarks marks;  // timing off
    w.marks = &marks;

    const double e = (double)eps;
    const int64_t T = (int64_t)std::floor(e * e * 1048576.0);
    const int64_t Tc = std::min<int64_t>(T, (int64_t)d * 1023 * 1023);
    const int dp = dp_for(d);
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    cudaError_t err = cudaMemsetAsync(w.status, 0, sizeof(unsigned), st);
    if (!err) err = cudaMemsetAsync(w.ctr, 0, kBytesCtr, st);
    if (!err) err = launch_prep_dense(w, points, n, d, dp, st);
    if (!err) err = launch_allpairs_simt(w, n, d, dp, Tc, min_pts, false, st);
    if (!err) err = launch_labels_allpairs(w, n, labels_out, nullptr, nullptr, st);
    if (!err && label_mode == DBSCAN_LABEL_COMPACT) err = launch_compact(w, n, labels_out, st);
    unsigned bits = 0;
    if (!err) err = cudaMemcpyAsync(&bits, w.status, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (!err) err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) {
        cudaGetLastError();
        return DBSCAN_ERR_CUDA;
    }
    if (bits & DB_EBIT_NOT_QUANTISED) return DBSCAN_ERR_NOT_QUANTISED;
    if (bits & DB_EBIT_TIMEOUT) return DBSCAN_ERR_TIMEOUT;
    if (bits) return DBSCAN_ERR_CUDA;
    return DBSCAN_OK;
}
