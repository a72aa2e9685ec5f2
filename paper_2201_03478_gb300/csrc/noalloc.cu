// noalloc.cu -- interp_tod_noalloc: the TOD evaluation of interp_tod for
// callers that must not allocate device memory during the call.
//
// Who needs it: code that runs while another component owns the device-memory
// budget (a caching allocator that must not see foreign cudaMalloc/cudaFree),
// and long-running acquisition or processing loops that cannot afford the
// implicit device synchronisation of cudaMalloc/cudaFree.  interp_tod may
// grow the plan's sort scratch with cudaMalloc when n exceeds every earlier
// call; this entry point never does.
//
// Its scratch (the pointing sort: per-sample stencil records, keys and
// permutation, the tile histogram and cursors) lives in one file-scope
// __device__ array of fixed size, held by every GPU that loads the library
// until the process exits:
//   kNoAllocMaxSamples (262,144) samples and kNoAllocMaxTiles (65,536) grid
//   tiles, 8.75 MiB per device.
// A call with n above kNoAllocMaxSamples is rejected with SL_ERR_ARG; the
// caller splits a longer TOD into chunks of at most that many samples.  The
// sort here keys samples by tile (not by cell), which keeps the histogram small.
#include <mutex>

#include "sl_internal.cuh"

namespace sl {

constexpr int64_t kNoAllocMaxSamples = 1 << 18;
constexpr int kNoAllocMaxTiles = 1 << 16;
// words (4 bytes): records (24 bytes each), keys, permutation, histogram, cursor, block sums
constexpr size_t kRecWords = (size_t)kNoAllocMaxSamples * (sizeof(StencilRec64) / 4);
constexpr size_t kBsumWords = (size_t)kNoAllocMaxTiles / 4096 + 2;
constexpr size_t kNoAllocWords = kRecWords + 2 * (size_t)kNoAllocMaxSamples + (kNoAllocMaxTiles + 1) +
                                  kNoAllocMaxTiles + kBsumWords + (kNoAllocMaxTiles + 1);

static __device__ __align__(256) unsigned g_noalloc_scratch[kNoAllocWords];

// Device address of g_noalloc_scratch per device ordinal.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device with cudaGetSymbolAddress (with that device current).
constexpr int kMaxDevices = 64;
static unsigned *g_scratch_ptr[kMaxDevices] = {nullptr};
static std::mutex g_scratch_mu;

static sl_status scratch_for_device(int device, unsigned **out) {
    if (device < 0 || device >= kMaxDevices)
        return set_error(SL_ERR_UNSUPPORTED, "interp_tod_noalloc: device ordinal %d >= %d", device, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[device]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr)
            return cuda_check(e != cudaSuccess ? e : cudaErrorInvalidSymbol,
                              "interp_tod_noalloc: cudaGetSymbolAddress of the static scratch");
        g_scratch_ptr[device] = (unsigned *)ptr;
    }
    *out = g_scratch_ptr[device];
    return SL_OK;
}

}  // namespace sl

using namespace sl;

extern "C" sl_status interp_tod_noalloc(sl_plan *p, const void *maps, const double *theta, const double *phi,
                                        const double *psi, int64_t n, double *tod) {
    if (!p) return set_error(SL_ERR_ARG, "interp_tod_noalloc: plan is NULL");
    sl_status st = cuda_check(cudaSetDevice(p->device), "cudaSetDevice");
    if (st != SL_OK) return st;
    if (n < 0 || n > kNoAllocMaxSamples)
        return set_error(SL_ERR_ARG, "interp_tod_noalloc: n=%lld outside [0, %lld] (the static scratch limit; "
                                     "split the TOD into chunks)", (long long)n, (long long)kNoAllocMaxSamples);
    if (p->ntiles > kNoAllocMaxTiles)
        return set_error(SL_ERR_UNSUPPORTED, "interp_tod_noalloc: the plan's grid has %d sort tiles, more than the "
                                             "static scratch holds (%d)", p->ntiles, kNoAllocMaxTiles);
    if (!maps || (n > 0 && (!theta || !phi || !psi || !tod)))
        return set_error(SL_ERR_ARG, "interp_tod_noalloc: NULL buffer");
    if (n == 0) return SL_OK;
    unsigned *base = nullptr;
    if ((st = scratch_for_device(p->device, &base)) != SL_OK) return st;
    SortBufs b;
    b.rec = base;                                          // 256-byte aligned records
    b.keys = base + kRecWords;
    b.perm = b.keys + kNoAllocMaxSamples;
    b.hist = b.perm + kNoAllocMaxSamples;                  // cleared by the sort before use
    b.cursor = b.hist + (kNoAllocMaxTiles + 1);
    b.bsum = b.cursor + kNoAllocMaxTiles;
    const int rec64 = plan_wide(p->precision);
    // FP32, TF32X3 and DF64 plans interpolate tile by tile from shared memory and need
    // the per-tile work list; FP64 plans gather per sample and do not.
    const int chunks = p->precision != SL_FP64;
    b.chunk_off = chunks ? b.bsum + kBsumWords : nullptr;
    if ((st = launch_sort_into(p, b, theta, phi, psi, n, 0, rec64, chunks)) != SL_OK) return st;
    return launch_interp(p, b, 0, maps, psi, n, tod);
}
