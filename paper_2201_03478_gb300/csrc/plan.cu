// plan.cu -- the C ABI of libsidelobe.so (include/sidelobe.h): argument
// validation, plan geometry, scratch management, the call sequences of the
// public entry points and per-kernel timing.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>
#include <cmath>
#include <vector>
#include <new>

#include "sl_internal.cuh"

namespace sl {

static thread_local char g_err[512] = "";

sl_status set_error(sl_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

cudaError_t allow_dyn_smem_fn(const void *kern, size_t sm) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> caps;   // (kernel, device) -> cap set
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    auto it = caps.find({kern, dev});
    if (it == caps.end()) {
        int optin = 0;
        cudaFuncAttributes fa;
        if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
        if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
        const int cap = optin - (int)fa.sharedSizeBytes;
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, cap)) != cudaSuccess) return e;
        it = caps.emplace(std::make_pair(kern, dev), cap).first;
    }
    return sm <= (size_t)it->second ? cudaSuccess : cudaErrorInvalidValue;
}

sl_status cuda_check(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return SL_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return set_error(SL_ERR_NOMEM, "%s: %s", what, cudaGetErrorString(e));
    }
    return set_error(SL_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ------------------------------------------------------------------ timing
int timing_begin(sl_plan *p, const char *name) {
    if (!p->timing) return -1;
    int idx = -1;
    for (size_t i = 0; i < p->timers.size(); ++i)
        if (p->timers[i].name == name) idx = (int)i;
    if (idx < 0) {
        p->timers.push_back(KernelTimer{name, 0, 0.0});
        idx = (int)p->timers.size() - 1;
    }
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return -1;
    if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return -1; }
    cudaEventRecord(a, p->stream);
    p->pending_ev.push_back(a);
    p->pending_ev.push_back(b);
    p->pending_idx.push_back(idx);
    return (int)p->pending_idx.size() - 1;
}

void timing_end(sl_plan *p, int slot) {
    if (slot < 0) return;
    cudaEventRecord(p->pending_ev[2 * slot + 1], p->stream);
}

static void timing_flush(sl_plan *p) {
    if (p->pending_idx.empty()) return;
    cudaStreamSynchronize(p->stream);
    for (size_t i = 0; i < p->pending_idx.size(); ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p->pending_ev[2 * i], p->pending_ev[2 * i + 1]) == cudaSuccess) {
            p->timers[p->pending_idx[i]].launches += 1;
            p->timers[p->pending_idx[i]].total_ms += ms;
        }
    }
    for (cudaEvent_t e : p->pending_ev) cudaEventDestroy(e);
    p->pending_ev.clear();
    p->pending_idx.clear();
}

// ------------------------------------------------------------------ allocation
static sl_status dalloc(sl_plan *p, void **ptr, size_t bytes, const char *what) {
    *ptr = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();
        return set_error(SL_ERR_NOMEM, "cudaMalloc(%zu bytes) for %s failed: %s", bytes, what,
                         cudaGetErrorString(e));
    }
    p->bytes_held += (int64_t)bytes;
    return SL_OK;
}

template <typename T>
static sl_status dalloc_t(sl_plan *p, T **ptr, size_t count, const char *what) {
    void *v = nullptr;
    sl_status st = dalloc(p, &v, count * sizeof(T), what);
    *ptr = (T *)v;
    return st;
}

static void dfree(void *ptr) {
    if (ptr) cudaFree(ptr);
}

static sl_status ensure_sort_capacity(sl_plan *p, int64_t n) {
    if (n <= p->sort_cap) return SL_OK;
    if (p->batch_refs > 0)
        return set_error(SL_ERR_ARG, "n=%lld exceeds the sort scratch (%lld samples) of a plan that a batch graph "
                                     "holds; reserve the capacity before the batch is created",
                         (long long)n, (long long)p->sort_cap);
    cudaStreamSynchronize(p->stream);
    dfree(p->sort.keys);
    dfree(p->sort.perm);
    dfree(p->sort.rec);
    if (p->sort_cap > 0)
        p->bytes_held -= p->sort_cap * (int64_t)(2 * sizeof(unsigned) + sizeof(StencilRec64)) + 4 * (int64_t)sizeof(unsigned);
    p->sort.keys = p->sort.perm = nullptr;
    p->sort.rec = nullptr;
    p->sort_cap = 0;
    sl_status st = dalloc_t(p, &p->sort.keys, (size_t)n, "sort keys");
    if (st != SL_OK) return st;
    st = dalloc_t(p, &p->sort.perm, (size_t)n + 4, "sort permutation");
    if (st != SL_OK) return st;
    st = dalloc(p, &p->sort.rec, (size_t)n * sizeof(StencilRec64), "stencil records");
    if (st != SL_OK) return st;
    p->sort_cap = n;
    return SL_OK;
}

// Per-key tables of the sort (their size follows the tile grid).
static sl_status alloc_sort_tables(sl_plan *p) {
    p->nkeys = sort_nkeys(p, 1);
    sl_status st = dalloc_t(p, &p->sort.hist, (size_t)p->nkeys + 1, "cell histogram");
    if (st == SL_OK) st = dalloc_t(p, &p->sort.cursor, (size_t)p->nkeys, "cell cursor");
    if (st == SL_OK) st = dalloc_t(p, &p->sort.bsum, (size_t)sort_nbsum(p->nkeys) + 2, "scan block sums");
    if (st == SL_OK) st = dalloc_t(p, &p->sort.chunk_off, (size_t)p->ntiles + 1, "tile chunks");
    return st;
}

static void free_sort_tables(sl_plan *p) {
    dfree(p->sort.hist);
    dfree(p->sort.cursor);
    dfree(p->sort.bsum);
    dfree(p->sort.chunk_off);
    p->sort.hist = p->sort.cursor = p->sort.bsum = p->sort.chunk_off = nullptr;
    p->bytes_held -= (int64_t)sizeof(unsigned) * ((p->nkeys + 1) + p->nkeys + (sort_nbsum(p->nkeys) + 2) +
                                                  (p->ntiles + 1));
}

// Shared memory the tile-staged kernels need at tile width tc.
static size_t tile_smem_need(const sl_plan *p, int tc) {
    size_t need = interp_adjoint_smem_tc(p, tc);
    if (plan_fp32(p->precision))
        need = std::max(need, std::max(interp_f32_tiled_smem_tc(p, tc), interp_f32_cells_smem_tc(p, tc)));
    if (p->precision == SL_DF64)
        need = std::max(need, std::max(interp_df_tiled_smem_tc(p, tc), interp_adjoint_df_smem_tc(p, tc)));
    return need;
}
constexpr size_t kSmemOptin = 232448;   // 227 KB of dynamic shared memory per CTA (sm_100 family)

static void set_tile_grid(sl_plan *p, int tc) {
    p->geom.tile_cols = tc;
    p->geom.ntr = (p->R + 1 + kTileRows - 1) / kTileRows;
    p->geom.ntc = (p->nphi + tc - 1) / tc;
    p->ntiles = p->geom.ntr * p->geom.ntc;
}

static sl_status ensure_adjoint_scratch(sl_plan *p) {
    sl_status st;
    if (!p->d_Abar) {
        st = dalloc_t(p, &p->d_Abar, (size_t)(p->K + 1) * (2 * p->L + 1) * (p->L + 1), "adjoint A");
        if (st != SL_OK) return st;
    }
    if (!p->d_Gadj) {
        if (plan_wide(p->precision)) {
            p->d_Gadj = (double2 *)p->d_G;
        } else {
            st = dalloc_t(p, &p->d_Gadj, (size_t)(p->K + 1) * p->R * (2 * p->L + 1), "adjoint G");
            if (st != SL_OK) return st;
        }
    }
    // the adjoint contraction runs in FP64: FP32 plans build the FP64 table and
    // start states (threshold 2^-64) on first use
    if (plan_wide(p->precision)) {
        p->d_ls_adj = p->d_ls;
        p->d_st64_adj = p->d_st64;
    } else if (!p->d_st64_adj) {
        const size_t nst = (size_t)(p->K + 1) * (p->L + 1) * 2 * p->npairs;
        if ((st = dalloc_t(p, &p->d_tab64, (size_t)(p->K + 1) * p->nalm, "recurrence table")) != SL_OK) return st;
        if ((st = launch_rtab(p)) != SL_OK) return st;
        if ((st = dalloc_t(p, &p->d_ls_adj, nst, "adjoint start l")) != SL_OK) return st;
        if ((st = dalloc_t(p, &p->d_st64_adj, nst, "adjoint start states")) != SL_OK) return st;
        if ((st = launch_advance(p, 0x1p-64, p->d_ls_adj, p->d_st64_adj, nullptr)) != SL_OK) return st;
    }
    return SL_OK;
}

static sl_status ensure_fbar(sl_plan *p) {
    if (p->d_Fbar) return SL_OK;
    return dalloc_t(p, &p->d_Fbar, (size_t)p->R * p->nphi * (p->K + 1), "adjoint cube");
}

// ------------------------------------------------------------------ validation
// Radices of the ring FFT.  Radix 8 takes fewer FP64 operations per point
// (FP64-class plans, whose FFT the FP64 pipe binds: 2.52 -> 2.34 ms at 2048
// points); FP32 plans keep radix 4, whose smaller register count keeps one more
// CTA per SM on the L1-bound FP32 FFT (radix 8 measured 0.348 -> 0.373 ms).
static bool factor_235(int n, int *rad, int *nrad, bool radix8) {
    int k = 0;
    while (radix8 && n % 8 == 0 && k < kMaxRadices) { rad[k++] = 8; n /= 8; }
    while (n % 4 == 0 && k < kMaxRadices) { rad[k++] = 4; n /= 4; }
    while (n % 2 == 0 && k < kMaxRadices) { rad[k++] = 2; n /= 2; }
    while (n % 3 == 0 && k < kMaxRadices) { rad[k++] = 3; n /= 3; }
    while (n % 5 == 0 && k < kMaxRadices) { rad[k++] = 5; n /= 5; }
    *nrad = k;
    return n == 1;
}

static sl_status validate(const sl_plan_desc *d, int *rad, int *nrad) {
    if (!d) return set_error(SL_ERR_ARG, "desc is NULL");
    if (d->lmax < 1 || d->lmax > 16384) return set_error(SL_ERR_ARG, "lmax=%d outside [1, 16384]", d->lmax);
    if (d->kmax < 0 || d->kmax > d->lmax || d->kmax > kMaxK)
        return set_error(SL_ERR_ARG, "kmax=%d outside [0, min(lmax, %d)]", d->kmax, kMaxK);
    if (d->ncomp != 1 && d->ncomp != 3) return set_error(SL_ERR_ARG, "ncomp=%d (must be 1 or 3)", d->ncomp);
    int p = d->interp_order ? d->interp_order : 4;
    if (p < 2 || (p & 1)) return set_error(SL_ERR_ARG, "interp_order=%d (must be even, >= 2)", d->interp_order);
    if (p > 6) return set_error(SL_ERR_UNSUPPORTED, "interp_order=%d (2, 4 and 6 are built)", d->interp_order);
    if (d->nrings < 4 || d->nrings > 65534) return set_error(SL_ERR_ARG, "nrings=%d outside [4, 65534]", d->nrings);
    if (!d->ring_theta) return set_error(SL_ERR_ARG, "ring_theta is NULL");
    const double *t = d->ring_theta;
    for (int r = 0; r < d->nrings; ++r) {
        if (!(t[r] > 0.0 && t[r] < M_PI)) return set_error(SL_ERR_ARG, "ring_theta[%d]=%g not in (0, pi)", r, t[r]);
        if (r > 0 && !(t[r] > t[r - 1])) return set_error(SL_ERR_ARG, "ring_theta not strictly ascending at %d", r);
        double mir = M_PI - t[d->nrings - 1 - r];
        if (fabs(mir - t[r]) > 1e-12) return set_error(SL_ERR_ARG, "ring_theta not N/S symmetric at ring %d", r);
    }
    if (d->nphi < 8 || d->nphi > kMaxNphi || (d->nphi & 1))
        return set_error(SL_ERR_ARG, "nphi=%d must be even and in [8, %d]", d->nphi, kMaxNphi);
    if (!factor_235(d->nphi, rad, nrad, !plan_fp32(d->precision)))
        return set_error(SL_ERR_UNSUPPORTED, "nphi=%d has a prime factor > 5", d->nphi);
    if ((int64_t)d->nrings * d->nphi * (d->kmax + 1) >= ((int64_t)1 << 31))
        return set_error(SL_ERR_UNSUPPORTED, "nrings * nphi * (kmax + 1) >= 2^31 (cube element offsets are 32-bit)");
    if (d->precision != SL_FP64 && d->precision != SL_FP32 && d->precision != SL_DF64 && d->precision != SL_TF32X3)
        return set_error(SL_ERR_ARG, "precision=%d unknown", d->precision);
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return set_error(SL_ERR_CUDA, "no CUDA device visible");
    }
    if (d->device < 0 || d->device >= ndev) return set_error(SL_ERR_ARG, "device=%d of %d", d->device, ndev);
    return SL_OK;
}

}  // namespace sl

using namespace sl;

// ====================================================================== C ABI
extern "C" {

const char *sl_last_error(void) { return g_err; }

void plan_destroy(sl_plan *p) {
    if (!p) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(p->device);
    cudaStreamSynchronize(p->stream);
    for (cudaEvent_t e : p->pending_ev) cudaEventDestroy(e);
    dfree(p->d_ring_theta);
    dfree(p->d_xr);
    dfree(p->d_y32);
    dfree(p->d_ring_ext);
    dfree(p->d_ring_fix);
    dfree(p->d_wden);
    dfree(p->d_lut);
    dfree(p->d_seed);
    dfree(p->d_seed_e);
    dfree(p->d_tab64);
    dfree(p->d_tab32);
    if (p->d_ls_adj && p->d_ls_adj != p->d_ls) dfree(p->d_ls_adj);
    if (p->d_st64_adj && p->d_st64_adj != p->d_st64) dfree(p->d_st64_adj);
    dfree(p->d_ls);
    dfree(p->d_st64);
    dfree(p->d_st32);
    dfree(p->d_sky32);
    dfree(p->d_beam32);
    dfree(p->d_tw64);
    dfree(p->d_tw32);
    dfree(p->d_fftperm);
    dfree(p->d_fftpos);
    dfree(p->d_ptw64);
    dfree(p->d_ptw32);
    if (p->d_Gadj && (void *)p->d_Gadj != p->d_G) dfree(p->d_Gadj);
    dfree(p->d_G);
    dfree(p->d_Fbar);
    dfree(p->d_Abar);
    dfree(p->d_offs64);
    dfree(p->d_rowtab32);
    dfree(p->d_skym32);
    dfree(p->d_Gm);
    dfree(p->d_err);
    dfree(p->d_orb);
    dfree(p->d_psitab);
    if (p->h_orb) cudaFreeHost(p->h_orb);
    if (p->orb_ev) cudaEventDestroy(p->orb_ev);
    dfree(p->d_rowtab_df);
    dfree(p->sort.hist);
    dfree(p->sort.cursor);
    dfree(p->sort.bsum);
    dfree(p->sort.chunk_off);
    dfree(p->sort.keys);
    dfree(p->sort.perm);
    dfree(p->sort.rec);
    if (p->side_fork) cudaEventDestroy(p->side_fork);
    if (p->side_join) cudaEventDestroy(p->side_join);
    if (p->side) cudaStreamDestroy(p->side);
    if (p->up) cudaStreamSynchronize(p->up);
    if (p->down) cudaStreamSynchronize(p->down);
    dfree(p->d_hin);
    dfree(p->d_htod);
    dfree(p->d_hmaps);
    for (int c = 0; c < 64; ++c) {
        if (p->h_arrived[c]) cudaEventDestroy(p->h_arrived[c]);
        if (p->h_done[c]) cudaEventDestroy(p->h_done[c]);
    }
    if (p->up) cudaStreamDestroy(p->up);
    if (p->down) cudaStreamDestroy(p->down);
    delete p;
    cudaSetDevice(prev);
}

sl_status sidelobe_plan_create(sl_plan **out, const sl_plan_desc *d) {
    if (!out) return set_error(SL_ERR_ARG, "out is NULL");
    *out = nullptr;
    int rad[kMaxRadices], nrad = 0;
    sl_status st = validate(d, rad, &nrad);
    if (st != SL_OK) return st;
    st = cuda_check(cudaSetDevice(d->device), "cudaSetDevice");
    if (st != SL_OK) return st;

    sl_plan *p = new (std::nothrow) sl_plan();
    if (!p) return set_error(SL_ERR_NOMEM, "host allocation of the plan failed");
    p->L = d->lmax;
    p->K = d->kmax;
    p->ncomp = d->ncomp;
    p->R = d->nrings;
    p->nphi = d->nphi;
    p->p = d->interp_order ? d->interp_order : 4;
    p->precision = d->precision;
    p->device = d->device;
    p->stream = (cudaStream_t)d->stream;
    p->npairs = (p->R + 1) / 2;
    p->nalm = (int64_t)(p->L + 1) * (p->L + 2) / 2;
    for (int i = 0; i < nrad; ++i) p->radices[i] = rad[i];
    p->nradix = nrad;

    const int R = p->R, L = p->L, K = p->K, half = p->p / 2, P = p->p;
    const double *th = d->ring_theta;

    // -------- geometry on the host in long double, then uploaded
    std::vector<double> ring_ext(R + 2 * half), wden((size_t)(R + 1) * P), xr(p->npairs),
        c2(p->npairs), s2(p->npairs), cs(p->npairs);
    std::vector<float> y32(p->npairs);
    for (int row = -half; row < R + half; ++row) {
        double v;
        if (row < 0) v = -th[-1 - row];
        else if (row >= R) v = 2.0 * M_PI - th[2 * R - 1 - row];
        else v = th[row];
        ring_ext[row + half] = v;
    }
    for (int i = -1; i <= R - 1; ++i) {
        for (int a = 0; a < P; ++a) {
            long double ta = ring_ext[i - half + 1 + a + half], den = 1.0L;
            for (int b = 0; b < P; ++b)
                if (b != a) den *= ta - (long double)ring_ext[i - half + 1 + b + half];
            wden[(size_t)(i + 1) * P + a] = (double)(1.0L / den);
        }
    }
    // per base row i: theta(i0+a) - theta(i0), i0 = i - p/2 + 1 (double) and the
    // same offsets followed by wden in float and in double-float
    std::vector<double> offs64((size_t)(R + 1) * P);
    std::vector<float> rowtab32((size_t)(R + 1) * 2 * P);
    std::vector<float2> rowtab_df((size_t)(R + 1) * 2 * P);
    auto split = [](long double v) {
        const float h = (float)v;
        return make_float2(h, (float)(v - (long double)h));
    };
    for (int i = -1; i <= R - 1; ++i) {
        const double t0 = ring_ext[i + 1];            // row i0 = i - half + 1 sits at index i0 + half
        for (int a = 0; a < P; ++a) {
            const double o = (double)((long double)ring_ext[i + 1 + a] - (long double)t0);
            offs64[(size_t)(i + 1) * P + a] = o;
            rowtab32[(size_t)(i + 1) * 2 * P + a] = (float)o;
            rowtab32[(size_t)(i + 1) * 2 * P + P + a] = (float)wden[(size_t)(i + 1) * P + a];
            rowtab_df[(size_t)(i + 1) * 2 * P + a] = split(o);
            rowtab_df[(size_t)(i + 1) * 2 * P + P + a] = split(wden[(size_t)(i + 1) * P + a]);
        }
    }
    for (int r = 0; r < p->npairs; ++r) {
        long double t = th[r];
        xr[r] = (double)cosl(t);
        c2[r] = (double)cosl(t / 2);
        s2[r] = (double)sinl(t / 2);
        cs[r] = (double)(cosl(t / 2) * sinl(t / 2));
        y32[r] = (float)(2.0L * sinl(t / 2) * sinl(t / 2));
    }
    int nlut = 4 * (R + 1);
    std::vector<int> lut(nlut);
    {
        int i = -1;
        for (int b = 0; b < nlut; ++b) {
            double t0 = b * M_PI / nlut;
            while (i < R - 1 && ring_ext[i + 1 + half] <= t0) ++i;
            lut[b] = std::max(-1, i - 1);   // one row of margin against rounding of theta*scale
        }
    }
    std::vector<double2> tw64(p->nphi);
    std::vector<float2> tw32(p->nphi);
    for (int j = 0; j < p->nphi; ++j) {
        long double a = 2.0L * 3.14159265358979323846264338327950288L * j / p->nphi;
        tw64[j] = make_double2((double)cosl(a), (double)sinl(a));
        tw32[j] = make_float2((float)cosl(a), (float)sinl(a));
    }

    p->geom.R = R;
    p->geom.nphi = p->nphi;
    p->geom.K = K;
    p->geom.p = P;
    p->geom.half = half;
    p->geom.nlut = nlut;
    p->geom.lut_scale = nlut / M_PI;
    p->geom.lut_scale_f = (float)(nlut / M_PI);
    p->geom.phi_scale = p->nphi / (2.0 * M_PI);
    // round(nphi / (2 pi) 2^52) < 2^64 for nphi <= 16384 (the rounding stays unsigned)
    p->geom.phi_fix = (unsigned long long)(
        ldexpl((long double)p->nphi / (2.0L * 3.14159265358979323846264338327950288L), 52) + 0.5L);

    double *d_c2 = nullptr, *d_s2 = nullptr, *d_cs = nullptr;
#define TRY(x)                      \
    do {                            \
        st = (x);                   \
        if (st != SL_OK) goto fail; \
    } while (0)
    {   // tile width: 32 columns (16 when kmax > 16), at most nphi and within the
        // shared memory of the tile-staged kernels; one of 8, 16, 32
        int tc = (K <= 16) ? 32 : 16;
        while (tc > 8 && (tc > p->nphi || tile_smem_need(p, tc) > kSmemOptin)) tc >>= 1;
        if (tile_smem_need(p, tc) > kSmemOptin) {
            st = set_error(SL_ERR_UNSUPPORTED, "kmax=%d with interp_order=%d: a sort tile exceeds shared memory", K, P);
            goto fail;
        }
        set_tile_grid(p, tc);
    }
    TRY(dalloc_t(p, &p->d_ring_theta, R, "ring theta"));
    TRY(dalloc_t(p, &p->d_xr, p->npairs, "ring cos"));
    TRY(dalloc_t(p, &p->d_y32, p->npairs, "ring 1-cos"));
    TRY(dalloc_t(p, &p->d_ring_ext, ring_ext.size(), "ring ext"));
    TRY(dalloc_t(p, &p->d_wden, wden.size(), "lagrange denominators"));
    TRY(dalloc_t(p, &p->d_lut, lut.size(), "ring lut"));
    TRY(dalloc_t(p, &p->d_tw64, tw64.size(), "twiddles"));
    TRY(dalloc_t(p, &p->d_tw32, tw32.size(), "twiddles"));
    TRY(dalloc_t(p, &p->d_fftperm, (size_t)p->nphi, "fft slot table"));
    TRY(dalloc_t(p, &d_c2, p->npairs, "seed tmp"));
    TRY(dalloc_t(p, &d_s2, p->npairs, "seed tmp"));
    TRY(dalloc_t(p, &d_cs, p->npairs, "seed tmp"));
    TRY(cuda_check(cudaMemcpy(p->d_ring_theta, th, R * sizeof(double), cudaMemcpyHostToDevice), "upload"));
    TRY(cuda_check(cudaMemcpy(p->d_xr, xr.data(), xr.size() * sizeof(double), cudaMemcpyHostToDevice), "upload"));
    TRY(cuda_check(cudaMemcpy(p->d_y32, y32.data(), y32.size() * sizeof(float), cudaMemcpyHostToDevice), "upload"));
    TRY(cuda_check(cudaMemcpy(p->d_ring_ext, ring_ext.data(), ring_ext.size() * sizeof(double), cudaMemcpyHostToDevice), "upload"));
    {
        std::vector<long long> ring_fix(ring_ext.size());
        for (size_t q = 0; q < ring_ext.size(); ++q) ring_fix[q] = llroundl(ldexpl((long double)ring_ext[q], 60));
        TRY(dalloc_t(p, &p->d_ring_fix, ring_fix.size(), "ring fixed point"));
        TRY(cuda_check(cudaMemcpy(p->d_ring_fix, ring_fix.data(), ring_fix.size() * sizeof(long long),
                                  cudaMemcpyHostToDevice), "upload"));
    }
    TRY(cuda_check(cudaMemcpy(p->d_wden, wden.data(), wden.size() * sizeof(double), cudaMemcpyHostToDevice), "upload"));
    TRY(cuda_check(cudaMemcpy(p->d_lut, lut.data(), lut.size() * sizeof(int), cudaMemcpyHostToDevice), "upload"));
    TRY(cuda_check(cudaMemcpy(p->d_tw64, tw64.data(), tw64.size() * sizeof(double2), cudaMemcpyHostToDevice), "upload"));
    TRY(cuda_check(cudaMemcpy(p->d_tw32, tw32.data(), tw32.size() * sizeof(float2), cudaMemcpyHostToDevice), "upload"));
    {
        // In-place ring FFT.  Input q sits in slot pos(q): the digits of q in the
        // radix sequence, the last pass's radix least significant, reversed; the
        // table holds q for each slot.  Pass twiddles: for pass (span Ns, radix R),
        // entries (q - 1) Ns + kk = e^{+2 pi i kk q / (Ns R)}, q in [1, R), kk < Ns,
        // passes one after another (nphi - 1 entries in all).
        std::vector<int> slotq((size_t)p->nphi), qslot((size_t)p->nphi);
        for (int q = 0; q < p->nphi; ++q) {
            int pos = 0, mult = p->nphi, n = q;
            for (int i = p->nradix - 1; i >= 0; --i) {
                mult /= p->radices[i];
                pos += (n % p->radices[i]) * mult;
                n /= p->radices[i];
            }
            slotq[(size_t)pos] = q;
            qslot[(size_t)q] = pos;
        }
        std::vector<double2> ptw64((size_t)p->nphi, make_double2(0.0, 0.0));
        std::vector<float2> ptw32((size_t)p->nphi, make_float2(0.f, 0.f));
        size_t o = 0;
        long long Ns = 1;
        for (int i = 0; i < p->nradix; ++i) {
            const int Rp = p->radices[i];
            for (int q = 1; q < Rp; ++q)
                for (long long kk = 0; kk < Ns; ++kk, ++o) {
                    const long double a = 2.0L * 3.14159265358979323846264338327950288L * (long double)(kk * q) /
                                          (long double)(Ns * Rp);
                    ptw64[o] = make_double2((double)cosl(a), (double)sinl(a));
                    ptw32[o] = make_float2((float)cosl(a), (float)sinl(a));
                }
            Ns *= Rp;
        }
        TRY(dalloc_t(p, &p->d_fftpos, qslot.size(), "fft slot table"));
        TRY(cuda_check(cudaMemcpy(p->d_fftpos, qslot.data(), qslot.size() * sizeof(int), cudaMemcpyHostToDevice),
                       "upload"));
        TRY(dalloc_t(p, &p->d_ptw64, ptw64.size(), "pass twiddles"));
        TRY(dalloc_t(p, &p->d_ptw32, ptw32.size(), "pass twiddles"));
        TRY(cuda_check(cudaMemcpy(p->d_fftperm, slotq.data(), slotq.size() * sizeof(int), cudaMemcpyHostToDevice),
                       "upload"));
        TRY(cuda_check(cudaMemcpy(p->d_ptw64, ptw64.data(), ptw64.size() * sizeof(double2), cudaMemcpyHostToDevice),
                       "upload"));
        TRY(cuda_check(cudaMemcpy(p->d_ptw32, ptw32.data(), ptw32.size() * sizeof(float2), cudaMemcpyHostToDevice),
                       "upload"));
    }
    TRY(cuda_check(cudaMemcpy(d_c2, c2.data(), c2.size() * sizeof(double), cudaMemcpyHostToDevice), "upload"));
    TRY(cuda_check(cudaMemcpy(d_s2, s2.data(), s2.size() * sizeof(double), cudaMemcpyHostToDevice), "upload"));
    TRY(cuda_check(cudaMemcpy(d_cs, cs.data(), cs.size() * sizeof(double), cudaMemcpyHostToDevice), "upload"));
    TRY(dalloc_t(p, &p->d_offs64, offs64.size(), "row offsets"));
    TRY(dalloc_t(p, &p->d_rowtab32, rowtab32.size(), "row table"));
    TRY(dalloc_t(p, &p->d_rowtab_df, rowtab_df.size(), "row table"));
    TRY(cuda_check(cudaMemcpy(p->d_rowtab_df, rowtab_df.data(), rowtab_df.size() * sizeof(float2),
                              cudaMemcpyHostToDevice), "upload"));
    TRY(cuda_check(cudaMemcpy(p->d_offs64, offs64.data(), offs64.size() * sizeof(double), cudaMemcpyHostToDevice), "upload"));
    TRY(cuda_check(cudaMemcpy(p->d_rowtab32, rowtab32.data(), rowtab32.size() * sizeof(float), cudaMemcpyHostToDevice), "upload"));
    p->geom.ring_ext = p->d_ring_ext;
    p->geom.ring_fix = p->d_ring_fix;
    p->geom.wden = p->d_wden;
    p->geom.lut = p->d_lut;
    p->geom.offs64 = p->d_offs64;
    p->geom.rowtab32 = p->d_rowtab32;
    p->geom.rowtab_df = p->d_rowtab_df;

    {
        size_t nseed = (size_t)(K + 1) * (L + 1) * p->npairs;
        TRY(dalloc_t(p, &p->d_seed, nseed, "seeds"));
        TRY(dalloc_t(p, &p->d_seed_e, nseed, "seed exponents"));
    }
    TRY(launch_seeds(p, d_c2, d_s2, d_cs));
    // the FP64 table drives the plan-time advance in both precisions; FP32 plans
    // keep only its float form
    TRY(dalloc_t(p, &p->d_tab64, (size_t)(K + 1) * p->nalm, "recurrence table"));
    if (plan_fp32(p->precision)) {
        TRY(dalloc_t(p, &p->d_tab32, (size_t)(K + 1) * p->nalm, "recurrence table"));
        TRY(dalloc_t(p, &p->d_sky32, (size_t)p->ncomp * sky_row_stride(p->nalm), "FP32 sky"));
        TRY(dalloc_t(p, &p->d_beam32, (size_t)p->ncomp * (K + 1) * (L + 1), "FP32 beam"));
    }
    TRY(launch_rtab(p));
    {
        const size_t nst = (size_t)(K + 1) * (L + 1) * 2 * p->npairs;
        TRY(dalloc_t(p, &p->d_ls, nst, "start l"));
        if (plan_wide(p->precision)) TRY(dalloc_t(p, &p->d_st64, nst, "start states"));
        else TRY(dalloc_t(p, &p->d_st32, nst, "start states"));
    }
    TRY(launch_advance(p, plan_wide(p->precision) ? 0x1p-64 : 0x1p-30, p->d_ls, p->d_st64, p->d_st32));
    TRY(count_lsteps(p, &p->lsteps));
    if (plan_fp32(p->precision)) {
        TRY(cuda_check(cudaStreamSynchronize(p->stream), "plan advance"));
        dfree(p->d_tab64);
        p->d_tab64 = nullptr;
        p->bytes_held -= (int64_t)(K + 1) * p->nalm * (int64_t)sizeof(RTab64);
    }
    {
        size_t gel = (size_t)(K + 1) * R * (2 * L + 1);
        p->G_bytes = gel * (plan_wide(p->precision) ? sizeof(double2) : sizeof(float2));
        TRY(dalloc(p, &p->d_G, p->G_bytes, "spin-Legendre scratch G"));
    }
    TRY(alloc_sort_tables(p));
    if (plan_fp32(p->precision)) {
        // [0]: device flag of the bounded waits (FP32 interpolation, tensor-core contraction);
        // [1]: work counter of the FP32 interpolation
        TRY(dalloc_t(p, &p->d_err, 2, "error flag"));
        TRY(cuda_check(cudaMemset(p->d_err, 0, 2 * sizeof(int)), "error flag"));
    }
    TRY(cuda_check(cudaStreamSynchronize(p->stream), "plan seeds"));
    dfree(d_c2);
    dfree(d_s2);
    dfree(d_cs);
    p->bytes_held -= 3 * (int64_t)p->npairs * sizeof(double);
    *out = p;
    return SL_OK;
fail:
    cudaStreamSynchronize(p->stream);
    dfree(d_c2);
    dfree(d_s2);
    dfree(d_cs);
    {
        char keep[512];
        snprintf(keep, sizeof(keep), "%s", g_err);
        plan_destroy(p);
        snprintf(g_err, sizeof(g_err), "%s", keep);
    }
    return st;
#undef TRY
}

static sl_status enter(sl_plan *p) {
    if (!p) return set_error(SL_ERR_ARG, "plan is NULL");
    return cuda_check(cudaSetDevice(p->device), "cudaSetDevice");
}

sl_status synth_spin_maps(sl_plan *p, const double *sky, const double *beam, void *maps) {
    sl_status st = enter(p);
    if (st != SL_OK) return st;
    if (!sky || !beam || !maps) return set_error(SL_ERR_ARG, "synth_spin_maps: NULL buffer");
    st = launch_lcontract(p, sky, beam);
    if (st != SL_OK) return st;
    return launch_ringfft_synth(p, maps);
}

static sl_status ensure_side_stream(sl_plan *p) {
    if (p->side) return SL_OK;
    sl_status st = cuda_check(cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking), "side stream");
    if (st == SL_OK) st = cuda_check(cudaEventCreateWithFlags(&p->side_fork, cudaEventDisableTiming), "side event");
    if (st == SL_OK) st = cuda_check(cudaEventCreateWithFlags(&p->side_join, cudaEventDisableTiming), "side event");
    return st;
}

static sl_status check_ptg(const double *theta, const double *phi, const double *psi, int64_t n,
                           const void *io, const char *who) {
    if (n < 0 || n >= ((int64_t)1 << 31)) return set_error(SL_ERR_ARG, "%s: n=%lld outside [0, 2^31)", who, (long long)n);
    if (n > 0 && (!theta || !phi || !psi || !io)) return set_error(SL_ERR_ARG, "%s: NULL buffer", who);
    return SL_OK;
}

sl_status interp_tod(sl_plan *p, const void *maps, const double *theta, const double *phi,
                     const double *psi, int64_t n, double *tod) {
    sl_status st = enter(p);
    if (st != SL_OK) return st;
    if ((st = check_ptg(theta, phi, psi, n, tod, "interp_tod")) != SL_OK) return st;
    if (!maps) return set_error(SL_ERR_ARG, "interp_tod: maps is NULL");
    if (n == 0) return SL_OK;
    if ((st = ensure_sort_capacity(p, n)) != SL_OK) return st;
    const int rec64 = plan_wide(p->precision);
    // FP32 and DF64 plans interpolate tile by tile from shared memory (needs the work items)
    SortBufs b = p->sort;
    const int chunks = p->precision != SL_FP64;
    if (!chunks) b.chunk_off = nullptr;
    if ((st = launch_sort_into(p, b, theta, phi, psi, n, 1, rec64, chunks)) != SL_OK) return st;
    return launch_interp(p, b, 1, maps, psi, n, tod);
}

sl_status convolve_tod(sl_plan *p, const double *sky, const double *beam, void *maps, const double *theta,
                       const double *phi, const double *psi, int64_t n, double *tod) {
    sl_status st = enter(p);
    if (st != SL_OK) return st;
    if (!sky || !beam || !maps) return set_error(SL_ERR_ARG, "convolve_tod: NULL sky, beam or maps");
    if ((st = check_ptg(theta, phi, psi, n, tod, "convolve_tod")) != SL_OK) return st;
    if (n == 0) return synth_spin_maps(p, sky, beam, maps);
    // scratch first (it may synchronise the plan's stream), then the fork
    if ((st = ensure_sort_capacity(p, n)) != SL_OK) return st;
    if ((st = ensure_side_stream(p)) != SL_OK) return st;
    const int rec64 = plan_wide(p->precision);
    SortBufs b = p->sort;
    const int chunks = p->precision != SL_FP64;
    if (!chunks) b.chunk_off = nullptr;
    // fork point: everything queued on the plan's stream before the call
    if ((st = cuda_check(cudaEventRecord(p->side_fork, p->stream), "fork")) != SL_OK) return st;
    if ((st = cuda_check(cudaStreamWaitEvent(p->side, p->side_fork, 0), "fork wait")) != SL_OK) return st;
    const cudaStream_t main_stream = p->stream;
    p->stream = p->side;   // the sort's launches (and their timers) go to the side stream
    st = launch_sort_into(p, b, theta, phi, psi, n, 1, rec64, chunks);
    if (st == SL_OK) st = cuda_check(cudaEventRecord(p->side_join, p->side), "sort done");
    p->stream = main_stream;
    if (st != SL_OK) return st;
    if ((st = launch_lcontract(p, sky, beam)) != SL_OK) return st;
    if ((st = launch_ringfft_synth(p, maps)) != SL_OK) return st;
    if ((st = cuda_check(cudaStreamWaitEvent(p->stream, p->side_join, 0), "join")) != SL_OK) return st;
    return launch_interp(p, b, 1, maps, psi, n, tod);
}

// ---- end to end from host buffers
constexpr int kMaxHostPieces = 64;   // the size of sl_plan's h_arrived / h_done

// Doubles of sky and beam at the front of d_hin (the pointings follow them).
static size_t host_harmonic_doubles(const sl_plan *p) {
    return (size_t)2 * p->ncomp * p->nalm + (size_t)2 * p->ncomp * (p->K + 1) * (p->L + 1);
}

// Streams, events and device buffers of convolve_tod_host for n samples.
static sl_status ensure_host_path(sl_plan *p, int64_t n) {
    sl_status st = SL_OK;
    if (!p->up) {
        if ((st = cuda_check(cudaStreamCreateWithFlags(&p->up, cudaStreamNonBlocking), "upload stream")) != SL_OK)
            return st;
        if ((st = cuda_check(cudaStreamCreateWithFlags(&p->down, cudaStreamNonBlocking), "download stream")) != SL_OK)
            return st;
        for (int c = 0; c < kMaxHostPieces && st == SL_OK; ++c) {
            st = cuda_check(cudaEventCreateWithFlags(&p->h_arrived[c], cudaEventDisableTiming), "piece event");
            if (st == SL_OK) st = cuda_check(cudaEventCreateWithFlags(&p->h_done[c], cudaEventDisableTiming), "piece event");
        }
        if (st != SL_OK) return st;
    }
    if (!p->d_hmaps) {
        const size_t mb = (size_t)p->R * p->nphi * (p->K + 1) * (plan_wide(p->precision) ? 16 : 8);
        if ((st = dalloc(p, &p->d_hmaps, mb, "host-path cube")) != SL_OK) return st;
    }
    if (n > p->host_cap) {
        cudaStreamSynchronize(p->stream);
        const size_t fixed = host_harmonic_doubles(p);
        if (p->host_cap >= 0)
            p->bytes_held -= (int64_t)((fixed + 3 * (size_t)p->host_cap + (size_t)p->host_cap) * sizeof(double));
        dfree(p->d_hin);
        dfree(p->d_htod);
        p->d_hin = p->d_htod = nullptr;
        p->host_cap = -1;
        if ((st = dalloc_t(p, &p->d_hin, fixed + 3 * (size_t)n, "host-path inputs")) != SL_OK) return st;
        if ((st = dalloc_t(p, &p->d_htod, (size_t)n, "host-path TOD")) != SL_OK) return st;
        p->host_cap = n;
    }
    return SL_OK;
}

static sl_status host_pipeline(sl_plan *p, const double *sky, const double *beam, const double *theta,
                               const double *phi, const double *psi, int64_t n, int np, double *tod) {
    const size_t nsky = (size_t)2 * p->ncomp * p->nalm;
    double *d_sky = p->d_hin, *d_beam = d_sky + nsky;
    double *d_th = d_sky + host_harmonic_doubles(p), *d_ph = d_th + p->host_cap, *d_ps = d_ph + p->host_cap;
    sl_status st = cuda_check(cudaMemcpyAsync(d_sky, sky, nsky * sizeof(double), cudaMemcpyDefault, p->stream), "sky");
    if (st == SL_OK)
        st = cuda_check(cudaMemcpyAsync(d_beam, beam, (host_harmonic_doubles(p) - nsky) * sizeof(double),
                                        cudaMemcpyDefault, p->stream), "beam");
    // the pointings piece by piece on the upload stream, after the work queued so far
    if (st == SL_OK) st = cuda_check(cudaEventRecord(p->side_fork, p->stream), "fork");
    if (st == SL_OK) st = cuda_check(cudaStreamWaitEvent(p->up, p->side_fork, 0), "fork wait");
    for (int c = 0; c < np && st == SL_OK; ++c) {
        const int64_t a = n * c / np, b = n * (c + 1) / np;
        const size_t bytes = (size_t)(b - a) * sizeof(double);
        if (b > a) {
            st = cuda_check(cudaMemcpyAsync(d_th + a, theta + a, bytes, cudaMemcpyDefault, p->up), "theta");
            if (st == SL_OK) st = cuda_check(cudaMemcpyAsync(d_ph + a, phi + a, bytes, cudaMemcpyDefault, p->up), "phi");
            if (st == SL_OK) st = cuda_check(cudaMemcpyAsync(d_ps + a, psi + a, bytes, cudaMemcpyDefault, p->up), "psi");
        }
        if (st == SL_OK) st = cuda_check(cudaEventRecord(p->h_arrived[c], p->up), "piece arrived");
    }
    // the cube while they arrive; then each piece's TOD, copied back on the download stream
    if (st == SL_OK) st = synth_spin_maps(p, d_sky, d_beam, p->d_hmaps);
    for (int c = 0; c < np && st == SL_OK; ++c) {
        const int64_t a = n * c / np, b = n * (c + 1) / np;
        st = cuda_check(cudaStreamWaitEvent(p->stream, p->h_arrived[c], 0), "piece wait");
        if (st == SL_OK && b > a) st = interp_tod(p, p->d_hmaps, d_th + a, d_ph + a, d_ps + a, b - a, p->d_htod + a);
        if (st == SL_OK) st = cuda_check(cudaEventRecord(p->h_done[c], p->stream), "piece done");
        if (st == SL_OK) st = cuda_check(cudaStreamWaitEvent(p->down, p->h_done[c], 0), "download wait");
        if (st == SL_OK && b > a)
            st = cuda_check(cudaMemcpyAsync(tod + a, p->d_htod + a, (size_t)(b - a) * sizeof(double),
                                            cudaMemcpyDefault, p->down), "tod");
    }
    return st;
}

sl_status convolve_tod_host(sl_plan *p, const double *sky, const double *beam, const double *theta,
                            const double *phi, const double *psi, int64_t n, int pieces, double *tod) {
    sl_status st = enter(p);
    if (st != SL_OK) return st;
    if (!sky || !beam) return set_error(SL_ERR_ARG, "convolve_tod_host: NULL sky or beam");
    if ((st = check_ptg(theta, phi, psi, n, tod, "convolve_tod_host")) != SL_OK) return st;
    if (pieces < 1 || pieces > kMaxHostPieces)
        return set_error(SL_ERR_ARG, "convolve_tod_host: pieces=%d outside [1, %d]", pieces, kMaxHostPieces);
    const int np = (int)std::min<int64_t>(pieces, std::max<int64_t>(n, 1));
    if ((st = ensure_host_path(p, n)) != SL_OK) return st;
    if (n > 0 && (st = ensure_sort_capacity(p, (n + np - 1) / np)) != SL_OK) return st;
    if ((st = ensure_side_stream(p)) != SL_OK) return st;
    st = host_pipeline(p, sky, beam, theta, phi, psi, n, np, tod);
    // returns only when nothing of the call is in flight, also after an error
    const sl_status su = cuda_check(cudaStreamSynchronize(p->up), "upload stream synchronize");
    const sl_status sd = cuda_check(cudaStreamSynchronize(p->down), "download stream synchronize");
    const sl_status ss = sl_plan_sync(p);   // the plan's stream, and the error flag of the bounded waits
    if (st != SL_OK) return st;
    return su != SL_OK ? su : (sd != SL_OK ? sd : ss);
}

sl_status adjoint_interp(sl_plan *p, const double *theta, const double *phi, const double *psi,
                         const double *tod, int64_t n, double *maps_bar) {
    sl_status st = enter(p);
    if (st != SL_OK) return st;
    if ((st = check_ptg(theta, phi, psi, n, tod, "adjoint_interp")) != SL_OK) return st;
    if (!maps_bar) return set_error(SL_ERR_ARG, "adjoint_interp: maps_bar is NULL");
    size_t bytes = (size_t)p->R * p->nphi * (p->K + 1) * sizeof(double2);
    if ((st = cuda_check(cudaMemsetAsync(maps_bar, 0, bytes, p->stream), "memset maps_bar")) != SL_OK) return st;
    if (n == 0) return SL_OK;
    if ((st = ensure_sort_capacity(p, n)) != SL_OK) return st;
    if ((st = launch_sort_into(p, p->sort, theta, phi, psi, n, 1, 1, 1)) != SL_OK) return st;
    return launch_interp_adjoint(p, p->sort, 1, psi, tod, n, (double2 *)maps_bar);
}

sl_status adjoint_synth(sl_plan *p, const double *maps_bar, const double *sky, const double *beam,
                        double *sky_grad, double *beam_grad, int accumulate) {
    sl_status st = enter(p);
    if (st != SL_OK) return st;
    if (!maps_bar || !sky || !beam) return set_error(SL_ERR_ARG, "adjoint_synth: NULL buffer");
    if (!sky_grad && !beam_grad) return SL_OK;
    if ((st = ensure_adjoint_scratch(p)) != SL_OK) return st;
    if ((st = launch_ringdft_adjoint(p, (const double2 *)maps_bar)) != SL_OK) return st;
    if ((st = launch_lcontract_adjoint(p)) != SL_OK) return st;
    return launch_grad(p, sky, beam, sky_grad, beam_grad, accumulate);
}

sl_status adjoint_tod(sl_plan *p, const double *theta, const double *phi, const double *psi,
                      const double *tod, int64_t n, const double *sky, const double *beam,
                      double *sky_grad, double *beam_grad, int accumulate) {
    sl_status st = enter(p);
    if (st != SL_OK) return st;
    if ((st = check_ptg(theta, phi, psi, n, tod, "adjoint_tod")) != SL_OK) return st;
    if (!sky || !beam) return set_error(SL_ERR_ARG, "adjoint_tod: NULL sky/beam");
    if ((st = ensure_fbar(p)) != SL_OK) return st;
    if ((st = adjoint_interp(p, theta, phi, psi, tod, n, (double *)p->d_Fbar)) != SL_OK) return st;
    return adjoint_synth(p, (const double *)p->d_Fbar, sky, beam, sky_grad, beam_grad, accumulate);
}

sl_status sl_plan_get_sizes(const sl_plan *p, sl_plan_sizes *o) {
    if (!p || !o) return set_error(SL_ERR_ARG, "NULL argument");
    o->nalm = p->nalm;
    o->sky_doubles = (int64_t)p->ncomp * p->nalm * 2;
    o->beam_doubles = (int64_t)p->ncomp * (p->K + 1) * (p->L + 1) * 2;
    o->maps_bytes = (int64_t)p->R * p->nphi * (p->K + 1) * (plan_wide(p->precision) ? 16 : 8);
    o->scratch_bytes = p->bytes_held;
    o->lsteps = p->lsteps;
    o->tile_cols = p->geom.tile_cols;
    {
        int rg, kg;
        ring_fft_tile(p, &rg, &kg);
        o->fft_rings = rg;
        o->fft_korders = kg;
    }
    o->contraction_pairs = p->precision == SL_FP32 ? (p->lc_ppt ? p->lc_ppt : lcontract_f32_ppt(p->npairs)) : 0;
    return SL_OK;
}

sl_status sl_plan_reserve(sl_plan *p, int64_t n) {
    sl_status st = enter(p);
    if (st != SL_OK) return st;
    if (n < 0 || n >= ((int64_t)1 << 31)) return set_error(SL_ERR_ARG, "sl_plan_reserve: n=%lld outside [0, 2^31)", (long long)n);
    return ensure_sort_capacity(p, n);
}

sl_status sl_plan_set_tile_cols(sl_plan *p, int tc) {
    sl_status st = enter(p);
    if (st != SL_OK) return st;
    if (tc != 8 && tc != 16 && tc != 32) return set_error(SL_ERR_ARG, "tile width %d is not 8, 16 or 32", tc);
    if (tc > p->nphi) return set_error(SL_ERR_ARG, "tile width %d exceeds nphi=%d", tc, p->nphi);
    if (tc == p->geom.tile_cols) return SL_OK;
    int dev_smem = 0;
    cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
    const size_t need = tile_smem_need(p, tc);
    if (dev_smem > 0 && need > (size_t)dev_smem)
        return set_error(SL_ERR_UNSUPPORTED, "tile width %d needs %zu bytes of shared memory (device: %d)", tc,
                         need, dev_smem);
    if (p->batch_refs > 0) return set_error(SL_ERR_ARG, "the plan is held by a batch graph");
    if ((st = cuda_check(cudaStreamSynchronize(p->stream), "stream synchronize")) != SL_OK) return st;
    free_sort_tables(p);
    set_tile_grid(p, tc);
    return alloc_sort_tables(p);
}

sl_status sl_plan_set_fft_tile(sl_plan *p, int rings, int korders) {
    sl_status st = enter(p);
    if (st != SL_OK) return st;
    if (rings == 0 && korders == 0) {
        p->fft_rg = p->fft_kg = 0;
        return SL_OK;
    }
    if ((rings != 1 && rings != 2 && rings != 4) || (korders != 1 && korders != 2))
        return set_error(SL_ERR_ARG, "fft tile %d x %d: rings must be 1, 2 or 4 and korders 1 or 2", rings, korders);
    if (ring_fft_cluster_size(p) != 1)
        return set_error(SL_ERR_UNSUPPORTED, "nphi=%d: the ring FFT runs on clusters", p->nphi);
    int dev_smem = 0;
    cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
    const size_t need = ring_fft_ip_smem(p, rings, korders);
    if (need > (size_t)kFftSmemMax || (dev_smem > 0 && need > (size_t)dev_smem))
        return set_error(SL_ERR_UNSUPPORTED, "fft tile %d x %d needs %zu bytes of shared memory", rings, korders,
                         need);
    p->fft_rg = rings;
    p->fft_kg = korders;
    return SL_OK;
}

sl_status sl_plan_set_contraction_pairs(sl_plan *p, int pairs) {
    sl_status st = enter(p);
    if (st != SL_OK) return st;
    if (pairs != 0 && pairs != 2 && pairs != 4 && pairs != 8)
        return set_error(SL_ERR_ARG, "contraction pairs %d: 0 (automatic), 2, 4 or 8", pairs);
    if (p->precision != SL_FP32 && pairs != 0)
        return set_error(SL_ERR_UNSUPPORTED, "contraction pairs: only SL_FP32 plans have the choice");
    p->lc_ppt = pairs;
    return SL_OK;
}

sl_status sl_plan_set_stream(sl_plan *p, void *stream) {
    sl_status st = enter(p);
    if (st != SL_OK) return st;
    cudaStreamSynchronize(p->stream);
    p->stream = (cudaStream_t)stream;
    return SL_OK;
}

sl_status sl_plan_sync(sl_plan *p) {
    sl_status st = enter(p);
    if (st != SL_OK) return st;
    if ((st = cuda_check(cudaStreamSynchronize(p->stream), "stream synchronize")) != SL_OK) return st;
    if (p->d_err) {
        int flag = 0;
        if ((st = cuda_check(cudaMemcpy(&flag, p->d_err, sizeof(int), cudaMemcpyDeviceToHost), "error flag")) != SL_OK)
            return st;
        if (flag) {
            cudaMemset(p->d_err, 0, sizeof(int));
            return set_error(SL_ERR_TIMEOUT, "a bounded wait inside a kernel expired (FP32 interpolation or "
                                             "tensor-core contraction)");
        }
    }
    return SL_OK;
}

sl_status sl_plan_selftest_timeout(sl_plan *p) {
    sl_status st = enter(p);
    if (st != SL_OK) return st;
    if (!p->d_err) {
        if ((st = dalloc_t(p, &p->d_err, 1, "error flag")) != SL_OK) return st;
        if ((st = cuda_check(cudaMemset(p->d_err, 0, sizeof(int)), "error flag")) != SL_OK) return st;
    }
    return launch_wait_probe(p, p->d_err);
}

sl_status synth_spin_maps_multi(sl_plan *p, int nsky, const double *sky, const double *beam, void *maps) {
    sl_status st = enter(p);
    if (st != SL_OK) return st;
    if (!plan_fp32(p->precision))
        return set_error(SL_ERR_UNSUPPORTED, "synth_spin_maps_multi: FP32 plans only (the tensor-core path)");
    if (nsky < 1) return set_error(SL_ERR_ARG, "synth_spin_maps_multi: nsky=%d < 1", nsky);
    if (nsky > 65535)   // the ring FFT runs one grid row per sky
        return set_error(SL_ERR_UNSUPPORTED, "synth_spin_maps_multi: nsky=%d > 65535", nsky);
    if (!sky || !beam || !maps) return set_error(SL_ERR_ARG, "synth_spin_maps_multi: NULL buffer");
    if (nsky > p->msky_cap) {
        if (p->batch_refs > 0) return set_error(SL_ERR_ARG, "synth_spin_maps_multi: the plan is held by a batch graph");
        cudaStreamSynchronize(p->stream);
        const int64_t gsky = (int64_t)(p->K + 1) * p->R * (2 * p->L + 1);
        if (p->msky_cap > 0)
            p->bytes_held -= (int64_t)p->msky_cap * (int64_t)sizeof(float2) * (p->ncomp * sky_row_stride(p->nalm) + gsky);
        dfree(p->d_skym32);
        dfree(p->d_Gm);
        p->d_skym32 = nullptr;
        p->d_Gm = nullptr;
        p->msky_cap = 0;
        if ((st = dalloc_t(p, &p->d_skym32, (size_t)nsky * p->ncomp * sky_row_stride(p->nalm), "FP32 skies")) != SL_OK)
            return st;
        if ((st = dalloc_t(p, &p->d_Gm, (size_t)nsky * gsky, "multi-sky G")) != SL_OK) return st;
        p->msky_cap = nsky;
    }
    if (!p->d_err) {
        if ((st = dalloc_t(p, &p->d_err, 1, "error flag")) != SL_OK) return st;
        if ((st = cuda_check(cudaMemset(p->d_err, 0, sizeof(int)), "error flag")) != SL_OK) return st;
    }
    if ((st = launch_lcontract_mma(p, nsky, sky, beam, p->d_skym32, p->d_Gm, p->d_err)) != SL_OK) return st;
    return launch_ringfft_synth_from(p, p->d_Gm, nsky, maps);
}

// ------------------------------------------------------------------ orbital dipole
static sl_status orb_scratch(sl_plan *p, size_t bytes) {
    if (bytes <= p->orb_bytes) return SL_OK;
    cudaStreamSynchronize(p->stream);
    if (p->d_orb) {
        dfree(p->d_orb);
        p->bytes_held -= (int64_t)p->orb_bytes;
    }
    p->d_orb = nullptr;
    p->orb_bytes = 0;
    sl_status st = dalloc(p, (void **)&p->d_orb, bytes, "orbital dipole scratch");
    if (st == SL_OK) p->orb_bytes = bytes;
    return st;
}

constexpr size_t kOrbS = 16;   // doubles reserved for the moments at the start of the scratch

sl_status sl_orbital_moments(sl_plan *p, const double *beam, double *S) {
    sl_status st = enter(p);
    if (st != SL_OK) return st;
    if (!beam || !S) return set_error(SL_ERR_ARG, "sl_orbital_moments: NULL buffer");
    if ((st = orb_scratch(p, kOrbS * sizeof(double))) != SL_OK) return st;
    if ((st = launch_orb_moments(p, beam, p->d_orb)) != SL_OK) return st;
    if ((st = cuda_check(cudaMemcpyAsync(S, p->d_orb, 9 * sizeof(double), cudaMemcpyDeviceToHost, p->stream),
                         "moments copy")) != SL_OK)
        return st;
    return cuda_check(cudaStreamSynchronize(p->stream), "stream synchronize");
}

sl_status orbital_dipole_tod(sl_plan *p, const double *beam, double T0, double q, const double *theta,
                             const double *phi, const double *psi, int64_t n, const int64_t *period_start,
                             const double *beta, int64_t nper, int subsample, double *tod, int accumulate) {
    sl_status st = enter(p);
    if (st != SL_OK) return st;
    if (n < 0) return set_error(SL_ERR_ARG, "orbital_dipole_tod: n=%lld < 0", (long long)n);
    if (subsample < 1 || subsample > (1 << 16))
        return set_error(SL_ERR_ARG, "orbital_dipole_tod: subsample=%d outside [1, 65536]", subsample);
    if (!std::isfinite(T0) || !std::isfinite(q)) return set_error(SL_ERR_ARG, "orbital_dipole_tod: T0, q not finite");
    if (n == 0) return SL_OK;
    if (!beam || !theta || !phi || !psi || !tod || !period_start || !beta)
        return set_error(SL_ERR_ARG, "orbital_dipole_tod: NULL buffer");
    if (nper < 1 || period_start[0] != 0 || period_start[nper] != n)
        return set_error(SL_ERR_ARG, "orbital_dipole_tod: period_start must run from 0 to n over nper >= 1 periods");
    // the pinned staging buffer is reused: wait until the previous upload has left it
    if (p->orb_ev && (st = cuda_check(cudaEventSynchronize(p->orb_ev), "orbital staging")) != SL_OK) return st;
    // host tables: [start | noff] as int64, then beta [nper][3], the elimination
    // pivots c_j = 1 / (4 - c_{j-1}) (c_0 = 0) and the spline weights of the
    // positions r = 0 .. s between two nodes (B = r/s, A = 1 - B)
    constexpr int kPiv = 40;
    const size_t nw = 4 * ((size_t)subsample + 1);
    // layout [weights | pivots | start | noff | beta]: the weights (read as 32-byte
    // vectors) first, at a 32-byte aligned offset of the scratch
    const size_t tab_bytes = (nw + kPiv + 2 * (size_t)(nper + 1) + 3 * (size_t)nper) * sizeof(int64_t);
    if (tab_bytes > p->h_orb_bytes) {
        if (p->h_orb) cudaFreeHost(p->h_orb);
        p->h_orb = nullptr;
        p->h_orb_bytes = 0;
        if (cudaHostAlloc(&p->h_orb, tab_bytes, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            p->h_orb = nullptr;
            return set_error(SL_ERR_NOMEM, "orbital_dipole_tod: pinned staging of %zu bytes", tab_bytes);
        }
        p->h_orb_bytes = tab_bytes;
    }
    if (!p->orb_ev && (st = cuda_check(cudaEventCreateWithFlags(&p->orb_ev, cudaEventDisableTiming),
                                       "orbital event")) != SL_OK)
        return st;
    double *wt = reinterpret_cast<double *>(p->h_orb), *piv = wt + nw;
    int64_t *start = reinterpret_cast<int64_t *>(piv + kPiv), *noff = start + (nper + 1);
    double *bet = reinterpret_cast<double *>(noff + (nper + 1));
    piv[0] = 0.0;
    for (int j = 1; j < kPiv; ++j) piv[j] = 1.0 / (4.0 - piv[j - 1]);
    const double sd = (double)subsample, h2 = sd * sd / 6.0;
    for (int r = 0; r <= subsample; ++r) {
        const double B = (double)r / sd, A = 1.0 - B;
        wt[4 * r + 0] = A;
        wt[4 * r + 1] = B;
        wt[4 * r + 2] = (A * A * A - A) * h2;
        wt[4 * r + 3] = (B * B * B - B) * h2;
    }
    noff[0] = 0;
    for (int64_t k = 0; k < nper; ++k) {
        const int64_t np = period_start[k + 1] - period_start[k];
        if (np < 0) return set_error(SL_ERR_ARG, "orbital_dipole_tod: period_start decreases at period %lld", (long long)k);
        if (np >= ((int64_t)1 << 31))
            return set_error(SL_ERR_ARG, "orbital_dipole_tod: period %lld has 2^31 samples or more", (long long)k);
        start[k] = period_start[k];
        noff[k + 1] = noff[k] + (subsample > 1 && np > 0 ? (np - 1) / subsample + 1 : 0);
        for (int c = 0; c < 3; ++c) {
            bet[3 * k + c] = beta[3 * k + c];
            if (!std::isfinite(beta[3 * k + c])) return set_error(SL_ERR_ARG, "orbital_dipole_tod: beta not finite");
        }
    }
    start[nper] = n;
    const int64_t nnodes = noff[nper];
    const size_t need = kOrbS * sizeof(double) + tab_bytes + 2 * (size_t)nnodes * sizeof(double);
    if ((st = orb_scratch(p, need)) != SL_OK) return st;
    char *base = reinterpret_cast<char *>(p->d_orb);
    int64_t *d_tab = reinterpret_cast<int64_t *>(base + kOrbS * sizeof(double));
    double *d_nodes = reinterpret_cast<double *>(base + kOrbS * sizeof(double) + tab_bytes);
    if ((st = cuda_check(cudaMemcpyAsync(d_tab, p->h_orb, tab_bytes, cudaMemcpyHostToDevice, p->stream),
                         "orbital tables")) != SL_OK)
        return st;
    if ((st = cuda_check(cudaEventRecord(p->orb_ev, p->stream), "orbital event")) != SL_OK) return st;
    if ((st = launch_orb_moments(p, beam, p->d_orb)) != SL_OK) return st;
    OrbLaunch o;
    o.theta = theta;
    o.phi = phi;
    o.psi = psi;
    o.w = reinterpret_cast<const double *>(d_tab);
    o.piv = o.w + nw;
    o.start = d_tab + nw + kPiv;
    o.noff = o.start + (nper + 1);
    o.beta = reinterpret_cast<const double *>(o.noff + (nper + 1));
    o.S = p->d_orb;
    o.T0 = T0;
    o.q = q;
    o.n = n;
    o.nper = nper;
    o.nnodes = nnodes;
    o.s = subsample;
    o.y = d_nodes;
    o.M2 = d_nodes + nnodes;
    o.tod = tod;
    o.accumulate = accumulate != 0;
    return launch_orbital(p, o);
}

// ------------------------------------------------------------------ psi-grid variant
static sl_status check_npsi(const sl_plan *p, int npsi, const char *who) {
    if (npsi < 2 * p->K + 2 || npsi < p->p || (npsi & 1) || npsi > 8192)
        return set_error(SL_ERR_ARG, "%s: npsi=%d must be even, >= 2 kmax + 2 = %d, >= the interpolation order "
                                     "and <= 8192", who, npsi, 2 * p->K + 2);
    if ((int64_t)p->R * p->nphi * npsi >= ((int64_t)1 << 31))
        return set_error(SL_ERR_UNSUPPORTED, "%s: nrings * nphi * npsi >= 2^31", who);
    if (psi_cube_smem_bytes(p, npsi) > (size_t)kSmemOptin)
        return set_error(SL_ERR_UNSUPPORTED, "%s: npsi=%d too large for the phase table in shared memory", who, npsi);
    return SL_OK;
}

sl_status synth_psi_cube(sl_plan *p, const void *maps, int npsi, void *cube_psi) {
    sl_status st = enter(p);
    if (st != SL_OK) return st;
    if (!maps || !cube_psi) return set_error(SL_ERR_ARG, "synth_psi_cube: NULL buffer");
    if ((st = check_npsi(p, npsi, "synth_psi_cube")) != SL_OK) return st;
    const bool wide = plan_wide(p->precision);
    if (p->psitab_n != npsi) {
        if (p->batch_refs > 0) return set_error(SL_ERR_ARG, "synth_psi_cube: the plan is held by a batch graph");
        cudaStreamSynchronize(p->stream);
        const int K1 = p->K + 1;
        const size_t elem = wide ? sizeof(double2) : sizeof(float2);
        if (p->d_psitab) {
            dfree(p->d_psitab);
            p->bytes_held -= (int64_t)K1 * p->psitab_n * (int64_t)elem;
        }
        p->d_psitab = nullptr;
        p->psitab_n = 0;
        if ((st = dalloc(p, &p->d_psitab, (size_t)K1 * npsi * elem, "psi phase table")) != SL_OK) return st;
        // [k][n]: (w_k cos(2 pi k n / npsi), -w_k sin(2 pi k n / npsi)), w_0 = 1, w_k = 2; exact integer phase
        std::vector<double> t64(2 * (size_t)K1 * npsi);
        const long double two_pi = 6.283185307179586476925286766559L;
        for (int k = 0; k < K1; ++k)
            for (int n = 0; n < npsi; ++n) {
                const long double a = two_pi * (long double)(((int64_t)k * n) % npsi) / (long double)npsi;
                const long double w = k == 0 ? 1.0L : 2.0L;
                t64[2 * ((size_t)k * npsi + n)] = (double)(w * cosl(a));
                t64[2 * ((size_t)k * npsi + n) + 1] = (double)(-w * sinl(a));
            }
        if (wide) {
            st = cuda_check(cudaMemcpy(p->d_psitab, t64.data(), t64.size() * sizeof(double), cudaMemcpyHostToDevice),
                            "psi table upload");
        } else {
            std::vector<float> t32(t64.size());
            for (size_t i = 0; i < t64.size(); ++i) t32[i] = (float)t64[i];
            st = cuda_check(cudaMemcpy(p->d_psitab, t32.data(), t32.size() * sizeof(float), cudaMemcpyHostToDevice),
                            "psi table upload");
        }
        if (st != SL_OK) return st;
        p->psitab_n = npsi;
    }
    return launch_psi_cube(p, maps, npsi, p->d_psitab, cube_psi);
}

sl_status interp_tod_psi(sl_plan *p, const void *cube_psi, int npsi, const double *theta, const double *phi,
                         const double *psi, int64_t n, double *tod) {
    sl_status st = enter(p);
    if (st != SL_OK) return st;
    if ((st = check_ptg(theta, phi, psi, n, tod, "interp_tod_psi")) != SL_OK) return st;
    if (!cube_psi) return set_error(SL_ERR_ARG, "interp_tod_psi: cube_psi is NULL");
    if ((st = check_npsi(p, npsi, "interp_tod_psi")) != SL_OK) return st;
    if (n == 0) return SL_OK;
    if ((st = ensure_sort_capacity(p, n)) != SL_OK) return st;
    SortBufs b = p->sort;
    // FP32 plans: tile-staged from shared memory when the tile's npsi values fit
    if (plan_fp32(p->precision) && interp_psi_tiled_smem(p, npsi) <= kSmemOptin) {
        if ((st = launch_sort_into(p, b, theta, phi, psi, n, 1, 0, 1)) != SL_OK) return st;
        return launch_interp_psi_tiled(p, b, cube_psi, npsi, n, tod);
    }
    b.chunk_off = nullptr;
    if ((st = launch_sort_into(p, b, theta, phi, psi, n, 1, 1, 0)) != SL_OK) return st;
    return launch_interp_psi(p, b, cube_psi, npsi, psi, n, tod);
}

unsigned sl_debug_check_status(void) {
    // every unit's word is read (and cleared); the first nonzero one is reported
    const unsigned w[6] = {chk_sort(), chk_interp(), chk_interp_df(), chk_psigrid(), chk_orbital(), chk_fft()};
    for (unsigned v : w)
        if (v) return v;
    return 0u;
}

sl_status sl_plan_enable_timing(sl_plan *p, int enable) {
    sl_status st = enter(p);
    if (st != SL_OK) return st;
    timing_flush(p);
    p->timing = enable != 0;
    return SL_OK;
}

sl_status sl_plan_kernel_stats(sl_plan *p, sl_kernel_stat *out, int max, int *count, int reset) {
    sl_status st = enter(p);
    if (st != SL_OK) return st;
    timing_flush(p);
    int n = (int)p->timers.size();
    if (count) *count = n;
    for (int i = 0; i < n && i < max && out; ++i) {
        snprintf(out[i].name, sizeof(out[i].name), "%s", p->timers[i].name.c_str());
        out[i].launches = p->timers[i].launches;
        out[i].total_ms = p->timers[i].total_ms;
    }
    if (reset) p->timers.clear();
    return cuda_check(cudaGetLastError(), "timing");
}

}  // extern "C"
