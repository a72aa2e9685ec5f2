// sl_internal.cuh -- plan layout, small device helpers and kernel launch
// declarations shared by the translation units of libsidelobe.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sidelobe.h"

namespace sl {

// ---------------------------------------------------------------- constants
constexpr int kMaxK = 128;       // beam azimuthal band limit supported
// ring FFT length held in shared memory: two double-complex buffers of nphi
// (the FP64 synthesis and every plan's adjoint DFT) within 227 KB
// longest ring: the binning's fixed-point phi scale round(nphi / (2 pi) 2^52) fits 64 bits
// up to here; rings longer than one CTA's shared memory use a cluster FFT
constexpr int kMaxNphi = 16384;
constexpr int kFftSmemMax = 232448;    // dynamic shared memory per CTA (227 KB)
constexpr int kMaxRadices = 16;

// Scaled FP64 Wigner values: value = mantissa * 2^(600 * e), e <= 0; a value
// with e < 0 is below 2^-300 and contributes nothing.
constexpr double kScaleUp = 0x1p600;
constexpr double kScaleDn = 0x1p-600;
constexpr double kScaleThr = 0x1p300;
constexpr double kScaleLow = 0x1p-300;
// FP32 recurrences use value = mantissa * 2^(64 e), rescaled above 2^32.
constexpr float kScaleDn32 = 0x1p-64f;
constexpr float kScaleThr32 = 0x1p32f;

// Sort tiles: cells (base row i in [-1, R-1], base column j) grouped into
// tiles of kTileRows x tile_cols cells.
constexpr int kTileRows = 4;
// Work item of the tile-staged kernels: at most this many sorted samples of one tile.
constexpr int kWorkChunk = 2048;

// SL_FP32 and SL_TF32X3 plans share every FP32 layout; SL_FP64 and SL_DF64
// plans share every FP64 layout (G, cube, records, tables).
inline bool plan_fp32(int precision) { return precision == SL_FP32 || precision == SL_TF32X3; }
inline bool plan_wide(int precision) { return !plan_fp32(precision); }

// ---------------------------------------------------------------- geometry
// Everything the interpolation kernels need, passed by value.
struct InterpGeom {
    int R, nphi, K, p, half;      // half = p/2 ghost rows per pole
    const double *ring_ext;       // [R + 2 half]: theta of rows -half .. R+half-1
    const long long *ring_fix;    // the same colatitudes in fixed point, round(theta 2^60)
    const double *wden;           // [(R+1) * p]: 1 / prod_{b!=a}(theta_a - theta_b) per base row
    const int *lut;               // [nlut]: base row for theta bin
    int nlut;
    double lut_scale;             // nlut / pi
    float lut_scale_f;            // the same, in float
    double phi_scale;             // nphi / (2 pi)
    unsigned long long phi_fix;   // round(nphi / (2 pi) 2^52)
    int tile_cols, ntr, ntc;      // tile grid: ntr = ceil((R+1)/kTileRows), ntc = ceil(nphi/tile_cols)
    const double *offs64;         // [(R+1) * p]: theta(i0+a) - theta(i0), i0 = i - p/2 + 1, per base row i
    const float *rowtab32;        // [(R+1) * 2p]: the same offsets, then wden, in float
    const float2 *rowtab_df;      // [(R+1) * 2p]: the same, as double-float (hi, lo)
};

// Bounds-checked builds (-DSL_CHECKED, the variant _build.build(checked=True) makes):
// SL_GUARD(cond, site) is true in ordinary builds (no code); in checked builds it
// evaluates cond and, when it fails, records the site in this translation unit's
// status word and skips the access it guards.  The status words of all units are
// read by sl_debug_check_status.
#ifdef SL_CHECKED
static __device__ unsigned sl_chk_word;
__device__ __forceinline__ bool sl_guard(bool ok, unsigned site) {
    if (!ok) atomicCAS(&sl_chk_word, 0u, site);
    return ok;
}
#define SL_GUARD(cond, site) (::sl::sl_guard((cond), (site)))
#define SL_CHECK_READER(name)                                                  \
    unsigned name() {                                                          \
        unsigned v = 0;                                                        \
        cudaMemcpyFromSymbol(&v, sl_chk_word, sizeof(v));                      \
        const unsigned z = 0;                                                  \
        cudaMemcpyToSymbol(sl_chk_word, &z, sizeof(z));                        \
        return v;                                                              \
    }
#else
#define SL_GUARD(cond, site) (true)
#define SL_CHECK_READER(name) \
    unsigned name() { return 0u; }
#endif
// per-unit readers (each translation unit with guards defines its own)
unsigned chk_sort();
unsigned chk_interp();
unsigned chk_interp_df();
unsigned chk_psigrid();
unsigned chk_orbital();
unsigned chk_fft();

// p-point Lagrange weights (separable interpolation, any even p).  theta:
// nodes at offsets o[a] from the first stencil row (o[0] = 0), 1/prod(o_a - o_b)
// in wd; d0 = theta - theta(first row).  phi: uniform nodes x_b = b - p/2 + 1
// around the base column, f the fraction in [0, 1).  Products of all but one
// factor through prefix and suffix products.
template <int P, typename T>
__device__ __forceinline__ void lagrange_theta(T d0, const T *o, const T *wd, T wt[P]) {
    T d[P], pre[P + 1], suf[P + 1];
#pragma unroll
    for (int a = 0; a < P; ++a) d[a] = (a == 0) ? d0 : d0 - o[a];
    pre[0] = T(1);
    suf[P] = T(1);
#pragma unroll
    for (int a = 0; a < P; ++a) pre[a + 1] = pre[a] * d[a];
#pragma unroll
    for (int a = P - 1; a >= 0; --a) suf[a] = suf[a + 1] * d[a];
#pragma unroll
    for (int a = 0; a < P; ++a) wt[a] = wd[a] * (pre[a] * suf[a + 1]);
}

// 1 / prod_{c != b} (b - c) for uniform nodes: (-1)^(P-1-b) / (b! (P-1-b)!).
template <int P>
__host__ __device__ constexpr double uniform_inv_den(int b) {
    double f = 1.0;
    for (int c = 0; c < P; ++c)
        if (c != b) f *= (double)(b - c);
    return 1.0 / f;
}

template <int P, typename T>
__device__ __forceinline__ void lagrange_phi(T f, T wp[P]) {
    T d[P], pre[P + 1], suf[P + 1];
#pragma unroll
    for (int b = 0; b < P; ++b) d[b] = f - T(b - P / 2 + 1);
    pre[0] = T(1);
    suf[P] = T(1);
#pragma unroll
    for (int b = 0; b < P; ++b) pre[b + 1] = pre[b] * d[b];
#pragma unroll
    for (int b = P - 1; b >= 0; --b) suf[b] = suf[b + 1] * d[b];
#pragma unroll
    for (int b = 0; b < P; ++b) wp[b] = (pre[b] * suf[b + 1]) * T(uniform_inv_den<P>(b));
}

// p-point weights of a sample: theta rows from the record and the plan's row
// table, phi nodes -p/2+1 .. p/2.
template <int P>
__device__ __forceinline__ void weights64(const InterpGeom &g, int i, double d0, double f, double wt[P],
                                          double wp[P]) {
    double o[P], wd[P];
#pragma unroll
    for (int a = 0; a < P; ++a) {
        o[a] = __ldg(g.offs64 + (size_t)(i + 1) * P + a);
        wd[a] = __ldg(g.wden + (size_t)(i + 1) * P + a);
    }
    lagrange_theta<P>(d0, o, wd, wt);
    lagrange_phi<P>(f, wp);
}

// Element offsets of the stencil's rows (ring * nphi * K1) and columns (col * K1)
// -- a node is row + column -- and the mask of ghost rows (beyond a pole: the
// ring at phi + pi).
template <int P>
__device__ __forceinline__ unsigned stencil_offsets(const InterpGeom &g, int i, int j, int roff[P], int coff[P],
                                                    int coff_g[P]) {
    const int K1 = g.K + 1;
    unsigned ghost = 0;
#pragma unroll
    for (int a = 0; a < P; ++a) {
        const int row = i - P / 2 + 1 + a;
        int ring = row;
        if (row < 0) { ring = -1 - row; ghost |= 1u << a; }
        else if (row >= g.R) { ring = 2 * g.R - 1 - row; ghost |= 1u << a; }
        roff[a] = ring * g.nphi * K1;
    }
#pragma unroll
    for (int b = 0; b < P; ++b) {
        int col = j - P / 2 + 1 + b;
        col = (col < 0) ? col + g.nphi : (col >= g.nphi ? col - g.nphi : col);
        coff[b] = col * K1;
        int cg = col + g.nphi / 2;
        cg = (cg >= g.nphi) ? cg - g.nphi : cg;
        coff_g[b] = cg * K1;
    }
    return ghost;
}

// Work item v -> its tile: the last t with chunk_off[t] <= v.
__device__ __forceinline__ int find_tile(const unsigned *chunk_off, int ntiles, unsigned v) {
    int lo = 0, hi = ntiles - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (chunk_off[mid] <= v) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Per-sample stencil record written by the binning kernel: the colatitude
// offset from the stencil's first row, the phi fraction in [0, 1), and the
// cell ((i+1) << 16) | j; FP32 plans also keep psi reduced to [-pi, pi].
struct StencilRec64 {
    double dth, fph;
    unsigned cell, pad;
};
struct __align__(16) StencilRec32 {
    float dth, fph, psr;
    unsigned cell;
};

// Arguments of the tile-staged FP32 interpolation of one plan's sorted pointings.
struct TiledArgs {
    InterpGeom g;
    const float2 *maps;
    const StencilRec32 *rec;
    const unsigned *perm, *start, *chunk_off;
    int ntiles, ncell;
    double *tod;
};

// Device buffers of one pointing sort.
struct SortBufs {
    unsigned *keys;       // [n]
    unsigned *perm;       // [n + 4]: sorted position -> sample (the tail pads 16-byte bulk copies)
    void *rec;            // [n] StencilRec64 or StencilRec32, by sample
    unsigned *hist;       // [nkeys + 1]: key counts, then first position of each key
    unsigned *cursor;     // [nkeys]
    unsigned *bsum;       // [nkeys / 4096 + 2]
    unsigned *chunk_off;  // [ntiles + 1]
};

// Rescaled l-recurrence coefficients per (k, m, l), stored at
// [k][m(2L+1-m)/2 + l] (the sky's packing): y_{l+1} = (a x -+ b) y_l - y_{l-1},
// d_l = c y_l.  FP32 plans keep c'+- = a -+ b - 2 for the difference form.
struct __align__(32) RTab64 {
    double a, b, c, unused;
};
struct __align__(16) RTab32 {
    float a, cp, cm, c;
};

struct KernelTimer {
    std::string name;
    int64_t launches = 0;
    double total_ms = 0;
};

}  // namespace sl

struct sl_plan {
    int L, K, ncomp, R, nphi, p, precision, device;
    cudaStream_t stream;
    int npairs;            // ceil(R/2): north rings (equator ring pairs with itself)
    int64_t nalm;

    // geometry (device)
    double *d_ring_theta = nullptr;   // [R]
    double *d_xr = nullptr;           // [npairs] cos(theta) of north rings
    float *d_y32 = nullptr;           // [npairs] 1 - cos(theta) = 2 sin^2(theta/2), FP32
    double *d_ring_ext = nullptr;
    long long *d_ring_fix = nullptr;
    double *d_wden = nullptr;
    double *d_offs64 = nullptr;
    float *d_rowtab32 = nullptr;
    float2 *d_rowtab_df = nullptr;
    int *d_lut = nullptr;
    int nlut = 0;
    sl::InterpGeom geom;

    // seeds: [K+1][L+1][npairs] (mantissa for +k, -k) and exponents
    double2 *d_seed = nullptr;
    int2 *d_seed_e = nullptr;
    // rescaled recurrence tables [K+1][nalm] (one of the two, by precision)
    sl::RTab64 *d_tab64 = nullptr;
    sl::RTab32 *d_tab32 = nullptr;
    // per-call start states [K+1][L+1][2 signs][npairs]: first significant l and
    // the recurrence state there (FP64 plans: st64, FP32 plans: st32)
    int *d_ls = nullptr;
    double2 *d_st64 = nullptr;
    float2 *d_st32 = nullptr;
    int64_t lsteps = 0;               // recurrence steps per synth call
    // FP64 start states of the adjoint contraction (alias the above in FP64 plans)
    int *d_ls_adj = nullptr;
    double2 *d_st64_adj = nullptr;
    // FP32 copies of sky and beam (FP32 plans)
    float2 *d_sky32 = nullptr;
    float2 *d_beam32 = nullptr;

    // ring FFT
    double2 *d_tw64 = nullptr;        // [nphi] e^{+2 pi i j / nphi}
    float2 *d_tw32 = nullptr;
    int *d_fftperm = nullptr;         // [nphi] FFT input q held by slot s (in-place ring FFT)
    int *d_fftpos = nullptr;          // [nphi] slot of FFT input q (its inverse)
    double2 *d_ptw64 = nullptr;       // [nphi] per-pass twiddles of the in-place ring FFT
    float2 *d_ptw32 = nullptr;
    int fft_rg = 0, fft_kg = 0;       // rings x k orders per in-place FFT CTA (0: default)
    int lc_ppt = 0;                   // ring pairs per thread of the FP32 contraction (0: automatic)
    int radices[sl::kMaxRadices];
    int nradix = 0;

    // scratch
    void *d_G = nullptr;              // [K+1][2L+1][R] complex, ring index fastest (precision of the plan)
    size_t G_bytes = 0;
    double2 *d_Gadj = nullptr;        // FP64 copy for FP32 plans (adjoint), else aliases d_G
    double2 *d_Fbar = nullptr;        // [R][nphi][K+1] adjoint cube
    double2 *d_Abar = nullptr;        // [K+1][2L+1][L+1]
    // pointing sort (fine cell keys; per-sample scratch grown on demand)
    int ntiles = 0;
    int64_t nkeys = 0;
    sl::SortBufs sort = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    int64_t sort_cap = 0;

    int64_t bytes_held = 0;
    // multi-sky builds (FP32 plans): FP32 skies, per-sky G, and the device flag of
    // the tensor-core kernel's bounded waits; grown on demand
    float2 *d_skym32 = nullptr;
    float2 *d_Gm = nullptr;
    int *d_err = nullptr;
    int msky_cap = 0;
    // orbital dipole (grown on demand): moments, period tables, spline nodes
    double *d_orb = nullptr;
    size_t orb_bytes = 0;
    // psi-grid variant: phase table [K+1][npsi] of the current npsi
    void *d_psitab = nullptr;
    int psitab_n = 0;
    void *h_orb = nullptr;              // pinned staging of the period tables
    size_t h_orb_bytes = 0;
    cudaEvent_t orb_ev = nullptr;       // recorded after the last table upload
    cudaStream_t side = nullptr;        // convolve_tod: the pointing sort's stream (created on first use)
    cudaEvent_t side_fork = nullptr, side_join = nullptr;
    // convolve_tod_host (created and grown on first use): device copies of the host
    // inputs (sky, beam, then the three pointing arrays of host_cap samples each),
    // the cube, the TOD, the upload and download streams and the per-piece events
    double *d_hin = nullptr;
    double *d_htod = nullptr;
    void *d_hmaps = nullptr;
    int64_t host_cap = -1;
    cudaStream_t up = nullptr, down = nullptr;
    cudaEvent_t h_arrived[64] = {}, h_done[64] = {};
    // number of captured batch graphs that hold pointers into this plan's
    // scratch: while > 0 nothing may be reallocated (the graphs would dangle)
    int batch_refs = 0;

    // timing
    bool timing = false;
    std::vector<sl::KernelTimer> timers;
    std::vector<cudaEvent_t> pending_ev;     // pairs (start, stop)
    std::vector<int> pending_idx;
};

namespace sl {

// status helpers (plan.cu)
sl_status set_error(sl_status st, const char *fmt, ...);
sl_status cuda_check(cudaError_t e, const char *what);

// Dynamic shared-memory cap of a kernel (plan.cu).  Raises the function's
// cap, once per device, to the device's opt-in maximum less the kernel's
// static shared memory, and checks that `sm` bytes fit under it.  The cap is
// never lowered to one plan's size: a CUDA graph captured earlier keeps its
// nodes' own (possibly larger) sizes, and a node launched again on its own
// (a profiler replaying graph nodes one by one) is checked against the
// function's current cap.
cudaError_t allow_dyn_smem_fn(const void *kern, size_t sm);
template <typename F>
inline cudaError_t allow_dyn_smem(F *kern, size_t sm) {
    return allow_dyn_smem_fn(reinterpret_cast<const void *>(kern), sm);
}

// timing (plan.cu): returns an index; call timing_end after the launch
int timing_begin(sl_plan *p, const char *name);
void timing_end(sl_plan *p, int idx);

// row stride (complex elements) of the FP32 sky copies: nalm rounded up to even, so that
// every row starts on 16 bytes (the tensor-core contraction loads them with TMA)
inline int64_t sky_row_stride(int64_t nalm) { return (nalm + 1) & ~(int64_t)1; }

// orbital dipole (k_orbital.cu): device pointers of one call
struct OrbLaunch {
    const double *theta, *phi, *psi;
    const int64_t *start, *noff;
    const double *beta, *S;
    const double *piv;       // elimination pivots c_1 .. c_39 (c_0 = 0), the last one the limit
    const double *w;         // [s][4] spline weights per position between nodes
    double T0, q;
    int64_t n, nper, nnodes;
    int s;
    double *y, *M2, *tod;
    int accumulate;
};
sl_status launch_orb_moments(sl_plan *p, const double *beam, double *S);
// psi-grid variant (k_psigrid.cu)
size_t psi_cube_smem_bytes(const sl_plan *p, int npsi);
sl_status launch_psi_cube(sl_plan *p, const void *maps, int npsi, const void *tab, void *out);
sl_status launch_interp_psi(sl_plan *p, const SortBufs &b, const void *cube, int npsi, const double *psi, int64_t n,
                            double *tod);
size_t interp_psi_tiled_smem(const sl_plan *p, int npsi);
sl_status launch_interp_psi_tiled(sl_plan *p, const SortBufs &b, const void *cube, int npsi, int64_t n, double *tod);
sl_status launch_orbital(sl_plan *p, const OrbLaunch &o);

// launchers (one per translation unit)
sl_status launch_seeds(sl_plan *p, const double *d_c2, const double *d_s2, const double *d_cs);
sl_status launch_rtab(sl_plan *p);
sl_status launch_advance(sl_plan *p, double thr, int *ls, double2 *st64, float2 *st32);
sl_status count_lsteps(sl_plan *p, int64_t *out);
sl_status launch_lcontract(sl_plan *p, const double *sky, const double *beam);
// Many detectors (batch.cu): work items of the persistent FP32 contraction.
constexpr int kMaxBatchDets = 32;
struct LcBatchItem {
    int det, block, ppt;
    float cost;
};
int lcontract_f32_ppt(int npairs);
// items grouped by ring pairs per thread (8, 4, 2), counts[g] per group
constexpr int kLcBatchGroups = 3;
sl_status lcontract_f32_batch_items(sl_plan *const *plans, int n, std::vector<LcBatchItem> &items,
                                    int counts[kLcBatchGroups]);
// the group of a plan's blocks (by its ring pairs per thread: 8, 4, 2)
int lcontract_f32_group(const sl_plan *p);
// one launch per nonempty group g on gstream[g], after `ready` (recorded on
// `stream` once the FP32 copies are made and counters[kLcBatchGroups] zeroed
// there), its end recorded in gdone[g]; the caller joins the group streams
sl_status launch_lcontract_f32_batch(cudaStream_t stream, const cudaStream_t *gstream, const cudaEvent_t *gdone,
                                     cudaEvent_t ready, sl_plan *const *plans, const double *const *sky,
                                     const double *const *beam, int n, const LcBatchItem *items,
                                     const int counts[kLcBatchGroups], unsigned *counters);
sl_status launch_ringfft_synth(sl_plan *p, void *maps);
// nsky cubes from nsky consecutive G blocks (gridDim.y = nsky)
sl_status launch_ringfft_synth_from(sl_plan *p, const void *G, int nsky, void *maps);
// CTAs per cluster of the ring FFT (1: one CTA per ring; 0: unsupported nphi)
int ring_fft_cluster_size(const sl_plan *p);
// rings x k orders per CTA of the in-place ring FFT the plan uses (0, 0 for the cluster form)
void ring_fft_tile(const sl_plan *p, int *rg, int *kg);
// shared memory of the in-place ring FFT for RG rings x KG k orders
size_t ring_fft_ip_smem(const sl_plan *p, int rg, int kg);
// Multi-sky spin Legendre step on the tensor cores (k_multisky.cu), FP32 plans.
sl_status launch_lcontract_mma(sl_plan *p, int nsky, const double *sky, const double *beam, float2 *sky32,
                               float2 *G, int *err);
int lcontract_mma_group(int nsky);
sl_status launch_wait_probe(sl_plan *p, int *err);
// Sort of n pointings into b: fine (cell) or coarse (tile) keys, FP64 or FP32
// stencil records; with_chunks also builds the adjoint's per-tile work items.
int64_t sort_nkeys(const sl_plan *p, int fine);
int64_t sort_nbsum(int64_t nkeys);
sl_status launch_sort_into(sl_plan *p, const SortBufs &b, const double *theta, const double *phi,
                           const double *psi, int64_t n, int fine, int rec64, int with_chunks);
// Forward interpolation over a sort (records in the plan's precision).  FP32
// plans use the tile-staged kernel when the sort built work items (chunk_off).
TiledArgs fine_tiled_args(const sl_plan *p, const SortBufs &b, const void *maps, double *tod);
sl_status launch_interp_f32_cells(cudaStream_t stream, int device, const TiledArgs *dets, int nd, int tc, int P,
                                  int kmax_max, unsigned *work, int *err);
sl_status launch_interp(sl_plan *p, const SortBufs &b, int fine, const void *maps, const double *psi, int64_t n,
                        double *tod);
size_t interp_f32_tiled_smem(const sl_plan *p);
// Dynamic shared memory of the two tile-staged kernels for tile width tc.
size_t interp_f32_tiled_smem_tc(const sl_plan *p, int tc);
size_t interp_f32_cells_smem_tc(const sl_plan *p, int tc);
size_t interp_adjoint_smem_tc(const sl_plan *p, int tc);
// Double-float interpolation (SL_DF64 plans; k_interp_df.cu), over a sort made
// with rec64 = 1 and with_chunks = 1.
sl_status launch_interp_df(sl_plan *p, const SortBufs &b, int fine, const void *maps, const double *psi, int64_t n,
                           double *tod);
size_t interp_df_tiled_smem_tc(const sl_plan *p, int tc);
sl_status launch_interp_adjoint_df(sl_plan *p, const SortBufs &b, int fine, const double *psi, const double *tod,
                                   double2 *fbar);
size_t interp_adjoint_df_smem_tc(const sl_plan *p, int tc);
// Adjoint scatter over a sort made with rec64 = 1, with_chunks = 1.
sl_status launch_interp_adjoint(sl_plan *p, const SortBufs &b, int fine, const double *psi, const double *tod,
                                int64_t n, double2 *fbar);
sl_status launch_ringdft_adjoint(sl_plan *p, const double2 *fbar);
sl_status launch_lcontract_adjoint(sl_plan *p);
sl_status launch_grad(sl_plan *p, const double *sky, const double *beam, double *sky_grad,
                      double *beam_grad, int accumulate);

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// ---- conversions on the integer pipes.  GB300 runs FP64 at 1/64 of FP32, and
// FP64 conversions and compares occupy that pipe; the binning kernel does
// these steps on the bit patterns instead (exact, except the rounding noted).

// double -> float, round half away from zero on the magnitude; values below
// the float normal range give +-0, above it +-inf (NaN stays NaN).
__device__ __forceinline__ float d2f_bits(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const unsigned long long t = b & 0x7fffffffffffffffull;
    if (t > 0x7ff0000000000000ull) return __int_as_float(0x7fc00000);           // NaN
    const long long fb = (long long)((t + (1ull << 28)) >> 29) - ((long long)(1023 - 127) << 23);
    if (fb < (1ll << 23)) return __int_as_float((int)sign);                     // underflow, 0
    if (fb >= (255ll << 23)) return __int_as_float((int)(sign | 0x7f800000u));  // overflow, inf
    return __int_as_float((int)(sign | (unsigned)fb));
}

// fr * 2^-sh (0 <= fr < 2^sh, sh <= 52) as a double (exact) and a float (truncated).
__device__ __forceinline__ double frac_bits_d(unsigned long long fr, int sh) {
    if (fr == 0) return 0.0;
    const int p = 63 - __clzll((long long)fr);                 // leading one, p < sh
    const unsigned long long m = (fr << (52 - p)) & ((1ull << 52) - 1);
    return __longlong_as_double((long long)(((unsigned long long)(p - sh + 1023) << 52) | m));
}
__device__ __forceinline__ float frac_bits_f(unsigned long long fr, int sh) {
    if (fr == 0) return 0.f;
    const int p = 63 - __clzll((long long)fr);
    if (p - sh + 127 <= 0) return 0.f;
    const unsigned long long m = (p >= 23) ? (fr >> (p - 23)) : (fr << (23 - p));
    return __int_as_float((int)(((unsigned)(p - sh + 127) << 23) | ((unsigned)m & 0x7fffffu)));
}

// Locate the base row i in [-1, R-1] of the interpolation stencil: the largest
// i with theta_ext(i) <= theta.  The look-up bin comes from a float copy of
// theta (the table keeps one row of margin); the final compares are exact:
// for non-negative doubles the bit patterns order like the values, a negative
// theta stays at row -1 and NaN ends on a valid row (the result is NaN).
__device__ __forceinline__ int locate_row(const InterpGeom &g, double theta) {
    int b = __float2int_rz(d2f_bits(theta) * g.lut_scale_f);
    b = min(max(b, 0), g.nlut - 1);
    int i = __ldg(g.lut + b);
    const long long tb = __double_as_longlong(theta);
    // ring_ext index of row r is r + half (rows >= 0 are positive colatitudes)
    while (i < g.R - 1 && __double_as_longlong(__ldg(g.ring_ext + i + 1 + g.half)) <= tb) ++i;
    return i;
}

// phi -> base column j in [0, nphi) and fraction u - j in [0, 1), u = phi nphi / (2 pi):
// one FP64 multiply; floor and fraction from the bits of u (exact).  phi outside
// [0, 2 pi) is first reduced in FP64.
__device__ __forceinline__ int locate_col_bits(const InterpGeom &g, double phi, unsigned long long &fr, int &sh) {
    double u = phi * g.phi_scale;
    const double n = (double)g.nphi;
    if (!(u >= 0.0 && u < n)) u -= n * floor(u * (1.0 / n));   // rare; also maps NaN to NaN
    const unsigned long long b = (unsigned long long)__double_as_longlong(u);
    const int e = (int)((b >> 52) & 0x7ff) - 1023;
    const unsigned long long M = (b & ((1ull << 52) - 1)) | (1ull << 52);   // u = M 2^(e-52)
    if (e > 30) { fr = 0; sh = 1; return 0; }          // NaN or out of range: column 0
    if (e < 0) {                                       // u < 1: j = 0, fraction u (exact)
        if (e < -126) { fr = 0; sh = 1; } else { fr = M; sh = 52 - e; }
        return 0;
    }
    sh = 52 - e;
    int j = (int)(M >> sh);
    fr = M & ((1ull << sh) - 1);
    if (j > g.nphi - 1) { j = g.nphi - 1; fr = (1ull << sh) - 1; }
    return j;
}

// ---- coordinate arithmetic on the integer pipes ---------------------------
// On this GPU the FP64 unit runs at 1/64 of the FP32 rate, so the per-sample
// conversions of the binning kernel are done in 64-bit fixed point instead.

// x 2^S truncated toward zero, if |x| < 2^(62-S) (else false: NaN, inf, too
// large).  Exact when the last mantissa bit of x is worth at least 2^-S.
template <int S>
__device__ __forceinline__ bool to_fix(double x, long long &v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff) - 1023;
    if (e > 61 - S) return false;
    const unsigned long long M = (b & ((1ull << 52) - 1)) | (1ull << 52);   // x = M 2^(e-52)
    const int sh = e + S - 52;
    const unsigned long long a = (sh >= 0) ? (M << sh) : (sh > -64 ? (M >> -sh) : 0ull);
    v = (b >> 63) ? -(long long)a : (long long)a;
    return true;
}

// v 2^-S rounded to the nearest double / float (|v| < 2^63).
template <int S>
__device__ __forceinline__ double fix_to_d(long long v) {
    if (v == 0) return 0.0;
    const unsigned long long sgn = (v < 0) ? (1ull << 63) : 0ull;
    const unsigned long long a = (v < 0) ? (unsigned long long)(-v) : (unsigned long long)v;
    const int p = 63 - __clzll((long long)a);
    const unsigned long long m = (p > 52) ? ((a + (1ull << (p - 53))) >> (p - 52)) : (a << (52 - p));
    // m in [2^52, 2^53]; a carry into 2^53 moves into the exponent field
    return __longlong_as_double(
        (long long)(sgn | ((((unsigned long long)(p - S + 1023)) << 52) + (m - (1ull << 52)))));
}
template <int S>
__device__ __forceinline__ float fix_to_f(long long v) {
    if (v == 0) return 0.f;
    const unsigned sgn = (v < 0) ? 0x80000000u : 0u;
    const unsigned long long a = (v < 0) ? (unsigned long long)(-v) : (unsigned long long)v;
    const int p = 63 - __clzll((long long)a);
    const int E = p - S + 127;
    if (E <= 0) return __int_as_float((int)sgn);     // below the normal range: 0
    const unsigned long long m = (p > 23) ? ((a + (1ull << (p - 24))) >> (p - 23)) : (a << (23 - p));
    return __int_as_float((int)(sgn | (((unsigned)E << 23) + (unsigned)(m - (1ull << 23)))));
}

// phi -> base column j in [0, nphi) and fraction fr 2^-53 in [0, 1): u = phi
// nphi / (2 pi) as the 128-bit product of phi's mantissa and phi_fix.  Falls
// back to locate_col_bits for |phi| < 2^-20, |phi| >= 16, NaN and inf.
__device__ __forceinline__ int locate_col_fix(const InterpGeom &g, double phi, unsigned long long &fr, int &sh) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(phi);
    const int e = (int)((b >> 52) & 0x7ff) - 1023;
    if (e < -20 || e > 3) return locate_col_bits(g, phi, fr, sh);
    const unsigned long long M = (b & ((1ull << 52) - 1)) | (1ull << 52);
    unsigned long long lo = M * g.phi_fix, hi = __umul64hi(M, g.phi_fix);
    if (b >> 63) {                       // negate the 128-bit product
        lo = ~lo + 1ull;
        hi = ~hi + (lo == 0ull ? 1ull : 0ull);
    }
    // u = (hi:lo) 2^(e-104): integer part hi >> t, fraction bits [t, t+64), t = 40 - e in [37, 60]
    const int t = 40 - e;
    long long j = (long long)hi >> t;
    fr = ((lo >> t) | (hi << (64 - t))) >> 11;
    sh = 53;
    if ((unsigned long long)j >= (unsigned long long)g.nphi) {
        j %= g.nphi;
        if (j < 0) j += g.nphi;
    }
    return (int)j;
}

// phi -> base column j and fraction f (double).
__device__ __forceinline__ int locate_col(const InterpGeom &g, double phi, double &f) {
    unsigned long long fr;
    int sh;
    const int j = locate_col_bits(g, phi, fr, sh);
    f = frac_bits_d(fr, sh);
    return j;
}

}  // namespace sl
