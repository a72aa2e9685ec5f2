// k_multisky.cu -- the spin "Legendre" step (Sect. 2.1, Eqs. c_m and S) for
// many skies that share one beam, as a tensor-core product:
//
//   G^(s)_k(r, m) = sum_l A^(s)_{k,lm} d^l_{mk}(theta_r),   s = 0 .. nsky-1.
//
// For fixed (m, k, sign of k) this is W[r, l] x V[l, n]: W holds the rescaled
// Wigner values y_l of 128 ring pairs (generated on the fly by the FP32
// recurrence of the single-sky kernel, difference form on 1 - cos theta),
// V holds, per sky, the four real columns of the two complex sums
// (c_l A+, (-1)^l c_l A- for +k; c_l A-, (-1)^l c_l A+ for -k, A+ = sum_X s
// conj(b), A- = sum_X conj(s) conj(b)).  With one sky V has 4 columns and the
// product is a matrix-vector product; with many skies it is a dense tile
// product and runs on tcgen05:
//
//   * CTA = (m, k, sign, 128 ring pairs, group of up to 32 skies), M = 128,
//     N = 4 x skies, K = l in chunks of 32;
//   * W and V are split into TF32 high and low parts and multiplied as
//     hi x hi + hi x lo + lo x hi (three MMAs, FP32 accumulation in tensor
//     memory): ~2^-21 relative per product, the accuracy of the FP32 path;
//   * W lives in tensor memory: four producer warps, the thread that owns ring
//     pair r runs its recurrence and writes its row (TMEM lane r) with
//     tcgen05.st, the chunk's coefficients broadcast through shared memory;
//     V lives in shared memory, K-major with the 128-byte swizzle, built by
//     four other producer warps from sky rows brought in by TMA tensor loads
//     and per-chunk beam factors; both double buffered, so that while the MMAs
//     of one chunk run the producers build the next chunk;
//   * 256 TMEM columns and 105 KB of shared memory per CTA at 32 skies (B
//     buffers 64 KB, staging 39 KB): two CTAs per SM;
//   * one thread issues the MMAs and commits them to an mbarrier per buffer;
//     every wait is bounded and sets an error flag (the CTA then stops,
//     waits for its MMAs with a bound and frees its tensor memory).
// The V producers bind the kernel (the MMA thread waits on them); with more
// than 16 skies each W warp, otherwise idle on the MMAs, also builds the second
// 4-sky unit of its V partner.  Their work per sky and l is four FMAs per component.
#include <algorithm>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "mbar.cuh"
#include "sl_internal.cuh"

namespace sl {

constexpr int kMsRows = 128;      // ring pairs per CTA (MMA M)
constexpr int kMsLC = 32;         // l per chunk
constexpr int kMsThreads = 288;   // 4 W-producer warps, 4 V-producer warps, 1 MMA warp

struct MsArgs {
    int L, K, ncomp, R, npairs, nrc;     // nrc: ring chunks of 128 pairs
    int nsky, nsg, ngroups;              // skies, skies per CTA (multiple of 4), groups
    int64_t nalm;
    const float2 *sky;                   // [nsky][ncomp][salm], FP32 copy (rows padded to an even length)
    int64_t salm;                        // sky row stride: nalm rounded up to even (16-byte rows)
    const float2 *beam;                  // [ncomp][K+1][L+1], FP32 copy
    const float *y32;                    // [npairs] 1 - cos theta
    const int *ls;                       // [K+1][L+1][2][npairs] first significant l
    const float2 *st32;                  // start states (y, D)
    const RTab32 *tab32;                 // [K+1][nalm] {a', c'+, c'-, c}
    float2 *G;                           // [nsky][K+1][R][2L+1]
    int64_t gsky;                        // elements of one sky's G
    int *err;
};

// Shared-memory operand descriptor: K-major, 128-byte swizzle (rows of 128 B,
// 16-byte chunk c of row r stored at chunk c ^ (r & 7), 8-row groups 1024 B apart).
__device__ __forceinline__ uint64_t ms_sdesc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3fff) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// Instruction descriptor: kind::tf32, D in F32, A and B TF32 and K-major.
__device__ __forceinline__ uint32_t ms_idesc(int m, int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
// float index of element (row, k) of a [rows][32] tile in that layout
__device__ __forceinline__ int ms_sw(int row, int k) { return row * 32 + ((((k >> 2) ^ (row & 7))) << 2) + (k & 3); }

// TF32 split: hi keeps the 19 bits the tensor core reads, lo = x - hi (exact)
__device__ __forceinline__ void tf32_split(float x, float &hi, float &lo) {
    hi = __uint_as_float(__float_as_uint(x) & 0xffffe000u);
    lo = x - hi;
}

__device__ __forceinline__ void ms_write_two(const MsArgs &a, float2 *G, int m, int k, int pair, int neg, float2 acc1,
                                             float2 acc2) {
    const int rn = pair, rs = a.R - 1 - pair;
    // G[k][L +- m][r]: consecutive rows (ring pairs) of the CTA write contiguous runs
    float2 *gp = G + ((int64_t)k * (2 * a.L + 1) + a.L + m) * a.R;
    float2 *gm = G + ((int64_t)k * (2 * a.L + 1) + a.L - m) * a.R;
    const bool modd = m & 1, kodd = k & 1;
    if (!neg) {
        gp[rn] = acc1;
        if (m > 0 && rs != rn) {
            if (modd != kodd) { acc2.x = -acc2.x; acc2.y = -acc2.y; }
            gm[rs] = acc2;
        }
    } else {
        if (m > 0) {
            if (kodd) { acc1.x = -acc1.x; acc1.y = -acc1.y; }
            gm[rn] = acc1;
        }
        if (rs != rn) {
            if (modd) { acc2.x = -acc2.x; acc2.y = -acc2.y; }
            gp[rs] = acc2;
        }
    }
}

// TMEM columns of one CTA: the accumulator D in [0, N), the W operand (TF32
// high and low parts, two buffers of 32 columns each) from column 128.
constexpr int kMsTmemCols = 256;
constexpr int kMsAcol = 128;
constexpr int kMsNB = 2;            // operand buffers (chunks in flight)
constexpr int kMsNS = 3;            // staging slots of the sky values per V warp (work units in flight)
constexpr int kMsBoxX = 68;         // floats per TMA row: 34 float2 = 32 l plus the alignment slack
constexpr int kMsStageF = 832;      // floats per staging slot: [4 skies][<= 3 components][68], 128-byte multiple

// Roles (warp-specialized; no CTA-wide barrier inside the chunk loop):
//   warps 0-3  W producers: thread = ring pair = TMEM lane; per chunk the 32
//              recurrence steps, TF32 split, tcgen05.st into A buffer b;
//              arrive on full_a[b]; with more than 16 skies W warp w then builds
//              the unit of skies 16 + 4w .. + 3 into B buffer b (staged by V
//              warp 4 + w, handed over through slot_free) and arrives on full_b[b];
//   warps 4-7  V producers: lane = l - c0, warp over skies; sky x beam
//              columns into the swizzled B buffer b; arrive on full_b[b];
//   warp 8     MMA issuer (lane 0): waits full_a[b] and full_b[b], issues the
//              12 MMAs of the chunk, commits them to empty[b];
// the producers wait on empty[b] before refilling buffer b.  After the last
// chunk the W warps wait for its commit and read the accumulator.
// One work unit of the sky x beam columns: 4 skies (staged rows at src, this lane's l)
// into rows 4 s + q of the K-major swizzled B buffer (Bh, Bl: TF32 high and low parts).
// With A+ = sum_X s conj(b) and A- = sum_X conj(s) conj(b), the four columns are
// c (p1.x, p1.y), (-1)^l c (p2.x, p2.y), (p1, p2) = (A+, A-) for +k and (A-, A+) for -k:
//   c p1 = (xa + ys, yx - xb),  c p2 = (xa - ys, -(yx + xb)),
// xa = sum s.x c b.x, xb = sum s.x c b.y, ys = sum s.y sigma c b.y, yx = sum s.y sigma c b.x
// (the factors b* carry c_l, sigma = sign of k and the m = 0 rule).
template <int NC>
__device__ __forceinline__ void ms_build_unit(const float *src, float *Bh, float *Bl, const float *bxc,
                                              const float *byc, const float *bxs, const float *bys, float par,
                                              const int (&swz_off)[2][4]) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        float xa = 0.f, xb = 0.f, ys = 0.f, yx = 0.f;
#pragma unroll
        for (int X = 0; X < NC; ++X) {
            const float2 s2 = *reinterpret_cast<const float2 *>(src + (t * NC + X) * kMsBoxX);
            xa = fmaf(s2.x, bxc[X], xa);
            xb = fmaf(s2.x, byc[X], xb);
            ys = fmaf(s2.y, bys[X], ys);
            yx = fmaf(s2.y, bxs[X], yx);
        }
        const float vv[4] = {xa + ys, yx - xb, par * (xa - ys), -par * (yx + xb)};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            // row 4 s + q; the group's first sky is a multiple of 4, so (row & 7) = 4 (t & 1) + q
            const int off = 128 * t + swz_off[t & 1][q];
            float h, lo;
            tf32_split(vv[q], h, lo);
            Bh[off] = h;
            Bl[off] = lo;
        }
    }
}

// this lane's float offset in row q of the 4 rows of one sky, for an even (h = 0) or odd
// (h = 1) sky of a multiple-of-4 group: the 16-byte chunk (lane / 4) of a 128-byte row
// sits at chunk (lane / 4) ^ (row & 7), and row & 7 = 4 h + q
__device__ __forceinline__ void ms_swz_offsets(int lane, int (&swz_off)[2][4]) {
    const int ch = lane >> 2, lo4 = lane & 3;
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int q = 0; q < 4; ++q) swz_off[h][q] = q * 32 + ((ch ^ (4 * h + q)) << 2) + lo4;
}

// 288 threads, two CTAs per SM: the 18 warps spread 5, 5, 4, 4 over the SM's four
// 16,384-register partitions, so at most 96 registers a thread.
// NC = T/E/B components per sky (1 or 3), a compile-time count so that the V
// producers' component loops unroll and the four skies of a unit interleave.
template <int NC>
__global__ void __launch_bounds__(kMsThreads, 2) k_lcontract_mma(const MsArgs a,
                                                                  const __grid_constant__ CUtensorMap tmap) {
    extern __shared__ unsigned char ms_raw[];
    __shared__ __align__(8) uint64_t full_a[kMsNB], full_b[kMsNB], empty[kMsNB];
    __shared__ __align__(8) uint64_t stg_bar[4][kMsNS];    // TMA arrivals of each V warp's staging slots
    __shared__ __align__(8) uint64_t slot_free[4][kMsNS];  // consumer of a helped V warp's slot has finished
    __shared__ uint32_t tmem_base;
    __shared__ int s_lmin, s_fail;
    __shared__ float2 wcoef[4][kMsLC];                      // per W warp: (a, c+ or c-) of the chunk's l
    volatile int *fail = &s_fail;   // set by any role whose bounded wait ran out

    int b = blockIdx.x;
    const int grp = b % a.ngroups;
    b /= a.ngroups;
    const int rc = b % a.nrc;
    b /= a.nrc;
    const int neg = b & 1;
    b >>= 1;
    const int k = b % (a.K + 1);
    const int m = b / (a.K + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = 4 * a.nsg;
    const int64_t moff = (int64_t)m * (2 * a.L + 1 - m) / 2;
    const RTab32 *tab = a.tab32 + (int64_t)k * a.nalm + moff;

    // V operand buffers in shared memory, 1024-byte aligned: per buffer B_hi, B_lo [N][32]
    const uint32_t raw = smem_u32(ms_raw);
    float *base = reinterpret_cast<float *>(ms_raw + ((1024u - (raw & 1023u)) & 1023u));
    const int bfl = N * kMsLC;

    // W threads' recurrences (threads 0..127 own the rows = TMEM lanes)
    const int pair = rc * kMsRows + tid;
    float y = 0.f, D = 0.f, yc = 0.f;
    int ls = a.L + 1;
    if (tid < kMsRows && pair < a.npairs) {
        const int64_t si = (((int64_t)k * (a.L + 1) + m) * 2 + neg) * a.npairs + pair;
        ls = a.ls[si];
        const float2 st = a.st32[si];
        y = st.x;
        D = st.y;
        yc = a.y32[pair];
    }
    if (tid == 0) {
        s_lmin = 0x7fffffff;
        s_fail = 0;
    }
    __syncthreads();
    if (tid < kMsRows) atomicMin(&s_lmin, ls);
    __syncthreads();
    const int lstart = s_lmin;
    const int s_first = grp * a.nsg;

    if (lstart > a.L) {   // no ring of this CTA has a significant term: the sums are zero
        if (tid < kMsRows && pair < a.npairs)
            for (int s = 0; s < a.nsg && s_first + s < a.nsky; ++s)
                ms_write_two(a, a.G + (int64_t)(s_first + s) * a.gsky, m, k, pair, neg, make_float2(0.f, 0.f),
                             make_float2(0.f, 0.f));
        return;
    }
    const int nchunks = (a.L - lstart + kMsLC) / kMsLC;
    // With more than 16 skies a V warp has two units per chunk (skies 4 vw.. and 16 + 4 vw..);
    // when both hold skies, W warp vw builds the second one after its recurrence (the W
    // warps would otherwise idle on the MMAs while the V warps bind the kernel).
    const int npass = (a.nsg + 15) >> 4;
    auto passes_of = [&](int vw) { return min(npass, max(0, (a.nsg - 4 * vw + 15) >> 4)); };
    int nhelp = 0;
#pragma unroll
    for (int w = 0; w < 4; ++w) nhelp += (npass == 2 && passes_of(w) == 2) ? 1 : 0;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_base)), "r"(kMsTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int q = 0; q < 4 * kMsNS; ++q)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&stg_bar[q / kMsNS][q % kMsNS]))
                         : "memory");
        for (int q = 0; q < 4 * kMsNS; ++q)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&slot_free[q / kMsNS][q % kMsNS]))
                         : "memory");
        for (int q = 0; q < kMsNB; ++q) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&full_a[q])), "r"(kMsRows) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&full_b[q])), "r"(kMsRows + 32 * nhelp)
                         : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&empty[q])) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (warp < 4) {
        // ---------------------------------------------------------------- W producers
        // this warp's lane i holds the coefficients of l = c0 + i (prefetched one chunk ahead)
        RTab32 tcur = {0.f, 0.f, 0.f, 0.f}, tnext = {0.f, 0.f, 0.f, 0.f};
        // helper duty: the second unit of V warp `warp` (skies 16 + 4 warp ..), see the V producers
        const bool whelp = npass == 2 && passes_of(warp) == 2;
        const int lmin = max(m, k);
        const float2 *beam_k = a.beam + (int64_t)k * (a.L + 1);
        int swz_off[2][4];
        ms_swz_offsets(lane, swz_off);
        if (lstart + lane <= a.L) tcur = tab[lstart + lane];
        for (int c = 0; c < nchunks; ++c) {
            const int bi = c % kMsNB;
            const int c0 = lstart + c * kMsLC;
            if (c + 1 < nchunks && c0 + kMsLC + lane <= a.L) tnext = tab[c0 + kMsLC + lane];
            // the beam values of this lane's l for the helper unit (in flight during the recurrence)
            float2 wb[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
            const bool lok = c0 + lane <= a.L && c0 + lane >= lmin;
            if (whelp && lok) {
#pragma unroll
                for (int X = 0; X < NC; ++X) wb[X] = __ldg(beam_k + (int64_t)X * (a.K + 1) * (a.L + 1) + c0 + lane);
            }
            if (c >= kMsNB && !mbar_wait(smem_u32(&empty[bi]), ((c - kMsNB) / kMsNB) & 1)) *fail = 1;
            if (*fail) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // the chunk's coefficients, broadcast through shared memory (one load per step)
            __syncwarp();
            wcoef[warp][lane] = make_float2(tcur.a, neg ? tcur.cm : tcur.cp);
            __syncwarp();
            uint32_t hv[kMsLC], lv[kMsLC];
            if (__all_sync(0xffffffffu, c0 >= ls && c0 + kMsLC - 1 <= a.L)) {
                // every lane's recurrence runs through the whole chunk: no range tests
#pragma unroll
                for (int i = 0; i < kMsLC; ++i) {
                    const float2 t = wcoef[warp][i];
                    const float v = y;
                    D = fmaf(fmaf(-t.x, yc, t.y), y, D);
                    y += D;
                    float h, lo;
                    tf32_split(v, h, lo);
                    hv[i] = __float_as_uint(h);
                    lv[i] = __float_as_uint(lo);
                }
            } else {
#pragma unroll
                for (int i = 0; i < kMsLC; ++i) {
                    const int l = c0 + i;
                    const float2 t = wcoef[warp][i];
                    float v = 0.f;
                    if (l >= ls && l <= a.L) {
                        v = y;
                        D = fmaf(fmaf(-t.x, yc, t.y), y, D);
                        y += D;
                    }
                    float h, lo;
                    tf32_split(v, h, lo);
                    hv[i] = __float_as_uint(h);
                    lv[i] = __float_as_uint(lo);
                }
            }
            const uint32_t arow = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(kMsAcol + bi * 64);
            asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
                         "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
                         "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"
                         :: "r"(arow), "r"(hv[0]), "r"(hv[1]), "r"(hv[2]), "r"(hv[3]), "r"(hv[4]), "r"(hv[5]),
                            "r"(hv[6]), "r"(hv[7]), "r"(hv[8]), "r"(hv[9]), "r"(hv[10]), "r"(hv[11]), "r"(hv[12]),
                            "r"(hv[13]), "r"(hv[14]), "r"(hv[15]), "r"(hv[16]), "r"(hv[17]), "r"(hv[18]),
                            "r"(hv[19]), "r"(hv[20]), "r"(hv[21]), "r"(hv[22]), "r"(hv[23]), "r"(hv[24]),
                            "r"(hv[25]), "r"(hv[26]), "r"(hv[27]), "r"(hv[28]), "r"(hv[29]), "r"(hv[30]),
                            "r"(hv[31]) : "memory");
            asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
                         "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
                         "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"
                         :: "r"(arow + 32), "r"(lv[0]), "r"(lv[1]), "r"(lv[2]), "r"(lv[3]), "r"(lv[4]), "r"(lv[5]),
                            "r"(lv[6]), "r"(lv[7]), "r"(lv[8]), "r"(lv[9]), "r"(lv[10]), "r"(lv[11]), "r"(lv[12]),
                            "r"(lv[13]), "r"(lv[14]), "r"(lv[15]), "r"(lv[16]), "r"(lv[17]), "r"(lv[18]),
                            "r"(lv[19]), "r"(lv[20]), "r"(lv[21]), "r"(lv[22]), "r"(lv[23]), "r"(lv[24]),
                            "r"(lv[25]), "r"(lv[26]), "r"(lv[27]), "r"(lv[28]), "r"(lv[29]), "r"(lv[30]),
                            "r"(lv[31]) : "memory");
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(smem_u32(&full_a[bi]));
            if (whelp) {
                const int ui = 2 * c + 1, sl = ui % kMsNS;
                // V warp `warp` has read unit ui - 3 of this slot and issued unit ui into it
                if (c >= 1 && !mbar_wait(smem_u32(&slot_free[warp][sl]), ((ui - 3) / kMsNS) & 1)) *fail = 1;
                if (!*fail && !mbar_wait(smem_u32(&stg_bar[warp][sl]), (ui / kMsNS) & 1)) *fail = 1;
                if (*fail) break;
                // this lane's beam factors (l = c0 + lane), as the V producers form them
                const float cl = lok ? tcur.c : 0.f, sg = neg ? -cl : cl, sy = (m == 0) ? 0.f : sg;
                float bxc[3], byc[3], bxs[3], bys[3];
#pragma unroll
                for (int X = 0; X < 3; ++X) {
                    if (k == 0) wb[X].y = 0.f;
                    bxc[X] = cl * wb[X].x;
                    byc[X] = cl * wb[X].y;
                    bxs[X] = sy * wb[X].x;
                    bys[X] = sy * wb[X].y;
                }
                const float par = ((c0 + lane) & 1) ? -1.f : 1.f;
                float *Bh = base + bi * 2 * bfl + 128 * (16 + 4 * warp), *Bl = Bh + bfl;
                const int64_t x0 = moff + lstart + (int64_t)c * kMsLC;
                const float *wstage = base + 2 * kMsNB * bfl + warp * kMsNS * kMsStageF;
                ms_build_unit<NC>(wstage + sl * kMsStageF + 2 * ((int)(x0 & 1) + lane), Bh, Bl, bxc, byc, bxs,
                                  bys, par, swz_off);
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&slot_free[warp][sl]));
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(smem_u32(&full_b[bi]));
            }
            tcur = tnext;
        }
    } else if (warp < 8) {
        // ---------------------------------------------------------------- V producers
        // Work unit u = (chunk c, pass j): the 4 consecutive skies 4 vw + 16 j .. + 3 at
        // l = c0 + lane.  Lane 0 brings their T/E/B rows m, l = c0 .. c0 + 31 (from an even
        // alm index: the tensor map's rows start on 16 bytes) into this warp's staging slot
        // u mod 3 with one TMA tensor load, two units ahead of the unit being built.
        const int vw = warp - 4;
        const float2 *beam_k = a.beam + (int64_t)k * (a.L + 1);
        const int lmin = max(m, k);
        const int i = lane;
        int swz_off[2][4];
        ms_swz_offsets(lane, swz_off);
        const int nunits = nchunks * npass;
        // this warp's passes j < na hold skies (4 vw + 16 j < nsg); its staged units are
        // numbered ui = c na + j, slot ui mod 3, and issued two units ahead
        const int na = passes_of(vw), nact = nchunks * na;
        const bool helped = npass == 2 && na == 2;
        float *stage = base + 2 * kMsNB * bfl + vw * kMsNS * kMsStageF;
        const uint32_t tx_bytes = (uint32_t)(kMsBoxX * NC * 4 * sizeof(float));
        auto issue = [&](int ui) {
            if (lane != 0 || ui >= nact) return;
            const int c = ui / na, j = ui - c * na, s0 = 4 * vw + 16 * j;
            const int64_t x0 = moff + lstart + (int64_t)c * kMsLC;    // alm index of l = c0
            const int xf = (int)((x0 & ~(int64_t)1) * 2);              // in floats, a multiple of 4
            const uint32_t bar = smem_u32(&stg_bar[vw][ui % kMsNS]);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(tx_bytes)
                         : "memory");
            asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
                         "[%0], [%1, {%2, %3, %4}], [%5];"
                         :: "r"(smem_u32(stage + (ui % kMsNS) * kMsStageF)), "l"(&tmap), "r"(xf), "r"(0),
                            "r"(s_first + s0), "r"(bar)
                         : "memory");
        };
        issue(0);
        issue(1);
        // beam and c_l of the next two chunks are prefetched into registers
        float2 bn[3], bn2[3];
        float cn, cn2;
        auto beam_of = [&](int c, float2 *bo, float &co) {
            const int l = lstart + c * kMsLC + i;
            bo[0] = bo[1] = bo[2] = make_float2(0.f, 0.f);
            co = 0.f;
            if (c < nchunks && l <= a.L && l >= lmin) {
#pragma unroll
                for (int X = 0; X < 3; ++X)
                    if (X < NC) {
                        bo[X] = __ldg(beam_k + (int64_t)X * (a.K + 1) * (a.L + 1) + l);
                        if (k == 0) bo[X].y = 0.f;
                    }
                co = __ldg(&tab[l].c);
            }
        };
        beam_of(0, bn, cn);
        beam_of(1, bn2, cn2);
        float bxc[3], byc[3], bxs[3], bys[3], par = 1.f;
        auto chunk_factors = [&](int c) {
            const int l = lstart + c * kMsLC + i;
            // this lane's beam factors for the chunk (c_l folded in; sigma = sign of k
            // and the m = 0 rule -- Im s ignored -- folded into the factors of Im s)
            const float cl = cn, sg = neg ? -cl : cl, sy = (m == 0) ? 0.f : sg;
#pragma unroll
            for (int X = 0; X < 3; ++X) {
                bxc[X] = cl * bn[X].x;
                byc[X] = cl * bn[X].y;
                bxs[X] = sy * bn[X].x;
                bys[X] = sy * bn[X].y;
                bn[X] = bn2[X];
            }
            par = (l & 1) ? -1.f : 1.f;
            cn = cn2;
            beam_of(c + 2, bn2, cn2);
        };
        int ui_done = 0;                  // staged units consumed
        int issued = min(2, nact);        // units issued (the helped schedule)
        if (helped) {
            // Units 2c (this warp) and 2c + 1 (W warp vw) per chunk; unit u sits in slot u mod 3.
            // A copy lands in a slot only once the slot's previous unit has been read: unit
            // 2c + 3 goes into the slot of 2c, which this warp has just read; unit 2c + 2 into
            // the slot of 2c - 1, which W warp vw releases through slot_free.  This warp arrives
            // on the slot_free of 2c once 2c is read and 2c + 3 issued; W warp vw waits for that
            // before it tests the staging barrier of 2c + 3 (so no parity test runs two phases
            // away from its barrier).
            for (int c = 0; c < nchunks; ++c) {
                const int bi = c % kMsNB;
                chunk_factors(c);
                if (c >= kMsNB && !mbar_wait(smem_u32(&empty[bi]), ((c - kMsNB) / kMsNB) & 1)) *fail = 1;
                if (*fail) break;
                const int nx = 2 * c + 2;
                if (nx < nact) {
                    if (c >= 1 && !mbar_wait(smem_u32(&slot_free[vw][nx % kMsNS]), ((2 * c - 1) / kMsNS) & 1))
                        *fail = 1;
                    if (*fail) break;
                    issue(nx);
                    issued = nx + 1;
                }
                const int ui = 2 * c;
                if (!mbar_wait(smem_u32(&stg_bar[vw][ui % kMsNS]), (ui / kMsNS) & 1)) *fail = 1;
                if (*fail) break;
                float *Bh = base + bi * 2 * bfl + 128 * (4 * vw), *Bl = Bh + bfl;
                const int64_t x0 = moff + lstart + (int64_t)c * kMsLC;
                ms_build_unit<NC>(stage + (ui % kMsNS) * kMsStageF + 2 * ((int)(x0 & 1) + i), Bh, Bl, bxc, byc,
                                  bxs, bys, par, swz_off);
                __syncwarp();
                if (ui + 3 < nact) {
                    issue(ui + 3);
                    issued = ui + 4;
                }
                if (lane == 0) mbar_arrive(smem_u32(&slot_free[vw][ui % kMsNS]));
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(smem_u32(&full_b[bi]));
            }
            // after a failed wait: the last copy issued into each slot lands (bounded) before
            // the CTA's shared memory is released
            if (*fail && lane == 0)
                for (int u = max(0, issued - kMsNS); u < issued; ++u)
                    mbar_wait(smem_u32(&stg_bar[vw][u % kMsNS]), (u / kMsNS) & 1, 1000000ull);
        } else
        for (int u = 0; u < nunits; ++u) {
            const int c = u / npass, j = u - c * npass, bi = c % kMsNB, s0 = 4 * vw + 16 * j;
            if (j == 0) {
                chunk_factors(c);
                if (c >= kMsNB && !mbar_wait(smem_u32(&empty[bi]), ((c - kMsNB) / kMsNB) & 1)) *fail = 1;
            }
            if (*fail) break;
            if (j < na) {
                const int ui = c * na + j;
                __syncwarp();             // slot (ui + 2) mod 3 was last read in unit ui - 1
                issue(ui + 2);
                if (!mbar_wait(smem_u32(&stg_bar[vw][ui % kMsNS]), (ui / kMsNS) & 1)) *fail = 1;
                if (*fail) break;
                float *Bh = base + bi * 2 * bfl + 128 * s0, *Bl = Bh + bfl;
                // this lane's l sits at float2 (x0 & 1) + lane of each staged row
                const int64_t x0 = moff + lstart + (int64_t)c * kMsLC;
                ms_build_unit<NC>(stage + (ui % kMsNS) * kMsStageF + 2 * ((int)(x0 & 1) + i), Bh, Bl, bxc, byc,
                                  bxs, bys, par, swz_off);
                ui_done = ui + 1;
            }
            if (j == npass - 1) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(smem_u32(&full_b[bi]));
            }
        }
        // after a failed wait: the TMA loads still in flight land (bounded) before the
        // CTA's shared memory is released
        if (!helped && *fail && lane == 0)
            for (int ui = ui_done; ui < min(ui_done + kMsNS, nact); ++ui)
                mbar_wait(smem_u32(&stg_bar[vw][ui % kMsNS]), (ui / kMsNS) & 1, 1000000ull);
    } else if (lane == 0) {
        // ---------------------------------------------------------------- MMA issuer
        const uint32_t idesc = ms_idesc(kMsRows, N);
        int issued = -1;   // last chunk whose MMAs were committed
        for (int c = 0; c < nchunks; ++c) {
            const int bi = c % kMsNB;
            const uint32_t par = (c / kMsNB) & 1;
            if (!mbar_wait(smem_u32(&full_a[bi]), par) || !mbar_wait(smem_u32(&full_b[bi]), par)) *fail = 1;
            if (*fail) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const float *Bh = base + bi * 2 * bfl, *Bl = Bh + bfl;
            const uint32_t bh = smem_u32(Bh), bl = smem_u32(Bl);
            const uint32_t ahi = tmem + (uint32_t)(kMsAcol + bi * 64), alo = ahi + 32;
#pragma unroll
            for (int kk = 0; kk < kMsLC / 8; ++kk) {
                const uint64_t dbh = ms_sdesc(bh + kk * 32), dbl = ms_sdesc(bl + kk * 32);
                const uint32_t acc0 = (c > 0 || kk > 0) ? 1u : 0u;
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}"
                             :: "r"(tmem), "r"(ahi + kk * 8), "l"(dbh), "r"(idesc), "r"(acc0) : "memory");
                asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, 1;"
                             :: "r"(tmem), "r"(ahi + kk * 8), "l"(dbl), "r"(idesc) : "memory");
                asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, 1;"
                             :: "r"(tmem), "r"(alo + kk * 8), "l"(dbh), "r"(idesc) : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(smem_u32(&empty[bi])) : "memory");
            issued = c;
        }
        // MMAs still in flight (a failed wait elsewhere) must end before the dealloc
        if (*fail && issued >= 0) mbar_wait(smem_u32(&empty[issued % kMsNB]), (issued / kMsNB) & 1);
    }

    // the last chunk's commit means every MMA of the CTA has finished
    bool ok = true;
    if (warp < 4) {
        const int cl_ = nchunks - 1;
        ok = !*fail && mbar_wait(smem_u32(&empty[cl_ % kMsNB]), (cl_ / kMsNB) & 1);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (!ok) {
            if (lane == 0) atomicExch(a.err, 1);
        } else {
            // epilogue: lanes 32w..32w+31 are rows (ring pairs); 16 columns = 4 skies per load
            const int row = warp * 32 + lane, pr = rc * kMsRows + row;
            for (int cg = 0; cg < N / 16; ++cg) {
                uint32_t r[16];
                const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cg * 16);
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                             "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                             : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                               "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
                               "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                             : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (pr < a.npairs) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int sky = s_first + cg * 4 + q;
                        if (sky < a.nsky)
                            ms_write_two(a, a.G + (int64_t)sky * a.gsky, m, k, pr, neg,
                                         make_float2(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1])),
                                         make_float2(__uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3])));
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kMsTmemCols) : "memory");
}

// Failure-detection self-test: a wait on an mbarrier that nothing signals
// must expire and raise the error flag (the context stays usable).
__global__ void k_wait_probe(int *err, unsigned long long limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&bar)) : "memory");
    if (!mbar_wait(smem_u32(&bar), 0, limit_ns)) atomicExch(err, 1);
}

sl_status launch_wait_probe(sl_plan *p, int *err) {
    k_wait_probe<<<1, 32, 0, p->stream>>>(err, 50000000ull);
    return cuda_check(cudaGetLastError(), "k_wait_probe launch");
}

__global__ void k_to_f32_ms(const double2 *__restrict__ in, float2 *__restrict__ out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

// [nrows][nalm] complex128 -> [nrows][salm] complex64, the padding zeroed
__global__ void k_to_f32_rows(const double2 *__restrict__ in, float2 *__restrict__ out, int64_t nrows, int64_t nalm,
                              int64_t salm) {
    const int64_t n = nrows * salm;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / salm, c = i - r * salm;
        const double2 v = c < nalm ? in[r * nalm + c] : make_double2(0.0, 0.0);
        out[i] = make_float2((float)v.x, (float)v.y);
    }
}

// The 3-D tensor map over the FP32 skies: x = floats of a row (2 salm), y = component,
// z = sky; boxes of 68 floats x ncomp x 4 skies, zero fill outside.
static sl_status sky_tensor_map(CUtensorMap *tm, const float2 *sky32, int64_t salm, int ncomp, int nsky) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return set_error(SL_ERR_CUDA, "cuTensorMapEncodeTiled entry point unavailable");
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t dims[3] = {(cuuint64_t)(2 * salm), (cuuint64_t)ncomp, (cuuint64_t)nsky};
    const cuuint64_t strides[2] = {(cuuint64_t)(2 * salm * sizeof(float)), (cuuint64_t)(2 * salm * ncomp * sizeof(float))};
    const cuuint32_t box[3] = {(cuuint32_t)kMsBoxX, (cuuint32_t)ncomp, 4u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    const CUresult r = encode(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)sky32, dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(SL_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return SL_OK;
}

size_t lcontract_mma_smem(int nsg, int ncomp) {
    (void)ncomp;
    // B_hi, B_lo (two buffers), the four V warps' staging slots, alignment slack
    return 2 * kMsNB * (size_t)4 * nsg * kMsLC * sizeof(float) + (size_t)4 * kMsNS * kMsStageF * sizeof(float) + 1024;
}

int lcontract_mma_group(int nsky) {
    int nsg = std::min(32, nsky);
    return (nsg + 3) & ~3;
}

sl_status launch_lcontract_mma(sl_plan *p, int nsky, const double *sky, const double *beam, float2 *sky32,
                               float2 *G, int *err) {
    const int64_t salm = sky_row_stride(p->nalm);
    const int64_t nrows = (int64_t)nsky * p->ncomp, nb = (int64_t)p->ncomp * (p->K + 1) * (p->L + 1);
    k_to_f32_rows<<<(unsigned)std::min<int64_t>((nrows * salm + 255) / 256, 8192), 256, 0, p->stream>>>(
        (const double2 *)sky, sky32, nrows, p->nalm, salm);
    k_to_f32_ms<<<(unsigned)std::min<int64_t>((nb + 255) / 256, 4096), 256, 0, p->stream>>>((const double2 *)beam,
                                                                                             p->d_beam32, nb);
    MsArgs a;
    a.L = p->L;
    a.K = p->K;
    a.ncomp = p->ncomp;
    a.R = p->R;
    a.npairs = p->npairs;
    a.nrc = (p->npairs + kMsRows - 1) / kMsRows;
    a.nsky = nsky;
    a.nsg = lcontract_mma_group(nsky);
    a.ngroups = (nsky + a.nsg - 1) / a.nsg;
    a.nalm = p->nalm;
    a.sky = sky32;
    a.salm = salm;
    CUtensorMap tmap;
    sl_status st = sky_tensor_map(&tmap, sky32, salm, p->ncomp, nsky);
    if (st != SL_OK) return st;
    a.beam = p->d_beam32;
    a.y32 = p->d_y32;
    a.ls = p->d_ls;
    a.st32 = p->d_st32;
    a.tab32 = p->d_tab32;
    a.G = G;
    a.gsky = (int64_t)(p->K + 1) * p->R * (2 * p->L + 1);
    a.err = err;
    const int64_t nblk = (int64_t)(p->L + 1) * (p->K + 1) * 2 * a.nrc * a.ngroups;
    if (nblk > 0x7fffffff) return set_error(SL_ERR_UNSUPPORTED, "grid too large");
    const size_t sm = lcontract_mma_smem(a.nsg, a.ncomp);
    void (*kern)(const MsArgs, const CUtensorMap) = a.ncomp == 1 ? k_lcontract_mma<1> : k_lcontract_mma<3>;
    cudaError_t e = allow_dyn_smem(kern, sm);
    if (e != cudaSuccess) return cuda_check(e, "k_lcontract_mma smem attribute");
    const int slot = timing_begin(p, "lcontract_mma");
    kern<<<(unsigned)nblk, kMsThreads, sm, p->stream>>>(a, tmap);
    timing_end(p, slot);
    return cuda_check(cudaGetLastError(), "k_lcontract_mma launch");
}

}  // namespace sl
