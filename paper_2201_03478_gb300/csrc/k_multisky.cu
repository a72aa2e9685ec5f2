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
//   * CTA = (m, k, sign, 128 ring pairs, group of up to 64 skies), M = 128,
//     N = 4 x skies, K = l in chunks of 32 (one 128-byte swizzle row of TF32);
//   * W and V are split into TF32 high and low parts and multiplied as
//     hi x hi + hi x lo + lo x hi (three MMAs, FP32 accumulation in tensor
//     memory): ~2^-21 relative per product, the accuracy of the FP32 path;
//   * both operands live in shared memory, K-major with the 128-byte swizzle,
//     double buffered: while the MMAs of one chunk run, the CTA generates the
//     next chunk's W rows and V columns, from coefficients, sky and beam values
//     that cp.async copies have staged in shared memory two chunks ahead;
//   * one thread issues the MMAs and commits them to an mbarrier per buffer;
//     every wait is bounded and sets an error flag (the CTA then stops,
//     waits for its MMAs with a bound and frees its tensor memory).
#include <algorithm>

#include "sl_internal.cuh"

namespace sl {

constexpr int kMsRows = 128;      // ring pairs per CTA (MMA M)
constexpr int kMsLC = 32;         // l per chunk
constexpr int kMsThreads = 256;
constexpr unsigned long long kMsWaitNs = 1000000000ull;   // bound of every mbarrier wait: 1 s

struct MsArgs {
    int L, K, ncomp, R, npairs, nrc;     // nrc: ring chunks of 128 pairs
    int nsky, nsg, ngroups;              // skies, skies per CTA (multiple of 4), groups
    int64_t nalm;
    const float2 *sky;                   // [nsky][ncomp][nalm], FP32 copy
    const float2 *beam;                  // [ncomp][K+1][L+1], FP32 copy
    const float *y32;                    // [npairs] 1 - cos theta
    const int *ls;                       // [K+1][L+1][2][npairs] first significant l
    const float2 *st32;                  // start states (y, D)
    const RTab32 *tab32;                 // [K+1][nalm] {a', c'+, c'-, c}
    float2 *G;                           // [nsky][K+1][R][2L+1]
    int64_t gsky;                        // elements of one sky's G
    int *err;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

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

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the completion of the mbarrier phase of the given parity, for at
// most limit_ns of wall time; false when the limit expired.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned long long limit_ns = kMsWaitNs) {
    const unsigned long long t0 = globaltimer_ns();
    for (;;) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, q;\n\t}"
                     : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
        if (globaltimer_ns() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" :: "r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int NPEND>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" :: "n"(NPEND) : "memory"); }

// Staged inputs of one chunk: sky [nsg][ncomp][32], beam [ncomp][32], coefficients [32].
struct MsStage {
    float2 *sky, *beam;
    RTab32 *tab;
};

// The sky tile's rows (sky, X) are consecutive rows of the [nsky][ncomp][nalm]
// array: warp w copies rows w, w + 8, ..., lane = l - c0.
__device__ __forceinline__ void ms_prefetch(const MsArgs &a, const MsStage &st, const float2 *sky_rows,
                                            int row_limit, const float2 *beam_k, const RTab32 *tab, int c0) {
    const int lane = threadIdx.x & 31, l = c0 + lane;
    if (l <= a.L) {
        const int rows = a.nsg * a.ncomp;
        for (int r = threadIdx.x >> 5; r < rows; r += kMsThreads / 32)
            if (r < row_limit) cp_async8(st.sky + r * 32 + lane, sky_rows + (int64_t)r * a.nalm + l);
        const int X = threadIdx.x >> 5;
        if (X < a.ncomp) cp_async8(st.beam + X * 32 + lane, beam_k + (int64_t)X * (a.K + 1) * (a.L + 1) + l);
        if (threadIdx.x < 32) cp_async16(st.tab + lane, tab + l);
    }
    cp_async_commit();
}

// TF32 split: hi keeps the 19 bits the tensor core reads, lo = x - hi (exact)
__device__ __forceinline__ void tf32_split(float x, float &hi, float &lo) {
    hi = __uint_as_float(__float_as_uint(x) & 0xffffe000u);
    lo = x - hi;
}

__device__ __forceinline__ void ms_write_two(const MsArgs &a, float2 *G, int m, int k, int pair, int neg, float2 acc1,
                                             float2 acc2) {
    const int rn = pair, rs = a.R - 1 - pair;
    const int64_t row = 2 * (int64_t)a.L + 1, base = (int64_t)k * a.R;
    const bool modd = m & 1, kodd = k & 1;
    if (!neg) {
        G[(base + rn) * row + a.L + m] = acc1;
        if (m > 0 && rs != rn) {
            if (modd != kodd) { acc2.x = -acc2.x; acc2.y = -acc2.y; }
            G[(base + rs) * row + a.L - m] = acc2;
        }
    } else {
        if (m > 0) {
            if (kodd) { acc1.x = -acc1.x; acc1.y = -acc1.y; }
            G[(base + rn) * row + a.L - m] = acc1;
        }
        if (rs != rn) {
            if (modd) { acc2.x = -acc2.x; acc2.y = -acc2.y; }
            G[(base + rs) * row + a.L + m] = acc2;
        }
    }
}

__global__ void __launch_bounds__(kMsThreads, 1) k_lcontract_mma(const MsArgs a) {
    extern __shared__ unsigned char ms_raw[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_base;
    __shared__ int s_lmin, s_fail;

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

    // operand buffers, 1024-byte aligned: per buffer A_hi, A_lo [128][32], B_hi, B_lo [N][32]
    const uint32_t raw = smem_u32(ms_raw);
    float *base = reinterpret_cast<float *>(ms_raw + ((1024u - (raw & 1023u)) & 1023u));
    const int afl = kMsRows * kMsLC, bfl = N * kMsLC;
    float *buf[2] = {base, base + 2 * afl + 2 * bfl};
    float2 *const stage0 = reinterpret_cast<float2 *>(base + 4 * afl + 4 * bfl);
    const int nsky_el = a.nsg * a.ncomp * 32, nbeam_el = a.ncomp * 32;
    const int stage_el = nsky_el + nbeam_el + 64;   // 32 RTab32 = 64 float2
    auto stage_of = [&](int q) {
        float2 *sp = stage0 + q * stage_el;
        return MsStage{sp, sp + nsky_el, reinterpret_cast<RTab32 *>(sp + nsky_el + nbeam_el)};
    };

    // this thread's recurrence (threads 0..127 own the rows)
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
    int ncols = 32;
    while (ncols < N) ncols <<= 1;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_base)), "r"(ncols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = ms_idesc(kMsRows, N);

    int issued = -1;    // last chunk whose MMAs were committed
    const float2 *sky_rows = a.sky + (int64_t)s_first * a.ncomp * a.nalm + moff;
    const int row_limit = min(a.nsg, a.nsky - s_first) * a.ncomp;
    const float2 *beam_k = a.beam + (int64_t)k * (a.L + 1);
    ms_prefetch(a, stage_of(0), sky_rows, row_limit, beam_k, tab, lstart);
    ms_prefetch(a, stage_of(1), sky_rows, row_limit, beam_k, tab, lstart + kMsLC);
    for (int c = 0; c < nchunks; ++c) {
        const int bi = c & 1;
        // stage chunk c + 2 (its stage was last read by chunk c - 1, before the
        // barrier that preceded that chunk's MMAs; past lmax the group is empty),
        // then wait for chunk c's copies (two newer groups may stay in flight)
        ms_prefetch(a, stage_of((c + 2) % 3), sky_rows, row_limit, beam_k, tab, lstart + (c + 2) * kMsLC);
        cp_async_wait<2>();
        if (c >= 2 && !mbar_wait(smem_u32(&mbar[bi]), ((c - 2) >> 1) & 1)) s_fail = 1;
        __syncthreads();
        if (s_fail) break;
        float *Ah = buf[bi], *Al = Ah + afl, *Bh = Al + afl, *Bl = Bh + bfl;
        const MsStage st = stage_of(c % 3);
        const int c0 = lstart + c * kMsLC;
        if (tid < kMsRows) {
            // W row: y_l for l in [c0, c0 + 32), zero before the ring's start
            float w[kMsLC];
#pragma unroll
            for (int i = 0; i < kMsLC; ++i) {
                const int l = c0 + i;
                float v = 0.f;
                if (l >= ls && l <= a.L) {
                    v = y;
                    const RTab32 t = st.tab[i];
                    D = fmaf(fmaf(-t.a, yc, neg ? t.cm : t.cp), y, D);
                    y += D;
                }
                w[i] = v;
            }
#pragma unroll
            for (int q = 0; q < kMsLC / 4; ++q) {
                float4 h, lo;
                tf32_split(w[4 * q + 0], h.x, lo.x);
                tf32_split(w[4 * q + 1], h.y, lo.y);
                tf32_split(w[4 * q + 2], h.z, lo.z);
                tf32_split(w[4 * q + 3], h.w, lo.w);
                *reinterpret_cast<float4 *>(Ah + ms_sw(tid, 4 * q)) = h;
                *reinterpret_cast<float4 *>(Al + ms_sw(tid, 4 * q)) = lo;
            }
        }
        // V columns: item (sky s, four consecutive l), the four values of this sign each
        const int lmin = max(m, k);
        for (int e = tid; e < a.nsg * (kMsLC / 4); e += kMsThreads) {
            const int s = e >> 3, q = e & 7;
            float v[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = 4 * q + u, l = c0 + i;
                v[0][u] = v[1][u] = v[2][u] = v[3][u] = 0.f;
                if (l <= a.L && s_first + s < a.nsky && l >= lmin) {
                    float2 ap = {0.f, 0.f}, am = {0.f, 0.f};
                    for (int X = 0; X < a.ncomp; ++X) {
                        float2 sv = st.sky[(s * a.ncomp + X) * 32 + i];
                        if (m == 0) sv.y = 0.f;
                        float2 bv = st.beam[X * 32 + i];
                        if (k == 0) bv.y = 0.f;
                        ap.x += sv.x * bv.x + sv.y * bv.y;      // s conj(b)
                        ap.y += sv.y * bv.x - sv.x * bv.y;
                        am.x += sv.x * bv.x - sv.y * bv.y;      // conj(s) conj(b)
                        am.y -= sv.y * bv.x + sv.x * bv.y;
                    }
                    const float cl = st.tab[i].c, sc = (l & 1) ? -cl : cl;
                    const float2 p1 = neg ? am : ap, p2 = neg ? ap : am;
                    v[0][u] = cl * p1.x;
                    v[1][u] = cl * p1.y;
                    v[2][u] = sc * p2.x;
                    v[3][u] = sc * p2.y;
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int row = 4 * s + j, off = row * 32 + ((q ^ (row & 7)) << 2);
                float4 h, lo;
                tf32_split(v[j][0], h.x, lo.x);
                tf32_split(v[j][1], h.y, lo.y);
                tf32_split(v[j][2], h.z, lo.z);
                tf32_split(v[j][3], h.w, lo.w);
                *reinterpret_cast<float4 *>(Bh + off) = h;
                *reinterpret_cast<float4 *>(Bl + off) = lo;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            const uint32_t ah = smem_u32(Ah), al = smem_u32(Al), bh = smem_u32(Bh), bl = smem_u32(Bl);
#pragma unroll
            for (int kk = 0; kk < kMsLC / 8; ++kk) {
                const uint32_t off = kk * 32;   // 8 TF32 along K
                const uint64_t dah = ms_sdesc(ah + off), dal = ms_sdesc(al + off);
                const uint64_t dbh = ms_sdesc(bh + off), dbl = ms_sdesc(bl + off);
                const uint32_t acc0 = (c > 0 || kk > 0) ? 1u : 0u;
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
                             :: "r"(tmem), "l"(dah), "l"(dbh), "r"(idesc), "r"(acc0) : "memory");
                asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;"
                             :: "r"(tmem), "l"(dah), "l"(dbl), "r"(idesc) : "memory");
                asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;"
                             :: "r"(tmem), "l"(dal), "l"(dbh), "r"(idesc) : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(smem_u32(&mbar[bi])) : "memory");
        }
        issued = c;
    }
    cp_async_wait<0>();   // no copy into shared memory outlives the loop
    // every committed MMA has finished once the last commit has arrived
    bool ok = !s_fail;
    if (issued >= 0 && !mbar_wait(smem_u32(&mbar[issued & 1]), (issued >> 1) & 1)) ok = false;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) {
        if (tid == 0) atomicExch(a.err, 1);
    } else if (warp < 4) {
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
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(ncols) : "memory");
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

size_t lcontract_mma_smem(int nsg, int ncomp) {
    const size_t ops = 2 * (2 * (size_t)kMsRows * kMsLC + 2 * (size_t)4 * nsg * kMsLC) * 4;
    const size_t stage = 3 * ((size_t)nsg * ncomp * 32 + (size_t)ncomp * 32 + 64) * sizeof(float2);
    return ops + stage + 1024;
}

int lcontract_mma_group(int nsky) {
    int nsg = std::min(32, nsky);
    return (nsg + 3) & ~3;
}

sl_status launch_lcontract_mma(sl_plan *p, int nsky, const double *sky, const double *beam, float2 *sky32,
                               float2 *G, int *err) {
    const int64_t ns = (int64_t)nsky * p->ncomp * p->nalm, nb = (int64_t)p->ncomp * (p->K + 1) * (p->L + 1);
    k_to_f32_ms<<<(unsigned)std::min<int64_t>((ns + 255) / 256, 8192), 256, 0, p->stream>>>((const double2 *)sky,
                                                                                             sky32, ns);
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
    cudaError_t e = cudaFuncSetAttribute(k_lcontract_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return cuda_check(e, "k_lcontract_mma smem attribute");
    const int slot = timing_begin(p, "lcontract_mma");
    k_lcontract_mma<<<(unsigned)nblk, kMsThreads, sm, p->stream>>>(a);
    timing_end(p, slot);
    return cuda_check(cudaGetLastError(), "k_lcontract_mma launch");
}

}  // namespace sl
