// k_lcontract.cu -- the spin "Legendre" step of the cube (Sect. 2.1, Eqs. c_m
// and S):
//
//   G_k(r, m) = sum_{l >= max(|m|, k)} A_{k,lm} d^l_{mk}(theta_r),
//   A_{k,lm}  = sum_X s^X_lm conj(b^X_lk),      m in [-L, L], k in [0, K],
//
// written to G[k][m + L][r]: the ring index is fastest, so that the threads of a
// CTA (consecutive ring pairs at one m) write contiguous runs.
//
// Reflections.  Per north ring, two l-recurrences, d^l_{m,+k}(theta_r) and
// d^l_{m,-k}(theta_r), give four outputs through
//   d^l_{-m,k}(t)    = (-1)^{m+k} d^l_{m,-k}(t)
//   d^l_{ m,k}(pi-t) = (-1)^{l+m} d^l_{m,-k}(t)
//   d^l_{-m,k}(pi-t) = (-1)^{l-k} d^l_{m, k}(t)
// and the sky's real-field relation s_{l,-m} = (-1)^m conj(s_lm):
//   +k recurrence d1:  G(north, +m) = sum_l A+_l d1_l,
//                      G(south, -m) = (-1)^{m+k} sum_l (-1)^l A-_l d1_l
//   -k recurrence d2:  G(north, -m) = (-1)^k sum_l A-_l d2_l,
//                      G(south, +m) = (-1)^m sum_l (-1)^l A+_l d2_l
// with A+_l = sum_X s conj(b) and A-_l = sum_X conj(s) conj(b).
//
// Recurrence.  d^{l+1} = (a_l x - b_l) d^l - g_l d^{l-1} (x = cos theta; b
// changes sign with k) runs on rescaled values y_l = d_l / c_l with
// c_{l+1} = g_l c_{l-1}:  y_{l+1} = (a'_l x -+ b'_l) y_l - y_{l-1}, and c_l moves
// into the sum coefficients.  a', b', c_l come from the plan table (k_rtab).
// Each ring and sign starts at the plan's start state (k_advance): the first
// l at which the value is significant; the evanescent part before it (about
// 28% of the (ring, m, l) volume at lmax = 1024) is not run at all.
//
// FP64 plans: one thread per (north ring, sign of k): per l, 2 FP64 operations
// for the recurrence and 4 for the two complex x real sums.  FP32 plans: one
// thread per (two adjacent north rings, sign); the recurrence in the
// difference form  D_{l+1} = (c'_l - a'_l y) y_l + D_l,  y_{l+1} = y_l + D_{l+1}
// with y = 1 - cos(theta) and c' = a' -+ b' - 2 formed in double (keeps the
// FP32 recurrence accurate near the pole, where cos theta alone carries too
// few bits); sky x beam products from FP32 copies of sky and beam.
// DF64 plans: the FP64 plan's layout and start states, with the recurrence
// and the sums in double-float arithmetic (df.cuh): per l, two double-float
// products and two sums for the recurrence and four double-float
// multiply-accumulates, all on the FP32 pipes.
// The CTA stages the coefficients of a chunk of l in shared memory (double
// buffered in FP32); a thread steps only from its own start l.
#include <algorithm>

#include "df.cuh"
#include "sl_internal.cuh"

namespace sl {

constexpr int kNT = 256;          // threads per CTA
constexpr int kHalf = kNT / 2;    // threads per sign
constexpr int kF32Pairs = 4;      // ring pairs per thread of the FP32 contraction
constexpr int kLC64 = 64;         // l values staged per chunk (FP64)

struct __align__(16) Coef64 {
    double a, nb, pb, unused;     // a', -b', +b'
};
struct __align__(16) Acc64 {
    double2 ap, sam, am, sap;     // +k uses (ap, sam), -k uses (am, sap)
};

struct LcArgs {
    int L, K, ncomp, R, npairs, nchunk, ppt;  // ppt: ring pairs per thread
    int64_t nalm;
    const double2 *sky, *beam;       // FP64 inputs
    const float2 *sky32, *beam32;    // FP32 copies (FP32 plans)
    const double *xr;
    const float *y32;
    const int *ls;
    const double2 *st64;
    const float2 *st32;
    const RTab64 *tab64;
    const RTab32 *tab32;
    void *G;
};

__device__ __forceinline__ void block_mk(const LcArgs &a, int &m, int &k, int &pc) {
    int b = blockIdx.x;
    pc = b % a.nchunk;
    b /= a.nchunk;
    k = b % (a.K + 1);
    m = b / (a.K + 1);
}

__device__ __forceinline__ int64_t start_index(const LcArgs &a, int k, int m, int neg, int pair) {
    return (((int64_t)k * (a.L + 1) + m) * 2 + neg) * a.npairs + pair;
}

// Writes the two sums of one recurrence.  neg = 0 (+k): acc1 -> (north, +m),
// acc2 -> (south, -m); neg = 1 (-k): acc1 -> (north, -m), acc2 -> (south, +m).
template <typename C>
__device__ __forceinline__ void write_two(const LcArgs &a, int m, int k, int pair, int neg, C acc1, C acc2) {
    C *G = reinterpret_cast<C *>(a.G);
    const int rn = pair, rs = a.R - 1 - pair;
    // rows (k, L + m) and (k, L - m) of G
    C *gp = G + ((int64_t)k * (2 * a.L + 1) + a.L + m) * a.R;
    C *gm = G + ((int64_t)k * (2 * a.L + 1) + a.L - m) * a.R;
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

// Smallest start l over the CTA (L + 1 when no thread has work).
__device__ __forceinline__ int block_min(int v) {
    __shared__ int s_min;
    if (threadIdx.x == 0) s_min = 0x7fffffff;
    __syncthreads();
    atomicMin(&s_min, v);
    __syncthreads();
    return s_min;
}

// ------------------------------------------------------------------ FP64
__global__ void __launch_bounds__(kNT) k_lcontract_f64(const LcArgs a) {
    __shared__ Coef64 rc[kLC64];
    __shared__ Acc64 ac[kLC64];
    int m, k, pc;
    block_mk(a, m, k, pc);
    const int neg = threadIdx.x >= kHalf;
    const int pair = pc * kHalf + (threadIdx.x & (kHalf - 1));
    const bool active = pair < a.npairs;
    const int64_t moff = (int64_t)m * (2 * a.L + 1 - m) / 2;
    const RTab64 *tab = a.tab64 + (int64_t)k * a.nalm + moff;

    double x = 0.0, y = 0.0, yo = 0.0;
    int ls = a.L + 1;
    if (active) {
        const int64_t si = start_index(a, k, m, neg, pair);
        ls = a.ls[si];
        const double2 s = a.st64[si];
        yo = s.x;
        y = s.y;
        x = a.xr[pair];
    }
    double2 acc1 = {0, 0}, acc2 = {0, 0};
    const int lstart = block_min(ls);
    // coefficient slots of this thread's sign
    const int bofs = neg ? 2 : 1;     // index of -b' (for +k) or +b' (for -k) in Coef64
    const int cofs = neg ? 2 : 0;     // first double2 of (ap, sam) or (am, sap) in Acc64
    for (int c0 = lstart; c0 <= a.L; c0 += kLC64) {
        const int nc = min(kLC64, a.L - c0 + 1);
        __syncthreads();
        for (int i = threadIdx.x; i < nc; i += kNT) {
            const int l = c0 + i;
            const RTab64 t = tab[l];
            rc[i] = Coef64{t.a, -t.b, t.b, 0.0};
            double2 ap = {0.0, 0.0}, am = {0.0, 0.0};
            for (int X = 0; X < a.ncomp; ++X) {
                double2 s = a.sky[X * a.nalm + moff + l];
                if (m == 0) s.y = 0.0;
                double2 b = a.beam[((int64_t)X * (a.K + 1) + k) * (a.L + 1) + l];
                if (k == 0) b.y = 0.0;
                ap.x += s.x * b.x + s.y * b.y;      // s conj(b)
                ap.y += s.y * b.x - s.x * b.y;
                am.x += s.x * b.x - s.y * b.y;      // conj(s) conj(b)
                am.y -= s.y * b.x + s.x * b.y;
            }
            const double c = t.c, sc = (l & 1) ? -c : c;
            ac[i] = Acc64{make_double2(c * ap.x, c * ap.y), make_double2(sc * am.x, sc * am.y),
                          make_double2(c * am.x, c * am.y), make_double2(sc * ap.x, sc * ap.y)};
        }
        __syncthreads();
        const int i0 = max(0, ls - c0);
        const double *rcd = reinterpret_cast<const double *>(rc);
        const double2 *acd = reinterpret_cast<const double2 *>(ac);
#pragma unroll 4
        for (int i = i0; i < nc; ++i) {
            const double ra = rcd[4 * i], rb = rcd[4 * i + bofs];
            const double2 c1 = acd[4 * i + cofs], c2 = acd[4 * i + cofs + 1];
            acc1.x = fma(c1.x, y, acc1.x);
            acc1.y = fma(c1.y, y, acc1.y);
            acc2.x = fma(c2.x, y, acc2.x);
            acc2.y = fma(c2.y, y, acc2.y);
            const double yn = fma(fma(ra, x, rb), y, -yo);
            yo = y;
            y = yn;
        }
    }
    if (active) write_two<double2>(a, m, k, pair, neg, acc1, acc2);
}

// ------------------------------------------------------------------ FP32
struct Stage32 {
    RTab32 t;
    float2 s[3], b[3];
};

__device__ __forceinline__ void stage_load(const LcArgs &a, const RTab32 *tab, int64_t moff, int m, int k, int l,
                                           Stage32 &st) {
    st.t = tab[l];
#pragma unroll
    for (int X = 0; X < 3; ++X) {
        if (X < a.ncomp) {
            st.s[X] = a.sky32[X * a.nalm + moff + l];
            st.b[X] = a.beam32[((int64_t)X * (a.K + 1) + k) * (a.L + 1) + l];
            if (m == 0) st.s[X].y = 0.f;
            if (k == 0) st.b[X].y = 0.f;
        } else {
            st.s[X] = make_float2(0.f, 0.f);
            st.b[X] = make_float2(0.f, 0.f);
        }
    }
}

struct __align__(16) Acc32 {
    float2 ap, sam, am, sap;
};

__device__ __forceinline__ void stage_store(const Stage32 &st, int l, float4 *rc, Acc32 *ac) {
    float2 ap = {0.f, 0.f}, am = {0.f, 0.f};
#pragma unroll
    for (int X = 0; X < 3; ++X) {
        const float2 s = st.s[X], b = st.b[X];
        ap.x += s.x * b.x + s.y * b.y;      // s conj(b)
        ap.y += s.y * b.x - s.x * b.y;
        am.x += s.x * b.x - s.y * b.y;      // conj(s) conj(b)
        am.y -= s.y * b.x + s.x * b.y;
    }
    const float c = st.t.c, sc = (l & 1) ? -c : c;
    *rc = make_float4(st.t.a, st.t.cp, st.t.cm, 0.f);
    *ac = Acc32{make_float2(c * ap.x, c * ap.y), make_float2(sc * am.x, sc * am.y),
                make_float2(c * am.x, c * am.y), make_float2(sc * ap.x, sc * ap.y)};
}

struct Rec32 {
    float yc, y, D;
    int ls;
    float2 acc1, acc2;
};

__device__ __forceinline__ void rec32_step(Rec32 &s, float ra, float rc_, float2 c1, float2 c2) {
    s.acc1.x = fmaf(c1.x, s.y, s.acc1.x);
    s.acc1.y = fmaf(c1.y, s.y, s.acc1.y);
    s.acc2.x = fmaf(c2.x, s.y, s.acc2.x);
    s.acc2.y = fmaf(c2.y, s.y, s.acc2.y);
    s.D = fmaf(fmaf(-ra, s.yc, rc_), s.y, s.D);
    s.y += s.D;
}

// PPT ring pairs per thread (consecutive pairs): each staged coefficient load
// feeds PPT recurrence steps.
template <int PPT>
__global__ void __launch_bounds__(kNT) k_lcontract_f32(const LcArgs a) {
    __shared__ float4 rc[2][kNT];   // a', c'+, c'-, unused
    __shared__ Acc32 ac[2][kNT];
    int m, k, pc;
    block_mk(a, m, k, pc);
    const int neg = threadIdx.x >= kHalf;
    const int p0 = pc * (PPT * kHalf) + PPT * (threadIdx.x & (kHalf - 1));
    const int64_t moff = (int64_t)m * (2 * a.L + 1 - m) / 2;
    const RTab32 *tab = a.tab32 + (int64_t)k * a.nalm + moff;

    Rec32 S[PPT];
    int lme = a.L + 1, lmx = 0;
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        S[q].ls = a.L + 1;
        S[q].acc1 = S[q].acc2 = make_float2(0.f, 0.f);
        S[q].y = S[q].D = S[q].yc = 0.f;
        if (p0 + q < a.npairs) {
            const int64_t si = start_index(a, k, m, neg, p0 + q);
            S[q].ls = a.ls[si];
            const float2 st2 = a.st32[si];
            S[q].y = st2.x;
            S[q].D = st2.y;
            S[q].yc = a.y32[p0 + q];
        }
        lme = min(lme, S[q].ls);
        lmx = max(lmx, S[q].ls);
    }
    const int lstart = block_min(lme);
    const int cofs = neg ? 2 : 0;
    Stage32 st;
    {
        const int l = lstart + (int)threadIdx.x;
        if (l <= a.L) {
            stage_load(a, tab, moff, m, k, l, st);
            stage_store(st, l, &rc[0][threadIdx.x], &ac[0][threadIdx.x]);
        }
    }
    int buf = 0;
    for (int c0 = lstart; c0 <= a.L; c0 += kNT, buf ^= 1) {
        const int nc = min(kNT, a.L - c0 + 1);
        const int ln = c0 + kNT + (int)threadIdx.x;   // this thread's l in the next chunk
        const bool next = ln <= a.L;
        if (next) stage_load(a, tab, moff, m, k, ln, st);
        __syncthreads();
        const float4 *rcv = rc[buf];
        // (c1, c2) = (ap, sam) for +k, (am, sap) for -k: one 16-byte load each step
        const float4 *acv = reinterpret_cast<const float4 *>(ac[buf]) + (cofs >> 1);
        int i = max(0, lme - c0);
        // until every ring of the thread has started
        for (; i < nc && c0 + i < lmx; ++i) {
            const float4 r = rcv[i], cc = acv[2 * i];
            const float ra = r.x, rcc = neg ? r.z : r.y;    // c'- for -k, c'+ for +k
            const float2 c1 = make_float2(cc.x, cc.y), c2 = make_float2(cc.z, cc.w);
#pragma unroll
            for (int q = 0; q < PPT; ++q)
                if (c0 + i >= S[q].ls) rec32_step(S[q], ra, rcc, c1, c2);
        }
#pragma unroll 2
        for (; i < nc; ++i) {
            const float4 r = rcv[i], cc = acv[2 * i];
            const float ra = r.x, rcc = neg ? r.z : r.y;    // c'- for -k, c'+ for +k
            const float2 c1 = make_float2(cc.x, cc.y), c2 = make_float2(cc.z, cc.w);
#pragma unroll
            for (int q = 0; q < PPT; ++q) rec32_step(S[q], ra, rcc, c1, c2);
        }
        if (next) stage_store(st, ln, &rc[buf ^ 1][threadIdx.x], &ac[buf ^ 1][threadIdx.x]);
    }
#pragma unroll
    for (int q = 0; q < PPT; ++q)
        if (p0 + q < a.npairs) write_two<float2>(a, m, k, p0 + q, neg, S[q].acc1, S[q].acc2);
}

// ------------------------------------------------------------------ DF64
// Per l, staged: a' and b' as double-float, then (ap, sam, am, sap), each
// complex as (Re hi, Re lo, Im hi, Im lo).
struct __align__(16) CoefDF {
    float4 ab;
    float4 c[4];
};

__device__ __forceinline__ float4 df4(double2 v) {
    const dfl re = df_from_d(v.x), im = df_from_d(v.y);
    return make_float4(re.h, re.l, im.h, im.l);
}

// One recurrence (ring pair, sign) of the double-float kernel.
struct RecDF {
    dfl x, y, yo;
    dacc a1r, a1i, a2r, a2i;
    int ls;
};

__device__ __forceinline__ void rec_df_start(const LcArgs &a, int k, int m, int neg, int pair, RecDF &r) {
    r.x = r.y = r.yo = dfl{0.f, 0.f};
    dacc_zero(r.a1r);
    dacc_zero(r.a1i);
    dacc_zero(r.a2r);
    dacc_zero(r.a2i);
    r.ls = a.L + 1;
    if (pair < a.npairs) {
        const int64_t si = start_index(a, k, m, neg, pair);
        r.ls = a.ls[si];
        const double2 s = a.st64[si];
        r.yo = df_from_d(s.x);
        r.y = df_from_d(s.y);
        r.x = df_from_d(a.xr[pair]);
    }
}

// accumulate with y_l, then y_{l+1} = (a' x -+ b') y_l - y_{l-1}
__device__ __forceinline__ void rec_df_step(RecDF &r, dfl ra, dfl rb, float4 c1, float4 c2) {
    dacc_mac(r.a1r, dfl{c1.x, c1.y}, r.y);
    dacc_mac(r.a1i, dfl{c1.z, c1.w}, r.y);
    dacc_mac(r.a2r, dfl{c2.x, c2.y}, r.y);
    dacc_mac(r.a2i, dfl{c2.z, c2.w}, r.y);
    const dfl t = df_fma(ra, r.x, rb);
    const dfl yn = df_fma(t, r.y, df_neg(r.yo));
    r.yo = r.y;
    r.y = yn;
}

__device__ __forceinline__ void rec_df_write(const LcArgs &a, int m, int k, int pair, int neg, const RecDF &r) {
    if (pair >= a.npairs) return;
    const double2 acc1 = make_double2(df_to_d(dacc_get(r.a1r)), df_to_d(dacc_get(r.a1i)));
    const double2 acc2 = make_double2(df_to_d(dacc_get(r.a2r)), df_to_d(dacc_get(r.a2i)));
    write_two<double2>(a, m, k, pair, neg, acc1, acc2);
}

// Two adjacent ring pairs per thread (they share every coefficient load).
__global__ void __launch_bounds__(kNT) k_lcontract_df(const LcArgs a) {
    __shared__ CoefDF cf[kLC64];
    int m, k, pc;
    block_mk(a, m, k, pc);
    const int neg = threadIdx.x >= kHalf;
    const int p0 = pc * (2 * kHalf) + 2 * (threadIdx.x & (kHalf - 1));
    const int64_t moff = (int64_t)m * (2 * a.L + 1 - m) / 2;
    const RTab64 *tab = a.tab64 + (int64_t)k * a.nalm + moff;

    RecDF A, B;
    rec_df_start(a, k, m, neg, p0, A);
    rec_df_start(a, k, m, neg, p0 + 1, B);
    const int lme = min(A.ls, B.ls), lmx = max(A.ls, B.ls);
    const int lstart = block_min(lme);
    const int cofs = neg ? 2 : 0;        // (ap, sam) for +k, (am, sap) for -k
    const float bsg = neg ? 1.f : -1.f;  // -b' for +k, +b' for -k
    for (int c0 = lstart; c0 <= a.L; c0 += kLC64) {
        const int nc = min(kLC64, a.L - c0 + 1);
        __syncthreads();
        for (int i = threadIdx.x; i < nc; i += kNT) {
            const int l = c0 + i;
            const RTab64 t = tab[l];
            double2 ap = {0.0, 0.0}, am = {0.0, 0.0};
            for (int X = 0; X < a.ncomp; ++X) {
                double2 s = a.sky[X * a.nalm + moff + l];
                if (m == 0) s.y = 0.0;
                double2 b = a.beam[((int64_t)X * (a.K + 1) + k) * (a.L + 1) + l];
                if (k == 0) b.y = 0.0;
                ap.x += s.x * b.x + s.y * b.y;      // s conj(b)
                ap.y += s.y * b.x - s.x * b.y;
                am.x += s.x * b.x - s.y * b.y;      // conj(s) conj(b)
                am.y -= s.y * b.x + s.x * b.y;
            }
            const double c = t.c, sc = (l & 1) ? -c : c;
            const dfl ra = df_from_d(t.a), rb = df_from_d(t.b);
            CoefDF v;
            v.ab = make_float4(ra.h, ra.l, rb.h, rb.l);
            v.c[0] = df4(make_double2(c * ap.x, c * ap.y));
            v.c[1] = df4(make_double2(sc * am.x, sc * am.y));
            v.c[2] = df4(make_double2(c * am.x, c * am.y));
            v.c[3] = df4(make_double2(sc * ap.x, sc * ap.y));
            cf[i] = v;
        }
        __syncthreads();
        int i = max(0, lme - c0);
        // until both recurrences have started
        for (; i < nc && c0 + i < lmx; ++i) {
            const float4 ab = cf[i].ab, c1 = cf[i].c[cofs], c2 = cf[i].c[cofs + 1];
            const dfl ra = dfl{ab.x, ab.y}, rb = dfl{bsg * ab.z, bsg * ab.w};
            if (c0 + i >= A.ls) rec_df_step(A, ra, rb, c1, c2);
            if (c0 + i >= B.ls) rec_df_step(B, ra, rb, c1, c2);
        }
#pragma unroll 2
        for (; i < nc; ++i) {
            const float4 ab = cf[i].ab, c1 = cf[i].c[cofs], c2 = cf[i].c[cofs + 1];
            const dfl ra = dfl{ab.x, ab.y}, rb = dfl{bsg * ab.z, bsg * ab.w};
            rec_df_step(A, ra, rb, c1, c2);
            rec_df_step(B, ra, rb, c1, c2);
        }
    }
    rec_df_write(a, m, k, p0, neg, A);
    rec_df_write(a, m, k, p0 + 1, neg, B);
}

__global__ void k_to_f32(const double2 *__restrict__ in, float2 *__restrict__ out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

sl_status launch_lcontract(sl_plan *p, const double *sky, const double *beam) {
    if (p->precision == SL_TF32X3)   // one sky on the tensor cores
        return launch_lcontract_mma(p, 1, sky, beam, p->d_sky32, (float2 *)p->d_G, p->d_err);
    LcArgs a;
    a.L = p->L;
    a.K = p->K;
    a.ncomp = p->ncomp;
    a.R = p->R;
    a.npairs = p->npairs;
    a.ppt = (p->precision == SL_FP64) ? 1 : (p->precision == SL_DF64 ? 2 : kF32Pairs);
    a.nchunk = (p->npairs + a.ppt * kHalf - 1) / (a.ppt * kHalf);
    a.nalm = p->nalm;
    a.sky = (const double2 *)sky;
    a.beam = (const double2 *)beam;
    a.sky32 = p->d_sky32;
    a.beam32 = p->d_beam32;
    a.xr = p->d_xr;
    a.y32 = p->d_y32;
    a.ls = p->d_ls;
    a.st64 = p->d_st64;
    a.st32 = p->d_st32;
    a.tab64 = p->d_tab64;
    a.tab32 = p->d_tab32;
    a.G = p->d_G;
    const int64_t nblk = (int64_t)(p->L + 1) * (p->K + 1) * a.nchunk;
    if (nblk > 0x7fffffff) return set_error(SL_ERR_UNSUPPORTED, "grid too large");
    int slot;
    if (p->precision == SL_DF64) {
        slot = timing_begin(p, "lcontract_df");
        k_lcontract_df<<<(unsigned)nblk, kNT, 0, p->stream>>>(a);
    } else if (p->precision == SL_FP64) {
        slot = timing_begin(p, "lcontract_f64");
        k_lcontract_f64<<<(unsigned)nblk, kNT, 0, p->stream>>>(a);
    } else {
        const int64_t ns = (int64_t)p->ncomp * p->nalm, nb = (int64_t)p->ncomp * (p->K + 1) * (p->L + 1);
        k_to_f32<<<(unsigned)std::min<int64_t>((ns + 255) / 256, 4096), 256, 0, p->stream>>>(
            (const double2 *)sky, p->d_sky32, ns);
        k_to_f32<<<(unsigned)std::min<int64_t>((nb + 255) / 256, 4096), 256, 0, p->stream>>>(
            (const double2 *)beam, p->d_beam32, nb);
        slot = timing_begin(p, "lcontract_f32");
        k_lcontract_f32<kF32Pairs><<<(unsigned)nblk, kNT, 0, p->stream>>>(a);
    }
    timing_end(p, slot);
    return cuda_check(cudaGetLastError(), "k_lcontract launch");
}

}  // namespace sl
