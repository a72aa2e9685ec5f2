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
// for the recurrence and 4 for the two complex x real sums.  FP32 plans: eight
// ring pairs per thread of one sign, two at a time in the lanes of packed FP32x2
// instructions (k_lcontract_f32); the recurrence in the
// difference form  D_{l+1} = (c'_l - a'_l y) y_l + D_l,  y_{l+1} = y_l + D_{l+1}
// with y = 1 - cos(theta) and c' = a' -+ b' - 2 formed in double (keeps the
// FP32 recurrence accurate near the pole, where cos theta alone carries too
// few bits); sky x beam products from FP32 copies of sky and beam.
// DF64 plans: the FP64 plan's layout and start states, with the recurrence
// and the sums in double-float arithmetic (df.cuh): per l, two double-float
// products and two sums for the recurrence and four double-float
// multiply-accumulates, all on the FP32 pipes.
// FP64 and DF64: the CTA stages the coefficients of a chunk of l in shared
// memory and a thread steps only from its own start l.  FP32: each warp stages
// its own coefficients, 32 l at a time, and steps from its earliest start
// (recurrences not yet started hold an exact zero state).
#include <algorithm>
#include <vector>

#include "df.cuh"
#include "sl_internal.cuh"

namespace sl {

constexpr int kNT = 256;          // threads per CTA
constexpr int kHalf = kNT / 2;    // threads per sign
constexpr int kNT32 = 128;        // threads per CTA of the FP32 contraction: 64 per sign of k,
constexpr int kHalf32 = kNT32 / 2;   // 2, 4 or 8 ring pairs each (lcontract_f32_ppt)
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

// Block b -> (m, k, ring chunk pc).
__device__ __forceinline__ void block_mk_of(const LcArgs &a, int b, int &m, int &k, int &pc) {
    pc = b % a.nchunk;
    b /= a.nchunk;
    k = b % (a.K + 1);
    m = b / (a.K + 1);
}
__device__ __forceinline__ void block_mk(const LcArgs &a, int &m, int &k, int &pc) { block_mk_of(a, blockIdx.x, m, k, pc); }

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

// Per staged l and sign of k, what a step needs: (-a', c') with c' = c'+ for
// +k and c'- for -k, and the two sums' coefficients (ap, sam) for +k, (am, sap)
// for -k.  Threads of a warp read the same l: three 8-byte broadcasts per l
// (16-byte broadcasts of pre-duplicated values cost more shared-memory
// wavefronts than the register moves they save).
struct __align__(8) Stage32x2 {
    float2 r, c1, c2;
};

__device__ __forceinline__ void stage_store(const Stage32 &st, int l, Stage32x2 *plus, Stage32x2 *minus) {
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
    const float na = -st.t.a;
    *plus = Stage32x2{make_float2(na, st.t.cp), make_float2(c * ap.x, c * ap.y), make_float2(sc * am.x, sc * am.y)};
    *minus = Stage32x2{make_float2(na, st.t.cm), make_float2(c * am.x, c * am.y), make_float2(sc * ap.x, sc * ap.y)};
}

// Two recurrences (two ring pairs of one sign) in the two lanes of packed FP32
// pairs: every operation below is one two-lane instruction (__ffma2_rn,
// __fadd2_rn) doing what the scalar form does per lane, with the same rounding.
struct Rec32x2 {
    float2 yc, y, D;                  // 1 - cos theta, value, difference
    float2 a1r, a1i, a2r, a2i;        // the two complex sums, split into re and im pairs
    float2 ys, Ds;                    // start states, injected at the start l
    int ls0, ls1;                     // start l of each lane (L + 1: never)
};

// One l step; the per-l values come duplicated into both lanes.
struct Coef32x2 {
    float2 na, cr, c1r, c1i, c2r, c2i;
};

__device__ __forceinline__ Coef32x2 coef32x2(const Stage32x2 &v) {
    return Coef32x2{make_float2(v.r.x, v.r.x), make_float2(v.r.y, v.r.y), make_float2(v.c1.x, v.c1.x),
                    make_float2(v.c1.y, v.c1.y), make_float2(v.c2.x, v.c2.x), make_float2(v.c2.y, v.c2.y)};
}

// One l step of packed pairs Q0 .. NP-1, stage by stage across them (independent
// instructions between each producer and its consumer); first, for pairs Q0 ..
// Q1-1, the start states of the lanes whose start l is l (selects: before its
// start a recurrence holds exact zeros, and stepping zeros adds exact zeros).
template <int NP, int Q0, int Q1>
__device__ __forceinline__ void rec32x2_steps(Rec32x2 (&S)[NP], const Coef32x2 &c, int l) {
#pragma unroll
    for (int q = Q0; q < Q1; ++q) {
        const bool j0 = l == S[q].ls0, j1 = l == S[q].ls1;
        S[q].y.x = j0 ? S[q].ys.x : S[q].y.x;
        S[q].D.x = j0 ? S[q].Ds.x : S[q].D.x;
        S[q].y.y = j1 ? S[q].ys.y : S[q].y.y;
        S[q].D.y = j1 ? S[q].Ds.y : S[q].D.y;
    }
    float2 t[NP];
#pragma unroll
    for (int q = Q0; q < NP; ++q) t[q] = __ffma2_rn(c.na, S[q].yc, c.cr);
#pragma unroll
    for (int q = Q0; q < NP; ++q) {
        S[q].a1r = __ffma2_rn(c.c1r, S[q].y, S[q].a1r);
        S[q].a1i = __ffma2_rn(c.c1i, S[q].y, S[q].a1i);
    }
#pragma unroll
    for (int q = Q0; q < NP; ++q) S[q].D = __ffma2_rn(t[q], S[q].y, S[q].D);
#pragma unroll
    for (int q = Q0; q < NP; ++q) {
        S[q].a2r = __ffma2_rn(c.c2r, S[q].y, S[q].a2r);
        S[q].a2i = __ffma2_rn(c.c2i, S[q].y, S[q].a2i);
    }
#pragma unroll
    for (int q = Q0; q < NP; ++q) S[q].y = __fadd2_rn(S[q].y, S[q].D);
}

// Ramp steps i .. iend-1 of a batch with the last NA packed pairs begun, the last
// NB of them with every lane started (no injection left for those).
template <int NP, int NA, int NB>
__device__ __forceinline__ void rec32x2_ramp_loop(int &i, int iend, Rec32x2 (&S)[NP], const Stage32x2 *sv, int c0) {
    for (; i < iend; ++i) rec32x2_steps<NP, NP - NA, NP - NB>(S, coef32x2(sv[i]), c0 + i);
}
template <int NP>
__device__ __forceinline__ void rec32x2_ramp(int na, int nb, int &i, int iend, Rec32x2 (&S)[NP],
                                             const Stage32x2 *sv, int c0) {
#define SL_RAMP(A, B)                                                                                  \
    if constexpr (A <= NP && B <= A)                                                                   \
        if (na == A && nb == B) {                                                                      \
            rec32x2_ramp_loop<NP, (A <= NP ? A : 1), (A <= NP && B <= A ? B : 0)>(i, iend, S, sv, c0); \
            return;                                                                                    \
        }
    SL_RAMP(1, 0) SL_RAMP(1, 1) SL_RAMP(2, 0) SL_RAMP(2, 1) SL_RAMP(2, 2) SL_RAMP(3, 0) SL_RAMP(3, 1)
    SL_RAMP(3, 2) SL_RAMP(3, 3) SL_RAMP(4, 0) SL_RAMP(4, 1) SL_RAMP(4, 2) SL_RAMP(4, 3) SL_RAMP(4, 4)
#undef SL_RAMP
    i = iend;   // not reached: 1 <= na <= NP, 0 <= nb <= na
}

__device__ __forceinline__ void rec32x2_step(Rec32x2 &s, const Coef32x2 &c) {
    // sums with y_l: re/im of c1 y, c2 y
    s.a1r = __ffma2_rn(c.c1r, s.y, s.a1r);
    s.a1i = __ffma2_rn(c.c1i, s.y, s.a1i);
    s.a2r = __ffma2_rn(c.c2r, s.y, s.a2r);
    s.a2i = __ffma2_rn(c.c2i, s.y, s.a2i);
    // D_{l+1} = (c' - a' y_c) y_l + D_l,  y_{l+1} = y_l + D_{l+1}
    const float2 t = __ffma2_rn(c.na, s.yc, c.cr);
    s.D = __ffma2_rn(t, s.y, s.D);
    s.y = __fadd2_rn(s.y, s.D);
}

// PPT ring pairs per thread, two per packed recurrence.  A warp owns 32 * PPT
// consecutive ring pairs of one sign of k; packed pair q of lane j holds pairs
// base + 64 q + j (low lane) and base + 64 q + 32 + j (high lane), so that the
// 32 lanes of one packed pair cover 64 neighbouring rings, whose recurrences
// start at similar l (the start moves with the ring's distance from the pole).
// Until its start l a recurrence holds an exact zero state (it then adds exact
// zeros to its sums), and at the start l its start state is injected; packed
// pair q is not stepped at all before the earliest start among its lanes (a
// warp-uniform test), and the loop bounds are the warp's earliest and latest
// starts, so the lanes never diverge.  Each warp stages its own coefficients,
// 32 l at a time (one l per lane, double-buffered, the next batch loaded while
// the current one is used): no CTA-wide barrier, every warp runs from its own
// first start.  Each coefficient load from shared memory feeds PPT recurrence
// steps.
//
// lcontract_f32_warp runs one warp's share of one CTA block (the block index
// as in k_lcontract_f32; wpart = the warp's index in the block: 0-1 for +k,
// 2-3 for -k) with its staging buffers stw; the warps of a block are
// independent of each other.
template <int PPT>
__device__ __forceinline__ void lcontract_f32_warp(const LcArgs &a, int block, int wpart, Stage32x2 (*stw)[32]) {
    constexpr int NP = PPT / 2;
    int m, k, pc;
    block_mk_of(a, block, m, k, pc);
    const int neg = wpart >= 2;
    const int lane = threadIdx.x & 31, wsign = wpart & 1;
    const int base = pc * (PPT * kHalf32) + wsign * (32 * PPT);
    const int64_t moff = (int64_t)m * (2 * a.L + 1 - m) / 2;
    const RTab32 *tab = a.tab32 + (int64_t)k * a.nalm + moff;

    Rec32x2 S[NP];
    int qmin[NP];   // earliest start among the lanes of packed pair q (warp-uniform)
    int lme = a.L + 1, lmx = 0;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        float st[2][3];
        int ls[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int pair = base + 64 * q + 32 * h + lane;
            ls[h] = a.L + 1;
            st[h][0] = st[h][1] = st[h][2] = 0.f;
            if (pair < a.npairs) {
                const int64_t si = start_index(a, k, m, neg, pair);
                ls[h] = a.ls[si];
                const float2 st2 = a.st32[si];
                st[h][0] = st2.x;
                st[h][1] = st2.y;
                st[h][2] = a.y32[pair];
            }
        }
        S[q].ls0 = ls[0];
        S[q].ls1 = ls[1];
        S[q].ys = make_float2(st[0][0], st[1][0]);
        S[q].Ds = make_float2(st[0][1], st[1][1]);
        S[q].yc = make_float2(st[0][2], st[1][2]);
        S[q].y = S[q].D = make_float2(0.f, 0.f);
        S[q].a1r = S[q].a1i = S[q].a2r = S[q].a2i = make_float2(0.f, 0.f);
        qmin[q] = __reduce_min_sync(0xffffffffu, min(ls[0], ls[1]));
        lme = min(lme, qmin[q]);
        lmx = max(lmx, max(ls[0], ls[1]));
    }
    lmx = __reduce_max_sync(0xffffffffu, lmx);
    int qmax[NP];   // latest start among the lanes of packed pair q that start at all (warp-uniform)
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        const int s0 = S[q].ls0 <= a.L ? S[q].ls0 : -1, s1 = S[q].ls1 <= a.L ? S[q].ls1 : -1;
        qmax[q] = __reduce_max_sync(0xffffffffu, max(s0, s1));
    }
    // the packed pairs' earliest starts usually descend with q (ring pairs nearer the
    // equator start earlier): then they begin in the order NP-1, NP-2, .. 0 (warp-uniform)
    bool qdesc = true;
#pragma unroll
    for (int q = 1; q < NP; ++q) qdesc = qdesc && qmin[q] <= qmin[q - 1];
    Stage32 st;
    Stage32x2 dummy;
    auto stage_mine = [&](int l, Stage32x2 *dst) {   // this warp's sign only
        if (neg) stage_store(st, l, &dummy, dst);
        else stage_store(st, l, dst, &dummy);
    };
    if (lme + lane <= a.L) {
        stage_load(a, tab, moff, m, k, lme + lane, st);
        stage_mine(lme + lane, &stw[0][lane]);
    }
    int buf = 0;
    for (int c0 = lme; c0 <= a.L; c0 += 32, buf ^= 1) {
        const int nc = min(32, a.L - c0 + 1);
        const int ln = c0 + 32 + lane;   // this lane's l in the next batch
        const bool next = ln <= a.L;
        if (next) stage_load(a, tab, moff, m, k, ln, st);
        __syncwarp();
        const Stage32x2 *sv = stw[buf];
        int i = 0;
        // until every recurrence of the warp has started (up to and including the
        // last start l): inject start states; packed pairs none of whose lanes has
        // started are not stepped
        if (qdesc) {
            // in segments: the last na pairs begun, the last nb of them with every lane
            // started; those na step together, interleaved, and only the na - nb still
            // starting pay for the injection selects
            while (i < nc && c0 + i <= lmx) {
                const int l = c0 + i;
                int na = 0, nb = 0, lnext = lmx + 1;
                bool run = true;
#pragma unroll
                for (int q = NP - 1; q >= 0; --q)
                    if (run) {
                        if (qmin[q] <= l) ++na;
                        else { lnext = min(lnext, qmin[q]); run = false; }
                    }
                run = true;
#pragma unroll
                for (int q = NP - 1; q >= 0; --q)
                    if (run && q >= NP - na) {
                        if (qmax[q] < l) ++nb;
                        else { lnext = min(lnext, qmax[q] + 1); run = false; }
                    }
                rec32x2_ramp<NP>(na, nb, i, min(nc, lnext - c0), S, sv, c0);
            }
        } else {
            for (; i < nc && c0 + i <= lmx; ++i) {
                const int l = c0 + i;
                const Coef32x2 c = coef32x2(sv[i]);
#pragma unroll
                for (int q = 0; q < NP; ++q) {
                    if (l < qmin[q]) continue;
                    if (l == S[q].ls0) { S[q].y.x = S[q].ys.x; S[q].D.x = S[q].Ds.x; }
                    if (l == S[q].ls1) { S[q].y.y = S[q].ys.y; S[q].D.y = S[q].Ds.y; }
                    rec32x2_step(S[q], c);
                }
            }
        }
#pragma unroll 2
        for (; i < nc; ++i) rec32x2_steps<NP, 0, 0>(S, coef32x2(sv[i]), c0 + i);
        __syncwarp();   // the batch is read before the other buffer is overwritten next time round
        if (next) stage_mine(ln, &stw[buf ^ 1][lane]);
    }
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        const int pair = base + 64 * q + lane;
        if (pair < a.npairs)
            write_two<float2>(a, m, k, pair, neg, make_float2(S[q].a1r.x, S[q].a1i.x), make_float2(S[q].a2r.x, S[q].a2i.x));
        if (pair + 32 < a.npairs)
            write_two<float2>(a, m, k, pair + 32, neg, make_float2(S[q].a1r.y, S[q].a1i.y),
                              make_float2(S[q].a2r.y, S[q].a2i.y));
    }
}

// One block per (m, k, ring chunk); warp w takes part w.
template <int PPT>
__global__ void __launch_bounds__(kNT32, 4) k_lcontract_f32(const LcArgs a) {
    __shared__ Stage32x2 stg[kNT32 / 32][2][32];   // [warp][buffer][l in batch]
    const int warp = threadIdx.x >> 5;
    lcontract_f32_warp<PPT>(a, blockIdx.x, warp, stg[warp]);
}

// Ring pairs per thread of the FP32 contraction for a grid of npairs northern
// rings: the variant (2, 4 or 8, i.e. 128, 256 or 512 ring pairs per block)
// that leaves the fewest threads idle, the larger on a tie.
int lcontract_f32_ppt(int npairs) {
    int best = 8;
    double best_idle = 2.0;
    for (int ppt : {8, 4, 2}) {
        const int per = ppt * kHalf32;
        const int nb = (npairs + per - 1) / per;
        const double idle = 1.0 - (double)npairs / ((double)nb * per);
        if (idle < best_idle - 1e-9) {
            best_idle = idle;
            best = ppt;
        }
    }
    return best;
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

// The contraction's arguments for plan p (ppt and nchunk as its kernels use them).
static void make_lcargs(const sl_plan *p, const double *sky, const double *beam, LcArgs &a) {
    a.L = p->L;
    a.K = p->K;
    a.ncomp = p->ncomp;
    a.R = p->R;
    a.npairs = p->npairs;
    a.ppt = (p->precision == SL_FP64) ? 1
          : (p->precision == SL_DF64 ? 2 : (p->lc_ppt ? p->lc_ppt : lcontract_f32_ppt(p->npairs)));
    const int half = plan_fp32(p->precision) ? kHalf32 : kHalf;   // ring pairs per sign of a CTA / ppt
    a.nchunk = (p->npairs + a.ppt * half - 1) / (a.ppt * half);
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
}

// FP32 copies of a plan's sky and beam (the FP32 contraction reads them).
static sl_status launch_to_f32(sl_plan *p, cudaStream_t s, const double *sky, const double *beam) {
    const int64_t ns = (int64_t)p->ncomp * p->nalm, nb = (int64_t)p->ncomp * (p->K + 1) * (p->L + 1);
    k_to_f32<<<(unsigned)std::min<int64_t>((ns + 255) / 256, 4096), 256, 0, s>>>((const double2 *)sky, p->d_sky32, ns);
    k_to_f32<<<(unsigned)std::min<int64_t>((nb + 255) / 256, 4096), 256, 0, s>>>((const double2 *)beam, p->d_beam32, nb);
    return cuda_check(cudaGetLastError(), "k_to_f32 launch");
}

sl_status launch_lcontract(sl_plan *p, const double *sky, const double *beam) {
    if (p->precision == SL_TF32X3)   // one sky on the tensor cores
        return launch_lcontract_mma(p, 1, sky, beam, p->d_sky32, (float2 *)p->d_G, p->d_err);
    LcArgs a;
    make_lcargs(p, sky, beam, a);
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
        sl_status st = launch_to_f32(p, p->stream, sky, beam);
        if (st != SL_OK) return st;
        slot = timing_begin(p, "lcontract_f32");
        if (a.ppt == 8) k_lcontract_f32<8><<<(unsigned)nblk, kNT32, 0, p->stream>>>(a);
        else if (a.ppt == 4) k_lcontract_f32<4><<<(unsigned)nblk, kNT32, 0, p->stream>>>(a);
        else k_lcontract_f32<2><<<(unsigned)nblk, kNT32, 0, p->stream>>>(a);
    }
    timing_end(p, slot);
    return cuda_check(cudaGetLastError(), "k_lcontract launch");
}

// ------------------------------------------------------------------ many detectors
// Persistent launches for the FP32 contractions of up to kMaxBatchDets plans
// (detectors with their own lmax, kmax, grids, skies and beams): one launch
// per number of ring pairs per thread among them (one kernel variant each, at
// its full occupancy), the launches side by side on their own streams.  Every
// warp takes (block, part) units -- the part of a k_lcontract_f32 block one
// warp runs -- from its launch's counter over the launch's items, ordered by
// decreasing cost, and runs it with its detector's arguments (kernel
// parameters).  A block's four parts are independent and the launches share
// nothing, so no warp ever waits for another; the order balances the tail
// (largest blocks first), and a launch's CTAs take the SMs that another's
// finished CTAs leave.  (Claiming whole blocks per CTA, so that a block's four
// warps share L1, measured slower: the CTA then waits for its slowest warp.)
struct LcBatchArgs {
    int ndet, nitems;
    const LcBatchItem *items;
    unsigned *counter;                // zeroed before the launch
    LcArgs d[kMaxBatchDets];
};

template <int PPT>
__global__ void __launch_bounds__(kNT32, 4) k_lcontract_f32_batch(const __grid_constant__ LcBatchArgs B) {
    __shared__ Stage32x2 stg[kNT32 / 32][2][32];   // [warp][buffer][l in batch]
    // the detectors' arguments, copied once from the kernel parameters: read at a
    // run-time index, they are shared-memory loads instead of constant-cache misses
    __shared__ __align__(16) LcArgs s_args[kMaxBatchDets];
    static_assert(sizeof(LcArgs) % sizeof(int) == 0, "LcArgs copied as ints");
    {
        const int *src = reinterpret_cast<const int *>(B.d);
        int *dst = reinterpret_cast<int *>(s_args);
        const int nw = B.ndet * (int)(sizeof(LcArgs) / sizeof(int));
        for (int w = threadIdx.x; w < nw; w += blockDim.x) dst[w] = src[w];
        __syncthreads();
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned nunits = 4u * (unsigned)B.nitems;
    unsigned u = 0;
    if (lane == 0) u = atomicAdd(B.counter, 1u);
    u = __shfl_sync(0xffffffffu, u, 0);
    while (u < nunits) {
        // the next unit is claimed before this one runs: the atomic's round trip
        // overlaps the work instead of preceding it
        unsigned un = 0;
        if (lane == 0) un = atomicAdd(B.counter, 1u);
        const LcBatchItem it = B.items[u >> 2];
        lcontract_f32_warp<PPT>(s_args[it.det], it.block, (int)(u & 3u), stg[warp]);
        __syncwarp();
        u = __shfl_sync(0xffffffffu, un, 0);
    }
}

// Work items: every block of every detector, grouped by the detector's ring
// pairs per thread (8, 4, 2), each group by decreasing cost; counts[g] items in
// group g.
sl_status lcontract_f32_batch_items(sl_plan *const *plans, int n, std::vector<LcBatchItem> &items,
                                    int counts[kLcBatchGroups]) {
    items.clear();
    for (int g = 0; g < kLcBatchGroups; ++g) counts[g] = 0;
    for (int d = 0; d < n; ++d) {
        const sl_plan *p = plans[d];
        if (!plan_fp32(p->precision) || p->precision == SL_TF32X3)
            return set_error(SL_ERR_UNSUPPORTED, "batched contraction: plan %d is not an SL_FP32 plan", d);
        LcArgs a;
        make_lcargs(p, nullptr, nullptr, a);
        const int per = a.ppt * kHalf32;
        for (int m = 0; m <= p->L; ++m)
            for (int k = 0; k <= p->K; ++k)
                for (int c = 0; c < a.nchunk; ++c) {
                    // recurrence steps of the block (the evanescent zone ignored): l from max(m, k) to L
                    const int pairs = std::min(per, p->npairs - c * per);
                    const float cost = (float)(p->L + 1 - std::max(m, k)) * (float)pairs;
                    items.push_back(LcBatchItem{d, (m * (p->K + 1) + k) * a.nchunk + c, a.ppt, cost});
                }
    }
    // within a group: detector by detector (the largest first), each in block order
    // as a k_lcontract_f32 grid runs it -- the (m, k) blocks of one detector that
    // run together share its sky rows in L2 -- except that the detector's last
    // blocks wait for the end of the group
    std::vector<double> dcost(n, 0.0);
    for (const LcBatchItem &it : items) dcost[it.det] += it.cost;
    std::stable_sort(items.begin(), items.end(), [&](const LcBatchItem &x, const LcBatchItem &y) {
        if (x.ppt != y.ppt) return x.ppt > y.ppt;
        if (x.det != y.det) return dcost[x.det] != dcost[y.det] ? dcost[x.det] > dcost[y.det] : x.det < y.det;
        return false;
    });
    for (const LcBatchItem &it : items) ++counts[it.ppt == 8 ? 0 : (it.ppt == 4 ? 1 : 2)];
    return SL_OK;
}

int lcontract_f32_group(const sl_plan *p) {
    const int ppt = p->lc_ppt ? p->lc_ppt : lcontract_f32_ppt(p->npairs);
    return ppt == 8 ? 0 : (ppt == 4 ? 1 : 2);
}

sl_status launch_lcontract_f32_batch(cudaStream_t stream, const cudaStream_t *gstream, const cudaEvent_t *gdone,
                                     cudaEvent_t ready, sl_plan *const *plans, const double *const *sky,
                                     const double *const *beam, int n, const LcBatchItem *items,
                                     const int counts[kLcBatchGroups], unsigned *counters) {
    if (n < 1 || n > kMaxBatchDets) return set_error(SL_ERR_ARG, "batched contraction: %d plans (1..%d)", n, kMaxBatchDets);
    LcBatchArgs B;
    B.ndet = n;
    for (int d = 0; d < n; ++d) {
        sl_status st = launch_to_f32(plans[d], stream, sky[d], beam[d]);
        if (st != SL_OK) return st;
        make_lcargs(plans[d], sky[d], beam[d], B.d[d]);
    }
    sl_status st = cuda_check(cudaMemsetAsync(counters, 0, kLcBatchGroups * sizeof(unsigned), stream), "batch counters");
    if (st == SL_OK) st = cuda_check(cudaEventRecord(ready, stream), "batch counters ready");
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, plans[0]->device);
    int first = 0;
    for (int g = 0; g < kLcBatchGroups && st == SL_OK; first += counts[g], ++g) {
        if (counts[g] == 0) continue;
        void (*kern)(const LcBatchArgs) = g == 0 ? k_lcontract_f32_batch<8>
                                        : (g == 1 ? k_lcontract_f32_batch<4> : k_lcontract_f32_batch<2>);
        int per_sm = 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kNT32, 0);
        if (per_sm < 1) per_sm = 1;
        B.items = items + first;
        B.nitems = counts[g];
        B.counter = counters + g;
        const cudaStream_t s = gstream[g];
        st = cuda_check(cudaStreamWaitEvent(s, ready, 0), "batch group stream");
        if (st != SL_OK) break;
        kern<<<(unsigned)(nsm * per_sm), kNT32, 0, s>>>(B);
        st = cuda_check(cudaGetLastError(), "k_lcontract_f32_batch launch");
        if (st == SL_OK) st = cuda_check(cudaEventRecord(gdone[g], s), "batch group done");
    }
    return st;
}

}  // namespace sl
