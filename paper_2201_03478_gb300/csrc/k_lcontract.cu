// k_lcontract.cu -- the spin "Legendre" step of the cube (Sect. 2.1, Eqs. c_m
// and S):
//
//   G_k(r, m) = sum_{l >= max(|m|, k)} A_{k,lm} d^l_{mk}(theta_r),
//   A_{k,lm}  = sum_X s^X_lm conj(b^X_lk),      m in [-L, L], k in [0, K],
//
// written to G[k][r][m + L].
//
// One CTA per (m >= 0, k, block of north rings); one thread per north ring r.
// Each thread runs two l-recurrences, d^l_{m,+k}(theta_r) and d^l_{m,-k}(theta_r),
// and from them produces four outputs through the reflection identities
//   d^l_{-m,k}(t)    = (-1)^{m+k} d^l_{m,-k}(t)
//   d^l_{ m,k}(pi-t) = (-1)^{l+m} d^l_{m,-k}(t)
//   d^l_{-m,k}(pi-t) = (-1)^{l-k} d^l_{m, k}(t)
// and the sky's real-field relation s_{l,-m} = (-1)^m conj(s_lm):
//   G(north, +m) =               sum_l A+_l d1_l
//   G(south, +m) = (-1)^m        sum_l (-1)^l A+_l d2_l
//   G(north, -m) = (-1)^k        sum_l A-_l d2_l
//   G(south, -m) = (-1)^{m+k}    sum_l (-1)^l A-_l d1_l
// with A+_l = sum_X s conj(b), A-_l = sum_X conj(s) conj(b), d1 = d_{m,+k},
// d2 = d_{m,-k}.  The recurrence (in l, at fixed m, k):
//   d^{l+1} = (alpha_l x - beta_l) d^l - gamma_l d^{l-1},   x = cos(theta),
//   alpha_l = (2l+1)(l+1)/sqrt(((l+1)^2-m^2)((l+1)^2-k^2)),
//   beta_l  = (2l+1) m k /(l sqrt(...)),  gamma_l = (l+1) sqrt((l^2-m^2)(l^2-k^2))/(l sqrt(...)),
// (beta changes sign with k).  The CTA stages alpha, beta, gamma and the four
// signed coefficients for a chunk of l in shared memory; every thread then
// steps its two recurrences through the chunk.
//
// FP64 plans: the recurrence and the sums in double.  FP32 plans: the
// coefficients are formed in double and rounded; the recurrence runs in the
// difference form  D_{l+1} = (c_l - alpha_l y) d_l + gamma_l D_l,
// d_{l+1} = d_l + D_{l+1}, with y = 1 - cos(theta) and c_l = alpha_l -+ beta_l
// - gamma_l - 1 formed in double, which keeps the FP32 recurrence accurate
// near the pole, where cos(theta) alone carries too few bits.
#include "sl_internal.cuh"

namespace sl {

constexpr int kLC = 64;     // l values staged per chunk
constexpr int kNT = 256;    // threads (north rings) per CTA

struct __align__(32) Rec64 {
    double a, b, g, pad;
};
struct __align__(16) Acc64 {
    double2 ap, am, sap, sam;
};
struct __align__(16) Rec32 {
    float a, cp, cm, g;
};
struct __align__(16) Acc32 {
    float2 ap, am, sap, sam;
};

struct LcArgs {
    int L, K, ncomp, R, npairs, nchunk;
    int64_t nalm;
    const double2 *sky, *beam;
    const double *xr;
    const float *y32;
    const double2 *seed;
    const int2 *seed_e;
    void *G;
};

// Recurrence coefficients of the step l -> l+1 and the signed A coefficients,
// computed in double.
__device__ __forceinline__ void make_coefs(const LcArgs &a, int m, int k, int l, double &al,
                                           double &be, double &ga, double2 &ap, double2 &am) {
    const double lp = l + 1.0, ll = (double)l, dm = (double)m, dk = (double)k;
    const double A = (lp * lp - dm * dm) * (lp * lp - dk * dk);
    const double ra = 1.0 / sqrt(A);
    al = (2.0 * l + 1.0) * lp * ra;
    if (l > 0) {
        const double B = (ll * ll - dm * dm) * (ll * ll - dk * dk);
        be = (2.0 * l + 1.0) * dm * dk * ra / ll;
        ga = lp * sqrt(B) * ra / ll;
    } else {
        be = 0.0;
        ga = 0.0;
    }
    ap = make_double2(0.0, 0.0);
    am = make_double2(0.0, 0.0);
    const int64_t moff = (int64_t)m * (2 * a.L + 1 - m) / 2;
    for (int X = 0; X < a.ncomp; ++X) {
        double2 s = a.sky[X * a.nalm + moff + l];
        if (m == 0) s.y = 0.0;
        double2 b = a.beam[((int64_t)X * (a.K + 1) + k) * (a.L + 1) + l];
        if (k == 0) b.y = 0.0;
        // s conj(b)
        ap.x += s.x * b.x + s.y * b.y;
        ap.y += s.y * b.x - s.x * b.y;
        // conj(s) conj(b)
        am.x += s.x * b.x - s.y * b.y;
        am.y -= s.y * b.x + s.x * b.y;
    }
}

__device__ __forceinline__ void block_mk(const LcArgs &a, int &m, int &k, int &pair) {
    int b = blockIdx.x;
    const int pc = b % a.nchunk;
    b /= a.nchunk;
    k = b % (a.K + 1);
    m = b / (a.K + 1);
    pair = pc * kNT + threadIdx.x;
}

template <typename C>
__device__ __forceinline__ void write_out(const LcArgs &a, int m, int k, int pair, C NP, C SP, C NM, C SM) {
    C *G = reinterpret_cast<C *>(a.G);
    const int rn = pair, rs = a.R - 1 - pair;
    const int64_t row = 2 * (int64_t)a.L + 1;
    const int64_t base = (int64_t)k * a.R;
    const bool modd = m & 1, kodd = k & 1;
    G[(base + rn) * row + a.L + m] = NP;
    if (rs != rn) {
        if (modd) { SP.x = -SP.x; SP.y = -SP.y; }
        G[(base + rs) * row + a.L + m] = SP;
    }
    if (m > 0) {
        if (kodd) { NM.x = -NM.x; NM.y = -NM.y; }
        G[(base + rn) * row + a.L - m] = NM;
        if (rs != rn) {
            if (modd != kodd) { SM.x = -SM.x; SM.y = -SM.y; }
            G[(base + rs) * row + a.L - m] = SM;
        }
    }
}

// ------------------------------------------------------------------ FP64
__global__ void __launch_bounds__(kNT) k_lcontract_f64(const LcArgs a) {
    __shared__ Rec64 rc[kLC];
    __shared__ Acc64 ac[kLC];
    int m, k, pair;
    block_mk(a, m, k, pair);
    const int l0 = max(m, k);
    const bool active = pair < a.npairs;

    double x = 0.0, d1 = 0.0, d1o = 0.0, d2 = 0.0, d2o = 0.0;
    int e1 = 0, e2 = 0;
    double2 NP = {0, 0}, SP = {0, 0}, NM = {0, 0}, SM = {0, 0};
    if (active) {
        x = a.xr[pair];
        const int64_t si = ((int64_t)k * (a.L + 1) + m) * a.npairs + pair;
        const double2 sv = a.seed[si];
        const int2 se = a.seed_e[si];
        d1 = sv.x;
        e1 = se.x;
        d2 = sv.y;
        e2 = se.y;
    }
    for (int c0 = l0; c0 <= a.L; c0 += kLC) {
        const int nc = min(kLC, a.L - c0 + 1);
        __syncthreads();
        for (int i = threadIdx.x; i < nc; i += kNT) {
            const int l = c0 + i;
            double al, be, ga;
            double2 ap, am;
            make_coefs(a, m, k, l, al, be, ga, ap, am);
            rc[i] = Rec64{al, be, ga, 0.0};
            const double sg = (l & 1) ? -1.0 : 1.0;
            ac[i] = Acc64{ap, am, make_double2(sg * ap.x, sg * ap.y), make_double2(sg * am.x, sg * am.y)};
        }
        __syncthreads();
        if (!active) continue;
        int i = 0;
        // scaled phase: values below 2^-300 are carried with an exponent
        for (; i < nc && (e1 < 0 || e2 < 0); ++i) {
            const Rec64 r = rc[i];
            const Acc64 c = ac[i];
            if (e1 == 0) {
                NP.x = fma(c.ap.x, d1, NP.x);
                NP.y = fma(c.ap.y, d1, NP.y);
                SM.x = fma(c.sam.x, d1, SM.x);
                SM.y = fma(c.sam.y, d1, SM.y);
            }
            if (e2 == 0) {
                NM.x = fma(c.am.x, d2, NM.x);
                NM.y = fma(c.am.y, d2, NM.y);
                SP.x = fma(c.sap.x, d2, SP.x);
                SP.y = fma(c.sap.y, d2, SP.y);
            }
            const double n1 = fma(fma(r.a, x, -r.b), d1, -r.g * d1o);
            const double n2 = fma(fma(r.a, x, r.b), d2, -r.g * d2o);
            d1o = d1;
            d1 = n1;
            d2o = d2;
            d2 = n2;
            if (e1 < 0 && fabs(d1) > kScaleThr) {
                d1 *= kScaleDn;
                d1o *= kScaleDn;
                ++e1;
            }
            if (e2 < 0 && fabs(d2) > kScaleThr) {
                d2 *= kScaleDn;
                d2o *= kScaleDn;
                ++e2;
            }
        }
#pragma unroll 4
        for (; i < nc; ++i) {
            const Rec64 r = rc[i];
            const Acc64 c = ac[i];
            NP.x = fma(c.ap.x, d1, NP.x);
            NP.y = fma(c.ap.y, d1, NP.y);
            SM.x = fma(c.sam.x, d1, SM.x);
            SM.y = fma(c.sam.y, d1, SM.y);
            NM.x = fma(c.am.x, d2, NM.x);
            NM.y = fma(c.am.y, d2, NM.y);
            SP.x = fma(c.sap.x, d2, SP.x);
            SP.y = fma(c.sap.y, d2, SP.y);
            const double n1 = fma(fma(r.a, x, -r.b), d1, -r.g * d1o);
            const double n2 = fma(fma(r.a, x, r.b), d2, -r.g * d2o);
            d1o = d1;
            d1 = n1;
            d2o = d2;
            d2 = n2;
        }
    }
    if (active) write_out<double2>(a, m, k, pair, NP, SP, NM, SM);
}

// ------------------------------------------------------------------ FP32
__device__ __forceinline__ void to_scaled32(double v, int e600, float &mant, int &e64) {
    // value = v * 2^(600 e600) -> mant * 2^(64 e64), |mant| >= 2^-32 while e64 < 0
    if (v == 0.0) {
        mant = 0.f;
        e64 = 0;
        return;
    }
    int ex;
    const double f = frexp(v, &ex);       // v = f 2^ex, |f| in [0.5, 1)
    long tot = (long)ex + 600L * e600;
    int e = 0;
    if (tot < -32) {
        const long nsteps = (-32 - tot + 63) / 64;
        tot += 64 * nsteps;
        e = -(int)nsteps;
    }
    mant = (float)ldexp(f, (int)tot);
    e64 = e;
}

__global__ void __launch_bounds__(kNT) k_lcontract_f32(const LcArgs a) {
    __shared__ Rec32 rc[kLC];
    __shared__ Acc32 ac[kLC];
    int m, k, pair;
    block_mk(a, m, k, pair);
    const int l0 = max(m, k);
    const bool active = pair < a.npairs;

    float y = 0.f, d1 = 0.f, D1 = 0.f, d2 = 0.f, D2 = 0.f;
    int e1 = 0, e2 = 0;
    float2 NP = {0, 0}, SP = {0, 0}, NM = {0, 0}, SM = {0, 0};
    if (active) {
        y = a.y32[pair];
        const int64_t si = ((int64_t)k * (a.L + 1) + m) * a.npairs + pair;
        const double2 sv = a.seed[si];
        const int2 se = a.seed_e[si];
        to_scaled32(sv.x, se.x, d1, e1);
        to_scaled32(sv.y, se.y, d2, e2);
        D1 = d1;   // d^{l0-1} = 0
        D2 = d2;
    }
    for (int c0 = l0; c0 <= a.L; c0 += kLC) {
        const int nc = min(kLC, a.L - c0 + 1);
        __syncthreads();
        for (int i = threadIdx.x; i < nc; i += kNT) {
            const int l = c0 + i;
            double al, be, ga;
            double2 ap, am;
            make_coefs(a, m, k, l, al, be, ga, ap, am);
            rc[i] = Rec32{(float)al, (float)(al - be - ga - 1.0), (float)(al + be - ga - 1.0), (float)ga};
            const double sg = (l & 1) ? -1.0 : 1.0;
            ac[i] = Acc32{make_float2((float)ap.x, (float)ap.y), make_float2((float)am.x, (float)am.y),
                          make_float2((float)(sg * ap.x), (float)(sg * ap.y)),
                          make_float2((float)(sg * am.x), (float)(sg * am.y))};
        }
        __syncthreads();
        if (!active) continue;
        int i = 0;
        for (; i < nc && (e1 < 0 || e2 < 0); ++i) {
            const Rec32 r = rc[i];
            const Acc32 c = ac[i];
            if (e1 == 0) {
                NP.x = fmaf(c.ap.x, d1, NP.x);
                NP.y = fmaf(c.ap.y, d1, NP.y);
                SM.x = fmaf(c.sam.x, d1, SM.x);
                SM.y = fmaf(c.sam.y, d1, SM.y);
            }
            if (e2 == 0) {
                NM.x = fmaf(c.am.x, d2, NM.x);
                NM.y = fmaf(c.am.y, d2, NM.y);
                SP.x = fmaf(c.sap.x, d2, SP.x);
                SP.y = fmaf(c.sap.y, d2, SP.y);
            }
            D1 = fmaf(fmaf(-r.a, y, r.cp), d1, r.g * D1);
            d1 += D1;
            D2 = fmaf(fmaf(-r.a, y, r.cm), d2, r.g * D2);
            d2 += D2;
            if (e1 < 0 && fabsf(d1) > kScaleThr32) {
                d1 *= kScaleDn32;
                D1 *= kScaleDn32;
                ++e1;
            }
            if (e2 < 0 && fabsf(d2) > kScaleThr32) {
                d2 *= kScaleDn32;
                D2 *= kScaleDn32;
                ++e2;
            }
        }
#pragma unroll 4
        for (; i < nc; ++i) {
            const Rec32 r = rc[i];
            const Acc32 c = ac[i];
            NP.x = fmaf(c.ap.x, d1, NP.x);
            NP.y = fmaf(c.ap.y, d1, NP.y);
            SM.x = fmaf(c.sam.x, d1, SM.x);
            SM.y = fmaf(c.sam.y, d1, SM.y);
            NM.x = fmaf(c.am.x, d2, NM.x);
            NM.y = fmaf(c.am.y, d2, NM.y);
            SP.x = fmaf(c.sap.x, d2, SP.x);
            SP.y = fmaf(c.sap.y, d2, SP.y);
            D1 = fmaf(fmaf(-r.a, y, r.cp), d1, r.g * D1);
            d1 += D1;
            D2 = fmaf(fmaf(-r.a, y, r.cm), d2, r.g * D2);
            d2 += D2;
        }
    }
    if (active) write_out<float2>(a, m, k, pair, NP, SP, NM, SM);
}

sl_status launch_lcontract(sl_plan *p, const double *sky, const double *beam) {
    LcArgs a;
    a.L = p->L;
    a.K = p->K;
    a.ncomp = p->ncomp;
    a.R = p->R;
    a.npairs = p->npairs;
    a.nchunk = (p->npairs + kNT - 1) / kNT;
    a.nalm = p->nalm;
    a.sky = (const double2 *)sky;
    a.beam = (const double2 *)beam;
    a.xr = p->d_xr;
    a.y32 = p->d_y32;
    a.seed = p->d_seed;
    a.seed_e = p->d_seed_e;
    a.G = p->d_G;
    const int64_t nblk = (int64_t)(p->L + 1) * (p->K + 1) * a.nchunk;
    if (nblk > 0x7fffffff) return set_error(SL_ERR_UNSUPPORTED, "grid too large");
    int slot;
    if (p->precision == SL_FP64) {
        slot = timing_begin(p, "lcontract_f64");
        k_lcontract_f64<<<(unsigned)nblk, kNT, 0, p->stream>>>(a);
    } else {
        slot = timing_begin(p, "lcontract_f32");
        k_lcontract_f32<<<(unsigned)nblk, kNT, 0, p->stream>>>(a);
    }
    timing_end(p, slot);
    return cuda_check(cudaGetLastError(), "k_lcontract launch");
}

}  // namespace sl
