// k_adjoint.cu -- transpose of the spin "Legendre" step and the final
// sky x beam products (the gradients of the total convolution, Sect. 2.1,
// with respect to the sky s_lm and the beam b_lk).
//
// Contraction transpose (real inner product Re<x, y>):
//   Abar_{k,l,m} = sum_r d^l_{mk}(theta_r) Ghat_k(r, m),   m in [-L, L].
// With the reflections of the forward step, per north ring pair (d1 = d_{m,+k},
// d2 = d_{m,-k}, s_l = (-1)^l):
//   Abar_{+m}(l) = c_l sum_pairs [y1 Ghat(N,+m) + s_l y2 (-1)^m Ghat(S,+m)]
//   Abar_{-m}(l) = c_l sum_pairs [y2 (-1)^{m+k} Ghat(N,-m) + s_l y1 (-1)^k Ghat(S,-m)]
// where d = c y are the rescaled recurrence values of the forward kernel, run
// from the same FP64 start states (the evanescent zone is skipped).
// One CTA per (m >= 0, k, 128 ring pairs), one thread per (ring pair, sign of
// k).  Per chunk of 32 l: every thread steps its recurrence and writes y to
// shared memory (0 before its start l); then each of the 256 threads forms
// one of the 8 real dot products of one l over the CTA's 128 pairs.  The
// (l, value) results are combined with c_l and s_l and added atomically into
// Abar (zeroed first; the CTAs of other ring blocks add to the same entries).
//
// Products (A_{k,lm} = sum_X s^X_lm conj(b^X_lk), extended to m < 0 by
// s_{l,-m} = (-1)^m conj(s_lm)); g = d/dRe + i d/dIm:
//   sky,  m > 0: sum_k [b_lk Abar_{k,l,m} + (-1)^m conj(b_lk) conj(Abar_{k,l,-m})]
//   sky,  m = 0: sum_k Re(b_lk Abar_{k,l,0})
//   beam:        sum_{m=-l..l} s_lm conj(Abar_{k,lm})   (Re only for k = 0; 0 for l < k)
#include "df.cuh"
#include "sl_internal.cuh"

namespace sl {

constexpr int kNTA = 256;          // threads per CTA
constexpr int kPA = kNTA / 2;      // ring pairs per CTA
constexpr int kLCA = 32;           // l per chunk (kLCA * 8 dot products = kNTA threads)
constexpr int kWS = kPA + 1;       // padded row of the y tile (bank spread)

struct LcAdjArgs {
    int L, K, R, npairs, nchunk;
    int64_t nalm;
    const double *xr;
    const int *ls;
    const double2 *st64;
    const RTab64 *tab;
    const double2 *Ghat;   // [K+1][R][2L+1]
    double2 *Abar;         // [K+1][2L+1][L+1]
};

struct AdjSmem {
    double W[kLCA][2][kWS];        // y values [l][sign][pair]
    double Gv[8][kWS];             // dot-product partners [dot][pair]
    double dots[kLCA][8];
    double2 rc[kLCA];              // a', b'
    double cl[kLCA];               // c_l
    int qlo[2][kLCA];              // [sign][l - c0]: first pair whose y is nonzero at l (or later)
};


// Pairs below qlo[sign][i] have y = 0 at l = c0 + i (their recurrence starts
// later; the evanescent zone), so the dot products of that l start there: the
// skipped terms are exact zeros and the sums are unchanged.  Each thread enters
// its first nonzero l of the chunk; warp 0 turns the entries into prefix minima.
__device__ __forceinline__ void adj_qlo_mark(int (*qlo)[kLCA], bool active, int ls, int c0, int nc, int neg,
                                             int lp) {
    if (active && ls < c0 + nc) atomicMin(&qlo[neg][max(0, ls - c0)], lp);
}
__device__ __forceinline__ void adj_qlo_scan(int (*qlo)[kLCA]) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
#pragma unroll
        for (int sg = 0; sg < 2; ++sg) {
            int v = qlo[sg][lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v = min(v, t);
            }
            qlo[sg][lane] = v;
        }
    }
}

__global__ void __launch_bounds__(kNTA) k_lcontract_adj(const LcAdjArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AdjSmem &S = *reinterpret_cast<AdjSmem *>(smem_raw);
    auto &W = S.W;
    auto &Gv = S.Gv;
    auto &dots = S.dots;
    auto &rc = S.rc;
    auto &cl = S.cl;
    int b = blockIdx.x;
    const int pc = b % a.nchunk;
    b /= a.nchunk;
    const int k = b % (a.K + 1), m = b / (a.K + 1);
    const int neg = threadIdx.x >= kPA;
    const int lp = threadIdx.x & (kPA - 1);
    const int pair = pc * kPA + lp;
    const bool active = pair < a.npairs;
    const int64_t moff = (int64_t)m * (2 * a.L + 1 - m) / 2;
    const RTab64 *tab = a.tab + (int64_t)k * a.nalm + moff;

    double x = 0.0, y = 0.0, yo = 0.0;
    int ls = a.L + 1;
    // dot partners: 0/1 W+ . Ghat(N,+m); 2/3 W- . (-1)^m Ghat(S,+m);
    //               4/5 W- . (-1)^{m+k} Ghat(N,-m); 6/7 W+ . (-1)^k Ghat(S,-m)
    {
        double2 g0 = {0, 0}, g1 = {0, 0};
        if (active) {
            const int64_t si = (((int64_t)k * (a.L + 1) + m) * 2 + neg) * a.npairs + pair;
            ls = a.ls[si];
            yo = a.st64[si].x;
            y = a.st64[si].y;
            x = a.xr[pair];
            const int rn = pair, rs = a.R - 1 - pair;
            const int64_t row = 2 * (int64_t)a.L + 1;
            const double2 *Gk = a.Ghat + (int64_t)k * a.R * row;
            const double sm_ = (m & 1) ? -1.0 : 1.0, sk = (k & 1) ? -1.0 : 1.0;
            if (!neg) {
                g0 = Gk[rn * row + a.L + m];
                if (m > 0 && rs != rn) {
                    const double2 v = Gk[rs * row + a.L - m];
                    g1 = make_double2(sk * v.x, sk * v.y);
                }
            } else {
                if (rs != rn) {
                    const double2 v = Gk[rs * row + a.L + m];
                    g0 = make_double2(sm_ * v.x, sm_ * v.y);
                }
                if (m > 0) {
                    const double2 v = Gk[rn * row + a.L - m];
                    g1 = make_double2(sm_ * sk * v.x, sm_ * sk * v.y);
                }
            }
        }
        const int d0 = neg ? 2 : 0, d1 = neg ? 4 : 6;
        Gv[d0][lp] = g0.x;
        Gv[d0 + 1][lp] = g0.y;
        Gv[d1][lp] = g1.x;
        Gv[d1 + 1][lp] = g1.y;
    }
    // smallest start l over the CTA
    __shared__ int s_min;
    if (threadIdx.x == 0) s_min = 0x7fffffff;
    __syncthreads();
    atomicMin(&s_min, ls);
    __syncthreads();
    const int lstart = s_min;
    const double sb = neg ? 1.0 : -1.0;
    const int dl = threadIdx.x >> 3, dq = threadIdx.x & 7;     // this thread's (l, dot) in phase 2
    const int wsg = (dq == 0 || dq == 1 || dq == 6 || dq == 7) ? 0 : 1;   // W+ or W-
    double2 *Ap = a.Abar + ((int64_t)k * (2 * a.L + 1) + a.L + m) * (a.L + 1);
    double2 *Am = a.Abar + ((int64_t)k * (2 * a.L + 1) + a.L - m) * (a.L + 1);

    for (int c0 = lstart; c0 <= a.L; c0 += kLCA) {
        const int nc = min(kLCA, a.L - c0 + 1);
        __syncthreads();
        if (threadIdx.x < nc) {
            const RTab64 t = tab[c0 + threadIdx.x];
            rc[threadIdx.x] = make_double2(t.a, t.b);
            cl[threadIdx.x] = t.c;
        }
        if (threadIdx.x < 2 * kLCA) S.qlo[threadIdx.x / kLCA][threadIdx.x % kLCA] = kPA;
        __syncthreads();
        adj_qlo_mark(S.qlo, active, ls, c0, nc, neg, lp);
        // phase 1: recurrence values of this (pair, sign) for the chunk
        for (int i = 0; i < nc; ++i) {
            const int l = c0 + i;
            double v = 0.0;
            if (l >= ls) {
                v = y;
                const double2 r = rc[i];
                const double yn = fma(fma(r.x, x, sb * r.y), y, -yo);
                yo = y;
                y = yn;
            }
            W[i][neg][lp] = v;
        }
        for (int i = nc; i < kLCA; ++i) W[i][neg][lp] = 0.0;
        __syncthreads();
        adj_qlo_scan(S.qlo);
        __syncthreads();
        // phase 2: dot product (dl, dq) over the CTA's pairs with a nonzero y
        {
            const double *wr = W[dl][wsg];
            const double *gr = Gv[dq];
            double s0 = 0.0, s1 = 0.0;
#pragma unroll 8
            for (int q = S.qlo[wsg][dl] & ~1; q < kPA; q += 2) {
                s0 = fma(wr[q], gr[q], s0);
                s1 = fma(wr[q + 1], gr[q + 1], s1);
            }
            dots[dl][dq] = s0 + s1;
        }
        __syncthreads();
        // combine: Abar+ = c (D01 + s D23), Abar- = c (D45 + s D67)
        if (threadIdx.x < 4 * nc) {
            const int i = threadIdx.x >> 2, comp = threadIdx.x & 3;
            const int l = c0 + i;
            const double s = (l & 1) ? -1.0 : 1.0;
            const double c = cl[i];
            if (comp < 2) {
                const double v = c * (dots[i][comp] + s * dots[i][2 + comp]);
                atomicAdd(&Ap[l].x + comp, v);
            } else if (m > 0) {
                const double v = c * (dots[i][2 + comp] + s * dots[i][4 + comp]);
                atomicAdd(&Am[l].x + (comp - 2), v);
            }
        }
    }
}

// ------------------------------------------------------------------ DF64
// The same transpose for SL_DF64 plans: the recurrence and the dot products in
// double-float arithmetic (df.cuh), the c_l, s_l combination and the atomic
// additions into Abar in double.
struct AdjSmemDF {
    float2 W[kLCA][2][kWS];        // y values [l][sign][pair], double-float
    float2 Gv[8][kWS];
    double dots[kLCA][8];
    float4 rc[kLCA];               // a', b' as double-float
    double cl[kLCA];
    int qlo[2][kLCA];
};

__global__ void __launch_bounds__(kNTA) k_lcontract_adj_df(const LcAdjArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AdjSmemDF &S = *reinterpret_cast<AdjSmemDF *>(smem_raw);
    int b = blockIdx.x;
    const int pc = b % a.nchunk;
    b /= a.nchunk;
    const int k = b % (a.K + 1), m = b / (a.K + 1);
    const int neg = threadIdx.x >= kPA;
    const int lp = threadIdx.x & (kPA - 1);
    const int pair = pc * kPA + lp;
    const bool active = pair < a.npairs;
    const int64_t moff = (int64_t)m * (2 * a.L + 1 - m) / 2;
    const RTab64 *tab = a.tab + (int64_t)k * a.nalm + moff;

    dfl x = {0.f, 0.f}, y = {0.f, 0.f}, yo = {0.f, 0.f};
    int ls = a.L + 1;
    {
        double2 g0 = {0, 0}, g1 = {0, 0};
        if (active) {
            const int64_t si = (((int64_t)k * (a.L + 1) + m) * 2 + neg) * a.npairs + pair;
            ls = a.ls[si];
            yo = df_from_d(a.st64[si].x);
            y = df_from_d(a.st64[si].y);
            x = df_from_d(a.xr[pair]);
            const int rn = pair, rs = a.R - 1 - pair;
            const int64_t row = 2 * (int64_t)a.L + 1;
            const double2 *Gk = a.Ghat + (int64_t)k * a.R * row;
            const double sm_ = (m & 1) ? -1.0 : 1.0, sk = (k & 1) ? -1.0 : 1.0;
            if (!neg) {
                g0 = Gk[rn * row + a.L + m];
                if (m > 0 && rs != rn) {
                    const double2 v = Gk[rs * row + a.L - m];
                    g1 = make_double2(sk * v.x, sk * v.y);
                }
            } else {
                if (rs != rn) {
                    const double2 v = Gk[rs * row + a.L + m];
                    g0 = make_double2(sm_ * v.x, sm_ * v.y);
                }
                if (m > 0) {
                    const double2 v = Gk[rn * row + a.L - m];
                    g1 = make_double2(sm_ * sk * v.x, sm_ * sk * v.y);
                }
            }
        }
        const int d0 = neg ? 2 : 0, d1 = neg ? 4 : 6;
        const dfl a0 = df_from_d(g0.x), a1 = df_from_d(g0.y), b0 = df_from_d(g1.x), b1 = df_from_d(g1.y);
        S.Gv[d0][lp] = make_float2(a0.h, a0.l);
        S.Gv[d0 + 1][lp] = make_float2(a1.h, a1.l);
        S.Gv[d1][lp] = make_float2(b0.h, b0.l);
        S.Gv[d1 + 1][lp] = make_float2(b1.h, b1.l);
    }
    __shared__ int s_min;
    if (threadIdx.x == 0) s_min = 0x7fffffff;
    __syncthreads();
    atomicMin(&s_min, ls);
    __syncthreads();
    const int lstart = s_min;
    const float sb = neg ? 1.f : -1.f;
    const int dl = threadIdx.x >> 3, dq = threadIdx.x & 7;
    const int wsg = (dq == 0 || dq == 1 || dq == 6 || dq == 7) ? 0 : 1;
    double2 *Ap = a.Abar + ((int64_t)k * (2 * a.L + 1) + a.L + m) * (a.L + 1);
    double2 *Am = a.Abar + ((int64_t)k * (2 * a.L + 1) + a.L - m) * (a.L + 1);

    for (int c0 = lstart; c0 <= a.L; c0 += kLCA) {
        const int nc = min(kLCA, a.L - c0 + 1);
        __syncthreads();
        if (threadIdx.x < nc) {
            const RTab64 t = tab[c0 + threadIdx.x];
            const dfl ra = df_from_d(t.a), rb = df_from_d(t.b);
            S.rc[threadIdx.x] = make_float4(ra.h, ra.l, rb.h, rb.l);
            S.cl[threadIdx.x] = t.c;
        }
        if (threadIdx.x < 2 * kLCA) S.qlo[threadIdx.x / kLCA][threadIdx.x % kLCA] = kPA;
        __syncthreads();
        adj_qlo_mark(S.qlo, active, ls, c0, nc, neg, lp);
        for (int i = 0; i < nc; ++i) {
            const int l = c0 + i;
            float2 v = make_float2(0.f, 0.f);
            if (l >= ls) {
                v = make_float2(y.h, y.l);
                const float4 r = S.rc[i];
                const dfl t = df_fma(dfl{r.x, r.y}, x, dfl{sb * r.z, sb * r.w});
                const dfl yn = df_fma(t, y, df_neg(yo));
                yo = y;
                y = yn;
            }
            S.W[i][neg][lp] = v;
        }
        for (int i = nc; i < kLCA; ++i) S.W[i][neg][lp] = make_float2(0.f, 0.f);
        __syncthreads();
        adj_qlo_scan(S.qlo);
        __syncthreads();
        {
            const float2 *wr = S.W[dl][wsg];
            const float2 *gr = S.Gv[dq];
            dacc s0, s1;
            dacc_zero(s0);
            dacc_zero(s1);
#pragma unroll 4
            for (int q = S.qlo[wsg][dl] & ~1; q < kPA; q += 2) {
                const float2 w0 = wr[q], g0 = gr[q], w1 = wr[q + 1], g1 = gr[q + 1];
                dacc_mac(s0, dfl{w0.x, w0.y}, dfl{g0.x, g0.y});
                dacc_mac(s1, dfl{w1.x, w1.y}, dfl{g1.x, g1.y});
            }
            dacc_add(s0, dacc_get(s1));
            S.dots[dl][dq] = df_to_d(dacc_get(s0));
        }
        __syncthreads();
        if (threadIdx.x < 4 * nc) {
            const int i = threadIdx.x >> 2, comp = threadIdx.x & 3;
            const int l = c0 + i;
            const double s = (l & 1) ? -1.0 : 1.0;
            const double c = S.cl[i];
            if (comp < 2) {
                const double v = c * (S.dots[i][comp] + s * S.dots[i][2 + comp]);
                atomicAdd(&Ap[l].x + comp, v);
            } else if (m > 0) {
                const double v = c * (S.dots[i][2 + comp] + s * S.dots[i][4 + comp]);
                atomicAdd(&Am[l].x + (comp - 2), v);
            }
        }
    }
}

sl_status launch_lcontract_adjoint(sl_plan *p) {
    LcAdjArgs a;
    a.L = p->L;
    a.K = p->K;
    a.R = p->R;
    a.npairs = p->npairs;
    a.nchunk = (p->npairs + kPA - 1) / kPA;
    a.nalm = p->nalm;
    a.xr = p->d_xr;
    a.ls = p->d_ls_adj;
    a.st64 = p->d_st64_adj;
    a.tab = p->d_tab64;
    a.Ghat = p->d_Gadj;
    a.Abar = p->d_Abar;
    sl_status st = cuda_check(cudaMemsetAsync(p->d_Abar, 0,
                                              (size_t)(p->K + 1) * (2 * p->L + 1) * (p->L + 1) * sizeof(double2),
                                              p->stream),
                              "memset Abar");
    if (st != SL_OK) return st;
    const int64_t nblk = (int64_t)(p->L + 1) * (p->K + 1) * a.nchunk;
    const bool df = p->precision == SL_DF64;
    const size_t sm = df ? sizeof(AdjSmemDF) : sizeof(AdjSmem);
    void (*kern)(const LcAdjArgs) = df ? k_lcontract_adj_df : k_lcontract_adj;
    if ((st = cuda_check(allow_dyn_smem(kern, sm),
                         "k_lcontract_adj smem attribute")) != SL_OK)
        return st;
    int slot = timing_begin(p, df ? "lcontract_adj_df" : "lcontract_adj");
    kern<<<(unsigned)nblk, kNTA, sm, p->stream>>>(a);
    timing_end(p, slot);
    return cuda_check(cudaGetLastError(), "k_lcontract_adj launch");
}

// ------------------------------------------------------------------ products
__global__ void k_grad_sky(int L, int K, int64_t nalm, const double2 *__restrict__ beam,
                           const double2 *__restrict__ Abar, double2 *__restrict__ out, int accumulate) {
    const int m = blockIdx.y, X = blockIdx.z;
    const int l = m + blockIdx.x * blockDim.x + threadIdx.x;
    if (l > L) return;
    const int64_t row = L + 1;
    double2 g = {0.0, 0.0};
    const double sgn = (m & 1) ? -1.0 : 1.0;
    for (int k = 0; k <= K; ++k) {
        double2 b = beam[((int64_t)X * (K + 1) + k) * (L + 1) + l];
        if (k == 0) b.y = 0.0;
        const double2 ap = Abar[((int64_t)k * (2 * L + 1) + L + m) * row + l];
        // b * Abar_{+m}
        g.x += b.x * ap.x - b.y * ap.y;
        g.y += b.x * ap.y + b.y * ap.x;
        if (m > 0) {
            const double2 an = Abar[((int64_t)k * (2 * L + 1) + L - m) * row + l];
            // (-1)^m conj(b) conj(an) = (-1)^m conj(b * an)
            g.x += sgn * (b.x * an.x - b.y * an.y);
            g.y -= sgn * (b.x * an.y + b.y * an.x);
        }
    }
    if (m == 0) g.y = 0.0;
    double2 *o = out + (int64_t)X * nalm + (int64_t)m * (2 * L + 1 - m) / 2 + l;
    if (accumulate) {
        const double2 c = *o;
        g.x += c.x;
        g.y += c.y;
    }
    *o = g;
}

__global__ void k_grad_beam(int L, int K, int64_t nalm, const double2 *__restrict__ sky,
                            const double2 *__restrict__ Abar, double2 *__restrict__ out, int accumulate) {
    const int k = blockIdx.y, X = blockIdx.z;
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l > L) return;
    const int64_t row = L + 1;
    double2 g = {0.0, 0.0};
    if (l >= k) {
        const double2 *Ak = Abar + (int64_t)k * (2 * L + 1) * row;
        for (int m = 0; m <= l; ++m) {
            double2 s = sky[(int64_t)X * nalm + (int64_t)m * (2 * L + 1 - m) / 2 + l];
            if (m == 0) s.y = 0.0;
            const double2 ap = Ak[(int64_t)(L + m) * row + l];
            // s * conj(ap)
            g.x += s.x * ap.x + s.y * ap.y;
            g.y += s.y * ap.x - s.x * ap.y;
            if (m > 0) {
                const double2 an = Ak[(int64_t)(L - m) * row + l];
                const double sg = (m & 1) ? -1.0 : 1.0;
                // (-1)^m conj(s) conj(an) = (-1)^m conj(s * an)
                g.x += sg * (s.x * an.x - s.y * an.y);
                g.y -= sg * (s.x * an.y + s.y * an.x);
            }
        }
        if (k == 0) g.y = 0.0;
    }
    double2 *o = out + ((int64_t)X * (K + 1) + k) * (L + 1) + l;
    if (accumulate) {
        const double2 c = *o;
        g.x += c.x;
        g.y += c.y;
    }
    *o = g;
}

sl_status launch_grad(sl_plan *p, const double *sky, const double *beam, double *sky_grad, double *beam_grad,
                      int accumulate) {
    const int bs = 128;
    if (sky_grad) {
        dim3 grid((p->L + 1 + bs - 1) / bs, p->L + 1, p->ncomp);
        int slot = timing_begin(p, "grad_sky");
        k_grad_sky<<<grid, bs, 0, p->stream>>>(p->L, p->K, p->nalm, (const double2 *)beam, p->d_Abar,
                                              (double2 *)sky_grad, accumulate);
        timing_end(p, slot);
        sl_status st = cuda_check(cudaGetLastError(), "k_grad_sky launch");
        if (st != SL_OK) return st;
    }
    if (beam_grad) {
        dim3 grid((p->L + 1 + bs - 1) / bs, p->K + 1, p->ncomp);
        int slot = timing_begin(p, "grad_beam");
        k_grad_beam<<<grid, bs, 0, p->stream>>>(p->L, p->K, p->nalm, (const double2 *)sky, p->d_Abar,
                                               (double2 *)beam_grad, accumulate);
        timing_end(p, slot);
        return cuda_check(cudaGetLastError(), "k_grad_beam launch");
    }
    return SL_OK;
}

}  // namespace sl
