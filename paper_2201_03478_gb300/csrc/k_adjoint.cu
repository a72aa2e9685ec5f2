// k_adjoint.cu -- transpose of the spin "Legendre" step and the final
// sky x beam products (the gradients of the total convolution, Sect. 2.1,
// with respect to the sky s_lm and the beam b_lk).
//
// Contraction transpose (real inner product Re<x, y>):
//   Abar_{k,l,m} = sum_r d^l_{mk}(theta_r) Ghat_k(r, m),   m in [-L, L],
// organised like the forward kernel: one CTA per (m >= 0, k, 256 north rings),
// two recurrences per thread, the four reflections folded into
//   Abar_{+m} = sum_pairs [d1 Ghat(N,+m) + (-1)^{l+m} d2 Ghat(S,+m)]
//   Abar_{-m} = sum_pairs [(-1)^{m+k} d2 Ghat(N,-m) + (-1)^{l-k} d1 Ghat(S,-m)]
// Every l needs a sum over the CTA's rings: a 4-value warp reduce-scatter by
// shuffles, a cross-warp sum in shared memory per chunk of l, and one atomic
// add per (l, value) into Abar (zeroed first).  All warps step l together;
// a warp keeps checking the scaled representation until all its lanes have
// reached normal range.
//
// Products (A_{k,lm} = sum_X s^X_lm conj(b^X_lk), extended to m < 0 by
// s_{l,-m} = (-1)^m conj(s_lm)); g = d/dRe + i d/dIm:
//   sky,  m > 0: sum_k [b_lk Abar_{k,l,m} + (-1)^m conj(b_lk) conj(Abar_{k,l,-m})]
//   sky,  m = 0: sum_k Re(b_lk Abar_{k,l,0})
//   beam:        sum_{m=-l..l} s_lm conj(Abar_{k,lm})   (Re only for k = 0; 0 for l < k)
#include "sl_internal.cuh"

namespace sl {

constexpr int kNTA = 256;
constexpr int kLCA = 32;

struct __align__(32) RecA {
    double x, y, z, w;   // alpha, beta, gamma, unused
};

struct LcAdjArgs {
    int L, K, R, npairs, nchunk;
    const double *xr;
    const double2 *seed;
    const int2 *seed_e;
    const double2 *Ghat;   // [K+1][R][2L+1]
    double2 *Abar;         // [K+1][2L+1][L+1]
};

__device__ __forceinline__ void rec_coefs(int m, int k, int l, double &al, double &be, double &ga) {
    const double lp = l + 1.0, ll = (double)l, dm = (double)m, dk = (double)k;
    const double ra = 1.0 / sqrt((lp * lp - dm * dm) * (lp * lp - dk * dk));
    al = (2.0 * l + 1.0) * lp * ra;
    if (l > 0) {
        be = (2.0 * l + 1.0) * dm * dk * ra / ll;
        ga = lp * sqrt((ll * ll - dm * dm) * (ll * ll - dk * dk)) * ra / ll;
    } else {
        be = 0.0;
        ga = 0.0;
    }
}

__global__ void __launch_bounds__(kNTA) k_lcontract_adj(const LcAdjArgs a) {
    __shared__ RecA rc[kLCA];                       // alpha, beta, gamma
    __shared__ double red[kNTA / 32][kLCA][4];      // per-warp sums
    int b = blockIdx.x;
    const int pc = b % a.nchunk;
    b /= a.nchunk;
    const int k = b % (a.K + 1);
    const int m = b / (a.K + 1);
    const int pair = pc * kNTA + threadIdx.x;
    const int l0 = max(m, k);
    const bool active = pair < a.npairs;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    double x = 0.0, d1 = 0.0, d1o = 0.0, d2 = 0.0, d2o = 0.0;
    int e1 = 0, e2 = 0;
    double2 gnp = {0, 0}, gsp = {0, 0}, gnm = {0, 0}, gsm = {0, 0};
    if (active) {
        x = a.xr[pair];
        const int64_t si = ((int64_t)k * (a.L + 1) + m) * a.npairs + pair;
        const double2 sv = a.seed[si];
        const int2 se = a.seed_e[si];
        d1 = sv.x;
        e1 = se.x;
        d2 = sv.y;
        e2 = se.y;
        const int rn = pair, rs = a.R - 1 - pair;
        const int64_t row = 2 * (int64_t)a.L + 1;
        const double2 *Gk = a.Ghat + (int64_t)k * a.R * row;
        const double sm_ = (m & 1) ? -1.0 : 1.0, sk = (k & 1) ? -1.0 : 1.0;
        gnp = Gk[rn * row + a.L + m];
        if (rs != rn) {
            const double2 v = Gk[rs * row + a.L + m];
            gsp = make_double2(sm_ * v.x, sm_ * v.y);
        }
        if (m > 0) {
            const double2 v = Gk[rn * row + a.L - m];
            gnm = make_double2(sm_ * sk * v.x, sm_ * sk * v.y);
            if (rs != rn) {
                const double2 w = Gk[rs * row + a.L - m];
                gsm = make_double2(sk * w.x, sk * w.y);
            }
        }
    }
    bool slow = __any_sync(0xffffffffu, e1 < 0 || e2 < 0);
    double2 *Ap = a.Abar + ((int64_t)k * (2 * a.L + 1) + a.L + m) * (a.L + 1);
    double2 *Am = a.Abar + ((int64_t)k * (2 * a.L + 1) + a.L - m) * (a.L + 1);

    for (int c0 = l0; c0 <= a.L; c0 += kLCA) {
        const int nc = min(kLCA, a.L - c0 + 1);
        __syncthreads();
        for (int i = threadIdx.x; i < nc; i += kNTA) {
            double al, be, ga;
            rec_coefs(m, k, c0 + i, al, be, ga);
            rc[i] = RecA{al, be, ga, 0.0};
        }
        __syncthreads();
        for (int i = 0; i < nc; ++i) {
            const int l = c0 + i;
            const RecA r = rc[i];
            double u1, u2;   // d1, d2 as they contribute (0 while scaled)
            if (slow) {
                u1 = (e1 == 0) ? d1 : 0.0;
                u2 = (e2 == 0) ? d2 : 0.0;
            } else {
                u1 = d1;
                u2 = d2;
            }
            double v0, v1, v2, v3;   // Abar_{+m} (re, im), Abar_{-m} (re, im)
            if (l & 1) {
                v0 = fma(-u2, gsp.x, u1 * gnp.x);
                v1 = fma(-u2, gsp.y, u1 * gnp.y);
                v2 = fma(-u1, gsm.x, u2 * gnm.x);
                v3 = fma(-u1, gsm.y, u2 * gnm.y);
            } else {
                v0 = fma(u2, gsp.x, u1 * gnp.x);
                v1 = fma(u2, gsp.y, u1 * gnp.y);
                v2 = fma(u1, gsm.x, u2 * gnm.x);
                v3 = fma(u1, gsm.y, u2 * gnm.y);
            }
            // reduce-scatter over the warp: lane 0 -> v0, 8 -> v1, 16 -> v2, 24 -> v3
            {
                const bool hi = lane & 16;
                const double s0 = hi ? v0 : v2, s1 = hi ? v1 : v3;
                const double k0 = hi ? v2 : v0, k1 = hi ? v3 : v1;
                const double t0 = k0 + __shfl_xor_sync(0xffffffffu, s0, 16);
                const double t1 = k1 + __shfl_xor_sync(0xffffffffu, s1, 16);
                const bool b8 = lane & 8;
                double w = (b8 ? t1 : t0) + __shfl_xor_sync(0xffffffffu, b8 ? t0 : t1, 8);
                w += __shfl_xor_sync(0xffffffffu, w, 4);
                w += __shfl_xor_sync(0xffffffffu, w, 2);
                w += __shfl_xor_sync(0xffffffffu, w, 1);
                if ((lane & 7) == 0) red[warp][i][lane >> 3] = w;
            }
            // advance both recurrences
            const double n1 = fma(fma(r.x, x, -r.y), d1, -r.z * d1o);
            const double n2 = fma(fma(r.x, x, r.y), d2, -r.z * d2o);
            d1o = d1;
            d1 = n1;
            d2o = d2;
            d2 = n2;
            if (slow) {
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
                slow = __any_sync(0xffffffffu, e1 < 0 || e2 < 0);
            }
        }
        __syncthreads();
        // cross-warp sums, one atomic per (l, value)
        for (int t = threadIdx.x; t < nc * 4; t += kNTA) {
            const int i = t >> 2, c = t & 3;
            if (m == 0 && c >= 2) continue;
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < kNTA / 32; ++w) s += red[w][i][c];
            double *dst = (c < 2) ? &Ap[c0 + i].x : &Am[c0 + i].x;
            atomicAdd(dst + (c & 1), s);
        }
    }
}

sl_status launch_lcontract_adjoint(sl_plan *p) {
    LcAdjArgs a;
    a.L = p->L;
    a.K = p->K;
    a.R = p->R;
    a.npairs = p->npairs;
    a.nchunk = (p->npairs + kNTA - 1) / kNTA;
    a.xr = p->d_xr;
    a.seed = p->d_seed;
    a.seed_e = p->d_seed_e;
    a.Ghat = p->d_Gadj;
    a.Abar = p->d_Abar;
    sl_status st = cuda_check(cudaMemsetAsync(p->d_Abar, 0,
                                              (size_t)(p->K + 1) * (2 * p->L + 1) * (p->L + 1) * sizeof(double2),
                                              p->stream),
                              "memset Abar");
    if (st != SL_OK) return st;
    const int64_t nblk = (int64_t)(p->L + 1) * (p->K + 1) * a.nchunk;
    int slot = timing_begin(p, "lcontract_adj");
    k_lcontract_adj<<<(unsigned)nblk, kNTA, 0, p->stream>>>(a);
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
