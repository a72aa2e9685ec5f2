// k_seeds.cu -- FP64 starting values of the l-recurrence of the spin
// "Legendre" step (Sect. 2.1, Eqs. c_m and S: one spin-k transform per beam
// order k).  For every north ring r, k in [0, K] and m in [0, L] the kernel
// stores d^{l0}_{m,+k}(theta_r) and d^{l0}_{m,-k}(theta_r), l0 = max(m, k),
// as a mantissa and an exponent e (value = mantissa * 2^(600 e)).
//
// Closed forms at l0 (the single surviving term of Wigner's sum):
//   m <= k:  d^k_{m, k} = sqrt(C(2k, k+m)) c^{k+m} s^{k-m}
//            d^k_{m,-k} = (-1)^{k+m} sqrt(C(2k, k+m)) c^{k-m} s^{k+m}
//   m >= k:  d^m_{m, q} = (-1)^{m-q} sqrt(C(2m, m+q)) c^{m+q} s^{m-q},  q = +-k
// with c = cos(theta/2), s = sin(theta/2).  For m > k the kernel walks m
// upward with the ratio
//   d^m_{m,q} / d^{m-1}_{m-1,q} = -sqrt(2m (2m-1) / ((m+q)(m-q))) c s,
// so each seed costs O(1) instead of O(m).
#include <algorithm>

#include "sl_internal.cuh"

namespace sl {

struct Scaled {
    double v;
    int e;
};

__device__ __forceinline__ void renorm_down(Scaled &x) {
    // keep |v| >= 2^-300 while the true value is tiny
    if (x.v != 0.0 && fabs(x.v) < kScaleLow) {
        x.v *= kScaleUp;
        x.e -= 1;
    }
}

__global__ void k_seeds(int L, int K, int npairs, const double *__restrict__ c2,
                        const double *__restrict__ s2, const double *__restrict__ cs,
                        double2 *__restrict__ seed, int2 *__restrict__ seed_e) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int total = npairs * (K + 1) * 2;
    if (t >= total) return;
    const int pair = t % npairs;
    const int rest = t / npairs;
    const int neg = rest & 1;        // 0: q = +k, 1: q = -k
    const int k = rest >> 1;
    const int q = neg ? -k : k;
    const double c = c2[pair], s = s2[pair], csv = cs[pair];

    double *out_v = reinterpret_cast<double *>(seed) + neg;
    int *out_e = reinterpret_cast<int *>(seed_e) + neg;
    auto store = [&](int m, const Scaled &x) {
        size_t idx = ((size_t)k * (L + 1) + m) * npairs + pair;
        out_v[2 * idx] = x.v;
        out_e[2 * idx] = x.e;
    };

    // m = 0 .. k: l0 = k, direct products (k <= 63)
    Scaled last{1.0, 0};
    for (int m = 0; m <= k && m <= L; ++m) {
        // sqrt(C(2k, k+m)) as a running product
        double binom = 1.0;
        for (int i = 1; i <= k - m; ++i) binom = binom * (double)(k + m + i) / (double)i;
        Scaled x{sqrt(binom), 0};
        const int pc = neg ? (k - m) : (k + m);
        const int ps = neg ? (k + m) : (k - m);
        for (int i = 0; i < pc; ++i) { x.v *= c; renorm_down(x); }
        for (int i = 0; i < ps; ++i) { x.v *= s; renorm_down(x); }
        if (neg && ((k + m) & 1)) x.v = -x.v;
        store(m, x);
        last = x;
    }
    // m = k+1 .. L: upward ratio
    for (int m = k + 1; m <= L; ++m) {
        double ratio = sqrt((2.0 * m) * (2.0 * m - 1.0) / ((double)(m + q) * (double)(m - q)));
        last.v = -last.v * ratio * csv;
        renorm_down(last);
        store(m, last);
    }
}

// Rescaled recurrence coefficients.  With d^{l+1} = (al_l x - be_l) d^l - ga_l d^{l-1}
// (al, be, ga as in the recurrence of Wigner's d in l; be flips sign with k) and
// d_l = c_l y_l, choosing c_{l0} = c_{l0+1} = 1 and c_{l+1} = ga_l c_{l-1} (l > l0)
// gives y_{l+1} = (a_l x - b_l) y_l - y_{l-1} with a = al c_l/c_{l+1},
// b = be c_l/c_{l+1}.  One thread per (k, m) walks l = l0..L in double.
__global__ void k_rtab(int L, int K, int64_t nalm, RTab64 *__restrict__ t64, RTab32 *__restrict__ t32) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (L + 1) * (K + 1)) return;
    const int k = t / (L + 1), m = t % (L + 1);
    const int l0 = max(m, k);
    const int64_t off = (int64_t)k * nalm + (int64_t)m * (2 * L + 1 - m) / 2;
    for (int l = m; l < l0 && l <= L; ++l) {
        if (t64) t64[off + l] = RTab64{0.0, 0.0, 0.0, 0.0};
        if (t32) t32[off + l] = RTab32{0.f, 0.f, 0.f, 0.f};
    }
    const double dm = (double)m, dk = (double)k;
    double c_prev = 1.0, c_cur = 1.0;   // c_{l-1} (unused at l0), c_l
    for (int l = l0; l <= L; ++l) {
        const double lp = l + 1.0, ll = (double)l;
        const double ra = 1.0 / sqrt((lp * lp - dm * dm) * (lp * lp - dk * dk));
        const double al = (2.0 * l + 1.0) * lp * ra;
        double be = 0.0, ga = 0.0;
        if (l > 0) {
            be = (2.0 * l + 1.0) * dm * dk * ra / ll;
            ga = lp * sqrt((ll * ll - dm * dm) * (ll * ll - dk * dk)) * ra / ll;
        }
        const double c_next = (l == l0) ? 1.0 : ga * c_prev;
        const double q = c_cur / c_next;
        const double a = al * q, b = be * q;
        if (t64) t64[off + l] = RTab64{a, b, c_cur, 0.0};
        if (t32) t32[off + l] = RTab32{(float)a, (float)(a - b - 2.0), (float)(a + b - 2.0), (float)c_cur};
        c_prev = c_cur;
        c_cur = c_next;
    }
}

sl_status launch_rtab(sl_plan *p) {
    const int total = (p->L + 1) * (p->K + 1);
    const int bs = 64;
    int slot = timing_begin(p, "rtab");
    k_rtab<<<(total + bs - 1) / bs, bs, 0, p->stream>>>(p->L, p->K, p->nalm, p->d_tab64, p->d_tab32);
    timing_end(p, slot);
    return cuda_check(cudaGetLastError(), "k_rtab launch");
}

// Start states of the per-call recurrences.  For every (k, m, ring pair, sign
// of k) the rescaled FP64 recurrence (table a, b) is run from the seed at l0,
// with the scaled exponent, up to the first l at which the value reaches the
// significance threshold (2^-64 for FP64 plans, 2^-30 for FP32 plans); the
// terms before it are below thr * sum|A| and are dropped.  Stored: ls and the
// state at ls ({y_{ls-1}, y_ls} in double, or {y_ls, y_ls - y_{ls-1}} in float).
// ls = L + 1 marks a ring that never reaches the threshold below lmax.
// One CTA per (m, k, 128 ring pairs); thread t < 128: +k, t >= 128: -k.
constexpr int kAdvNT = 256;
constexpr int kAdvLC = 64;

__global__ void __launch_bounds__(kAdvNT) k_advance(int L, int K, int npairs, int nchunk, int64_t nalm,
                                                    double thr, const double *__restrict__ xr,
                                                    const double2 *__restrict__ seed,
                                                    const int2 *__restrict__ seed_e,
                                                    const RTab64 *__restrict__ tab, int *__restrict__ ls_out,
                                                    double2 *__restrict__ st64, float2 *__restrict__ st32) {
    __shared__ double2 rc[kAdvLC];
    int b = blockIdx.x;
    const int pc = b % nchunk;
    b /= nchunk;
    const int k = b % (K + 1), m = b / (K + 1);
    const int neg = threadIdx.x >= kAdvNT / 2;
    const int pair = pc * (kAdvNT / 2) + (threadIdx.x & (kAdvNT / 2 - 1));
    const bool active = pair < npairs;
    const int l0 = max(m, k);
    const RTab64 *tb = tab + (int64_t)k * nalm + (int64_t)m * (2 * L + 1 - m) / 2;
    double x = 0.0, y = 0.0, yo = 0.0;
    int e = 0, ls = L + 1;
    bool done = !active;
    if (active) {
        x = xr[pair];
        const int64_t si = ((int64_t)k * (L + 1) + m) * npairs + pair;
        y = neg ? seed[si].y : seed[si].x;
        e = neg ? seed_e[si].y : seed_e[si].x;
    }
    const double sb = neg ? 1.0 : -1.0;    // -k: a x + b, +k: a x - b
    for (int c0 = l0; c0 <= L; c0 += kAdvLC) {
        const int nc = min(kAdvLC, L - c0 + 1);
        __syncthreads();
        for (int i = threadIdx.x; i < nc; i += kAdvNT) rc[i] = make_double2(tb[c0 + i].a, tb[c0 + i].b);
        __syncthreads();
        if (!done) {
            for (int i = 0; i < nc; ++i) {
                if (e == 0 && fabs(y) >= thr) {
                    ls = c0 + i;
                    done = true;
                    break;
                }
                const double2 r = rc[i];
                const double yn = fma(fma(r.x, x, sb * r.y), y, -yo);
                yo = y;
                y = yn;
                if (e < 0 && fabs(y) > kScaleThr) {
                    y *= kScaleDn;
                    yo *= kScaleDn;
                    ++e;
                }
            }
        }
        if (__syncthreads_and(done)) break;
    }
    if (!active) return;
    const int64_t o = (((int64_t)k * (L + 1) + m) * 2 + neg) * npairs + pair;
    ls_out[o] = ls;
    if (st64) st64[o] = make_double2(yo, y);
    if (st32) st32[o] = make_float2((float)y, (float)(y - yo));
}

sl_status launch_advance(sl_plan *p, double thr, int *ls, double2 *st64, float2 *st32) {
    const int nchunk = (p->npairs + kAdvNT / 2 - 1) / (kAdvNT / 2);
    const int64_t nblk = (int64_t)(p->L + 1) * (p->K + 1) * nchunk;
    int slot = timing_begin(p, "advance");
    k_advance<<<(unsigned)nblk, kAdvNT, 0, p->stream>>>(p->L, p->K, p->npairs, nchunk, p->nalm, thr, p->d_xr,
                                                        p->d_seed, p->d_seed_e, p->d_tab64, ls, st64, st32);
    timing_end(p, slot);
    return cuda_check(cudaGetLastError(), "k_advance launch");
}

// Number of recurrence steps the per-call contraction runs: sum of (L + 1 - ls).
__global__ void k_count_lsteps(int L, int64_t n, const int *__restrict__ ls, unsigned long long *__restrict__ out) {
    unsigned long long s = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += (unsigned long long)max(0, L + 1 - ls[i]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

sl_status count_lsteps(sl_plan *p, int64_t *out) {
    unsigned long long *d = nullptr, h = 0;
    sl_status st = cuda_check(cudaMalloc(&d, sizeof(unsigned long long)), "count alloc");
    if (st != SL_OK) return st;
    const int64_t n = (int64_t)(p->K + 1) * (p->L + 1) * 2 * p->npairs;
    cudaMemsetAsync(d, 0, sizeof(unsigned long long), p->stream);
    k_count_lsteps<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 8), 256, 0, p->stream>>>(p->L, n, p->d_ls, d);
    st = cuda_check(cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, p->stream), "count copy");
    if (st == SL_OK) st = cuda_check(cudaStreamSynchronize(p->stream), "count sync");
    cudaFree(d);
    *out = (int64_t)h;
    return st;
}

sl_status launch_seeds(sl_plan *p, const double *d_c2, const double *d_s2, const double *d_cs) {
    const int total = p->npairs * (p->K + 1) * 2;
    const int bs = 128;
    int slot = timing_begin(p, "seeds");
    k_seeds<<<(total + bs - 1) / bs, bs, 0, p->stream>>>(p->L, p->K, p->npairs, d_c2, d_s2, d_cs,
                                                        p->d_seed, p->d_seed_e);
    timing_end(p, slot);
    return cuda_check(cudaGetLastError(), "k_seeds launch");
}

}  // namespace sl
