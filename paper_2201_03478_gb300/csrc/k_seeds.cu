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
