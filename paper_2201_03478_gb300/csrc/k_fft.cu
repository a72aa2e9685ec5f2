// k_fft.cu -- the phi direction of the cube (Sect. 2.1, step 1 of the
// two-step algorithm: the synthesis along each ring) and its transpose.
//
// Synthesis (one CTA per group of up to 4 rings x 2 orders k, in place):
//   H(q)  = sum_{m = q mod nphi, |m| <= L} G_k(r, m)     (exact alias folding,
//           G stored [k][m + L][r])
//   F_k(r, phi_j) = sum_q H(q) e^{+2 pi i q j / nphi}    (inverse DFT)
// written to maps[r][j][k].
// Transpose (one CTA per (ring r, k)):
//   X(q) = sum_j Fbar_k(r, j) e^{-2 pi i q j / nphi},   Ghat_k(r, m) = X(m mod nphi).
//
// Rings too long for one CTA's shared memory (two buffers of nphi complex
// values) are transformed by a thread-block cluster of C = 2, 4 or 8 CTAs: the
// two buffers are spread over the CTAs' shared memory (element e in CTA e / S,
// S = nphi / C, read and written through distributed shared memory), the
// cluster synchronises after each pass, and each CTA gathers and writes its
// own slice of the ring.
//
// The synthesis DFT is a decimation-in-time mixed-radix FFT (radices 8, 4, 2, 3,
// 5) in place in shared memory on digit-reversed input; the transpose and the
// cluster form use a self-sorting (Stockham) FFT with two buffers.  Twiddles
// come from a table e^{+2 pi i j/nphi} built in long double on the host.  Each
// Stockham pass computes, for butterfly t in [0, N/R):
//   kk = t mod Ns,  v_q = x[t + q N/R] w^{s q kk N/(Ns R)},  v = DFT_R(v),
//   y[(t div Ns) Ns R + kk + q Ns] = v_q,  Ns <- Ns R.
#include <cooperative_groups.h>

#include "sl_internal.cuh"

namespace sl {

template <typename T> struct CplxOf;
template <> struct CplxOf<double> { using type = double2; };
template <> struct CplxOf<float> { using type = float2; };

template <typename C> __device__ __forceinline__ C mk(double x, double y);
template <> __device__ __forceinline__ double2 mk<double2>(double x, double y) { return make_double2(x, y); }
template <> __device__ __forceinline__ float2 mk<float2>(double x, double y) { return make_float2((float)x, (float)y); }

template <typename C> __device__ __forceinline__ C add(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C sub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C> __device__ __forceinline__ C mulc(C a, C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
// multiply by -i (FWD) or +i (inverse)
template <typename C, bool INV> __device__ __forceinline__ C rot(C a) {
    C r;
    if (INV) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
    return r;
}
// scale by a constant, in the transform's own precision (an FP32 value times a
// double would run on the FP64 pipe)
__device__ __forceinline__ double2 scal(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 scal(float2 a, double s) {
    const float f = (float)s;
    return make_float2(a.x * f, a.y * f);
}

// cos/sin of 2 pi/3, 2 pi/5, 4 pi/5 and cos pi/4 (from their closed forms)
constexpr double kS3 = 0.86602540378443864676;   // sqrt(3)/2
constexpr double kS2 = 0.70710678118654752440;   // sqrt(2)/2
constexpr double kC51 = 0.30901699437494742410;  // (sqrt(5)-1)/4
constexpr double kS51 = 0.95105651629515357212;
constexpr double kC52 = -0.80901699437494742410;
constexpr double kS52 = 0.58778525229247312917;

template <typename C, bool INV>
__device__ __forceinline__ void dft_small(int R, C *v) {
    if (R == 2) {
        C a = v[0], b = v[1];
        v[0] = add(a, b);
        v[1] = sub(a, b);
    } else if (R == 4) {
        C s02 = add(v[0], v[2]), d02 = sub(v[0], v[2]);
        C s13 = add(v[1], v[3]), d13 = rot<C, INV>(sub(v[1], v[3]));
        v[0] = add(s02, s13);
        v[2] = sub(s02, s13);
        v[1] = add(d02, d13);
        v[3] = sub(d02, d13);
    } else if (R == 3) {
        C t1 = add(v[1], v[2]);
        C t2 = rot<C, INV>(scal(sub(v[1], v[2]), kS3));
        C a = sub(v[0], scal(t1, 0.5));
        v[0] = add(v[0], t1);
        v[1] = add(a, t2);
        v[2] = sub(a, t2);
    } else if (R == 8) {
        // 4-point transforms of the even and the odd inputs (J = rot: +-i), then
        // X_k = E_k + W^k O_k, X_{k+4} = E_k - W^k O_k with W = e^{+-2 pi i/8}:
        // W O = (O + J O)/sqrt2, W^2 O = J O, W^3 O = (J O - O)/sqrt2
        const C e0 = add(v[0], v[4]), e1 = sub(v[0], v[4]);
        const C e2 = add(v[2], v[6]), e3 = rot<C, INV>(sub(v[2], v[6]));
        const C o0 = add(v[1], v[5]), o1 = sub(v[1], v[5]);
        const C o2 = add(v[3], v[7]), o3 = rot<C, INV>(sub(v[3], v[7]));
        const C E0 = add(e0, e2), E2 = sub(e0, e2), E1 = add(e1, e3), E3 = sub(e1, e3);
        const C O0 = add(o0, o2), O2 = sub(o0, o2), O1 = add(o1, o3), O3 = sub(o1, o3);
        const C t1 = scal(add(O1, rot<C, INV>(O1)), kS2);
        const C t2 = rot<C, INV>(O2);
        const C t3 = scal(sub(rot<C, INV>(O3), O3), kS2);
        v[0] = add(E0, O0);
        v[4] = sub(E0, O0);
        v[1] = add(E1, t1);
        v[5] = sub(E1, t1);
        v[2] = add(E2, t2);
        v[6] = sub(E2, t2);
        v[3] = add(E3, t3);
        v[7] = sub(E3, t3);
    } else {  // 5
        C t1 = add(v[1], v[4]), t2 = add(v[2], v[3]);
        C t3 = sub(v[1], v[4]), t4 = sub(v[2], v[3]);
        C a1 = add(v[0], add(scal(t1, kC51), scal(t2, kC52)));
        C a2 = add(v[0], add(scal(t1, kC52), scal(t2, kC51)));
        C b1 = rot<C, INV>(add(scal(t3, kS51), scal(t4, kS52)));
        C b2 = rot<C, INV>(sub(scal(t3, kS52), scal(t4, kS51)));
        v[0] = add(v[0], add(t1, t2));
        v[1] = add(a1, b1);
        v[4] = sub(a1, b1);
        v[2] = add(a2, b2);
        v[3] = sub(a2, b2);
    }
}

struct Radices {
    int n;
    unsigned long long code;   // radix of pass i in bits [4i, 4i + 4)
};

template <typename C, bool INV, int R>
__device__ __forceinline__ void fft_pass(const C *__restrict__ src, C *__restrict__ dst, int N, int Ns,
                                         const C *__restrict__ tw) {
    const int NR = N / R;
    const int stride = N / (Ns * R);
    // Ns = R_0 R_1 ... of the passes done; shifts and masks when it is a power of two
    const bool p2 = (Ns & (Ns - 1)) == 0;
    const int lg = __ffs(Ns) - 1;
    for (int t = threadIdx.x; t < NR; t += blockDim.x) {
        const int kk = p2 ? (t & (Ns - 1)) : t % Ns;
        const int blk = p2 ? (t >> lg) : t / Ns;
        C v[R];
#pragma unroll
        for (int q = 0; q < R; ++q) v[q] = src[t + q * NR];
        if (Ns > 1) {
            // one table read per butterfly: w^2 .. w^(R-1) as products of w
            C w = tw[kk * stride];
            if (!INV) w.y = -w.y;
            C wq = w;
#pragma unroll
            for (int q = 1; q < R; ++q) {
                v[q] = mulc(v[q], wq);
                if (q + 1 < R) wq = mulc(wq, w);
            }
        }
        dft_small<C, INV>(R, v);
        const int base = blk * Ns * R + kk;
#pragma unroll
        for (int q = 0; q < R; ++q) dst[base + q * Ns] = v[q];
    }
}

// Transforms buf0 (length N) in shared memory, using buf1 as the second
// buffer; returns the buffer holding the result.
template <typename C, bool INV>
__device__ C *fft_smem(C *buf0, C *buf1, int N, const Radices &rad, const C *__restrict__ tw) {
    C *src = buf0, *dst = buf1;
    int Ns = 1;
    for (int pass = 0; pass < rad.n; ++pass) {
        const int R = (int)((rad.code >> (4 * pass)) & 15);
        switch (R) {
            case 8: fft_pass<C, INV, 8>(src, dst, N, Ns, tw); break;
            case 4: fft_pass<C, INV, 4>(src, dst, N, Ns, tw); break;
            case 2: fft_pass<C, INV, 2>(src, dst, N, Ns, tw); break;
            case 3: fft_pass<C, INV, 3>(src, dst, N, Ns, tw); break;
            default: fft_pass<C, INV, 5>(src, dst, N, Ns, tw); break;
        }
        __syncthreads();
        C *tmp = src;
        src = dst;
        dst = tmp;
        Ns *= R;
    }
    return src;
}

constexpr int kRingGroup = 4;   // rings per sector of an FP32 G row (cluster form)

// ------------------------------------------------------------------ in-place multi-ring form
// One CTA transforms RG consecutive rings x KG consecutive k (TT = RG KG
// transforms).  Shared memory holds units of TT values, unit e = element e of
// every transform (t = ring-slot KG + k-slot), so each butterfly loads and
// stores whole units and reads its twiddles once for all TT transforms.  The
// G reads of a CTA cover RG adjacent rings of one (k, m) row (G is ring-fastest)
// and its cube writes KG adjacent k of one (ring, j) (the cube is k-fastest).
// The transform runs in place (decimation in time): slot s receives the input
// q = slotq[s] (and q sits in slot qslot[q]), the digit reversal of s in the radix sequence (the last pass's
// radix least significant), and pass p (radix R, span Ns = product of the
// earlier radices) combines, for each block of Ns R slots and kk < Ns, the slots
// kk + q Ns (q < R) after the twiddles e^{+2 pi i kk q/(Ns R)} -- each butterfly
// reads and writes the same R slots, so one buffer suffices.  Units are placed
// with an XOR swizzle, unit e at e ^ ((e / U) mod U), U units per 128-byte bank
// row, so that the strided butterflies of the first passes do not collide on
// the same banks.
template <typename C, int TT>
struct alignas(TT * sizeof(C) >= 16 ? 16 : TT * sizeof(C)) FftUnit {
    C v[TT];
};

template <int UB>
struct Swz {   // UB bytes per unit
    static constexpr int U = UB >= 128 ? 1 : 128 / UB;
    static constexpr int lg = U >= 16 ? 4 : U >= 8 ? 3 : U >= 4 ? 2 : U >= 2 ? 1 : 0;
    static __device__ __forceinline__ int at(int e) { return e ^ ((e >> lg) & (U - 1)); }
    static int units(int n) { return (n + U - 1) / U * U; }   // slots allocated for n units
};

template <typename C, int R, int TT>
__device__ __forceinline__ void dit_pass(C *x, int N, int Ns, const C *__restrict__ ptw) {
    using Ut = FftUnit<C, TT>;
    using S = Swz<TT * (int)sizeof(C)>;
    Ut *xu = reinterpret_cast<Ut *>(x);
    const bool p2 = (Ns & (Ns - 1)) == 0;
    const int lg = __ffs(Ns) - 1;
    for (int b = threadIdx.x; b < N / R; b += blockDim.x) {
        const int kk = p2 ? (b & (Ns - 1)) : b % Ns;
        const int g = p2 ? (b >> lg) : b / Ns;
        const int e0 = g * Ns * R + kk;
        Ut u[R];
#pragma unroll
        for (int q = 0; q < R; ++q) u[q] = xu[S::at(e0 + q * Ns)];
        C w[R];
#pragma unroll
        for (int q = 1; q < R; ++q) w[q] = Ns > 1 ? __ldg(ptw + (q - 1) * Ns + kk) : mk<C>(1.0, 0.0);
#pragma unroll
        for (int t = 0; t < TT; ++t) {
            C v[R];
            v[0] = u[0].v[t];
#pragma unroll
            for (int q = 1; q < R; ++q) v[q] = Ns > 1 ? mulc(u[q].v[t], w[q]) : u[q].v[t];
            dft_small<C, true>(R, v);
#pragma unroll
            for (int q = 0; q < R; ++q) u[q].v[t] = v[q];
        }
#pragma unroll
        for (int q = 0; q < R; ++q) xu[S::at(e0 + q * Ns)] = u[q];
    }
}

template <typename T, int RG, int KG>
__global__ void __launch_bounds__(256) k_ringfft_synth_ip(int L, int K, int R, int N, Radices rad,
                                                          const typename CplxOf<T>::type *__restrict__ G,
                                                          const typename CplxOf<T>::type *__restrict__ ptw,
                                                          const int *__restrict__ slotq,
                                                          const int *__restrict__ qslot,
                                                          typename CplxOf<T>::type *__restrict__ maps) {
    using C = typename CplxOf<T>::type;
    constexpr int TT = RG * KG;
    using S = Swz<TT * (int)sizeof(C)>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *x = reinterpret_cast<C *>(smem_raw);   // units [slot][TT]
    // CTA order: the k groups of one ring group adjacent (they share the cube's sectors)
    const int nkg = (K + KG) / KG;
    const int kg = (int)blockIdx.x % nkg;
    const int r0 = ((int)blockIdx.x / nkg) * RG, k0 = kg * KG;
    // blockIdx.y: sky of a multi-sky build (consecutive G and cube blocks)
    G += (int64_t)blockIdx.y * (K + 1) * R * (2 * L + 1);
    maps += (int64_t)blockIdx.y * R * N * (K + 1);
    const bool p2n = (N & (N - 1)) == 0;
    const int lgn = __ffs(N) - 1;
    // gather, slot by slot: lanes run over the ring slot, then the k slot, then
    // the slot s; slot s receives the first alias m >= -L of its input q =
    // slotq[s] by an asynchronous copy (zero when there is none), so that every
    // copy of the CTA is in flight at once
    const int total = N * TT;
    for (int u = threadIdx.x; u < total; u += blockDim.x) {
        const int ri = u % RG, ki = (u / RG) % KG, sl = u / TT;
        const int k = k0 + ki, r = r0 + ri;
        int q = __ldg(slotq + sl);
        if (!SL_GUARD(q >= 0 && q < N, 0x601u)) q = 0;
        const int m = q - N * (p2n ? (q + L) >> lgn : (q + L) / N);   // smallest m >= -L, m = q (mod N)
        const bool ok = k <= K && r < R && m <= L;
        const C *src = ok ? G + ((int64_t)k * (2 * L + 1) + (m + L)) * R + r : G;
        const unsigned dst = (unsigned)__cvta_generic_to_shared(x + S::at(sl) * TT + ri * KG + ki);
        if (sizeof(C) == 8)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(src),
                         "r"(ok ? 8 : 0) : "memory");
        else
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src),
                         "r"(ok ? 16 : 0) : "memory");
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    // the further aliases (2L + 1 > N): m = N - L + i, i < min(N, 2L + 1 - N), are
    // the aliases after the first of distinct q, each with its own multiples of N
    const int next = min(N, 2 * L + 1 - N);
    for (int u = threadIdx.x; u < next * TT; u += blockDim.x) {
        const int ri = u % RG, ki = (u / RG) % KG, i = u / TT;
        const int k = k0 + ki, r = r0 + ri;
        if (k > K || r >= R) continue;
        const int m0 = N - L + i;
        C acc = mk<C>(0.0, 0.0);
        for (int m = m0; m <= L; m += N) acc = add(acc, G[((int64_t)k * (2 * L + 1) + (m + L)) * R + r]);
        const int q = ((m0 % N) + N) % N;   // m0 < 0 when L > N
        int sq = __ldg(qslot + q);
        if (!SL_GUARD(sq >= 0 && sq < N, 0x602u)) continue;
        C *d = x + S::at(sq) * TT + ri * KG + ki;
        *d = add(*d, acc);
    }
    __syncthreads();
    int Ns = 1, off = 0;
    for (int pass = 0; pass < rad.n; ++pass) {
        const int Rp = (int)((rad.code >> (4 * pass)) & 15);
        switch (Rp) {
            case 8:   // FP64-class plans only: compiled for double2 alone, since a radix-8
                      // pass in the FP32 kernel raises its registers for every radix
                if constexpr (sizeof(C) == sizeof(double2)) dit_pass<C, 8, TT>(x, N, Ns, ptw + off);
                break;
            case 4: dit_pass<C, 4, TT>(x, N, Ns, ptw + off); break;
            case 2: dit_pass<C, 2, TT>(x, N, Ns, ptw + off); break;
            case 3: dit_pass<C, 3, TT>(x, N, Ns, ptw + off); break;
            default: dit_pass<C, 5, TT>(x, N, Ns, ptw + off); break;
        }
        __syncthreads();
        off += Ns * (Rp - 1);
        Ns *= Rp;
    }
    // write: lanes run over the k slot, then the ring slot, then j
    for (int u = threadIdx.x; u < total; u += blockDim.x) {
        const int ki = u % KG, ri = (u / KG) % RG, j = u / TT;
        const int k = k0 + ki, r = r0 + ri;
        if (k <= K && r < R) maps[((int64_t)r * N + j) * (K + 1) + k] = x[S::at(j) * TT + ri * KG + ki];
    }
}

__global__ void __launch_bounds__(256) k_ringdft_adjoint(int L, int K, int R, int N, Radices rad,
                                                         const double2 *__restrict__ fbar,
                                                         const double2 *__restrict__ tw,
                                                         double2 *__restrict__ Ghat) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2 *buf0 = reinterpret_cast<double2 *>(smem_raw);
    double2 *buf1 = buf0 + N;
    const int k = blockIdx.x % (K + 1);
    const int r = blockIdx.x / (K + 1);
    const double2 *in = fbar + (int64_t)r * N * (K + 1) + k;
    for (int j = threadIdx.x; j < N; j += blockDim.x) buf0[j] = in[(int64_t)j * (K + 1)];
    __syncthreads();
    const double2 *res = fft_smem<double2, false>(buf0, buf1, N, rad, tw);
    double2 *g = Ghat + ((int64_t)k * R + r) * (2 * L + 1);
    for (int m = -L + (int)threadIdx.x; m <= L; m += blockDim.x) {
        int q = m % N;
        if (q < 0) q += N;
        g[m + L] = res[q];
    }
}

// ------------------------------------------------------------------ cluster form
// Element e of a distributed buffer: CTA e / S of the cluster, slot e mod S.
template <typename C>
struct DistBuf {
    C *local;          // this CTA's slots (the same offset in every CTA of the cluster)
    int S, lgS;        // slots per CTA; log2 S when S is a power of two, else -1
    __device__ __forceinline__ C *at(cooperative_groups::cluster_group &cl, int e) const {
        const int r = lgS >= 0 ? e >> lgS : e / S;
        return cl.map_shared_rank(local, r) + (e - r * S);
    }
};

template <typename C, bool INV, int R>
__device__ __forceinline__ void fft_pass_cl(cooperative_groups::cluster_group &cl, const DistBuf<C> &src,
                                            const DistBuf<C> &dst, int N, int Ns, const C *__restrict__ tw,
                                            int g0, int gstride) {
    const int NR = N / R;
    const int stride = N / (Ns * R);
    const bool p2 = (Ns & (Ns - 1)) == 0;
    const int lg = __ffs(Ns) - 1;
    for (int t = g0; t < NR; t += gstride) {
        const int kk = p2 ? (t & (Ns - 1)) : t % Ns;
        const int blk = p2 ? (t >> lg) : t / Ns;
        C v[R];
#pragma unroll
        for (int q = 0; q < R; ++q) v[q] = *src.at(cl, t + q * NR);
        if (Ns > 1) {
            C w = tw[kk * stride];
            if (!INV) w.y = -w.y;
            C wq = w;
#pragma unroll
            for (int q = 1; q < R; ++q) {
                v[q] = mulc(v[q], wq);
                if (q + 1 < R) wq = mulc(wq, w);
            }
        }
        dft_small<C, INV>(R, v);
        const int base = blk * Ns * R + kk;
#pragma unroll
        for (int q = 0; q < R; ++q) *dst.at(cl, base + q * Ns) = v[q];
    }
}

// All passes over the cluster; returns which buffer (0 or 1) holds the result.
template <typename C, bool INV>
__device__ int fft_cluster(cooperative_groups::cluster_group &cl, const DistBuf<C> &b0, const DistBuf<C> &b1,
                           int N, const Radices &rad, const C *__restrict__ tw) {
    const int g0 = (int)cl.block_rank() * blockDim.x + threadIdx.x, gstride = (int)cl.num_blocks() * blockDim.x;
    int cur = 0, Ns = 1;
    for (int pass = 0; pass < rad.n; ++pass) {
        const int R = (int)((rad.code >> (4 * pass)) & 15);
        const DistBuf<C> &src = cur ? b1 : b0, &dst = cur ? b0 : b1;
        switch (R) {
            case 8:   // FP64-class plans only (as in the in-place form)
                if constexpr (sizeof(C) == sizeof(double2)) fft_pass_cl<C, INV, 8>(cl, src, dst, N, Ns, tw, g0, gstride);
                break;
            case 4: fft_pass_cl<C, INV, 4>(cl, src, dst, N, Ns, tw, g0, gstride); break;
            case 2: fft_pass_cl<C, INV, 2>(cl, src, dst, N, Ns, tw, g0, gstride); break;
            case 3: fft_pass_cl<C, INV, 3>(cl, src, dst, N, Ns, tw, g0, gstride); break;
            default: fft_pass_cl<C, INV, 5>(cl, src, dst, N, Ns, tw, g0, gstride); break;
        }
        cl.sync();
        cur ^= 1;
        Ns *= R;
    }
    return cur;
}

template <typename T>
__global__ void __launch_bounds__(256) k_ringfft_synth_cl(int L, int K, int R, int N, Radices rad,
                                                          const typename CplxOf<T>::type *__restrict__ G,
                                                          const typename CplxOf<T>::type *__restrict__ tw,
                                                          typename CplxOf<T>::type *__restrict__ maps) {
    using C = typename CplxOf<T>::type;
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nc = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    const int S = N / nc;
    DistBuf<C> b0{reinterpret_cast<C *>(smem_raw), S, (S & (S - 1)) == 0 ? __ffs(S) - 1 : -1};
    DistBuf<C> b1{b0.local + S, S, b0.lgS};
    // cluster index -> (ring, k): kRingGroup consecutive rings fastest (they share the sectors of G)
    int b = blockIdx.x / nc;
    const int rlo = b % kRingGroup;
    b /= kRingGroup;
    const int k = b % (K + 1);
    const int r = (b / (K + 1)) * kRingGroup + rlo;
    if (r >= R) return;   // uniform over the cluster
    G += (int64_t)blockIdx.y * (K + 1) * R * (2 * L + 1);
    maps += (int64_t)blockIdx.y * R * N * (K + 1);
    const C *g = G + (int64_t)k * (2 * L + 1) * R + r;
    for (int qq = threadIdx.x; qq < S; qq += blockDim.x) {
        const int q = rank * S + qq;
        int m = q - N * ((q + L) / N);
        C acc = mk<C>(0.0, 0.0);
        for (; m <= L; m += N) acc = add(acc, g[(int64_t)(m + L) * R]);
        b0.local[qq] = acc;
    }
    cl.sync();
    const int cur = fft_cluster<C, true>(cl, b0, b1, N, rad, tw);
    const C *res = cur ? b1.local : b0.local;
    C *out = maps + (int64_t)r * N * (K + 1) + k;
    for (int jj = threadIdx.x; jj < S; jj += blockDim.x) out[(int64_t)(rank * S + jj) * (K + 1)] = res[jj];
    cl.sync();   // no CTA leaves while another may still read its shared memory
}

__global__ void __launch_bounds__(256) k_ringdft_adjoint_cl(int L, int K, int R, int N, Radices rad,
                                                            const double2 *__restrict__ fbar,
                                                            const double2 *__restrict__ tw,
                                                            double2 *__restrict__ Ghat) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nc = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    const int S = N / nc;
    DistBuf<double2> b0{reinterpret_cast<double2 *>(smem_raw), S, (S & (S - 1)) == 0 ? __ffs(S) - 1 : -1};
    DistBuf<double2> b1{b0.local + S, S, b0.lgS};
    const int cidx = blockIdx.x / nc;
    const int k = cidx % (K + 1);
    const int r = cidx / (K + 1);
    const double2 *in = fbar + (int64_t)r * N * (K + 1) + k;
    for (int jj = threadIdx.x; jj < S; jj += blockDim.x) b0.local[jj] = in[(int64_t)(rank * S + jj) * (K + 1)];
    cl.sync();
    const int cur = fft_cluster<double2, false>(cl, b0, b1, N, rad, tw);
    const DistBuf<double2> &res = cur ? b1 : b0;
    double2 *g = Ghat + ((int64_t)k * R + r) * (2 * L + 1);
    for (int m = -L + rank * (int)blockDim.x + (int)threadIdx.x; m <= L; m += nc * (int)blockDim.x) {
        int q = m % N;
        if (q < 0) q += N;
        g[m + L] = *res.at(cl, q);
    }
    cl.sync();
}

// CTAs per cluster for a ring of N complex T2 values (two buffers): 1 when they fit
// one CTA's shared memory, else the smallest of 2, 4, 8 that fits and divides N.
static int fft_cluster_size(int N, size_t elem) {
    for (int c = 1; c <= 8; c *= 2)
        if (N % c == 0 && 2 * (size_t)(N / c) * elem <= (size_t)kFftSmemMax) return c;
    return 0;
}

static Radices radices_of(const sl_plan *p) {
    Radices r;
    r.n = p->nradix;
    r.code = 0;
    for (int i = 0; i < p->nradix; ++i) r.code |= (unsigned long long)p->radices[i] << (4 * i);
    return r;
}

SL_CHECK_READER(chk_fft)

// The synthesis runs in place (one buffer of nphi values per transform): one CTA
// while a single transform fits, else the two-buffer cluster form.
int ring_fft_cluster_size(const sl_plan *p) {
    const size_t elem = plan_wide(p->precision) ? sizeof(double2) : sizeof(float2);
    if ((size_t)p->nphi * elem <= (size_t)kFftSmemMax) return 1;
    return fft_cluster_size(p->nphi, elem);
}

size_t ring_fft_ip_smem(const sl_plan *p, int rg, int kg) {
    const int ub = rg * kg * (plan_wide(p->precision) ? (int)sizeof(double2) : (int)sizeof(float2));
    const int U = ub >= 128 ? 1 : 128 / ub;
    return (size_t)((p->nphi + U - 1) / U * U) * ub;   // slots rounded up to whole swizzle groups
}

// Default tile: 2 rings x 1 order within kFftIpBudget bytes of shared memory,
// else 1 x 1 (measured at lmax 1024, 1024 x 2048 rings, kmax 16, FP32 and FP64:
// 2 x 1 fastest, before 1 x 2, 1 x 1, 2 x 2, 4 x 1 and 4 x 2 -- the larger tiles
// lose more to fewer resident CTAs than they gain from wider requests).
constexpr size_t kFftIpBudget = 64 * 1024;

void ring_fft_tile(const sl_plan *p, int *rg, int *kg) {
    *rg = *kg = 0;
    if (ring_fft_cluster_size(p) != 1) return;
    if (p->fft_rg > 0) {
        *rg = p->fft_rg;
        *kg = p->fft_kg;
        return;
    }
    static const int cand[2][2] = {{2, 1}, {1, 1}};
    for (const auto &c : cand)
        if (ring_fft_ip_smem(p, c[0], c[1]) <= kFftIpBudget || (c[0] == 1 && c[1] == 1)) {
            *rg = c[0];
            *kg = c[1];
            return;
        }
}

template <typename T, int RG, int KG>
static cudaError_t launch_ip(sl_plan *p, const void *G, int nsky, void *maps) {
    using C = typename CplxOf<T>::type;
    const size_t sm = ring_fft_ip_smem(p, RG, KG);
    cudaError_t e = allow_dyn_smem(k_ringfft_synth_ip<T, RG, KG>, sm);
    if (e != cudaSuccess) return e;
    const unsigned nblk = (unsigned)(((p->R + RG - 1) / RG) * ((p->K + KG) / KG));
    const C *ptw = plan_wide(p->precision) ? (const C *)p->d_ptw64 : (const C *)p->d_ptw32;
    k_ringfft_synth_ip<T, RG, KG><<<dim3(nblk, (unsigned)nsky), 256, sm, p->stream>>>(
        p->L, p->K, p->R, p->nphi, radices_of(p), (const C *)G, ptw, p->d_fftperm, p->d_fftpos, (C *)maps);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_ip_tile(sl_plan *p, int rg, int kg, const void *G, int nsky, void *maps) {
    switch (rg * 4 + kg) {
        case 4 * 4 + 2: return launch_ip<T, 4, 2>(p, G, nsky, maps);
        case 2 * 4 + 2: return launch_ip<T, 2, 2>(p, G, nsky, maps);
        case 4 * 4 + 1: return launch_ip<T, 4, 1>(p, G, nsky, maps);
        case 2 * 4 + 1: return launch_ip<T, 2, 1>(p, G, nsky, maps);
        case 1 * 4 + 2: return launch_ip<T, 1, 2>(p, G, nsky, maps);
        default: return launch_ip<T, 1, 1>(p, G, nsky, maps);
    }
}

template <typename K_, typename... Args>
static cudaError_t launch_cluster(K_ kern, dim3 grid, int csize, size_t sm, cudaStream_t st, Args... args) {
    cudaError_t e = allow_dyn_smem(kern, sm);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

sl_status launch_ringfft_synth_from(sl_plan *p, const void *G, int nsky, void *maps) {
    const int ngrp = (p->R + kRingGroup - 1) / kRingGroup;
    const dim3 nblk((unsigned)(ngrp * kRingGroup * (p->K + 1)), (unsigned)nsky);
    int slot;
    const int csize = ring_fft_cluster_size(p);
    if (csize < 1) return set_error(SL_ERR_UNSUPPORTED, "nphi=%d: ring too long for an 8-CTA cluster", p->nphi);
    if (csize > 1) {
        const dim3 grid(nblk.x * (unsigned)csize, nblk.y);
        cudaError_t e;
        if (plan_wide(p->precision)) {
            const size_t sm = 2 * (size_t)(p->nphi / csize) * sizeof(double2);
            slot = timing_begin(p, "ringfft_f64");
            e = launch_cluster(k_ringfft_synth_cl<double>, grid, csize, sm, p->stream, p->L, p->K, p->R, p->nphi,
                               radices_of(p), (const double2 *)G, (const double2 *)p->d_tw64, (double2 *)maps);
        } else {
            const size_t sm = 2 * (size_t)(p->nphi / csize) * sizeof(float2);
            slot = timing_begin(p, "ringfft_f32");
            e = launch_cluster(k_ringfft_synth_cl<float>, grid, csize, sm, p->stream, p->L, p->K, p->R, p->nphi,
                               radices_of(p), (const float2 *)G, (const float2 *)p->d_tw32, (float2 *)maps);
        }
        timing_end(p, slot);
        return cuda_check(e, "k_ringfft_synth_cl launch");
    }
    int rg, kg;
    ring_fft_tile(p, &rg, &kg);
    cudaError_t e;
    if (plan_wide(p->precision)) {
        slot = timing_begin(p, "ringfft_f64");
        e = launch_ip_tile<double>(p, rg, kg, G, nsky, maps);
    } else {
        slot = timing_begin(p, "ringfft_f32");
        e = launch_ip_tile<float>(p, rg, kg, G, nsky, maps);
    }
    timing_end(p, slot);
    return cuda_check(e, "k_ringfft_synth_ip launch");
}

sl_status launch_ringfft_synth(sl_plan *p, void *maps) { return launch_ringfft_synth_from(p, p->d_G, 1, maps); }

sl_status launch_ringdft_adjoint(sl_plan *p, const double2 *fbar) {
    const unsigned nblk = (unsigned)((p->K + 1) * p->R);
    const int csize = fft_cluster_size(p->nphi, sizeof(double2));
    if (csize < 1) return set_error(SL_ERR_UNSUPPORTED, "nphi=%d: ring too long for an 8-CTA cluster", p->nphi);
    if (csize > 1) {
        const size_t sm = 2 * (size_t)(p->nphi / csize) * sizeof(double2);
        int slot = timing_begin(p, "ringdft_adj");
        cudaError_t e = launch_cluster(k_ringdft_adjoint_cl, dim3(nblk * (unsigned)csize), csize, sm, p->stream, p->L,
                                       p->K, p->R, p->nphi, radices_of(p), fbar, (const double2 *)p->d_tw64,
                                       p->d_Gadj);
        timing_end(p, slot);
        return cuda_check(e, "k_ringdft_adjoint_cl launch");
    }
    const size_t sm = 2 * (size_t)p->nphi * sizeof(double2);
    cudaError_t e = allow_dyn_smem(k_ringdft_adjoint, sm);
    if (e != cudaSuccess) return cuda_check(e, "k_ringdft_adjoint smem attribute");
    int slot = timing_begin(p, "ringdft_adj");
    k_ringdft_adjoint<<<nblk, 256, sm, p->stream>>>(p->L, p->K, p->R, p->nphi, radices_of(p), fbar, p->d_tw64,
                                                    p->d_Gadj);
    timing_end(p, slot);
    return cuda_check(cudaGetLastError(), "k_ringdft_adjoint launch");
}

}  // namespace sl
