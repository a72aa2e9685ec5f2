// k_fft.cu -- the phi direction of the cube (Sect. 2.1, step 1 of the
// two-step algorithm: the synthesis along each ring) and its transpose.
//
// Synthesis (one CTA per (ring r, k)):
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
// The DFT is a self-sorting (Stockham) mixed-radix FFT with radices 4, 2, 3, 5
// entirely in shared memory, twiddles from a table e^{+2 pi i j/nphi} built in
// long double on the host.  Each pass computes, for butterfly t in [0, N/R):
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
template <typename C> __device__ __forceinline__ C scal(C a, double s) {
    C r;
    r.x = a.x * s;
    r.y = a.y * s;
    return r;
}

// cos/sin of 2 pi/3, 2 pi/5, 4 pi/5 (from their closed forms)
constexpr double kS3 = 0.86602540378443864676;   // sqrt(3)/2
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
    unsigned long long code;   // radix of pass i in bits [3i, 3i + 3)
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
        const int R = (int)((rad.code >> (3 * pass)) & 7);
        switch (R) {
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

constexpr int kRingGroup = 4;   // rings per sector of an FP32 G row

template <typename T>
__global__ void __launch_bounds__(256) k_ringfft_synth(int L, int K, int R, int N, Radices rad,
                                                       const typename CplxOf<T>::type *__restrict__ G,
                                                       const typename CplxOf<T>::type *__restrict__ tw,
                                                       typename CplxOf<T>::type *__restrict__ maps) {
    using C = typename CplxOf<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf0 = reinterpret_cast<C *>(smem_raw);
    C *buf1 = buf0 + N;
    // CTA order: kRingGroup consecutive rings fastest, then k, then the ring
    // group, so that the rings sharing a sector of G (ring index fastest) and the
    // k values sharing a sector of the cube ([r][j][k]) run close together
    int b = blockIdx.x;
    const int rlo = b % kRingGroup;
    b /= kRingGroup;
    const int k = b % (K + 1);
    const int r = (b / (K + 1)) * kRingGroup + rlo;
    if (r >= R) return;
    // blockIdx.y: sky of a multi-sky build (consecutive G and cube blocks)
    G += (int64_t)blockIdx.y * (K + 1) * R * (2 * L + 1);
    maps += (int64_t)blockIdx.y * R * N * (K + 1);
    const C *g = G + (int64_t)k * (2 * L + 1) * R + r;
    // the first alias of kGather values of q per thread is loaded before any is used
    constexpr int kGather = 8;
    const bool p2n = (N & (N - 1)) == 0;
    const int lgn = __ffs(N) - 1;
    for (int q0 = threadIdx.x; q0 < N; q0 += kGather * blockDim.x) {
        C v[kGather];
#pragma unroll
        for (int i = 0; i < kGather; ++i) {
            const int q = q0 + i * (int)blockDim.x;
            const int m = q - N * (p2n ? (q + L) >> lgn : (q + L) / N);   // smallest m >= -L, m = q (mod N)
            v[i] = (q < N && m <= L) ? g[(int64_t)(m + L) * R] : mk<C>(0.0, 0.0);
        }
#pragma unroll
        for (int i = 0; i < kGather; ++i) {
            const int q = q0 + i * (int)blockDim.x;
            if (q < N) {
                C acc = v[i];
                for (int m = q - N * (p2n ? (q + L) >> lgn : (q + L) / N) + N; m <= L; m += N)
                    acc = add(acc, g[(int64_t)(m + L) * R]);
                buf0[q] = acc;
            }
        }
    }
    __syncthreads();
    const C *res = fft_smem<C, true>(buf0, buf1, N, rad, tw);
    C *out = maps + (int64_t)r * N * (K + 1) + k;
    for (int j = threadIdx.x; j < N; j += blockDim.x) out[(int64_t)j * (K + 1)] = res[j];
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
        const int R = (int)((rad.code >> (3 * pass)) & 7);
        const DistBuf<C> &src = cur ? b1 : b0, &dst = cur ? b0 : b1;
        switch (R) {
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
    // cluster index -> (ring, k), rings of a sector together as in k_ringfft_synth
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

int ring_fft_cluster_size(const sl_plan *p) {
    return fft_cluster_size(p->nphi, plan_wide(p->precision) ? sizeof(double2) : sizeof(float2));
}

template <typename K_, typename... Args>
static cudaError_t launch_cluster(K_ kern, dim3 grid, int csize, size_t sm, cudaStream_t st, Args... args) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
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

static Radices radices_of(const sl_plan *p) {
    Radices r;
    r.n = p->nradix;
    r.code = 0;
    for (int i = 0; i < p->nradix; ++i) r.code |= (unsigned long long)p->radices[i] << (3 * i);
    return r;
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
    if (plan_wide(p->precision)) {
        const size_t sm = 2 * (size_t)p->nphi * sizeof(double2);
        cudaFuncSetAttribute(k_ringfft_synth<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        slot = timing_begin(p, "ringfft_f64");
        k_ringfft_synth<double><<<nblk, 256, sm, p->stream>>>(p->L, p->K, p->R, p->nphi, radices_of(p),
                                                              (const double2 *)G, p->d_tw64, (double2 *)maps);
    } else {
        const size_t sm = 2 * (size_t)p->nphi * sizeof(float2);
        cudaFuncSetAttribute(k_ringfft_synth<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        slot = timing_begin(p, "ringfft_f32");
        k_ringfft_synth<float><<<nblk, 256, sm, p->stream>>>(p->L, p->K, p->R, p->nphi, radices_of(p),
                                                             (const float2 *)G, p->d_tw32, (float2 *)maps);
    }
    timing_end(p, slot);
    return cuda_check(cudaGetLastError(), "k_ringfft_synth launch");
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
    cudaFuncSetAttribute(k_ringdft_adjoint, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int slot = timing_begin(p, "ringdft_adj");
    k_ringdft_adjoint<<<nblk, 256, sm, p->stream>>>(p->L, p->K, p->R, p->nphi, radices_of(p), fbar, p->d_tw64,
                                                    p->d_Gadj);
    timing_end(p, slot);
    return cuda_check(cudaGetLastError(), "k_ringdft_adjoint launch");
}

}  // namespace sl
