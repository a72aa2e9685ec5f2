// k_interp_df.cu -- step 2 of the two-step algorithm (Sect. 2.1) for SL_DF64
// plans: the same 4-point Lagrange interpolation and conjugate-pair phase sum
// as the FP64 kernel,
//
//   c = Re S_0 + 2 sum_{k>=1} Re(e^{ik psi} S_k),   S_k = sum_q w_q F_k(node q),
//
// with the weights, the stencil sums and the phase recurrence in double-float
// arithmetic (df.cuh) on the FP32 pipes.  Layout as the FP32 tile-staged
// kernel: one CTA per work item (<= kWorkChunk sorted samples of one tile),
// the tile's nodes (rows tr*4-2 .. tr*4+4, columns tc*TC-1 .. tc*TC+TC+1,
// every k) staged in shared memory as [k][row][col] float4 (Re hi, Re lo,
// Im hi, Im lo), converted from the double cube while staging, ghost rows
// folded in with (-1)^k.  cos psi and sin psi come from the FP64 sincos (on
// the otherwise idle FP64 pipe).
#include "df.cuh"
#include "sl_internal.cuh"

namespace sl {

struct DfArgs {
    InterpGeom g;
    const double2 *maps;
    const StencilRec64 *rec;
    const double *psi;
    const unsigned *perm, *start, *chunk_off;
    int ntiles, ncell;
    double *tod;       // forward: written; adjoint: the input TOD
    double2 *fbar;     // adjoint cube (adjoint only)
};

__device__ __forceinline__ dfl df_ld(const float2 *p) {
    const float2 v = __ldg(p);
    return dfl{v.x, v.y};
}

// p-point Lagrange weights in double-float (the same prefix / suffix products
// as lagrange_theta and lagrange_phi).
template <int P>
__device__ __forceinline__ void weights_df(const float2 *rt, dfl d0, dfl f, dfl wt[P], dfl wp[P]) {
    dfl d[P], pre[P + 1], suf[P + 1];
    const dfl one = df_make(1.f, 0.f);
#pragma unroll
    for (int a = 0; a < P; ++a) d[a] = (a == 0) ? d0 : df_sub(d0, df_ld(rt + a));
    pre[0] = one;
    suf[P] = one;
#pragma unroll
    for (int a = 0; a < P; ++a) pre[a + 1] = df_mul(pre[a], d[a]);
#pragma unroll
    for (int a = P - 1; a >= 0; --a) suf[a] = df_mul(suf[a + 1], d[a]);
#pragma unroll
    for (int a = 0; a < P; ++a) wt[a] = df_mul(df_ld(rt + P + a), df_mul(pre[a], suf[a + 1]));
#pragma unroll
    for (int b = 0; b < P; ++b) d[b] = df_sub(f, df_make((float)(b - P / 2 + 1), 0.f));
#pragma unroll
    for (int b = 0; b < P; ++b) pre[b + 1] = df_mul(pre[b], d[b]);
#pragma unroll
    for (int b = P - 1; b >= 0; --b) suf[b] = df_mul(suf[b + 1], d[b]);
#pragma unroll
    for (int b = 0; b < P; ++b) {
        const double inv = uniform_inv_den<P>(b);
        const float ih = (float)inv;
        wp[b] = df_mul(df_mul(pre[b], suf[b + 1]), df_make(ih, (float)(inv - (double)ih)));
    }
}

template <int TC, int P>
__global__ void __launch_bounds__(256) k_interp_df_tiled(const DfArgs A) {
    constexpr int TW = TC + P - 1, NR = kTileRows + P - 1, NN = NR * TW;
    const InterpGeom &g = A.g;
    const int K1 = g.K + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4 *node = reinterpret_cast<float4 *>(smem_raw);   // [K1][NR][TW]
    const int e_step_n = (int)blockDim.x / K1, e_step_k = (int)blockDim.x - e_step_n * K1;
    const int e0_n = (int)threadIdx.x / K1, e0_k = (int)threadIdx.x - e0_n * K1;
    const unsigned nchunks = A.chunk_off[A.ntiles];
    int staged_tile = -1;
    for (unsigned v = blockIdx.x; v < nchunks; v += gridDim.x) {
        const int tile = find_tile(A.chunk_off, A.ntiles, v);
        const unsigned c = v - A.chunk_off[tile];
        const unsigned s_beg = A.start[(int64_t)tile * A.ncell] + c * kWorkChunk;
        const unsigned s_end = min(A.start[(int64_t)(tile + 1) * A.ncell], s_beg + kWorkChunk);
        const int tr = tile / g.ntc, tcol = tile - tr * g.ntc;
        const int rowlo = tr * kTileRows - P / 2, collo = tcol * TC - P / 2 + 1;
        if (tile != staged_tile) {
            __syncthreads();
            // element e = node * K1 + k, walked with blockDim.x steps
            for (int nd = e0_n, k = e0_k; nd < NN;) {
                const int r = nd / TW, cc = nd - r * TW;
                const int row = rowlo + r;
                float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
                if (row >= -P / 2 && row <= g.R - 1 + P / 2) {
                    int ring = row, col = collo + cc;
                    if (row < 0 || row >= g.R) {
                        ring = (row < 0) ? -1 - row : 2 * g.R - 1 - row;
                        col += g.nphi >> 1;
                    }
                    if (col < 0) col += g.nphi;
                    if (col >= g.nphi) col -= g.nphi;
                    if (col >= g.nphi) col -= g.nphi;
                    if (!SL_GUARD(ring >= 0 && ring < g.R && col >= 0 && col < g.nphi, 0x301u)) ring = col = 0;
                    double2 d = __ldg(A.maps + ((int64_t)ring * g.nphi + col) * K1 + k);
                    if (ring != row && (k & 1)) { d.x = -d.x; d.y = -d.y; }
                    const dfl re = df_from_d(d.x), im = df_from_d(d.y);
                    val = make_float4(re.h, re.l, im.h, im.l);
                }
                node[k * NN + nd] = val;
                nd += e_step_n;
                k += e_step_k;
                if (k >= K1) { k -= K1; ++nd; }
            }
            __syncthreads();
            staged_tile = tile;
        }
        for (unsigned t = s_beg + threadIdx.x; t < s_end; t += blockDim.x) {
            const unsigned s = A.perm[t];
            const StencilRec64 r = A.rec[s];
            const int i = (int)(r.cell >> 16) - 1, j = (int)(r.cell & 0xffffu);
            double sp, cp;
            sincos(__ldg(A.psi + s), &sp, &cp);
            // Lagrange weights in double-float
            dfl wt[P], wp[P];
            weights_df<P>(g.rowtab_df + (size_t)(i + 1) * 2 * P, df_from_d(r.dth), df_from_d(r.fph), wt, wp);
            dfl w[P * P];
#pragma unroll
            for (int q = 0; q < P * P; ++q) w[q] = df_mul(wt[q / P], wp[q % P]);
            int nb0 = (i - P / 2 + 1 - rowlo) * TW + (j - P / 2 + 1 - collo);
            if (!SL_GUARD(nb0 >= 0 && nb0 + (P - 1) * TW + (P - 1) < NN, 0x302u)) nb0 = 0;
            const float4 *nb = node + nb0;
            const dfl two = df_make(2.f, 0.f);
            // C_k = 2 cos(k psi), S_k = 2 sin(k psi): X_{k+1} = (2 cos psi) X_k - X_{k-1}
            const dfl c1 = df_from_d(2.0 * cp);
            dfl Ck = c1, Sk = df_from_d(2.0 * sp), Ckm = two, Skm = df_make(0.f, 0.f);
            dacc acc;
            {
                dacc sr;
                dacc_zero(sr);
#pragma unroll
                for (int q = 0; q < P * P; ++q) {
                    const float4 v4 = nb[(q / P) * TW + (q % P)];
                    dacc_mac(sr, w[q], dfl{v4.x, v4.y});
                }
                acc = sr;
            }
            nb += NN;
            for (int k = 1; k < K1; ++k, nb += NN) {
                dacc sr, si;
                dacc_zero(sr);
                dacc_zero(si);
#pragma unroll
                for (int q = 0; q < P * P; ++q) {
                    const float4 v4 = nb[(q / P) * TW + (q % P)];
                    dacc_mac(sr, w[q], dfl{v4.x, v4.y});
                    dacc_mac(si, w[q], dfl{v4.z, v4.w});
                }
                dacc_mac(acc, Ck, dacc_get(sr));
                dacc_mac(acc, df_neg(Sk), dacc_get(si));
                const dfl cn = df_fma(c1, Ck, df_neg(Ckm)), sn = df_fma(c1, Sk, df_neg(Skm));
                Ckm = Ck;
                Skm = Sk;
                Ck = cn;
                Sk = sn;
            }
            A.tod[s] = df_to_d(dacc_get(acc));
        }
    }
}

// ------------------------------------------------------------------ adjoint
// The transpose of the interpolation for SL_DF64 plans: the FP64 kernel's tile
// scatter with the weights, the phases and the shared-memory accumulation in
// double-float (each accumulator an unnormalised high/low pair); the tile is
// flushed to the double adjoint cube with atomic additions.
constexpr int kNBD = 64;   // samples staged per batch (32 when kmax + 1 > 64, to fit shared memory)
__host__ __device__ __forceinline__ int kNBD_of(int K1) { return K1 > 64 ? kNBD / 2 : kNBD; }

template <int P>
__global__ void k_interp_adjoint_df(const DfArgs A) {
    constexpr int NQ = P * P;
    const InterpGeom &g = A.g;
    const int K1 = g.K + 1;
    const int TC = g.tile_cols;
    const int tw = TC + P - 1, th_rows = kTileRows + P - 1, nnode = th_rows * tw;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4 *acc = reinterpret_cast<float4 *>(smem_raw);               // [nnode][K1] (Re h, Re l, Im h, Im l)
    float4 *PH = acc + (size_t)nnode * K1;                            // [kNBD][K1]
    float2 *W = reinterpret_cast<float2 *>(PH + (size_t)kNBD_of(K1) * K1);   // [kNBD][NQ]
    int *LOC = reinterpret_cast<int *>(W + (size_t)kNBD_of(K1) * NQ);        // [kNBD]

    const unsigned nchunks = A.chunk_off[A.ntiles];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    for (int e = threadIdx.x; e < nnode * K1; e += blockDim.x) acc[e] = make_float4(0.f, 0.f, 0.f, 0.f);

    for (unsigned v = blockIdx.x; v < nchunks; v += gridDim.x) {
        const int tile = find_tile(A.chunk_off, A.ntiles, v);
        const unsigned c = v - A.chunk_off[tile];
        const unsigned s_beg = A.start[(int64_t)tile * A.ncell] + c * kWorkChunk;
        const unsigned s_end = min(A.start[(int64_t)(tile + 1) * A.ncell], s_beg + kWorkChunk);
        const int tr = tile / g.ntc, tcol = tile % g.ntc;
        const int rowlo = tr * kTileRows - P / 2, collo = tcol * TC - P / 2 + 1;
        __syncthreads();
        for (unsigned b0 = s_beg; b0 < s_end; b0 += (unsigned)kNBD_of(K1)) {
            const int nb = (int)min((unsigned)kNBD_of(K1), s_end - b0);
            // phase A: per-sample weights, node location and phases eps_k y e^{-ik psi}
            if ((int)threadIdx.x < nb) {
                const unsigned s = A.perm[b0 + threadIdx.x];
                const StencilRec64 r = A.rec[s];
                const int i = (int)(r.cell >> 16) - 1, j = (int)(r.cell & 0xffffu);
                dfl wt[P], wp[P];
                weights_df<P>(g.rowtab_df + (size_t)(i + 1) * 2 * P, df_from_d(r.dth), df_from_d(r.fph), wt, wp);
                float2 *ws = W + threadIdx.x * NQ;
#pragma unroll
                for (int ra = 0; ra < P; ++ra)
#pragma unroll
                    for (int cb = 0; cb < P; ++cb) {
                        const dfl w = df_mul(wt[ra], wp[cb]);
                        ws[ra * P + cb] = make_float2(w.h, w.l);
                    }
                int loc = (i - P / 2 + 1 - rowlo) * tw + (j - P / 2 + 1 - collo);
                if (!SL_GUARD(loc >= 0 && loc + (P - 1) * tw + (P - 1) < nnode, 0x303u)) loc = 0;
                LOC[threadIdx.x] = loc;
                double sp, cp;
                sincos(__ldg(A.psi + s), &sp, &cp);
                const double yv = A.tod[s];
                const dfl y1 = df_from_d(yv), y2 = df_from_d(2.0 * yv), c2 = df_from_d(2.0 * cp);
                dfl ck = df_make(1.f, 0.f), sk = df_make(0.f, 0.f), ckm = df_from_d(cp), skm = df_from_d(-sp);
                float4 *Ps = PH + (size_t)threadIdx.x * K1;
                for (int k = 0; k <= g.K; ++k) {
                    const dfl sc = (k == 0) ? y1 : y2;
                    const dfl re = df_mul(sc, ck), im = df_neg(df_mul(sc, sk));
                    Ps[k] = make_float4(re.h, re.l, im.h, im.l);
                    const dfl cn = df_fma(c2, ck, df_neg(ckm)), sn = df_fma(c2, sk, df_neg(skm));
                    ckm = ck;
                    skm = sk;
                    ck = cn;
                    sk = sn;
                }
            }
            __syncthreads();
            // phase B: warp w owns k-pairs w, w + nwarps, ...; lanes over (node, k
            // parity); register sums while the cell stays the same (cell order),
            // added to the shared tile when it changes
            constexpr int NE = (2 * NQ + 31) / 32;
            for (int kp = warp; 2 * kp <= g.K; kp += nwarps) {
                dacc rr[NE], ri[NE];
#pragma unroll
                for (int t = 0; t < NE; ++t) {
                    dacc_zero(rr[t]);
                    dacc_zero(ri[t]);
                }
                int cur_loc = nb > 0 ? LOC[0] : 0;
                for (int sidx = 0; sidx <= nb; ++sidx) {
                    const int loc = (sidx < nb) ? LOC[sidx] : -1;
                    if (loc != cur_loc) {       // warp-uniform
#pragma unroll
                        for (int t = 0; t < NE; ++t) {
                            const int e = lane + 32 * t;
                            const int q = e % NQ, kk = 2 * kp + e / NQ;
                            if (e < 2 * NQ && kk <= g.K) {
                                float4 &dst = acc[(size_t)(cur_loc + (q / P) * tw + (q % P)) * K1 + kk];
                                const float4 c = dst;
                                dacc sr{c.x, c.y}, si{c.z, c.w};
                                dacc_add(sr, dacc_get(rr[t]));
                                dacc_add(si, dacc_get(ri[t]));
                                dst = make_float4(sr.h, sr.l, si.h, si.l);
                            }
                            dacc_zero(rr[t]);
                            dacc_zero(ri[t]);
                        }
                        __syncwarp(0xffffffffu);
                        cur_loc = loc;
                    }
                    if (sidx == nb) break;
#pragma unroll
                    for (int t = 0; t < NE; ++t) {
                        const int e = lane + 32 * t;
                        const int q = e % NQ, kk = 2 * kp + e / NQ;
                        if (e < 2 * NQ && kk <= g.K) {
                            const float2 w = W[sidx * NQ + q];
                            const float4 ph = PH[(size_t)sidx * K1 + kk];
                            dacc_mac(rr[t], dfl{w.x, w.y}, dfl{ph.x, ph.y});
                            dacc_mac(ri[t], dfl{w.x, w.y}, dfl{ph.z, ph.w});
                        }
                    }
                }
            }
            __syncthreads();
        }
        // flush the tile (ghost rows fold onto their ring at phi + pi with (-1)^k)
        for (int e = threadIdx.x; e < nnode * K1; e += blockDim.x) {
            const float4 val = acc[e];
            if (val.x == 0.f && val.y == 0.f && val.z == 0.f && val.w == 0.f) continue;
            acc[e] = make_float4(0.f, 0.f, 0.f, 0.f);
            const int kk = e % K1;
            const int node = e / K1;
            const int row = rowlo + node / tw;
            int col = collo + node % tw;
            if (row < -P / 2 || row > g.R - 1 + P / 2) continue;
            int ring = row;
            double sg = 1.0;
            if (row < 0 || row >= g.R) {
                ring = (row < 0) ? -1 - row : 2 * g.R - 1 - row;
                col += g.nphi / 2;
                if (kk & 1) sg = -1.0;
            }
            col %= g.nphi;
            if (col < 0) col += g.nphi;
            if (!SL_GUARD(ring >= 0 && ring < g.R, 0x304u)) continue;
            double2 *o = A.fbar + ((int64_t)ring * g.nphi + col) * K1 + kk;
            atomicAdd(&o->x, sg * ((double)val.x + (double)val.y));
            atomicAdd(&o->y, sg * ((double)val.z + (double)val.w));
        }
    }
}

size_t interp_adjoint_df_smem_tc(const sl_plan *p, int tc) {
    const int K1 = p->K + 1, P = p->p;
    const int nnode = (kTileRows + P - 1) * (tc + P - 1);
    return (size_t)nnode * K1 * sizeof(float4) + (size_t)kNBD_of(K1) * K1 * sizeof(float4) +
           (size_t)kNBD_of(K1) * P * P * sizeof(float2) + (size_t)kNBD_of(K1) * sizeof(int);
}

sl_status launch_interp_adjoint_df(sl_plan *p, const SortBufs &b, int fine, const double *psi, const double *tod,
                                   double2 *fbar) {
    if (!b.chunk_off) return set_error(SL_ERR_ARG, "adjoint interpolation needs the per-tile work list");
    DfArgs a;
    a.g = p->geom;
    a.maps = nullptr;
    a.rec = (const StencilRec64 *)b.rec;
    a.psi = psi;
    a.perm = b.perm;
    a.start = b.hist;
    a.chunk_off = b.chunk_off;
    a.ntiles = p->ntiles;
    a.ncell = fine ? kTileRows * p->geom.tile_cols : 1;
    a.tod = const_cast<double *>(tod);   // read only here
    a.fbar = fbar;
    const int K1 = p->K + 1;
    const size_t sm = interp_adjoint_df_smem_tc(p, p->geom.tile_cols);
    int nwarps = (K1 + 1) / 2;
    if (nwarps < 2) nwarps = 2;
    if (nwarps > 16) nwarps = 16;
    void (*kern)(const DfArgs);
    switch (p->p) {
        case 2: kern = k_interp_adjoint_df<2>; break;
        case 4: kern = k_interp_adjoint_df<4>; break;
        case 6: kern = k_interp_adjoint_df<6>; break;
        default: return set_error(SL_ERR_UNSUPPORTED, "interp_order %d", p->p);
    }
    cudaError_t e = allow_dyn_smem(kern, sm);
    if (e != cudaSuccess) return cuda_check(e, "k_interp_adjoint_df smem attribute");
    int per_sm = 1, nsm = 152;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * nwarps, sm);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device);
    if (per_sm < 1) per_sm = 1;
    const int slot = timing_begin(p, "interp_adj_df");
    kern<<<(unsigned)(nsm * per_sm), 32 * nwarps, sm, p->stream>>>(a);
    timing_end(p, slot);
    return cuda_check(cudaGetLastError(), "k_interp_adjoint_df launch");
}

size_t interp_df_tiled_smem_tc(const sl_plan *p, int tc) {
    return (size_t)(kTileRows + p->p - 1) * (tc + p->p - 1) * (p->K + 1) * sizeof(float4);
}

sl_status launch_interp_df(sl_plan *p, const SortBufs &b, int fine, const void *maps, const double *psi, int64_t n,
                           double *tod) {
    if (!b.chunk_off) return set_error(SL_ERR_ARG, "double-float interpolation needs the per-tile work list");
    DfArgs a;
    a.g = p->geom;
    a.maps = (const double2 *)maps;
    a.rec = (const StencilRec64 *)b.rec;
    a.psi = psi;
    a.perm = b.perm;
    a.start = b.hist;
    a.chunk_off = b.chunk_off;
    a.ntiles = p->ntiles;
    a.ncell = fine ? kTileRows * p->geom.tile_cols : 1;
    a.tod = tod;
    a.fbar = nullptr;
    const size_t sm = interp_df_tiled_smem_tc(p, p->geom.tile_cols);
    void (*kern)(const DfArgs) = nullptr;
#define SL_TILED(TCV, PV) \
    if (p->geom.tile_cols == TCV && p->p == PV) kern = k_interp_df_tiled<TCV, PV>;
    SL_TILED(32, 4) SL_TILED(16, 4) SL_TILED(8, 4)
    SL_TILED(32, 2) SL_TILED(16, 2) SL_TILED(8, 2)
    SL_TILED(32, 6) SL_TILED(16, 6) SL_TILED(8, 6)
#undef SL_TILED
    if (!kern) return set_error(SL_ERR_UNSUPPORTED, "tile width %d, interp_order %d", p->geom.tile_cols, p->p);
    cudaError_t e = allow_dyn_smem(kern, sm);
    if (e != cudaSuccess) return cuda_check(e, "k_interp_df_tiled smem attribute");
    int per_sm = 1, nsm = 152;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, sm);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device);
    if (per_sm < 1) per_sm = 1;
    const int slot = timing_begin(p, "interp_df");
    kern<<<(unsigned)(nsm * per_sm), 256, sm, p->stream>>>(a);
    timing_end(p, slot);
    (void)n;
    return cuda_check(cudaGetLastError(), "k_interp_df launch");
}

SL_CHECK_READER(chk_interp_df)

}  // namespace sl
