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
    double *tod;
};

__device__ __forceinline__ dfl df_ld(const float2 *p) {
    const float2 v = __ldg(p);
    return dfl{v.x, v.y};
}

template <int TC>
__global__ void __launch_bounds__(256) k_interp_df_tiled(const DfArgs A) {
    constexpr int TW = TC + 3, NR = kTileRows + 3, NN = NR * TW;
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
        const int rowlo = tr * kTileRows - 2, collo = tcol * TC - 1;
        if (tile != staged_tile) {
            __syncthreads();
            // element e = node * K1 + k, walked with blockDim.x steps
            for (int nd = e0_n, k = e0_k; nd < NN;) {
                const int r = nd / TW, cc = nd - r * TW;
                const int row = rowlo + r;
                float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
                if (row >= -2 && row <= g.R + 1) {
                    int ring = row, col = collo + cc;
                    if (row < 0 || row >= g.R) {
                        ring = (row < 0) ? -1 - row : 2 * g.R - 1 - row;
                        col += g.nphi >> 1;
                    }
                    if (col < 0) col += g.nphi;
                    if (col >= g.nphi) col -= g.nphi;
                    if (col >= g.nphi) col -= g.nphi;
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
            const float2 *rt = g.rowtab_df + (size_t)(i + 1) * 8;
            const dfl d0 = df_from_d(r.dth), f = df_from_d(r.fph);
            const dfl d1 = df_sub(d0, df_ld(rt + 1)), d2 = df_sub(d0, df_ld(rt + 2)), d3 = df_sub(d0, df_ld(rt + 3));
            const dfl p01 = df_mul(d0, d1), p23 = df_mul(d2, d3);
            const dfl wt[4] = {df_mul(df_ld(rt + 4), df_mul(d1, p23)), df_mul(df_ld(rt + 5), df_mul(d0, p23)),
                               df_mul(df_ld(rt + 6), df_mul(p01, d3)), df_mul(df_ld(rt + 7), df_mul(p01, d2))};
            const dfl one = df_make(1.f, 0.f), two = df_make(2.f, 0.f);
            const dfl a = df_add(f, one), cm = df_sub(f, one), d = df_sub(f, two);
            const dfl cd = df_mul(cm, d), ab = df_mul(a, f);
            // 1/6 and 1/2 as double-float: 1/6 = h + l exactly to 2^-48
            const dfl sixth = df_make(0.16666667163372039795f, -4.9670538793103396892e-09f);
            const dfl wp[4] = {df_neg(df_mul(df_mul(f, cd), sixth)), df_mul(df_mul(a, cd), df_make(0.5f, 0.f)),
                               df_neg(df_mul(df_mul(ab, d), df_make(0.5f, 0.f))), df_mul(df_mul(ab, cm), sixth)};
            dfl w[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) w[q] = df_mul(wt[q >> 2], wp[q & 3]);
            const float4 *nb = node + (i - 1 - rowlo) * TW + (j - 1 - collo);
            // C_k = 2 cos(k psi), S_k = 2 sin(k psi): X_{k+1} = (2 cos psi) X_k - X_{k-1}
            const dfl c1 = df_from_d(2.0 * cp);
            dfl Ck = c1, Sk = df_from_d(2.0 * sp), Ckm = two, Skm = df_make(0.f, 0.f);
            dacc acc;
            {
                dacc sr;
                dacc_zero(sr);
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const float4 v4 = nb[(q >> 2) * TW + (q & 3)];
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
                for (int q = 0; q < 16; ++q) {
                    const float4 v4 = nb[(q >> 2) * TW + (q & 3)];
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

size_t interp_df_tiled_smem_tc(const sl_plan *p, int tc) {
    return (size_t)(kTileRows + 3) * (tc + 3) * (p->K + 1) * sizeof(float4);
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
    const size_t sm = interp_df_tiled_smem_tc(p, p->geom.tile_cols);
    void (*kern)(const DfArgs);
    switch (p->geom.tile_cols) {
        case 32: kern = k_interp_df_tiled<32>; break;
        case 16: kern = k_interp_df_tiled<16>; break;
        case 8: kern = k_interp_df_tiled<8>; break;
        default: return set_error(SL_ERR_UNSUPPORTED, "tile width %d", p->geom.tile_cols);
    }
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
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

}  // namespace sl
