// k_interp.cu -- step 2 of the two-step algorithm (Sect. 2.1): the cube is
// evaluated at each pointing and summed over k with the conjugate-pair phases
//
//   c = Re S_0 + 2 sum_{k>=1} Re(e^{ik psi} S_k),   S_k = sum_{a,b} wt_a wp_b F_k(row a, col b),
//
// plus its transpose.  The paper leaves the interpolation scheme open; here it
// is separable 4-point Lagrange: wt from the actual (extended) ring
// colatitudes, wp for uniform phi nodes j-1..j+2 (periodic).  Stencil rows
// beyond a pole are ghost rows: row -1-q is ring q and row R+q is ring R-1-q,
// read at phi + pi with the factor (-1)^k (d^l_{mk}(-t) = (-1)^{m-k} d^l_{mk}(t)).
//
// The binning kernel has already turned each pointing into a stencil record
// (cell (i, j), theta - theta(i-1), the phi fraction) in double precision.
// Forward FP64: one thread per sample in sorted order (samples of one cell are
// adjacent, so the lanes of a warp read the same nodes).  Forward FP32: one CTA
// per work item, the tile's nodes staged in shared memory first.
// Adjoint: one CTA per work item (<= kChunk samples of one tile); the tile's
// nodes (with a 3-node halo) are accumulated in shared memory, each warp
// owning a disjoint set of k so that no two threads update the same word, and
// the tile is flushed to the global adjoint cube with atomic adds.
#include <algorithm>

#include "sl_internal.cuh"

namespace sl {

constexpr int kChunkA = kWorkChunk;

// ------------------------------------------------------------------ forward FP64
// One thread per sample: combined weights w_a w_b per node, read through L1.
template <int P>
__global__ void __launch_bounds__(256) k_interp_f64(const InterpGeom g, const double2 *__restrict__ maps,
                                                    const StencilRec64 *__restrict__ rec,
                                                    const double *__restrict__ psi, const unsigned *__restrict__ perm,
                                                    int64_t n, double *__restrict__ tod) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const unsigned s = perm[t];
        const StencilRec64 r = rec[s];
        const int i = (int)(r.cell >> 16) - 1, j = (int)(r.cell & 0xffffu);
        double wt[P], wp[P];
        weights64<P>(g, i, r.dth, r.fph, wt, wp);
        int roff[P], coff[P], coffg[P];
        const unsigned ghost = stencil_offsets<P>(g, i, j, roff, coff, coffg);
        // node offsets and combined weights (ghost rows read the ring at phi + pi)
        int off[P * P];
        double w[P * P];
#pragma unroll
        for (int a = 0; a < P; ++a)
#pragma unroll
            for (int b = 0; b < P; ++b) {
                off[a * P + b] = roff[a] + (((ghost >> a) & 1u) ? coffg[b] : coff[b]);
                w[a * P + b] = wt[a] * wp[b];
                if (!SL_GUARD(off[a * P + b] >= 0 &&
                                  (int64_t)off[a * P + b] + g.K < (int64_t)g.R * g.nphi * (g.K + 1),
                              0x201u))
                    off[a * P + b] = 0;
            }
        double sp, cp;
        sincos(psi[s], &sp, &cp);
        // k = 0: only Re S_0 enters the TOD
        double acc = 0.0;
#pragma unroll
        for (int q = 0; q < P * P; ++q) acc = fma(w[q], __ldg(maps + off[q]).x, acc);
        // C_k = 2 cos(k psi), S_k = 2 sin(k psi) by the Chebyshev three-term
        // recurrence X_{k+1} = (2 cos psi) X_k - X_{k-1}
        const double c1 = 2.0 * cp;
        double Ck = c1, Sk = 2.0 * sp, Ckm = 2.0, Skm = 0.0;
        for (int k = 1; k <= g.K; ++k) {
            if (ghost) {   // (-1)^k on ghost rows: flip their weights between k-1 and k
#pragma unroll
                for (int a = 0; a < P; ++a)
                    if (ghost & (1u << a))
#pragma unroll
                        for (int b = 0; b < P; ++b) w[a * P + b] = -w[a * P + b];
            }
            double sr = 0.0, si = 0.0;
#pragma unroll
            for (int q = 0; q < P * P; ++q) {
                const double2 v = __ldg(maps + off[q] + k);
                sr = fma(w[q], v.x, sr);
                si = fma(w[q], v.y, si);
            }
            acc = fma(Ck, sr, acc);
            acc = fma(-Sk, si, acc);
            const double cn = fma(c1, Ck, -Ckm), sn = fma(c1, Sk, -Skm);
            Ckm = Ck;
            Skm = Sk;
            Ck = cn;
            Sk = sn;
        }
        tod[s] = acc;
    }
}

// ------------------------------------------------------------------ forward FP32, tile-staged
// One CTA per work item (<= kChunkA sorted samples of one tile).  The tile's
// stencil nodes -- rows tr*4-2 .. tr*4+4 and columns tc*TC-1 .. tc*TC+TC+1,
// every k -- are staged into shared memory with coalesced loads (consecutive
// threads read consecutive k of one node); ghost rows are folded in while
// staging (ring at phi + pi, factor (-1)^k).  Shared layout [k pair][row][col]
// of float4 (F_k, F_k+1), k padded to an even count: the 16 stencil nodes of a
// sample sit at compile-time offsets from its first node, and one k pair is
// one 128-bit load.  Samples are then evaluated from shared memory; the lanes
// of a warp mostly share one cell (broadcast reads).
struct TiledArgs {
    InterpGeom g;
    const float2 *maps;
    const StencilRec32 *rec;
    const unsigned *perm, *start, *chunk_off;
    int ntiles, ncell;
    double *tod;
};

template <int TC, int P>
__global__ void __launch_bounds__(256) k_interp_f32_tiled(const TiledArgs A) {
    constexpr int TW = TC + P - 1, NR = kTileRows + P - 1, NN = NR * TW;   // staged nodes per k pair
    const InterpGeom &g = A.g;
    const int K1 = g.K + 1, KH = (K1 + 1) >> 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4 *node = reinterpret_cast<float4 *>(smem_raw);   // [KH][NR][TW]
    // staging walk: element e = node * KH + kp, advanced by blockDim.x per step
    const int e_step_n = (int)blockDim.x / KH, e_step_k = (int)blockDim.x - e_step_n * KH;
    const int e0_n = (int)threadIdx.x / KH, e0_k = (int)threadIdx.x - e0_n * KH;
    const unsigned nchunks = A.chunk_off[A.ntiles];
    int staged_tile = -1;
    for (unsigned v = blockIdx.x; v < nchunks; v += gridDim.x) {
        const int tile = find_tile(A.chunk_off, A.ntiles, v);
        const unsigned c = v - A.chunk_off[tile];
        const unsigned s_beg = A.start[(int64_t)tile * A.ncell] + c * kChunkA;
        const unsigned s_end = min(A.start[(int64_t)(tile + 1) * A.ncell], s_beg + kChunkA);
        const int tr = tile / g.ntc, tcol = tile - tr * g.ntc;
        const int rowlo = tr * kTileRows - P / 2, collo = tcol * TC - P / 2 + 1;
        if (tile != staged_tile) {
            __syncthreads();
            for (int nd = e0_n, kp = e0_k; nd < NN;) {
                const int r = nd / TW, cc = nd - r * TW;
                const int row = rowlo + r, k = 2 * kp;
                float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
                if (row >= -P / 2 && row <= g.R - 1 + P / 2) {
                    int ring = row, col = collo + cc;
                    bool flip = false;
                    if (row < 0 || row >= g.R) {
                        ring = (row < 0) ? -1 - row : 2 * g.R - 1 - row;
                        col += g.nphi >> 1;
                    }
                    // col in [-1, 1.5 nphi + TC + 2): at most two wraps
                    if (col < 0) col += g.nphi;
                    if (col >= g.nphi) col -= g.nphi;
                    if (col >= g.nphi) col -= g.nphi;
                    flip = ring != row;
                    if (!SL_GUARD(ring >= 0 && ring < g.R && col >= 0 && col < g.nphi, 0x202u)) ring = col = 0;
                    const float2 *src = A.maps + ((int64_t)ring * g.nphi + col) * K1 + k;
                    const float2 v0 = __ldg(src);
                    const float2 v1 = (k + 1 < K1) ? __ldg(src + 1) : make_float2(0.f, 0.f);
                    // ghost rows: (-1)^k, i.e. the odd member of the pair flips
                    val = flip ? make_float4(v0.x, v0.y, -v1.x, -v1.y) : make_float4(v0.x, v0.y, v1.x, v1.y);
                }
                node[kp * NN + nd] = val;
                nd += e_step_n;
                kp += e_step_k;
                if (kp >= KH) { kp -= KH; ++nd; }
            }
            __syncthreads();
            staged_tile = tile;
        }
        for (unsigned t = s_beg + threadIdx.x; t < s_end; t += blockDim.x) {
            const unsigned s = A.perm[t];
            const StencilRec32 r = A.rec[s];
            const int i = (int)(r.cell >> 16) - 1, j = (int)(r.cell & 0xffffu);
            float o[P], wd[P], wt[P], wp[P];
#pragma unroll
            for (int a = 0; a < P; ++a) {
                o[a] = __ldg(g.rowtab32 + (size_t)(i + 1) * 2 * P + a);
                wd[a] = __ldg(g.rowtab32 + (size_t)(i + 1) * 2 * P + P + a);
            }
            lagrange_theta<P>(r.dth, o, wd, wt);
            lagrange_phi<P>(r.fph, wp);
            float w[P * P];
#pragma unroll
            for (int q = 0; q < P * P; ++q) w[q] = wt[q / P] * wp[q % P];
            int nb0 = (i - P / 2 + 1 - rowlo) * TW + (j - P / 2 + 1 - collo);
            if (!SL_GUARD(nb0 >= 0 && nb0 + (P - 1) * TW + (P - 1) < NN, 0x203u)) nb0 = 0;
            const float4 *nb = node + nb0;
            float sz, cz;
            sincosf(r.psr, &sz, &cz);
            // z^k for the pair (k, k+1), starting at (1, z)
            float z0r = 1.f, z0i = 0.f, z1r = cz, z1i = sz;
            const float z2r = cz * cz - sz * sz, z2i = 2.f * cz * sz;
            float acc0 = 0.f, acc1 = 0.f;
            for (int kp = 0; kp < KH; ++kp, nb += NN) {
                float sr0 = 0.f, si0 = 0.f, sr1 = 0.f, si1 = 0.f;
#pragma unroll
                for (int q = 0; q < P * P; ++q) {
                    const float4 v = nb[(q / P) * TW + (q % P)];
                    sr0 = fmaf(w[q], v.x, sr0);
                    si0 = fmaf(w[q], v.y, si0);
                    sr1 = fmaf(w[q], v.z, sr1);
                    si1 = fmaf(w[q], v.w, si1);
                }
                if (kp == 0) acc0 = sr0;
                else acc1 = fmaf(z0r, sr0, fmaf(-z0i, si0, acc1));
                acc1 = fmaf(z1r, sr1, fmaf(-z1i, si1, acc1));   // padding slot holds zeros
                const float n0r = z0r * z2r - z0i * z2i, n0i = z0r * z2i + z0i * z2r;
                const float n1r = z1r * z2r - z1i * z2i, n1i = z1r * z2i + z1i * z2r;
                z0r = n0r; z0i = n0i; z1r = n1r; z1i = n1i;
            }
            A.tod[s] = (double)acc0 + 2.0 * (double)acc1;
        }
    }
}

SL_CHECK_READER(chk_interp)

size_t interp_f32_tiled_smem_tc(const sl_plan *p, int tc) {
    const int KH = (p->K + 2) / 2;
    return (size_t)(kTileRows + p->p - 1) * (tc + p->p - 1) * KH * sizeof(float4);
}

size_t interp_f32_tiled_smem(const sl_plan *p) { return interp_f32_tiled_smem_tc(p, p->geom.tile_cols); }

// ------------------------------------------------------------------ adjoint
// maps_bar_k(node) += y wt_a wp_b sigma_{a,k} eps_k e^{-ik psi},  eps_0 = 1, eps_k = 2.
struct AdjArgs {
    InterpGeom g;
    const double *psi, *y;
    const StencilRec64 *rec;
    const unsigned *perm, *start, *chunk_off;
    int ntiles, ncell;
    double2 *fbar;
};

constexpr int kNB = 64;   // samples staged per batch (32 when kmax + 1 > 64, to fit shared memory)
__host__ __device__ __forceinline__ int kNB_of(int K1) { return K1 > 64 ? kNB / 2 : kNB; }

template <int P>
__global__ void k_interp_adjoint(const AdjArgs A) {
    constexpr int NQ = P * P;               // stencil nodes
    const InterpGeom &g = A.g;
    const int K1 = g.K + 1;
    const int TC = g.tile_cols;
    const int tw = TC + P - 1;              // smem tile columns
    const int th_rows = kTileRows + P - 1;  // smem tile rows
    const int nnode = th_rows * tw;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2 *acc = reinterpret_cast<double2 *>(smem_raw);            // [nnode][K1]
    double2 *PH = acc + (size_t)nnode * K1;                           // [kNB][K1]
    double *W = reinterpret_cast<double *>(PH + (size_t)kNB_of(K1) * K1);    // [kNB][NQ]
    int *LOC = reinterpret_cast<int *>(W + (size_t)kNB_of(K1) * NQ);         // [kNB] node index of the first stencil node

    const unsigned nchunks = A.chunk_off[A.ntiles];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;

    for (int e = threadIdx.x; e < nnode * K1; e += blockDim.x) acc[e] = make_double2(0.0, 0.0);

    for (unsigned v = blockIdx.x; v < nchunks; v += gridDim.x) {
        // tile of this work item: largest t with chunk_off[t] <= v
        int lo = 0, hi = A.ntiles - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (A.chunk_off[mid] <= v) lo = mid; else hi = mid - 1;
        }
        const int tile = lo;
        const unsigned c = v - A.chunk_off[tile];
        const unsigned s_beg = A.start[(int64_t)tile * A.ncell] + c * kChunkA;
        const unsigned s_end = min(A.start[(int64_t)(tile + 1) * A.ncell], s_beg + kChunkA);
        const int tr = tile / g.ntc, tcol = tile % g.ntc;
        const int rowlo = tr * kTileRows - P / 2;   // stencil rows i-P/2+1 .., base row i >= tr*4-1
        const int collo = tcol * TC - P / 2 + 1;
        __syncthreads();
        for (unsigned b0 = s_beg; b0 < s_end; b0 += (unsigned)kNB_of(K1)) {
            const int nb = (int)min((unsigned)kNB_of(K1), s_end - b0);
            // phase A: per-sample weights, node location and phases
            if ((int)threadIdx.x < nb) {
                const unsigned s = A.perm[b0 + threadIdx.x];
                const StencilRec64 r = A.rec[s];
                const int i = (int)(r.cell >> 16) - 1, j = (int)(r.cell & 0xffffu);
                double wt[P], wp[P];
                weights64<P>(g, i, r.dth, r.fph, wt, wp);
                double *ws = W + threadIdx.x * NQ;
#pragma unroll
                for (int ra = 0; ra < P; ++ra)
#pragma unroll
                    for (int cb = 0; cb < P; ++cb) ws[ra * P + cb] = wt[ra] * wp[cb];
                int loc = (i - P / 2 + 1 - rowlo) * tw + (j - P / 2 + 1 - collo);
                if (!SL_GUARD(loc >= 0 && loc + (P - 1) * tw + (P - 1) < nnode, 0x204u)) loc = 0;
                LOC[threadIdx.x] = loc;
                double sp, cp;
                sincos(A.psi[s], &sp, &cp);
                const double y = A.y[s], c2 = 2.0 * cp;
                double ck = 1.0, sk = 0.0, ckm = cp, skm = -sp;
                double2 *Ps = PH + (size_t)threadIdx.x * K1;
                for (int k = 0; k <= g.K; ++k) {
                    const double sc = (k == 0) ? y : 2.0 * y;
                    Ps[k] = make_double2(sc * ck, -sc * sk);     // eps_k y e^{-ik psi}
                    const double cn = fma(c2, ck, -ckm), sn = fma(c2, sk, -skm);
                    ckm = ck;
                    skm = sk;
                    ck = cn;
                    sk = sn;
                }
            }
            __syncthreads();
            // phase B: warp w owns k-pairs w, w + nwarps, ...; a lane handles the
            // entries (node q, k parity) = lane, lane + 32, ... of the 2 P^2.
            // Samples are in cell order, so consecutive samples mostly share
            // their stencil: a lane sums in registers while the cell stays
            // the same and adds to the shared tile when it changes.
            constexpr int NE = (2 * NQ + 31) / 32;
            for (int kp = warp; 2 * kp <= g.K; kp += nwarps) {
                double2 racc[NE];
#pragma unroll
                for (int t = 0; t < NE; ++t) racc[t] = make_double2(0.0, 0.0);
                int cur_loc = nb > 0 ? LOC[0] : 0;
                for (int sidx = 0; sidx <= nb; ++sidx) {
                    const int loc = (sidx < nb) ? LOC[sidx] : -1;
                    if (loc != cur_loc) {       // warp-uniform: flush the previous cell's sums
#pragma unroll
                        for (int t = 0; t < NE; ++t) {
                            const int e = lane + 32 * t;
                            const int q = e % NQ, kk = 2 * kp + e / NQ;
                            if (e < 2 * NQ && kk <= g.K) {
                                double2 &dst = acc[(size_t)(cur_loc + (q / P) * tw + (q % P)) * K1 + kk];
                                double2 c = dst;
                                c.x += racc[t].x;
                                c.y += racc[t].y;
                                dst = c;
                            }
                            racc[t] = make_double2(0.0, 0.0);
                        }
                        // the next cell's stencil may overlap: order this warp's updates
                        __syncwarp(0xffffffffu);
                        cur_loc = loc;
                    }
                    if (sidx == nb) break;
#pragma unroll
                    for (int t = 0; t < NE; ++t) {
                        const int e = lane + 32 * t;
                        const int q = e % NQ, kk = 2 * kp + e / NQ;
                        if (e < 2 * NQ && kk <= g.K) {
                            const double w = W[sidx * NQ + q];
                            const double2 ph = PH[(size_t)sidx * K1 + kk];
                            racc[t].x = fma(w, ph.x, racc[t].x);
                            racc[t].y = fma(w, ph.y, racc[t].y);
                        }
                    }
                }
            }
            __syncthreads();
        }
        // flush the tile (ghost rows fold onto their ring at phi + pi with (-1)^k)
        for (int e = threadIdx.x; e < nnode * K1; e += blockDim.x) {
            const double2 val = acc[e];
            if (val.x == 0.0 && val.y == 0.0) continue;
            acc[e] = make_double2(0.0, 0.0);
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
            if (!SL_GUARD(ring >= 0 && ring < g.R, 0x205u)) continue;
            double2 *o = A.fbar + ((int64_t)ring * g.nphi + col) * K1 + kk;
            atomicAdd(&o->x, sg * val.x);
            atomicAdd(&o->y, sg * val.y);
        }
    }
}

static unsigned grid_for(int64_t n, int bs) {
    int64_t b = (n + bs - 1) / bs;
    const int64_t cap = 152 * 32;
    return (unsigned)(b < cap ? (b > 0 ? b : 1) : cap);
}

sl_status launch_interp(sl_plan *p, const SortBufs &b, int fine, const void *maps, const double *psi, int64_t n,
                        double *tod) {
    int slot;
    if (p->precision == SL_DF64) return launch_interp_df(p, b, fine, maps, psi, n, tod);
    if (p->precision == SL_FP64) {
        void (*kern)(const InterpGeom, const double2 *, const StencilRec64 *, const double *, const unsigned *,
                     int64_t, double *);
        switch (p->p) {
            case 2: kern = k_interp_f64<2>; break;
            case 4: kern = k_interp_f64<4>; break;
            case 6: kern = k_interp_f64<6>; break;
            default: return set_error(SL_ERR_UNSUPPORTED, "interp_order %d", p->p);
        }
        slot = timing_begin(p, "interp_f64");
        kern<<<grid_for(n, 256), 256, 0, p->stream>>>(p->geom, (const double2 *)maps, (const StencilRec64 *)b.rec,
                                                       psi, b.perm, n, tod);
    } else {
        if (!b.chunk_off) return set_error(SL_ERR_ARG, "FP32 interpolation needs the per-tile work list");
        TiledArgs a;
        a.g = p->geom;
        a.maps = (const float2 *)maps;
        a.rec = (const StencilRec32 *)b.rec;
        a.perm = b.perm;
        a.start = b.hist;
        a.chunk_off = b.chunk_off;
        a.ntiles = p->ntiles;
        a.ncell = fine ? kTileRows * p->geom.tile_cols : 1;
        a.tod = tod;
        const size_t sm = interp_f32_tiled_smem(p);
        void (*kern)(const TiledArgs) = nullptr;
#define SL_TILED(TCV, PV) \
    if (p->geom.tile_cols == TCV && p->p == PV) kern = k_interp_f32_tiled<TCV, PV>;
        SL_TILED(32, 4) SL_TILED(16, 4) SL_TILED(8, 4)
        SL_TILED(32, 2) SL_TILED(16, 2) SL_TILED(8, 2)
        SL_TILED(32, 6) SL_TILED(16, 6) SL_TILED(8, 6)
#undef SL_TILED
        if (!kern) return set_error(SL_ERR_UNSUPPORTED, "tile width %d, interp_order %d", p->geom.tile_cols, p->p);
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return cuda_check(e, "k_interp_f32_tiled smem attribute");
        int per_sm = 1, nsm = 152;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, sm);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device);
        if (per_sm < 1) per_sm = 1;
        slot = timing_begin(p, "interp_f32");
        kern<<<(unsigned)(nsm * per_sm), 256, sm, p->stream>>>(a);
    }
    timing_end(p, slot);
    return cuda_check(cudaGetLastError(), "k_interp launch");
}

size_t interp_adjoint_smem_tc(const sl_plan *p, int tc) {
    const int K1 = p->K + 1, P = p->p;
    const int nnode = (kTileRows + P - 1) * (tc + P - 1);
    return (size_t)nnode * K1 * sizeof(double2) + (size_t)kNB_of(K1) * K1 * sizeof(double2) +
           (size_t)kNB_of(K1) * P * P * sizeof(double) + (size_t)kNB_of(K1) * sizeof(int);
}

sl_status launch_interp_adjoint(sl_plan *p, const SortBufs &b, int fine, const double *psi, const double *tod,
                                int64_t n, double2 *fbar) {
    if (p->precision == SL_DF64) return launch_interp_adjoint_df(p, b, fine, psi, tod, fbar);
    AdjArgs a;
    a.g = p->geom;
    a.psi = psi;
    a.y = tod;
    a.rec = (const StencilRec64 *)b.rec;
    a.perm = b.perm;
    a.start = b.hist;
    a.chunk_off = b.chunk_off;
    a.ntiles = p->ntiles;
    a.ncell = fine ? kTileRows * p->geom.tile_cols : 1;
    a.fbar = fbar;
    const int K1 = p->K + 1;
    const size_t sm = interp_adjoint_smem_tc(p, p->geom.tile_cols);
    int nwarps = (K1 + 1) / 2;
    if (nwarps < 2) nwarps = 2;
    if (nwarps > 16) nwarps = 16;
    void (*kern)(const AdjArgs);
    switch (p->p) {
        case 2: kern = k_interp_adjoint<2>; break;
        case 4: kern = k_interp_adjoint<4>; break;
        case 6: kern = k_interp_adjoint<6>; break;
        default: return set_error(SL_ERR_UNSUPPORTED, "interp_order %d", p->p);
    }
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return cuda_check(e, "k_interp_adjoint smem attribute");
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * nwarps, sm);
    if (per_sm < 1) per_sm = 1;
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device);
    int slot = timing_begin(p, "interp_adj");
    kern<<<(unsigned)(nsm * per_sm), 32 * nwarps, sm, p->stream>>>(a);
    timing_end(p, slot);
    (void)n;
    return cuda_check(cudaGetLastError(), "k_interp_adjoint launch");
}

}  // namespace sl
