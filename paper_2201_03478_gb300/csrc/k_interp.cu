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
#include <climits>

#include "mbar.cuh"
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

// ------------------------------------------------------------------ forward FP32, cell groups
// The path interp_tod takes for FP32 plans.  The fine sort orders each tile's
// samples by cell, so a thread evaluates S samples of ONE cell together (S = 2
// for p <= 4; 1 for p = 6, where two samples' weights would not fit in
// registers): every node value it loads from shared memory feeds S sums, which
// halves the shared-memory traffic per multiply-add -- the bound of the
// one-sample form (k_interp_f32_tiled, kept for the tile-keyed sort of
// interp_tod_noalloc).  The (re, im) sums run as packed two-lane FP32
// multiply-adds (__ffma2_rn), half the issue slots of scalar ones.  The k sum
// is a Horner scheme in z = e^{i psi}, from k = K down to 1:
//   h <- h z + S_k,   c = Re S_0 + 2 Re(z h)   (the last step in FP64).
//
// Warp-specialized, no CTA-wide barrier after the set-up.  Warp 0 stages;
// warps 1-7 evaluate.  The staging warp takes chunks of kCellIPC consecutive
// work items (<= kChunkA sorted samples of one tile) from a global counter and
// cuts them into sub-items of <= kCellSub samples.  All its global -> shared
// traffic is asynchronous (cp.async and one bulk copy), so one latency covers
// a whole tile or sub-item.
//   node buffers (2):   node0[NR][TW] = Re F_0 (k = 0 enters the TOD through
//                       its real part only), node[KP][NR][TW] = float4
//                       (F_{2j+1}, F_{2j+2}), KP = ceil(K/2) (an odd K's unused
//                       slot holds zeros), the tile's four base rows of the row
//                       table and its cells' first sorted positions.  Same tile,
//                       halo and ghost-row rule as the tiled kernel (ghost rows
//                       get their (-1)^k sign in a pass after the copies land);
//                       refilled when the tile changes.
//   record buffers (2): a sub-item's sample indices (one bulk copy), its stencil
//                       records (cp.async gathers through those indices), its
//                       group table (per cell ceil(count / S) groups, prefix
//                       offsets) and a header.
// Handoff by mbarriers: nfull and rfull (32 staging lanes' arrivals plus 32
// arrivals on completion of their cp.async copies), nempty and rempty (7
// evaluating warps); a private barrier paces the bulk copy.  Every wait is
// bounded (mbar.cuh); an expired wait raises the plan's error flag and the warp
// stops (SL_ERR_TIMEOUT at the next sl_plan_sync).
constexpr int kCellSub = 1024;        // samples per record buffer
constexpr int kCellSidx = kCellSub + 8;   // sample-index slots: a 16-byte aligned superset of the sub-item
constexpr int kCellConsumers = 7;     // evaluating warps per CTA (plus one staging warp)
constexpr int kCellIPC = 8;           // work items per chunk taken from the counter

struct CellMeta {
    int nbuf, rowlo, collo, tr;
    unsigned ngroups;                 // 0xffffffff: no more work for this CTA
    unsigned poff;                    // first sample index of the sub-item within its slots
    int det;                          // detector (plan) of the sub-item
};

// Parameters of one launch: one detector (interp_tod) or many (a batch).
struct CellArgs {
    int ndet, kpmax;                  // detectors; node pairs ceil(kmax/2) of the largest kmax
    unsigned *work;                   // work counter (zeroed before the launch)
    int *err;                         // device error flag of the bounded waits
    TiledArgs d[kMaxBatchDets];
};

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes) : "memory");
}
// 4-byte copy; with ok == false nothing is read and the destination is zero-filled
__device__ __forceinline__ void cp_async4(void *dst, const void *src, bool ok) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" :: "r"(smem_u32(dst)), "l"(src), "r"(ok ? 4 : 0)
                 : "memory");
}

// Exact float -> double by integer operations only (normal, subnormal, zero,
// infinity, NaN): the FP64 pipe runs at 1/64 of the FP32 rate, and the
// hardware conversion runs on it.
__device__ __forceinline__ double f2d_exact(float x) {
    const unsigned u = __float_as_uint(x), e = (u >> 23) & 0xffu;
    unsigned m = u & 0x7fffffu;
    unsigned de;
    if (e == 0xffu) {
        de = 0x7ffu;
    } else if (e != 0u) {
        de = e + 896u;
    } else if (m == 0u) {
        de = 0u;
    } else {   // subnormal m 2^-149: the leading one at bit b moves to the implicit bit
        const unsigned b = 31u - (unsigned)__clz(m);
        m = (m << (23u - b)) & 0x7fffffu;
        de = b + 874u;
    }
    return __longlong_as_double((long long)(((unsigned long long)(u & 0x80000000u) << 32) |
                                            ((unsigned long long)de << 52) | ((unsigned long long)m << 29)));
}

template <int TC, int P>
__global__ void __launch_bounds__(256, 2) k_interp_f32_cells(const __grid_constant__ CellArgs C) {
    constexpr int TW = TC + P - 1, NR = kTileRows + P - 1, NN = NR * TW;
    constexpr int NCELL = kTileRows * TC, NQ = P * P, CPL = NCELL / 32, ROWT = kTileRows * 2 * P;
    constexpr int S = (P <= 4) ? 2 : 1;
    constexpr unsigned kEnd = 0xffffffffu;
    const int KPM = C.kpmax;   // node pairs of the largest kmax: the node buffers' stride
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4 *nodeb = reinterpret_cast<float4 *>(smem_raw);                             // [2][KPM * NN]
    StencilRec32 *srecb = reinterpret_cast<StencilRec32 *>(nodeb + 2 * (size_t)KPM * NN);   // [2][kCellSub]
    unsigned *ssidb = reinterpret_cast<unsigned *>(srecb + 2 * kCellSub);            // [2][kCellSidx]
    unsigned *cstb = ssidb + 2 * kCellSidx;                                          // [2][NCELL + 1]
    float *node0b = reinterpret_cast<float *>(cstb + 2 * (NCELL + 1));               // [2][NN]
    float *srowb = node0b + 2 * NN;                                                  // [2][ROWT]
    unsigned *goffb = reinterpret_cast<unsigned *>(srowb + 2 * ROWT);                // [2][NCELL + 1]
    unsigned *cbegb = goffb + 2 * (NCELL + 1);                                       // [2][NCELL]
    unsigned *cendb = cbegb + 2 * NCELL;                                             // [2][NCELL]
    __shared__ CellMeta meta[2];
    __shared__ unsigned gctr[2];                   // groups of each record buffer claimed so far
    __shared__ unsigned dcum[kMaxBatchDets + 1];   // first global work item of each detector
    __shared__ __align__(8) unsigned long long bars[9];
    const uint32_t rfull = smem_u32(&bars[0]), rempty = smem_u32(&bars[2]);
    const uint32_t nfull = smem_u32(&bars[4]), nempty = smem_u32(&bars[6]), pbar = smem_u32(&bars[8]);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(rfull + 8 * b, 64);
            mbar_init(rempty + 8 * b, kCellConsumers);
            mbar_init(nfull + 8 * b, 64);
            mbar_init(nempty + 8 * b, kCellConsumers);
        }
        mbar_init(pbar, 1);
    }
    __syncthreads();

    if (warp == 0) {
        // ------------------------------------------------ staging warp
        {   // work items of the detectors, one after another
            const unsigned nd = lane < C.ndet ? C.d[lane].chunk_off[C.d[lane].ntiles] : 0u;
            unsigned x = nd;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane < C.ndet) dcum[lane + 1] = x;
            if (lane == 0) dcum[0] = 0u;
            __syncwarp();
        }
        const unsigned nchunks = dcum[C.ndet];
        bool ok = true;
        int tile = -1, tile_det = -1, det = -1, tcur = 0;
        unsigned nfill = 0, u = 0, pphase = 0;
        int nb = 0, rowlo = 0, collo = 0, tr = 0;
        for (;;) {
            unsigned v0 = 0;
            if (lane == 0) v0 = atomicAdd(C.work, 1u) * kCellIPC;
            v0 = __shfl_sync(0xffffffffu, v0, 0);
            if (v0 >= nchunks || !ok) break;
            const unsigned v_end = min(nchunks, v0 + kCellIPC);
            det = -1;
            for (unsigned v = v0; v < v_end && ok; ++v) {
                int dv = 0;
                while (dv + 1 < C.ndet && dcum[dv + 1] <= v) ++dv;
                const TiledArgs &A = C.d[dv];
                const InterpGeom &g = A.g;
                const int K = g.K, K1 = K + 1, KP = (K + 1) >> 1, KE = KP + 1;
                const unsigned vl = v - dcum[dv];
                if (dv != det) {
                    det = dv;
                    tcur = find_tile(A.chunk_off, A.ntiles, vl);
                }
                while (tcur + 1 < A.ntiles && A.chunk_off[tcur + 1] <= vl) ++tcur;
                const unsigned c = vl - A.chunk_off[tcur];
                if (tcur != tile || det != tile_det) {
                    nb = nfill & 1;
                    if (nfill >= 2) ok = __all_sync(0xffffffffu, mbar_wait(nempty + 8 * nb, ((nfill - 2) >> 1) & 1));
                    if (!ok) break;
                    tr = tcur / g.ntc;
                    const int tcol = tcur - tr * g.ntc;
                    rowlo = tr * kTileRows - P / 2;
                    collo = tcol * TC - P / 2 + 1;
                    float4 *node = nodeb + (size_t)nb * KPM * NN;
                    float *node0 = node0b + nb * NN;
                    // first sorted position of each cell of the tile (and the tile's end): a
                    // cp.async group of its own, issued first, so that the group tables below
                    // wait for these copies only and not for the node copies behind them
                    // (earlier record gathers still pending join this group)
                    cp_async_commit();
                    const int64_t cb = (int64_t)tcur * NCELL;
                    for (int t = lane; t <= NCELL; t += 32) cp_async4(cstb + nb * (NCELL + 1) + t, A.start + cb + t, true);
                    cp_async_commit();
                    // node (column cc, k slot w) of row r for idx = cc * KE + w, stepped by 32
                    // lanes with counters instead of a division per element
                    const int q32 = 32 / KE, r32 = 32 - q32 * KE;
                    const int cc0 = lane / KE, w0 = lane - cc0 * KE;
                    bool polar = false;
                    for (int r = 0; r < NR; ++r) {
                        const int row = rowlo + r;
                        const bool inr = row >= -P / 2 && row <= g.R - 1 + P / 2;
                        const bool ghost = row < 0 || row >= g.R;
                        polar |= inr && ghost;
                        const int ring = !inr ? 0 : (row < 0 ? -1 - row : (row >= g.R ? 2 * g.R - 1 - row : row));
                        const int cshift = ghost ? (g.nphi >> 1) : 0;
                        const float2 *rsrc = A.maps + (int64_t)ring * g.nphi * K1;
                        int cc = cc0, w = w0;
                        for (int idx = lane; idx < TW * KE; idx += 32) {
                            int col = collo + cc + cshift;
                            if (col < 0) col += g.nphi;
                            if (col >= g.nphi) col -= g.nphi;
                            if (col >= g.nphi) col -= g.nphi;
                            if (!SL_GUARD(col >= 0 && col < g.nphi, 0x205u)) col = 0;
                            const float2 *src = rsrc + (int64_t)col * K1;
                            const int nd = r * TW + cc;
                            if (w == 0) {
                                cp_async4(node0 + nd, src, inr);
                            } else {
                                const int k = 2 * w - 1;
                                float2 *d2 = reinterpret_cast<float2 *>(node + (w - 1) * NN + nd);
                                cp_async8(d2, src + k, inr);
                                cp_async8(d2 + 1, src + (k + 1 <= K ? k + 1 : k), inr && k + 1 <= K);
                            }
                            w += r32;
                            cc += q32;
                            if (w >= KE) {
                                w -= KE;
                                ++cc;
                            }
                        }
                    }
                    // the row table of the tile's base rows (i + 1 = tr * 4 .. tr * 4 + 3, at most R)
                    for (int t = lane; t < ROWT; t += 32) {
                        const int ri = tr * kTileRows + t / (2 * P);
                        cp_async4(srowb + nb * ROWT + t, g.rowtab32 + (size_t)(ri <= g.R ? ri : 0) * 2 * P + t % (2 * P),
                                  ri <= g.R);
                    }
                    cp_async_commit();
                    if (__any_sync(0xffffffffu, polar)) {
                        cp_async_wait_all();   // the ghost rows are fixed up in place once they land
                        __syncwarp();
                        // ghost rows: (-1)^k, i.e. the odd member (k = 2j + 1) of every pair flips
                        for (int r = 0; r < NR; ++r) {
                            const int row = rowlo + r;
                            if (!(row < 0 || row >= g.R)) continue;
                            for (int idx = lane; idx < TW * KP; idx += 32) {
                                const int jj = idx / TW, cc = idx - jj * TW;
                                float4 &e = node[jj * NN + r * TW + cc];
                                e.x = -e.x;
                                e.y = -e.y;
                            }
                        }
                        __syncwarp();
                    } else {
                        // the group tables below read the cell starts: this lane's copies of them
                        // (all but the most recent group), then the warp's; the node copies land on
                        // their own and are tracked by nfull
                        cp_async_wait<1>();
                        __syncwarp();
                    }
                    mbar_arrive_cp_async(nfull + 8 * nb);
                    mbar_arrive(nfull + 8 * nb);
                    tile = tcur;
                    tile_det = det;
                    ++nfill;
                }
                const unsigned *cst = cstb + nb * (NCELL + 1);
                const unsigned s_beg = cst[0] + c * kChunkA;
                const unsigned s_end = min(cst[NCELL], s_beg + kChunkA);
                for (unsigned sb = s_beg; sb < s_end && ok; sb += kCellSub, ++u) {
                    const unsigned se = min(s_end, sb + kCellSub);
                    const int rb = u & 1;
                    if (u >= 2) ok = __all_sync(0xffffffffu, mbar_wait(rempty + 8 * rb, ((u - 2) >> 1) & 1));
                    if (!ok) break;
                    // sample indices: one bulk copy of a 16-byte aligned superset
                    const unsigned sb4 = sb & ~3u, se4 = (se + 3u) & ~3u, poff = sb - sb4;
                    unsigned *ssid = ssidb + rb * kCellSidx;
                    if (lane == 0) {
                        mbar_arrive_expect_tx(pbar, (se4 - sb4) * 4u);
                        bulk_copy_g2s(ssid, A.perm + sb4, (se4 - sb4) * 4u, pbar);
                    }
                    // group table: per cell ceil(count / S) groups, exclusive prefix over the cells
                    unsigned cnt[CPL], gbv[CPL], gev[CPL], lsum = 0;
#pragma unroll
                    for (int q = 0; q < CPL; ++q) {
                        const int cc = lane * CPL + q;
                        unsigned gb = max(cst[cc], sb), ge = min(cst[cc + 1], se);
                        if (ge < gb) ge = gb;
                        gbv[q] = gb - sb;
                        gev[q] = ge - sb;
                        cnt[q] = (ge - gb + S - 1) / S;
                        lsum += cnt[q];
                    }
                    unsigned x = lsum;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
                        if (lane >= o) x += y;
                    }
                    unsigned pre = x - lsum;
                    unsigned *goff = goffb + rb * (NCELL + 1);
#pragma unroll
                    for (int q = 0; q < CPL; ++q) {
                        const int cc = lane * CPL + q;
                        goff[cc] = pre;
                        cbegb[rb * NCELL + cc] = gbv[q];
                        cendb[rb * NCELL + cc] = gev[q];
                        pre += cnt[q];
                    }
                    if (lane == 31) goff[NCELL] = x;
                    const unsigned total = __shfl_sync(0xffffffffu, x, 31);
                    if (lane == 0) {
                        meta[rb] = CellMeta{nb, rowlo, collo, tr, total, poff, det};
                        gctr[rb] = 0u;
                    }
                    // the records, gathered through the indices
                    ok = __all_sync(0xffffffffu, mbar_wait(pbar, pphase));
                    pphase ^= 1u;
                    if (!ok) break;
                    StencilRec32 *srec = srecb + rb * kCellSub;
                    for (unsigned t = lane; t < se - sb; t += 32) cp_async16(srec + t, A.rec + ssid[poff + t]);
                    mbar_arrive_cp_async(rfull + 8 * rb);
                    mbar_arrive(rfull + 8 * rb);
                }
            }
        }
        if (ok) {   // end marker
            const int rb = u & 1;
            if (u >= 2) ok = __all_sync(0xffffffffu, mbar_wait(rempty + 8 * rb, ((u - 2) >> 1) & 1));
            if (ok) {
                if (lane == 0) meta[rb].ngroups = kEnd;
                mbar_arrive_cp_async(rfull + 8 * rb);
                mbar_arrive(rfull + 8 * rb);
            }
        }
        if (!ok) {
            cp_async_wait_all();
            mbar_wait(pbar, pphase, 10000000ull);   // a bulk copy that may still be in flight
            if (lane == 0) atomicExch(C.err, 1);
        }
        return;
    }

    // ---------------------------------------------------- evaluating warps
    int cur_nb = -1;
    unsigned nfill = 0;
    bool ok = true;
    for (unsigned u = 0;; ++u) {
        const int rb = u & 1;
        ok = __all_sync(0xffffffffu, mbar_wait(rfull + 8 * rb, (u >> 1) & 1));
        if (!ok) break;
        const unsigned ngroups = meta[rb].ngroups;
        if (ngroups == kEnd) break;
        const int mnb = meta[rb].nbuf;
        if (mnb != cur_nb) {   // the next node fill (fills alternate between the two buffers)
            __syncwarp();
            if (cur_nb >= 0 && lane == 0) mbar_arrive(nempty + 8 * cur_nb);
            ok = __all_sync(0xffffffffu, mbar_wait(nfull + 8 * mnb, (nfill >> 1) & 1));
            if (!ok) break;
            cur_nb = mnb;
            ++nfill;
        }
        const int m_rowlo = meta[rb].rowlo, m_collo = meta[rb].collo, m_tr = meta[rb].tr;
        const TiledArgs &A = C.d[meta[rb].det];
        const int KP = (A.g.K + 1) >> 1;
        const float4 *node = nodeb + (size_t)cur_nb * KPM * NN;
        const float *node0 = node0b + cur_nb * NN;
        const float *srow = srowb + cur_nb * ROWT;
        const StencilRec32 *srec = srecb + rb * kCellSub;
        const unsigned *ssid = ssidb + rb * kCellSidx + meta[rb].poff;
        const unsigned *goff = goffb + rb * (NCELL + 1);
        const unsigned *cbeg = cbegb + rb * NCELL, *cend = cendb + rb * NCELL;
        // groups are claimed 32 at a time (one per lane) from the buffer's counter, so
        // the warps finish a sub-item together and its buffer is released early
        for (;;) {
            unsigned gclaim = 0;
            if (lane == 0) gclaim = atomicAdd(&gctr[rb], 32u);
            gclaim = __shfl_sync(0xffffffffu, gclaim, 0);
            if (gclaim >= ngroups) break;
            const unsigned gi = gclaim + lane;
            if (gi >= ngroups) continue;
            // the group's cell: the last cell whose first group is <= gi (never an empty one)
            int lo = 0, hi = NCELL - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (goff[mid] <= gi) lo = mid; else hi = mid - 1;
            }
            const unsigned t0 = cbeg[lo] + S * (gi - goff[lo]);   // sub-item-local sorted position
            const unsigned tl = cend[lo];
            unsigned sidx[S], rcell[S];
            float rdth[S], rfph[S], rpsr[S];
#pragma unroll
            for (int q = 0; q < S; ++q) {
                const unsigned t = (t0 + q < tl) ? t0 + q : t0;
                sidx[q] = ssid[t];
                const StencilRec32 rr = srec[t];
                rdth[q] = rr.dth;
                rfph[q] = rr.fph;
                rpsr[q] = rr.psr;
                rcell[q] = rr.cell;
            }
            const int i = (int)(rcell[0] >> 16) - 1, j = (int)(rcell[0] & 0xffffu);
            int li = i + 1 - m_tr * kTileRows;
            if (!SL_GUARD(li >= 0 && li < kTileRows, 0x207u)) li = 0;
            float o[P], wd[P];
#pragma unroll
            for (int a = 0; a < P; ++a) {
                o[a] = srow[li * 2 * P + a];
                wd[a] = srow[li * 2 * P + P + a];
            }
            float2 W[S][NQ];
            float zc[S], zs[S];
#pragma unroll
            for (int q = 0; q < S; ++q) {
                float wt[P], wp[P];
                lagrange_theta<P>(rdth[q], o, wd, wt);
                lagrange_phi<P>(rfph[q], wp);
#pragma unroll
                for (int e = 0; e < NQ; ++e) {
                    const float w = wt[e / P] * wp[e % P];
                    W[q][e] = make_float2(w, w);
                }
                sincosf(rpsr[q], &zs[q], &zc[q]);
            }
            int nb0 = (i - P / 2 + 1 - m_rowlo) * TW + (j - P / 2 + 1 - m_collo);
            if (!SL_GUARD(nb0 >= 0 && nb0 + (P - 1) * TW + (P - 1) < NN && (S == 1 || rcell[S - 1] == rcell[0]),
                          0x206u))
                nb0 = 0;
            // k = 0: Re S_0
            float a0[S];
#pragma unroll
            for (int q = 0; q < S; ++q) a0[q] = 0.f;
#pragma unroll
            for (int e = 0; e < NQ; ++e) {
                const float f = node0[nb0 + (e / P) * TW + (e % P)];
#pragma unroll
                for (int q = 0; q < S; ++q) a0[q] = fmaf(W[q][e].x, f, a0[q]);
            }
            // k = K .. 1, two at a time, Horner in z
            float hr[S], hi_[S];
#pragma unroll
            for (int q = 0; q < S; ++q) hr[q] = hi_[q] = 0.f;
            const float4 *nbp = node + (size_t)(KP - 1) * NN + nb0;
            for (int jj = KP - 1; jj >= 0; --jj, nbp -= NN) {
                float2 sa[S], sb2[S];
#pragma unroll
                for (int q = 0; q < S; ++q) sa[q] = sb2[q] = make_float2(0.f, 0.f);
#pragma unroll
                for (int e = 0; e < NQ; ++e) {
                    const float4 vv = nbp[(e / P) * TW + (e % P)];
                    const float2 lo2 = make_float2(vv.x, vv.y), hi2 = make_float2(vv.z, vv.w);
#pragma unroll
                    for (int q = 0; q < S; ++q) {
                        sa[q] = __ffma2_rn(W[q][e], lo2, sa[q]);
                        sb2[q] = __ffma2_rn(W[q][e], hi2, sb2[q]);
                    }
                }
#pragma unroll
                for (int q = 0; q < S; ++q) {
                    // h <- (h z + S_{2jj+2}) z + S_{2jj+1}
                    const float nr = fmaf(hr[q], zc[q], fmaf(-hi_[q], zs[q], sb2[q].x));
                    const float ni = fmaf(hr[q], zs[q], fmaf(hi_[q], zc[q], sb2[q].y));
                    hr[q] = fmaf(nr, zc[q], fmaf(-ni, zs[q], sa[q].x));
                    hi_[q] = fmaf(nr, zs[q], fmaf(ni, zc[q], sa[q].y));
                }
            }
#pragma unroll
            for (int q = 0; q < S; ++q)
                if (q == 0 || t0 + q < tl) {
                    const float pz = fmaf(zc[q], hr[q], -zs[q] * hi_[q]);   // Re(z h)
                    A.tod[sidx[q]] = fma(2.0, f2d_exact(pz), f2d_exact(a0[q]));
                }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(rempty + 8 * rb);
    }
    if (!ok && lane == 0) atomicExch(C.err, 1);
}

size_t interp_f32_cells_smem(int K, int P, int tc) {
    const int KP = (K + 1) / 2, NN = (kTileRows + P - 1) * (tc + P - 1), ncell = kTileRows * tc;
    return 2 * ((size_t)KP * NN * sizeof(float4) + (size_t)kCellSub * sizeof(StencilRec32) +
                (size_t)kCellSidx * sizeof(unsigned) + (size_t)(ncell + 1) * sizeof(unsigned) +
                (size_t)NN * sizeof(float) + (size_t)kTileRows * 2 * P * sizeof(float)) +
           (size_t)(2 * (ncell + 1) + 4 * ncell) * sizeof(unsigned);
}

size_t interp_f32_cells_smem_tc(const sl_plan *p, int tc) { return interp_f32_cells_smem(p->K, p->p, tc); }

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

TiledArgs fine_tiled_args(const sl_plan *p, const SortBufs &b, const void *maps, double *tod) {
    TiledArgs a;
    a.g = p->geom;
    a.maps = (const float2 *)maps;
    a.rec = (const StencilRec32 *)b.rec;
    a.perm = b.perm;
    a.start = b.hist;
    a.chunk_off = b.chunk_off;
    a.ntiles = p->ntiles;
    a.ncell = kTileRows * p->geom.tile_cols;
    a.tod = tod;
    return a;
}

// One persistent launch of k_interp_f32_cells over nd detectors' work items
// (their sorts done; all with tile width tc and interpolation order P; kmax
// at most kmax_max).  work and err: a counter (zeroed here) and the error flag.
sl_status launch_interp_f32_cells(cudaStream_t stream, int device, const TiledArgs *dets, int nd, int tc, int P,
                                  int kmax_max, unsigned *work, int *err) {
    if (nd < 1 || nd > kMaxBatchDets) return set_error(SL_ERR_ARG, "FP32 interpolation: %d detectors (1..%d)", nd, kMaxBatchDets);
    CellArgs C;
    C.ndet = nd;
    C.kpmax = (kmax_max + 1) / 2;
    C.work = work;
    C.err = err;
    for (int d = 0; d < nd; ++d) C.d[d] = dets[d];
    const size_t sm = interp_f32_cells_smem(kmax_max, P, tc);
    void (*kern)(const CellArgs) = nullptr;
#define SL_CELLS(TCV, PV) \
    if (tc == TCV && P == PV) kern = k_interp_f32_cells<TCV, PV>;
    SL_CELLS(32, 4) SL_CELLS(16, 4) SL_CELLS(8, 4)
    SL_CELLS(32, 2) SL_CELLS(16, 2) SL_CELLS(8, 2)
    SL_CELLS(32, 6) SL_CELLS(16, 6) SL_CELLS(8, 6)
#undef SL_CELLS
    if (!kern) return set_error(SL_ERR_UNSUPPORTED, "tile width %d, interp_order %d", tc, P);
    cudaError_t e = allow_dyn_smem(kern, sm);
    if (e != cudaSuccess) return cuda_check(e, "k_interp_f32_cells smem attribute");
    if ((e = cudaMemsetAsync(work, 0, sizeof(unsigned), stream)) != cudaSuccess) return cuda_check(e, "work counter");
    int per_sm = 1, nsm = 152;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, sm);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    if (per_sm < 1) per_sm = 1;
    kern<<<(unsigned)(nsm * per_sm), 256, sm, stream>>>(C);
    return cuda_check(cudaGetLastError(), "k_interp_f32_cells launch");
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
        if (fine) {   // cell-sorted samples: S samples of a cell per thread
            if (!p->d_err) return set_error(SL_ERR_ARG, "FP32 interpolation needs the plan's error flag");
            slot = timing_begin(p, "interp_f32");
            sl_status st = launch_interp_f32_cells(p->stream, p->device, &a, 1, p->geom.tile_cols, p->p, p->K,
                                                   reinterpret_cast<unsigned *>(p->d_err + 1), p->d_err);
            timing_end(p, slot);
            return st;
        }
        // tile-keyed sort (interp_tod_noalloc): one sample per thread
        const size_t sm = interp_f32_tiled_smem(p);
        void (*kern)(const TiledArgs) = nullptr;
#define SL_TILED(TCV, PV) \
    if (p->geom.tile_cols == TCV && p->p == PV) kern = k_interp_f32_tiled<TCV, PV>;
        SL_TILED(32, 4) SL_TILED(16, 4) SL_TILED(8, 4)
        SL_TILED(32, 2) SL_TILED(16, 2) SL_TILED(8, 2)
        SL_TILED(32, 6) SL_TILED(16, 6) SL_TILED(8, 6)
#undef SL_TILED
        if (!kern) return set_error(SL_ERR_UNSUPPORTED, "tile width %d, interp_order %d", p->geom.tile_cols, p->p);
        cudaError_t e = allow_dyn_smem(kern, sm);
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
    cudaError_t e = allow_dyn_smem(kern, sm);
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
