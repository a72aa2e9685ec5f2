// k_psigrid.cu -- step 2 of the two-step algorithm as the paper states it
// (Sect. 2.1): a Fourier transform over the beam order turns the cube
// F_k(theta_r, phi_j) into c(theta_r, phi_j, psi_n) on a uniform psi grid,
//
//   c(r, j, n) = Re F_0 + 2 sum_{k=1}^{K} Re(e^{ik psi_n} F_k(r, j)),  psi_n = 2 pi n / npsi
//
// (the conjugate-pair sum of Eq. c_m at the grid angles), and the TOD is
// interpolated from that real cube in all three angles.  The paper leaves the
// scheme open; here: p-point Lagrange in theta (actual ring colatitudes) and
// phi (uniform, periodic) as on the exact-phase path, times p-point Lagrange
// on the periodic psi grid.  A ghost row past a pole holds (-1)^k F_k(ring,
// phi + pi), which is c(ring, phi + pi, psi + pi): column + nphi/2 and psi
// index + npsi/2 (npsi even).
//
// k_psi_cube: one CTA per 64 consecutive (ring, phi) nodes; their F_k and the
//   phase table [k][n] = (w_k cos(2 pi k n / npsi), -w_k sin(...)), w_0 = 1,
//   w_k = 2, sit in shared memory; one thread per output value (n fastest, so
//   the stores are coalesced).  Output layout [R][nphi][npsi].
// k_interp_psi: one thread per sample in cell-sorted order (the plan's sort),
//   p^3 reads of the real cube per sample instead of p^2 (K + 1) complex ones.
// k_interp_psi_tiled (FP32 plans): one CTA per work item of a sort tile; the
//   tile's stencil nodes (all npsi values, ghost rows already shifted by pi in
//   phi and psi) are staged in shared memory with coalesced loads, then each
//   sample reads its p^3 values from there.
#include <algorithm>

#include "sl_internal.cuh"

namespace sl {

constexpr int kPsiNodes = 64;    // (ring, phi) nodes per CTA of k_psi_cube

template <typename T> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };

template <typename T>
__global__ void __launch_bounds__(256) k_psi_cube(const typename Vec2<T>::type *__restrict__ maps,
                                                  const typename Vec2<T>::type *__restrict__ tab, int K1, int npsi,
                                                  int64_t nnode, T *__restrict__ out) {
    using T2 = typename Vec2<T>::type;
    extern __shared__ __align__(16) unsigned char psm[];
    T2 *s_tab = reinterpret_cast<T2 *>(psm);                 // [K1][npsi]
    T2 *s_f = s_tab + (size_t)K1 * npsi;                     // [kPsiNodes][K1]
    const int64_t node0 = (int64_t)blockIdx.x * kPsiNodes;
    const int nn = (int)min((int64_t)kPsiNodes, nnode - node0);
    for (int i = threadIdx.x; i < K1 * npsi; i += blockDim.x) s_tab[i] = tab[i];
    const T2 *src = maps + node0 * K1;
    for (int i = threadIdx.x; i < nn * K1; i += blockDim.x) s_f[i] = src[i];
    __syncthreads();
    T *dst = out + node0 * npsi;
    for (int o = threadIdx.x; o < nn * npsi; o += blockDim.x) {
        const int v = o / npsi, n = o - v * npsi;
        const T2 *f = s_f + v * K1;
        T acc = T(0);
        for (int k = 0; k < K1; ++k) {
            const T2 w = s_tab[k * npsi + n], x = f[k];
            acc = fma(w.x, x.x, acc);
            acc = fma(w.y, x.y, acc);
        }
        dst[o] = acc;
    }
}

// One thread per sample (sorted).  T: cube element type; the sum is taken in T
// (FP64 plans: double; FP32 plans: float, as on their exact-phase path).
template <int P, typename T>
__global__ void __launch_bounds__(256) k_interp_psi(const InterpGeom g, int npsi, const T *__restrict__ cube,
                                                    const StencilRec64 *__restrict__ rec,
                                                    const double *__restrict__ psi, const unsigned *__restrict__ perm,
                                                    int64_t n, double *__restrict__ tod) {
    // node strides of the psi cube: npsi reals per (ring, phi) node
    InterpGeom gq = g;
    gq.K = npsi - 1;
    const double vscale = (double)npsi / (2.0 * 3.14159265358979323846);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const unsigned s = perm[t];
        const StencilRec64 r = rec[s];
        const int i = (int)(r.cell >> 16) - 1, j = (int)(r.cell & 0xffffu);
        double wt[P], wp[P];
        weights64<P>(g, i, r.dth, r.fph, wt, wp);
        int roff[P], coff[P], coffg[P];
        const unsigned ghost = stencil_offsets<P>(gq, i, j, roff, coff, coffg);
        // psi: periodic uniform grid
        double v = psi[s] * vscale;
        v -= (double)npsi * floor(v / (double)npsi);
        int n0 = (int)floor(v);
        if (n0 >= npsi) n0 = npsi - 1;
        if (n0 < 0) n0 = 0;
        double wq[P];
        lagrange_phi<P, double>(v - (double)n0, wq);
        int q[P], qg[P];
#pragma unroll
        for (int c = 0; c < P; ++c) {
            int a = n0 - P / 2 + 1 + c;
            a = a < 0 ? a + npsi : (a >= npsi ? a - npsi : a);
            q[c] = a;
            int b = a + npsi / 2;
            qg[c] = b >= npsi ? b - npsi : b;
        }
        T acc = T(0);
#pragma unroll
        for (int a = 0; a < P; ++a) {
            const bool gh = (ghost >> a) & 1u;
            T ra = T(0);
#pragma unroll
            for (int b = 0; b < P; ++b) {
                int no = roff[a] + (gh ? coffg[b] : coff[b]);
                if (!SL_GUARD(no >= 0 && (int64_t)no + npsi <= (int64_t)g.R * g.nphi * npsi, 0x401u)) no = 0;
                const T *node = cube + no;
                T rb = T(0);
#pragma unroll
                for (int c = 0; c < P; ++c) rb = fma((T)wq[c], __ldg(node + (gh ? qg[c] : q[c])), rb);
                ra = fma((T)wp[b], rb, ra);
            }
            acc = fma((T)wt[a], ra, acc);
        }
        tod[s] = (double)acc;
    }
}

struct PsiTiledArgs {
    InterpGeom g;
    int npsi;
    const float *cube;
    const StencilRec32 *rec;
    const unsigned *perm, *start, *chunk_off;
    int ntiles, ncell;
    double *tod;
};

template <int TC, int P>
__global__ void __launch_bounds__(256) k_interp_psi_tiled(const PsiTiledArgs A) {
    constexpr int TW = TC + P - 1, NR = kTileRows + P - 1, NN = NR * TW;
    const InterpGeom &g = A.g;
    const int npsi = A.npsi;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *node = reinterpret_cast<float *>(smem_raw);   // [NN][npsi]
    const float vscale = (float)npsi / 6.28318530717958647692f;
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
            for (int e = threadIdx.x; e < NN * npsi; e += blockDim.x) {
                const int nd = e / npsi, n = e - nd * npsi;
                const int r = nd / TW, cc = nd - r * TW;
                const int row = rowlo + r;
                float val = 0.f;
                if (row >= -P / 2 && row <= g.R - 1 + P / 2) {
                    int ring = row, col = collo + cc, q = n;
                    if (row < 0 || row >= g.R) {   // ghost row: ring at phi + pi, psi + pi
                        ring = (row < 0) ? -1 - row : 2 * g.R - 1 - row;
                        col += g.nphi >> 1;
                        q += npsi >> 1;
                        if (q >= npsi) q -= npsi;
                    }
                    if (col < 0) col += g.nphi;
                    if (col >= g.nphi) col -= g.nphi;
                    if (col >= g.nphi) col -= g.nphi;
                    val = __ldg(A.cube + ((int64_t)ring * g.nphi + col) * npsi + q);
                }
                node[e] = val;
            }
            __syncthreads();
            staged_tile = tile;
        }
        for (unsigned t = s_beg + threadIdx.x; t < s_end; t += blockDim.x) {
            const unsigned s = A.perm[t];
            const StencilRec32 r = A.rec[s];
            const int i = (int)(r.cell >> 16) - 1, j = (int)(r.cell & 0xffffu);
            float o[P], wd[P], wt[P], wp[P], wq[P];
#pragma unroll
            for (int a = 0; a < P; ++a) {
                o[a] = __ldg(g.rowtab32 + (size_t)(i + 1) * 2 * P + a);
                wd[a] = __ldg(g.rowtab32 + (size_t)(i + 1) * 2 * P + P + a);
            }
            lagrange_theta<P>(r.dth, o, wd, wt);
            lagrange_phi<P>(r.fph, wp);
            // psi (reduced to [-pi, pi) by the binning) on the periodic grid
            float vq = r.psr * vscale;
            if (vq < 0.f) vq += (float)npsi;
            int n0 = (int)floorf(vq);
            if (n0 >= npsi) n0 = npsi - 1;
            if (n0 < 0) n0 = 0;
            lagrange_phi<P>(vq - (float)n0, wq);
            int q[P];
#pragma unroll
            for (int cq = 0; cq < P; ++cq) {
                int a = n0 - P / 2 + 1 + cq;
                q[cq] = a < 0 ? a + npsi : (a >= npsi ? a - npsi : a);
            }
            int nb0 = (i - P / 2 + 1 - rowlo) * TW + (j - P / 2 + 1 - collo);
            if (!SL_GUARD(nb0 >= 0 && nb0 + (P - 1) * TW + (P - 1) < NN, 0x402u)) nb0 = 0;
            const float *nb = node + nb0 * npsi;
            float acc = 0.f;
#pragma unroll
            for (int a = 0; a < P; ++a) {
                float ra = 0.f;
#pragma unroll
                for (int b = 0; b < P; ++b) {
                    const float *nd = nb + (a * TW + b) * npsi;
                    float rb = 0.f;
#pragma unroll
                    for (int cq = 0; cq < P; ++cq) rb = fmaf(wq[cq], nd[q[cq]], rb);
                    ra = fmaf(wp[b], rb, ra);
                }
                acc = fmaf(wt[a], ra, acc);
            }
            A.tod[s] = (double)acc;
        }
    }
}

size_t interp_psi_tiled_smem(const sl_plan *p, int npsi) {
    return (size_t)(kTileRows + p->p - 1) * (p->geom.tile_cols + p->p - 1) * npsi * sizeof(float);
}

sl_status launch_interp_psi_tiled(sl_plan *p, const SortBufs &b, const void *cube, int npsi, int64_t n, double *tod) {
    (void)n;
    PsiTiledArgs a;
    a.g = p->geom;
    a.npsi = npsi;
    a.cube = (const float *)cube;
    a.rec = (const StencilRec32 *)b.rec;
    a.perm = b.perm;
    a.start = b.hist;
    a.chunk_off = b.chunk_off;
    a.ntiles = p->ntiles;
    a.ncell = kTileRows * p->geom.tile_cols;
    a.tod = tod;
    const size_t sm = interp_psi_tiled_smem(p, npsi);
    void (*kern)(const PsiTiledArgs) = nullptr;
#define SL_PT(TCV, PV) \
    if (p->geom.tile_cols == TCV && p->p == PV) kern = k_interp_psi_tiled<TCV, PV>;
    SL_PT(32, 4) SL_PT(16, 4) SL_PT(8, 4)
    SL_PT(32, 2) SL_PT(16, 2) SL_PT(8, 2)
    SL_PT(32, 6) SL_PT(16, 6) SL_PT(8, 6)
#undef SL_PT
    if (!kern) return set_error(SL_ERR_UNSUPPORTED, "tile width %d, interp_order %d", p->geom.tile_cols, p->p);
    cudaError_t e = allow_dyn_smem(kern, sm);
    if (e != cudaSuccess) return cuda_check(e, "k_interp_psi_tiled smem attribute");
    int per_sm = 1, nsm = 152;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, sm);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device);
    if (per_sm < 1) per_sm = 1;
    const int slot = timing_begin(p, "interp_psi_f32");
    kern<<<(unsigned)(nsm * per_sm), 256, sm, p->stream>>>(a);
    timing_end(p, slot);
    return cuda_check(cudaGetLastError(), "k_interp_psi_tiled launch");
}

template <typename T>
static size_t psi_cube_smem(int K1, int npsi) {
    return ((size_t)K1 * npsi + (size_t)kPsiNodes * K1) * sizeof(typename Vec2<T>::type);
}

size_t psi_cube_smem_bytes(const sl_plan *p, int npsi) {
    return plan_wide(p->precision) ? psi_cube_smem<double>(p->K + 1, npsi) : psi_cube_smem<float>(p->K + 1, npsi);
}

sl_status launch_psi_cube(sl_plan *p, const void *maps, int npsi, const void *tab, void *out) {
    const int K1 = p->K + 1;
    const int64_t nnode = (int64_t)p->R * p->nphi;
    const unsigned nb = (unsigned)((nnode + kPsiNodes - 1) / kPsiNodes);
    int slot;
    if (plan_wide(p->precision)) {
        const size_t sm = psi_cube_smem<double>(K1, npsi);
        cudaError_t e = allow_dyn_smem(k_psi_cube<double>, sm);
        if (e != cudaSuccess) return cuda_check(e, "k_psi_cube smem attribute");
        slot = timing_begin(p, "psi_cube_f64");
        k_psi_cube<double><<<nb, 256, sm, p->stream>>>((const double2 *)maps, (const double2 *)tab, K1, npsi, nnode,
                                                       (double *)out);
    } else {
        const size_t sm = psi_cube_smem<float>(K1, npsi);
        cudaError_t e = allow_dyn_smem(k_psi_cube<float>, sm);
        if (e != cudaSuccess) return cuda_check(e, "k_psi_cube smem attribute");
        slot = timing_begin(p, "psi_cube_f32");
        k_psi_cube<float><<<nb, 256, sm, p->stream>>>((const float2 *)maps, (const float2 *)tab, K1, npsi, nnode,
                                                      (float *)out);
    }
    timing_end(p, slot);
    return cuda_check(cudaGetLastError(), "k_psi_cube launch");
}

sl_status launch_interp_psi(sl_plan *p, const SortBufs &b, const void *cube, int npsi, const double *psi, int64_t n,
                            double *tod) {
    const unsigned nb = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)152 * 64);
    const bool wide = plan_wide(p->precision);
    int slot = timing_begin(p, wide ? "interp_psi_f64" : "interp_psi_f32");
#define SL_PSI(PV)                                                                                                 \
    if (p->p == PV) {                                                                                             \
        if (wide)                                                                                                  \
            k_interp_psi<PV, double><<<nb, 256, 0, p->stream>>>(p->geom, npsi, (const double *)cube,               \
                                                                (const StencilRec64 *)b.rec, psi, b.perm, n, tod); \
        else                                                                                                       \
            k_interp_psi<PV, float><<<nb, 256, 0, p->stream>>>(p->geom, npsi, (const float *)cube,                 \
                                                               (const StencilRec64 *)b.rec, psi, b.perm, n, tod);  \
    }
    SL_PSI(2) SL_PSI(4) SL_PSI(6)
#undef SL_PSI
    timing_end(p, slot);
    return cuda_check(cudaGetLastError(), "k_interp_psi launch");
}

SL_CHECK_READER(chk_psigrid)

}  // namespace sl
