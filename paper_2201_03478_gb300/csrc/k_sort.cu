// k_sort.cu -- binning of the pointings before interpolation (the cube is read
// through p x p stencils, Sect. 2.1 interpolation step): a counting sort of
// the samples by grid cell, plus a per-sample stencil record.
//
// A sample's cell is (base row i, base column j) of its stencil.  Cells are
// grouped into tiles of kTileRows x tile_cols; the sort key is either the tile
// (coarse) or the cell in tile-major order (fine), so that both orders list
// each tile's samples contiguously.  With fine keys the samples of one cell
// are adjacent and neighbouring threads read the same cube nodes.
//
//   k_bin:        pointing -> (i, j) in double; key; record {theta - theta(i-1),
//                 phi fraction, [reduced psi], cell}; key histogram
//   k_scan_local / k_scan1 / k_scan_add:  exclusive prefix sum of the histogram
//                 -> first position of every key (and a cursor copy)
//   k_scatter_agg: perm[cursor[key]++] = s, the cursor atomics aggregated per
//                 chunk of samples in shared memory (order within a key unspecified)
//   k_tile_chunks: work items of at most kChunk samples per tile (adjoint)
#include "sl_internal.cuh"

namespace sl {

constexpr int kChunk = kWorkChunk;
constexpr int kScanBlock = 4096;    // keys per CTA of k_scan_local (1024 threads x 4)

// Runs of equal keys among the warp's lanes (the active lanes are a prefix of
// the warp: lanes 0 .. nact - 1): the run of this lane starts at lane *head and
// holds *cnt lanes.  One atomic per run replaces one per lane; lanes of a scan
// that share a cell are almost always adjacent, and a key that recurs after
// another key just starts another run.  (Grouping all equal keys with
// __match_any_sync costs a multi-pass instruction per lane group, which bound
// the binning and the scatter.)
__device__ __forceinline__ void key_run(unsigned key, bool ok, unsigned lane, int *head, unsigned *cnt) {
    const unsigned prev = __shfl_up_sync(0xffffffffu, key, 1);
    const unsigned act = __ballot_sync(0xffffffffu, ok);
    const unsigned heads = __ballot_sync(0xffffffffu, ok && (lane == 0 || key != prev));
    const unsigned upto = (lane == 31) ? 0xffffffffu : ((2u << lane) - 1u);   // lanes 0 .. lane
    *head = 31 - __clz(heads & upto);
    const unsigned after = heads & ~upto;
    const int next = after ? __ffs(after) - 1 : 32;
    const int nact = __popc(act);
    *cnt = (unsigned)(min(next, nact) - *head);
}

// Samples [*beg, *end) of this CTA in k_bin: one contiguous slice
// of the TOD per CTA (a multiple of blockDim.x long), walked blockDim.x at a
// time.  A scan repeats the same circle on the sky every few thousand samples,
// so a grid-stride walk -- every resident CTA on one contiguous stretch of the
// TOD -- sends hundreds of warps to the same cells' counters at once, and
// their atomics serialise; slices put the CTAs on different stretches.
__device__ __forceinline__ void cta_slice(int64_t n, int64_t *beg, int64_t *end) {
    const int64_t per = ((n + gridDim.x - 1) / gridDim.x + blockDim.x - 1) / blockDim.x * blockDim.x;
    *beg = min(n, (int64_t)blockIdx.x * per);
    *end = min(n, *beg + per);
}

template <bool REC64>
__global__ void __launch_bounds__(256) k_bin(const InterpGeom g, int fine, const double *__restrict__ theta,
                                             const double *__restrict__ phi, const double *__restrict__ psi,
                                             int64_t n, unsigned *__restrict__ keys, void *__restrict__ rec,
                                             unsigned *__restrict__ hist) {
    const unsigned lane = threadIdx.x & 31;
    int64_t sbeg, send;
    cta_slice(n, &sbeg, &send);
    for (int64_t s0 = sbeg; s0 < send; s0 += blockDim.x) {
        const int64_t s = s0 + threadIdx.x;
        const bool ok = s < send;
        unsigned key = 0xffffffffu;
        if (ok) {
            const double th = theta[s];
            const int i = locate_row(g, th);
            unsigned long long fr;
            int sh;
            const int j = locate_col_fix(g, phi[s], fr, sh);
            // tile_cols is 8, 16 or 32 and i + 1 >= 0: shifts and masks instead of divisions
            const int tlg = __ffs(g.tile_cols) - 1;
            const int tr = (int)((unsigned)(i + 1) / kTileRows), li = (i + 1) - tr * kTileRows;
            const int tc = j >> tlg, lj = j & (g.tile_cols - 1);
            const unsigned tile = (unsigned)tr * (unsigned)g.ntc + (unsigned)tc;
            key = fine ? tile * (unsigned)(kTileRows * g.tile_cols) + (unsigned)(li * g.tile_cols + lj) : tile;
            [[maybe_unused]] const unsigned nkeys = (unsigned)(g.ntr * g.ntc) * (fine ? (unsigned)(kTileRows * g.tile_cols) : 1u);
            if (!SL_GUARD(i >= -1 && i < g.R && j >= 0 && j < g.nphi && key < nkeys, 0x101u)) key = 0;
            keys[s] = key;
            // theta - theta(i0), i0 = i - p/2 + 1 the first stencil row (index i0 + half = i + 1),
            // in 2^-60 fixed point (exact for theta >= 2^-8)
            long long tf = 0;
            const bool tfix = to_fix<60>(th, tf);
            const long long dfix = tf - __ldg(g.ring_fix + i + 1);
            const unsigned cell = ((unsigned)(i + 1) << 16) | (unsigned)j;
            if (REC64) {
                const double dth = tfix ? fix_to_d<60>(dfix) : th - __ldg(g.ring_ext + i + 1);
                reinterpret_cast<StencilRec64 *>(rec)[s] = StencilRec64{dth, frac_bits_d(fr, sh), cell, 0u};
            } else {
                const float dth = tfix ? fix_to_f<60>(dfix) : d2f_bits(th - __ldg(g.ring_ext + i + 1));
                // psi reduced to [-pi, pi] in 2^-59 fixed point; |psi| >= 8 (and NaN) in FP64
                const double ps = psi[s];
                long long pf;
                float psr;
                if (to_fix<59>(ps, pf)) {
                    constexpr long long kPi59 = 1811004864519280711ll, k2Pi59 = 3622009729038561421ll;
                    if (pf > kPi59) pf -= k2Pi59;
                    else if (pf < -kPi59) pf += k2Pi59;
                    psr = fix_to_f<59>(pf);
                } else {
                    psr = d2f_bits(ps - 6.283185307179586 * rint(ps * 0.15915494309189535));
                }
                reinterpret_cast<StencilRec32 *>(rec)[s] = StencilRec32{dth, frac_bits_f(fr, sh), psr, cell};
            }
        }
        int head;
        unsigned cnt;
        key_run(key, ok, lane, &head, &cnt);
        if (ok && (int)lane == head) atomicAdd(hist + key, cnt);
    }
}

// Block-wide exclusive scan of 1024 values (one per thread); returns the total.
__device__ __forceinline__ unsigned block_exclusive_scan(unsigned v, unsigned &excl) {
    __shared__ unsigned s_w[32];
    __shared__ unsigned s_tot;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned a = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, a, o);
        if ((int)lane >= o) a += y;
    }
    if (lane == 31) s_w[warp] = a;
    __syncthreads();
    if (warp == 0) {
        unsigned w = s_w[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, w, o);
            if ((int)lane >= o) w += y;
        }
        s_w[lane] = w;
        if (lane == 31) s_tot = w;
    }
    __syncthreads();
    excl = (warp ? s_w[warp - 1] : 0u) + a - v;
    const unsigned tot = s_tot;
    __syncthreads();
    return tot;
}

// Per CTA: exclusive scan of data[b*4096 .. +4096) in place, block total to bsum[b].
__global__ void __launch_bounds__(1024) k_scan_local(int64_t n, unsigned *__restrict__ data,
                                                      unsigned *__restrict__ bsum) {
    const int64_t base = (int64_t)blockIdx.x * kScanBlock + 4 * threadIdx.x;
    unsigned v[4], t = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        v[q] = (base + q < n) ? data[base + q] : 0u;
        t += v[q];
    }
    unsigned ex;
    const unsigned tot = block_exclusive_scan(t, ex);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (base + q < n) data[base + q] = ex;
        ex += v[q];
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// Single CTA: exclusive scan of data[0..n) in place; data[n] = total.
__global__ void __launch_bounds__(1024) k_scan1(int n, unsigned *__restrict__ data) {
    unsigned carry = 0;
    for (int base = 0; base < n; base += 1024) {
        const int t = base + threadIdx.x;
        const unsigned v = (t < n) ? data[t] : 0u;
        unsigned ex;
        const unsigned tot = block_exclusive_scan(v, ex);
        if (t < n) data[t] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) data[n] = carry;
}

__global__ void k_scan_add(int64_t n, unsigned *__restrict__ data, const unsigned *__restrict__ bsum,
                           unsigned *__restrict__ cursor, unsigned total_slot_from_bsum) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned v = data[i] + bsum[i / kScanBlock];
        data[i] = v;
        cursor[i] = v;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) data[n] = bsum[total_slot_from_bsum];
}

// The scatter with its atomics aggregated per chunk of kAggChunk samples: a
// shared-memory hash table gives every sample of the chunk its rank among the
// chunk's samples of the same key (a shared atomic); then one global atomic per
// distinct key reserves the key's range, these atomics issued eight at a time
// and independent of each other, so their round trips overlap; last, each
// sample goes to its range start plus its rank.  Along a scan a 4096-sample
// chunk holds about two visits of every cell of a circle; a per-lane scatter
// (one returning atomic per run of equal keys in a warp) waited for one
// round trip per warp and 32 samples.
constexpr int kAggThreads = 256, kAggPer = 16, kAggChunk = kAggThreads * kAggPer;
constexpr int kAggLog = 13, kAggSlots = 1 << kAggLog;   // > 2 x the distinct keys of a chunk
static_assert(kAggSlots >= kAggChunk, "the hash table must hold every distinct key of a chunk");
constexpr unsigned kNoKey = 0xffffffffu;

__global__ void __launch_bounds__(kAggThreads) k_scatter_agg(int64_t n, int64_t nkeys, const unsigned *__restrict__ keys,
                                                             unsigned *__restrict__ cursor,
                                                             unsigned *__restrict__ perm) {
    extern __shared__ __align__(16) unsigned agg_smem[];
    unsigned *hkey = agg_smem, *hval = agg_smem + kAggSlots;   // key per slot; count, then range start
    const int64_t per = (n + (int64_t)gridDim.x * kAggChunk - 1) / ((int64_t)gridDim.x * kAggChunk) * kAggChunk;
    const int64_t sbeg = min(n, (int64_t)blockIdx.x * per), send = min(n, sbeg + per);
    for (int64_t c0 = sbeg; c0 < send; c0 += kAggChunk) {
        for (int i = threadIdx.x; i < kAggSlots / 4; i += kAggThreads) {
            reinterpret_cast<uint4 *>(hkey)[i] = make_uint4(kNoKey, kNoKey, kNoKey, kNoKey);
            reinterpret_cast<uint4 *>(hval)[i] = make_uint4(0u, 0u, 0u, 0u);
        }
        __syncthreads();
        unsigned slot[kAggPer], rank[kAggPer];
#pragma unroll
        for (int j = 0; j < kAggPer; ++j) {
            const int64_t s = c0 + (int64_t)j * kAggThreads + threadIdx.x;
            slot[j] = kAggSlots;
            rank[j] = 0u;
            if (s < send) {
                unsigned key = keys[s];
                if (!SL_GUARD(key < nkeys, 0x102u)) key = 0;
                unsigned h = (key * 2654435761u) >> (32 - kAggLog);
                // linear probing; the table holds more slots than the chunk has samples,
                // so a free or matching slot is always found within kAggSlots probes
                for (int probe = 0; probe < kAggSlots; ++probe) {
                    const unsigned prev = atomicCAS(&hkey[h], kNoKey, key);
                    if (prev == kNoKey || prev == key) break;
                    h = (h + 1u) & (kAggSlots - 1);
                }
                slot[j] = h;
                rank[j] = atomicAdd(&hval[h], 1u);
            }
        }
        __syncthreads();
        for (int i0 = threadIdx.x; i0 < kAggSlots; i0 += 8 * kAggThreads) {
            unsigned got[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int i = i0 + q * kAggThreads;
                const unsigned k = hkey[i];
                got[q] = (k != kNoKey) ? atomicAdd(cursor + k, hval[i]) : 0u;
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int i = i0 + q * kAggThreads;
                if (hkey[i] != kNoKey) hval[i] = got[q];
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kAggPer; ++j) {
            if (slot[j] >= kAggSlots) continue;
            const int64_t s = c0 + (int64_t)j * kAggThreads + threadIdx.x;
            const unsigned pos = hval[slot[j]] + rank[j];
            if (SL_GUARD(pos < n, 0x103u)) perm[pos] = (unsigned)s;
        }
        __syncthreads();   // the table is cleared for the next chunk
    }
}

// chunk_off[t] = ceil(#samples of tile t / kChunk); scanned by k_scan1 afterwards.
__global__ void k_tile_chunks(int ntiles, int ncell, const unsigned *__restrict__ start,
                              unsigned *__restrict__ chunk_off) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    const unsigned c = start[(int64_t)(t + 1) * ncell] - start[(int64_t)t * ncell];
    chunk_off[t] = (c + kChunk - 1) / kChunk;
}

SL_CHECK_READER(chk_sort)

static unsigned grid_for(int64_t n, int bs) {
    int64_t b = (n + bs - 1) / bs;
    const int64_t cap = 152 * 16;
    return (unsigned)(b < cap ? (b > 0 ? b : 1) : cap);
}

int64_t sort_nkeys(const sl_plan *p, int fine) {
    return fine ? (int64_t)p->ntiles * kTileRows * p->geom.tile_cols : (int64_t)p->ntiles;
}

int64_t sort_nbsum(int64_t nkeys) { return (nkeys + kScanBlock - 1) / kScanBlock; }

sl_status launch_sort_into(sl_plan *p, const SortBufs &b, const double *theta, const double *phi,
                           const double *psi, int64_t n, int fine, int rec64, int with_chunks) {
    const int64_t nkeys = sort_nkeys(p, fine), nb = sort_nbsum(nkeys);
    const int ncell = fine ? kTileRows * p->geom.tile_cols : 1;
    sl_status st = cuda_check(cudaMemsetAsync(b.hist, 0, (nkeys + 1) * sizeof(unsigned), p->stream), "memset hist");
    if (st != SL_OK) return st;
    int slot = timing_begin(p, "bin");
    if (rec64)
        k_bin<true><<<grid_for(n, 256), 256, 0, p->stream>>>(p->geom, fine, theta, phi, psi, n, b.keys, b.rec, b.hist);
    else
        k_bin<false><<<grid_for(n, 256), 256, 0, p->stream>>>(p->geom, fine, theta, phi, psi, n, b.keys, b.rec, b.hist);
    timing_end(p, slot);
    if ((st = cuda_check(cudaGetLastError(), "k_bin launch")) != SL_OK) return st;
    slot = timing_begin(p, "scan");
    k_scan_local<<<(unsigned)nb, 1024, 0, p->stream>>>(nkeys, b.hist, b.bsum);
    k_scan1<<<1, 1024, 0, p->stream>>>((int)nb, b.bsum);
    k_scan_add<<<(unsigned)std::min<int64_t>((nkeys + 255) / 256, 152 * 16), 256, 0, p->stream>>>(
        nkeys, b.hist, b.bsum, b.cursor, (unsigned)nb);
    timing_end(p, slot);
    if ((st = cuda_check(cudaGetLastError(), "k_scan launch")) != SL_OK) return st;
    slot = timing_begin(p, "scatter");
    {
        const size_t sm = 2 * (size_t)kAggSlots * sizeof(unsigned);
        if ((st = cuda_check(allow_dyn_smem(k_scatter_agg, sm), "k_scatter_agg smem attribute")) != SL_OK) return st;
        const int64_t nchunk = (n + kAggChunk - 1) / kAggChunk;
        const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(nchunk, 152 * 3 * 4));
        k_scatter_agg<<<grid, kAggThreads, sm, p->stream>>>(n, nkeys, b.keys, b.cursor, b.perm);
    }
    timing_end(p, slot);
    if ((st = cuda_check(cudaGetLastError(), "k_scatter_agg launch")) != SL_OK) return st;
    if (with_chunks) {
        k_tile_chunks<<<(p->ntiles + 255) / 256, 256, 0, p->stream>>>(p->ntiles, ncell, b.hist, b.chunk_off);
        k_scan1<<<1, 1024, 0, p->stream>>>(p->ntiles, b.chunk_off);
        st = cuda_check(cudaGetLastError(), "k_tile_chunks launch");
    }
    return st;
}

}  // namespace sl
