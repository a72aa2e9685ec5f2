// k_sort.cu -- binning of the pointings before interpolation (the cube is read
// through p x p stencils, Sect. 2.1 interpolation step): a counting sort of
// the samples by grid tile.  A sample's cell is (base row i, base column j) of
// its stencil; tiles group kTileRows x tile_cols cells.
//
//   k_bin:      key[s] = tile(i, j), histogram of keys (warp-aggregated atomics)
//   k_scan:     exclusive prefix sum -> tile start offsets (and cursor copy),
//               plus per-tile chunk offsets used by the adjoint scatter
//   k_scatter:  perm[cursor[key]++] = s  (order within a tile is unspecified)
#include "sl_internal.cuh"

namespace sl {

constexpr int kChunk = 2048;   // adjoint work item: at most this many samples of one tile

__global__ void __launch_bounds__(256) k_bin(const InterpGeom g, const double *__restrict__ theta,
                                             const double *__restrict__ phi, int64_t n,
                                             unsigned *__restrict__ keys, unsigned *__restrict__ hist) {
    const unsigned lane = threadIdx.x & 31;
    for (int64_t s0 = (int64_t)blockIdx.x * blockDim.x; s0 < n; s0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = s0 + threadIdx.x;
        const bool ok = s < n;
        unsigned key = 0xffffffffu;
        if (ok) {
            const int i = locate_row(g, theta[s]);
            double f;
            const int j = locate_col(g, phi[s], f);
            key = tile_key(g, i, j);
            keys[s] = key;
        }
        const unsigned act = __ballot_sync(0xffffffffu, ok);
        if (ok) {
            const unsigned peers = __match_any_sync(act, key);
            const int leader = __ffs(peers) - 1;
            if ((int)lane == leader) atomicAdd(hist + key, (unsigned)__popc(peers));
        }
    }
}

// Single CTA: exclusive scan of hist[0..ntiles) into start (hist, in place,
// with hist[ntiles] = n), cursor = start, chunk_off = prefix of ceil(cnt/kChunk).
__global__ void __launch_bounds__(1024) k_scan(int ntiles, unsigned *__restrict__ hist,
                                               unsigned *__restrict__ cursor,
                                               unsigned *__restrict__ chunk_off) {
    __shared__ unsigned s_tot[32], s_ch[32];
    __shared__ unsigned carry_tot, carry_ch;
    if (threadIdx.x == 0) {
        carry_tot = 0;
        carry_ch = 0;
    }
    __syncthreads();
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < ntiles; base += 1024) {
        const int t = base + threadIdx.x;
        const unsigned c = (t < ntiles) ? hist[t] : 0u;
        const unsigned ch = (c + kChunk - 1) / kChunk;
        unsigned a = c, b = ch;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned ya = __shfl_up_sync(0xffffffffu, a, o);
            const unsigned yb = __shfl_up_sync(0xffffffffu, b, o);
            if ((int)lane >= o) {
                a += ya;
                b += yb;
            }
        }
        if (lane == 31) {
            s_tot[warp] = a;
            s_ch[warp] = b;
        }
        __syncthreads();
        if (warp == 0) {
            unsigned wa = s_tot[lane], wb = s_ch[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned ya = __shfl_up_sync(0xffffffffu, wa, o);
                const unsigned yb = __shfl_up_sync(0xffffffffu, wb, o);
                if ((int)lane >= o) {
                    wa += ya;
                    wb += yb;
                }
            }
            s_tot[lane] = wa;
            s_ch[lane] = wb;
        }
        __syncthreads();
        const unsigned pre_a = (warp ? s_tot[warp - 1] : 0u) + a - c + carry_tot;
        const unsigned pre_b = (warp ? s_ch[warp - 1] : 0u) + b - ch + carry_ch;
        if (t < ntiles) {
            hist[t] = pre_a;
            cursor[t] = pre_a;
            chunk_off[t] = pre_b;
        }
        __syncthreads();
        if (threadIdx.x == 1023) {
            carry_tot = pre_a + c;
            carry_ch = pre_b + ch;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        hist[ntiles] = carry_tot;
        chunk_off[ntiles] = carry_ch;
    }
}

__global__ void __launch_bounds__(256) k_scatter(int64_t n, const unsigned *__restrict__ keys,
                                                 unsigned *__restrict__ cursor, unsigned *__restrict__ perm) {
    const unsigned lane = threadIdx.x & 31;
    for (int64_t s0 = (int64_t)blockIdx.x * blockDim.x; s0 < n; s0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = s0 + threadIdx.x;
        const bool ok = s < n;
        const unsigned key = ok ? keys[s] : 0xffffffffu;
        const unsigned act = __ballot_sync(0xffffffffu, ok);
        if (ok) {
            const unsigned peers = __match_any_sync(act, key);
            const int leader = __ffs(peers) - 1;
            const unsigned rank = __popc(peers & ((1u << lane) - 1u));
            unsigned base = 0;
            if ((int)lane == leader) base = atomicAdd(cursor + key, (unsigned)__popc(peers));
            base = __shfl_sync(peers, base, leader);
            perm[base + rank] = (unsigned)s;
        }
    }
}

static unsigned grid_for(int64_t n, int bs) {
    int64_t b = (n + bs - 1) / bs;
    const int64_t cap = 152 * 16;
    return (unsigned)(b < cap ? (b > 0 ? b : 1) : cap);
}

sl_status launch_sort(sl_plan *p, const double *theta, const double *phi, int64_t n) {
    sl_status st = cuda_check(cudaMemsetAsync(p->d_hist, 0, (p->ntiles + 1) * sizeof(unsigned), p->stream),
                              "memset hist");
    if (st != SL_OK) return st;
    int slot = timing_begin(p, "bin");
    k_bin<<<grid_for(n, 256), 256, 0, p->stream>>>(p->geom, theta, phi, n, p->d_keys, p->d_hist);
    timing_end(p, slot);
    if ((st = cuda_check(cudaGetLastError(), "k_bin launch")) != SL_OK) return st;
    slot = timing_begin(p, "scan");
    k_scan<<<1, 1024, 0, p->stream>>>(p->ntiles, p->d_hist, p->d_cursor, p->d_chunk_off);
    timing_end(p, slot);
    if ((st = cuda_check(cudaGetLastError(), "k_scan launch")) != SL_OK) return st;
    slot = timing_begin(p, "scatter");
    k_scatter<<<grid_for(n, 256), 256, 0, p->stream>>>(n, p->d_keys, p->d_cursor, p->d_perm);
    timing_end(p, slot);
    return cuda_check(cudaGetLastError(), "k_scatter launch");
}

// Same three kernels as launch_sort, into caller-provided scratch (no plan
// scratch, no allocation).  hist must hold ntiles + 1 entries, cursor ntiles,
// chunk_off ntiles + 1, keys and perm n each.
sl_status launch_sort_into(sl_plan *p, const double *theta, const double *phi, int64_t n, unsigned *keys,
                           unsigned *perm, unsigned *hist, unsigned *cursor, unsigned *chunk_off) {
    sl_status st = cuda_check(cudaMemsetAsync(hist, 0, (p->ntiles + 1) * sizeof(unsigned), p->stream),
                              "memset hist");
    if (st != SL_OK) return st;
    k_bin<<<grid_for(n, 256), 256, 0, p->stream>>>(p->geom, theta, phi, n, keys, hist);
    if ((st = cuda_check(cudaGetLastError(), "k_bin launch")) != SL_OK) return st;
    k_scan<<<1, 1024, 0, p->stream>>>(p->ntiles, hist, cursor, chunk_off);
    if ((st = cuda_check(cudaGetLastError(), "k_scan launch")) != SL_OK) return st;
    k_scatter<<<grid_for(n, 256), 256, 0, p->stream>>>(n, keys, cursor, perm);
    return cuda_check(cudaGetLastError(), "k_scatter launch");
}

}  // namespace sl
