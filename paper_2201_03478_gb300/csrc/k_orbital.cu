// k_orbital.cu -- the orbital dipole and quadrupole seen through the full 4pi
// beam (Sect. 3.3, Eqs. dipole and dipole_fast), with the paper's acceleration:
// the rotation into the beam frame at every s-th sample of a pointing period,
// a cubic spline in between, and the remainder of each period exact.
//
//   D~ = T0 [ S . beta' + q beta'^T S2 beta' ],   beta' = R^T beta,
//   R = Rz(phi) Ry(theta) Rz(psi)  (the beam-to-sky rotation of Sect. 2.1),
//
// with S = (S_x, S_y, S_z) and S2 the symmetric matrix of S_xx ... S_yz: the
// moments int v B dOmega of the temperature beam in its own frame.  Only the
// l <= 2 beam coefficients enter them (closed forms in k_orb_moments).
//
// Kernels (all FP64):
//   k_orb_moments  one thread: the nine moments from b_lk, l <= 2
//   k_orb_nodes    one thread per spline node: Eq. dipole_fast at that sample
//   k_orb_spline   one warp per pointing period: second derivatives of the
//                  natural cubic spline through the period's nodes
//   k_orb_eval     one thread per sample: the spline between nodes, Eq.
//                  dipole_fast after the last node (or everywhere when s = 1)
//
// The spline system M_{j-1} + 4 M_j + M_{j+1} = 6 (y_{j+1} - 2 y_j + y_{j-1}) / s^2
// (M_0 = M_{n-1} = 0) is solved by the tridiagonal elimination
//   dp_j = (rhs_j - dp_{j-1}) c_j,  M_j = dp_j - c_j M_{j+1},  c_j = 1 / (4 - c_{j-1}),
// whose pivots c_j reach their limit 2 - sqrt(3) (to the last bit) within
// kOrbPivots rows.  Both sweeps are first-order recurrences with a factor of
// magnitude c_j <= 0.268, so a run of rows started from zero differs from the
// true values by that factor's powers times the true value before the run: a
// warp stages 2048 rows in shared memory, gives each lane 64 consecutive rows,
// runs them from zero (lane 0 from the true carry), and adds the carry of the
// lane before it over the first kOrbFix rows (0.268^45 < 1e-25: the rest is
// below rounding).
//
// Between nodes the spline is w0 y_j + w1 y_{j+1} + w2 M_j + w3 M_{j+1} with
// weights of r = t - j s only (B = r/s, A = 1 - B, w2 = (A^3 - A) s^2/6,
// w3 = (B^3 - B) s^2/6), tabulated on the host: four FP64 operations a sample.
#include <cmath>

#include "sl_internal.cuh"

namespace sl {

constexpr int kOrbEvalPerThread = 8;   // samples per thread of k_orb_eval
constexpr int kOrbRun = 64;            // rows per lane and sweep round of k_orb_spline
constexpr int kOrbPivots = 40;         // pivots tabulated; the last one is the limit
constexpr int kOrbFix = 45;            // rows that take the carry of the lane before

// Eq. dipole_fast at one sample.  beta' = Rz(-psi) Ry(-theta) Rz(-phi) beta.
__device__ __forceinline__ double orb_value(const double *__restrict__ S, double T0, double q, double th,
                                            double ph, double ps, const double *__restrict__ b) {
    double st, ct, sp, cp, ss, cs;
    sincos(th, &st, &ct);
    sincos(ph, &sp, &cp);
    sincos(ps, &ss, &cs);
    const double u = cp * b[0] + sp * b[1];      // Rz(-phi)
    const double v = -sp * b[0] + cp * b[1];
    const double x1 = ct * u - st * b[2];        // Ry(-theta)
    const double z = st * u + ct * b[2];
    const double x = cs * x1 + ss * v;           // Rz(-psi)
    const double y = -ss * x1 + cs * v;
    const double lin = S[0] * x + S[1] * y + S[2] * z;
    const double quad = S[3] * x * x + S[4] * y * y + S[5] * z * z +
                        2.0 * (S[6] * x * y + S[7] * x * z + S[8] * y * z);
    return T0 * (lin + q * quad);
}

// The nine moments of the temperature beam (component 0 of [ncomp][K+1][L+1]).
// Writing each v in spherical harmonics (Condon-Shortley phase) and using
// b_{l,-m} = (-1)^m conj(b_lm):  z = sqrt(4pi/3) Y10, x + iy = -sqrt(8pi/3) Y11,
// 1 = sqrt(4pi) Y00, z^2 = sqrt(4pi)/3 Y00 + (4/3) sqrt(pi/5) Y20,
// (x + iy)^2 = sqrt(32pi/15) Y22, (x + iy) z = -sqrt(8pi/15) Y21.
__global__ void k_orb_moments(const double2 *__restrict__ beam, int L, int K, double *__restrict__ S) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    auto b = [&](int l, int k) -> double2 {
        return (l <= L && k <= K && k <= l) ? beam[(int64_t)k * (L + 1) + l] : make_double2(0.0, 0.0);
    };
    const double pi = 3.14159265358979323846;
    const double b00 = b(0, 0).x, b10 = b(1, 0).x, b20 = b(2, 0).x;
    const double2 b11 = b(1, 1), b21 = b(2, 1), b22 = b(2, 2);
    const double mono = sqrt(4.0 * pi) / 3.0 * b00;
    const double c22 = sqrt(32.0 * pi / 15.0), c21 = sqrt(8.0 * pi / 15.0), c20 = sqrt(pi / 5.0);
    S[0] = -2.0 * sqrt(2.0 * pi / 3.0) * b11.x;
    S[1] = 2.0 * sqrt(2.0 * pi / 3.0) * b11.y;
    S[2] = sqrt(4.0 * pi / 3.0) * b10;
    S[3] = mono - 2.0 / 3.0 * c20 * b20 + 0.5 * c22 * b22.x;
    S[4] = mono - 2.0 / 3.0 * c20 * b20 - 0.5 * c22 * b22.x;
    S[5] = mono + 4.0 / 3.0 * c20 * b20;
    S[6] = -0.5 * c22 * b22.y;
    S[7] = -c21 * b21.x;
    S[8] = c21 * b21.y;
}

struct OrbArgs {
    const double *theta, *phi, *psi;
    const int64_t *start;     // [nper + 1] first sample of each period
    const int64_t *noff;      // [nper + 1] first node of each period
    const double *beta;       // [nper][3]
    const double *S;          // [9]
    const double *piv;        // [kOrbPivots] c_j (c_0 = 0); c_j = piv[kOrbPivots - 1] beyond
    const double4_32a *w;     // [s + 1] spline weights (w0, w1, w2, w3) of r = 0 .. s
    double T0, q;
    int64_t n, nper, nnodes;
    int s;
    double *y, *M2;           // [nnodes] node values and spline second derivatives
    double *tod;
    int accumulate;
};

// largest p in [lo, hi) with v[p] <= x, given v[lo] <= x < v[hi]
__device__ __forceinline__ int64_t orb_find(const int64_t *__restrict__ v, int64_t lo, int64_t hi, int64_t x) {
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (v[mid] <= x) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(256) k_orb_nodes(const OrbArgs a) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < a.nnodes;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = orb_find(a.noff, 0, a.nper, g);
        const int64_t i = a.start[p] + (int64_t)a.s * (g - a.noff[p]);
        a.y[g] = orb_value(a.S, a.T0, a.q, a.theta[i], a.phi[i], a.psi[i], a.beta + 3 * p);
    }
}

constexpr int kOrbWarps = 1;                      // periods (warps) per CTA of k_orb_spline (33 KB of static shared memory each)
constexpr int kOrbRound = 32 * kOrbRun;           // rows per sweep round
constexpr int kOrbPad = kOrbRound + kOrbRound / kOrbRun;

// shared-memory slot of round row q: one pad slot per lane run, so that the 32
// lanes (rows 64 l + i) fall on distinct bank pairs
__device__ __forceinline__ int orb_pad(int q) { return q + (q >> 6); }

// One warp per period: the two sweeps of the elimination in rounds of
// kOrbRound rows staged in shared memory (coalesced loads and stores; each lane
// runs its 64 rows from shared memory; see the header).
__global__ void __launch_bounds__(32 * kOrbWarps) k_orb_spline(const OrbArgs a) {
    __shared__ double s_piv[kOrbPivots];
    __shared__ double s_y[kOrbWarps][kOrbRound + 2];
    __shared__ double s_d[kOrbWarps][kOrbPad];
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    for (int j = threadIdx.x; j < kOrbPivots; j += blockDim.x) s_piv[j] = a.piv[j];
    __syncthreads();
    const int64_t p = (int64_t)blockIdx.x * kOrbWarps + wq;
    if (p >= a.nper) return;
    const int64_t g0 = a.noff[p], M = a.noff[p + 1] - g0;
    const double *__restrict__ y = a.y + g0;
    double *__restrict__ m2 = a.M2 + g0;
    double *sy = s_y[wq], *sd = s_d[wq];
    if (M < 3) {
        for (int64_t j = lane; j < M; j += 32) m2[j] = 0.0;
        return;
    }
    if (lane == 0) {
        m2[0] = 0.0;
        m2[M - 1] = 0.0;
    }
    auto piv = [&](int64_t j) { return s_piv[j < kOrbPivots ? j : kOrbPivots - 1]; };
    const double r6 = 6.0 / ((double)a.s * (double)a.s);
    // forward sweep over rows 1 .. M-2: dp_j = (rhs_j - dp_{j-1}) c_j, dp_0 = 0
    double carry = 0.0;
    for (int64_t base = 1; base <= M - 2; base += kOrbRound) {
        const int rows = (int)min((int64_t)kOrbRound, M - 1 - base);
        for (int k = lane; k < rows + 2; k += 32) sy[k] = y[base - 1 + k];
        __syncwarp();
        for (int k = lane; k < rows; k += 32) sd[orb_pad(k)] = r6 * (sy[k + 2] - 2.0 * sy[k + 1] + sy[k]);
        __syncwarp();
        const int lo = lane * kOrbRun, hi = min(lo + kOrbRun, rows);
        double d = lane == 0 ? carry : 0.0;
        for (int q = lo; q < hi; ++q) {
            d = (sd[orb_pad(q)] - d) * piv(base + q);
            sd[orb_pad(q)] = d;
        }
        const double before = __shfl_up_sync(0xffffffffu, d, 1);
        if (lane > 0 && lo < hi) {
            double corr = before;
            for (int q = lo; q < min(hi, lo + kOrbFix); ++q) {
                corr *= -piv(base + q);
                sd[orb_pad(q)] += corr;
            }
        }
        // the next round starts after lane 31's rows (its carry term there is
        // below 0.268^64 of the value; with fewer rows the period has ended)
        carry = __shfl_sync(0xffffffffu, d, 31);
        __syncwarp();
        for (int k = lane; k < rows; k += 32) m2[base + k] = sd[orb_pad(k)];
        __syncwarp();
    }
    // backward sweep: M_j = dp_j - c_j M_{j+1}, M_{M-1} = 0; round row q is j = top - q
    carry = 0.0;
    for (int64_t top = M - 2; top >= 1; top -= kOrbRound) {
        const int rows = (int)min((int64_t)kOrbRound, top);
        for (int k = lane; k < rows; k += 32) sd[orb_pad(k)] = m2[top - k];
        __syncwarp();
        const int lo = lane * kOrbRun, hi = min(lo + kOrbRun, rows);
        double m = lane == 0 ? carry : 0.0;
        for (int q = lo; q < hi; ++q) {
            m = sd[orb_pad(q)] - piv(top - q) * m;
            sd[orb_pad(q)] = m;
        }
        const double above = __shfl_up_sync(0xffffffffu, m, 1);
        if (lane > 0 && lo < hi) {
            double corr = above;
            for (int q = lo; q < min(hi, lo + kOrbFix); ++q) {
                corr *= -piv(top - q);
                sd[orb_pad(q)] += corr;
            }
        }
        carry = __shfl_sync(0xffffffffu, m, 31);
        __syncwarp();
        for (int k = lane; k < rows; k += 32) m2[top - k] = sd[orb_pad(k)];
        __syncwarp();
    }
}

__global__ void __launch_bounds__(256) k_orb_eval(const OrbArgs a) {
    __shared__ int64_t s_p[2];
    const int64_t c0 = (int64_t)blockIdx.x * blockDim.x * kOrbEvalPerThread;
    const int64_t c1 = min(a.n, c0 + (int64_t)blockDim.x * kOrbEvalPerThread);
    if (threadIdx.x == 0) {
        s_p[0] = orb_find(a.start, 0, a.nper, c0);
        s_p[1] = orb_find(a.start, 0, a.nper, c1 - 1);
    }
    __syncthreads();
    const int64_t p0 = s_p[0], p1 = s_p[1];
    const unsigned su = (unsigned)a.s;
#pragma unroll 2
    for (int r = 0; r < kOrbEvalPerThread; ++r) {
        const int64_t i = c0 + threadIdx.x + (int64_t)r * blockDim.x;
        if (i >= c1) break;
        const int64_t p = p0 == p1 ? p0 : orb_find(a.start, p0, p1 + 1, i);
        const unsigned t = (unsigned)(i - a.start[p]);      // periods hold < 2^31 samples
        double val;
        bool exact = su == 1;
        if (!exact) {
            const int64_t g0 = a.noff[p];
            const unsigned M = (unsigned)(a.noff[p + 1] - g0);
            const unsigned jt = t / su;
            if (jt >= M || (jt == M - 1 && t != jt * su)) {
                exact = true;                                   // after the last node
            } else if (M == 1) {
                val = a.y[g0];
            } else {
                const unsigned j = jt < M - 1 ? jt : M - 2;
                if (SL_GUARD(g0 + j + 1 < a.nnodes && t - j * su <= su, 0x501u)) {
                    const double4_32a w = a.w[t - j * su];         // r = t - j s (s at the last node)
                    const double *yy = a.y + g0 + j, *mm = a.M2 + g0 + j;
                    val = w.x * yy[0] + w.y * yy[1] + w.z * mm[0] + w.w * mm[1];
                } else {
                    val = 0.0;
                }
            }
        }
        if (exact) val = orb_value(a.S, a.T0, a.q, a.theta[i], a.phi[i], a.psi[i], a.beta + 3 * p);
        a.tod[i] = a.accumulate ? a.tod[i] + val : val;
    }
}

sl_status launch_orb_moments(sl_plan *p, const double *beam, double *S) {
    k_orb_moments<<<1, 32, 0, p->stream>>>((const double2 *)beam, p->L, p->K, S);
    return cuda_check(cudaGetLastError(), "k_orb_moments launch");
}

sl_status launch_orbital(sl_plan *p, const OrbLaunch &o) {
    OrbArgs a;
    a.theta = o.theta;
    a.phi = o.phi;
    a.psi = o.psi;
    a.start = o.start;
    a.noff = o.noff;
    a.beta = o.beta;
    a.S = o.S;
    a.piv = o.piv;
    a.w = reinterpret_cast<const double4_32a *>(o.w);
    a.T0 = o.T0;
    a.q = o.q;
    a.n = o.n;
    a.nper = o.nper;
    a.nnodes = o.nnodes;
    a.s = o.s;
    a.y = o.y;
    a.M2 = o.M2;
    a.tod = o.tod;
    a.accumulate = o.accumulate;
    int slot;
    if (a.s > 1 && a.nnodes > 0) {
        const int64_t nb = std::min<int64_t>((a.nnodes + 255) / 256, 152 * 32);
        slot = timing_begin(p, "orb_nodes");
        k_orb_nodes<<<(unsigned)nb, 256, 0, p->stream>>>(a);
        timing_end(p, slot);
        sl_status st = cuda_check(cudaGetLastError(), "k_orb_nodes launch");
        if (st != SL_OK) return st;
        slot = timing_begin(p, "orb_spline");
        k_orb_spline<<<(unsigned)((a.nper + kOrbWarps - 1) / kOrbWarps), 32 * kOrbWarps, 0, p->stream>>>(a);
        timing_end(p, slot);
        if ((st = cuda_check(cudaGetLastError(), "k_orb_spline launch")) != SL_OK) return st;
    }
    const int64_t per_cta = 256 * kOrbEvalPerThread;
    const int64_t nb = (a.n + per_cta - 1) / per_cta;
    if (nb > 0x7fffffff) return set_error(SL_ERR_UNSUPPORTED, "orbital_dipole_tod: n too large");
    slot = timing_begin(p, a.s == 1 ? "orb_exact" : "orb_eval");
    k_orb_eval<<<(unsigned)nb, 256, 0, p->stream>>>(a);
    timing_end(p, slot);
    return cuda_check(cudaGetLastError(), "k_orb_eval launch");
}

SL_CHECK_READER(chk_orbital)

}  // namespace sl

extern "C" sl_status sl_quad_factor(double nu_hz, double T0, double *q) {
    if (!q) return sl::set_error(SL_ERR_ARG, "sl_quad_factor: NULL output");
    if (!(nu_hz > 0.0 && nu_hz < HUGE_VAL && T0 > 0.0 && T0 < HUGE_VAL))
        return sl::set_error(SL_ERR_ARG, "sl_quad_factor: nu=%g and T0=%g must be finite and > 0", nu_hz, T0);
    const double h = 6.62607015e-34, kb = 1.380649e-23;   // exact SI values
    const double a = h * nu_hz / (kb * T0);
    *q = 0.5 * a * (std::exp(a) + 1.0) / std::expm1(a);
    return SL_OK;
}
