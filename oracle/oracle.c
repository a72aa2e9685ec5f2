/*
 * oracle.c -- plain, slow FP64 CPU oracle for the spin-harmonic total
 * convolution of Galloway et al., "BeyondPlanck VIII: Sidelobe corrections"
 * (arXiv:2201.03478), Sect. 2.1.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may call this code.  The CUDA library
 * shares nothing with it (no headers, tables or helpers) and never links it.
 *
 * What is computed (Sect. 2.1, Eq. totalconvolver with an active zyz rotation
 * R = Rz(phi) Ry(theta) Rz(psi) and D^l_{mk}(a,b,g) = e^{-ima} d^l_{mk}(b) e^{-ikg}):
 *
 *   c(theta, phi, psi) = sum_{l,m,k} s_lm conj(b_lk) d^l_{mk}(theta) e^{im phi} e^{ik psi}
 *
 * Negative m (sky) and negative k (beam) entries follow the real-field
 * relations s_{l,-m} = (-1)^m conj(s_lm) and Eq. breal; Im of m=0 and k=0
 * entries is ignored.  Polarised input (ncomp = 3, T/E/B) is the sum of the
 * three scalar convolutions, A_{k,lm} = sum_X s^X_lm conj(b^X_lk).
 *
 * Packing: sky [ncomp][nalm] complex, idx(l,m) = m(2L+1-m)/2 + l (m >= 0);
 * beam [ncomp][K+1][L+1] complex; cube [nrings][nphi][K+1] complex.
 *
 * Everything runs in double precision, plain loops; OpenMP only splits
 * independent outer loops.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

static int imax(int a, int b) { return a > b ? a : b; }
static int iabs(int a) { return a < 0 ? -a : a; }
static int odd(int a) { return (a % 2) != 0; }

/* ---------------------------------------------------------------------------
 * Wigner d^l_{mk}(beta) by Wigner's explicit sum, in long double.
 *   d^l_{mk} = sum_s (-1)^{m-k+s} sqrt((l+m)!(l-m)!(l+k)!(l-k)!)
 *              / ((l+k-s)! s! (m-k+s)! (l-m-s)!)
 *              cos(b/2)^{2l+k-m-2s} sin(b/2)^{m-k+2s}
 * Valid for small l (factorials of 2l must fit); used to pin the recurrence.
 * ------------------------------------------------------------------------- */
static long double factl(int n)
{
    long double f = 1.0L;
    for (int i = 2; i <= n; ++i) f *= (long double)i;
    return f;
}

long double or_wigner_d_explicit(int l, int m, int k, long double beta)
{
    if (iabs(m) > l || iabs(k) > l) return 0.0L;
    long double c = cosl(beta / 2), s = sinl(beta / 2);
    long double pref = sqrtl(factl(l + m) * factl(l - m) * factl(l + k) * factl(l - k));
    int slo = imax(0, k - m), shi = (l + k < l - m) ? l + k : l - m;
    long double sum = 0.0L;
    for (int t = slo; t <= shi; ++t) {
        long double den = factl(l + k - t) * factl(t) * factl(m - k + t) * factl(l - m - t);
        int ec = 2 * l + k - m - 2 * t, es = m - k + 2 * t;
        long double term = pref / den;
        for (int i = 0; i < ec; ++i) term *= c;
        for (int i = 0; i < es; ++i) term *= s;
        sum += odd(m - k + t) ? -term : term;
    }
    return sum;
}

/* ---------------------------------------------------------------------------
 * d^l_{mk}(beta) for l = 0..lmax by the three-term recurrence in l:
 *   l sqrt(((l+1)^2-m^2)((l+1)^2-k^2)) d^{l+1}
 *     = (2l+1) (l(l+1) cos b - m k) d^l - (l+1) sqrt((l^2-m^2)(l^2-k^2)) d^{l-1},
 * started at l0 = max(|m|,|k|) from the single surviving term of Wigner's sum
 * (evaluated through log-factorials in long double).  Values too small for
 * double range are carried as mantissa * 2^(600 E) with E < 0 and reported
 * as 0 until the recurrence has grown them back to E = 0; a value with E < 0
 * is below 2^-300 in magnitude.
 * ------------------------------------------------------------------------- */
void or_wigner_d_seq(int lmax, int m, int k, double beta, double *out)
{
    int l0 = imax(iabs(m), iabs(k));
    for (int l = 0; l <= lmax && l < l0; ++l) out[l] = 0.0;
    if (l0 > lmax) return;

    int s0 = imax(0, k - m);                 /* the only admissible s at l = l0 */
    int ec = 2 * l0 + k - m - 2 * s0, es = m - k + 2 * s0;
    long double ch = cosl((long double)beta / 2), sh = sinl((long double)beta / 2);
    if ((ec > 0 && ch == 0.0L) || (es > 0 && sh == 0.0L)) {
        for (int l = l0; l <= lmax; ++l) out[l] = 0.0;
        return;
    }
    long double lg = 0.5L * (lgammal(l0 + m + 1.0L) + lgammal(l0 - m + 1.0L) +
                             lgammal(l0 + k + 1.0L) + lgammal(l0 - k + 1.0L)) -
                     lgammal(l0 + k - s0 + 1.0L) - lgammal(s0 + 1.0L) -
                     lgammal(m - k + s0 + 1.0L) - lgammal(l0 - m - s0 + 1.0L);
    if (ec > 0) lg += ec * logl(fabsl(ch));
    if (es > 0) lg += es * logl(fabsl(sh));
    int sign = odd(m - k + s0) ? -1 : 1;
    if (ch < 0 && odd(ec)) sign = -sign;
    if (sh < 0 && odd(es)) sign = -sign;

    long double lg2 = lg / logl(2.0L);
    int E = 0;
    while (lg2 < -300.0L) { lg2 += 600.0L; --E; }
    double dcur = sign * (double)exp2l(lg2), dprev = 0.0;
    double x = cos(beta);
    out[l0] = (E == 0) ? dcur : 0.0;
    for (int l = l0; l < lmax; ++l) {
        double dnext;
        if (l == 0) {
            dnext = x * dcur;                 /* m = k = 0: Legendre P_1 */
        } else {
            double lp = l + 1.0, ll = (double)l;
            double A = (lp * lp - (double)m * m) * (lp * lp - (double)k * k);
            double B = (ll * ll - (double)m * m) * (ll * ll - (double)k * k);
            dnext = ((2.0 * l + 1.0) * (ll * lp * x - (double)m * k) * dcur -
                     lp * sqrt(B) * dprev) / (ll * sqrt(A));
        }
        dprev = dcur;
        dcur = dnext;
        if (E < 0 && fabs(dcur) > 0x1p300) {
            dcur *= 0x1p-600;
            dprev *= 0x1p-600;
            ++E;
        }
        out[l + 1] = (E == 0) ? dcur : 0.0;
    }
}

/* ---------------------------------------------------------------------------
 * Extended coefficient access (real-field relations, Sect. 2.1 Eq. breal).
 * ------------------------------------------------------------------------- */
static cplx sky_at(const cplx *sky, int L, int l, int m)
{
    int am = iabs(m);
    cplx v = sky[(size_t)am * (2 * L + 1 - am) / 2 + l];
    if (am == 0) return creal(v);
    if (m < 0) return odd(am) ? -conj(v) : conj(v);
    return v;
}

static cplx beam_at(const cplx *beam, int L, int l, int k)
{
    int ak = iabs(k);
    cplx v = beam[(size_t)ak * (L + 1) + l];
    if (ak == 0) return creal(v);
    if (k < 0) return odd(ak) ? -conj(v) : conj(v);
    return v;
}

/* A_{k,lm} = sum_X s^X_lm conj(b^X_lk), any sign of m and k. */
static cplx coef_A(const cplx *sky, const cplx *beam, int L, int K, int ncomp,
                   int l, int m, int k)
{
    size_t nalm = (size_t)(L + 1) * (L + 2) / 2;
    cplx a = 0;
    for (int X = 0; X < ncomp; ++X)
        a += sky_at(sky + X * nalm, L, l, m) *
             conj(beam_at(beam + (size_t)X * (K + 1) * (L + 1), L, l, k));
    return a;
}

/* ---------------------------------------------------------------------------
 * Exact per-sample convolution (Eq. totalconvolver): the full sum over
 * l, m in [-l, l], k in [-K, K].  Returns real and imaginary parts; the
 * imaginary part vanishes for real sky and beam (Eq. breal pairs).
 * ------------------------------------------------------------------------- */
void or_conv_exact(int L, int K, int ncomp, const double *sky_, const double *beam_,
                   int64_t n, const double *theta, const double *phi, const double *psi,
                   double *out_re, double *out_im)
{
    const cplx *sky = (const cplx *)sky_, *beam = (const cplx *)beam_;
#pragma omp parallel
    {
        double *d = (double *)malloc(sizeof(double) * (L + 1));
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < n; ++i) {
            cplx tot = 0;
            for (int m = -L; m <= L; ++m) {
                for (int k = -K; k <= K; ++k) {
                    or_wigner_d_seq(L, m, k, theta[i], d);
                    cplx acc = 0;
                    for (int l = imax(iabs(m), iabs(k)); l <= L; ++l)
                        acc += coef_A(sky, beam, L, K, ncomp, l, m, k) * d[l];
                    tot += acc * cexp(I * (m * phi[i] + k * psi[i]));
                }
            }
            out_re[i] = creal(tot);
            out_im[i] = cimag(tot);
        }
        free(d);
    }
}

/* ---------------------------------------------------------------------------
 * Spin "Legendre" step of the cube (Sect. 2.1 Eqs. c_m, S):
 *   G_k(r, m) = sum_{l >= max(|m|,k)} A_{k,lm} d^l_{mk}(theta_r)
 * for k = 0..K, every ring r and m in [-L, L].  G is [K+1][nrings][2L+1].
 * ------------------------------------------------------------------------- */
void or_cube_G(int L, int K, int ncomp, const double *sky_, const double *beam_,
               int nrings, const double *ring_theta, double *G_)
{
    const cplx *sky = (const cplx *)sky_, *beam = (const cplx *)beam_;
    cplx *G = (cplx *)G_;
    int nm = 2 * L + 1;
#pragma omp parallel
    {
        double *d = (double *)malloc(sizeof(double) * (L + 1));
#pragma omp for collapse(2) schedule(dynamic, 1)
        for (int k = 0; k <= K; ++k)
            for (int r = 0; r < nrings; ++r)
                for (int m = -L; m <= L; ++m) {
                    or_wigner_d_seq(L, m, k, ring_theta[r], d);
                    cplx acc = 0;
                    for (int l = imax(iabs(m), k); l <= L; ++l)
                        acc += coef_A(sky, beam, L, K, ncomp, l, m, k) * d[l];
                    G[((size_t)k * nrings + r) * nm + (m + L)] = acc;
                }
        free(d);
    }
}

/* Adjoint of or_cube_G with respect to A (real inner product Re<x, y>):
 *   Abar_{k,lm} = sum_r d^l_{mk}(theta_r) Ghat_k(r, m),   Abar is [K+1][2L+1][L+1]. */
void or_cube_G_adjoint(int L, int K, int nrings, const double *ring_theta,
                       const double *Ghat_, double *Abar_)
{
    const cplx *Ghat = (const cplx *)Ghat_;
    cplx *Abar = (cplx *)Abar_;
    int nm = 2 * L + 1;
#pragma omp parallel
    {
        double *d = (double *)malloc(sizeof(double) * (L + 1));
#pragma omp for collapse(2) schedule(dynamic, 1)
        for (int k = 0; k <= K; ++k)
            for (int m = -L; m <= L; ++m) {
                cplx *row = Abar + ((size_t)k * nm + (m + L)) * (L + 1);
                for (int l = 0; l <= L; ++l) row[l] = 0;
                for (int r = 0; r < nrings; ++r) {
                    or_wigner_d_seq(L, m, k, ring_theta[r], d);
                    cplx g = Ghat[((size_t)k * nrings + r) * nm + (m + L)];
                    for (int l = imax(iabs(m), k); l <= L; ++l) row[l] += d[l] * g;
                }
            }
        free(d);
    }
}

/* ---------------------------------------------------------------------------
 * Interpolation of the cube at pointings (Sect. 2.1 leaves the scheme to
 * the implementer; reading: separable p-point Lagrange).  Rows are the p rings around theta on the ring list extended
 * past the poles: row -1-q is ring q at colatitude -theta_q, row R+q is ring
 * R-1-q at colatitude 2 pi - theta_{R-1-q}; a ghost row holds
 * (-1)^k F_k(ring, phi + pi), because d^l_{mk}(-t) = (-1)^{m-k} d^l_{mk}(t).
 * Columns are p uniform phi nodes (periodic).  TOD (Sect. 2.1, conjugate pairs):
 *   c = Re S_0 + 2 sum_{k>=1} Re(e^{ik psi} S_k),  S_k = sum w_a w_b F_k(node).
 * ------------------------------------------------------------------------- */
typedef struct {
    int ring;      /* real ring index */
    int ghost;     /* 1 when the row lies beyond a pole */
    double theta;  /* colatitude of the row on the extended axis */
} row_t;

static row_t row_info(int R, const double *rt, int row)
{
    row_t o;
    if (row < 0) {
        o.ring = -1 - row; o.ghost = 1; o.theta = -rt[o.ring];
    } else if (row >= R) {
        o.ring = 2 * R - 1 - row; o.ghost = 1; o.theta = 2.0 * M_PI - rt[o.ring];
    } else {
        o.ring = row; o.ghost = 0; o.theta = rt[row];
    }
    return o;
}

/* largest i in [-1, R-1] with theta_ext(i) <= theta (theta_ext(-1) = -theta_0) */
static int locate_row(int R, const double *rt, double theta)
{
    if (!(theta >= rt[0])) return -1;
    int lo = 0, hi = R - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (rt[mid] <= theta) lo = mid; else hi = mid - 1;
    }
    return lo;
}

typedef struct {
    int rows[8], cols[8];
    row_t ri[8];
    double wt[8], wp[8];
} stencil_t;

static void make_stencil(int R, const double *rt, int nphi, int p, double theta, double phi,
                         stencil_t *st)
{
    int i = locate_row(R, rt, theta);
    for (int a = 0; a < p; ++a) {
        st->rows[a] = i - p / 2 + 1 + a;
        st->ri[a] = row_info(R, rt, st->rows[a]);
    }
    for (int a = 0; a < p; ++a) {
        double w = 1.0;
        for (int b = 0; b < p; ++b)
            if (b != a) w *= (theta - st->ri[b].theta) / (st->ri[a].theta - st->ri[b].theta);
        st->wt[a] = w;
    }
    double u = phi * nphi / (2.0 * M_PI);
    u -= nphi * floor(u / nphi);
    double j = floor(u), f = u - j;
    for (int b = 0; b < p; ++b) {
        double xb = b - p / 2 + 1, w = 1.0;
        for (int c = 0; c < p; ++c) {
            double xc = c - p / 2 + 1;
            if (c != b) w *= (f - xc) / (xb - xc);
        }
        st->wp[b] = w;
        long col = (long)j - p / 2 + 1 + b;
        col %= nphi;
        if (col < 0) col += nphi;
        st->cols[b] = (int)col;
    }
}

void or_interp(int K, int R, const double *rt, int nphi, int p, const double *cube_,
               int64_t n, const double *theta, const double *phi, const double *psi,
               double *tod)
{
    const cplx *cube = (const cplx *)cube_;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        stencil_t st;
        make_stencil(R, rt, nphi, p, theta[i], phi[i], &st);
        double c = 0.0;
        for (int k = 0; k <= K; ++k) {
            cplx S = 0;
            for (int a = 0; a < p; ++a) {
                int ring = st.ri[a].ring;
                double sgn = (st.ri[a].ghost && odd(k)) ? -1.0 : 1.0;
                for (int b = 0; b < p; ++b) {
                    int col = st.cols[b];
                    if (st.ri[a].ghost) col = (col + nphi / 2) % nphi;
                    S += st.wt[a] * st.wp[b] * sgn *
                         cube[((size_t)ring * nphi + col) * (K + 1) + k];
                }
            }
            if (k == 0) c += creal(S);
            else c += 2.0 * creal(cexp(I * (k * psi[i])) * S);
        }
        tod[i] = c;
    }
}

/* Adjoint of or_interp (real inner products):
 *   cube_bar_k(node) += y w_a w_b sigma eps_k e^{-ik psi}, eps_0 = 1, eps_k = 2.
 * cube_bar must be zeroed by the caller.  Serial on purpose (plain). */
void or_interp_adjoint(int K, int R, const double *rt, int nphi, int p, int64_t n,
                       const double *theta, const double *phi, const double *psi,
                       const double *tod, double *cube_bar_)
{
    cplx *cb = (cplx *)cube_bar_;
    for (int64_t i = 0; i < n; ++i) {
        stencil_t st;
        make_stencil(R, rt, nphi, p, theta[i], phi[i], &st);
        for (int k = 0; k <= K; ++k) {
            cplx ph = (k == 0 ? 1.0 : 2.0) * tod[i] * cexp(-I * (k * psi[i]));
            for (int a = 0; a < p; ++a) {
                int ring = st.ri[a].ring;
                double sgn = (st.ri[a].ghost && odd(k)) ? -1.0 : 1.0;
                for (int b = 0; b < p; ++b) {
                    int col = st.cols[b];
                    if (st.ri[a].ghost) col = (col + nphi / 2) % nphi;
                    cb[((size_t)ring * nphi + col) * (K + 1) + k] +=
                        st.wt[a] * st.wp[b] * sgn * ph;
                }
            }
        }
    }
}
