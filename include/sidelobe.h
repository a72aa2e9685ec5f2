/*
 * sidelobe.h -- C ABI of libsidelobe.so: the spin-harmonic sidelobe
 * convolution of Galloway et al., "BeyondPlanck VIII: Sidelobe corrections"
 * (arXiv:2201.03478), on one NVIDIA GB300 (sm_103a).
 *
 * The operation (Sect. 2.1).  For a real sky s (harmonic coefficients s_lm,
 * Eq. convolution) and a real beam b (b_lk, Eq. breal), with the beam's
 * boresight on +z and the pointing rotation R = Rz(phi) Ry(theta) Rz(psi),
 *
 *   c(theta, phi, psi) = sum_{l,m,k} s_lm conj(b_lk) d^l_{mk}(theta) e^{im phi} e^{ik psi}
 *                                                         (Eq. totalconvolver)
 *
 * is computed in the paper's two steps: (1) for each beam order k = 0..kmax a
 * spin-k synthesis gives the cube F_k(theta_r, phi_j) on iso-latitude rings
 * (Eqs. c_m and S: F_k is the paper's  _{k}S  up to its sign convention for
 * spin harmonics); (2) the cube is interpolated at each pointing and summed
 * with e^{ik psi} phases using the conjugate pairs F_{-k} = conj(F_k)
 * (Sect. 2.1, the pair formula before Eq. S):
 *
 *   c = Re S_0 + 2 sum_{k>=1} Re(e^{ik psi} S_k),  S_k = interpolated F_k.
 *
 * The paper does not fix the interpolation scheme; this library uses
 * separable p-point Lagrange interpolation in theta (at the actual ring
 * colatitudes) and phi (uniform, periodic), p = 2, 4 or 6, with p/2 ghost
 * rows past each pole that hold (-1)^k F_k(ring, phi + pi).
 *
 * Polarised input (ncomp = 3, T/E/B) is the sum of three scalar
 * convolutions: A_{k,lm} = sum_X s^X_lm conj(b^X_lk).
 *
 * Memory.  Every pointer argument of the compute calls is a DEVICE pointer
 * on the plan's device; the caller owns those buffers.  The plan owns its
 * own tables and scratch (allocated by sidelobe_plan_create, and for the
 * pointing sort grown on demand by the first call with a larger n).
 *
 * Packing.
 *   sky  : double [ncomp][nalm][2] (re, im), nalm = (lmax+1)(lmax+2)/2,
 *          m-major: idx(l, m) = m(2 lmax + 1 - m)/2 + l, 0 <= m <= l.
 *          Im of m = 0 entries is ignored.  s_{l,-m} = (-1)^m conj(s_lm).
 *   beam : double [ncomp][kmax+1][lmax+1][2]; entries with l < k are
 *          ignored; Im of k = 0 entries is ignored; b_{l,-k} = (-1)^k conj(b_lk).
 *   maps : the cube, [nrings][nphi][kmax+1] complex, k fastest;
 *          double2 in SL_FP64 and SL_DF64 plans, float2 in SL_FP32 and
 *          SL_TF32X3 plans.
 *          phi_j = 2 pi j / nphi on every ring.
 *   theta, phi, psi : double [n], radians; theta in [0, pi].
 *   tod  : double [n].
 *
 * Execution.  All compute calls are asynchronous on the plan's stream and
 * return after enqueuing.  Argument errors are reported synchronously;
 * launch errors are reported by the call that launched; faults inside a
 * kernel surface at the next synchronising call (sl_plan_sync).  A plan is
 * not re-entrant: one host thread and one stream at a time.
 *
 * Errors.  Every call returns an sl_status; on anything but SL_OK,
 * sl_last_error() gives a message (thread-local, valid until the next call
 * from the same thread).  No call ever terminates the process.
 */
#ifndef SIDELOBE_H
#define SIDELOBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sl_plan sl_plan;

typedef enum {
    SL_OK = 0,
    SL_ERR_ARG = -1,          /* bad argument (null pointer, size, layout) */
    SL_ERR_UNSUPPORTED = -2,  /* valid but not supported (e.g. nphi with a prime factor > 5) */
    SL_ERR_NOMEM = -3,        /* device allocation failed */
    SL_ERR_CUDA = -4,         /* CUDA runtime error (launch, copy, device fault) */
    SL_ERR_TIMEOUT = -5       /* a bounded device-side wait expired */
} sl_status;

typedef enum {
    SL_FP64 = 0,  /* everything in double precision */
    SL_FP32 = 1,  /* FP64 seeds and recurrence coefficients, pointing->grid
                     conversion, psi reduction and final TOD value; FP32
                     recurrence, sky x beam products, contraction, ring FFT,
                     maps and interpolation sums */
    SL_TF32X3 = 2, /* SL_FP32 with the l-contraction on the tensor cores
                     (tcgen05, the FP32 recurrence values and the sky x beam
                     columns split into TF32 high and low parts, three
                     products, FP32 accumulation; the multi-sky kernel with
                     one sky) */
    SL_DF64 = 4   /* FP64-class results from the FP32 pipes: the layouts,
                     tables, FFT and coordinates of SL_FP64 (maps are double2),
                     with the l-contraction and the interpolation sums run in
                     double-float arithmetic (pairs of floats, ~48-bit
                     significands), and so do the transposes of both in
                     adjoint_tod.  (SL_FP32 and SL_TF32X3 plans run adjoint_tod
                     in FP64.) */
} sl_precision;

typedef struct {
    int lmax;                  /* sky and beam band limit L >= 1 */
    int kmax;                  /* beam azimuthal band limit K, 0 <= K <= min(L, 128) */
    int ncomp;                 /* 1 (T) or 3 (T, E, B) */
    int nrings;                /* R in [4, 65534] */
    const double *ring_theta;  /* HOST [nrings]: strictly ascending colatitudes in (0, pi),
                                  symmetric: theta[R-1-r] == pi - theta[r] (to 1e-12);
                                  copied at plan creation */
    int nphi;                  /* Phi: even, >= 8, of the form 2^a 3^b 5^c, <= 16384; rings longer
                                  than one CTA's shared memory run on a cluster of 2-8 CTAs;
                                  nrings * nphi * (kmax + 1) < 2^31 */
    int interp_order;          /* p: 2, 4 or 6 points per axis (0 selects 4) */
    int precision;             /* sl_precision */
    int device;                /* CUDA device ordinal */
    void *stream;              /* cudaStream_t for all work; NULL = legacy default stream */
} sl_plan_desc;

/* Builds a plan: validates the description, uploads the ring geometry and
 * computes on the device the FP64 recurrence seeds d^{l0}_{m,+-k}(theta_r),
 * l0 = max(m, k), for every ring pair, m and k (Sect. 2.1: the spin-k
 * transforms of Eq. S).  Synchronises the stream before returning.
 * *out receives the plan (NULL on error).  Free with plan_destroy. */
sl_status sidelobe_plan_create(sl_plan **out, const sl_plan_desc *desc);

/* Step 1 of the two-step algorithm (Sect. 2.1): the cube
 *   F_k(theta_r, phi_j) = sum_{l,m} A_{k,lm} d^l_{mk}(theta_r) e^{im phi_j},
 *   A_{k,lm} = sum_X s^X_lm conj(b^X_lk),   k = 0..kmax,
 * written to maps (layout above; fully overwritten).  sky and beam are device
 * pointers in the packing above.  m is folded modulo nphi when 2 lmax + 1 >
 * nphi, which is exact at the nodes. */
sl_status synth_spin_maps(sl_plan *plan, const double *sky, const double *beam, void *maps);

/* Step 1 for many skies sharing one beam (no counterpart in the paper, which
 * convolves one sky at a time; sampling sky posteriors convolves many sky
 * realisations with one beam): for s < nsky, maps[s] is what synth_spin_maps
 * gives for sky[s] and beam.  FP32 plans only (else SL_ERR_UNSUPPORTED): the
 * l-contraction of all skies runs per (m, k) as one tensor-core tile product
 * (tcgen05; the rescaled Wigner values and the sky x beam columns are split
 * into TF32 high and low parts, three products, FP32 accumulation in tensor
 * memory), with the accuracy of the FP32 path.  nsky in [1, 65535] (larger:
 * SL_ERR_UNSUPPORTED; call once per group of skies).
 *   sky  : device double [nsky][ncomp][nalm][2], the packing above per sky;
 *   beam : device, the packing above (shared by every sky);
 *   maps : device float2 [nsky][nrings][nphi][kmax+1], fully overwritten.
 * The plan grows scratch for FP32 skies and per-sky G on the first call with a
 * larger nsky (8 (ncomp nalm + (kmax+1) nrings (2 lmax+1)) bytes per sky).  A
 * bounded wait inside the kernel that expires is reported as SL_ERR_TIMEOUT
 * by the next sl_plan_sync. */
sl_status synth_spin_maps_multi(sl_plan *plan, int nsky, const double *sky, const double *beam, void *maps);

/* Step 2 (Sect. 2.1, conjugate pairs): for i < n,
 *   tod[i] = Re S_0 + 2 sum_{k>=1} Re(e^{ik psi_i} S_k),
 * S_k the p-point Lagrange interpolation of F_k at (theta_i, phi_i).
 * The pointings are binned into grid tiles and sorted by a counting sort on
 * the device first; tod is written in the caller's order.  n = 0 is a no-op.
 * n < 2^31. */
sl_status interp_tod(sl_plan *plan, const void *maps, const double *theta, const double *phi,
                     const double *psi, int64_t n, double *tod);

/* Adjoint of interp_tod o synth_spin_maps with respect to the packed real
 * parameters of sky and beam (Re and Im of each stored entry; Im of m = 0 and
 * k = 0 entries and beam entries with l < k are not parameters and get 0):
 *   sky_grad  = d<c(sky, beam), tod>/d sky   (beam held fixed),
 *   beam_grad = d<c(sky, beam), tod>/d beam  (sky held fixed),
 * i.e. the gradients of sum_i tod_i c_i.  Shapes are those of sky and beam.
 * accumulate != 0 adds to the output buffers instead of overwriting them.
 * Either gradient pointer may be NULL to skip it. */
sl_status adjoint_tod(sl_plan *plan, const double *theta, const double *phi, const double *psi,
                      const double *tod, int64_t n, const double *sky, const double *beam,
                      double *sky_grad, double *beam_grad, int accumulate);

/* The whole forward operator in one call (Sect. 2.1: the cube of step 1, then
 * the TOD of step 2): the result of synth_spin_maps(plan, sky, beam, maps)
 * followed by interp_tod(plan, maps, theta, phi, psi, n, tod) -- maps and tod
 * are both written, bit for bit as by those two calls.  The pointing sort
 * needs the pointings only, so it runs on a second stream that the plan owns,
 * forked from the plan's stream when the call is made (after all work queued
 * there before), concurrently with the l-contraction and the ring FFT on the
 * plan's stream; the interpolation waits for both.  Arguments, layouts and
 * errors as the two calls (n may be 0: then only maps is written).  The call
 * may be captured into a CUDA graph from the plan's stream like the others. */
sl_status convolve_tod(sl_plan *plan, const double *sky, const double *beam, void *maps, const double *theta,
                       const double *phi, const double *psi, int64_t n, double *tod);

/* convolve_tod from HOST buffers, for callers that keep their data on the host
 * (no counterpart in the paper): sky, beam, theta, phi, psi and tod are host
 * pointers with the layouts of convolve_tod.  The call copies sky and beam to
 * device buffers that the plan owns and builds the cube there (synth_spin_maps);
 * meanwhile it uploads the pointings in `pieces` consecutive pieces on a stream of
 * its own, interpolates each piece on the plan's stream as soon as it has arrived
 * (interp_tod) and copies its TOD back on a third stream.  Unlike the device
 * calls it is synchronous: it returns when the whole TOD is in tod and nothing of
 * the call is in flight, with SL_ERR_TIMEOUT if a bounded wait inside a kernel
 * expired.  The copies start after the work queued on the plan's stream before
 * the call.  pieces in [1, 64] (fewer when n is smaller); SL_ERR_ARG otherwise.
 * For the copies to overlap the computation the host buffers must be page-locked
 * (cudaHostAlloc, pinned tensors); pageable buffers work, with serialised copies.
 * The plan's device buffers of this call (inputs, cube, TOD: about 32 bytes per
 * sample plus the cube) are allocated on first use and grown when n exceeds
 * every earlier call; each piece's sort uses the plan's sort scratch. */
sl_status convolve_tod_host(sl_plan *plan, const double *sky, const double *beam, const double *theta,
                            const double *phi, const double *psi, int64_t n, int pieces, double *tod);

/* The two halves of adjoint_tod, for callers that keep the adjoint cube.
 * adjoint_interp: maps_bar (maps layout, always double2) = transpose of the
 * interpolation and phase sum applied to tod; overwritten.
 * adjoint_synth: gradients from maps_bar (transpose of synth_spin_maps
 * followed by the sky x beam products). */
sl_status adjoint_interp(sl_plan *plan, const double *theta, const double *phi, const double *psi,
                         const double *tod, int64_t n, double *maps_bar);
sl_status adjoint_synth(sl_plan *plan, const double *maps_bar, const double *sky, const double *beam,
                        double *sky_grad, double *beam_grad, int accumulate);

/* interp_tod for callers that must not allocate device memory during the
 * call (no counterpart in the paper).  Some callers cannot allocate: code
 * that runs while another component owns the device-memory budget (a
 * caching allocator that must not see foreign cudaMalloc/cudaFree calls), and
 * long-running acquisition loops that cannot take the implicit device
 * synchronisation of cudaMalloc/cudaFree.  interp_tod may grow the plan's sort
 * scratch with cudaMalloc when n exceeds every earlier call; this entry point
 * never allocates: its sort scratch is one static device array of 8.75 MiB
 * that every GPU loading the library holds until the process exits.
 *
 * Same arguments, layout and result as interp_tod (the plan is created
 * beforehand with sidelobe_plan_create).  Limits: n <= 262,144 samples per
 * call (larger n returns SL_ERR_ARG: split the TOD into chunks) and plan
 * grids of at most 65,536 sort tiles (else SL_ERR_UNSUPPORTED).
 *
 * The first call on a device looks up the static array's device address
 * (cudaGetSymbolAddress, with that device current) and caches it; make that
 * first call before any stream capture.  Every call on a device shares the one
 * array and leaves its contents behind (the sort clears what must start at
 * zero), so calls that overlap on the GPU -- concurrent streams, or several
 * host threads -- race and give wrong results: serialise them. */
sl_status interp_tod_noalloc(sl_plan *plan, const void *maps, const double *theta, const double *phi,
                             const double *psi, int64_t n, double *tod);

/* ---------------------------------------------------------------------------
 * psi-grid variant of step 2 (Sect. 2.1: the Fourier transform over the beam
 * order that turns c(theta, phi, k) into c(theta, phi, psi), Eq. c_m).
 *
 * synth_psi_cube: from the cube maps (DEVICE, [nrings][nphi][kmax+1] complex,
 *   the plan's precision) to the real cube (DEVICE, [nrings][nphi][npsi]; double
 *   for FP64 and DF64 plans, float for FP32 and TF32X3 plans)
 *     c(r, j, n) = Re F_0 + 2 sum_{k=1}^{kmax} Re(e^{ik psi_n} F_k(r, j)),
 *     psi_n = 2 pi n / npsi.
 * interp_tod_psi: the TOD (DEVICE, n doubles) at the pointings from that cube:
 *   p-point Lagrange in theta and phi as interp_tod, times p-point Lagrange on
 *   the periodic psi grid (p = the plan's interp_order); ghost rows past a pole
 *   read the ring at phi + pi and psi + pi.  Sums in the plan's precision.
 * npsi: even, >= 2 kmax + 2, >= p, <= 8192.  At grid angles psi = psi_n the
 * result is the exact phase sum of interp_tod; between them it carries the psi
 * interpolation error (smaller as npsi grows).  Errors: SL_ERR_ARG (NULL
 * buffers, npsi out of range), SL_ERR_UNSUPPORTED (nrings nphi npsi >= 2^31).
 * Like interp_tod, interp_tod_psi uses the plan's sort scratch. */
sl_status synth_psi_cube(sl_plan *plan, const void *maps, int npsi, void *cube_psi);
sl_status interp_tod_psi(sl_plan *plan, const void *cube_psi, int npsi, const double *theta, const double *phi,
                         const double *psi, int64_t n, double *tod);

/* ---------------------------------------------------------------------------
 * Orbital dipole and quadrupole through the full 4pi beam (Sect. 3.3, Eqs.
 * dipole_simple, dipole and dipole_fast).  The satellite velocity beta = v/c
 * (one 3-vector per pointing period, in the frame of the pointings) gives the
 * sky signal D(n) = T0 [beta.n + q (beta.n)^2]; seen through the beam it is
 *
 *   D~ = T0 [ S_x b'_x + S_y b'_y + S_z b'_z + q ( S_xx b'_x^2 + S_yy b'_y^2
 *             + S_zz b'_z^2 + 2 S_xy b'_x b'_y + 2 S_xz b'_x b'_z + 2 S_yz b'_y b'_z ) ],
 *
 * b' = R^T beta with R = Rz(phi) Ry(theta) Rz(psi) (the rotation of the
 * convolution above), S_v = int v B dOmega the moments of the temperature beam
 * B = sum b_lk Y_lk in its own frame (boresight +z); only l <= 2 enters.
 *
 * sl_orbital_moments: the nine moments {S_x, S_y, S_z, S_xx, S_yy, S_zz, S_xy,
 *   S_xz, S_yz} of the beam (DEVICE, the plan's beam layout; component 0 is
 *   the temperature beam) into S (HOST, 9 doubles).  Synchronises the stream.
 *
 * orbital_dipole_tod: the TOD D~ for n samples (theta, phi, psi: DEVICE, n
 *   doubles; tod: DEVICE, n doubles, overwritten or, with accumulate != 0,
 *   added to).  The samples form nper consecutive pointing periods:
 *   period_start (HOST, nper + 1 int64, 0 = period_start[0] <= ... <=
 *   period_start[nper] = n) and beta (HOST, [nper][3] doubles).  T0 [K] and q
 *   (the quadrupole factor (a/2)(e^a + 1)/(e^a - 1), a = h nu / (k_B T0)) scale
 *   the result.  subsample = s: within each period the rotation is evaluated at
 *   local samples 0, s, 2s, ... only, a natural cubic spline through those node
 *   values gives the samples between them, and the samples after the last node
 *   (the remainder that s does not divide) are evaluated exactly (the paper's
 *   acceleration, s = 20 there); s = 1 evaluates every sample exactly.
 *   1 <= s <= 65536; a period holds fewer than 2^31 samples.  The period
 *   tables go through a pinned staging buffer of the plan into device scratch
 *   (both grown on demand; growth synchronises the stream); the call returns
 *   once the previous call's upload has left the staging buffer.  Errors:
 *   SL_ERR_ARG for NULL buffers, n < 0, s out of range, non-finite T0, q or
 *   beta, or period_start not running from 0 to n; SL_ERR_NOMEM if the
 *   scratch cannot grow. */
sl_status sl_orbital_moments(sl_plan *plan, const double *beam, double *S);

/* The quadrupole factor q of Eq. dipole_simple (Sect. 3.3): q = (a/2)(e^a + 1)/(e^a - 1),
 * a = h nu / (k_B T0), with the exact SI values of h and k_B; nu in Hz, T0 in K.
 * Written to *q (HOST).  SL_ERR_ARG for a NULL output or nu, T0 not finite and > 0. */
sl_status sl_quad_factor(double nu_hz, double T0, double *q);
sl_status orbital_dipole_tod(sl_plan *plan, const double *beam, double T0, double q, const double *theta,
                             const double *phi, const double *psi, int64_t n, const int64_t *period_start,
                             const double *beta, int64_t nper, int subsample, double *tod, int accumulate);

/* Frees the plan and everything it owns (after synchronising its stream).
 * NULL is a no-op. */
void plan_destroy(sl_plan *plan);

/* ---- plan utilities ---------------------------------------------------- */

/* Sizes a caller needs to allocate buffers. */
typedef struct {
    int64_t nalm;          /* sky entries per component */
    int64_t sky_doubles;   /* ncomp * nalm * 2 */
    int64_t beam_doubles;  /* ncomp * (kmax+1) * (lmax+1) * 2 */
    int64_t maps_bytes;    /* nrings * nphi * (kmax+1) * (16 or 8) */
    int64_t scratch_bytes; /* device memory the plan holds right now */
    int64_t lsteps;        /* recurrence steps one synth_spin_maps runs: sum over
                              (north ring, m, k, sign of k) of the l it visits
                              (the evanescent part below the significance
                              threshold is skipped) */
    int64_t tile_cols;     /* phi columns per sort tile (the tile is 4 rows high) */
    int64_t fft_rings;     /* rings x k orders one CTA of the ring FFT transforms */
    int64_t fft_korders;   /* (both 0 when the rings need the cluster form) */
    int64_t contraction_pairs;   /* SL_FP32 plans: ring pairs per thread of the contraction (else 0) */
} sl_plan_sizes;
sl_status sl_plan_get_sizes(const sl_plan *plan, sl_plan_sizes *out);

/* Re-targets the plan to another stream of the same device (synchronises the
 * old stream first). */
sl_status sl_plan_set_stream(sl_plan *plan, void *stream);

/* Grows the plan's pointing-sort scratch to hold n samples now, so that later
 * interp_tod / adjoint calls with at most n samples allocate nothing.
 * n in [0, 2^31).  SL_ERR_ARG while a batch graph holds the plan and n exceeds
 * the current capacity. */
sl_status sl_plan_reserve(sl_plan *plan, int64_t n);

/* Sets the width (phi columns: 8, 16 or 32, at most nphi) of the sort tiles,
 * the unit of the FP32 interpolation's shared-memory staging and of the
 * adjoint's.  Results do not depend on it; speed does (see sl_batch_create's
 * autotuner).  Reallocates the per-tile tables: SL_ERR_ARG while a batch graph
 * holds the plan; SL_ERR_UNSUPPORTED when the staged tile would not fit in
 * shared memory. */
sl_status sl_plan_set_tile_cols(sl_plan *plan, int tile_cols);

/* Sets how many rings (1, 2 or 4) and beam orders k (1 or 2) one CTA of the
 * ring FFT of synth_spin_maps transforms together (Sect. 2.1, step 1: the
 * transform along each ring of every F_k): its G reads then cover that many
 * adjacent rings and its cube writes that many adjacent k.  0, 0 restores the
 * default.  Results do not depend on it (every transform runs the same
 * arithmetic); speed does.  SL_ERR_ARG for other values; SL_ERR_UNSUPPORTED
 * when rings x korders transforms of nphi values do not fit in one CTA's shared
 * memory, or when the rings are long enough to need the cluster form. */
sl_status sl_plan_set_fft_tile(sl_plan *plan, int rings, int korders);

/* SL_FP32 plans: how many ring pairs (2, 4 or 8) each thread of the
 * l-contraction of synth_spin_maps steps together, i.e. 128, 256 or 512 ring
 * pairs per CTA (Sect. 2.1, Eqs. c_m and S: the spin "Legendre" step); 0
 * restores the automatic choice (the variant that leaves the fewest threads
 * idle for the plan's rings).  Results do not depend on it (the same
 * arithmetic per recurrence); speed does.  SL_ERR_ARG for other values;
 * SL_ERR_UNSUPPORTED for a nonzero value on plans of other precisions. */
sl_status sl_plan_set_contraction_pairs(sl_plan *plan, int pairs);

/* Synchronises the plan's stream; reports device faults as SL_ERR_CUDA and an
 * expired bounded wait inside a kernel (synth_spin_maps_multi) as
 * SL_ERR_TIMEOUT (the flag is then cleared; the context stays usable). */
sl_status sl_plan_sync(sl_plan *plan);

/* Failure-detection self-test: enqueues a kernel whose bounded wait (50 ms) on
 * a barrier that nothing signals must expire and raise the plan's error flag,
 * so that the next sl_plan_sync returns SL_ERR_TIMEOUT. */
sl_status sl_plan_selftest_timeout(sl_plan *plan);

/* Measured arithmetic peak of `device` (no counterpart in the paper: the
 * denominator of the roofline fractions reported for the ALU-bound kernels).
 * kind 0: FP64 fused multiply-add; 1: FP32 fused multiply-add; 2: packed FP32
 * (two lanes per instruction).  Runs 8 independent chains per thread on 8
 * CTAs of 256 threads per SM for about 17-20 ms, best of three timed launches
 * after a warm-up, and stores flops per second (2 per lane multiply-add) in
 * *flops_per_s.  Touches no memory; synchronises its own stream.
 * SL_ERR_ARG for a NULL output or another kind. */
sl_status sl_measure_alu_peak(int device, int kind, double *flops_per_s);

/* Per-kernel timing.  While enabled, every launch is bracketed by CUDA events
 * on the plan's stream.  sl_plan_kernel_stats fills, for up to max entries,
 * the kernel name, the number of launches and the summed device milliseconds
 * since the last reset (synchronises the stream).  Returns the number of
 * distinct kernels in *count. */
typedef struct {
    char name[32];
    int64_t launches;
    double total_ms;
} sl_kernel_stat;
sl_status sl_plan_enable_timing(sl_plan *plan, int enable);
sl_status sl_plan_kernel_stats(sl_plan *plan, sl_kernel_stat *out, int max, int *count, int reset);

/* ---- batches of detectors ------------------------------------------------
 *
 * A batch runs the whole forward path (synth_spin_maps + interp_tod) of many
 * detectors -- each with its own plan (lmax, kmax, grid, precision), sky,
 * beam and pointing stream -- as one CUDA graph (no counterpart in the paper,
 * which convolves one detector at a time).  Detectors are spread over a few
 * streams inside the graph so that small ones overlap; one graph launch
 * replaces the per-detector launches.
 *
 * sl_batch_create validates the items, reserves each plan's sort scratch for
 * its n, optionally autotunes (flags & SL_BATCH_AUTOTUNE: per detector the
 * tile width among 8, 16, 32 by timing interp_tod on its own pointings; then
 * the number of streams among 1, 2, 4, 8 by timing graph replays), and
 * captures the graph on `stream`.  It runs the path while tuning, so the
 * items' inputs must be valid by then.  The graph holds the items' pointers:
 * later runs read whatever those buffers hold, and the plans may not grow or
 * re-tile their scratch until the batch is destroyed (such calls return
 * SL_ERR_ARG).  Every item needs its own plan; plans must be on one device.
 * The plans' streams are left as they were.
 *
 * sl_batch_run enqueues one replay on the batch's stream (asynchronous). */
typedef struct sl_batch sl_batch;

typedef struct {
    sl_plan *plan;
    const double *sky, *beam;             /* device, the plan's packing */
    void *maps;                           /* device, the plan's maps layout (written) */
    const double *theta, *phi, *psi;      /* device [n] */
    int64_t n;
    double *tod;                          /* device [n] (written) */
} sl_batch_item;

/* SL_BATCH_PERSISTENT: the persistent form -- persistent launches for every
 * detector's l-contraction (one per number of ring pairs per thread among the
 * detectors, side by side) and one for every detector's interpolation, the
 * ring FFTs and pointing sorts between them, all in the graph.  Needs SL_FP32
 * plans with one interp_order, at most 32 items; the plans are given one
 * sort-tile width (the autotuner's choice, else the smallest default).  With
 * SL_BATCH_AUTOTUNE the tuner picks per detector the contraction's ring pairs
 * per thread and the ring FFT tile (timing its cube build), then the common
 * tile width (timing graph replays). */
enum { SL_BATCH_AUTOTUNE = 1, SL_BATCH_PERSISTENT = 2 };

typedef struct {
    int nitems;
    int nstreams;             /* streams the graph spreads the detectors over */
    double tuned_ms;          /* replay time measured for that choice (0 without autotuning) */
    double serial_ms;         /* the same detectors one after another on one stream, no graph
                                 (measured while autotuning; 0 otherwise) */
    int kernel_nodes;         /* kernel launches one run of the graph makes */
    int graph_nodes;          /* all nodes of the graph (kernels, memsets, events) */
    int persistent;           /* 1 for the persistent form (SL_BATCH_PERSISTENT) */
} sl_batch_info;

sl_status sl_batch_create(sl_batch **out, const sl_batch_item *items, int nitems, void *stream, int flags);
sl_status sl_batch_run(sl_batch *batch);
/* Synchronises the batch's stream; reports device faults as SL_ERR_CUDA and an
 * expired bounded wait of the persistent interpolation as SL_ERR_TIMEOUT (the
 * flag is then cleared). */
sl_status sl_batch_sync(sl_batch *batch);
sl_status sl_batch_get_info(const sl_batch *batch, sl_batch_info *info);
void sl_batch_destroy(sl_batch *batch);

/* Bounds-checked builds (the library compiled with -DSL_CHECKED): every data-
 * dependent gather and scatter index of the binning, scatter, interpolation
 * (forward and adjoint, all precisions), psi-grid, orbital and ring-FFT
 * (its digit-reversal tables) kernels is tested
 * before the access; a failed test skips the access and records a site code.
 * Returns the code of a recorded failure since the last call (0: none) and
 * clears the record; synchronises the device.  Ordinary builds: always 0. */
unsigned sl_debug_check_status(void);

/* Thread-local message describing the last non-OK status of this thread. */
const char *sl_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SIDELOBE_H */
