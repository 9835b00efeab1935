/*
 * hradon -- fast hyperbolic Radon transform on sm_103a (C ABI).
 *
 * Computes the hyperbolic Radon transform of a common-midpoint gather,
 *
 *     R_h f(tau, q) = int f( sqrt(tau^2 + q^2 x^2), x ) dx            (Eq. (1))
 *                   = 2 int_0^inf f( sqrt(tau^2 + q^2 x^2), x ) dx   (Eq. (3)),
 *
 * and its adjoint (defined by <R_h f, g> = <f, R_h* g>, Eq. (16)) with the
 * log-polar method of Nikitin, Andersson, Carlsson and Duchkov
 * (arXiv:1604.07651, Sections 2-4): after the change of variables
 * (s, y) = (t^2, x^2) the transform is a straight-line Radon transform, which
 * becomes a convolution in log-polar coordinates (Eq. (6)-(7)) evaluated by
 * cubic B-spline gridding, FFT and B-spline interpolation (Eq. (14)-(17)).
 *
 * Grids (physical units, any consistent set, e.g. s, km, s/km):
 *   gather   f[k][j] = f(t_j, x_k),  t_j = j dt (j < Nt),  x_k = k dx (k < Nx)
 *   image    g[l][i] = R f(tau_i, q_l), tau_i = tau0 + i dtau (i < Ntau),
 *            q_l = qmin + l (qmax - qmin)/(Nq - 1) (l < Nq)
 * Both arrays are row-major float32 with the time axis fastest:
 * f is [Nx][Nt], g is [Nq][Ntau]. The gather is zero outside
 * [0, (Nt-1)dt] x [0, (Nx-1)dx] (Eq. (11)).
 *
 * Ownership: every data pointer passed to radon_fwd / radon_adj /
 * radon_direct_* is a device pointer owned by the caller, on the plan's
 * device. The plan owns its tables, kernel spectra and work buffers
 * (allocated by radon_plan_create*, freed by radon_plan_destroy). Outputs
 * are overwritten, never accumulated. Calls are asynchronous on the given
 * stream (a cudaStream_t passed as void*, NULL = the legacy default
 * stream). The transform calls (radon_fwd, radon_adj, the batch, solver and
 * no-alloc calls) never make the host wait; plan and batch creation and
 * destruction, radon_plan_profile_read and the two inspection calls
 * (radon_plan_piece_lattice, radon_plan_piece_samples) synchronise. A plan may be used
 * by one stream at a time.
 *
 * Errors: every function returns a radon_status and never aborts;
 * radon_last_error() gives a message for the calling thread's last failure.
 * Everything a failed creation had allocated is released.
 *
 * Testing the out-of-memory path: when the environment variable
 * RADON_FAIL_ALLOC_AT holds n > 0 at the start of radon_plan_create* or
 * radon_batch_create*, the n-th device allocation of that creation fails
 * as if the device were out of memory, and the call returns RADON_ERR_OOM.
 */
#ifndef HRADON_H
#define HRADON_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RADON_OK = 0,
    RADON_ERR_INVALID_ARG = 1, /* bad size, spacing, range, pointer or descriptor field */
    RADON_ERR_OOM = 2,         /* device or host allocation failed */
    RADON_ERR_CUDA = 3,        /* a CUDA runtime call or kernel launch failed */
    RADON_ERR_UNSUPPORTED = 4  /* sizes beyond what the kernels handle (see radon_plan_create_ex) */
} radon_status;

typedef struct radon_plan_s* radon_plan;

#define RADON_MAX_TSPLIT 8

/*
 * Problem and method parameters.
 *   Nt, Nx, Ntau >= 2, Nq >= 1; dt, dx > 0; 0 <= qmin <= qmax (qmin < qmax if Nq > 1);
 *   tau0 >= 0; dtau > 0 (0 selects (Nt-1) dt / (Ntau-1), i.e. tau on [0, T]).
 *   sigma   : the log-polar sample spacing of Eq. (18) is divided by sigma (> 0).
 *   omega_c : half-width, in cycles per lattice cell, of the frequency
 *             rectangle L of Eq. (14) and (17) (0 < omega_c < 0.5).
 *   tsplit  : split points of the time integral, Eq. (19), as fractions of
 *             T = (Nt-1) dt in (0, 1); the split uses a smooth partition of
 *             unity in t (raised cosine in log t over [b/1.25, 1.25 b]).
 *   n_qsplit: number of slowness pieces (Section 5), >= 1; each gets its
 *             own log-polar setup.
 *   device  : CUDA device ordinal, or -1 for the calling thread's current device.
 *   rows_per_band: lattice rows one CTA of the row-FFT kernels holds, 1..6,
 *             or 0 to have radon_plan_create_ex (and radon_batch_create, when
 *             every descriptor asks for it) time each feasible value on the
 *             device and keep the fastest; radon_plan_desc reports the choice.
 *             It changes the work split only, not the results.
 *   spline_order: degree of the B-spline of the gridding, the deconvolution
 *             and the interpolation (Eq. (14)-(17)): 3 (cubic, the default)
 *             or 5 (quintic, the higher-order kernel of Section 7: six taps
 *             per axis, three guard cells per lattice side; more accurate
 *             on smooth data, about twice the tap work). The plans of one
 *             batch must share it.
 */
typedef struct {
    int Nt, Nx, Ntau, Nq;
    double dt, dx;
    double qmin, qmax;
    double tau0, dtau;
    double sigma, omega_c;
    int n_tsplit;
    double tsplit[RADON_MAX_TSPLIT];
    int n_qsplit;
    int device;
    int rows_per_band;
    int spline_order;
} radon_desc;

/* Geometry of one sub-problem of a plan (for tests and diagnostics). */
typedef struct {
    int jt_lo, jt_hi;        /* gather samples of the time piece */
    int l_lo, l_hi;          /* output columns of the slowness piece */
    double alpha, beta;      /* rotation and sector opening (Section 2.1) */
    double a, O1, O2;        /* square side and centre (Section 2.1) */
    double a_r, r_max;       /* radial extent of the lines meeting the data */
    double dphi_rule, deta_rule; /* spacing of Eq. (18) */
    double dtheta, drho, theta0, rho0;
    int Ntheta, Nrho;        /* lattice, including two guard cells per side */
    int Ptheta, Prho;        /* zero-padded FFT sizes */
    int k1max, k2max;        /* frequency rectangle L in bins */
    double theta_m;          /* kernel window |theta| <= theta_m */
    /* forward gridding work split (0 from radon_geometry, which builds no tables):
       lattice tiles, work units, tiles cut into several units, and the most
       chunks (runs of <= 8 samples of one trace) one tile holds */
    int grid_tiles, grid_units, grid_split_tiles, grid_max_tile_chunks;
} radon_piece_info;

/*
 * Fill *d with the default method parameters for the given problem:
 * tau0 = 0, dtau = (Nt-1) dt/(Ntau-1), sigma = 1.1, omega_c = 0.4,
 * time splits at 0.25 T and 0.5 T, one slowness piece, current device,
 * 3 rows per band, cubic B-splines.
 * Returns RADON_ERR_INVALID_ARG for a NULL d.
 */
radon_status radon_desc_init(radon_desc* d, int Nt, int Nx, int Ntau, int Nq, double dt,
                             double dx, double qmin, double qmax);

/*
 * Plan for the grids above with qmin = 0 and default method parameters.
 * Equivalent to radon_desc_init(&d, Nt, Nx, Ntau, Nq, dt, dx, 0, qmax) and
 * radon_plan_create_ex(out, &d). Synchronous; runs FP64 plan-time kernels.
 */
radon_status radon_plan_create(radon_plan* out, int Nt, int Nx, int Ntau, int Nq, double dt,
                               double dx, double qmax);

/*
 * Plan for an arbitrary descriptor. Computes every sub-problem's geometry
 * in FP64 on the host (Sections 2.1, 2.2, 4), its kernel spectrum
 * chi_L zeta_hat / B3_hat^2 with an FP64 quadrature on the device, and the
 * lookup tables; allocates the work buffers. On failure *out is NULL.
 * RADON_ERR_UNSUPPORTED if a lattice needs more shared memory per block
 * than the device offers (FFT lengths above 12288 along rho or 6144 along
 * theta on GB300, or time pieces x lattice length along rho x 4 bytes above
 * it for the output interpolation's profiles).
 */
radon_status radon_plan_create_ex(radon_plan* out, const radon_desc* d);

/*
 * Plan on unequally spaced offsets and/or slownesses (Section 4: the
 * log-polar method carries over to unequally spaced grids; the gridding
 * takes every sample at its own position). x: d->Nx offsets in km, strictly
 * increasing, x[0] >= 0 (the largest is X of Eq. (12)), in place of k * dx;
 * q: d->Nq slownesses in s/km, strictly increasing, q[0] >= 0, in place of
 * the regular grid from qmin to qmax. Host arrays, copied; either may be
 * NULL (the descriptor's regular grid); time and intercept time stay
 * regular. d->dx, d->qmin and d->qmax must still pass the descriptor checks;
 * with q given the plan's descriptor (radon_plan_desc) reports
 * qmin = q[0] and qmax = q[Nq-1]. The gridding weight of sample (t_j, x_k)
 * takes the trapezoid weight of x_k among the given offsets, and the lattice
 * spacing of Eq. (18) is taken over equally spaced offsets of the same range
 * [x_0, X] (the largest gap would coarsen the lattice). The adjoint is the
 * exact transpose as before; radon_mute applies its line to the given
 * slownesses. Errors as radon_plan_create_ex, plus RADON_ERR_INVALID_ARG for
 * offsets or slownesses that are not finite, negative or not strictly
 * increasing, given offsets with Nx < 2, or a single given slowness <= 0.
 */
radon_status radon_plan_create_grid(radon_plan* out, const radon_desc* d, const double* x, const double* q);

/* Release everything the plan owns. NULL is accepted. Synchronises the plan's device. */
radon_status radon_plan_destroy(radon_plan p);

/*
 * Forward transform: g = R_h f. f: device [Nx][Nt] float32 (read only),
 * g: device [Nq][Ntau] float32 (overwritten). f and g must not overlap.
 */
radon_status radon_fwd(radon_plan p, const float* f, float* g, void* stream);

/*
 * Adjoint transform: f = R_h* g, the exact transpose of radon_fwd up to
 * FP32 rounding. g: device [Nq][Ntau], f: device [Nx][Nt] (overwritten).
 */
radon_status radon_adj(radon_plan p, const float* g, float* f, void* stream);

/* Number of sub-problems (time pieces x slowness pieces) of a plan. */
radon_status radon_plan_num_pieces(radon_plan p, int* n);

/* Geometry of sub-problem `piece` (0 <= piece < num_pieces). */
radon_status radon_plan_piece_info(radon_plan p, int piece, radon_piece_info* info);

/*
 * Geometry of every sub-problem for a descriptor, computed on the host only
 * (no device is touched): writes min(*npieces, max_infos) entries of infos
 * (infos may be NULL when max_infos is 0) and sets *npieces to the total
 * count, slowness-piece major as in a plan. Same checks as radon_plan_create_ex.
 */
radon_status radon_geometry(const radon_desc* d, int* npieces, radon_piece_info* infos,
                            int max_infos);
/* As radon_geometry on given offsets / slownesses (x, q as in
 * radon_plan_create_grid; either may be NULL), host only. */
radon_status radon_geometry_grid(const radon_desc* d, const double* x, const double* q, int* npieces,
                                 radon_piece_info* infos, int max_infos);

/*
 * Inspection of one sub-problem (0 <= piece < num_pieces), for tests and
 * diagnostics. Both calls synchronise the device and copy to host memory.
 *
 * radon_plan_piece_lattice: the lattice [Ntheta][Nrho] (row-major floats) as
 * the last radon_fwd or radon_adj on the plan left it: after radon_fwd the
 * convolved lattice of Eq. (16)-(17), Q = IFFT(FFT(G) K) restricted to the
 * lattice, which the output interpolation reads; after radon_adj the
 * lattice of the transposed convolution (conj K) of the interpolation's
 * transpose, which the adjoint gridding reads. (radon_fwd_noalloc works in
 * the caller's area and leaves the plan's lattice as it was.) `count` is the
 * room of `out` in floats; less than Ntheta * Nrho is RADON_ERR_INVALID_ARG.
 *
 * radon_plan_piece_samples: the lattice position and weight of every gather
 * sample of the piece's time range, [Nx][jt_hi - jt_lo + 1] entries (trace
 * major): theta[e] and rho[e] in cells (theta index (phi - theta0) / dtheta
 * and rho index (eta - rho0) / drho of Eq. (10)), weight[e] the gridding
 * weight of Eq. (14)-(15) without the sample value (window, 2 a^2 tb e^-eta,
 * quadrature weights, 1 / (dtheta drho)). A weight of 0 marks a sample the
 * piece does not grid (muted, or outside the piece's window); its positions
 * are then undefined. Computed in FP64 at plan creation, stored as first
 * tap and FP32 fraction (positions to about 6e-8 cells). Any of the three
 * outputs may be NULL; `count` less than the number of entries is
 * RADON_ERR_INVALID_ARG.
 */
radon_status radon_plan_piece_lattice(radon_plan p, int piece, float* out, size_t count);
radon_status radon_plan_piece_samples(radon_plan p, int piece, double* theta, double* rho, float* weight,
                                      size_t count);

/* The descriptor the plan was built from (defaults resolved). */
radon_status radon_plan_desc(radon_plan p, radon_desc* d);

/* Device bytes owned by the plan. */
radon_status radon_plan_device_bytes(radon_plan p, size_t* bytes);

/*
 * Direct summation over hyperbolas on the GPU (FP32), the O(N^3) comparator:
 * Eq. (3) discretised as in the paper's reference (Section 5): Keys cubic
 * interpolation in t, trapezoid in x. Same grids and layouts as above with
 * q_l = qmin + l dq. Device pointers; asynchronous on stream.
 */
radon_status radon_direct_fwd(const float* f, float* g, int Nt, int Nx, int Ntau, int Nq,
                              double dt, double dx, double tau0, double dtau, double qmin,
                              double dq, void* stream);
/* Its exact transpose. */
radon_status radon_direct_adj(const float* g, float* f, int Nt, int Nx, int Ntau, int Nq,
                              double dt, double dx, double tau0, double dtau, double qmin,
                              double dq, void* stream);

/*
 * Per-stage timing (off by default). While enabled, every kernel launch of
 * radon_fwd / radon_adj is bracketed by CUDA events recorded on the launch
 * stream. Stages: 0 gridding (forward), 1 row FFT (forward), 2 column
 * FFT*K*IFFT (forward), 3 inverse row FFT (forward), 4 output interpolation
 * (forward), 5 theta spread of the column profiles + row FFT (adjoint), 6
 * column FFT*conj(K)*IFFT (adjoint), 7 inverse row FFT (adjoint), 8 gather
 * of the samples (adjoint), 9 rho profiles of the output columns (adjoint).
 */
#define RADON_NSTAGES 10
radon_status radon_plan_set_profiling(radon_plan p, int enable);

/*
 * Totals since the last read: for each stage, the summed kernel time in ms,
 * the number of launches, and the algorithmic bytes those launches must move
 * (inputs read once plus outputs written once; lattice-sized intermediates
 * counted at their stored size). Synchronises the recorded events, then
 * resets the totals. Any output pointer may be NULL.
 */
radon_status radon_plan_profile_read(radon_plan p, double ms[RADON_NSTAGES],
                                     long long launches[RADON_NSTAGES],
                                     double bytes[RADON_NSTAGES]);

/*
 * Batches of gathers of different sizes (many CMP gathers at once). The
 * batch holds one plan per descriptor (all on the first descriptor's
 * device) and runs every stage of the transform as ONE launch over all
 * sub-problems of all gathers, with descriptors and block maps in device
 * memory; the calls are therefore also cheap to capture in a CUDA graph.
 * Data are packed back to back: gather i occupies elements
 * [f_offsets[i], f_offsets[i+1]) of the packed gather buffer ([Nx][Nt],
 * time fastest) and image i [g_offsets[i], g_offsets[i+1]) of the packed image
 * buffer ([Nq][Ntau]); radon_batch_layout fills the n+1 offsets (elements).
 * radon_batch_fwd reads FP32 (in_type RADON_IN_F32) or BF16 (RADON_IN_BF16,
 * stored as raw bfloat16) gathers and computes in FP32; the image and the
 * adjoint's output are FP32. Asynchronous on `stream`; the batch may be used
 * on one stream at a time. Errors as for radon_plan_create_ex / radon_fwd.
 */
typedef struct radon_batch_s* radon_batch;
#define RADON_IN_F32 0
#define RADON_IN_BF16 1
radon_status radon_batch_create(radon_batch* out, int n, const radon_desc* descs);
/* As radon_batch_create on given grids: x[i] / q[i] are gather i's offsets /
 * slownesses as in radon_plan_create_grid (x or q itself, or any entry, may
 * be NULL: the regular grid). */
radon_status radon_batch_create_grid(radon_batch* out, int n, const radon_desc* descs, const double* const* x,
                                     const double* const* q);
radon_status radon_batch_destroy(radon_batch b);
radon_status radon_batch_layout(radon_batch b, int* n, long long* f_offsets, long long* g_offsets);
radon_status radon_batch_plan(radon_batch b, int i, radon_desc* d);
radon_status radon_batch_fwd(radon_batch b, const void* f, int in_type, float* g, void* stream);
radon_status radon_batch_adj(radon_batch b, const float* g, float* f, void* stream);

/*
 * Sparse Radon inversion by iterative soft thresholding (Section 3, the
 * iterations (iters) and, with a trace mask, (itersmd)): runs `iters`
 * iterations of
 *   g <- S_{c2 mu}( y + c2 R_h (f - chi_S R_h* y) ),  S_m(v) = sign(v) max(|v| - m/2, 0),
 * the proximal-gradient method of min_g ||chi_S R_h* g - f||^2 + mu ||g||_1,
 * with y = g (accelerate = 0, the paper's iteration) or the FISTA
 * extrapolation y = g_n + ((t_{n-1} - 1)/t_n)(g_n - g_{n-1}),
 * t_n = (1 + sqrt(1 + 4 t_{n-1}^2))/2, t_0 = 1 (accelerate = 1).
 *   f     [Nx][Nt] device FP32 data, zero on missing traces (read only);
 *   mask  [Nx] device FP32 trace weights chi_S (1 recorded, 0 missing), or
 *         NULL for every trace;
 *   g     [Nq][Ntau] device FP32: the starting iterate in, the result out;
 *   c2    step c^2 > 0 with c^2 ||R_h||^2 < 1 for convergence (radon_opnorm);
 *   mu    sparsity weight >= 0;
 *   work  device scratch, 256-byte aligned, of radon_ista_work_bytes bytes,
 *         owned by the caller and not used by anything else during the call.
 * Asynchronous on `stream`; no host synchronisation. Errors: INVALID_ARG for
 * NULL pointers, iters < 0, c2 <= 0, mu < 0, non-finite c2 or mu, or a short
 * or misaligned work area; CUDA for launch failures.
 */
radon_status radon_ista_work_bytes(radon_plan p, size_t* bytes);
radon_status radon_ista(radon_plan p, const float* f, const float* mask, float* g, int iters,
                        float c2, float mu, int accelerate, void* work, size_t work_bytes,
                        void* stream);

/*
 * Power iteration for the step bound of radon_ista: starting from v0
 * ([Nq][Ntau] device FP32, any vector not orthogonal to the top singular
 * vector), `iters` >= 1 steps of v <- R_h R_h* v / ||R_h R_h* v||; writes
 * ||R_h R_h* v|| of the last step, which increases to ||R_h||^2, to *norm2
 * (one device float). Scratch `work` of radon_opnorm_work_bytes bytes,
 * 256-byte aligned. Asynchronous on `stream`. Same errors as radon_ista.
 */
radon_status radon_opnorm_work_bytes(radon_plan p, size_t* bytes);
radon_status radon_opnorm(radon_plan p, const float* v0, int iters, float* norm2, void* work,
                          size_t work_bytes, void* stream);

/*
 * Radon-domain mute (Section 6, multiple attenuation): out = g with the
 * outputs (tau_i, q_l) on one side of the line q = q0 + slope * tau set to
 * zero. side RADON_KEEP_BELOW zeroes q > q0 + slope tau (keeps the
 * primaries, smaller slowness), RADON_KEEP_ABOVE zeroes q <= q0 + slope tau
 * (keeps the multiples); q_l is the plan's slowness grid (regular or given),
 * the comparison in FP64. g, out: [Nq][Ntau] device FP32 (may be the same
 * buffer). Asynchronous on `stream`.
 */
#define RADON_KEEP_BELOW 0
#define RADON_KEEP_ABOVE 1
radon_status radon_mute(radon_plan p, const float* g, float* out, double q0, double slope, int side,
                        void* stream);

/*
 * Multiple attenuation: g = the sparse Radon image of f after `iters`
 * soft-thresholding iterations (radon_ista with every trace; g is the
 * starting iterate in and the image out), then
 *   f_out = f - R_h*( g restricted to q > q0 + slope * tau ),
 * the gather with the multiples' part of the image subtracted. f, f_out:
 * [Nx][Nt] device FP32 (distinct); work: radon_demultiple_work_bytes bytes,
 * 256-byte aligned. Errors as radon_ista.
 */
radon_status radon_demultiple_work_bytes(radon_plan p, size_t* bytes);
radon_status radon_demultiple(radon_plan p, const float* f, double q0, double slope, int iters,
                              float c2, float mu, int accelerate, float* g, float* f_out, void* work,
                              size_t work_bytes, void* stream);

/*
 * Forward transform that allocates nothing, for callers that cannot call
 * cudaMalloc when they run (a host framework that has reserved the whole
 * device for its own pool, deployments with a fixed device footprint, loops
 * that cannot take the device-wide synchronisation cudaMalloc/cudaFree can
 * cause). The paper has no counterpart; this is a deployment variant of
 * radon_fwd with the same arguments and the same result (up to FP32
 * rounding order).
 *
 * Its work memory (spectra, lattices, piece descriptors) is a static device
 * array of RADON_NOALLOC_MAX_BYTES that every GPU loading this library holds
 * until the process exits; the plan's own work buffers are not used. Plans
 * whose work memory exceeds it (2048^2 gathers with default parameters need
 * about 76 MB) or that have more than 32 pieces are rejected with
 * RADON_ERR_UNSUPPORTED and a message giving the bytes needed. The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.
 * All calls on a device share the one array and it keeps the last call's
 * contents: calls whose work overlaps on the GPU (different streams, or
 * different host threads) race and give wrong results; serialise them.
 */
#define RADON_NOALLOC_MAX_BYTES (32u << 20)
radon_status radon_fwd_noalloc(radon_plan p, const float* f, float* g, void* stream);

/* Message of the calling thread's last failed call ("" if none). */
const char* radon_last_error(void);

/* Library version string. */
const char* radon_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HRADON_H */
