/*
 * mf.h -- C ABI of the GB300 meshfree log-likelihood library (libmf.so).
 *
 * The library evaluates the online stage of the meshfree likelihood
 * interpolation of Sec. II D for large batches of sampler points: rotate the
 * intrinsic point into the metric eigenbasis, evaluate the Gaussian RBF
 * interpolants with their polynomial tail (Eq. rbfcoeff) for every SVD
 * coefficient of every mode/detector overlap series and for the mode cross
 * terms, rebuild each detector's overlap at its delay with a cubic spline
 * through 10 samples (Eq. SVD + Sec. II D), and combine them with the
 * extrinsic amplitudes into lnL (Eqs. logl_basic, projected_h_fd,
 * hplus_hcross_decomposed1/2, logl_complete).
 *
 * Conventions shared by every entry point:
 *   - Return value: MF_OK (0) or a negative MF_E_* code; mf_error_string()
 *     names it.  Nothing aborts the process.
 *   - Host inputs (const double* / const int*) are copied before return; the
 *     caller keeps ownership.  Device pointers (mf_loglike*) are borrowed for
 *     the duration of the asynchronous call; the caller keeps them alive until
 *     the stream has passed the call.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *   - The handle owns all device memory it allocates; mf_free releases it.
 *   - All work runs on the GPU.  There is no CPU fallback: without a CUDA
 *     device the calls return MF_E_CUDA.
 *   - A handle is not thread-safe: calls on one handle must be serialised by
 *     the caller (different handles are independent).
 */
#ifndef MF_H
#define MF_H

#include <stddef.h>

#if defined(__GNUC__)
#define MF_API __attribute__((visibility("default")))
#else
#define MF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mf_handle mf_handle;

enum {
    MF_OK = 0,
    MF_E_INVAL = -1,    /* bad argument (NULL, size out of range, wrong order) */
    MF_E_NOMEM = -2,    /* device or host allocation failed                    */
    MF_E_CUDA = -3,     /* a CUDA runtime / library call failed                */
    MF_E_ILLCOND = -4,  /* RBF system not positive definite / too ill-conditioned */
    MF_E_RANGE = -5,    /* some queries left the sampled time window (their lnL = NaN) */
    MF_E_TIMEOUT = -6,  /* a bounded device-side wait gave up                  */
    MF_E_NOTIMPL = -7,  /* option not implemented                              */
    MF_E_STATE = -8     /* handle not fully configured for this call           */
};

/* Radial kernel phi of Eq. (rbfcoeff), with s = eps r:
 *   MF_RBF_GAUSSIAN  exp(-s^2)          positive definite (any tail)
 *   MF_RBF_PHS3      s^3                cubic polyharmonic spline; conditionally
 *                                       positive definite of order 2: needs the
 *                                       affine tail (tail_degree 1); eps only
 *                                       scales it
 *   MF_RBF_MQ        sqrt(1 + s^2)      multiquadric; conditionally definite of
 *                                       order 1: needs tail_degree >= 0
 *   MF_RBF_IMQ       1 / sqrt(1 + s^2)  inverse multiquadric; positive definite
 * (the paper's rule after Eq. rbfcoeff: order r needs monomials of degree
 * r - 1 or more).  The FP16 forms take only the kernels bounded by 1
 * (Gaussian, IMQ); BF16 and FP32 forms take all four. */
typedef enum { MF_RBF_GAUSSIAN = 0, MF_RBF_PHS3 = 1, MF_RBF_MQ = 2, MF_RBF_IMQ = 3 } mf_rbf;

/* Arithmetic of the Phi.W contraction (the interpolant evaluation).
 *   FP32        : FP32 SIMT FMAs (the plain form).
 *   BF16/FP16   : one tcgen05 MMA with 16-bit Phi and W, FP32 accumulation.
 *   *_WSPLIT    : Phi.W_hi + Phi.W_lo (W split into two 16-bit parts).
 *   *_3TERM     : Phi_hi.W_hi + Phi_hi.W_lo + Phi_lo.W_hi.
 * FP16 forms scale Phi by 2^14 and each W column by a power of two so that
 * both stay in the normal FP16 range; the scale is undone in FP32. */
typedef enum {
    MF_FORM_FP32 = 0,
    MF_FORM_BF16 = 1,
    MF_FORM_FP16 = 2,
    MF_FORM_BF16_WSPLIT = 3,
    MF_FORM_FP16_WSPLIT = 4,
    MF_FORM_BF16_3TERM = 5,
    MF_FORM_FP16_3TERM = 6,
    MF_FORM_MLP = 7          /* trained surrogate network (mf_train_surrogate) */
} mf_form;

/* Name of a status code (static string). */
MF_API const char *mf_error_string(int status);

/* Library version string, e.g. "mf 0.1 sm_103a". */
MF_API const char *mf_version(void);

/*
 * SVD compression of one overlap matrix (Eq. SVD).
 *   z      : host, [N][M][2] FP64 (re, im) -- row n = overlap series at node n.
 *   coef   : host out, [N][rank][2]  -- C_{n,i} = sum_t z_n(t) conj(u_i(t)).
 *   basis  : host out, [rank][M][2]  -- orthonormal u_i (rows of V^H),
 *            ordered by decreasing singular value.
 *   sv     : host out or NULL, [rank] singular values.
 * Runs on the GPU in FP64 with the library's own kernels: block subspace
 * iteration on Z with rank + 10 columns (Gram-Schmidt applied twice, a
 * one-sided Jacobi SVD of the small triangular factor), until the leading
 * `rank` right singular vectors, weighted by their singular values, change
 * by less than 1e-12 s_1 between iterations (at most 30 iterations); then
 * C = Z V.  The singular values are accurate to rounding of s_1 (Z^H Z is
 * never formed).  Deterministic: the start block is a fixed pseudo-random
 * pattern and every reduction has a fixed order.  The basis is orthonormal
 * even when Z has rank r < rank (for instance Z = 0): the rows beyond r then
 * complete the set, with singular values and coefficients at rounding level
 * (0 for Z = 0).  Synchronous.
 * Requires N >= M (at least as many nodes as time samples),
 * 1 <= rank <= M <= 8192.
 */
MF_API int mf_svd_compress(const double *z, int N, int M, int rank, double *coef, double *basis,
                    double *sv, void *stream);

/*
 * Build the interpolants (Eq. rbfcoeff) for K columns at N nodes.
 *   nodes       : host [N][4] FP64, node coordinates in the metric eigenbasis.
 *   node_values : host [N][K] FP64, the quantities interpolated: per
 *                 (detector, mode) the rank real parts then rank imaginary
 *                 parts of the SVD coefficients; then per detector the cross
 *                 terms sigma: n_modes real diagonals, Re of the strict upper
 *                 triangle (row-major), Im of the strict upper triangle.
 *   rbf, eps    : radial kernel and shape parameter (eps > 0).
 *   tail_degree : -1 (none), 0 (constant) or 1 (affine: 1, x1..x4); at
 *                 least the kernel's minimum (mf_rbf), else MF_E_INVAL.
 * Solves [Phi P; P^T 0][a; b] = [F; 0] on the GPU in FP64 with the
 * library's own kernels.  Positive definite kernels (Gaussian, IMQ):
 * Cholesky of Phi plus the tail Schur complement; cond = cond(Phi).
 * Conditionally definite kernels (PHS3, MQ): the null-space method, Q R = P
 * (Householder), Cholesky of the projected +/-(Q^T Phi Q) on the null space
 * of P^T, then the tail coefficients from R; cond = that of the projected
 * matrix.  Returns MF_E_ILLCOND if the (projected) matrix is not numerically
 * positive definite, e.g. for duplicate nodes.  Synchronous on `stream`.
 * Limits: 1 <= N <= 65536, 1 <= K <= 4096; N > number of tail terms.
 */
MF_API int mf_build(const double *nodes, const double *node_values, int N, int K, mf_rbf rbf,
             double eps, int tail_degree, void *stream, mf_handle **out);

/*
 * Column layout of the handle's K columns (must match node_values above):
 * n_det detectors, n_modes modes with (l, m) pairs in ell_m [n_modes][2]
 * (m > 0; the negative-m mode h_{l,-m} is the one interpolated, Eqs.
 * hplus_hcross_decomposed1/2), `rank` SVD coefficients per mode.  Requires
 * K == n_det*n_modes*2*rank + n_det*n_modes^2.  Supported modes: (2,2),
 * (2,1), (3,3), (3,2), (4,4); n_modes <= 5; n_det <= 8; rank <= 128.
 */
MF_API int mf_set_layout(mf_handle *h, int n_det, int n_modes, const int *ell_m, int rank);

/*
 * Host-only planner: the device column layout a handle with this layout
 * would take for a form whose passes are at most pass_max columns wide
 * (16..512, a multiple of 16; 176 for MF_FORM_FP32, 256 for the tcgen05
 * cluster design) and, with pass_count > 0, exactly that many passes.
 * Per detector its mode groups (interleaved Re/Im of a run of SVD
 * coefficients, padded to 8 columns) then its cross-term group, packed
 * contiguously into the fewest passes that fit, the widest pass minimised;
 * a mode's coefficients are split into runs when whole modes do not fit.
 *   n_pass, pass_width [<= 48], Kdev: out, the passes and their padded total.
 *   user_of_dev: out or NULL, [Kdev] node_values column of each device
 *                column (-1 for padding); cap = its length.
 * Touches no GPU.  MF_E_INVAL if nothing fits or an argument is out of range.
 */
MF_API int mf_plan_layout(int n_det, int n_modes, int rank, int pass_max, int pass_count, int *n_pass,
                          int *pass_width, int *Kdev, int *user_of_dev, int cap);

/*
 * SVD basis vectors of every (detector, mode) overlap series (Eq. SVD).
 *   basis : host [n_det][n_modes][rank][M][2] FP64 (re, im).
 *   t0, dt: time of sample 0 and the sample spacing (seconds).
 * The series is evaluated at t = t_c + dt_k with a not-a-knot cubic spline
 * through the 10 samples j-4..j+5, j = floor((t - t0)/dt) (Sec. II D).
 */
MF_API int mf_set_basis(mf_handle *h, const double *basis, int M, double t0, double dt);

/*
 * Frozen antenna patterns and delays (Eq. projected_h_fd):
 *   det : host [n_det][3] = F+(psi=0), Fx(psi=0), dt_k (seconds from
 *         geocentre); F+(psi) = F+0 cos2psi + Fx0 sin2psi,
 *         Fx(psi) = -F+0 sin2psi + Fx0 cos2psi.
 *   d_ref: luminosity distance at which the node overlaps were computed;
 *         the amplitude of a query is d_ref / d_L.
 */
MF_API int mf_set_detectors(mf_handle *h, const double *det, double d_ref);

/*
 * Sky-dependent antenna patterns and delays (Eq. projected_h_td, long-
 * wavelength response), in place of mf_set_detectors: mf_loglike then needs
 * E >= 7 extrinsic columns, the last two being the source's right ascension
 * alpha and declination delta (rad).  For channel k (a detector, or one
 * frequency band of a detector whose signal lasts long enough for the Earth
 * to turn: Sec. II B, 3G detectors) at the epoch t_c + tau_k:
 *   hour angle h = gmst0 + omega (t_c + tau_k) - alpha,
 *   source direction w = (cos delta cos h, -cos delta sin h, sin delta),
 *   wave-frame axes X = cos psi X0 + sin psi Y0, Y = -sin psi X0 + cos psi Y0
 *   with X0 = (-sin h, -cos h, 0), Y0 = (-cos h sin delta, sin h sin delta,
 *   cos delta),
 *   F+ = D : (X X - Y Y), Fx = D : (X Y + Y X), delay dt_k = -(r_k . w).
 *   tensor : host [n_det][3][3] FP64 detector tensors D_k (symmetric; for
 *            arms u, v: (u u^T - v v^T) / 2), Earth-fixed frame.
 *   pos    : host [n_det][3] detector positions divided by c (seconds,
 *            |.| <= 1), Earth-fixed frame.
 *   tau    : host [n_det] epoch offsets (seconds, |.| <= 1e7), or NULL (0).
 *   gmst0  : Greenwich sidereal angle (rad) at t_c = 0; omega: the Earth's
 *            rotation rate (rad/s).  d_ref as in mf_set_detectors.
 * The delay enters the spline time t_c + dt_k (Sec. II D), so every channel's
 * basis must cover t_c + dt_k +- 5 samples (else NaN and MF_E_RANGE).
 * MF_E_STATE before mf_set_layout; MF_E_INVAL for non-finite or out-of-range
 * values.  mf_set_detectors switches back to frozen patterns.
 */
MF_API int mf_set_sky(mf_handle *h, const double *tensor, const double *pos, const double *tau,
                      double gmst0, double omega, double d_ref);

/*
 * Sampler frame -> metric eigenbasis (Sec. II D, Delta-e coordinates):
 * x = R (theta - centre), R = rows of metric eigenvectors by ascending
 * eigenvalue, each row's largest-|.| entry positive.  metric: host [4][4]
 * symmetric positive definite, or NULL for R = I.  centre: host [4] or NULL
 * for 0.  The 4x4 eigendecomposition runs on the GPU (FP64 Jacobi).
 */
MF_API int mf_set_rotation(mf_handle *h, const double *metric, const double *centre);

/*
 * General affine frame instead of mf_set_rotation: x = A (theta - centre)
 * with A host [4][4] row-major (any invertible map, e.g. the rotation into
 * the metric eigenbasis followed by a division by the ellipsoid's semi-axes,
 * which is what mf_place_nodes returns), centre host [4] or NULL.
 */
MF_API int mf_set_frame(mf_handle *h, const double *A, const double *centre);

/* Select the Phi.W arithmetic (default MF_FORM_FP32).  Converts the weights
 * for the form on first use (synchronous on the legacy stream).  Returns
 * MF_E_NOTIMPL for an FP16 form on a handle built with MF_RBF_PHS3 or
 * MF_RBF_MQ (their values leave the FP16 range), MF_E_STATE for MF_FORM_MLP
 * before mf_train_surrogate; the previous form stays selected then. */
MF_API int mf_set_form(mf_handle *h, mf_form form);

/*
 * lnL for Q queries, asynchronous on `stream` (Eq. logl_complete read with
 * the -1/2 ||h||^2 of Eq. logl_basic):
 *   lnL_q = sum_k [ Re sum_mu conj(c_k,mu) z_k,mu(t_c + dt_k)
 *                   - 1/2 sum_mu,nu conj(c_k,mu) sigma_k,mu,nu c_k,nu ],
 *   c_k,mu = (d_ref/d_L) 1/2 [ (F+ + i Fx) Y_{l,-m} + (-1)^l (F+ - i Fx) conj(Y_{l,m}) ],
 *   Y = -2Y_lm(iota, phi_c).
 * intrinsic : device [Q][4] FP32, sampler-frame coordinates; 16-byte aligned
 *             (rows are read as float4), else MF_E_INVAL.
 * extrinsic : device [Q][E] FP32, E >= 5, columns (d_L [Mpc], cos iota,
 *             psi, phi_c, t_c [s]); after mf_set_sky E >= 7 and columns 5, 6
 *             are (alpha, delta) [rad].
 * out_lnL   : device [Q] FP32, written by the call.
 * Queries whose spline stencil leaves the sampled window get NaN and are
 * counted; mf_sync_status() reports them.  Q == 0 is a no-op.  Q <= 2^26.
 */
MF_API int mf_loglike(mf_handle *h, const float *intrinsic, const float *extrinsic, int Q, int E,
               float *out_lnL, void *stream);

/*
 * mf_loglike without any device allocation in the call.  The paper has no
 * counterpart: this is a service for callers that cannot allocate device
 * memory while they run -- callers that give all device memory to their own
 * fixed pool at start-up, and real-time sampler loops that forbid
 * allocation (and the synchronisation it can bring) once they run.
 * Same arguments and results as mf_loglike with the plain FP32 form (the
 * handle must be in MF_FORM_FP32, else MF_E_STATE; the handle's device must
 * be the current device, else MF_E_STATE).  When the columns need
 * several passes, the partial sums live in one fixed array of
 * MF_NOALLOC_MAX_PARTIAL floats (16 MiB) inside the library, which every GPU
 * that loads the library keeps until the process exits:
 *   - n_pass * Q above MF_NOALLOC_MAX_PARTIAL returns MF_E_INVAL (n_pass is
 *     mf_query "n_pass"); nothing is launched.
 *   - All calls on a device share the array; calls that overlap on the GPU
 *     (other streams, other handles) race and must be serialised by the caller.
 *   - The first call on each device looks up the array's device address and
 *     caches it; make that first call before any stream capture starts.  The
 *     cached address does not survive cudaDeviceReset: after a reset, do not
 *     call this entry point on that device again in the same process.
 */
#define MF_NOALLOC_MAX_PARTIAL 4194304
MF_API int mf_loglike_noalloc(mf_handle *h, const float *intrinsic, const float *extrinsic, int Q,
                              int E, float *out_lnL, void *stream);

/*
 * Interpolated columns only (the Phi.W stage, Eq. rbfcoeff), in the
 * node_values column order: out [Q][K] device FP32, computed in the handle's
 * current form (FP32 SIMT, or the tcgen05 kernel of a 16-bit form with its
 * epilogue writing columns instead of lnL; the FP16 column scales are
 * undone), or in MF_FORM_MLP the trained network's de-standardised
 * outputs for every query (no radius fallback; these are exactly the
 * columns the surrogate's fused lnL epilogue combines).  intrinsic as in
 * mf_loglike.  Asynchronous on `stream`.
 */
MF_API int mf_eval_columns(mf_handle *h, const float *intrinsic, int Q, float *out, void *stream);

/* ------------------------------------------------------------------------
 * Batched events: many interpolants (events, e.g. independent sampler runs
 * with their own nodes, SVD rank and batch size) evaluated by ONE persistent
 * tcgen05 launch (plus one combine launch), replayed from a CUDA graph.  The
 * per-query result of every event is exactly mf_loglike's (Eq.
 * logl_complete); only the scheduling differs.
 *
 * mf_batch_create plans a batch over `n_events` (1..128) handles that share
 * one tcgen05 form (MF_FORM_BF16 .. MF_FORM_FP16_3TERM, set beforehand) and
 * the same number of modes; layout, basis and detectors must be set.
 *   Q_plan[e]      : host, the batch size expected for event e (shapes the
 *                    timing runs; calls may use any sizes).
 *   autotune_shape : 1 = time every launch shape that fits (passes per event
 *                    = cluster size, weight-ring depth) on synthetic queries
 *                    of the planned sizes and keep the fastest; 0 = fewest
 *                    passes, deepest ring, no timing.
 * The plan re-lays out every handle in the chosen number of column passes
 * (the "pass_count" option of mf_set_option, which mf_loglike honours too).
 * The batch keeps pointers to the handles: free the batch before them.
 * Changing a handle's form, layout, basis, detectors, rotation or pass
 * options afterwards makes mf_batch_loglike return MF_E_STATE.
 * Errors: MF_E_INVAL (arguments, mixed forms or mode counts), MF_E_STATE
 * (a handle not ready or not in a tcgen05 form), MF_E_NOTIMPL (no shape
 * fits), MF_E_TIMEOUT (a timing run's bounded wait gave up).  On error the
 * handles get their previous layout back and *out is NULL. */
typedef struct mf_batch mf_batch;
MF_API int mf_batch_create(mf_handle *const *hs, int n_events, const int *Q_plan,
                           int autotune_shape, void *stream, mf_batch **out);

/* Enqueue lnL for every event of the batch on `stream` (asynchronous).
 * intrinsic[e] / extrinsic[e] / out_lnL[e]: device pointers as in
 * mf_loglike for event e, Q[e] queries (0 allowed, then the pointers may be
 * NULL), E >= 5 the extrinsic row stride of all events, sum of Q <= 2^30.
 * The first call, and any call whose pointers or sizes differ from the
 * previous call's, captures the launches into the batch's CUDA graph
 * (updating it in place); an identical call replays it.  A call with larger
 * sizes than any before grows a scratch buffer and synchronises `stream`
 * first.  Out-of-window queries get NaN as in mf_loglike; the counts and
 * device status are read with mf_batch_sync_status. */
MF_API int mf_batch_loglike(mf_batch *b, const float *const *intrinsic,
                            const float *const *extrinsic, const int *Q, int E,
                            float *const *out_lnL, void *stream);

/* "timing": 1 = CUDA events around each mf_batch_loglike (read with
 * mf_batch_query "kernel_ms"); "graph": 0 = launch directly, 1 (default) =
 * capture / replay. */
MF_API int mf_batch_set_option(mf_batch *b, const char *key, double value);

/* "n_events", "n_pass" (passes per event = cluster size), "ring" (weight
 * ring depth), "nbox" (widest pass), "clusters" (resident clusters
 * launched), "n_items" (work items of the last call), "captures",
 * "replays", "launches" (kernel launches per call), "n_tuned" (shapes timed
 * by the autotuner), "kernel_ms" (last call, "timing" on; waits for it). */
MF_API int mf_batch_query(const mf_batch *b, const char *key, double *value);

/* The autotuner's i-th timed shape and its time (ms) per batch launch. */
MF_API int mf_batch_tuning(const mf_batch *b, int i, int *n_pass, int *ring, double *ms);

/* Wait for `stream`; MF_E_TIMEOUT if a bounded device wait gave up, else
 * MF_E_RANGE with *n_bad = out-of-window queries over all events, else
 * MF_OK.  Resets the counters. */
MF_API int mf_batch_sync_status(mf_batch *b, void *stream, long long *n_bad);

MF_API void mf_batch_free(mf_batch *b);

/* One-shot convenience: plan (no timing), run, wait for `stream`, free. */
MF_API int mf_loglike_batch(mf_handle *const *hs, int n_events, const float *const *intrinsic,
                            const float *const *extrinsic, const int *Q, int E,
                            float *const *out_lnL, void *stream);

/* ------------------------------------------------------------------------
 * Surrogate network (no counterpart in the paper: a learned stand-in for the
 * interpolants of Eq. rbfcoeff, with the RBF path as its fallback): a
 * fully connected network n_in -> hidden (x n_hidden) -> n_out with SiLU
 * activations, FP32 master weights, BF16 GEMM operands and FP32
 * accumulation, trained on the GPU by the library's own forward, backward
 * and Adam kernels.  Layers l: z_l = W_l h_{l-1} + b_l, h_l = SiLU(z_l),
 * output y = z_last; loss = mean over rows and outputs of (y - t)^2.
 * Flat parameter order (set/get): per layer W_l [out][in] row-major, then
 * b_l [out].
 * Limits: 1 <= n_in <= 16; hidden a multiple of 16 up to 256; n_hidden >= 1
 * (at most 7); n_out a multiple of 8.  MF_E_INVAL otherwise. */
typedef struct mf_mlp mf_mlp;
typedef struct mf_mlp_train_params {
    int steps;                 /* Adam steps */
    int batch;                 /* minibatch rows (multiple of 8; capped at n) */
    float lr, lr_min;          /* cosine schedule from lr to lr_min over the steps */
    float beta1, beta2, eps;   /* Adam constants; <= 0 selects 0.9, 0.999, 1e-8 */
    unsigned long long seed;   /* minibatch order */
} mf_mlp_train_params;
/* Seeded initialisation: every W and b uniform in +-1/sqrt(fan_in). */
MF_API int mf_mlp_create(int n_in, int hidden, int n_hidden, int n_out, unsigned long long seed,
                         mf_mlp **out);
MF_API void mf_mlp_free(mf_mlp *m);
MF_API long long mf_mlp_n_params(const mf_mlp *m);
/* Host FP32 arrays of mf_mlp_n_params floats; both synchronise the device. */
MF_API int mf_mlp_set_params(mf_mlp *m, const float *host);
MF_API int mf_mlp_get_params(const mf_mlp *m, float *host);
/* Y [B][n_out] = network(X [B][n_in]); device FP32, Y 16-byte aligned.
 * Asynchronous on `stream`. */
MF_API int mf_mlp_forward(mf_mlp *m, const float *X, int B, float *Y, void *stream);
/* Gradient of the loss on exactly the rows X [B][n_in], T [B][n_out]
 * (device FP32, B a multiple of 8): host_grad (n_params floats, flat
 * order) and *host_loss, either may be NULL.  Synchronous; parameters are
 * unchanged.  MF_E_TIMEOUT if a bounded device wait gave up. */
MF_API int mf_mlp_gradient(mf_mlp *m, const float *X, const float *T, int B, float *host_grad,
                           double *host_loss, void *stream);
/* Train on the n rows X [n][n_in], T [n][n_out] (device FP32): `steps`
 * Adam steps on minibatches of `batch` rows taken in a scrambled order
 * (row j of step s = (a_s + j c) mod n, a_s drawn from the seed and the
 * step), one CUDA-graph replay per step.  Resets the Adam moments.
 * Synchronous (waits for `stream`). */
MF_API int mf_mlp_train(mf_mlp *m, const float *X, const float *T, int n,
                        const mf_mlp_train_params *p, void *stream);
/* "n_params", "loss" (mean squared residual of the last training step),
 * "steps_done", "train_ms" (wall time of the last mf_mlp_train on the GPU). */
MF_API int mf_mlp_query(const mf_mlp *m, const char *key, double *value);

/* ------------------------------------------------------------------------
 * Learned surrogate of a handle's interpolant (form MF_FORM_MLP; not in the
 * paper: it replaces only the Phi.W stage, the time interpolation, amplitudes
 * and quadratic form of Eqs. SVD, projected_h_fd and logl_complete are the
 * RBF path's).  A
 * network 4 -> hidden (x n_hidden) -> K' (K' = K rounded up to 8), SiLU,
 * maps the metric-eigenbasis point x = R (theta - centre) to the per-column
 * standardised interpolated columns (node_values order); it is trained on
 * the GPU (mf_mlp kernels) on n_train points labelled by the FP64 RBF
 * interpolant, itself evaluated on the GPU (FP64 kernel sums and the
 * library's own FP64 GEMM against the FP64 weights).
 *   train_intrinsic : device [n_train][4] FP32 sampler-frame points (16-byte
 *                     aligned), drawn from the region the sampler explores.
 *   held_*          : device held-out queries [n_held][4], [n_held][E].
 * The held-out gate compares the network's lnL with the plain FP32 RBF
 * path's on the held-out queries: it passes when max |dlnL| <= gate_max and
 * the median <= gate_median (defaults 0.1 and 0.01).  In MF_FORM_MLP,
 * mf_loglike then evaluates the network (chunks of 65536 queries: input
 * layer, hidden GEMMs, final GEMM fused with the lnL epilogue) and sends
 * queries with |x| beyond the training radius (r_gate; by default the
 * largest training |x|) to the FP32 RBF path: those queries are compacted
 * on the device and the RBF launch reads their count there, so the call
 * never waits for the GPU (mf_query "fallback_rate" reads the last call's
 * count and waits for it); if the gate failed, the RBF path serves every
 * query.  mf_query: "fallback_rate",
 * "surrogate_gate", "surrogate_heldout_max" / "_median" / "_p99",
 * "surrogate_train_ms", "surrogate_label_ms", "surrogate_gate_ms",
 * "surrogate_loss", "surrogate_r_gate", "surrogate_n_params".
 * Synchronous; the handle keeps its form (select MF_FORM_MLP afterwards).
 * Zero fields of the parameters select: steps 20000, batch 4096, hidden
 * 256, n_hidden 3, lr 1e-3 -> lr_min 1e-5 (cosine). */
typedef struct mf_surrogate_params {
    int steps, batch, hidden, n_hidden;
    float lr, lr_min;
    float gate_max, gate_median;
    float r_gate;              /* training radius in x; 0 = largest training |x| */
    unsigned long long seed;
} mf_surrogate_params;
MF_API int mf_train_surrogate(mf_handle *h, const float *train_intrinsic, int n_train,
                              const float *held_intrinsic, const float *held_extrinsic, int n_held,
                              int E, const mf_surrogate_params *params, void *stream);

/* ------------------------------------------------------------------------
 * Start-up generation (Sec. II C) from data, on the GPU.
 *
 * Frequency-domain stand-in templates (no waveform model of the paper is
 * available here): mode (l, m) at intrinsic point theta, with F = 2 f / m,
 *   h_{l,-m}(f) = amp (F/f_ref)^(-7/6) exp(-i (m/2) sum_a s_a theta_a u_a(F/f_ref))
 * for F_lo(theta) <= F <= f_hi, F_lo = f_lo exp(cut_rate cut_dir . theta),
 * u_a(x) = x^p_a - 1 - p_a (x - 1); 0 elsewhere.  One-sided frequency grid
 * f_j = j / (L dt), j = 0 .. L/2. */
typedef struct mf_wave {
    int n_modes;
    int ell_m[5][2];
    double amp[5];
    double f_lo, f_hi, f_ref;
    double powers[4], scales[4];
    double cut_dir[4], cut_rate;
    int L;                    /* FFT length: power of two, 16 .. 8192 */
    double dt;                /* sample spacing of the overlap series (s) */
} mf_wave;

/* Node placement (Sec. II C 1): the constant-match ellipsoid
 * x^T g x <= mismatch of the metric g (host [4][4], SPD; Eq. MisMatch),
 * semi-axes a_d = sqrt(mismatch / lambda_d) along the eigenvectors (ascending
 * eigenvalue, rows of R as in mf_set_rotation), the longest (d = 0) times
 * `squeeze` in (0, 1]; nodes theta_n = centre + R^T (a * y_n) with y_n the
 * first N points of the 4-D Halton sequence (bases 2, 3, 5, 7; indices
 * skip+1, skip+2, ...) mapped to [-1,1]^4 that fall in the unit ball,
 * selected in index order on the GPU.
 *   theta : host out [N][4] (sampler frame);  y : host out [N][4] or NULL
 *   (whitened nodes, the unit ball);  frame : host out [4][4] or NULL,
 *   A = diag(1/a) R, so that y = A (theta - centre) (for mf_set_frame). */
MF_API int mf_place_nodes(const double *metric, const double *centre, double mismatch, double squeeze, int N,
                          long long skip, double *theta, double *y, double *frame);

/* Squeeze factor (Sec. II C 1): the true match (Eq. Match: normalised
 * overlap of the dominant-mode templates, modulus, maximised over the L
 * circular time shifts) from the centre to centre + t a_0 e_0 along the
 * longest axis, t = i / n_t (i = 1..n_t), each point one CTA with an
 * inverse FFT; *kappa = the first t where it falls below 1 - mismatch
 * (linear interpolation; 1 if it never does).  psd host [L/2+1];
 * match_out host [n_t] or NULL.  Synchronous. */
MF_API int mf_squeeze_factor(const mf_wave *w, const double *psd, const double *metric, const double *centre,
                             double mismatch, int n_t, double *kappa, double *match_out);

/* Node overlaps (Sec. II C 2) of N nodes against n_det detectors' data:
 *   z[k][mu][n][s] = 4 df sum_j conj(h_mu(f_j; theta_n)) d_k(f_j) / S_k(f_j)
 *                    exp(2 pi i f_j t_s),  t_s = (s - M/2) dt, s = 0..M-1
 * (the circular time shifts of an inverse FFT of length L, FP64, one CTA per
 * (node, mode)), and the cross terms
 *   sigma[k][n][mu][nu] = 4 df sum_j conj(h_mu) h_nu / S_k   (Hermitian).
 *   theta : host [N][4];  data : host [n_det][L/2+1][2] (re, im);
 *   psd : host [n_det][L/2+1];  z : host out [n_det][n_modes][N][M][2];
 *   sigma : host out [n_det][N][n_modes][n_modes][2].  Synchronous. */
MF_API int mf_standin_overlaps(const mf_wave *w, const double *theta, int N, const double *data,
                               const double *psd, int n_det, int M, double *z, double *sigma, void *stream);

/* ------------------------------------------------------------------------
 * Nested sampling over the online likelihood (the paper samples the
 * posterior with nested sampling and random-walk proposals in the metric
 * eigenbasis Delta-e: Secs. III A, III C), batched for the GPU.
 *
 * State of a point (dim 9, or 11 for a handle with sky-dependent patterns),
 * with a uniform prior on the domain:
 *   v[0..3] x in the Delta-e ball |x| <= r_ball (theta = centre + R^T x),
 *   v[4] u in [0,1] with d_L^3 = dl_min^3 + u (dl_max^3 - dl_min^3),
 *   v[5] cos iota in [-1,1], v[6] psi in [0,pi), v[7] phi_c in [0,2pi),
 *   v[8] t_c in [-tc_half, tc_half], v[9] alpha in [0,2pi),
 *   v[10] sin delta in [-1,1].
 * Each iteration the `batch` lowest-likelihood live points die (the j-th,
 * in ascending lnL, shrinks log X by 1/(n_live - j)); each is replaced by a
 * surviving point moved by `walks` random-walk steps v + scale sd z (sd:
 * per-dimension spread of the live points; z standard normal), a step being
 * kept if it stays in the domain and its lnL exceeds the largest lnL that
 * died.  All walkers step together: one proposal kernel, one mf_loglike call
 * over the batch (the handle's current form), one acceptance kernel.  The
 * scale adapts as scale *= exp(accepted fraction - 0.5) per iteration.
 * Random numbers are the splitmix64 outputs of `seed` at counters
 * ((iter * 65536 + walker) * 1024 + step) * 64 + slot.  Stops when the live
 * points can add less than dlogz to log Z (or after max_iter iterations);
 * the last live points are then added with equal shares of the remaining
 * volume.
 *   out_v [max_out][dim], out_lnl [max_out], out_logwt [max_out] (host):
 *     the dead points then the final live points, in order, with their log
 *     posterior weight lnL + log dX (unnormalised); n_samples in *res may
 *     exceed max_out (the rest is not stored).  NULL with max_out = 0.
 *   test_sigma > 0 selects a diagnostic likelihood with a known evidence
 *     instead of the handle's: lnL = -|x - test_mu|^2 / (2 test_sigma^2)
 *     (h may then be NULL: identity rotation, zero centre, dim 9).
 * Synchronous (waits for `stream` once per iteration).  MF_E_INVAL for
 * sizes out of range (8 <= n_live <= 65536, 1 <= batch < n_live,
 * 1 <= walks <= 1000), MF_E_STATE for an unconfigured handle. */
typedef struct mf_ns_params {
    int n_live, batch, walks, max_iter;
    double dlogz;             /* stopping threshold on the remaining log-evidence */
    double scale0;            /* initial step scale (<= 0: 1) */
    double r_ball;            /* intrinsic prior: Delta-e ball radius */
    double dl_min, dl_max;    /* d_L prior range (uniform in volume), Mpc */
    double tc_half;           /* t_c prior half-width, s */
    unsigned long long seed;
    double test_sigma;        /* > 0: diagnostic Gaussian likelihood */
    double test_mu[4];
} mf_ns_params;
typedef struct mf_ns_result {
    double logz, logz_err;    /* log evidence and sqrt(H / n_live) */
    double info;              /* information H (nats) */
    double accept, scale;     /* accepted fraction of walk steps; final scale */
    double wall_ms;           /* wall time of the call */
    long long n_samples;      /* dead + final live points */
    long long n_like;         /* likelihood evaluations */
    int iterations, converged, dim;
} mf_ns_result;
MF_API int mf_nested_sample(mf_handle *h, const mf_ns_params *p, mf_ns_result *res, double *out_v,
                            double *out_lnl, double *out_logwt, int max_out, void *stream);

/* Importance weights of posterior samples (Sec. III A): w_i proportional to
 * exp(logwt_i + log_ratio_i) (log_ratio = log target prior - log sampling
 * prior, or NULL for 1), normalised to sum 1, and the effective sample size
 * N_eff = (sum w)^2 / sum w^2.  Host arrays of n.  MF_E_INVAL if no weight is
 * finite. */
MF_API int mf_reweight(const double *logwt, const double *log_ratio, int n, double *w, double *n_eff);

/* Tuning / instrumentation knobs (host-side, take effect at the next call):
 *   "timing"   : 1 = record CUDA events around the main lnL kernel of each
 *                mf_loglike (read back with mf_query "kernel_ms"), 0 = off.
 *   "pass_max" : widest column pass (16..512, multiple of 16) the tcgen05
 *                forms may use; re-lays out the weights.
 *   "tc_design": tcgen05 kernel design: 0 = thread-block clusters sharing
 *                the RBF tile in shared memory (one launch per run of at
 *                most "tc_chunk" passes); 1 = the RBF tile in tensor
 *                memory, one CTA per column pass (passes <= 192 columns);
 *                -1 (default) = 1 when the columns fit in one such pass,
 *                else 0.  Re-lays out the weights; mf_query "tc_design"
 *                reports the design in use.
 *   "tc_nbs"   : depth (2..6) of the weight-tile ring of the tcgen05
 *                kernels, lowered to what fits in shared memory; 0 (default)
 *                = 4 for the cluster design, 6 for the tensor-memory design
 *                (likewise lowered).
 *   "tc_pair"  : 1 (default) = the 3-term forms pair two query tiles per
 *                cluster when 2 x passes <= 8 (weight tiles multicast to
 *                both) and the larger clusters keep at least 93 % of the
 *                resident CTAs of the single launch (mf_query "tc_paired"
 *                tells the last launch's choice); 0 = never.  Results are
 *                the same either way.
 *   "tc_rot"   : 1 (default) = query tile t of the tcgen05 kernels visits the
 *                node blocks starting at block 11 floor(t / 2) mod n_kb (the
 *                clusters, which start together, then fetch different weight
 *                tiles); 0 = every tile starts at block 0.  Changes the order
 *                of the FP32 sums (results differ in rounding only); batched
 *                launches take each member's setting.
 *   "tc_chunk" : passes per cluster launch at most (2..8); 0 (default) = as
 *                many as one CTA's shared memory stages (4 for the 3-term
 *                forms).  Columns needing more passes run as several
 *                launches, each over a run of passes; results are the same
 *                for every value.
 *   "pass_count": 0 (default) = as few column passes as "pass_max" allows;
 *                1..8 = exactly this many for the tcgen05 forms (contiguous
 *                groups, widest pass minimised; the FP32 form keeps its own
 *                rule); re-lays out the weights, MF_E_INVAL if they do not
 *                fit (the previous layout is kept). */
MF_API int mf_set_option(mf_handle *h, const char *key, double value);

/* Wait for `stream`, then report device-side status accumulated since the
 * last call: MF_OK, or MF_E_RANGE with *n_bad (if non-NULL) = number of
 * out-of-window queries.  Resets the counter. */
MF_API int mf_sync_status(mf_handle *h, void *stream, long long *n_bad);

/* Scalar diagnostics: "cond" (2-norm condition estimate of Phi), "lambda_min",
 * "lambda_max", "cancel" (max over sampled nodes/columns of sum_n |a_n phi_n|
 * / max |F|), "N", "K", "Kdev" (padded device columns), "n_pass" (column
 * passes of the current form), "form", "launches" (kernel launches per
 * mf_loglike), "kernel_ms" (main-kernel time of the last mf_loglike when the
 * "timing" option is on; waits for that kernel). */
MF_API int mf_query(const mf_handle *h, const char *key, double *value);

/* Copy the FP64 weights [(N+P)][K] (a rows, then tail b rows) to host. */
MF_API int mf_get_weights(const mf_handle *h, double *W_host, size_t count);

MF_API void mf_free(mf_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* MF_H */
