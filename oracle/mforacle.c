/*
 * FP64 CPU oracle for the meshfree log-likelihood (TEST INFRASTRUCTURE).
 *
 * Plain, slow, obviously-correct loops that follow the paper's online stage
 * step by step (Sec. II D).  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file; the GPU library shares no
 * code with it.
 *
 *  - RBF interpolant with polynomial tail ........ Eq. (rbfcoeff)
 *  - SVD reconstruction of the overlap series .... Eq. (SVD)
 *  - cubic spline through ~10 samples ............ Sec. II D (online stage)
 *  - spin-weighted spherical harmonics ........... Eq. (h_spherical_harmonic_basis)
 *  - polarisations from negative-m modes ......... Eqs. (hplus_hcross_decomposed1/2)
 *  - frozen antenna patterns + detector delay .... Eq. (projected_h_fd)
 *  - sky-dependent patterns F(alpha, delta, psi, t)
 *    and geocentre-to-detector delays ............ Eqs. (projected_h_td/fd)
 *  - lnL = sum_k <h|d> - 1/2 ||h||^2 ............. Eqs. (logl_basic), (logl_complete)
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int N, K, P;            /* nodes, interpolated columns, tail terms (0,1,5) */
    const double *nodes;    /* [N][4] nodes in the metric eigenbasis            */
    const double *W;        /* [(N+P)][K] RBF weights a (N rows) then tail b    */
    double eps;             /* shape parameter of the radial kernel (rbf below)  */
    int n_det, n_modes, rank, M;
    const int *ell_m;       /* [n_modes][2]                                     */
    const double *basis;    /* [n_det][n_modes][rank][M][2] (re, im)            */
    double t0, dt;          /* time of sample 0 and sample spacing              */
    const double *det;      /* [n_det][3] = F+(psi=0), Fx(psi=0), delay dt_k    */
    double d_ref;           /* reference distance of the node overlaps          */
    const double *R;        /* [4][4] rows = metric eigenvectors                */
    const double *centre;   /* [4] ellipsoid centre                              */
    int stencil;            /* number of spline samples (10)                    */
    /* sky mode (sky != 0): per query, detector k's antenna patterns and delay
     * follow from the source's right ascension and declination (extrinsic
     * columns 5 and 6) and the Earth's rotation angle at t_c + tau_k        */
    int sky;
    const double *dtensor;  /* [n_det][3][3] detector tensors, Earth-fixed frame */
    const double *dpos;     /* [n_det][3] detector positions / c (seconds)       */
    const double *tau;      /* [n_det] epoch of channel k relative to t_c (s)    */
    double gmst0;           /* Greenwich sidereal angle at t_c = 0 (rad)         */
    double omega_e;         /* Earth's sidereal rotation rate (rad/s)            */
    int rbf;                /* radial kernel, s = eps r: 0 Gaussian exp(-s^2),
                             * 1 cubic polyharmonic s^3, 2 multiquadric
                             * sqrt(1 + s^2), 3 inverse multiquadric
                             * 1 / sqrt(1 + s^2)                                 */
} oracle_model;

/* ---------------------------------------------------------------- helpers */
static double fact(int n) {
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= (double)i;
    return f;
}

/* Wigner small-d matrix element d^l_{mp,m}(theta), explicit sum form. */
static double wigner_d(int l, int mp, int m, double theta) {
    double c = cos(0.5 * theta), s = sin(0.5 * theta);
    int kmin = (m - mp > 0) ? m - mp : 0;
    int kmax = (l + m < l - mp) ? l + m : l - mp;
    double pref = sqrt(fact(l + m) * fact(l - m) * fact(l + mp) * fact(l - mp));
    double sum = 0.0;
    for (int k = kmin; k <= kmax; ++k) {
        double den = fact(l + m - k) * fact(k) * fact(l - k - mp) * fact(k - m + mp);
        double sgn = ((k - m + mp) % 2 == 0) ? 1.0 : -1.0;
        sum += sgn * pref / den * pow(c, 2 * l - 2 * k + m - mp) * pow(s, 2 * k - m + mp);
    }
    return sum;
}

/* Spin-weighted spherical harmonic sY_lm(theta, phi)
 *   = (-1)^s sqrt((2l+1)/(4 pi)) d^l_{m,-s}(theta) e^{i m phi}. */
void oracle_sylm(int s, int l, int m, double theta, double phi, double *re, double *im) {
    double sgn = (s % 2 == 0) ? 1.0 : -1.0;
    double mag = sgn * sqrt((2.0 * l + 1.0) / (4.0 * M_PI)) * wigner_d(l, m, -s, theta);
    *re = mag * cos(m * phi);
    *im = mag * sin(m * phi);
}

/* Dense Gaussian elimination with partial pivoting: solves A x = b in place
 * (A is n x n row-major, b has nrhs columns, row-major [n][nrhs]). */
static int gauss_solve(int n, double *A, double *b, int nrhs) {
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(A[r * n + col]) > fabs(A[piv * n + col])) piv = r;
        if (A[piv * n + col] == 0.0) return -1;
        if (piv != col) {
            for (int c = 0; c < n; ++c) { double t = A[col*n+c]; A[col*n+c] = A[piv*n+c]; A[piv*n+c] = t; }
            for (int c = 0; c < nrhs; ++c) { double t = b[col*nrhs+c]; b[col*nrhs+c] = b[piv*nrhs+c]; b[piv*nrhs+c] = t; }
        }
        for (int r = col + 1; r < n; ++r) {
            double f = A[r * n + col] / A[col * n + col];
            if (f == 0.0) continue;
            for (int c = col; c < n; ++c) A[r * n + c] -= f * A[col * n + c];
            for (int c = 0; c < nrhs; ++c) b[r * nrhs + c] -= f * b[col * nrhs + c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        for (int c = 0; c < nrhs; ++c) {
            double acc = b[r * nrhs + c];
            for (int k = r + 1; k < n; ++k) acc -= A[r * n + k] * b[k * nrhs + c];
            b[r * nrhs + c] = acc / A[r * n + r];
        }
    }
    return 0;
}

/* Not-a-knot cubic spline through n >= 4 samples y_0..y_{n-1} at abscissae
 * 0..n-1, evaluated at x in [0, n-1].  Unknowns are the knot second
 * derivatives; interior rows impose C2 continuity, the two end rows make the
 * third derivative continuous across knots 1 and n-2 (not-a-knot). */
double oracle_spline(int n, const double *y, double x) {
    double *A = (double *)calloc((size_t)n * n, sizeof(double));
    double *m2 = (double *)calloc((size_t)n, sizeof(double));
    A[0 * n + 0] = 1.0; A[0 * n + 1] = -2.0; A[0 * n + 2] = 1.0;
    for (int i = 1; i < n - 1; ++i) {
        A[i * n + i - 1] = 1.0; A[i * n + i] = 4.0; A[i * n + i + 1] = 1.0;
        m2[i] = 6.0 * (y[i + 1] - 2.0 * y[i] + y[i - 1]);
    }
    A[(n - 1) * n + n - 3] = 1.0; A[(n - 1) * n + n - 2] = -2.0; A[(n - 1) * n + n - 1] = 1.0;
    gauss_solve(n, A, m2, 1);
    int i = (int)floor(x);
    if (i < 0) i = 0;
    if (i > n - 2) i = n - 2;
    double t = x - i, w = 1.0 - t;
    double v = w * y[i] + t * y[i + 1] + ((w * w * w - w) * m2[i] + (t * t * t - t) * m2[i + 1]) / 6.0;
    free(A); free(m2);
    return v;
}

/* Rotate a sampler-frame point into the metric eigenbasis: x = R (theta - c). */
static void rotate(const oracle_model *m, const double *theta, double *x) {
    for (int i = 0; i < 4; ++i) {
        double acc = 0.0;
        for (int j = 0; j < 4; ++j) acc += m->R[i * 4 + j] * (theta[j] - m->centre[j]);
        x[i] = acc;
    }
}

/* The radial kernel phi(r) at squared distance r2 (Eq. rbfcoeff). */
static double rbf_phi(const oracle_model *m, double r2) {
    double s2 = m->eps * m->eps * r2;
    switch (m->rbf) {
        case 1: return s2 * sqrt(s2);
        case 2: return sqrt(1.0 + s2);
        case 3: return 1.0 / sqrt(1.0 + s2);
        default: return exp(-s2);
    }
}

/* Eq. (rbfcoeff): f_k(x) = sum_n a_nk phi(|x - y_n|) + sum_p b_pk p_p(x). */
static void rbf_eval_point(const oracle_model *m, const double *x, double *f) {
    for (int k = 0; k < m->K; ++k) f[k] = 0.0;
    for (int n = 0; n < m->N; ++n) {
        double r2 = 0.0;
        for (int i = 0; i < 4; ++i) { double d = x[i] - m->nodes[n * 4 + i]; r2 += d * d; }
        double phi = rbf_phi(m, r2);
        const double *w = m->W + (size_t)n * m->K;
        for (int k = 0; k < m->K; ++k) f[k] += phi * w[k];
    }
    double mono[5] = {1.0, x[0], x[1], x[2], x[3]};
    for (int p = 0; p < m->P; ++p) {
        const double *w = m->W + (size_t)(m->N + p) * m->K;
        for (int k = 0; k < m->K; ++k) f[k] += mono[p] * w[k];
    }
}

void oracle_rbf_eval(const oracle_model *m, int Q, const double *x, double *f) {
    #pragma omp parallel for schedule(dynamic, 16)
    for (int q = 0; q < Q; ++q) rbf_eval_point(m, x + (size_t)q * 4, f + (size_t)q * m->K);
}

/* Antenna patterns and delay of channel k for a source at right ascension
 * alpha and declination delta with polarisation angle psi (Eq. projected_h_td
 * at the epoch t_c + tau_k; the long-wavelength detector response):
 *   h = GMST(t_c + tau_k) - alpha is the source's Greenwich hour angle,
 *   w = (cos d cos h, -cos d sin h, sin d) the unit vector towards the source,
 *   X0 = (-sin h, -cos h, 0) and Y0 = (-cos h sin d, sin h sin d, cos d) the
 *   wave-frame axes at psi = 0, X = cos psi X0 + sin psi Y0,
 *   Y = -sin psi X0 + cos psi Y0,
 *   F+ = D : (X X - Y Y),  Fx = D : (X Y + Y X),  D the detector tensor,
 *   dt = -(r . w) with r the detector position over c: the wave reaches a
 *   detector on the source's side of the Earth before the geocentre. */
void oracle_sky_response(const oracle_model *m, int k, double tc, double alpha, double delta,
                         double psi, double *fp, double *fx, double *dt) {
    double h = m->gmst0 + m->omega_e * (tc + m->tau[k]) - alpha;
    double sd = sin(delta), cd = cos(delta), sh = sin(h), ch = cos(h);
    double w[3] = {cd * ch, -cd * sh, sd};
    double X0[3] = {-sh, -ch, 0.0};
    double Y0[3] = {-ch * sd, sh * sd, cd};
    double X[3], Y[3];
    for (int i = 0; i < 3; ++i) {
        X[i] = cos(psi) * X0[i] + sin(psi) * Y0[i];
        Y[i] = -sin(psi) * X0[i] + cos(psi) * Y0[i];
    }
    const double *D = m->dtensor + (size_t)k * 9;
    double p = 0.0, x = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            p += D[i * 3 + j] * (X[i] * X[j] - Y[i] * Y[j]);
            x += D[i * 3 + j] * (X[i] * Y[j] + Y[i] * X[j]);
        }
    const double *r = m->dpos + (size_t)k * 3;
    *fp = p;
    *fx = x;
    *dt = -(r[0] * w[0] + r[1] * w[1] + r[2] * w[2]);
}

/* Per-mode complex amplitude multiplying the negative-m mode in a detector
 * with antenna patterns (F+, Fx) (Eqs. hplus_hcross_decomposed1/2
 * substituted into Eq. projected_h_fd):
 *   h^k = sum_mu c_mu h_{l,-m},
 *   c_mu = (d_ref/d_L) * 1/2 [ (F+ + i Fx) Y_{l,-m} + (-1)^l (F+ - i Fx) conj(Y_{l,m}) ]
 * with Y = -2Y evaluated at (iota, phi_c). */
static void amplitudes_from_f(const oracle_model *m, double fp, double fx, double dL, double cosi,
                              double phic, double *c_re, double *c_im) {
    double iota = acos(cosi);
    double a = m->d_ref / dL;
    for (int mu = 0; mu < m->n_modes; ++mu) {
        int l = m->ell_m[2 * mu], mm = m->ell_m[2 * mu + 1];
        double yn_re, yn_im, yp_re, yp_im;
        oracle_sylm(-2, l, -mm, iota, phic, &yn_re, &yn_im);
        oracle_sylm(-2, l, mm, iota, phic, &yp_re, &yp_im);
        double sl = (l % 2 == 0) ? 1.0 : -1.0;
        /* (F+ + i Fx)(yn) */
        double t1r = fp * yn_re - fx * yn_im, t1i = fp * yn_im + fx * yn_re;
        /* (F+ - i Fx) conj(yp) = (fp - i fx)(yp_re - i yp_im) */
        double t2r = fp * yp_re - fx * yp_im, t2i = -fp * yp_im - fx * yp_re;
        c_re[mu] = 0.5 * a * (t1r + sl * t2r);
        c_im[mu] = 0.5 * a * (t1i + sl * t2i);
    }
}

/* Frozen antenna patterns of detector k (F+0, Fx0 at psi = 0):
 * F+(psi) = F+0 cos 2psi + Fx0 sin 2psi, Fx(psi) = -F+0 sin 2psi + Fx0 cos 2psi. */
void oracle_amplitudes(const oracle_model *m, int k, double dL, double cosi, double psi,
                       double phic, double *c_re, double *c_im) {
    double fp0 = m->det[k * 3 + 0], fx0 = m->det[k * 3 + 1];
    double fp = fp0 * cos(2.0 * psi) + fx0 * sin(2.0 * psi);
    double fx = -fp0 * sin(2.0 * psi) + fx0 * cos(2.0 * psi);
    amplitudes_from_f(m, fp, fx, dL, cosi, phic, c_re, c_im);
}

/* Column of Re(C_i) for (det k, mode mu, coefficient i); Im follows at +rank. */
static int col_coef(const oracle_model *m, int k, int mu, int i) {
    return (k * m->n_modes + mu) * 2 * m->rank + i;
}
static int col_sigma0(const oracle_model *m, int k) {
    return m->n_det * m->n_modes * 2 * m->rank + k * m->n_modes * m->n_modes;
}

/* lnL of one query from its interpolated columns f[K] (node_values order):
 * time interpolation, amplitudes and Eq. logl_complete.  Returns 0, or 1
 * when the spline stencil leaves the sampled time window (then *out = NaN),
 * or 2 when c^H Sigma c is not real to 1e-9 relative (the cross terms were
 * not unpacked into a Hermitian Sigma; *out is still written). */
static int loglike_from_columns(const oracle_model *m, const double *f, const double *ext,
                                double *out) {
    const int nm = m->n_modes, S = m->stencil, half = S / 2 - 1;
    double c_re[8], c_im[8], ys_re[32], ys_im[32];
    double lnl = 0.0;
    int herm_bad = 0;
    for (int k = 0; k < m->n_det; ++k) {
        double fp, fx, dtk;
        if (m->sky) {
            oracle_sky_response(m, k, ext[4], ext[5], ext[6], ext[2], &fp, &fx, &dtk);
        } else {
            double fp0 = m->det[k * 3 + 0], fx0 = m->det[k * 3 + 1];
            fp = fp0 * cos(2.0 * ext[2]) + fx0 * sin(2.0 * ext[2]);
            fx = -fp0 * sin(2.0 * ext[2]) + fx0 * cos(2.0 * ext[2]);
            dtk = m->det[k * 3 + 2];
        }
        double t = (double)ext[4] + dtk;
        double s = (t - m->t0) / m->dt;
        int j = (int)floor(s);
        double u = s - j;
        if (j - half < 0 || j - half + S - 1 > m->M - 1) { *out = NAN; return 1; }
        amplitudes_from_f(m, fp, fx, ext[0], ext[1], ext[3], c_re, c_im);
        /* <h^k | d^k> = Re sum_mu conj(c_mu) z_mu(t_c + dt_k) */
        for (int mu = 0; mu < nm; ++mu) {
            /* Eq. (SVD): z(t_r) = sum_i C_i u_i(t_r) on the S stencil samples */
            for (int r = 0; r < S; ++r) { ys_re[r] = 0.0; ys_im[r] = 0.0; }
            for (int i = 0; i < m->rank; ++i) {
                double cr = f[col_coef(m, k, mu, i)], ci = f[col_coef(m, k, mu, i) + m->rank];
                const double *b = m->basis + ((((size_t)k * nm + mu) * m->rank + i) * m->M) * 2;
                for (int r = 0; r < S; ++r) {
                    double br = b[2 * (j - half + r)], bi = b[2 * (j - half + r) + 1];
                    ys_re[r] += cr * br - ci * bi;
                    ys_im[r] += cr * bi + ci * br;
                }
            }
            double zr = oracle_spline(S, ys_re, half + u);
            double zi = oracle_spline(S, ys_im, half + u);
            lnl += c_re[mu] * zr + c_im[mu] * zi;
        }
        /* ||h^k||^2 = c^H Sigma c with Sigma rebuilt from the packed columns */
        double sr[64], si[64];
        int base = col_sigma0(m, k), p = 0;
        int nup = nm * (nm - 1) / 2;
        for (int a = 0; a < nm; ++a) { sr[a * nm + a] = f[base + a]; si[a * nm + a] = 0.0; }
        for (int a = 0; a < nm; ++a)
            for (int b = a + 1; b < nm; ++b, ++p) {
                sr[a * nm + b] = f[base + nm + p];       si[a * nm + b] = f[base + nm + nup + p];
                sr[b * nm + a] = f[base + nm + p];       si[b * nm + a] = -f[base + nm + nup + p];
            }
        double q_re = 0.0, q_im = 0.0;
        for (int a = 0; a < nm; ++a)
            for (int b = 0; b < nm; ++b) {
                /* conj(c_a) Sigma_ab c_b */
                double xr = sr[a * nm + b] * c_re[b] - si[a * nm + b] * c_im[b];
                double xi = sr[a * nm + b] * c_im[b] + si[a * nm + b] * c_re[b];
                q_re += c_re[a] * xr + c_im[a] * xi;
                q_im += c_re[a] * xi - c_im[a] * xr;
            }
        /* Sigma Hermitian => c^H Sigma c real (Eq. conjugation_symmetry) */
        if (!(fabs(q_im) <= 1e-9 * fabs(q_re) + 1e-300)) herm_bad = 1;
        lnl -= 0.5 * q_re;
    }
    *out = lnl;
    return herm_bad ? 2 : 0;
}

/* lnL for Q queries; intrinsic [Q][4] (sampler frame), extrinsic [Q][E]
 * = (d_L, cos iota, psi, phi_c, t_c) and, in sky mode, (alpha, delta).  Inputs are the FP32 values the GPU
 * receives, promoted to FP64.  Returns the number of out-of-window queries;
 * *n_herm = queries whose c^H Sigma c had an imaginary part. */
int oracle_loglike(const oracle_model *m, int Q, const float *intrinsic, const float *extrinsic,
                   int E, double *out, int nthreads, int *n_herm) {
    int bad = 0, herm = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    #pragma omp parallel reduction(+:bad, herm)
    {
        double *f = (double *)malloc(sizeof(double) * (size_t)m->K);
        #pragma omp for schedule(dynamic, 8)
        for (int q = 0; q < Q; ++q) {
            double th[4], ex[7] = {0, 0, 0, 0, 0, 0, 0};
            for (int i = 0; i < 4; ++i) th[i] = (double)intrinsic[(size_t)q * 4 + i];
            for (int i = 0; i < (E < 7 ? E : 7); ++i) ex[i] = (double)extrinsic[(size_t)q * E + i];
            double x[4];
            rotate(m, th, x);
            rbf_eval_point(m, x, f);
            const int st = loglike_from_columns(m, f, ex, out + q);
            bad += st == 1;
            herm += st == 2;
        }
        free(f);
    }
    *n_herm = herm;
    return bad;
}

/* lnL for Q queries whose interpolated columns are given: F [Q][K] in the
 * node_values column order (e.g. a surrogate's prediction), extrinsic as in
 * oracle_loglike.  Returns the number of out-of-window queries; *n_herm as
 * in oracle_loglike. */
int oracle_loglike_columns(const oracle_model *m, int Q, const double *F, const float *extrinsic,
                           int E, double *out, int nthreads, int *n_herm) {
    int bad = 0, herm = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    #pragma omp parallel for reduction(+:bad, herm) schedule(dynamic, 8)
    for (int q = 0; q < Q; ++q) {
        double ex[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int i = 0; i < (E < 7 ? E : 7); ++i) ex[i] = (double)extrinsic[(size_t)q * E + i];
        const int st = loglike_from_columns(m, F + (size_t)q * m->K, ex, out + q);
        bad += st == 1;
        herm += st == 2;
    }
    *n_herm = herm;
    return bad;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
