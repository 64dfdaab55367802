// Start-up stage on the GPU in FP64 (not part of the per-query path):
//   * RBF interpolant construction, Eq. (rbfcoeff).  Positive definite kernels
//     (Gaussian, IMQ): Cholesky of Phi, the tail handled through the Schur
//     complement (P^T Phi^-1 P) b = P^T Phi^-1 F, a = Phi^-1 (F - P b) (so
//     P^T a = 0).  Conditionally definite kernels (PHS3 of order 2, MQ of
//     order 1, with a tail of at least the matching degree): the null-space
//     method -- Householder Q R = P, a = Q [0; c] with
//     (s Q2^T Phi Q2) c = s Q2^T F positive definite (s = -1 for MQ), then
//     R b = Q1^T (F - Phi a).  Power / inverse iteration give the condition
//     number of the matrix factored; a cancellation probe follows.
//   * 4x4 metric eigendecomposition (cyclic Jacobi) for the Delta-e rotation
//     (Sec. II D) and the 10-sample not-a-knot spline operator (Sec. II D).
// The Cholesky factorisation and triangular solves are this library's own
// FP64 kernels (mf_chol.cu), as is the SVD compression of the overlap
// matrices (mf_svd.cu); the matrix assembly, Schur step, iterations and
// small solves are kernels here.
#include "mf_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

namespace mf {
int chol_factor(double *A, int N, double *diag0, int *err, cudaStream_t st);
int chol_solve(const double *L, int N, double *X, int ncols, cudaStream_t st);
namespace {

template <class T>
struct DevBuf {
    T *p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
    cudaError_t alloc(size_t n) { return cudaMalloc((void **)&p, n * sizeof(T)); }
};

__global__ void assemble_phi64(const double *__restrict__ y, int N, double eps2, int kind,
                               double *__restrict__ A) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y;
    if (j >= N) return;
    double r2 = 0.0;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        double t = y[i * 4 + d] - y[j * 4 + d];
        r2 += t * t;
    }
    A[(size_t)i * N + j] = rbf_phi64(kind, eps2 * r2);
}

// B (column-major N x (K+P)): columns 0..K-1 = F^T rows, K.. = tail monomials.
__global__ void assemble_rhs(const double *__restrict__ F, const double *__restrict__ y, int N,
                             int K, int P, double *__restrict__ B) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    int c = blockIdx.y;
    if (n >= N) return;
    double v;
    if (c < K) v = F[(size_t)n * K + c];
    else {
        int p = c - K;
        v = (p == 0) ? 1.0 : y[n * 4 + p - 1];
    }
    B[(size_t)c * N + n] = v;
}

// T[p][c] = sum_n P[n][p] X[c][n]  (X column-major N x (K+P))
__global__ void tail_dots(const double *__restrict__ X, const double *__restrict__ y, int N,
                          int P, double *__restrict__ T, int ncols) {
    int c = blockIdx.x;
    __shared__ double red[5][256];
    double acc[5] = {0, 0, 0, 0, 0};
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        double x = X[(size_t)c * N + n];
        acc[0] += x;
        for (int p = 1; p < P; ++p) acc[p] += y[n * 4 + p - 1] * x;
    }
    for (int p = 0; p < 5; ++p) red[p][threadIdx.x] = acc[p];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int p = 0; p < 5; ++p) red[p][threadIdx.x] += red[p][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int p = 0; p < P; ++p) T[(size_t)p * ncols + c] = red[p][0];
}

// b[:,k] = S^-1 T[:,k] with S = T[:, K..K+P-1] (P <= 5), Gaussian elimination
// with partial pivoting per column; then W rows N..N+P-1 = b.
__global__ void solve_tail(const double *__restrict__ T, int K, int P, int ncols,
                           double *__restrict__ b, int *__restrict__ err) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    double S[5][6];
    for (int i = 0; i < P; ++i) {
        for (int j = 0; j < P; ++j) S[i][j] = T[(size_t)i * ncols + K + j];
        S[i][P] = T[(size_t)i * ncols + k];
    }
    for (int col = 0; col < P; ++col) {
        int piv = col;
        for (int r = col + 1; r < P; ++r)
            if (fabs(S[r][col]) > fabs(S[piv][col])) piv = r;
        if (S[piv][col] == 0.0) { *err = 1; return; }
        if (piv != col)
            for (int c = 0; c <= P; ++c) { double t = S[col][c]; S[col][c] = S[piv][c]; S[piv][c] = t; }
        for (int r = col + 1; r < P; ++r) {
            double f = S[r][col] / S[col][col];
            for (int c = col; c <= P; ++c) S[r][c] -= f * S[col][c];
        }
    }
    for (int r = P - 1; r >= 0; --r) {
        double acc = S[r][P];
        for (int c = r + 1; c < P; ++c) acc -= S[r][c] * b[(size_t)c * K + k];
        b[(size_t)r * K + k] = acc / S[r][r];
    }
}

// W[n][k] = X_F[k][n] - sum_p X_P[p][n] b[p][k]  (n < N);  W[N+p][k] = b[p][k]
__global__ void form_weights(const double *__restrict__ X, const double *__restrict__ b, int N,
                             int K, int P, double *__restrict__ W) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    int n = blockIdx.y;
    if (k >= K) return;
    if (n < N) {
        double v = X[(size_t)k * N + n];
        for (int p = 0; p < P; ++p) v -= X[(size_t)(K + p) * N + n] * b[(size_t)p * K + k];
        W[(size_t)n * K + k] = v;
    } else {
        W[(size_t)n * K + k] = b[(size_t)(n - N) * K + k];
    }
}

__global__ void matvec64(const double *__restrict__ A, const double *__restrict__ x, int N,
                         double *__restrict__ y) {
    int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    int lane = threadIdx.x & 31;
    if (row >= N) return;
    double acc = 0.0;
    for (int j = lane; j < N; j += 32) acc += A[(size_t)row * N + j] * x[j];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) y[row] = acc;
}

// x <- y / |y|, nrm <- |y|  (single block)
__global__ void normalize64(const double *__restrict__ y, int N, double *__restrict__ x,
                            double *__restrict__ nrm) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) acc += y[i] * y[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    double n = sqrt(red[0]);
    for (int i = threadIdx.x; i < N; i += blockDim.x) x[i] = (n > 0) ? y[i] / n : 0.0;
    if (threadIdx.x == 0) *nrm = n;
}

__global__ void fill64(double *x, int N, double v) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) x[i] = v;
}

// max over sampled nodes i and columns k of sum_n |a_nk| phi(y_i, y_n)
__global__ void cancellation_probe(const double *__restrict__ y, const double *__restrict__ W,
                                   int N, int K, double eps2, int kind, int stride,
                                   double *__restrict__ out) {
    int i = blockIdx.x * stride;
    if (i >= N) return;
    double best = 0.0;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        double acc = 0.0;
        for (int n = 0; n < N; ++n) {
            double r2 = 0.0;
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                double t = y[i * 4 + d] - y[n * 4 + d];
                r2 += t * t;
            }
            acc += fabs(W[(size_t)n * K + k]) * fabs(rbf_phi64(kind, eps2 * r2));
        }
        best = fmax(best, acc);
    }
    __shared__ double red[256];
    red[threadIdx.x] = best;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

// ------------------------------------------ null-space method (PHS3, MQ)
// Householder QR of the tail matrix P [N][np] (monomials 1, y_1..y_4 of the
// nodes), one CTA: P = H_0 .. H_{np-1} [R; 0], H_c = I - tau_c v_c v_c^T,
// v_c zero above row c.  Pw [np][N] workspace; V [np][N]; R [np][np].
__device__ double block_sum64(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    return s;
}

__global__ void __launch_bounds__(1024) tail_qr(const double *__restrict__ y, int N, int np,
                                                double *__restrict__ Pw, double *__restrict__ V,
                                                double *__restrict__ tau, double *__restrict__ R) {
    __shared__ double red[32];
    for (int i = threadIdx.x; i < N; i += blockDim.x)
        for (int p = 0; p < np; ++p) Pw[(size_t)p * N + i] = p == 0 ? 1.0 : y[i * 4 + p - 1];
    for (int i = threadIdx.x; i < np * np; i += blockDim.x) R[i] = 0.0;
    __syncthreads();
    for (int c = 0; c < np; ++c) {
        double *x = Pw + (size_t)c * N, *v = V + (size_t)c * N;
        double s = 0.0;
        for (int i = c + threadIdx.x; i < N; i += blockDim.x) s += x[i] * x[i];
        const double nrm = sqrt(block_sum64(s, red));
        const double x0 = x[c];
        const double alpha = x0 >= 0.0 ? -nrm : nrm;
        for (int i = threadIdx.x; i < N; i += blockDim.x) v[i] = i < c ? 0.0 : (i == c ? x0 - alpha : x[i]);
        __syncthreads();
        double t = 0.0;
        for (int i = c + threadIdx.x; i < N; i += blockDim.x) t += v[i] * v[i];
        const double vtv = block_sum64(t, red);
        const double tc = vtv > 0.0 ? 2.0 / vtv : 0.0;
        if (threadIdx.x == 0) {
            tau[c] = tc;
            R[c * np + c] = alpha;
        }
        for (int j = c + 1; j < np; ++j) {
            double *z = Pw + (size_t)j * N;
            double d = 0.0;
            for (int i = c + threadIdx.x; i < N; i += blockDim.x) d += v[i] * z[i];
            d = block_sum64(d, red) * tc;
            for (int i = c + threadIdx.x; i < N; i += blockDim.x) z[i] -= d * v[i];
            __syncthreads();
            if (threadIdx.x == 0) R[c * np + j] = z[c];
        }
        __syncthreads();
    }
}

// out = v . w (one CTA)
__global__ void dot64(const double *__restrict__ v, const double *__restrict__ w, int N, double *__restrict__ out) {
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) s += v[i] * w[i];
    s = block_sum64(s, red);
    if (threadIdx.x == 0) *out = s;
}

// X <- H X H for symmetric X [N][N], H = I - tau v v^T, given w = X v and
// c = v . w:  X - tau (v w^T + w v^T) + tau^2 c v v^T
__global__ void sym_reflect(double *__restrict__ X, int N, const double *__restrict__ v, const double *__restrict__ w,
                            const double *__restrict__ tau, const double *__restrict__ c) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= N) return;
    const double t = *tau;
    X[(size_t)i * N + j] += -t * (v[i] * w[j] + w[i] * v[j]) + t * t * (*c) * v[i] * v[j];
}

// G <- H G for the K columns of G (column-major, column k at G + k N); one
// CTA per column
__global__ void reflect_cols(double *__restrict__ G, int N, const double *__restrict__ v,
                             const double *__restrict__ tau) {
    __shared__ double red[32];
    double *g = G + (size_t)blockIdx.x * N;
    double s = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) s += v[i] * g[i];
    const double u = block_sum64(s, red) * (*tau);
    for (int i = threadIdx.x; i < N; i += blockDim.x) g[i] -= u * v[i];
}

// B [n2][n2] = sgn * X[np:, np:]   (X [N][N] row-major)
__global__ void extract_block(const double *__restrict__ X, int N, int np, double sgn, double *__restrict__ B) {
    const int n2 = N - np;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= n2) return;
    B[(size_t)i * n2 + j] = sgn * X[(size_t)(i + np) * N + np + j];
}

// C [K][n2] (column-major) = sgn * G[np:, :]   (G column-major N x K)
__global__ void extract_rows(const double *__restrict__ G, int N, int np, double sgn, double *__restrict__ C) {
    const int n2 = N - np;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (i >= n2) return;
    C[(size_t)k * n2 + i] = sgn * G[(size_t)k * N + np + i];
}

// A [K][N] (column-major) = [0 (np rows); C]
__global__ void embed_rows(const double *__restrict__ C, int N, int np, double *__restrict__ A) {
    const int n2 = N - np;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (i >= N) return;
    A[(size_t)k * N + i] = i < np ? 0.0 : C[(size_t)k * n2 + i - np];
}

// T[p][k] = G[k][p] - sum_j X[p][np + j] C[k][j]   (p < np; one CTA per (k, p))
__global__ void tail_rhs(const double *__restrict__ X, const double *__restrict__ G, const double *__restrict__ C,
                         int N, int np, int K, double *__restrict__ T) {
    __shared__ double red[32];
    const int k = blockIdx.x, p = blockIdx.y;
    const int n2 = N - np;
    double s = 0.0;
    for (int j = threadIdx.x; j < n2; j += blockDim.x) s += X[(size_t)p * N + np + j] * C[(size_t)k * n2 + j];
    s = block_sum64(s, red);
    if (threadIdx.x == 0) T[(size_t)p * K + k] = G[(size_t)k * N + p] - s;
}

// b = R^-1 T (R upper triangular np x np), column by column; W rows:
// W[n][k] = A[k][n] (n < N), W[N + p][k] = b[p][k]
__global__ void tail_back_solve(const double *__restrict__ R, int np, const double *__restrict__ T, int K,
                                double *__restrict__ W, int N) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    double b[5];
    for (int r = np - 1; r >= 0; --r) {
        double acc = T[(size_t)r * K + k];
        for (int c = r + 1; c < np; ++c) acc -= R[r * np + c] * b[c];
        b[r] = acc / R[r * np + r];
        W[(size_t)(N + r) * K + k] = b[r];
    }
}

__global__ void transpose_weights(const double *__restrict__ A, int N, int K, double *__restrict__ W) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    if (k >= K) return;
    W[(size_t)n * K + k] = A[(size_t)k * N + n];
}

__global__ void absmax64(const double *__restrict__ x, size_t n, double *__restrict__ out) {
    __shared__ double red[256];
    double m = 0.0;
    for (size_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(x[i]));
    red[threadIdx.x] = m;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// Cyclic Jacobi on a symmetric 4x4 (FP64, one thread); rows of R = eigenvectors
// sorted by ascending eigenvalue, each with its largest-|.| entry positive.
__global__ void jacobi4(const double *__restrict__ Ain, double *__restrict__ R,
                        double *__restrict__ lam) {
    double A[4][4], V[4][4];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            A[i][j] = 0.5 * (Ain[i * 4 + j] + Ain[j * 4 + i]);
            V[i][j] = (i == j) ? 1.0 : 0.0;
        }
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) {
                tot += A[i][j] * A[i][j];
                if (i != j) off += A[i][j] * A[i][j];
            }
        if (off <= 1e-32 * tot) break;
        for (int p = 0; p < 3; ++p)
            for (int q = p + 1; q < 4; ++q) {
                if (A[p][q] == 0.0) continue;
                double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < 4; ++k) {   // A <- J^T A J
                    double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 4; ++k) {
                    double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 4; ++k) {   // V <- V J (columns = eigenvectors)
                    double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - s * vkq;
                    V[k][q] = s * vkp + c * vkq;
                }
            }
    }
    int ord[4] = {0, 1, 2, 3};
    for (int i = 0; i < 4; ++i)
        for (int j = i + 1; j < 4; ++j)
            if (A[ord[j]][ord[j]] < A[ord[i]][ord[i]]) { int t = ord[i]; ord[i] = ord[j]; ord[j] = t; }
    for (int r = 0; r < 4; ++r) {
        int c = ord[r];
        int big = 0;
        for (int k = 1; k < 4; ++k)
            if (fabs(V[k][c]) > fabs(V[big][c])) big = k;
        double sg = V[big][c] < 0 ? -1.0 : 1.0;
        for (int k = 0; k < 4; ++k) R[r * 4 + k] = sg * V[k][c];
        lam[r] = A[c][c];
    }
}

// Rows 4 and 5 of G = A^-1 Rm, the map from 10 samples to the knot second
// derivatives of the not-a-knot cubic spline (unit spacing): interior rows
// m_{i-1} + 4 m_i + m_{i+1} = 6 (y_{i-1} - 2 y_i + y_{i+1}); end rows
// m_0 - 2 m_1 + m_2 = 0 and m_7 - 2 m_8 + m_9 = 0 (continuous third derivative).
__global__ void spline_operator(double *__restrict__ G45) {
    const int n = kStencil;
    double A[kStencil][2 * kStencil];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < 2 * n; ++j) A[i][j] = 0.0;
    A[0][0] = 1.0; A[0][1] = -2.0; A[0][2] = 1.0;
    A[n - 1][n - 3] = 1.0; A[n - 1][n - 2] = -2.0; A[n - 1][n - 1] = 1.0;
    for (int i = 1; i < n - 1; ++i) {
        A[i][i - 1] = 1.0; A[i][i] = 4.0; A[i][i + 1] = 1.0;
        A[i][n + i - 1] = 6.0; A[i][n + i] = -12.0; A[i][n + i + 1] = 6.0;
    }
    for (int c = 0; c < n; ++c) {     // Gauss-Jordan with partial pivoting
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        for (int j = 0; j < 2 * n; ++j) { double t = A[c][j]; A[c][j] = A[piv][j]; A[piv][j] = t; }
        double d = A[c][c];
        for (int j = 0; j < 2 * n; ++j) A[c][j] /= d;
        for (int r = 0; r < n; ++r)
            if (r != c) {
                double f = A[r][c];
                for (int j = 0; j < 2 * n; ++j) A[r][j] -= f * A[c][j];
            }
    }
    for (int j = 0; j < n; ++j) {
        G45[j] = A[kStencilLo][n + j];
        G45[n + j] = A[kStencilLo + 1][n + j];
    }
}

// SVD helpers: Zc = column-major copy of Z (N x M); basis rows from V^H.
// Cubic coefficients of the 10-sample not-a-knot spline on [j, j+1]:
//   S(u) = y4 + u (y5 - y4 - m4/3 - m5/6) + u^2 m4/2 + u^3 (m5 - m4)/6,
// m4, m5 = knot second derivatives (rows 4, 5 of the spline operator) of the
// samples y_r = u_i(j - 4 + r).  Entries whose window leaves [0, M) are zero.
struct Stencil45 { double g4[kStencil], g5[kStencil]; };

__global__ void cubic_table(const double2 *__restrict__ basis, int nblk, int rank, int M,
                            Stencil45 g, float4 *__restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    int b = blockIdx.z;
    if (i >= rank || b >= nblk) return;
    float4 *o = out + (((size_t)b * M + j) * rank + i) * 2;
    int s0 = j - kStencilLo;
    if (s0 < 0 || s0 + kStencil > M) {
        o[0] = make_float4(0.f, 0.f, 0.f, 0.f);
        o[1] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const double2 *y = basis + ((size_t)b * rank + i) * M + s0;
    double m4r = 0, m4i = 0, m5r = 0, m5i = 0;
    for (int r = 0; r < kStencil; ++r) {
        double2 v = y[r];
        m4r += g.g4[r] * v.x; m4i += g.g4[r] * v.y;
        m5r += g.g5[r] * v.x; m5i += g.g5[r] * v.y;
    }
    double2 y4 = y[kStencilLo], y5 = y[kStencilLo + 1];
    o[0] = make_float4((float)y4.x, (float)y4.y,
                       (float)(y5.x - y4.x - m4r / 3.0 - m5r / 6.0),
                       (float)(y5.y - y4.y - m4i / 3.0 - m5i / 6.0));
    o[1] = make_float4((float)(0.5 * m4r), (float)(0.5 * m4i), (float)((m5r - m4r) / 6.0),
                       (float)((m5i - m4i) / 6.0));
}

}  // namespace

int build_cubic_table(mf_handle *h, const double *basis_host) {
    const int nblk = h->n_det * h->n_modes, rank = h->rank, M = h->M;
    DevBuf<double2> b;
    size_t n = (size_t)nblk * rank * M;
    MF_CUDA(b.alloc(n));
    MF_CUDA(cudaMemcpy(b.p, basis_host, sizeof(double2) * n, cudaMemcpyHostToDevice));
    if (h->d_cubic) cudaFree(h->d_cubic);
    h->d_cubic = nullptr;
    MF_CUDA(cudaMalloc((void **)&h->d_cubic, sizeof(float4) * 2 * n));
    Stencil45 g;
    for (int r = 0; r < kStencil; ++r) { g.g4[r] = h->G4[r]; g.g5[r] = h->G5[r]; }
    dim3 grid((rank + 31) / 32, M, nblk);
    cubic_table<<<grid, 32>>>(b.p, nblk, rank, M, g, h->d_cubic);
    MF_CUDA(cudaGetLastError());
    MF_CUDA(cudaDeviceSynchronize());
    return MF_OK;
}

void log_msg(const char *fmt, ...) {
    static const bool on = getenv("MF_LOG") != nullptr;
    if (!on) return;
    va_list ap;
    va_start(ap, fmt);
    fprintf(stderr, "[mf] ");
    vfprintf(stderr, fmt, ap);
    fprintf(stderr, "\n");
    va_end(ap);
}

int cuda_status(cudaError_t e) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return MF_E_NOMEM;
    }
    return MF_E_CUDA;
}

int compute_stencil(mf_handle *h) {
    DevBuf<double> g;
    MF_CUDA(g.alloc(2 * kStencil));
    spline_operator<<<1, 1>>>(g.p);
    MF_CUDA(cudaGetLastError());
    double G[2 * kStencil];
    MF_CUDA(cudaMemcpy(G, g.p, sizeof(G), cudaMemcpyDeviceToHost));
    for (int j = 0; j < kStencil; ++j) {
        h->G4[j] = G[j];
        h->G5[j] = G[kStencil + j];
    }
    h->have_stencil = true;
    return MF_OK;
}

// Largest eigenvalue (power iteration), Cholesky factor in place, smallest
// eigenvalue (inverse iteration with the factor) of the SPD matrix A [n][n].
// MF_E_ILLCOND when a pivot is not positive beyond rounding.
static int factor_estimate(double *A, int n, double *lmax_out, double *lmin_out, cudaStream_t st) {
    DevBuf<double> x, y, nrm, diag0;
    DevBuf<int> cerr;
    MF_CUDA(x.alloc(n));
    MF_CUDA(y.alloc(n));
    MF_CUDA(nrm.alloc(1));
    MF_CUDA(diag0.alloc(n));
    MF_CUDA(cerr.alloc(1));
    MF_CUDA(cudaMemsetAsync(cerr.p, 0, sizeof(int), st));
    fill64<<<(n + 255) / 256, 256, 0, st>>>(x.p, n, 1.0 / std::sqrt((double)n));
    double lmax = 0.0;
    for (int it = 0; it < 60; ++it) {
        matvec64<<<(n + 7) / 8, 256, 0, st>>>(A, x.p, n, y.p);
        normalize64<<<1, 256, 0, st>>>(y.p, n, x.p, nrm.p);
    }
    MF_CUDA(cudaGetLastError());
    MF_CUDA(cudaMemcpyAsync(&lmax, nrm.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    // A = L L^T (FP64, blocked right-looking)
    int rc = chol_factor(A, n, diag0.p, cerr.p, st);
    if (rc) return rc;
    int hc = 0;
    MF_CUDA(cudaMemcpyAsync(&hc, cerr.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    MF_CUDA(cudaStreamSynchronize(st));
    if (hc != 0) return MF_E_ILLCOND;
    fill64<<<(n + 255) / 256, 256, 0, st>>>(x.p, n, 1.0 / std::sqrt((double)n));
    double inv = 0.0;
    for (int it = 0; it < 40; ++it) {
        MF_CUDA(cudaMemcpyAsync(y.p, x.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        rc = chol_solve(A, n, y.p, 1, st);
        if (rc) return rc;
        normalize64<<<1, 256, 0, st>>>(y.p, n, x.p, nrm.p);
    }
    MF_CUDA(cudaGetLastError());
    MF_CUDA(cudaMemcpyAsync(&inv, nrm.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    MF_CUDA(cudaStreamSynchronize(st));
    *lmax_out = lmax;
    *lmin_out = (inv > 0) ? 1.0 / inv : 0.0;
    return MF_OK;
}

// Positive definite kernels: Cholesky of Phi and the tail's Schur complement.
static int rbf_build_pd(mf_handle *h, double *A, const double *F, cudaStream_t st, double *lmax, double *lmin) {
    const int N = h->N, K = h->K, P = h->P;
    const int ncols = K + P;
    DevBuf<double> B, T, b;
    DevBuf<int> err;
    MF_CUDA(B.alloc((size_t)N * ncols));
    MF_CUDA(T.alloc((size_t)5 * ncols));
    MF_CUDA(b.alloc((size_t)(P > 0 ? P : 1) * K));
    MF_CUDA(err.alloc(1));
    MF_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
    int rc = factor_estimate(A, N, lmax, lmin, st);
    if (rc) return rc;
    // solve Phi X = [F | P]
    assemble_rhs<<<dim3((N + 255) / 256, ncols), 256, 0, st>>>(F, h->d_nodes64, N, K, P, B.p);
    MF_CUDA(cudaGetLastError());
    rc = chol_solve(A, N, B.p, ncols, st);
    if (rc) return rc;
    if (P > 0) {
        tail_dots<<<ncols, 256, 0, st>>>(B.p, h->d_nodes64, N, P, T.p, ncols);
        solve_tail<<<(K + 127) / 128, 128, 0, st>>>(T.p, K, P, ncols, b.p, err.p);
        MF_CUDA(cudaGetLastError());
    }
    form_weights<<<dim3((K + 127) / 128, N + P), 128, 0, st>>>(B.p, b.p, N, K, P, h->d_W64);
    MF_CUDA(cudaGetLastError());
    int herr = 0;
    MF_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    MF_CUDA(cudaStreamSynchronize(st));
    return herr ? MF_E_ILLCOND : MF_OK;
}

// Conditionally definite kernels (PHS3: s = +1, MQ: s = -1): the null-space
// method.  With Q R = P (Householder) and a = Q [0; c], the saddle system
// becomes (s X22) c = s G2 and R b = G1 - X12 c, where X = Q^T Phi Q and
// G = Q^T F; s X22 is positive definite for a kernel of order <= tail
// degree + 1 (Micchelli).
static int rbf_build_cpd(mf_handle *h, double *A, const double *F, cudaStream_t st, double *lmax, double *lmin) {
    const int N = h->N, K = h->K, np = h->P, n2 = N - np;
    const double sgn = h->rbf == MF_RBF_MQ ? -1.0 : 1.0;
    DevBuf<double> Pw, V, tau, R, w, c, B2, G, C2, Af, T;
    MF_CUDA(Pw.alloc((size_t)np * N));
    MF_CUDA(V.alloc((size_t)np * N));
    MF_CUDA(tau.alloc(np));
    MF_CUDA(R.alloc((size_t)np * np));
    MF_CUDA(w.alloc(N));
    MF_CUDA(c.alloc(1));
    MF_CUDA(B2.alloc((size_t)n2 * n2));
    MF_CUDA(G.alloc((size_t)N * K));
    MF_CUDA(C2.alloc((size_t)n2 * K));
    MF_CUDA(Af.alloc((size_t)N * K));
    MF_CUDA(T.alloc((size_t)np * K));
    tail_qr<<<1, 1024, 0, st>>>(h->d_nodes64, N, np, Pw.p, V.p, tau.p, R.p);
    MF_CUDA(cudaGetLastError());
    std::vector<double> Rh((size_t)np * np);
    MF_CUDA(cudaMemcpyAsync(Rh.data(), R.p, sizeof(double) * np * np, cudaMemcpyDeviceToHost, st));
    MF_CUDA(cudaStreamSynchronize(st));
    double rmax = 0.0;
    for (int i = 0; i < np; ++i) rmax = std::max(rmax, std::fabs(Rh[i * np + i]));
    for (int i = 0; i < np; ++i)
        if (!(std::fabs(Rh[i * np + i]) > 1e-12 * rmax)) return MF_E_ILLCOND;   // the tail is not unisolvent
    // X = Q^T Phi Q, one reflector at a time
    for (int i = 0; i < np; ++i) {
        const double *v = V.p + (size_t)i * N;
        matvec64<<<(N + 7) / 8, 256, 0, st>>>(A, v, N, w.p);
        dot64<<<1, 256, 0, st>>>(v, w.p, N, c.p);
        sym_reflect<<<dim3((N + 255) / 256, N), 256, 0, st>>>(A, N, v, w.p, tau.p + i, c.p);
    }
    extract_block<<<dim3((n2 + 255) / 256, n2), 256, 0, st>>>(A, N, np, sgn, B2.p);
    MF_CUDA(cudaGetLastError());
    int rc = factor_estimate(B2.p, n2, lmax, lmin, st);
    if (rc) return rc;
    // G = Q^T F (column-major N x K)
    assemble_rhs<<<dim3((N + 255) / 256, K), 256, 0, st>>>(F, h->d_nodes64, N, K, 0, G.p);
    for (int i = 0; i < np; ++i) reflect_cols<<<K, 256, 0, st>>>(G.p, N, V.p + (size_t)i * N, tau.p + i);
    extract_rows<<<dim3((n2 + 255) / 256, K), 256, 0, st>>>(G.p, N, np, sgn, C2.p);
    MF_CUDA(cudaGetLastError());
    rc = chol_solve(B2.p, n2, C2.p, K, st);
    if (rc) return rc;
    // a = Q [0; c]
    embed_rows<<<dim3((N + 255) / 256, K), 256, 0, st>>>(C2.p, N, np, Af.p);
    for (int i = np - 1; i >= 0; --i) reflect_cols<<<K, 256, 0, st>>>(Af.p, N, V.p + (size_t)i * N, tau.p + i);
    // R b = G1 - X12 c
    tail_rhs<<<dim3(K, np), 256, 0, st>>>(A, G.p, C2.p, N, np, K, T.p);
    transpose_weights<<<dim3((K + 127) / 128, N), 128, 0, st>>>(Af.p, N, K, h->d_W64);
    tail_back_solve<<<(K + 127) / 128, 128, 0, st>>>(R.p, np, T.p, K, h->d_W64, N);
    MF_CUDA(cudaGetLastError());
    MF_CUDA(cudaStreamSynchronize(st));
    return MF_OK;
}

int rbf_build(mf_handle *h, const double *F_host, cudaStream_t st) {
    const int N = h->N, K = h->K, P = h->P;
    const int kind = (int)h->rbf;
    DevBuf<double> A, F, cancel, fmax_d;
    MF_CUDA(A.alloc((size_t)N * N));
    MF_CUDA(F.alloc((size_t)N * K));
    MF_CUDA(fmax_d.alloc(1));
    MF_CUDA(cudaMemcpyAsync(F.p, F_host, sizeof(double) * (size_t)N * K, cudaMemcpyHostToDevice, st));
    const double eps2 = h->eps * h->eps;
    assemble_phi64<<<dim3((N + 255) / 256, N), 256, 0, st>>>(h->d_nodes64, N, eps2, kind, A.p);
    MF_CUDA(cudaGetLastError());
    MF_CUDA(cudaMalloc((void **)&h->d_W64, sizeof(double) * (size_t)(N + P) * K));
    double lmax = 0.0, lmin = 0.0;
    const bool pd = h->rbf == MF_RBF_GAUSSIAN || h->rbf == MF_RBF_IMQ;
    int rc = pd ? rbf_build_pd(h, A.p, F.p, st, &lmax, &lmin) : rbf_build_cpd(h, A.p, F.p, st, &lmax, &lmin);
    if (rc) return rc;

    // cancellation probe on up to 16 nodes
    const int stride = std::max(1, N / 16);
    const int nprobe = (N + stride - 1) / stride;
    MF_CUDA(cancel.alloc(nprobe));
    cancellation_probe<<<nprobe, 256, 0, st>>>(h->d_nodes64, h->d_W64, N, K, eps2, kind, stride, cancel.p);
    absmax64<<<1, 256, 0, st>>>(F.p, (size_t)N * K, fmax_d.p);
    MF_CUDA(cudaGetLastError());
    std::vector<double> can(nprobe);
    double fm = 0.0;
    MF_CUDA(cudaMemcpyAsync(can.data(), cancel.p, sizeof(double) * nprobe, cudaMemcpyDeviceToHost, st));
    MF_CUDA(cudaMemcpyAsync(&fm, fmax_d.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    MF_CUDA(cudaStreamSynchronize(st));
    h->lam_max = lmax;
    h->lam_min = lmin;
    h->cond = (h->lam_min > 0) ? h->lam_max / h->lam_min : INFINITY;
    double cm = 0.0;
    for (double v : can) cm = std::max(cm, v);
    h->cancel = (fm > 0) ? cm / fm : 0.0;
    return MF_OK;
}

int metric_eig(const double *metric, double *R_out) {
    DevBuf<double> a, r, l;
    MF_CUDA(a.alloc(16));
    MF_CUDA(r.alloc(16));
    MF_CUDA(l.alloc(4));
    MF_CUDA(cudaMemcpy(a.p, metric, 16 * sizeof(double), cudaMemcpyHostToDevice));
    jacobi4<<<1, 1>>>(a.p, r.p, l.p);
    MF_CUDA(cudaGetLastError());
    double lam[4];
    MF_CUDA(cudaMemcpy(R_out, r.p, 16 * sizeof(double), cudaMemcpyDeviceToHost));
    MF_CUDA(cudaMemcpy(lam, l.p, 4 * sizeof(double), cudaMemcpyDeviceToHost));
    for (int i = 0; i < 4; ++i)
        if (!(lam[i] > 0)) return MF_E_INVAL;   // metric must be positive definite
    return MF_OK;
}

}  // namespace mf
