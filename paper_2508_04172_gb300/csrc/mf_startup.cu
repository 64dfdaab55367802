// Start-up stage on the GPU in FP64 (not part of the per-query path):
//   * RBF interpolant construction, Eq. (rbfcoeff): Cholesky of the Gaussian
//     matrix Phi, the tail handled through the Schur complement
//     (P^T Phi^-1 P) b = P^T Phi^-1 F, a = Phi^-1 (F - P b)  (so P^T a = 0),
//     plus power / inverse iteration for cond(Phi) and a cancellation probe.
//   * SVD compression of an overlap matrix, Eq. (SVD): dense FP64 SVD of the
//     node-by-time matrix, projection C = Z V.
//   * 4x4 metric eigendecomposition (cyclic Jacobi) for the Delta-e rotation
//     (Sec. II D) and the 10-sample not-a-knot spline operator (Sec. II D).
// The Cholesky factorisation and triangular solves are this library's own
// FP64 kernels (mf_chol.cu); the SVD uses cuSOLVER and its projection GEMM
// cuBLAS; the matrix assembly, Schur step, iterations and small solves are
// kernels here.
#include "mf_internal.cuh"

#include <cublas_v2.h>
#include <cusolverDn.h>

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

struct Libs {
    cusolverDnHandle_t sol = nullptr;
    cublasHandle_t blas = nullptr;
    ~Libs() {
        if (sol) cusolverDnDestroy(sol);
        if (blas) cublasDestroy(blas);
    }
};

template <class T>
struct DevBuf {
    T *p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
    cudaError_t alloc(size_t n) { return cudaMalloc((void **)&p, n * sizeof(T)); }
};

__global__ void assemble_phi64(const double *__restrict__ y, int N, double eps2,
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
    A[(size_t)i * N + j] = exp(-eps2 * r2);
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
                                   int N, int K, double eps2, int stride,
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
            acc += fabs(W[(size_t)n * K + k]) * exp(-eps2 * r2);
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
__global__ void transpose_z(const cuDoubleComplex *__restrict__ Z, int N, int M,
                            cuDoubleComplex *__restrict__ Zc) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    int n = blockIdx.y;
    if (t < M) Zc[(size_t)t * N + n] = Z[(size_t)n * M + t];
}

__global__ void pick_basis(const cuDoubleComplex *__restrict__ VT, int M, int rank,
                           cuDoubleComplex *__restrict__ Vsel) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y;
    if (t < M) Vsel[(size_t)i * M + t] = VT[(size_t)t * M + i];
}

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

int rbf_build(mf_handle *h, const double *F_host, cudaStream_t st) {
    const int N = h->N, K = h->K, P = h->P;
    const int ncols = K + P;
    DevBuf<double> A, B, F, T, b, x, y, nrm, cancel, fmax_d, diag0;
    DevBuf<int> err, cerr;
    MF_CUDA(A.alloc((size_t)N * N));
    MF_CUDA(B.alloc((size_t)N * ncols));
    MF_CUDA(F.alloc((size_t)N * K));
    MF_CUDA(T.alloc((size_t)5 * ncols));
    MF_CUDA(b.alloc((size_t)(P > 0 ? P : 1) * K));
    MF_CUDA(x.alloc(N));
    MF_CUDA(y.alloc(N));
    MF_CUDA(nrm.alloc(1));
    MF_CUDA(err.alloc(1));
    MF_CUDA(cerr.alloc(1));
    MF_CUDA(fmax_d.alloc(1));
    MF_CUDA(diag0.alloc(N));
    MF_CUDA(cudaMemcpyAsync(F.p, F_host, sizeof(double) * (size_t)N * K, cudaMemcpyHostToDevice, st));
    MF_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
    MF_CUDA(cudaMemsetAsync(cerr.p, 0, sizeof(int), st));

    const double eps2 = h->eps * h->eps;
    assemble_phi64<<<dim3((N + 255) / 256, N), 256, 0, st>>>(h->d_nodes64, N, eps2, A.p);
    MF_CUDA(cudaGetLastError());
    // lambda_max by power iteration (before the factorization overwrites Phi)
    fill64<<<(N + 255) / 256, 256, 0, st>>>(x.p, N, 1.0 / std::sqrt((double)N));
    double lmax = 0.0;
    for (int it = 0; it < 60; ++it) {
        matvec64<<<(N + 7) / 8, 256, 0, st>>>(A.p, x.p, N, y.p);
        normalize64<<<1, 256, 0, st>>>(y.p, N, x.p, nrm.p);
    }
    MF_CUDA(cudaGetLastError());
    MF_CUDA(cudaMemcpyAsync(&lmax, nrm.p, sizeof(double), cudaMemcpyDeviceToHost, st));

    // Phi = L L^T (FP64, blocked right-looking); a pivot that is not positive
    // beyond rounding means Phi is numerically singular
    int rc = chol_factor(A.p, N, diag0.p, cerr.p, st);
    if (rc) return rc;
    int hc = 0;
    MF_CUDA(cudaMemcpyAsync(&hc, cerr.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    MF_CUDA(cudaStreamSynchronize(st));
    if (hc != 0) return MF_E_ILLCOND;

    // lambda_min by inverse iteration with the Cholesky factor
    fill64<<<(N + 255) / 256, 256, 0, st>>>(x.p, N, 1.0 / std::sqrt((double)N));
    double inv = 0.0;
    for (int it = 0; it < 40; ++it) {
        MF_CUDA(cudaMemcpyAsync(y.p, x.p, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
        rc = chol_solve(A.p, N, y.p, 1, st);
        if (rc) return rc;
        normalize64<<<1, 256, 0, st>>>(y.p, N, x.p, nrm.p);
    }
    MF_CUDA(cudaGetLastError());
    MF_CUDA(cudaMemcpyAsync(&inv, nrm.p, sizeof(double), cudaMemcpyDeviceToHost, st));

    // solve Phi X = [F | P]
    assemble_rhs<<<dim3((N + 255) / 256, ncols), 256, 0, st>>>(F.p, h->d_nodes64, N, K, P, B.p);
    MF_CUDA(cudaGetLastError());
    rc = chol_solve(A.p, N, B.p, ncols, st);
    if (rc) return rc;
    MF_CUDA(cudaMalloc((void **)&h->d_W64, sizeof(double) * (size_t)(N + P) * K));
    if (P > 0) {
        tail_dots<<<ncols, 256, 0, st>>>(B.p, h->d_nodes64, N, P, T.p, ncols);
        solve_tail<<<(K + 127) / 128, 128, 0, st>>>(T.p, K, P, ncols, b.p, err.p);
        MF_CUDA(cudaGetLastError());
    }
    form_weights<<<dim3((K + 127) / 128, N + P), 128, 0, st>>>(B.p, b.p, N, K, P, h->d_W64);
    MF_CUDA(cudaGetLastError());
    int herr = 0;
    MF_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));

    // cancellation probe on up to 16 nodes
    const int stride = std::max(1, N / 16);
    const int nprobe = (N + stride - 1) / stride;
    MF_CUDA(cancel.alloc(nprobe));
    cancellation_probe<<<nprobe, 256, 0, st>>>(h->d_nodes64, h->d_W64, N, K, eps2, stride,
                                               cancel.p);
    absmax64<<<1, 256, 0, st>>>(F.p, (size_t)N * K, fmax_d.p);
    MF_CUDA(cudaGetLastError());
    std::vector<double> can(nprobe);
    double fm = 0.0;
    MF_CUDA(cudaMemcpyAsync(can.data(), cancel.p, sizeof(double) * nprobe, cudaMemcpyDeviceToHost, st));
    MF_CUDA(cudaMemcpyAsync(&fm, fmax_d.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    MF_CUDA(cudaStreamSynchronize(st));
    if (herr) return MF_E_ILLCOND;
    h->lam_max = lmax;
    h->lam_min = (inv > 0) ? 1.0 / inv : 0.0;
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

int svd_compress(const double *z, int N, int M, int rank, double *coef, double *basis, double *sv,
                 cudaStream_t st) {
    if (N < M) return MF_E_INVAL;   // one row per node; more nodes than samples
    Libs L;
    MF_LIBCALL(cusolverDnCreate(&L.sol));
    MF_LIBCALL(cublasCreate(&L.blas));
    MF_LIBCALL(cusolverDnSetStream(L.sol, st));
    MF_LIBCALL(cublasSetStream(L.blas, st));
    DevBuf<cuDoubleComplex> Z, Zc, VT, Vsel, C, work;
    DevBuf<double> S, rwork;
    DevBuf<int> info;
    MF_CUDA(Z.alloc((size_t)N * M));
    MF_CUDA(Zc.alloc((size_t)N * M));
    MF_CUDA(VT.alloc((size_t)M * M));
    MF_CUDA(Vsel.alloc((size_t)rank * M));
    MF_CUDA(C.alloc((size_t)N * rank));
    MF_CUDA(S.alloc(M));
    MF_CUDA(rwork.alloc(5 * (size_t)M));
    MF_CUDA(info.alloc(1));
    MF_CUDA(cudaMemcpyAsync(Z.p, z, sizeof(cuDoubleComplex) * (size_t)N * M, cudaMemcpyHostToDevice, st));
    transpose_z<<<dim3((M + 255) / 256, N), 256, 0, st>>>(Z.p, N, M, Zc.p);
    MF_CUDA(cudaGetLastError());
    // Z = U S V^H (FP64 Householder bidiagonalisation + QR); only V^H is formed
    int lwork = 0;
    MF_LIBCALL(cusolverDnZgesvd_bufferSize(L.sol, N, M, &lwork));
    MF_CUDA(work.alloc((size_t)lwork + 1));
    signed char jobu = 'N', jobvt = 'A';
    MF_LIBCALL(cusolverDnZgesvd(L.sol, jobu, jobvt, N, M, Zc.p, N, S.p, nullptr, 1, VT.p, M,
                                work.p, lwork, rwork.p, info.p));
    pick_basis<<<dim3((M + 255) / 256, rank), 256, 0, st>>>(VT.p, M, rank, Vsel.p);
    MF_CUDA(cudaGetLastError());
    // C[n][i] = sum_t Z[n][t] conj(u_i[t]):  column-major (rank x N) = U^H T, with
    // T = Z^T (memory [N][M]) and U (M x rank) = basis rows stored [rank][M]
    cuDoubleComplex a1 = make_cuDoubleComplex(1.0, 0.0), a0 = make_cuDoubleComplex(0.0, 0.0);
    MF_LIBCALL(cublasZgemm(L.blas, CUBLAS_OP_C, CUBLAS_OP_N, rank, N, M, &a1, Vsel.p, M, Z.p, M,
                           &a0, C.p, rank));
    int hinfo = 0;
    MF_CUDA(cudaMemcpyAsync(&hinfo, info.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    MF_CUDA(cudaMemcpyAsync(coef, C.p, sizeof(cuDoubleComplex) * (size_t)N * rank, cudaMemcpyDeviceToHost, st));
    MF_CUDA(cudaMemcpyAsync(basis, Vsel.p, sizeof(cuDoubleComplex) * (size_t)rank * M, cudaMemcpyDeviceToHost, st));
    if (sv) MF_CUDA(cudaMemcpyAsync(sv, S.p, sizeof(double) * rank, cudaMemcpyDeviceToHost, st));
    MF_CUDA(cudaStreamSynchronize(st));
    if (hinfo != 0) log_msg("svd: gesvd info = %d (N = %d, M = %d)", hinfo, N, M);
    return hinfo == 0 ? MF_OK : MF_E_CUDA;
}

}  // namespace mf
