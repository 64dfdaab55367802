// FP64 Cholesky factorisation and triangular solves of the RBF interpolation
// matrix (Eq. rbfcoeff: Phi is symmetric positive definite for the Gaussian
// kernel), written for the start-up stage on the GPU.
//
// Factorisation: blocked, right-looking, lower.  For each panel of kNb
// columns starting at k0:
//   chol_diag    one CTA factors the kNb x kNb diagonal block in shared
//                memory (unblocked Cholesky) and flags a pivot that is not
//                positive beyond rounding (d <= kPivTol * Phi_jj before
//                factoring: Phi numerically singular -> MF_E_ILLCOND);
//   chol_panel   one warp per row below the block: L_ik = A_ik L_kk^-T by
//                forward substitution against L_kk in shared memory;
//   chol_update  the trailing lower triangle, 64 x 64 tiles:
//                A_ij -= L_i,panel L_j,panel^T (i >= j).
// Solves (X column-major [ncols][N]): L Y = B then L^T X = Y, each as
// diagonal-block substitutions (one thread per right-hand side) followed by
// a 64 x 64-tiled update of the remaining rows.
//
// A is row-major N x N; the factor overwrites its lower triangle (the upper
// triangle is left as assembled and never read).
#include "mf_internal.cuh"

#include <algorithm>
#include <cmath>

namespace mf {
namespace {

constexpr int kNb = 32;           // panel width
constexpr int kTileR = 64;        // update tile (rows x columns)
constexpr double kPivTol = 1e-14; // relative pivot floor

// ---------------------------------------------------------------- factor
__global__ void __launch_bounds__(256) chol_diag(double *__restrict__ A, int N, int k0,
                                                 const double *__restrict__ diag0, int *__restrict__ err) {
    __shared__ double L[kNb][kNb + 1];
    const int nb = min(kNb, N - k0);
    for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
        const int i = t / nb, j = t % nb;
        L[i][j] = (j <= i) ? A[(size_t)(k0 + i) * N + k0 + j] : 0.0;
    }
    __syncthreads();
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        if (threadIdx.x == 0) {
            const double d = L[j][j];
            if (!(d > kPivTol * diag0[k0 + j])) {   // also catches NaN
                bad = 1;
                L[j][j] = 1.0;
            } else {
                L[j][j] = sqrt(d);
            }
        }
        __syncthreads();
        const double djj = L[j][j];
        for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) L[i][j] /= djj;
        __syncthreads();
        // trailing update inside the block: L[i][c] -= L[i][j] L[c][j], j < c <= i
        for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
            const int i = t / nb, c = t % nb;
            if (c > j && c <= i) L[i][c] -= L[i][j] * L[c][j];
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
        const int i = t / nb, j = t % nb;
        if (j <= i) A[(size_t)(k0 + i) * N + k0 + j] = L[i][j];
    }
    if (threadIdx.x == 0 && bad) atomicOr(err, 1);
}

// rows k0 + nb .. N-1: row i of the panel solves L_kk x = a_i (x = L_ik^T)
__global__ void __launch_bounds__(256) chol_panel(double *__restrict__ A, int N, int k0) {
    __shared__ double L[kNb][kNb + 1];
    const int nb = kNb;   // only called when a full panel remains below
    for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
        const int i = t / nb, j = t % nb;
        L[i][j] = (j <= i) ? A[(size_t)(k0 + i) * N + k0 + j] : 0.0;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int row = k0 + nb + blockIdx.x * 8 + warp; row < N; row += gridDim.x * 8) {
        double *a = A + (size_t)row * N + k0;
        double v = a[lane];                       // kNb == 32: one column per lane
        for (int j = 0; j < nb; ++j) {
            const double xj = __shfl_sync(0xffffffffu, v, j) / L[j][j];
            if (lane == j) v = xj;
            if (lane > j) v -= xj * L[lane][j];
        }
        a[lane] = v;
    }
}

// Map a linear tile index to (ti, tj) with ti >= tj (lower-triangle tiles).
__device__ __forceinline__ void tri_index(int t, int &ti, int &tj) {
    int i = (int)floor((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((i + 1) * (i + 2) / 2 <= t) ++i;
    while (i * (i + 1) / 2 > t) --i;
    ti = i;
    tj = t - i * (i + 1) / 2;
}

// A[i][j] -= sum_m L[i][k0+m] L[j][k0+m] for the lower triangle of the
// trailing matrix (rows and columns from s = k0 + kNb).
__global__ void __launch_bounds__(256) chol_update(double *__restrict__ A, int N, int k0) {
    __shared__ double Li[kTileR][kNb + 1], Lj[kTileR][kNb + 1];
    const int s = k0 + kNb;
    int ti, tj;
    tri_index(blockIdx.x, ti, tj);
    const int i0 = s + ti * kTileR, j0 = s + tj * kTileR;
    for (int t = threadIdx.x; t < kTileR * kNb; t += blockDim.x) {
        const int r = t / kNb, m = t % kNb;
        Li[r][m] = (i0 + r < N) ? A[(size_t)(i0 + r) * N + k0 + m] : 0.0;
        Lj[r][m] = (j0 + r < N) ? A[(size_t)(j0 + r) * N + k0 + m] : 0.0;
    }
    __syncthreads();
    const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;   // 4 x 4 outputs each
    double acc[4][4] = {};
#pragma unroll 4
    for (int m = 0; m < kNb; ++m) {
        double a[4], b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            a[u] = Li[tr + 16 * u][m];
            b[u] = Lj[tc + 16 * u][m];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int i = i0 + tr + 16 * u, j = j0 + tc + 16 * v;
            if (i < N && j <= i) A[(size_t)i * N + j] -= acc[u][v];
        }
}

// ----------------------------------------------------------------- solves
// Forward substitution on the diagonal block [k0, k0+nb) for every column c:
// X[c][k0+j] = (X[c][k0+j] - sum_{m<j} L[k0+j][k0+m] X[c][k0+m]) / L_jj.
__global__ void __launch_bounds__(128) trsv_fwd_diag(const double *__restrict__ A, int N, int k0,
                                                     double *__restrict__ X, int ncols) {
    __shared__ double L[kNb][kNb + 1];
    const int nb = min(kNb, N - k0);
    for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
        const int i = t / nb, j = t % nb;
        L[i][j] = (j <= i) ? A[(size_t)(k0 + i) * N + k0 + j] : 0.0;
    }
    __syncthreads();
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncols) return;
    double *x = X + (size_t)c * N + k0;
    double v[kNb];
#pragma unroll
    for (int j = 0; j < kNb; ++j) v[j] = (j < nb) ? x[j] : 0.0;
#pragma unroll
    for (int j = 0; j < kNb; ++j) {
        if (j < nb) {
            double a = v[j];
#pragma unroll
            for (int m = 0; m < j; ++m) a -= L[j][m] * v[m];
            v[j] = a / L[j][j];
        }
    }
#pragma unroll
    for (int j = 0; j < kNb; ++j)
        if (j < nb) x[j] = v[j];
}

// Backward substitution with L^T on the diagonal block [k0, k0+nb):
// X[c][k0+j] = (X[c][k0+j] - sum_{m>j} L[k0+m][k0+j] X[c][k0+m]) / L_jj.
__global__ void __launch_bounds__(128) trsv_bwd_diag(const double *__restrict__ A, int N, int k0,
                                                     double *__restrict__ X, int ncols) {
    __shared__ double L[kNb][kNb + 1];
    const int nb = min(kNb, N - k0);
    for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
        const int i = t / nb, j = t % nb;
        L[i][j] = (j <= i) ? A[(size_t)(k0 + i) * N + k0 + j] : 0.0;
    }
    __syncthreads();
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncols) return;
    double *x = X + (size_t)c * N + k0;
    double v[kNb];
#pragma unroll
    for (int j = 0; j < kNb; ++j) v[j] = (j < nb) ? x[j] : 0.0;
#pragma unroll
    for (int j = kNb - 1; j >= 0; --j) {
        if (j < nb) {
            double a = v[j];
#pragma unroll
            for (int m = j + 1; m < kNb; ++m)
                if (m < nb) a -= L[m][j] * v[m];
            v[j] = a / L[j][j];
        }
    }
#pragma unroll
    for (int j = 0; j < kNb; ++j)
        if (j < nb) x[j] = v[j];
}

// Update after a solved block [k0, k0+nb) of every column:
//   forward  (bwd = 0): X[c][i] -= sum_m L[i][k0+m] X[c][k0+m]    for i in [k0+nb, N)
//   backward (bwd = 1): X[c][i] -= sum_m L[k0+m][i] X[c][k0+m]    for i in [0, k0)
// Tiles of 64 rows x 64 columns (grid.x over rows, grid.y over columns).
__global__ void __launch_bounds__(256) trsv_update(const double *__restrict__ A, int N, int k0, int nb,
                                                   double *__restrict__ X, int ncols, int bwd) {
    __shared__ double Lt[kTileR][kNb + 1];   // [row][m]
    __shared__ double Xs[kTileR][kNb + 1];   // [column][m]
    const int r_lo = bwd ? 0 : k0 + nb;
    const int i0 = r_lo + blockIdx.x * kTileR, c0 = blockIdx.y * kTileR;
    const int r_hi = bwd ? k0 : N;
    for (int t = threadIdx.x; t < kTileR * kNb; t += blockDim.x) {
        // forward: consecutive threads walk along a row of L (m fastest);
        // backward: along a row of L^T's source, i.e. r fastest
        const int r = bwd ? t % kTileR : t / kNb, m = bwd ? t / kTileR : t % kNb;
        double lv = 0.0;
        if (i0 + r < r_hi && m < nb)
            lv = bwd ? A[(size_t)(k0 + m) * N + i0 + r] : A[(size_t)(i0 + r) * N + k0 + m];
        Lt[r][m] = lv;
    }
    for (int t = threadIdx.x; t < kTileR * kNb; t += blockDim.x) {
        const int r = t / kNb, m = t % kNb;
        Xs[r][m] = (c0 + r < ncols && m < nb) ? X[(size_t)(c0 + r) * N + k0 + m] : 0.0;
    }
    __syncthreads();
    const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;
    double acc[4][4] = {};
#pragma unroll 4
    for (int m = 0; m < kNb; ++m) {
        double a[4], b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            a[u] = Lt[tr + 16 * u][m];
            b[u] = Xs[tc + 16 * u][m];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int i = i0 + tr + 16 * u, c = c0 + tc + 16 * v;
            if (i < r_hi && c < ncols) X[(size_t)c * N + i] -= acc[u][v];
        }
}

__global__ void copy_diag(const double *__restrict__ A, int N, double *__restrict__ d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) d[i] = A[(size_t)i * N + i];
}

}  // namespace

// Lower Cholesky factor of the row-major SPD matrix A (in place).  diag0
// (device, N) receives A's diagonal before factoring; err (device int) is
// OR-ed with 1 when a pivot is not positive beyond rounding.  Asynchronous.
int chol_factor(double *A, int N, double *diag0, int *err, cudaStream_t st) {
    copy_diag<<<(N + 255) / 256, 256, 0, st>>>(A, N, diag0);
    MF_CUDA(cudaGetLastError());
    for (int k0 = 0; k0 < N; k0 += kNb) {
        chol_diag<<<1, 256, 0, st>>>(A, N, k0, diag0, err);
        const int rest = N - k0 - kNb;
        if (rest > 0) {
            const int blocks = std::min((rest + 7) / 8, 1024);
            chol_panel<<<blocks, 256, 0, st>>>(A, N, k0);
            const int T = (rest + kTileR - 1) / kTileR;
            chol_update<<<T * (T + 1) / 2, 256, 0, st>>>(A, N, k0);
        }
        MF_CUDA(cudaGetLastError());
    }
    return MF_OK;
}

// X <- A^-1 X for the factor L of chol_factor (A = L L^T); X column-major
// [ncols][N].  Asynchronous.
int chol_solve(const double *L, int N, double *X, int ncols, cudaStream_t st) {
    const dim3 dg((ncols + 127) / 128);
    for (int k0 = 0; k0 < N; k0 += kNb) {
        const int nb = std::min(kNb, N - k0);
        trsv_fwd_diag<<<dg, 128, 0, st>>>(L, N, k0, X, ncols);
        const int rows = N - k0 - nb;
        if (rows > 0)
            trsv_update<<<dim3((rows + kTileR - 1) / kTileR, (ncols + kTileR - 1) / kTileR), 256, 0, st>>>(
                L, N, k0, nb, X, ncols, 0);
        MF_CUDA(cudaGetLastError());
    }
    const int last = (N - 1) / kNb * kNb;
    for (int k0 = last; k0 >= 0; k0 -= kNb) {
        const int nb = std::min(kNb, N - k0);
        trsv_bwd_diag<<<dg, 128, 0, st>>>(L, N, k0, X, ncols);
        if (k0 > 0)
            trsv_update<<<dim3((k0 + kTileR - 1) / kTileR, (ncols + kTileR - 1) / kTileR), 256, 0, st>>>(
                L, N, k0, nb, X, ncols, 1);
        MF_CUDA(cudaGetLastError());
    }
    return MF_OK;
}

}  // namespace mf
