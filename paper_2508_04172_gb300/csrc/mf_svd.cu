// SVD compression of a node-by-time overlap matrix (Eq. SVD) on the GPU in
// FP64, with this library's own kernels.
//
// The rank-l truncation of Z (N x M complex, row n = the overlap series at
// node n) needs the l dominant right singular vectors V_l; the coefficients
// are then C = Z V_l and the basis rows u_i = conj(V_l[:, i]).  They are found
// by block subspace iteration on Z itself (never on Z^H Z, which would square
// the condition number), with b = l + 10 columns:
//   Y = Z W                       (N x b)
//   Q = orth(Y)                   (classical Gram-Schmidt applied twice; a
//                                  numerically dependent column restarts from
//                                  a pseudo-random vector, Kahan-Parlett rule)
//   X = Z^H Q = Q_X R             (M x b, the same orthonormalisation)
//   R^H P = U S                   (one-sided Jacobi on the b x b factor)
//   W <- Q_X P, ordered by S      (the Ritz vectors; S = singular values of Q^H Z)
// until the leading l Ritz vectors, weighted by their singular values, move
// by less than 1e-12 s_1 between iterations (at least 2, at most 30
// iterations).  The singular values come from the Jacobi step on the small
// factor, which keeps them accurate to rounding of s_1 (no squaring).
//
// The FP64 rate of this GPU is low, so every step that touches the N x M
// matrix spreads over all SMs (tiled complex GEMM, split over k when the
// output has few tiles); the Gram-Schmidt runs as six launches per column
// with the cross-CTA sums done by the last CTA to finish (no waiting between
// CTAs); only the b x b Jacobi runs in one CTA.
//
// The file also holds the real FP64 GEMM that labels the surrogate's
// training set with the interpolant itself (dgemm_rm).
#include "mf_internal.cuh"

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

namespace mf {
namespace {

constexpr int kT = 32;          // GEMM output tile (complex elements)
constexpr int kKc = 16;         // GEMM k-chunk
constexpr int kOver = 10;       // oversampling columns
constexpr int kMinIter = 2;
constexpr int kMaxIter = 30;
constexpr double kTol = 1e-12;  // weighted subspace change, relative to s_1
constexpr int kCgsThreads = 128;
constexpr int kJacThreads = 1024;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
// conj(a) * b
__device__ __forceinline__ double2 cdotc(double2 a, double2 b) {
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 warp_sum2(double2 v) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, o);
        v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// ------------------------------------------------------------ complex GEMM
// C[m][n] (+)= sum_k opA(A)[m][k] opB(B)[k][n], row-major complex:
//   opA 0: A stored [m][k] (lda);  1: A^H, A stored [k][m] (lda)
//   opB 0: B stored [k][n] (ldb);  1: B^H, B stored [n][k] (ldb)
// blockIdx.z = k-split part: part z covers k in [z*kpart, (z+1)*kpart) and
// writes C + z*m*ldc (the parts are summed by sum_parts in a fixed order).
__global__ void __launch_bounds__(256) cgemm(int m, int n, int k, int kpart, const double2 *__restrict__ A, int lda,
                                             int opA, const double2 *__restrict__ B, int ldb, int opB,
                                             double2 *__restrict__ C, int ldc) {
    __shared__ double2 As[kKc][kT + 1], Bs[kKc][kT + 1];
    const int m0 = blockIdx.y * kT, n0 = blockIdx.x * kT;
    const int kb = blockIdx.z * kpart, ke = min(k, kb + kpart);
    C += (size_t)blockIdx.z * m * ldc;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;   // 2 x 2 outputs each
    double2 acc[2][2] = {};
    for (int k0 = kb; k0 < ke; k0 += kKc) {
        for (int t = threadIdx.x; t < kKc * kT; t += blockDim.x) {
            // each operand is read along its contiguous index: (kc, ic) walks k
            // fastest, (kr, ir) walks the m / n index fastest
            const int kc = t % kKc, ic = t / kKc, kr = t / kT, ir = t % kT;
            if (opA) {
                As[kr][ir] = (m0 + ir < m && k0 + kr < ke) ? cconj(A[(size_t)(k0 + kr) * lda + m0 + ir])
                                                           : make_double2(0.0, 0.0);
            } else {
                As[kc][ic] = (m0 + ic < m && k0 + kc < ke) ? A[(size_t)(m0 + ic) * lda + k0 + kc]
                                                           : make_double2(0.0, 0.0);
            }
            if (opB) {
                Bs[kc][ic] = (n0 + ic < n && k0 + kc < ke) ? cconj(B[(size_t)(n0 + ic) * ldb + k0 + kc])
                                                           : make_double2(0.0, 0.0);
            } else {
                Bs[kr][ir] = (n0 + ir < n && k0 + kr < ke) ? B[(size_t)(k0 + kr) * ldb + n0 + ir]
                                                           : make_double2(0.0, 0.0);
            }
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < kKc; ++kk) {
            const double2 a[2] = {As[kk][ty], As[kk][ty + 16]};
            const double2 b[2] = {Bs[kk][tx], Bs[kk][tx + 16]};
#pragma unroll
            for (int u = 0; u < 2; ++u)
#pragma unroll
                for (int v = 0; v < 2; ++v) {
                    acc[u][v].x = fma(a[u].x, b[v].x, fma(-a[u].y, b[v].y, acc[u][v].x));
                    acc[u][v].y = fma(a[u].x, b[v].y, fma(a[u].y, b[v].x, acc[u][v].y));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            const int r = m0 + ty + 16 * u, c = n0 + tx + 16 * v;
            if (r < m && c < n) C[(size_t)r * ldc + c] = acc[u][v];
        }
}

// out[i][j] = sum_z part[z][i][j]  (z ascending), i < m, j < n
__global__ void sum_parts(const double2 *__restrict__ part, int nz, int m, int n, double2 *__restrict__ out, int ldo) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)m * n) return;
    const int i = (int)(t / n), j = (int)(t % n);
    double2 s = make_double2(0.0, 0.0);
    for (int z = 0; z < nz; ++z) {
        const double2 v = part[(size_t)z * m * n + (size_t)i * n + j];
        s.x += v.x;
        s.y += v.y;
    }
    out[(size_t)i * ldo + j] = s;
}

// --------------------------------------------- Gram-Schmidt (twice), per column
// Y [rows][b] row-major is orthonormalised column by column in place; CTA c
// owns rows [c*chunk, min(rows, (c+1)*chunk)).  R [b][b] (row-major, zeroed
// by the caller) receives Y_in = Q R up to rounding.  Cross-CTA sums: every
// CTA writes its partial, the last CTA to arrive (atomic ticket) adds them in
// CTA order and writes the total; nobody waits.
//
// Column j is projected twice against q_0..q_{j-1}.  If the second
// projection shrinks it by more than the factor kAlpha, what is left is
// rounding noise (the column depends numerically on the previous ones, as
// the blocks of a low-rank Z do): the Kahan-Parlett rule sets R_jj = 0 and
// column j restarts from a fixed pseudo-random vector, projected twice in
// turn, so that Q stays orthonormal.
constexpr double kAlpha = 0.5;

struct CgsWork {
    double2 *part;     // [nblk][b] partial dots
    double *pnorm;     // [nblk] partial squared norms
    double2 *c0, *c1;  // [b] projection coefficients of two consecutive passes
    double *sc;        // [0] |v1|^2 after the first projection, [1] |v2|^2 after the
                       // second, [2] squared norm of what the column finally holds
    int *dep;          // [1] column numerically dependent (restarted)
    unsigned *ticket;  // [1] arrival counter (zero between launches)
};

// One launch of the per-column sequence (fields unused when null / zero).
struct CgsPass {
    int normalize_prev;       // scale column j-1 to unit norm first (R_{j-1,j-1} too)
    int guard;                // only when column j was found dependent
    int fill;                 // column j <- the restart vector
    const double2 *coef_in;   // y_j -= sum_i q_i coef_in[i]
    double2 *coef_out;        // coef_out[i] = <q_i, y_j> after the update
    int r_mode;               // coef_out into R[:, j]: 1 set, 2 add
    double *norm_out;         // |y_j|^2 after the update
    double *norm_out2;        // a second copy of it
    int set_dep;              // dep = |v2|^2 <= kAlpha^2 |v1|^2
};

__device__ bool last_to_arrive(unsigned *ticket) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
        if (last) *ticket = 0u;   // every CTA has arrived: safe to re-arm
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}
__device__ __forceinline__ double unit_uniform(uint64_t key) {   // [-1, 1)
    return (double)(mix64(key + 0x9E3779B97F4A7C15ull) >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

__global__ void __launch_bounds__(kCgsThreads) cgs_pass(double2 *__restrict__ Y, int rows, int b, int j, int chunk,
                                                        CgsPass p, CgsWork w, double2 *__restrict__ R) {
    extern __shared__ double2 csh[];
    __shared__ double red[kCgsThreads / 32];
    if (p.guard && !__ldcg(w.dep)) return;   // the same flag for every CTA
    const int r0 = blockIdx.x * chunk, r1 = min(rows, r0 + chunk);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (p.normalize_prev && j > 0) {
        const double nrm = sqrt(__ldcg(w.sc + 2));
        const double inv = nrm > 1e-300 ? 1.0 / nrm : 0.0;
        if (R && blockIdx.x == 0 && threadIdx.x == 0)
            R[(size_t)(j - 1) * b + j - 1] = make_double2(__ldcg(w.dep) ? 0.0 : sqrt(__ldcg(w.sc + 1)), 0.0);
        for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
            const double2 v = Y[(size_t)r * b + j - 1];
            Y[(size_t)r * b + j - 1] = make_double2(v.x * inv, v.y * inv);
        }
        __syncthreads();
    }
    if (j >= b) return;
    if (p.fill)
        for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
            const uint64_t key = ((uint64_t)r * (uint64_t)b + (uint64_t)j) * 2u;
            Y[(size_t)r * b + j] = make_double2(unit_uniform(key), unit_uniform(key + 1));
        }
    if (p.coef_in) {
        for (int i = threadIdx.x; i < j; i += blockDim.x) csh[i] = __ldcg(p.coef_in + i);
        __syncthreads();
        for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
            double2 v = Y[(size_t)r * b + j];
            for (int i = 0; i < j; ++i) {
                const double2 q = cmul(Y[(size_t)r * b + i], csh[i]);
                v.x -= q.x;
                v.y -= q.y;
            }
            Y[(size_t)r * b + j] = v;
        }
    }
    __syncthreads();
    if (p.coef_out)
        for (int i = warp; i < j; i += nw) {
            double2 s = make_double2(0.0, 0.0);
            for (int r = r0 + lane; r < r1; r += 32) {
                const double2 q = cdotc(Y[(size_t)r * b + i], Y[(size_t)r * b + j]);
                s.x += q.x;
                s.y += q.y;
            }
            s = warp_sum2(s);
            if (lane == 0) w.part[(size_t)blockIdx.x * b + i] = s;
        }
    if (p.norm_out) {
        double s = 0.0;
        for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
            const double2 v = Y[(size_t)r * b + j];
            s += v.x * v.x + v.y * v.y;
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) red[warp] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int i = 0; i < nw; ++i) t += red[i];
            w.pnorm[blockIdx.x] = t;
        }
    }
    if (!last_to_arrive(w.ticket)) return;
    if (p.coef_out)
        for (int i = threadIdx.x; i < j; i += blockDim.x) {
            double2 s = make_double2(0.0, 0.0);
            for (int c = 0; c < (int)gridDim.x; ++c) {
                const double2 v = __ldcg(w.part + (size_t)c * b + i);
                s.x += v.x;
                s.y += v.y;
            }
            p.coef_out[i] = s;
            if (R && p.r_mode) {
                double2 *e = R + (size_t)i * b + j;
                *e = p.r_mode == 2 ? make_double2(e->x + s.x, e->y + s.y) : s;
            }
        }
    if (p.norm_out && threadIdx.x == 0) {
        double t = 0.0;
        for (int c = 0; c < (int)gridDim.x; ++c) t += __ldcg(w.pnorm + c);
        *p.norm_out = t;
        if (p.norm_out2) *p.norm_out2 = t;
        if (p.set_dep) *w.dep = (t <= kAlpha * kAlpha * __ldcg(w.sc)) ? 1 : 0;
    }
}

// ------------------------------------------------ one-sided Jacobi (one CTA)
// A [n][n] column-major (A[c*n + r] = row r of column c), n even.  Rotates
// pairs of columns until every pair is orthogonal to tol (relative), with the
// unitary accumulated in P (column-major, starts at I): A_in P = A_out, whose
// column norms are the singular values s[c].  Round-robin ordering: each step
// rotates n/2 disjoint pairs at once.
__global__ void __launch_bounds__(kJacThreads) jacobi_onesided(double2 *__restrict__ A, double2 *__restrict__ P, int n,
                                                               int max_sweeps, double tol, double *__restrict__ s,
                                                               int *__restrict__ sweeps_out) {
    extern __shared__ double jsh[];
    const int h = n / 2;
    double *rc = jsh, *rs = rc + h, *pc = rs + h, *ps = pc + h;
    int *top = (int *)(ps + h), *bot = top + h;
    __shared__ int rotated;
    for (size_t i = threadIdx.x; i < (size_t)n * n; i += blockDim.x)
        P[i] = make_double2((i / n) == (i % n) ? 1.0 : 0.0, 0.0);
    for (int i = threadIdx.x; i < h; i += blockDim.x) {
        top[i] = 2 * i;
        bot[i] = 2 * i + 1;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) rotated = 0;
        __syncthreads();
        for (int step = 0; step < n - 1; ++step) {
            for (int k = warp; k < h; k += nw) {
                const int p = min(top[k], bot[k]), q = max(top[k], bot[k]);
                const double2 *ap = A + (size_t)p * n, *aq = A + (size_t)q * n;
                double al = 0.0, be = 0.0;
                double2 ga = make_double2(0.0, 0.0);
                for (int r = lane; r < n; r += 32) {
                    const double2 x = ap[r], y = aq[r];
                    al += x.x * x.x + x.y * x.y;
                    be += y.x * y.x + y.y * y.y;
                    const double2 g = cdotc(x, y);
                    ga.x += g.x;
                    ga.y += g.y;
                }
                for (int o = 16; o > 0; o >>= 1) {
                    al += __shfl_down_sync(0xffffffffu, al, o);
                    be += __shfl_down_sync(0xffffffffu, be, o);
                }
                ga = warp_sum2(ga);
                if (lane == 0) {
                    const double ab = sqrt(ga.x * ga.x + ga.y * ga.y);
                    double c = 1.0, sn = 0.0, cp = 1.0, sp = 0.0;
                    if (ab > 1e-300 && ab > tol * sqrt(al * be)) {
                        // 2x2 Hermitian Gram [[al, ga], [conj(ga), be]]: phase
                        // e^{i phi} = ga/|ga| removed, then the real symmetric
                        // Jacobi rotation (tangent of the smaller angle)
                        cp = ga.x / ab;
                        sp = ga.y / ab;
                        const double tau = (be - al) / (2.0 * ab);
                        const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + t * t);
                        sn = t * c;
                        rotated = 1;
                    }
                    rc[k] = c;
                    rs[k] = sn;
                    pc[k] = cp;
                    ps[k] = sp;
                }
            }
            __syncthreads();
            // [a_p, a_q] <- [a_p, a_q] U,  U = [[c, s], [-s e^{-i phi}, c e^{-i phi}]]
            for (int t = threadIdx.x; t < n * h; t += blockDim.x) {
                const int k = t / n, r = t % n;
                const double c = rc[k], sn = rs[k];
                if (sn == 0.0 && c == 1.0) continue;
                const int p = min(top[k], bot[k]), q = max(top[k], bot[k]);
                const double2 em = make_double2(pc[k], -ps[k]);
                double2 *ap = A + (size_t)p * n + r, *aq = A + (size_t)q * n + r;
                const double2 x = *ap, y = cmul(*aq, em);
                *ap = make_double2(c * x.x - sn * y.x, c * x.y - sn * y.y);
                *aq = make_double2(sn * x.x + c * y.x, sn * x.y + c * y.y);
                double2 *vp = P + (size_t)p * n + r, *vq = P + (size_t)q * n + r;
                const double2 u = *vp, v = cmul(*vq, em);
                *vp = make_double2(c * u.x - sn * v.x, c * u.y - sn * v.y);
                *vq = make_double2(sn * u.x + c * v.x, sn * u.y + c * v.y);
            }
            __syncthreads();
            if (threadIdx.x == 0 && h > 1) {
                // round-robin: index top[0] stays, the others move one place
                const int last_top = top[h - 1];
                for (int k = h - 1; k > 1; --k) top[k] = top[k - 1];
                top[1] = bot[0];
                for (int k = 0; k < h - 1; ++k) bot[k] = bot[k + 1];
                bot[h - 1] = last_top;
            }
            __syncthreads();
        }
        const int any = rotated;
        __syncthreads();
        if (!any) break;
    }
    for (int c = warp; c < n; c += nw) {
        double t = 0.0;
        for (int r = lane; r < n; r += 32) {
            const double2 x = A[(size_t)c * n + r];
            t += x.x * x.x + x.y * x.y;
        }
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) s[c] = sqrt(t);
    }
    if (threadIdx.x == 0 && sweeps_out) *sweeps_out = sweep;
}

// A [n][n] column-major = R^H for R [b][b] row-major (rows / columns >= b zero)
__global__ void r_adjoint(const double2 *__restrict__ R, int b, int n, double2 *__restrict__ A) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * n) return;
    const int c = t / n, r = t % n;   // A[r][c] = conj(R[c][r])
    A[t] = (r < b && c < b) ? cconj(R[(size_t)c * b + r]) : make_double2(0.0, 0.0);
}

// Pp [b][b] row-major: column c = column perm[c] of P (column-major, n x n)
__global__ void gather_perm(const double2 *__restrict__ P, int n, int b, const int *__restrict__ perm,
                            double2 *__restrict__ Pp) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= b * b) return;
    const int i = t / b, c = t % b;
    Pp[t] = P[(size_t)perm[c] * n + i];
}

// Deterministic start block [M][b]: the splitmix64 finaliser of the element
// index, uniform in [-1, 1) per component.
__global__ void start_block(double2 *__restrict__ W, size_t count) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const double sc = 2.0 / 9007199254740992.0;
    const double re = (double)(mix64(2 * i + 0x9E3779B97F4A7C15ull) >> 11) * sc - 1.0;
    const double im = (double)(mix64(2 * i + 1 + 0x9E3779B97F4A7C15ull) >> 11) * sc - 1.0;
    W[i] = make_double2(re, im);
}

// res[c] = sum_r |Wn[r][c] - T[r][c]|^2, c < l  (Wn: ld b; T: ld l); one CTA per column
__global__ void col_residual(const double2 *__restrict__ Wn, int b, const double2 *__restrict__ T, int l, int M,
                             double *__restrict__ res) {
    __shared__ double red[8];
    const int c = blockIdx.x;
    double s = 0.0;
    for (int r = threadIdx.x; r < M; r += blockDim.x) {
        const double2 a = Wn[(size_t)r * b + c], t = T[(size_t)r * l + c];
        const double dx = a.x - t.x, dy = a.y - t.y;
        s += dx * dx + dy * dy;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
        res[c] = t;
    }
}

// basis [l][M] = conj(W[:, :l])^T  (W: [M][b])
__global__ void basis_rows(const double2 *__restrict__ W, int M, int b, int l, double2 *__restrict__ basis) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)M * l) return;
    const int c = (int)(t / M), r = (int)(t % M);
    basis[t] = cconj(W[(size_t)r * b + c]);
}

template <class T>
struct Buf {
    T *p = nullptr;
    ~Buf() { if (p) cudaFree(p); }
    cudaError_t alloc(size_t n) { return cudaMalloc((void **)&p, std::max<size_t>(n, 1) * sizeof(T)); }
};

struct Svd {
    cudaStream_t st;
    int nsm;
    Buf<double2> gpart;      // k-split partial outputs
    size_t gpart_n = 0;

    // C = opA(A) opB(B), split over k when the output has few tiles
    int gemm(int m, int n, int k, const double2 *A, int lda, int opA, const double2 *B, int ldb, int opB, double2 *C,
             int ldc) {
        const int tiles = ((m + kT - 1) / kT) * ((n + kT - 1) / kT);
        int nz = 1;
        if (tiles < 4 * nsm) nz = std::max(1, std::min((4 * nsm + tiles - 1) / tiles, k / 512));
        int kpart = (k + nz - 1) / nz;
        kpart = (kpart + kKc - 1) / kKc * kKc;
        nz = (k + kpart - 1) / kpart;
        dim3 grid((n + kT - 1) / kT, (m + kT - 1) / kT, nz);
        if (nz == 1) {
            cgemm<<<grid, 256, 0, st>>>(m, n, k, kpart, A, lda, opA, B, ldb, opB, C, ldc);
            MF_CUDA(cudaGetLastError());
            return MF_OK;
        }
        const size_t need = (size_t)nz * m * n;
        if (need > gpart_n) {
            if (gpart.p) cudaFree(gpart.p);
            gpart.p = nullptr;
            MF_CUDA(gpart.alloc(need));
            gpart_n = need;
        }
        cgemm<<<grid, 256, 0, st>>>(m, n, k, kpart, A, lda, opA, B, ldb, opB, gpart.p, n);
        MF_CUDA(cudaGetLastError());
        sum_parts<<<(unsigned)((size_t)m * n + 255) / 256, 256, 0, st>>>(gpart.p, nz, m, n, C, ldc);
        MF_CUDA(cudaGetLastError());
        return MF_OK;
    }

    // Y [rows][b] <- orth(Y), R (zeroed here) with Y_in = Y_out R
    int orth(double2 *Y, int rows, int b, double2 *R, CgsWork &w) {
        const int nblk = std::max(1, std::min(nsm, (rows + 15) / 16));
        const int chunk = (rows + nblk - 1) / nblk;
        const int nb = (rows + chunk - 1) / chunk;
        if (R) MF_CUDA(cudaMemsetAsync(R, 0, sizeof(double2) * (size_t)b * b, st));
        const size_t dsm = sizeof(double2) * (size_t)b;
        double *v1 = w.sc, *v2 = w.sc + 1, *fin = w.sc + 2;
        for (int j = 0; j <= b; ++j) {
            // first projection (after scaling column j-1), second projection,
            // then the restart of a dependent column (no-ops otherwise)
            CgsPass p1{1, 0, 0, nullptr, w.c0, 1, nullptr, nullptr, 0};
            CgsPass p2{0, 0, 0, w.c0, w.c1, 2, v1, nullptr, 0};
            CgsPass p3{0, 0, 0, w.c1, nullptr, 0, v2, fin, 1};
            CgsPass p4{0, 1, 1, nullptr, w.c0, 0, nullptr, nullptr, 0};
            CgsPass p5{0, 1, 0, w.c0, w.c1, 0, nullptr, nullptr, 0};
            CgsPass p6{0, 1, 0, w.c1, nullptr, 0, fin, nullptr, 0};
            cgs_pass<<<nb, kCgsThreads, dsm, st>>>(Y, rows, b, j, chunk, p1, w, R);
            if (j == b) break;
            cgs_pass<<<nb, kCgsThreads, dsm, st>>>(Y, rows, b, j, chunk, p2, w, R);
            cgs_pass<<<nb, kCgsThreads, dsm, st>>>(Y, rows, b, j, chunk, p3, w, R);
            cgs_pass<<<nb, kCgsThreads, dsm, st>>>(Y, rows, b, j, chunk, p4, w, R);
            cgs_pass<<<nb, kCgsThreads, dsm, st>>>(Y, rows, b, j, chunk, p5, w, R);
            cgs_pass<<<nb, kCgsThreads, dsm, st>>>(Y, rows, b, j, chunk, p6, w, R);
        }
        MF_CUDA(cudaGetLastError());
        return MF_OK;
    }
};

// ------------------------------------------------------------- real GEMM
// C[m][n] = A[m][k] B[k][n], row-major FP64, 64 x 64 outputs per CTA
constexpr int kDT = 64, kDK = 16;
__global__ void __launch_bounds__(256) dgemm_kernel(int m, int n, int k, const double *__restrict__ A, int lda,
                                                    const double *__restrict__ B, int ldb, double *__restrict__ C,
                                                    int ldc) {
    __shared__ double As[kDK][kDT + 1], Bs[kDK][kDT];
    const int m0 = blockIdx.y * kDT, n0 = blockIdx.x * kDT;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;   // 4 x 4 outputs each, stride 16
    double acc[4][4] = {};
    for (int k0 = 0; k0 < k; k0 += kDK) {
        for (int t = threadIdx.x; t < kDK * kDT; t += blockDim.x) {
            const int kk = t % kDK, i = t / kDK;          // A: along k
            As[kk][i] = (m0 + i < m && k0 + kk < k) ? A[(size_t)(m0 + i) * lda + k0 + kk] : 0.0;
            const int kb = t / kDT, j = t % kDT;          // B: along n
            Bs[kb][j] = (n0 + j < n && k0 + kb < k) ? B[(size_t)(k0 + kb) * ldb + n0 + j] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < kDK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = As[kk][ty + 16 * u];
                b[u] = Bs[kk][tx + 16 * u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int r = m0 + ty + 16 * u, c = n0 + tx + 16 * v;
            if (r < m && c < n) C[(size_t)r * ldc + c] = acc[u][v];
        }
}

}  // namespace

int dgemm_rm(int m, int n, int k, const double *A, int lda, const double *B, int ldb, double *C, int ldc,
             cudaStream_t st) {
    if (m <= 0 || n <= 0) return MF_OK;
    dim3 grid((n + kDT - 1) / kDT, (m + kDT - 1) / kDT);
    dgemm_kernel<<<grid, 256, 0, st>>>(m, n, k, A, lda, B, ldb, C, ldc);
    MF_CUDA(cudaGetLastError());
    return MF_OK;
}

// See mf_svd_compress (mf.h).  z, coef, basis, sv are host arrays.
int svd_compress(const double *z, int N, int M, int rank, double *coef, double *basis, double *sv, cudaStream_t st) {
    if (N < M) return MF_E_INVAL;   // one row per node; more nodes than samples
    const int l = rank;
    const int b = std::min(M, l + kOver);
    const int n = b + (b & 1);      // the Jacobi pairs columns: even size
    int dev = 0;
    MF_CUDA(cudaGetDevice(&dev));
    Svd S;
    S.st = st;
    MF_CUDA(cudaDeviceGetAttribute(&S.nsm, cudaDevAttrMultiProcessorCount, dev));
    const int nblk = std::max(1, std::min(S.nsm, (std::max(N, M) + 15) / 16));
    Buf<double2> Z, W, Wn, Y, X, R, A, P, Pp, Sm, T, C, Bas, part, c0, c1;
    Buf<double> pnorm, sc, sig, res;
    Buf<unsigned> ticket;
    Buf<int> perm, sweeps, dep;
    MF_CUDA(Z.alloc((size_t)N * M));
    MF_CUDA(W.alloc((size_t)M * b));
    MF_CUDA(Wn.alloc((size_t)M * b));
    MF_CUDA(Y.alloc((size_t)N * b));
    MF_CUDA(X.alloc((size_t)M * b));
    MF_CUDA(R.alloc((size_t)b * b));
    MF_CUDA(A.alloc((size_t)n * n));
    MF_CUDA(P.alloc((size_t)n * n));
    MF_CUDA(Pp.alloc((size_t)b * b));
    MF_CUDA(Sm.alloc((size_t)l * l));
    MF_CUDA(T.alloc((size_t)M * l));
    MF_CUDA(C.alloc((size_t)N * l));
    MF_CUDA(Bas.alloc((size_t)l * M));
    MF_CUDA(part.alloc((size_t)nblk * b));
    MF_CUDA(c0.alloc(b));
    MF_CUDA(c1.alloc(b));
    MF_CUDA(pnorm.alloc(nblk));
    MF_CUDA(sc.alloc(3));
    MF_CUDA(dep.alloc(1));
    MF_CUDA(sig.alloc(n));
    MF_CUDA(res.alloc(l));
    MF_CUDA(ticket.alloc(1));
    MF_CUDA(perm.alloc(b));
    MF_CUDA(sweeps.alloc(1));
    MF_CUDA(cudaMemsetAsync(ticket.p, 0, sizeof(unsigned), st));
    MF_CUDA(cudaMemsetAsync(dep.p, 0, sizeof(int), st));
    MF_CUDA(cudaMemsetAsync(sc.p, 0, 3 * sizeof(double), st));
    MF_CUDA(cudaMemcpyAsync(Z.p, z, sizeof(double2) * (size_t)N * M, cudaMemcpyHostToDevice, st));
    CgsWork w{part.p, pnorm.p, c0.p, c1.p, sc.p, dep.p, ticket.p};
    const size_t jsm = (sizeof(double) * 4 + sizeof(int) * 2) * (size_t)(n / 2);
    if (jsm > 48 * 1024) MF_CUDA(cudaFuncSetAttribute(jacobi_onesided, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)jsm));

    start_block<<<(unsigned)(((size_t)M * b + 255) / 256), 256, 0, st>>>(W.p, (size_t)M * b);
    MF_CUDA(cudaGetLastError());
    std::vector<double> hs(n), hres(l), hsv(b);
    std::vector<int> order(n);
    int rc;
    for (int it = 0; it < kMaxIter; ++it) {
        if ((rc = S.gemm(N, b, M, Z.p, M, 0, W.p, b, 0, Y.p, b))) return rc;          // Y = Z W
        if ((rc = S.orth(Y.p, N, b, nullptr, w))) return rc;                          // Q = orth(Y)
        if ((rc = S.gemm(M, b, N, Z.p, M, 1, Y.p, b, 0, X.p, b))) return rc;          // X = Z^H Q
        if ((rc = S.orth(X.p, M, b, R.p, w))) return rc;                               // X = Q_X R
        r_adjoint<<<(n * n + 255) / 256, 256, 0, st>>>(R.p, b, n, A.p);
        MF_CUDA(cudaGetLastError());
        jacobi_onesided<<<1, kJacThreads, jsm, st>>>(A.p, P.p, n, 60, n * 2.3e-16, sig.p, sweeps.p);
        MF_CUDA(cudaGetLastError());
        MF_CUDA(cudaMemcpyAsync(hs.data(), sig.p, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
        MF_CUDA(cudaStreamSynchronize(st));
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return hs[a] > hs[c]; });
        MF_CUDA(cudaMemcpyAsync(perm.p, order.data(), sizeof(int) * b, cudaMemcpyHostToDevice, st));
        gather_perm<<<(b * b + 255) / 256, 256, 0, st>>>(P.p, n, b, perm.p, Pp.p);
        MF_CUDA(cudaGetLastError());
        if ((rc = S.gemm(M, b, b, X.p, b, 0, Pp.p, b, 0, Wn.p, b))) return rc;        // W' = Q_X P
        for (int i = 0; i < b; ++i) hsv[i] = hs[order[i]];
        bool done = false;
        if (it + 1 >= kMinIter) {
            // weighted change of the leading l Ritz vectors: |W'_c - W W^H W'_c|
            if ((rc = S.gemm(l, l, M, W.p, b, 1, Wn.p, b, 0, Sm.p, l))) return rc;    // S = W_l^H W'_l
            if ((rc = S.gemm(M, l, l, W.p, b, 0, Sm.p, l, 0, T.p, l))) return rc;      // T = W_l S
            col_residual<<<l, 256, 0, st>>>(Wn.p, b, T.p, l, M, res.p);
            MF_CUDA(cudaGetLastError());
            MF_CUDA(cudaMemcpyAsync(hres.data(), res.p, sizeof(double) * l, cudaMemcpyDeviceToHost, st));
            MF_CUDA(cudaStreamSynchronize(st));
            double e = 0.0;
            for (int c = 0; c < l; ++c) e += hsv[c] * hsv[c] * hres[c];
            done = std::sqrt(e) <= kTol * hsv[0] || hsv[0] == 0.0;
        }
        std::swap(W.p, Wn.p);
        if (done) break;
    }
    if ((rc = S.gemm(N, l, M, Z.p, M, 0, W.p, b, 0, C.p, l))) return rc;              // C = Z V_l
    basis_rows<<<(unsigned)(((size_t)M * l + 255) / 256), 256, 0, st>>>(W.p, M, b, l, Bas.p);
    MF_CUDA(cudaGetLastError());
    MF_CUDA(cudaMemcpyAsync(coef, C.p, sizeof(double2) * (size_t)N * l, cudaMemcpyDeviceToHost, st));
    MF_CUDA(cudaMemcpyAsync(basis, Bas.p, sizeof(double2) * (size_t)l * M, cudaMemcpyDeviceToHost, st));
    MF_CUDA(cudaStreamSynchronize(st));
    if (sv)
        for (int i = 0; i < l; ++i) sv[i] = hsv[i];
    return MF_OK;
}

}  // namespace mf
