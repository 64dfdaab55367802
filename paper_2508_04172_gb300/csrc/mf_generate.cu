// Start-up generation on the GPU (Sec. II C): node placement in the squeezed
// constant-match ellipsoid with a Halton sequence (Sec. II C 1), node
// overlaps z(t) over circular time shifts and mode cross terms sigma from
// synthetic detector data (Sec. II C 2), and the squeeze factor from the
// true match along the ellipsoid's longest axis (Eqs. Match, MisMatch).
//
// The templates are the frequency-domain stand-in declared in mf.h
// (mf_wave): per mode (l, m), with F = 2 f / m,
//   h_{l,-m}(f) = amp (F/f_ref)^(-7/6) exp(-i (m/2) sum_a s_a theta_a u_a(F/f_ref))
// on F_lo(theta) <= F <= f_hi, F_lo = f_lo exp(c_r c_v . theta),
// u_a(x) = x^p_a - 1 - p_a (x - 1).  The u_a and amplitudes depend on the
// frequency only and are tabulated once per call; a template is then 4 FMAs
// and one sincos per frequency.
//
// Overlaps: one CTA per (node, mode) forms P_j = 4 df conj(h_j) d_j / S_j
// for each detector, stores it bit-reversed in shared memory and runs an
// in-place radix-2 inverse FFT of length L (FP64, twiddles from a table
// built with sincospi); the M samples t_s = s dt, s = -M/2 .. M/2-1 (circular
// indices) are written out.
#include "mf_internal.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace mf {
namespace {

constexpr int kFftThreads = 512;
constexpr int kMaxL = 8192;       // FFT length limit (L complex doubles in shared memory)

struct WaveDev {
    int n_modes, nf, L;
    int em[kMaxModes];
    double f_lo, f_hi, f_ref, df, cut_rate;
    double cut_dir[4];
};

__device__ __forceinline__ int bitrev(int j, int logL) { return (int)(__brev((unsigned)j) >> (32 - logL)); }

// tables: U[mu][a][j] = s_a u_a(F_j / f_ref), A[mu][j] = amp (F_j/f_ref)^(-7/6) (0 outside [f_lo0, f_hi])
__global__ void wave_tables(const mf_wave w, int nf, double df, double *__restrict__ U, double *__restrict__ A) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int mu = blockIdx.y;
    if (j >= nf) return;
    const int m = w.ell_m[mu][1];
    const double F = 2.0 * (double)j * df / (double)m;
    const double x = F / w.f_ref;
    const bool inb = F > 0.0 && F <= w.f_hi;
    for (int a = 0; a < 4; ++a)
        U[((size_t)mu * 4 + a) * nf + j] = inb ? w.scales[a] * (pow(x, w.powers[a]) - 1.0 - w.powers[a] * (x - 1.0)) : 0.0;
    A[(size_t)mu * nf + j] = inb ? w.amp[mu] * pow(x, -7.0 / 6.0) : 0.0;
}

__global__ void twiddles(int L, double2 *__restrict__ tw) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= L / 2) return;
    double s, c;
    sincospi(2.0 * (double)j / (double)L, &s, &c);
    tw[j] = make_double2(c, s);   // exp(+2 pi i j / L)
}

// template value of mode mu at frequency bin j for theta (F_lo from theta)
__device__ __forceinline__ double2 tmpl(const WaveDev &w, int mu, int j, const double *U, const double *A,
                                        const double (&th)[4], double f_lo) {
    const double a = A[(size_t)mu * w.nf + j];
    const double F = 2.0 * (double)j * w.df / (double)w.em[mu];
    if (a == 0.0 || F < f_lo) return make_double2(0.0, 0.0);
    const double *u = U + (size_t)mu * 4 * w.nf + j;
    const double psi = th[0] * u[0] + th[1] * u[w.nf] + th[2] * u[2 * w.nf] + th[3] * u[3 * w.nf];
    double s, c;
    sincos(-0.5 * (double)w.em[mu] * psi, &s, &c);
    return make_double2(a * c, a * s);
}

__device__ __forceinline__ double band_edge(const WaveDev &w, const double (&th)[4]) {
    return w.f_lo * exp(w.cut_rate * (w.cut_dir[0] * th[0] + w.cut_dir[1] * th[1] + w.cut_dir[2] * th[2] +
                                      w.cut_dir[3] * th[3]));
}

// in-place radix-2 inverse FFT of X[0..L) (input in bit-reversed order)
__device__ __forceinline__ void ifft_smem(double2 *X, int L, int logL, const double2 *__restrict__ tw) {
    for (int s = 1; s <= logL; ++s) {
        const int half = 1 << (s - 1);
        const int stride = L >> s;              // twiddle index step
        for (int b = threadIdx.x; b < L / 2; b += blockDim.x) {
            const int grp = b >> (s - 1), k = b & (half - 1);
            const int i = grp * 2 * half + k;
            const double2 wv = __ldg(tw + k * stride);
            const double2 u = X[i], v = X[i + half];
            const double2 t = make_double2(v.x * wv.x - v.y * wv.y, v.x * wv.y + v.y * wv.x);
            X[i] = make_double2(u.x + t.x, u.y + t.y);
            X[i + half] = make_double2(u.x - t.x, u.y - t.y);
        }
        __syncthreads();
    }
}

// one CTA per (node n, mode mu): z[k][mu][n][0..M) for every detector k
__global__ void __launch_bounds__(kFftThreads) overlap_fft(const WaveDev w, int logL, const double *__restrict__ U,
                                                           const double *__restrict__ A,
                                                           const double2 *__restrict__ tw,
                                                           const double *__restrict__ theta, int N,
                                                           const double2 *__restrict__ data,
                                                           const double *__restrict__ psd, int n_det, int M,
                                                           double2 *__restrict__ z) {
    extern __shared__ double2 X[];
    const int n = blockIdx.x, mu = blockIdx.y;
    double th[4];
    for (int a = 0; a < 4; ++a) th[a] = theta[(size_t)n * 4 + a];
    const double f_lo = band_edge(w, th);
    for (int k = 0; k < n_det; ++k) {
        for (int j = threadIdx.x; j < w.L; j += blockDim.x) {
            double2 p = make_double2(0.0, 0.0);
            if (j < w.nf) {
                const double2 h = tmpl(w, mu, j, U, A, th, f_lo);
                const double2 d = data[(size_t)k * w.nf + j];
                const double g = 4.0 * w.df / psd[(size_t)k * w.nf + j];
                // conj(h) d
                p = make_double2(g * (h.x * d.x + h.y * d.y), g * (h.x * d.y - h.y * d.x));
            }
            X[bitrev(j, logL)] = p;
        }
        __syncthreads();
        ifft_smem(X, w.L, logL, tw);
        for (int s = threadIdx.x; s < M; s += blockDim.x) {
            const int idx = ((s - M / 2) % w.L + w.L) % w.L;
            z[(((size_t)k * w.n_modes + mu) * N + n) * M + s] = X[idx];
        }
        __syncthreads();
    }
}

// one CTA per node: sigma[k][n][mu][nu] = 4 df sum_j conj(h_mu) h_nu / S_k
__global__ void __launch_bounds__(256) cross_terms(const WaveDev w, const double *__restrict__ U,
                                                   const double *__restrict__ A, const double *__restrict__ theta,
                                                   int N, const double *__restrict__ psd, int n_det,
                                                   double2 *__restrict__ sigma) {
    __shared__ double red[256];
    const int n = blockIdx.x;
    double th[4];
    for (int a = 0; a < 4; ++a) th[a] = theta[(size_t)n * 4 + a];
    const double f_lo = band_edge(w, th);
    const int nm = w.n_modes;
    for (int k = 0; k < n_det; ++k)
        for (int mu = 0; mu < nm; ++mu)
            for (int nu = mu; nu < nm; ++nu) {
                double sr = 0.0, si = 0.0;
                for (int j = threadIdx.x; j < w.nf; j += blockDim.x) {
                    const double2 a = tmpl(w, mu, j, U, A, th, f_lo);
                    const double2 b = tmpl(w, nu, j, U, A, th, f_lo);
                    const double g = 1.0 / psd[(size_t)k * w.nf + j];
                    sr += g * (a.x * b.x + a.y * b.y);
                    si += g * (a.x * b.y - a.y * b.x);
                }
                double v[2] = {sr, si};
                for (int c = 0; c < 2; ++c) {
                    red[threadIdx.x] = v[c];
                    __syncthreads();
                    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
                        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
                        __syncthreads();
                    }
                    v[c] = red[0];
                    __syncthreads();
                }
                if (threadIdx.x == 0) {
                    const double2 s = make_double2(4.0 * w.df * v[0], 4.0 * w.df * v[1]);
                    sigma[(((size_t)k * N + n) * nm + mu) * nm + nu] = s;
                    sigma[(((size_t)k * N + n) * nm + nu) * nm + mu] = make_double2(s.x, -s.y);
                }
            }
}

// one CTA per point b: match of the dominant-mode templates at thA and thB[b]
// (Eq. Match: modulus of the normalised overlap, maximised over the L shifts)
__global__ void __launch_bounds__(kFftThreads) match_fft(const WaveDev w, int logL, const double *__restrict__ U,
                                                         const double *__restrict__ A,
                                                         const double2 *__restrict__ tw, const double *__restrict__ thA,
                                                         const double *__restrict__ thB, const double *__restrict__ psd,
                                                         double *__restrict__ out) {
    extern __shared__ double2 X[];
    __shared__ double red[3][kFftThreads];
    double ta[4], tb[4];
    for (int a = 0; a < 4; ++a) {
        ta[a] = thA[a];
        tb[a] = thB[(size_t)blockIdx.x * 4 + a];
    }
    const double la = band_edge(w, ta), lb = band_edge(w, tb);
    double saa = 0.0, sbb = 0.0;
    for (int j = threadIdx.x; j < w.L; j += blockDim.x) {
        double2 p = make_double2(0.0, 0.0);
        if (j < w.nf) {
            const double2 ha = tmpl(w, 0, j, U, A, ta, la), hb = tmpl(w, 0, j, U, A, tb, lb);
            const double g = 1.0 / psd[j];
            saa += g * (ha.x * ha.x + ha.y * ha.y);
            sbb += g * (hb.x * hb.x + hb.y * hb.y);
            p = make_double2(g * (hb.x * ha.x + hb.y * ha.y), g * (hb.x * ha.y - hb.y * ha.x));   // conj(hb) ha
        }
        X[bitrev(j, logL)] = p;
    }
    red[0][threadIdx.x] = saa;
    red[1][threadIdx.x] = sbb;
    __syncthreads();
    ifft_smem(X, w.L, logL, tw);
    double best = 0.0;
    for (int j = threadIdx.x; j < w.L; j += blockDim.x) best = fmax(best, X[j].x * X[j].x + X[j].y * X[j].y);
    red[2][threadIdx.x] = best;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            red[0][threadIdx.x] += red[0][threadIdx.x + o];
            red[1][threadIdx.x] += red[1][threadIdx.x + o];
            red[2][threadIdx.x] = fmax(red[2][threadIdx.x], red[2][threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = sqrt(red[2][0]) / sqrt(red[0][0] * red[1][0]);
}

// Halton coordinate of index i in base b as the exact fraction
// (mirrored digits) / b^ndigits, rounded once
__device__ __forceinline__ double radical_inverse(long long i, int b) {
    long long num = 0, den = 1;
    while (i > 0) {
        const long long d = i % b;
        i /= b;
        num = num * b + d;
        den *= b;
    }
    return (double)num / (double)den;
}

// ordered selection of the first N Halton points (indices skip+1, ...) in the
// unit ball; one CTA of 1024 threads walks the candidates in chunks
__global__ void __launch_bounds__(1024) halton_ball(long long skip, int N, double *__restrict__ y,
                                                    int *__restrict__ status) {
    __shared__ int warp_cnt[32];
    __shared__ int base_cnt;
    if (threadIdx.x == 0) base_cnt = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (long long c0 = skip + 1; c0 < skip + 1 + 64ll * N + 4096; c0 += blockDim.x) {
        const long long i = c0 + threadIdx.x;
        double v[4];
        const int bases[4] = {2, 3, 5, 7};
        for (int a = 0; a < 4; ++a) v[a] = __dsub_rn(__dmul_rn(2.0, radical_inverse(i, bases[a])), 1.0);
        // sum of squares in a fixed order, no contraction (the same rounding as a plain evaluation)
        double r2 = __dmul_rn(v[0], v[0]);
        r2 = __dadd_rn(r2, __dmul_rn(v[1], v[1]));
        r2 = __dadd_rn(r2, __dmul_rn(v[2], v[2]));
        r2 = __dadd_rn(r2, __dmul_rn(v[3], v[3]));
        const bool in = r2 <= 1.0;
        const unsigned bal = __ballot_sync(0xffffffffu, in);
        if (lane == 0) warp_cnt[wid] = __popc(bal);
        __syncthreads();
        int before = base_cnt;
        for (int q = 0; q < wid; ++q) before += warp_cnt[q];
        const int pos = before + __popc(bal & ((1u << lane) - 1u));
        if (in && pos < N)
            for (int a = 0; a < 4; ++a) y[(size_t)pos * 4 + a] = v[a];
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int q = 0; q < 32; ++q) tot += warp_cnt[q];
            base_cnt += tot;
        }
        __syncthreads();
        if (base_cnt >= N) break;
    }
    if (threadIdx.x == 0) *status = base_cnt >= N ? 0 : 1;
}

WaveDev wave_dev(const mf_wave &w) {
    WaveDev d;
    memset(&d, 0, sizeof(d));
    d.n_modes = w.n_modes;
    d.L = w.L;
    d.nf = w.L / 2 + 1;
    for (int mu = 0; mu < w.n_modes; ++mu) d.em[mu] = w.ell_m[mu][1];
    d.f_lo = w.f_lo;
    d.f_hi = w.f_hi;
    d.f_ref = w.f_ref;
    d.df = 1.0 / ((double)w.L * w.dt);
    d.cut_rate = w.cut_rate;
    for (int a = 0; a < 4; ++a) d.cut_dir[a] = w.cut_dir[a];
    return d;
}

int check_wave(const mf_wave *w) {
    if (!w || w->n_modes < 1 || w->n_modes > kMaxModes || w->L < 16 || w->L > kMaxL || (w->L & (w->L - 1)) ||
        !(w->dt > 0) || !(w->f_ref > 0) || !(w->f_hi > 0) || !(w->f_lo >= 0) || !std::isfinite(w->cut_rate))
        return MF_E_INVAL;
    for (int mu = 0; mu < w->n_modes; ++mu)
        if (w->ell_m[mu][1] < 1 || w->ell_m[mu][0] < w->ell_m[mu][1]) return MF_E_INVAL;
    return MF_OK;
}

struct DevTables {
    double *U = nullptr, *A = nullptr;
    double2 *tw = nullptr;
    ~DevTables() {
        if (U) cudaFree(U);
        if (A) cudaFree(A);
        if (tw) cudaFree(tw);
    }
    int make(const mf_wave &w, cudaStream_t st) {
        const int nf = w.L / 2 + 1;
        MF_CUDA(cudaMalloc((void **)&U, sizeof(double) * 4 * nf * w.n_modes));
        MF_CUDA(cudaMalloc((void **)&A, sizeof(double) * nf * w.n_modes));
        MF_CUDA(cudaMalloc((void **)&tw, sizeof(double2) * (w.L / 2)));
        wave_tables<<<dim3((nf + 255) / 256, w.n_modes), 256, 0, st>>>(w, nf, 1.0 / ((double)w.L * w.dt), U, A);
        twiddles<<<(w.L / 2 + 255) / 256, 256, 0, st>>>(w.L, tw);
        MF_CUDA(cudaGetLastError());
        return MF_OK;
    }
};

int ilog2(int L) {
    int s = 0;
    while ((1 << s) < L) ++s;
    return s;
}

}  // namespace
}  // namespace mf

using namespace mf;

extern "C" int mf_place_nodes(const double *metric, const double *centre, double mismatch, double squeeze, int N,
                              long long skip, double *theta, double *y, double *frame) {
    if (!metric || !centre || !theta || N < 1 || N > (1 << 20) || !(mismatch > 0 && mismatch < 1) ||
        !(squeeze > 0 && squeeze <= 1) || skip < 0 || skip > (1ll << 40))
        return MF_E_INVAL;
    double R[16];
    int rc = metric_eig(metric, R);
    if (rc) return rc;
    double a[4];
    for (int d = 0; d < 4; ++d) {
        double lam = 0.0;
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) lam += R[4 * d + i] * metric[4 * i + j] * R[4 * d + j];
        a[d] = std::sqrt(mismatch / lam);
    }
    a[0] *= squeeze;
    double *dy = nullptr;
    int *dst = nullptr;
    MF_CUDA(cudaMalloc((void **)&dy, sizeof(double) * 4 * (size_t)N));
    if (cudaMalloc((void **)&dst, sizeof(int)) != cudaSuccess) {
        cudaFree(dy);
        return MF_E_NOMEM;
    }
    halton_ball<<<1, 1024>>>(skip, N, dy, dst);
    std::vector<double> hy((size_t)4 * N);
    int hst = 1;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(hy.data(), dy, sizeof(double) * 4 * (size_t)N, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&hst, dst, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(dy);
    cudaFree(dst);
    if (e != cudaSuccess) return cuda_status(e);
    if (hst) return MF_E_INVAL;
    // theta = c + R^T (a * y); frame A = diag(1/a) R maps theta - c back to y
    for (int n = 0; n < N; ++n)
        for (int i = 0; i < 4; ++i) {
            double t = centre[i];
            for (int d = 0; d < 4; ++d) t += R[4 * d + i] * a[d] * hy[(size_t)4 * n + d];
            theta[(size_t)4 * n + i] = t;
        }
    if (y) std::copy(hy.begin(), hy.end(), y);
    if (frame)
        for (int d = 0; d < 4; ++d)
            for (int i = 0; i < 4; ++i) frame[4 * d + i] = R[4 * d + i] / a[d];
    return MF_OK;
}

extern "C" int mf_standin_overlaps(const mf_wave *w, const double *theta, int N, const double *data,
                                   const double *psd, int n_det, int M, double *z, double *sigma, void *stream) {
    int rc = check_wave(w);
    if (rc) return rc;
    if (!theta || !data || !psd || !z || !sigma || N < 1 || n_det < 1 || n_det > kMaxDet || M < 1 || M > w->L)
        return MF_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const int nf = w->L / 2 + 1, nm = w->n_modes, L = w->L, logL = ilog2(L);
    DevTables T;
    rc = T.make(*w, st);
    if (rc) return rc;
    double *dth = nullptr, *dpsd = nullptr;
    double2 *ddata = nullptr, *dz = nullptr, *dsig = nullptr;
    auto cleanup = [&]() {
        for (void *p : {(void *)dth, (void *)dpsd, (void *)ddata, (void *)dz, (void *)dsig})
            if (p) cudaFree(p);
    };
    cudaError_t e;
    if ((e = cudaMalloc((void **)&dth, sizeof(double) * 4 * (size_t)N)) != cudaSuccess ||
        (e = cudaMalloc((void **)&dpsd, sizeof(double) * (size_t)n_det * nf)) != cudaSuccess ||
        (e = cudaMalloc((void **)&ddata, sizeof(double2) * (size_t)n_det * nf)) != cudaSuccess ||
        (e = cudaMalloc((void **)&dz, sizeof(double2) * (size_t)n_det * nm * N * M)) != cudaSuccess ||
        (e = cudaMalloc((void **)&dsig, sizeof(double2) * (size_t)n_det * N * nm * nm)) != cudaSuccess) {
        cleanup();
        return cuda_status(e);
    }
    WaveDev wd = wave_dev(*w);
    const size_t smem = sizeof(double2) * (size_t)L;
    if ((e = cudaMemcpyAsync(dth, theta, sizeof(double) * 4 * (size_t)N, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(dpsd, psd, sizeof(double) * (size_t)n_det * nf, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(ddata, data, sizeof(double2) * (size_t)n_det * nf, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(overlap_fft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) {
        cleanup();
        return cuda_status(e);
    }
    overlap_fft<<<dim3((unsigned)N, (unsigned)nm), kFftThreads, smem, st>>>(wd, logL, T.U, T.A, T.tw, dth, N, ddata,
                                                                            dpsd, n_det, M, dz);
    cross_terms<<<(unsigned)N, 256, 0, st>>>(wd, T.U, T.A, dth, N, dpsd, n_det, dsig);
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(z, dz, sizeof(double2) * (size_t)n_det * nm * N * M, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(sigma, dsig, sizeof(double2) * (size_t)n_det * N * nm * nm, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess) {
        cleanup();
        return cuda_status(e);
    }
    cleanup();
    return MF_OK;
}

extern "C" int mf_squeeze_factor(const mf_wave *w, const double *psd, const double *metric, const double *centre,
                                 double mismatch, int n_t, double *kappa, double *match_out) {
    int rc = check_wave(w);
    if (rc) return rc;
    if (!psd || !metric || !centre || !kappa || n_t < 1 || n_t > 4096 || !(mismatch > 0 && mismatch < 1))
        return MF_E_INVAL;
    double R[16];
    rc = metric_eig(metric, R);
    if (rc) return rc;
    double lam0 = 0.0;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) lam0 += R[i] * metric[4 * i + j] * R[j];
    const double a0 = std::sqrt(mismatch / lam0);
    std::vector<double> tb((size_t)4 * n_t);
    for (int b = 0; b < n_t; ++b) {
        const double t = (double)(b + 1) / (double)n_t;
        for (int i = 0; i < 4; ++i) tb[(size_t)4 * b + i] = centre[i] + R[i] * (t * a0);
    }
    const int nf = w->L / 2 + 1, L = w->L, logL = ilog2(L);
    DevTables T;
    rc = T.make(*w, nullptr);
    if (rc) return rc;
    double *dA = nullptr, *dB = nullptr, *dpsd = nullptr, *dout = nullptr;
    auto cleanup = [&]() {
        for (void *p : {(void *)dA, (void *)dB, (void *)dpsd, (void *)dout})
            if (p) cudaFree(p);
    };
    cudaError_t e;
    if ((e = cudaMalloc((void **)&dA, sizeof(double) * 4)) != cudaSuccess ||
        (e = cudaMalloc((void **)&dB, sizeof(double) * 4 * (size_t)n_t)) != cudaSuccess ||
        (e = cudaMalloc((void **)&dpsd, sizeof(double) * nf)) != cudaSuccess ||
        (e = cudaMalloc((void **)&dout, sizeof(double) * n_t)) != cudaSuccess) {
        cleanup();
        return cuda_status(e);
    }
    const size_t smem = sizeof(double2) * (size_t)L;
    std::vector<double> m(n_t);
    if ((e = cudaMemcpy(dA, centre, sizeof(double) * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(dB, tb.data(), sizeof(double) * 4 * (size_t)n_t, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(dpsd, psd, sizeof(double) * nf, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(match_fft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) {
        cleanup();
        return cuda_status(e);
    }
    match_fft<<<(unsigned)n_t, kFftThreads, smem>>>(wave_dev(*w), logL, T.U, T.A, T.tw, dA, dB, dpsd, dout);
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpy(m.data(), dout, sizeof(double) * n_t, cudaMemcpyDeviceToHost)) != cudaSuccess) {
        cleanup();
        return cuda_status(e);
    }
    cleanup();
    // first crossing of 1 - mismatch, linearly interpolated (1 if none)
    const double target = 1.0 - mismatch;
    double k = 1.0, pt = 0.0, pm = 1.0;
    for (int b = 0; b < n_t; ++b) {
        const double t = (double)(b + 1) / (double)n_t;
        if (m[b] < target) {
            k = pt + (t - pt) * (pm - target) / (pm - m[b]);
            break;
        }
        pt = t;
        pm = m[b];
    }
    *kappa = k;
    if (match_out) std::copy(m.begin(), m.end(), match_out);
    return MF_OK;
}
