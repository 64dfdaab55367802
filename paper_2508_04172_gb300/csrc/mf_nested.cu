// Nested sampling driver over the online likelihood (Sec. II D; the paper
// samples with nested sampling, random-walk proposals, in the metric
// eigenbasis Delta-e, Sec. III C), and importance reweighting to a target
// prior with the effective sample size N_eff = (sum w)^2 / sum w^2 (Sec. III A).
//
// State of a point (D = 9, or 11 with sky-dependent patterns), uniform prior
// on the domain:
//   0..3  x    in the Delta-e ball |x| <= r_ball (intrinsic; theta = c + R^T x)
//   4     u    in [0, 1]: d_L^3 = dl_min^3 + u (dl_max^3 - dl_min^3) (uniform in volume)
//   5     cos iota in [-1, 1]
//   6     psi  in [0, pi)   (periodic)
//   7     phi_c in [0, 2 pi) (periodic)
//   8     t_c  in [-tc_half, tc_half]
//   9     alpha in [0, 2 pi) (periodic; sky mode)
//   10    sin delta in [-1, 1] (sky mode)
// Iteration: the `batch` lowest-likelihood live points die (ascending lnL;
// the j-th removed of N live shrinks log X by 1 / (N - j)); each is replaced
// by a copy of a surviving live point moved by `walks` random-walk steps
// v' = v + scale sd_d z_d (sd_d the live points' standard deviation per
// dimension, z standard normal), a step being kept when v' lies in the domain
// and lnL(v') > L*, the largest lnL that died.  All walkers move together:
// one proposal kernel, one mf_loglike call over the batch, one acceptance
// kernel per step.  The scale adapts after each iteration as
// scale *= exp(acc - 0.5) (acc = accepted fraction of the steps).
// Random numbers: output number `c` of the splitmix64 generator seeded
// with `seed` (counter-based, identical on host and device):
//   c = ((iter * 65536 + walker) * 1024 + step) * 64 + slot.
#include "mf_internal.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <numeric>
#include <vector>

namespace mf {
namespace {

constexpr int kMaxDim = 11;
constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr double kPi = 3.1415926535897932384626433832795;

__host__ __device__ __forceinline__ uint64_t sm64(uint64_t seed, uint64_t c) {
    uint64_t z = seed + (c + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ double uni(uint64_t seed, uint64_t c) {
    return (double)(sm64(seed, c) >> 11) * (1.0 / 9007199254740992.0);   // [0, 1)
}
__host__ __device__ __forceinline__ uint64_t ctr(uint64_t iter, uint64_t walker, uint64_t step, uint64_t slot) {
    return ((iter * 65536ull + walker) * 1024ull + step) * 64ull + slot;
}
// standard normal number d of (iter, walker, step): Box-Muller on slots 2d, 2d+1
__host__ __device__ __forceinline__ double gauss(uint64_t seed, uint64_t iter, uint64_t walker, uint64_t step, int d) {
    const double u1 = 1.0 - uni(seed, ctr(iter, walker, step, 2 * d));
    const double u2 = uni(seed, ctr(iter, walker, step, 2 * d + 1));
    return sqrt(-2.0 * log(u1)) * cos(kTwoPi * u2);
}

struct Domain {
    int D;
    double r_ball, dl_min3, dl_max3, tc_half;
};

// periodic dimensions wrap; returns false outside the domain
__host__ __device__ __forceinline__ bool in_domain(const Domain &dm, double *v) {
    const double r2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + v[3] * v[3];
    if (!(r2 <= dm.r_ball * dm.r_ball)) return false;
    if (!(v[4] >= 0.0 && v[4] <= 1.0)) return false;
    if (!(v[5] >= -1.0 && v[5] <= 1.0)) return false;
    v[6] -= kPi * floor(v[6] / kPi);
    v[7] -= kTwoPi * floor(v[7] / kTwoPi);
    if (!(fabs(v[8]) <= dm.tc_half)) return false;
    if (dm.D > 9) {
        v[9] -= kTwoPi * floor(v[9] / kTwoPi);
        if (!(v[10] >= -1.0 && v[10] <= 1.0)) return false;
    }
    return true;
}

struct Frame {
    double R[16], c[4];
};

// state -> sampler-frame intrinsic row and extrinsic row (FP32, as mf_loglike takes them)
__device__ __forceinline__ void to_query(const Domain &dm, const Frame &f, const double *v, float *th, float *ex,
                                         int E) {
    for (int i = 0; i < 4; ++i) {
        double t = f.c[i];
        for (int k = 0; k < 4; ++k) t += f.R[4 * k + i] * v[k];   // theta = c + R^T x
        th[i] = (float)t;
    }
    ex[0] = (float)cbrt(dm.dl_min3 + v[4] * (dm.dl_max3 - dm.dl_min3));
    ex[1] = (float)v[5];
    ex[2] = (float)v[6];
    ex[3] = (float)v[7];
    ex[4] = (float)v[8];
    if (E >= 7) {
        ex[5] = (float)(dm.D > 9 ? v[9] : 0.0);
        ex[6] = (float)(dm.D > 9 ? asin(v[10]) : 0.0);
    }
}

// initial live points: uniform on the domain (rejection for the ball)
__global__ void ns_init(Domain dm, Frame f, uint64_t seed, int n, double *__restrict__ V, float *__restrict__ th,
                        float *__restrict__ ex, int E) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= n) return;
    double v[kMaxDim];
    for (int t = 0; t < 1000; ++t) {   // ball acceptance 0.31: 1000 tries never run out in practice
        for (int d = 0; d < 4; ++d) v[d] = dm.r_ball * (2.0 * uni(seed, ctr(0, w, t, d)) - 1.0);
        if (v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + v[3] * v[3] <= dm.r_ball * dm.r_ball) break;
    }
    v[4] = uni(seed, ctr(0, w, 1000, 4));
    v[5] = 2.0 * uni(seed, ctr(0, w, 1000, 5)) - 1.0;
    v[6] = kPi * uni(seed, ctr(0, w, 1000, 6));
    v[7] = kTwoPi * uni(seed, ctr(0, w, 1000, 7));
    v[8] = dm.tc_half * (2.0 * uni(seed, ctr(0, w, 1000, 8)) - 1.0);
    if (dm.D > 9) {
        v[9] = kTwoPi * uni(seed, ctr(0, w, 1000, 9));
        v[10] = 2.0 * uni(seed, ctr(0, w, 1000, 10)) - 1.0;
    }
    for (int d = 0; d < dm.D; ++d) V[(size_t)w * dm.D + d] = v[d];
    to_query(dm, f, v, th + (size_t)w * 4, ex + (size_t)w * E, E);
}

// proposal of walker w at step s: P[w] = V[w] + scale sd z (flag 0 if outside)
__global__ void ns_propose(Domain dm, Frame f, uint64_t seed, uint64_t iter, int step, int k,
                           const double *__restrict__ V, const double *__restrict__ sd, const double *__restrict__ scale,
                           double *__restrict__ P, unsigned char *__restrict__ ok, float *__restrict__ th,
                           float *__restrict__ ex, int E) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= k) return;
    double v[kMaxDim];
    const double sc = *scale;
    for (int d = 0; d < dm.D; ++d) v[d] = V[(size_t)w * dm.D + d] + sc * sd[d] * gauss(seed, iter, w, step, d);
    const bool in = in_domain(dm, v);
    for (int d = 0; d < dm.D; ++d) P[(size_t)w * dm.D + d] = v[d];
    ok[w] = in ? 1 : 0;
    // an out-of-domain proposal is still evaluated (at the walker's own point)
    // so that the batch stays one fixed-size call; it is never accepted
    to_query(dm, f, in ? v : V + (size_t)w * dm.D, th + (size_t)w * 4, ex + (size_t)w * E, E);
}

__global__ void ns_accept(int D, int k, const double *__restrict__ lstar, const double *__restrict__ P,
                          const unsigned char *__restrict__ ok, const float *__restrict__ lnl_new,
                          double *__restrict__ V, double *__restrict__ L, unsigned long long *__restrict__ n_acc) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= k) return;
    const double l = (double)lnl_new[w];
    if (ok[w] && l > *lstar) {
        for (int d = 0; d < D; ++d) V[(size_t)w * D + d] = P[(size_t)w * D + d];
        L[w] = l;
        atomicAdd(n_acc, 1ull);
    }
}

// diagnostic likelihood: lnL = -|x - mu|^2 / (2 s^2) on the intrinsic part
__global__ void ns_gauss_lnl(const float *__restrict__ th, const Frame f, double s, const double *__restrict__ mu,
                             int n, float *__restrict__ out, double *__restrict__ out64) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= n) return;
    double r2 = 0.0;
    for (int i = 0; i < 4; ++i) {
        double x = 0.0;
        for (int j = 0; j < 4; ++j) x += f.R[4 * i + j] * ((double)th[(size_t)w * 4 + j] - f.c[j]);
        const double d = x - mu[i];
        r2 += d * d;
    }
    const double l = -0.5 * r2 / (s * s);
    out[w] = (float)l;
    if (out64) out64[w] = l;
}

double logaddexp(double a, double b) {
    if (a == -INFINITY) return b;
    if (b == -INFINITY) return a;
    const double m = std::max(a, b);
    return m + std::log1p(std::exp(-std::fabs(a - b)));
}

}  // namespace
}  // namespace mf

using namespace mf;

extern "C" int mf_nested_sample(mf_handle *h, const mf_ns_params *p, mf_ns_result *res, double *out_v,
                                double *out_lnl, double *out_logwt, int max_out, void *stream) {
    if (!p || !res || p->n_live < 8 || p->n_live > 65536 || p->batch < 1 || p->batch >= p->n_live ||
        p->walks < 1 || p->walks > 1000 || !(p->dlogz > 0) || p->max_iter < 1 || p->max_iter > (1 << 20) ||
        !(p->r_ball > 0) || !(p->dl_min > 0) || !(p->dl_max > p->dl_min) || !(p->tc_half > 0))
        return MF_E_INVAL;
    if (max_out < 0 || (max_out > 0 && (!out_v || !out_lnl || !out_logwt))) return MF_E_INVAL;
    const bool gauss_test = p->test_sigma > 0;
    if (!gauss_test) {
        if (!h) return MF_E_INVAL;
        if (!h->have_layout || !h->have_basis || !h->have_det) return MF_E_STATE;
    }
    const bool sky = !gauss_test && h->sky;
    const int D = sky ? 11 : 9;
    const int E = sky ? 7 : 5;
    const int N = p->n_live, k = p->batch;
    cudaStream_t st = (cudaStream_t)stream;
    Domain dm{D, p->r_ball, p->dl_min * p->dl_min * p->dl_min, p->dl_max * p->dl_max * p->dl_max, p->tc_half};
    Frame fr;
    if (h) {
        for (int i = 0; i < 16; ++i) fr.R[i] = h->R[i];
        for (int i = 0; i < 4; ++i) fr.c[i] = h->centre[i];
    } else {
        for (int i = 0; i < 16; ++i) fr.R[i] = (i % 5 == 0) ? 1.0 : 0.0;
        for (int i = 0; i < 4; ++i) fr.c[i] = 0.0;
    }
    const uint64_t seed = p->seed;
    // device buffers
    double *dV = nullptr, *dL = nullptr, *dW = nullptr, *dWL = nullptr, *dP = nullptr, *dsd = nullptr,
           *dscale = nullptr, *dlstar = nullptr, *dmu = nullptr, *dL64 = nullptr;
    float *dth = nullptr, *dex = nullptr, *dout = nullptr;
    unsigned char *dok = nullptr;
    unsigned long long *dacc = nullptr;
    auto cleanup = [&]() {
        for (void *q : {(void *)dV, (void *)dL, (void *)dW, (void *)dWL, (void *)dP, (void *)dsd, (void *)dscale,
                        (void *)dlstar, (void *)dmu, (void *)dL64, (void *)dth, (void *)dex, (void *)dout,
                        (void *)dok, (void *)dacc})
            if (q) cudaFree(q);
    };
    auto fail = [&](cudaError_t e) { cleanup(); return cuda_status(e); };
    cudaError_t e = cudaSuccess;
#define NS_ALLOC(ptr, bytes) \
    if ((e = cudaMalloc((void **)&ptr, bytes)) != cudaSuccess) return fail(e)
    NS_ALLOC(dV, sizeof(double) * N * D);
    NS_ALLOC(dL, sizeof(double) * N);
    NS_ALLOC(dW, sizeof(double) * k * D);
    NS_ALLOC(dWL, sizeof(double) * k);
    NS_ALLOC(dP, sizeof(double) * k * D);
    NS_ALLOC(dsd, sizeof(double) * D);
    NS_ALLOC(dscale, sizeof(double));
    NS_ALLOC(dlstar, sizeof(double));
    NS_ALLOC(dmu, sizeof(double) * 4);
    NS_ALLOC(dL64, sizeof(double) * N);
    NS_ALLOC(dth, sizeof(float) * 4 * N);
    NS_ALLOC(dex, sizeof(float) * E * N);
    NS_ALLOC(dout, sizeof(float) * N);
    NS_ALLOC(dok, k);
    NS_ALLOC(dacc, sizeof(unsigned long long));
#undef NS_ALLOC
    if ((e = cudaMemcpyAsync(dmu, p->test_mu, sizeof(double) * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return fail(e);
    long long n_like = 0;
    // likelihood of n rows of (dth, dex) into dout (FP32) and dL64 (FP64 copy)
    auto lnl = [&](int n) -> int {
        n_like += n;
        if (gauss_test) {
            ns_gauss_lnl<<<(n + 127) / 128, 128, 0, st>>>(dth, fr, p->test_sigma, dmu, n, dout, nullptr);
            return cudaGetLastError() == cudaSuccess ? MF_OK : MF_E_CUDA;
        }
        return mf_loglike(h, dth, dex, n, E, dout, stream);
    };
    const auto t_start = std::chrono::steady_clock::now();
    // initial live points
    ns_init<<<(N + 127) / 128, 128, 0, st>>>(dm, fr, seed, N, dV, dth, dex, E);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
    int rc = lnl(N);
    if (rc) { cleanup(); return rc; }
    std::vector<float> hl(N);
    std::vector<double> hL(N), hV((size_t)N * D);
    if ((e = cudaMemcpyAsync(hl.data(), dout, sizeof(float) * N, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(hV.data(), dV, sizeof(double) * N * D, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return fail(e);
    for (int i = 0; i < N; ++i) hL[i] = hl[i];
    double logX = 0.0, logZ = -INFINITY, Hacc = 0.0, scale = p->scale0 > 0 ? p->scale0 : 1.0;
    long long n_dead = 0, n_acc_tot = 0, n_steps_tot = 0;
    std::vector<int> order(N);
    std::vector<double> wk((size_t)k * D), wl(k), sd(D);
    int it = 0;
    bool converged = false;
    for (it = 1; it <= p->max_iter; ++it) {
        // the batch lowest live points die, in ascending lnL (ties by index)
        std::iota(order.begin(), order.end(), 0);
        std::sort(order.begin(), order.end(), [&](int a, int b) {
            return hL[a] < hL[b] || (hL[a] == hL[b] && a < b);
        });
        const double lstar = hL[order[k - 1]];
        for (int j = 0; j < k; ++j) {
            const int i = order[j];
            const double lx_new = logX - 1.0 / (double)(N - j);
            const double logw = hL[i] + logX + std::log1p(-std::exp(lx_new - logX));
            const double z_new = logaddexp(logZ, logw);
            // information H = sum_i w_i lnL_i / Z - log Z, accumulated as in Skilling's recursion
            Hacc = (logZ == -INFINITY ? 0.0 : std::exp(logZ - z_new) * (Hacc + logZ)) +
                   std::exp(logw - z_new) * hL[i] - z_new;
            logZ = z_new;
            if (n_dead < max_out) {
                for (int d = 0; d < D; ++d) out_v[n_dead * D + d] = hV[(size_t)i * D + d];
                out_lnl[n_dead] = hL[i];
                out_logwt[n_dead] = logw;
            }
            ++n_dead;
            logX = lx_new;
        }
        // stop when the live points can add less than dlogz to log Z
        double lmax = hL[order[N - 1]];
        if (logaddexp(logZ, logX + lmax) - logZ < p->dlogz) { converged = true; break; }
        // walkers start from surviving points chosen uniformly (host draws, slot 63 of step 1023)
        for (int j = 0; j < k; ++j) {
            const int pick = k + (int)(uni(seed, ctr(it, j, 1023, 63)) * (double)(N - k));
            const int src = order[std::min(pick, N - 1)];
            for (int d = 0; d < D; ++d) wk[(size_t)j * D + d] = hV[(size_t)src * D + d];
            wl[j] = hL[src];
        }
        // per-dimension spread of the surviving live points
        for (int d = 0; d < D; ++d) {
            double m = 0.0, s2 = 0.0;
            for (int q = k; q < N; ++q) m += hV[(size_t)order[q] * D + d];
            m /= (double)(N - k);
            for (int q = k; q < N; ++q) {
                const double t = hV[(size_t)order[q] * D + d] - m;
                s2 += t * t;
            }
            sd[d] = std::sqrt(s2 / (double)(N - k - 1 > 0 ? N - k - 1 : 1));
        }
        if ((e = cudaMemcpyAsync(dW, wk.data(), sizeof(double) * k * D, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(dWL, wl.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(dsd, sd.data(), sizeof(double) * D, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(dscale, &scale, sizeof(double), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(dlstar, &lstar, sizeof(double), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
            (e = cudaMemsetAsync(dacc, 0, sizeof(unsigned long long), st)) != cudaSuccess)
            return fail(e);
        for (int s = 0; s < p->walks; ++s) {
            ns_propose<<<(k + 127) / 128, 128, 0, st>>>(dm, fr, seed, (uint64_t)it, s, k, dW, dsd, dscale, dP, dok,
                                                         dth, dex, E);
            if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
            rc = lnl(k);
            if (rc) { cleanup(); return rc; }
            ns_accept<<<(k + 127) / 128, 128, 0, st>>>(D, k, dlstar, dP, dok, dout, dW, dWL, dacc);
            if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
        }
        unsigned long long nacc = 0;
        if ((e = cudaMemcpyAsync(wk.data(), dW, sizeof(double) * k * D, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(wl.data(), dWL, sizeof(double) * k, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(&nacc, dacc, sizeof(nacc), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return fail(e);
        // the walkers replace the dead points in place
        for (int j = 0; j < k; ++j) {
            const int i = order[j];
            for (int d = 0; d < D; ++d) hV[(size_t)i * D + d] = wk[(size_t)j * D + d];
            hL[i] = wl[j];
        }
        const double acc = (double)nacc / (double)((long long)k * p->walks);
        scale *= std::exp(acc - 0.5);
        n_acc_tot += (long long)nacc;
        n_steps_tot += (long long)k * p->walks;
    }
    // the remaining live points share the last volume equally
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int a, int b) { return hL[a] < hL[b] || (hL[a] == hL[b] && a < b); });
    for (int q = 0; q < N; ++q) {
        const int i = order[q];
        const double logw = hL[i] + logX - std::log((double)N);
        const double z_new = logaddexp(logZ, logw);
        Hacc = std::exp(logZ - z_new) * (Hacc + logZ) + std::exp(logw - z_new) * hL[i] - z_new;
        logZ = z_new;
        if (n_dead < max_out) {
            for (int d = 0; d < D; ++d) out_v[n_dead * D + d] = hV[(size_t)i * D + d];
            out_lnl[n_dead] = hL[i];
            out_logwt[n_dead] = logw;
        }
        ++n_dead;
    }
    const auto t_end = std::chrono::steady_clock::now();
    cleanup();
    res->logz = logZ;
    res->info = Hacc;
    res->logz_err = std::sqrt(std::max(Hacc, 0.0) / (double)N);
    res->n_samples = n_dead;
    res->n_like = n_like;
    res->iterations = converged ? it : p->max_iter;
    res->converged = converged ? 1 : 0;
    res->accept = n_steps_tot ? (double)n_acc_tot / (double)n_steps_tot : 0.0;
    res->scale = scale;
    res->dim = D;
    res->wall_ms = std::chrono::duration<double, std::milli>(t_end - t_start).count();
    return MF_OK;
}

extern "C" int mf_reweight(const double *logwt, const double *log_ratio, int n, double *w, double *n_eff) {
    if (!logwt || n < 1 || !w) return MF_E_INVAL;
    double m = -INFINITY;
    for (int i = 0; i < n; ++i) {
        const double a = logwt[i] + (log_ratio ? log_ratio[i] : 0.0);
        w[i] = a;
        m = std::max(m, a);
    }
    if (!std::isfinite(m)) return MF_E_INVAL;
    double s = 0.0, s2 = 0.0;
    for (int i = 0; i < n; ++i) {
        w[i] = std::exp(w[i] - m);
        s += w[i];
    }
    for (int i = 0; i < n; ++i) {
        w[i] /= s;
        s2 += w[i] * w[i];
    }
    if (n_eff) *n_eff = 1.0 / s2;   // (sum w)^2 / sum w^2 with sum w = 1
    return MF_OK;
}
