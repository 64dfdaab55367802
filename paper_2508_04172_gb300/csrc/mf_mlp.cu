// Surrogate network: a fully connected SiLU network n_in -> hidden x
// n_hidden -> n_out with FP32 master weights, BF16 GEMM operands and FP32
// accumulation.  Training runs entirely on the GPU (forward, MSE loss,
// backward, Adam), one step per replay of a captured CUDA graph.
//
// Layers l = 0 .. L-1 (L = n_hidden + 1): z_l = W_l h_{l-1} + b_l,
// h_l = SiLU(z_l) for l < L-1, y = z_{L-1}; h_{-1} = x.  Layer 0 has only
// n_in (<= 16) inputs and runs as plain FMAs; every other layer, forward
// and backward, is a tcgen05 GEMM with a fused epilogue:
//   forward     h_l      = SiLU(h_{l-1} W_l^T + b_l)             EPI_SILU
//   loss        dY       = 2 (y - t) / (B n_out), db_{L-1}       EPI_MSE
//   backward    dz_l     = (dz_{l+1} W_{l+1}) * SiLU'(z_l), db_l  EPI_DSILU
//               dW_l     = dz_l^T h_{l-1}                        EPI_F32
// Activations and back-propagated gradients are written both row-major and
// transposed so that every GEMM reads K-major operands.
#include "mf_mlp_kernels.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

struct mf_mlp {
    int n_in = 0, H = 0, nh = 0, n_out = 0, L = 0;
    long long n_params = 0;
    std::vector<int> off, in, out;                 // per layer: flat offset, fan-in, fan-out
    float *d_p = nullptr, *d_g = nullptr;          // master FP32 parameters, gradient
    float *d_m = nullptr, *d_v = nullptr;          // Adam moments
    std::vector<__nv_bfloat16 *> W, Wt;            // per layer BF16 [out][in], [in][out] (layer 0: none)
    mf::TrainState *d_st = nullptr;
    unsigned *d_err = nullptr;
    // workspace for `cap` rows
    int cap = 0;
    float *Xb = nullptr, *Tb = nullptr;
    std::vector<__nv_bfloat16 *> Hs, Hts, dZ, dZt;  // per hidden layer
    std::vector<float *> Zs;
    float *dZ0 = nullptr;
    __nv_bfloat16 *dY = nullptr, *dYt = nullptr;
    // training step for `plan_rows` rows
    int plan_rows = 0;
    std::vector<mf::GemmPlan> fwd, bwd;
    cudaStream_t cap_st = nullptr;
    cudaGraphExec_t step_exec = nullptr;
    float train_ms = 0.f;
    long long steps_done = 0;
};

namespace mf {
namespace {

const EpiParams &zero_epi() {
    static EpiParams z = [] {
        EpiParams e;
        memset(&e, 0, sizeof(e));
        return e;
    }();
    return z;
}

template <int EPI>
int launch_plan_epi(const GemmPlan &pl, const EpiParams &epi, int nm, cudaStream_t st) {
    const size_t smem = gemm_smem_bytes(pl.g.NT);
    dim3 grid((unsigned)((pl.g.M + kTile - 1) / kTile), (unsigned)pl.grid_y);
    void *kern = nullptr;
    if (EPI == EPI_LNL) {
        switch (nm) {
            case 1: kern = (void *)gemm_kernel<EPI_LNL, 1>; break;
            case 2: kern = (void *)gemm_kernel<EPI_LNL, 2>; break;
            case 3: kern = (void *)gemm_kernel<EPI_LNL, 3>; break;
            case 4: kern = (void *)gemm_kernel<EPI_LNL, 4>; break;
            case 5: kern = (void *)gemm_kernel<EPI_LNL, 5>; break;
            default: return MF_E_NOTIMPL;
        }
    } else {
        kern = (void *)gemm_kernel<EPI, 1>;
    }
    MF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    void *args[4] = {(void *)&pl.ta, (void *)&pl.tb, (void *)&pl.g, (void *)&epi};
    MF_CUDA(cudaLaunchKernel(kern, grid, dim3(kGemmThreads), args, smem, st));
    return MF_OK;
}

int launch_plan(const GemmPlan &pl, cudaStream_t st, const EpiParams *epi = nullptr, int nm = 1) {
    const EpiParams &e = epi ? *epi : zero_epi();
    switch (pl.epi) {
        case EPI_SILU: return launch_plan_epi<EPI_SILU>(pl, e, nm, st);
        case EPI_MSE: return launch_plan_epi<EPI_MSE>(pl, e, nm, st);
        case EPI_DSILU: return launch_plan_epi<EPI_DSILU>(pl, e, nm, st);
        case EPI_F32: return launch_plan_epi<EPI_F32>(pl, e, nm, st);
        case EPI_LNL: return launch_plan_epi<EPI_LNL>(pl, e, nm, st);
        default: return MF_E_INVAL;
    }
}

// C[M][N] = A[M][K] B[N][K]^T with A, B BF16 row-major; NT columns per CTA.
int make_plan(GemmPlan &pl, int epi, const void *A, int M, int K, const void *B, int N, int NT,
              const GemmArgs &g, unsigned *err) {
    if (NT < 16 || NT > 256 || NT % 16 || K % 8) return MF_E_INVAL;
    int rc = make_tmap(&pl.ta, const_cast<void *>(A), 1, K, M, kTile);
    if (rc) return rc;
    rc = make_tmap(&pl.tb, const_cast<void *>(B), 1, K, N, NT);
    if (rc) return rc;
    pl.g = g;
    pl.g.M = M;
    pl.g.N = N;
    pl.g.K = K;
    pl.g.NT = NT;
    pl.g.err = err;
    pl.epi = epi;
    pl.grid_y = (N + NT - 1) / NT;
    return MF_OK;
}

int nt_for(int n) { return std::min(256, (n + 15) / 16 * 16); }

LayerTab layer_tab(const mf_mlp *m) {
    LayerTab t;
    memset(&t, 0, sizeof(t));
    t.n_layers = m->L;
    for (int l = 0; l < m->L; ++l) {
        t.off[l] = m->off[l];
        t.in[l] = m->in[l];
        t.out[l] = m->out[l];
        t.W[l] = m->W[l];
        t.Wt[l] = m->Wt[l];
    }
    t.off[m->L] = (int)m->n_params;
    return t;
}

void free_work(mf_mlp *m) {
    auto fr = [](void *p) { if (p) cudaFree(p); };
    fr(m->Xb); fr(m->Tb); fr(m->dZ0); fr(m->dY); fr(m->dYt);
    for (auto p : m->Hs) fr(p);
    for (auto p : m->Hts) fr(p);
    for (auto p : m->dZ) fr(p);
    for (auto p : m->dZt) fr(p);
    for (auto p : m->Zs) fr(p);
    m->Xb = m->Tb = m->dZ0 = nullptr;
    m->dY = m->dYt = nullptr;
    m->Hs.clear(); m->Hts.clear(); m->dZ.clear(); m->dZt.clear(); m->Zs.clear();
    m->cap = 0;
    m->plan_rows = 0;
    if (m->step_exec) cudaGraphExecDestroy(m->step_exec);
    m->step_exec = nullptr;
}

int ensure_work(mf_mlp *m, int rows) {
    if (rows <= m->cap) return MF_OK;
    free_work(m);
    const size_t R = (size_t)rows, H = (size_t)m->H;
    auto al = [](void **p, size_t bytes) { return cudaMalloc(p, bytes) == cudaSuccess; };
    bool ok = al((void **)&m->Xb, 4 * R * m->n_in) && al((void **)&m->Tb, 4 * R * m->n_out) &&
              al((void **)&m->dZ0, 4 * R * H) && al((void **)&m->dY, 2 * R * m->n_out) &&
              al((void **)&m->dYt, 2 * R * m->n_out);
    for (int l = 0; l < m->nh && ok; ++l) {
        __nv_bfloat16 *a = nullptr, *b = nullptr, *c = nullptr, *d = nullptr;
        float *z = nullptr;
        ok = al((void **)&a, 2 * R * H) && al((void **)&b, 2 * R * H) && al((void **)&c, 2 * R * H) &&
             al((void **)&d, 2 * R * H) && al((void **)&z, 4 * R * H);
        m->Hs.push_back(a);
        m->Hts.push_back(b);
        m->dZ.push_back(c);
        m->dZt.push_back(d);
        m->Zs.push_back(z);
    }
    if (!ok) {
        cudaGetLastError();
        free_work(m);
        return MF_E_NOMEM;
    }
    m->cap = rows;
    return MF_OK;
}

// GEMM plans of one training step on `rows` rows of Xb/Tb (forward with
// saved activations, loss, backward).
int build_train_plans(mf_mlp *m, int rows) {
    if (m->plan_rows == rows) return MF_OK;
    m->fwd.clear();
    m->bwd.clear();
    if (m->step_exec) cudaGraphExecDestroy(m->step_exec);
    m->step_exec = nullptr;
    const int H = m->H, L = m->L, nh = m->nh;
    int rc;
    for (int l = 1; l < nh; ++l) {   // hidden GEMM layers
        GemmArgs g{};
        g.bias = m->d_p + m->off[l] + H * H;
        g.out_bf = m->Hs[l];
        g.out_t = m->Hts[l];
        g.out_f = m->Zs[l];
        GemmPlan pl;
        rc = make_plan(pl, EPI_SILU, m->Hs[l - 1], rows, H, m->W[l], H, nt_for(H), g, m->d_err);
        if (rc) return rc;
        m->fwd.push_back(pl);
    }
    {   // output layer + loss
        const int lo = L - 1;
        GemmArgs g{};
        g.bias = m->d_p + m->off[lo] + m->n_out * H;
        g.aux = m->Tb;
        g.out_bf = m->dY;
        g.out_t = m->dYt;
        g.colsum = m->d_g + m->off[lo] + m->n_out * H;
        g.loss = &m->d_st->loss_acc;
        g.gscale = 2.f / ((float)rows * (float)m->n_out);
        GemmPlan pl;
        rc = make_plan(pl, EPI_MSE, m->Hs[nh - 1], rows, H, m->W[lo], m->n_out, nt_for(m->n_out), g, m->d_err);
        if (rc) return rc;
        m->fwd.push_back(pl);
    }
    // backward: for each layer from the output down, its weight gradient and
    // the gradient of the layer below
    for (int l = L - 1; l >= 1; --l) {
        const __nv_bfloat16 *dz = (l == L - 1) ? m->dY : m->dZ[l];
        const __nv_bfloat16 *dzt = (l == L - 1) ? m->dYt : m->dZt[l];
        {   // dW_l = dz_l^T h_{l-1}:  [out_l][B] x [in_l][B]^T
            GemmArgs g{};
            g.out_f = m->d_g + m->off[l];
            GemmPlan pl;
            rc = make_plan(pl, EPI_F32, dzt, m->out[l], rows, m->Hts[l - 1], m->in[l], 64, g, m->d_err);
            if (rc) return rc;
            m->bwd.push_back(pl);
        }
        {   // dz_{l-1} = (dz_l W_l) * SiLU'(z_{l-1}):  [B][out_l] x [in_l][out_l]^T
            GemmArgs g{};
            g.aux = m->Zs[l - 1];
            g.colsum = m->d_g + m->off[l - 1] + m->out[l - 1] * m->in[l - 1];
            if (l - 1 >= 1) {
                g.out_bf = m->dZ[l - 1];
                g.out_t = m->dZt[l - 1];
            } else {
                g.out_f = m->dZ0;
            }
            GemmPlan pl;
            rc = make_plan(pl, EPI_DSILU, dz, rows, m->out[l], m->Wt[l], m->in[l], nt_for(m->in[l]), g,
                           m->d_err);
            if (rc) return rc;
            m->bwd.push_back(pl);
        }
    }
    m->plan_rows = rows;
    return MF_OK;
}

// Forward + backward on Xb/Tb (rows rows); gradients accumulate into d_g
// (zeroed beforehand), the loss sum into the train state.
int enqueue_fwd_bwd(mf_mlp *m, int rows, cudaStream_t st) {
    const int H = m->H;
    const long long n0 = (long long)rows * H;
    layer1_kernel<<<(unsigned)((n0 + 255) / 256), 256, 0, st>>>(m->Xb, rows, m->n_in, m->d_p, m->d_p + H * m->n_in,
                                                                H, m->Hs[0], m->Hts[0], m->Zs[0]);
    MF_CUDA(cudaGetLastError());
    for (auto &pl : m->fwd) {
        int rc = launch_plan(pl, st);
        if (rc) return rc;
    }
    for (auto &pl : m->bwd) {
        int rc = launch_plan(pl, st);
        if (rc) return rc;
    }
    layer1_wgrad_kernel<<<H, 256, 0, st>>>(m->dZ0, m->Xb, rows, m->n_in, H, m->d_g);
    MF_CUDA(cudaGetLastError());
    return MF_OK;
}

int refresh_copies(mf_mlp *m, cudaStream_t st) {
    adam_kernel<<<256, 256, 0, st>>>(m->d_p, m->d_g, m->d_m, m->d_v, (int)m->n_params, layer_tab(m), m->d_st, 0);
    MF_CUDA(cudaGetLastError());
    return MF_OK;
}

uint64_t splitmix(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void destroy_mlp(mf_mlp *m) {
    if (!m) return;
    free_work(m);
    auto fr = [](void *p) { if (p) cudaFree(p); };
    fr(m->d_p); fr(m->d_g); fr(m->d_m); fr(m->d_v); fr(m->d_st); fr(m->d_err);
    for (auto p : m->W) fr(p);
    for (auto p : m->Wt) fr(p);
    if (m->cap_st) cudaStreamDestroy(m->cap_st);
    delete m;
}

}  // namespace
}  // namespace mf

using namespace mf;

extern "C" {

int mf_mlp_create(int n_in, int hidden, int n_hidden, int n_out, unsigned long long seed, mf_mlp **out) {
    if (!out) return MF_E_INVAL;
    *out = nullptr;
    if (n_in < 1 || n_in > kMlpMaxIn || hidden < 16 || hidden > 256 || hidden % 16 || n_hidden < 1 ||
        n_hidden + 1 > kMlpMaxLayers || n_out < 8 || n_out % 8 || n_out > (1 << 16))
        return MF_E_INVAL;
    mf_mlp *m = new (std::nothrow) mf_mlp();
    if (!m) return MF_E_NOMEM;
    m->n_in = n_in;
    m->H = hidden;
    m->nh = n_hidden;
    m->n_out = n_out;
    m->L = n_hidden + 1;
    long long p = 0;
    for (int l = 0; l < m->L; ++l) {
        const int fi = l == 0 ? n_in : hidden, fo = l == m->L - 1 ? n_out : hidden;
        m->off.push_back((int)p);
        m->in.push_back(fi);
        m->out.push_back(fo);
        p += (long long)fi * fo + fo;
    }
    m->n_params = p;
    // PyTorch-style initialisation U(-1/sqrt(fan_in), 1/sqrt(fan_in)), seeded
    std::vector<float> h(p);
    uint64_t s = seed;
    for (int l = 0; l < m->L; ++l) {
        const double a = 1.0 / std::sqrt((double)m->in[l]);
        const long long n = (long long)m->in[l] * m->out[l] + m->out[l];
        for (long long i = 0; i < n; ++i)
            h[m->off[l] + i] = (float)(a * (2.0 * ((splitmix(s) >> 11) * (1.0 / 9007199254740992.0)) - 1.0));
    }
    bool ok = cudaMalloc((void **)&m->d_p, 4 * p) == cudaSuccess && cudaMalloc((void **)&m->d_g, 4 * p) == cudaSuccess &&
              cudaMalloc((void **)&m->d_m, 4 * p) == cudaSuccess && cudaMalloc((void **)&m->d_v, 4 * p) == cudaSuccess &&
              cudaMalloc((void **)&m->d_st, sizeof(TrainState)) == cudaSuccess &&
              cudaMalloc((void **)&m->d_err, 16 * sizeof(unsigned)) == cudaSuccess &&
              cudaStreamCreateWithFlags(&m->cap_st, cudaStreamNonBlocking) == cudaSuccess;
    for (int l = 0; l < m->L && ok; ++l) {
        __nv_bfloat16 *a = nullptr, *b = nullptr;
        if (l > 0)
            ok = cudaMalloc((void **)&a, 2 * (size_t)m->in[l] * m->out[l]) == cudaSuccess &&
                 cudaMalloc((void **)&b, 2 * (size_t)m->in[l] * m->out[l]) == cudaSuccess;
        m->W.push_back(a);
        m->Wt.push_back(b);
    }
    if (!ok) {
        cudaGetLastError();
        destroy_mlp(m);
        return MF_E_NOMEM;
    }
    cudaMemcpy(m->d_p, h.data(), 4 * p, cudaMemcpyHostToDevice);
    cudaMemset(m->d_g, 0, 4 * p);
    cudaMemset(m->d_m, 0, 4 * p);
    cudaMemset(m->d_v, 0, 4 * p);
    cudaMemset(m->d_st, 0, sizeof(TrainState));
    cudaMemset(m->d_err, 0, 16 * sizeof(unsigned));
    int rc = refresh_copies(m, nullptr);
    if (rc == MF_OK && cudaDeviceSynchronize() != cudaSuccess) rc = MF_E_CUDA;
    if (rc) {
        destroy_mlp(m);
        return rc;
    }
    *out = m;
    return MF_OK;
}

void mf_mlp_free(mf_mlp *m) { destroy_mlp(m); }

long long mf_mlp_n_params(const mf_mlp *m) { return m ? m->n_params : -1; }

int mf_mlp_set_params(mf_mlp *m, const float *host) {
    if (!m || !host) return MF_E_INVAL;
    MF_CUDA(cudaMemcpy(m->d_p, host, 4 * m->n_params, cudaMemcpyHostToDevice));
    int rc = refresh_copies(m, nullptr);
    if (rc) return rc;
    MF_CUDA(cudaDeviceSynchronize());
    return MF_OK;
}

int mf_mlp_get_params(const mf_mlp *m, float *host) {
    if (!m || !host) return MF_E_INVAL;
    MF_CUDA(cudaDeviceSynchronize());
    MF_CUDA(cudaMemcpy(host, m->d_p, 4 * m->n_params, cudaMemcpyDeviceToHost));
    return MF_OK;
}

int mf_mlp_forward(mf_mlp *m, const float *X, int B, float *Y, void *stream) {
    if (!m || B < 0 || B > (1 << 24)) return MF_E_INVAL;
    if (B == 0) return MF_OK;
    if (!X || !Y || ((uintptr_t)Y & 15)) return MF_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ensure_work(m, B);
    if (rc) return rc;
    const int H = m->H;
    const long long n0 = (long long)B * H;
    layer1_kernel<<<(unsigned)((n0 + 255) / 256), 256, 0, st>>>(X, B, m->n_in, m->d_p, m->d_p + H * m->n_in, H,
                                                                m->Hs[0], nullptr, nullptr);
    MF_CUDA(cudaGetLastError());
    for (int l = 1; l < m->L; ++l) {
        const bool last = l == m->L - 1;
        GemmArgs g{};
        g.bias = m->d_p + m->off[l] + m->out[l] * m->in[l];
        GemmPlan pl;
        if (last) {
            g.out_f = Y;
            rc = make_plan(pl, EPI_F32, m->Hs[l - 1], B, H, m->W[l], m->n_out, nt_for(m->n_out), g, m->d_err);
        } else {
            g.out_bf = m->Hs[l];
            rc = make_plan(pl, EPI_SILU, m->Hs[l - 1], B, H, m->W[l], H, nt_for(H), g, m->d_err);
        }
        if (rc) return rc;
        rc = launch_plan(pl, st);
        if (rc) return rc;
    }
    return MF_OK;
}

int mf_mlp_gradient(mf_mlp *m, const float *X, const float *T, int B, float *host_grad, double *host_loss,
                    void *stream) {
    if (!m || !X || !T || B < 8 || B % 8 || B > (1 << 22)) return MF_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ensure_work(m, B);
    if (rc) return rc;
    rc = build_train_plans(m, B);
    if (rc) return rc;
    MF_CUDA(cudaMemcpyAsync(m->Xb, X, 4 * (size_t)B * m->n_in, cudaMemcpyDeviceToDevice, st));
    MF_CUDA(cudaMemcpyAsync(m->Tb, T, 4 * (size_t)B * m->n_out, cudaMemcpyDeviceToDevice, st));
    MF_CUDA(cudaMemsetAsync(m->d_g, 0, 4 * m->n_params, st));
    MF_CUDA(cudaMemsetAsync(&m->d_st->loss_acc, 0, sizeof(float), st));
    rc = enqueue_fwd_bwd(m, B, st);
    if (rc) return rc;
    MF_CUDA(cudaStreamSynchronize(st));
    unsigned err = 0;
    MF_CUDA(cudaMemcpy(&err, m->d_err, sizeof(err), cudaMemcpyDeviceToHost));
    if (err) return MF_E_TIMEOUT;
    if (host_grad) MF_CUDA(cudaMemcpy(host_grad, m->d_g, 4 * m->n_params, cudaMemcpyDeviceToHost));
    if (host_loss) {
        float s = 0.f;
        MF_CUDA(cudaMemcpy(&s, &m->d_st->loss_acc, sizeof(float), cudaMemcpyDeviceToHost));
        *host_loss = (double)s / ((double)B * m->n_out);
    }
    MF_CUDA(cudaMemset(m->d_g, 0, 4 * m->n_params));
    return MF_OK;
}

int mf_mlp_train(mf_mlp *m, const float *X, const float *T, int n, const mf_mlp_train_params *tp,
                 void *stream) {
    if (!m || !X || !T || !tp || n < 1) return MF_E_INVAL;
    const int B = std::min(tp->batch, n);
    if (B < 8 || B % 8 || tp->steps < 0 || !(tp->lr > 0) || !(tp->lr_min >= 0)) return MF_E_INVAL;
    if (tp->steps == 0) return MF_OK;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ensure_work(m, B);
    if (rc) return rc;
    rc = build_train_plans(m, B);
    if (rc) return rc;
    TrainState s{};
    s.step = 0;
    s.total = tp->steps;
    s.lr_max = tp->lr;
    s.lr_min = tp->lr_min;
    s.beta1 = tp->beta1 > 0 ? tp->beta1 : 0.9f;
    s.beta2 = tp->beta2 > 0 ? tp->beta2 : 0.999f;
    s.eps = tp->eps > 0 ? tp->eps : 1e-8f;
    s.rows = B;
    s.n_out = m->n_out;
    s.seed = tp->seed;
    MF_CUDA(cudaStreamSynchronize(st));
    MF_CUDA(cudaMemcpy(m->d_st, &s, sizeof(s), cudaMemcpyHostToDevice));
    MF_CUDA(cudaMemset(m->d_g, 0, 4 * m->n_params));
    MF_CUDA(cudaMemset(m->d_m, 0, 4 * m->n_params));
    MF_CUDA(cudaMemset(m->d_v, 0, 4 * m->n_params));
    // a stride coprime to n walks the training set in a scrambled order
    long long stride = 1000003;
    while (std::gcd(stride, (long long)n) != 1) stride += 2;
    // one training step, captured once (the data pointers are part of it)
    if (m->step_exec) cudaGraphExecDestroy(m->step_exec);
    m->step_exec = nullptr;
    cudaGraph_t graph = nullptr;
    MF_CUDA(cudaStreamBeginCapture(m->cap_st, cudaStreamCaptureModeRelaxed));
    gather_kernel<<<256, 256, 0, m->cap_st>>>(X, T, n, m->n_in, m->n_out, m->d_st, stride, m->Xb, m->Tb);
    rc = enqueue_fwd_bwd(m, B, m->cap_st);
    if (rc == MF_OK) {
        adam_kernel<<<256, 256, 0, m->cap_st>>>(m->d_p, m->d_g, m->d_m, m->d_v, (int)m->n_params, layer_tab(m),
                                                m->d_st, 1);
        step_end_kernel<<<1, 1, 0, m->cap_st>>>(m->d_st);
    }
    cudaError_t ec = cudaStreamEndCapture(m->cap_st, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    MF_CUDA(ec);
    cudaError_t ei = cudaGraphInstantiate(&m->step_exec, graph, 0);
    cudaGraphDestroy(graph);
    MF_CUDA(ei);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
    for (int i = 0; i < tp->steps; ++i) MF_CUDA(cudaGraphLaunch(m->step_exec, st));
    cudaEventRecord(e1, st);
    cudaError_t es = cudaEventSynchronize(e1);
    cudaEventElapsedTime(&m->train_ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    MF_CUDA(es);
    m->steps_done += tp->steps;
    unsigned err = 0;
    MF_CUDA(cudaMemcpy(&err, m->d_err, sizeof(err), cudaMemcpyDeviceToHost));
    return err ? MF_E_TIMEOUT : MF_OK;
}

int mf_mlp_query(const mf_mlp *m, const char *key, double *value) {
    if (!m || !key || !value) return MF_E_INVAL;
    std::string k(key);
    if (k == "n_params") *value = (double)m->n_params;
    else if (k == "train_ms") *value = m->train_ms;
    else if (k == "steps_done") *value = (double)m->steps_done;
    else if (k == "loss") {
        TrainState s;
        MF_CUDA(cudaDeviceSynchronize());
        MF_CUDA(cudaMemcpy(&s, m->d_st, sizeof(s), cudaMemcpyDeviceToHost));
        *value = s.last_loss;
    } else
        return MF_E_INVAL;
    return MF_OK;
}

}  // extern "C"
