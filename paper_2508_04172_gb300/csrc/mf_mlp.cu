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
    MF_CUDA(cudaLaunchKernel(kern, grid, dim3(EPI == EPI_LNL ? kGemmThreadsLnl : kGemmThreads), args, smem, st));
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
// Column tile of the hidden-layer GEMMs (N = hidden): 128 columns keep three
// CTAs (128 TMEM columns each) per SM, so more epilogue warps hide latency.
int nt_hidden(int n) { return std::min(128, (n + 15) / 16 * 16); }

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
        rc = make_plan(pl, EPI_SILU, m->Hs[l - 1], rows, H, m->W[l], H, nt_hidden(H), g, m->d_err);
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
            rc = make_plan(pl, EPI_DSILU, dz, rows, m->out[l], m->Wt[l], m->in[l], nt_hidden(m->in[l]), g,
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
            rc = make_plan(pl, EPI_SILU, m->Hs[l - 1], B, H, m->W[l], H, nt_hidden(H), g, m->d_err);
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

// ===================================================================
// The surrogate of an interpolant handle: the network above trained to
// map the metric-eigenbasis point x to the handle's interpolated columns
// F(x) (Eq. rbfcoeff), labelled by the FP64 RBF interpolant on the GPU,
// served through the same time-interpolation / amplitude / quadratic-form
// epilogue as the RBF path (Eqs. SVD, projected_h_fd, logl_complete).
// The plain FP32 RBF path is the fallback: for every query when the
// held-out gate fails, and for queries outside the training radius.
// ===================================================================

struct mf_surrogate {
    mf_mlp *net = nullptr;
    int K = 0, K_out = 0;                 // user columns, network outputs (K rounded to 8)
    double *d_mu = nullptr, *d_s = nullptr;   // per user column: mean, scale of the targets
    float r_gate = 0.f;                   // training radius: queries beyond it use the RBF path
    bool gate = false;                    // held-out gate passed
    double ho_max = 0, ho_median = 0, ho_p99 = 0;
    float train_ms = 0, label_ms = 0, gate_ms = 0, loss = 0;
    int n_train = 0;
    // inference weights for the current device layout
    __nv_bfloat16 *d_Wdev = nullptr;      // [Kdev][H] de-standardised final layer, device order
    float *d_bdev = nullptr;              // [Kdev]
    int Kdev = 0, nbox = 0;
    unsigned layout_gen = ~0u;
    // inference scratch (grown on demand)
    int chunk_cap = 0;
    __nv_bfloat16 *d_h[2] = {nullptr, nullptr};   // [chunk][H] ping-pong activations
    float *d_part = nullptr;                      // [n_pass][chunk]
    int q_cap = 0, e_cap = 0, np_cap = 0;
    unsigned char *d_flag = nullptr;              // [Q] query outside the training radius
    int *d_list = nullptr;                        // [Q] indices of those queries
    int *d_count = nullptr;                       // number of them
    float *d_ci = nullptr, *d_ce = nullptr, *d_co = nullptr, *d_cpart = nullptr;   // compacted copies
    double fallback_rate = 0;
    int last_launches = 0;                        // kernels launched by the last mf_loglike
    float *d_colbuf = nullptr;                    // [chunk][Kdev] network columns (mf_eval_columns)
    size_t colbuf_cap = 0;
    bool fb_pending = false;                      // fallback count of the last call still on the device
    int fb_Q = 0;
};

namespace mf {
namespace {

constexpr int kSurChunk = 1 << 16;       // queries per network chunk (activations stay in L2)
constexpr int kLabelRows = 4096;         // label rows per FP64 GEMM

// x = R (theta - centre) in FP64 and FP32; |x| per row.
__global__ void sur_rotate_kernel(const float *__restrict__ th, int n, const double *__restrict__ Rc,
                                  double *__restrict__ x64, float *__restrict__ x32, float *__restrict__ rad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double d[4], r2 = 0.0;
    for (int k = 0; k < 4; ++k) d[k] = (double)th[(size_t)i * 4 + k] - Rc[16 + k];
    for (int a = 0; a < 4; ++a) {
        double v = 0.0;
        for (int k = 0; k < 4; ++k) v += Rc[4 * a + k] * d[k];
        x64[(size_t)i * 4 + a] = v;
        x32[(size_t)i * 4 + a] = (float)v;
        r2 += v * v;
    }
    rad[i] = (float)sqrt(r2);
}

// Augmented RBF row of every point (Eq. rbfcoeff): phi(eps |x - y_n|) for
// the N nodes (kernel `kind`, mf_rbf), then the tail monomials 1, x_1..x_4
// (first P of them).
__global__ void sur_phi_kernel(const double *__restrict__ x, int rows, const double *__restrict__ nodes, int N,
                               int P, double eps2, int kind, double *__restrict__ phi) {
    const int NP = N + P;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < (long long)rows * NP;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx / NP), n = (int)(idx % NP);
        const double *xi = x + (size_t)i * 4;
        double v;
        if (n < N) {
            const double *y = nodes + (size_t)n * 4;
            double r2 = 0.0;
            for (int k = 0; k < 4; ++k) r2 += (xi[k] - y[k]) * (xi[k] - y[k]);
            v = rbf_phi64(kind, eps2 * r2);
        } else {
            const int q = n - N;
            v = q == 0 ? 1.0 : xi[q - 1];
        }
        phi[idx] = v;
    }
}

// Per user column: mean and scale (standard deviation, floored at 1e-4 of
// the largest column's) of the labels F [n][K].
__global__ void sur_colstats_kernel(const double *__restrict__ F, int n, int K, double *__restrict__ mu,
                                    double *__restrict__ sd) {
    const int c = blockIdx.x;
    double s = 0.0, s2 = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double v = F[(size_t)i * K + c];
        s += v;
        s2 += v * v;
    }
    __shared__ double a[256], b[256];
    a[threadIdx.x] = s;
    b[threadIdx.x] = s2;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) {
            a[threadIdx.x] += a[threadIdx.x + k];
            b[threadIdx.x] += b[threadIdx.x + k];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double m = a[0] / n;
        mu[c] = m;
        sd[c] = sqrt(fmax(0.0, b[0] / n - m * m));
    }
}

__global__ void sur_floor_scale_kernel(double *sd, int K) {
    double mx = 0.0;
    for (int c = 0; c < K; ++c) mx = fmax(mx, sd[c]);
    const double fl = fmax(1e-4 * mx, 1e-300);
    for (int c = 0; c < K; ++c) sd[c] = fmax(sd[c], fl);
}

// Network targets (F - mu) / s in FP32 [n][K_out] (padding columns 0).
__global__ void sur_targets_kernel(const double *__restrict__ F, int n, int K, int K_out,
                                   const double *__restrict__ mu, const double *__restrict__ sd,
                                   float *__restrict__ T) {
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < (long long)n * K_out;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx / K_out), c = (int)(idx % K_out);
        T[idx] = c < K ? (float)((F[(size_t)i * K + c] - mu[c]) / sd[c]) : 0.f;
    }
}

// Final layer in the device column layout, de-standardised:
// W_dev[d] = s_u W_L[u], b_dev[d] = s_u b_L[u] + mu_u (u = user column of d).
__global__ void sur_devweights_kernel(const float *__restrict__ WL, const float *__restrict__ bL, int H,
                                      const int *__restrict__ user_of_dev, int Kdev,
                                      const double *__restrict__ mu, const double *__restrict__ sd,
                                      __nv_bfloat16 *__restrict__ Wdev, float *__restrict__ bdev) {
    const int d = blockIdx.x;
    const int u = user_of_dev[d];
    for (int k = threadIdx.x; k < H; k += blockDim.x)
        Wdev[(size_t)d * H + k] = __float2bfloat16_rn(u >= 0 ? (float)(sd[u] * (double)WL[(size_t)u * H + k]) : 0.f);
    if (threadIdx.x == 0) bdev[d] = u >= 0 ? (float)(sd[u] * (double)bL[u] + mu[u]) : 0.f;
}

// Network input layer for lnL queries: x = R (theta - centre) (FP32, as the
// RBF path), first layer -> H1 (one thread per query, the H outputs written
// as 16-byte vectors); flags queries with |x| > r_gate.
__global__ void __launch_bounds__(128) sur_input_kernel(const float *__restrict__ th, int Q, const RotParams rot,
                                 const float *__restrict__ W1, const float *__restrict__ b1, int H,
                                 __nv_bfloat16 *__restrict__ H1, float r_gate, unsigned char *__restrict__ flag,
                                 int *__restrict__ count) {
    __shared__ float4 w[256];     // [H] rows of W1 (4 inputs)
    __shared__ float bb[256];
    for (int o = threadIdx.x; o < H; o += blockDim.x) {
        w[o] = make_float4(W1[4 * o], W1[4 * o + 1], W1[4 * o + 2], W1[4 * o + 3]);
        bb[o] = b1[o];
    }
    __syncthreads();
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= Q) return;
    const float4 t = *reinterpret_cast<const float4 *>(th + (size_t)q * 4);
    const float d[4] = {t.x - rot.centre[0], t.y - rot.centre[1], t.z - rot.centre[2], t.w - rot.centre[3]};
    float x[4], r2 = 0.f;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        x[a] = rot.R[4 * a] * d[0] + rot.R[4 * a + 1] * d[1] + rot.R[4 * a + 2] * d[2] + rot.R[4 * a + 3] * d[3];
        r2 = fmaf(x[a], x[a], r2);
    }
    uint4 *row = reinterpret_cast<uint4 *>(H1 + (size_t)q * H);
    for (int o0 = 0; o0 < H; o0 += 8) {
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const float4 ww = w[o0 + e];
            float z = fmaf(ww.x, x[0], bb[o0 + e]);
            z = fmaf(ww.y, x[1], z);
            z = fmaf(ww.z, x[2], z);
            z = fmaf(ww.w, x[3], z);
            v[e] = silu_f(z);
        }
        uint4 p;
        p.x = Half2<1>::pack(v[0], v[1]);
        p.y = Half2<1>::pack(v[2], v[3]);
        p.z = Half2<1>::pack(v[4], v[5]);
        p.w = Half2<1>::pack(v[6], v[7]);
        row[o0 / 8] = p;
    }
    if (flag) {
        const bool out = !(sqrtf(r2) <= r_gate);
        flag[q] = out;
        if (out) atomicAdd(count, 1);
    }
}

// Gather the flagged queries (any order) into compact copies.
__global__ void sur_compact_kernel(const unsigned char *__restrict__ flag, int Q, const float *__restrict__ th,
                                   const float *__restrict__ ext, int E, int *__restrict__ slot,
                                   int *__restrict__ list, float *__restrict__ ci, float *__restrict__ ce) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= Q || !flag[q]) return;
    const int j = atomicAdd(slot, 1);
    list[j] = q;
    reinterpret_cast<float4 *>(ci)[j] = reinterpret_cast<const float4 *>(th)[q];
    for (int k = 0; k < E; ++k) ce[(size_t)j * E + k] = ext[(size_t)q * E + k];
}

__global__ void sur_scatter_kernel(const int *__restrict__ list, const int *__restrict__ count,
                                   const float *__restrict__ v, float *__restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < *count) out[list[j]] = v[j];
}

// Network columns in the device layout -> node_values order (one thread per
// (query, device column); padding columns are dropped).
__global__ void sur_gather_cols(const float *__restrict__ dev, int Qc, int Kdev, const int *__restrict__ user_of_dev,
                                int K, float *__restrict__ out) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)Qc * Kdev) return;
    const int q = (int)(i / (size_t)Kdev), c = (int)(i % (size_t)Kdev);
    const int u = user_of_dev[c];
    if (u >= 0) out[(size_t)q * K + u] = dev[i];
}

void free_infer(mf_surrogate *s) {
    auto fr = [](void *p) { if (p) cudaFree(p); };
    fr(s->d_h[0]); fr(s->d_h[1]); fr(s->d_part);
    fr(s->d_flag); fr(s->d_list); fr(s->d_count); fr(s->d_ci); fr(s->d_ce); fr(s->d_co); fr(s->d_cpart);
    s->d_h[0] = s->d_h[1] = nullptr;
    s->d_part = nullptr;
    s->d_flag = nullptr;
    s->d_list = s->d_count = nullptr;
    s->d_ci = s->d_ce = s->d_co = s->d_cpart = nullptr;
    s->chunk_cap = s->q_cap = s->e_cap = s->np_cap = 0;
}

void destroy_surrogate(mf_surrogate *s) {
    if (!s) return;
    free_infer(s);
    if (s->net) destroy_mlp(s->net);
    auto fr = [](void *p) { if (p) cudaFree(p); };
    fr(s->d_mu); fr(s->d_s); fr(s->d_Wdev); fr(s->d_bdev); fr(s->d_colbuf);
    delete s;
}

int ensure_infer(mf_surrogate *s, int chunk, int Q, int E, int n_pass) {
    const int H = s->net->H;
    if (chunk > s->chunk_cap) {
        for (int k = 0; k < 2; ++k) {
            if (s->d_h[k]) cudaFree(s->d_h[k]);
            s->d_h[k] = nullptr;
        }
        if (s->d_part) cudaFree(s->d_part);
        s->d_part = nullptr;
        s->chunk_cap = 0;
        MF_CUDA(cudaMalloc((void **)&s->d_h[0], 2 * (size_t)chunk * H));
        MF_CUDA(cudaMalloc((void **)&s->d_h[1], 2 * (size_t)chunk * H));
        MF_CUDA(cudaMalloc((void **)&s->d_part, 4 * (size_t)chunk * kMaxPass));
        s->chunk_cap = chunk;
    }
    if (Q > s->q_cap || E > s->e_cap || n_pass > s->np_cap) {
        auto fr = [](void *p) { if (p) cudaFree(p); };
        fr(s->d_flag); fr(s->d_list); fr(s->d_count); fr(s->d_ci); fr(s->d_ce); fr(s->d_co); fr(s->d_cpart);
        s->q_cap = s->e_cap = s->np_cap = 0;
        const size_t q = (size_t)Q, e = (size_t)std::max(E, 5);
        MF_CUDA(cudaMalloc((void **)&s->d_flag, q));
        MF_CUDA(cudaMalloc((void **)&s->d_list, 4 * q));
        MF_CUDA(cudaMalloc((void **)&s->d_count, 8));
        MF_CUDA(cudaMalloc((void **)&s->d_ci, 16 * q));
        MF_CUDA(cudaMalloc((void **)&s->d_ce, 4 * q * e));
        MF_CUDA(cudaMalloc((void **)&s->d_co, 4 * q));
        MF_CUDA(cudaMalloc((void **)&s->d_cpart, 4 * q * (size_t)n_pass));
        s->q_cap = (int)q;
        s->e_cap = (int)e;
        s->np_cap = n_pass;
    }
    return MF_OK;
}

}  // namespace

// Final-layer weights of the surrogate in the handle's current device
// layout (rebuilt whenever the layout changes).
int surrogate_prepare(mf_handle *h) {
    mf_surrogate *s = h->sur;
    if (!s || !s->net) return MF_E_STATE;
    const int H = s->net->H, L = s->net->L;
    if (s->d_Wdev) cudaFree(s->d_Wdev);
    if (s->d_bdev) cudaFree(s->d_bdev);
    s->d_Wdev = nullptr;
    s->d_bdev = nullptr;
    MF_CUDA(cudaMalloc((void **)&s->d_Wdev, 2 * (size_t)h->Kdev * H));
    MF_CUDA(cudaMalloc((void **)&s->d_bdev, 4 * (size_t)h->Kdev));
    const float *WL = s->net->d_p + s->net->off[L - 1];
    sur_devweights_kernel<<<h->Kdev, 256>>>(WL, WL + (size_t)s->K_out * H, H, h->d_user_of_dev, h->Kdev, s->d_mu,
                                            s->d_s, s->d_Wdev, s->d_bdev);
    MF_CUDA(cudaGetLastError());
    MF_CUDA(cudaDeviceSynchronize());
    s->Kdev = h->Kdev;
    int nbox = 0;
    for (auto &p : h->passes) nbox = std::max(nbox, p.width);
    s->nbox = nbox;
    return MF_OK;
}

void free_surrogate(mf_handle *h) {
    destroy_surrogate(h->sur);
    h->sur = nullptr;
}

// The network's interpolated columns (node_values order) for Q queries:
// the same input layer and hidden GEMMs as the lnL path, the final layer
// stored in FP32 (the accumulators the fused lnL epilogue reads) and
// gathered into the user column order.  Every query goes through the
// network, whatever its radius or the gate.
int eval_columns_surrogate(mf_handle *h, const float *intr, int Q, float *out, cudaStream_t st) {
    mf_surrogate *s = h->sur;
    if (!s || !s->net || !s->d_Wdev) return MF_E_STATE;
    mf_mlp *m = s->net;
    const int H = m->H;
    const int np = (int)h->passes.size();
    const int chunk = std::min(Q, 1 << 14);
    int rc = ensure_infer(s, chunk, Q, 5, np);
    if (rc) return rc;
    const size_t need = (size_t)chunk * h->Kdev;
    if (need > s->colbuf_cap) {
        if (s->d_colbuf) cudaFree(s->d_colbuf);
        s->d_colbuf = nullptr;
        s->colbuf_cap = 0;
        MF_CUDA(cudaMalloc((void **)&s->d_colbuf, 4 * need));
        s->colbuf_cap = need;
    }
    const RotParams rot = make_rot(h);
    for (int q0 = 0; q0 < Q; q0 += chunk) {
        const int Qc = std::min(chunk, Q - q0);
        sur_input_kernel<<<(unsigned)((Qc + 127) / 128), 128, 0, st>>>(
            intr + (size_t)q0 * 4, Qc, rot, m->d_p, m->d_p + H * 4, H, s->d_h[0], 1e30f, s->d_flag + q0,
            s->d_count);
        MF_CUDA(cudaGetLastError());
        int cur = 0;
        for (int l = 1; l < m->L - 1; ++l) {
            GemmArgs g{};
            g.bias = m->d_p + m->off[l] + H * H;
            g.out_bf = s->d_h[cur ^ 1];
            GemmPlan pl;
            rc = make_plan(pl, EPI_SILU, s->d_h[cur], Qc, H, m->W[l], H, nt_hidden(H), g, h->d_err);
            if (rc) return rc;
            rc = launch_plan(pl, st);
            if (rc) return rc;
            cur ^= 1;
        }
        GemmArgs g{};
        g.bias = s->d_bdev;
        g.out_f = s->d_colbuf;
        GemmPlan pl;
        rc = make_plan(pl, EPI_F32, s->d_h[cur], Qc, H, s->d_Wdev, h->Kdev, nt_for(std::min(h->Kdev, 128)), g,
                       h->d_err);
        if (rc) return rc;
        rc = launch_plan(pl, st);
        if (rc) return rc;
        const size_t n = (size_t)Qc * h->Kdev;
        sur_gather_cols<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(s->d_colbuf, Qc, h->Kdev, h->d_user_of_dev,
                                                                      h->K, out + (size_t)q0 * h->K);
        MF_CUDA(cudaGetLastError());
    }
    return MF_OK;
}

// lnL through the network: chunks of queries through the hidden layers,
// the final layer fused with the lnL epilogue per column pass, then the
// plain FP32 RBF path for queries outside the training radius.  Uses the
// FP32 weights of the handle (prepared with the surrogate form).
int loglike_surrogate(mf_handle *h, const float *intr, const float *ext, int Q, int E, float *out,
                      cudaStream_t st, bool force_net) {
    mf_surrogate *s = h->sur;
    if (!s || !s->net || !s->d_Wdev || !h->d_W32) return MF_E_STATE;
    const int np = (int)h->passes.size();
    if (!s->gate && !force_net) {   // held-out gate failed: the RBF path serves everything
        s->fallback_rate = 1.0;
        s->fb_pending = false;
        s->last_launches = np > 1 ? 2 : 1;
        int rc = ensure_infer(s, 1, Q, E, np);
        if (rc) return rc;
        rc = launch_fp32(h, intr, ext, Q, E, out, st, np > 1 ? s->d_cpart : nullptr);
        if (rc) return rc;
        if (np > 1) return launch_combine(s->d_cpart, np, Q, out, st, h->d_bad);
        return MF_OK;
    }
    mf_mlp *m = s->net;
    const int H = m->H;
    const int chunk = std::min(Q, kSurChunk);
    int rc = ensure_infer(s, chunk, Q, E, np);
    if (rc) return rc;
    MF_CUDA(cudaMemsetAsync(s->d_count, 0, 8, st));
    const int n_chunks = (Q + chunk - 1) / chunk;
    s->last_launches = n_chunks * (1 + (m->L - 2) + 1 + (np > 1 ? 1 : 0));
    const RotParams rot = make_rot(h);
    const EpiParams epi = make_epi(h);
    for (int q0 = 0; q0 < Q; q0 += chunk) {
        const int Qc = std::min(chunk, Q - q0);
        sur_input_kernel<<<(unsigned)((Qc + 127) / 128), 128, 0, st>>>(
            intr + (size_t)q0 * 4, Qc, rot, m->d_p, m->d_p + H * 4, H, s->d_h[0], force_net ? 1e30f : s->r_gate,
            s->d_flag + q0, s->d_count);
        MF_CUDA(cudaGetLastError());
        int cur = 0;
        for (int l = 1; l < m->L - 1; ++l) {
            GemmArgs g{};
            g.bias = m->d_p + m->off[l] + H * H;
            g.out_bf = s->d_h[cur ^ 1];
            GemmPlan pl;
            rc = make_plan(pl, EPI_SILU, s->d_h[cur], Qc, H, m->W[l], H, nt_hidden(H), g, h->d_err);
            if (rc) return rc;
            rc = launch_plan(pl, st);
            if (rc) return rc;
            cur ^= 1;
        }
        GemmArgs g{};
        g.bias = s->d_bdev;
        g.ext = ext + (size_t)q0 * E;
        g.E = E;
        g.lnl_out = out + q0;
        g.partial = s->d_part;
        GemmPlan pl;
        rc = make_plan(pl, EPI_LNL, s->d_h[cur], Qc, H, s->d_Wdev, h->Kdev, s->nbox, g, h->d_err);
        if (rc) return rc;
        pl.grid_y = np;
        rc = launch_plan(pl, st, &epi, h->n_modes);
        if (rc) return rc;
        if (np > 1) {
            rc = launch_combine(s->d_part, np, Qc, out + q0, st, h->d_bad);
            if (rc) return rc;
        }
    }
    if (force_net) {
        s->fallback_rate = 0.0;
        s->fb_pending = false;
        return MF_OK;
    }
    // queries outside the training radius: compacted on the device and
    // evaluated by the plain RBF path, whose launch reads their count on the
    // device (no host synchronisation: the call stays asynchronous and can be
    // captured in a CUDA graph); results are scattered back in place
    MF_CUDA(cudaMemsetAsync(s->d_count + 1, 0, 4, st));
    sur_compact_kernel<<<(Q + 255) / 256, 256, 0, st>>>(s->d_flag, Q, intr, ext, E, s->d_count + 1, s->d_list,
                                                        s->d_ci, s->d_ce);
    MF_CUDA(cudaGetLastError());
    rc = launch_fp32(h, s->d_ci, s->d_ce, Q, E, s->d_co, st, np > 1 ? s->d_cpart : nullptr, s->d_count + 1);
    if (rc) return rc;
    if (np > 1) {
        rc = launch_combine(s->d_cpart, np, Q, s->d_co, st, h->d_bad, s->d_count + 1);
        if (rc) return rc;
    }
    sur_scatter_kernel<<<(Q + 255) / 256, 256, 0, st>>>(s->d_list, s->d_count + 1, s->d_co, out);
    MF_CUDA(cudaGetLastError());
    s->last_launches += 3 + (np > 1 ? 1 : 0);
    s->fb_pending = true;     // the rate is read from the device count when queried
    s->fb_Q = Q;
    return MF_OK;
}

}  // namespace mf

namespace {

// host-side quantiles of |a - b| over finite pairs
void abs_diff_stats(const std::vector<float> &a, const std::vector<float> &b, double &mx, double &med, double &p99) {
    std::vector<double> d;
    d.reserve(a.size());
    for (size_t i = 0; i < a.size(); ++i)
        if (std::isfinite(a[i]) && std::isfinite(b[i])) d.push_back(std::fabs((double)a[i] - (double)b[i]));
    mx = med = p99 = d.empty() ? INFINITY : 0.0;
    if (d.empty()) return;
    std::sort(d.begin(), d.end());
    mx = d.back();
    med = d[d.size() / 2];
    p99 = d[std::min(d.size() - 1, (size_t)(0.99 * (double)d.size()))];
}

}  // namespace

extern "C" {

int mf_train_surrogate(mf_handle *h, const float *train_intrinsic, int n_train, const float *held_intrinsic,
                       const float *held_extrinsic, int n_held, int E, const mf_surrogate_params *sp,
                       void *stream) {
    if (!h || !train_intrinsic || !sp || n_train < 64 || E < 5) return MF_E_INVAL;
    if (n_held < 0 || (n_held > 0 && (!held_intrinsic || !held_extrinsic))) return MF_E_INVAL;
    if (((uintptr_t)train_intrinsic & 15) || ((uintptr_t)held_intrinsic & 15)) return MF_E_INVAL;
    if (!h->have_layout || !h->have_basis || !h->have_det) return MF_E_STATE;
    if (h->sky && E < 7) return MF_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    MF_CUDA(cudaStreamSynchronize(st));
    const mf_form prev = h->form;
    mf::free_surrogate(h);
    mf_surrogate *s = new (std::nothrow) mf_surrogate();
    if (!s) return MF_E_NOMEM;
    h->sur = s;
    s->K = h->K;
    s->K_out = (h->K + 7) / 8 * 8;
    s->n_train = n_train;
    const int hidden = sp->hidden > 0 ? sp->hidden : 256;
    const int n_hidden = sp->n_hidden > 0 ? sp->n_hidden : 3;
    int rc = mf_mlp_create(4, hidden, n_hidden, s->K_out, sp->seed, &s->net);
    if (rc) { mf::free_surrogate(h); return rc; }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // ---- labels: the FP64 RBF interpolant at the rotated training points
    cudaEventRecord(e0, st);
    const int NP = h->N + h->P, K = h->K;
    double *x64 = nullptr, *Rc = nullptr, *F = nullptr, *phi = nullptr;
    float *x32 = nullptr, *rad = nullptr, *T = nullptr;
    auto cleanup = [&]() {
        for (void *p : {(void *)x64, (void *)Rc, (void *)F, (void *)phi, (void *)x32, (void *)rad, (void *)T})
            if (p) cudaFree(p);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    };
    const int lrows = std::min(n_train, mf::kLabelRows);
    bool ok = cudaMalloc((void **)&x64, 32 * (size_t)n_train) == cudaSuccess &&
              cudaMalloc((void **)&Rc, 20 * sizeof(double)) == cudaSuccess &&
              cudaMalloc((void **)&F, 8 * (size_t)n_train * K) == cudaSuccess &&
              cudaMalloc((void **)&phi, 8 * (size_t)lrows * NP) == cudaSuccess &&
              cudaMalloc((void **)&x32, 16 * (size_t)n_train) == cudaSuccess &&
              cudaMalloc((void **)&rad, 4 * (size_t)n_train) == cudaSuccess &&
              cudaMalloc((void **)&T, 4 * (size_t)n_train * s->K_out) == cudaSuccess &&
              cudaMalloc((void **)&s->d_mu, 8 * (size_t)K) == cudaSuccess &&
              cudaMalloc((void **)&s->d_s, 8 * (size_t)K) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        cleanup();
        mf::free_surrogate(h);
        return MF_E_NOMEM;
    }
    double Rh[20];
    memcpy(Rh, h->R, 16 * sizeof(double));
    memcpy(Rh + 16, h->centre, 4 * sizeof(double));
    cudaMemcpy(Rc, Rh, sizeof(Rh), cudaMemcpyHostToDevice);
    mf::sur_rotate_kernel<<<(n_train + 255) / 256, 256, 0, st>>>(train_intrinsic, n_train, Rc, x64, x32, rad);
    for (int r0 = 0; r0 < n_train && rc == MF_OK; r0 += lrows) {
        const int rows = std::min(lrows, n_train - r0);
        mf::sur_phi_kernel<<<1024, 256, 0, st>>>(x64 + (size_t)r0 * 4, rows, h->d_nodes64, h->N, h->P,
                                                 h->eps * h->eps, (int)h->rbf, phi);
        // F[rows][K] = Phi[rows][NP] W[NP][K]
        rc = mf::dgemm_rm(rows, K, NP, phi, NP, h->d_W64, K, F + (size_t)r0 * K, K, st);
    }
    if (rc) { cleanup(); mf::free_surrogate(h); return rc; }
    mf::sur_colstats_kernel<<<K, 256, 0, st>>>(F, n_train, K, s->d_mu, s->d_s);
    mf::sur_floor_scale_kernel<<<1, 1, 0, st>>>(s->d_s, K);
    mf::sur_targets_kernel<<<1024, 256, 0, st>>>(F, n_train, K, s->K_out, s->d_mu, s->d_s, T);
    cudaEventRecord(e1, st);
    cudaError_t ce = cudaEventSynchronize(e1);
    if (ce != cudaSuccess) { cleanup(); mf::free_surrogate(h); MF_CUDA(ce); }
    cudaEventElapsedTime(&s->label_ms, e0, e1);
    {
        std::vector<float> r(n_train);
        cudaMemcpy(r.data(), rad, 4 * (size_t)n_train, cudaMemcpyDeviceToHost);
        s->r_gate = sp->r_gate > 0 ? sp->r_gate : *std::max_element(r.begin(), r.end());
    }
    // ---- training
    mf_mlp_train_params tp{};
    tp.steps = sp->steps > 0 ? sp->steps : 20000;
    tp.batch = sp->batch > 0 ? sp->batch : 4096;
    tp.lr = sp->lr > 0 ? sp->lr : 1e-3f;
    tp.lr_min = sp->lr_min > 0 ? sp->lr_min : 1e-5f;
    tp.seed = sp->seed;
    rc = mf_mlp_train(s->net, x32, T, n_train, &tp, stream);
    s->train_ms = s->net->train_ms;
    double loss = 0;
    if (rc == MF_OK) rc = mf_mlp_query(s->net, "loss", &loss);
    s->loss = (float)loss;
    cleanup();
    if (rc) { mf::free_surrogate(h); return rc; }
    // ---- held-out gate: the network's lnL against the plain FP32 RBF path
    rc = mf::prepare_form(h, MF_FORM_FP32);
    if (rc == MF_OK) rc = mf::surrogate_prepare(h);
    if (rc == MF_OK && n_held > 0) {
        float *a = nullptr, *b = nullptr;
        if (cudaMalloc((void **)&a, 4 * (size_t)n_held) != cudaSuccess ||
            cudaMalloc((void **)&b, 4 * (size_t)n_held) != cudaSuccess) {
            cudaGetLastError();
            rc = MF_E_NOMEM;
        } else {
            cudaEvent_t g0, g1;
            cudaEventCreate(&g0);
            cudaEventCreate(&g1);
            cudaEventRecord(g0, st);
            rc = mf::loglike_surrogate(h, held_intrinsic, held_extrinsic, n_held, E, a, st, true);
            cudaEventRecord(g1, st);
            if (rc == MF_OK) rc = mf_loglike(h, held_intrinsic, held_extrinsic, n_held, E, b, stream);
            if (rc == MF_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = MF_E_CUDA;
            cudaEventElapsedTime(&s->gate_ms, g0, g1);
            cudaEventDestroy(g0);
            cudaEventDestroy(g1);
            if (rc == MF_OK) {
                std::vector<float> ha(n_held), hb(n_held);
                cudaMemcpy(ha.data(), a, 4 * (size_t)n_held, cudaMemcpyDeviceToHost);
                cudaMemcpy(hb.data(), b, 4 * (size_t)n_held, cudaMemcpyDeviceToHost);
                abs_diff_stats(ha, hb, s->ho_max, s->ho_median, s->ho_p99);
            }
        }
        if (a) cudaFree(a);
        if (b) cudaFree(b);
        // the held-out runs' out-of-window counts are not the caller's
        long long nb = 0;
        if (mf_sync_status(h, stream, &nb) == MF_E_TIMEOUT && rc == MF_OK) rc = MF_E_TIMEOUT;
    }
    const float gmax = sp->gate_max > 0 ? sp->gate_max : 0.1f;
    const float gmed = sp->gate_median > 0 ? sp->gate_median : 0.01f;
    s->gate = rc == MF_OK && n_held > 0 && s->ho_max <= gmax && s->ho_median <= gmed;
    // back to the caller's form (the surrogate stays trained)
    int rc2 = mf::prepare_form(h, prev);
    if (rc) { mf::free_surrogate(h); return rc; }
    return rc2;
}

}  // extern "C"

namespace mf {
int surrogate_query(const mf_handle *h, const std::string &k, double *v) {
    mf_surrogate *s = h->sur;
    if (!s) return MF_E_STATE;
    if (k == "fallback_rate" && s->fb_pending) {
        // the count of the last call, once the device has produced it
        int n = 0;
        MF_CUDA(cudaMemcpy(&n, s->d_count + 1, sizeof(int), cudaMemcpyDeviceToHost));
        s->fallback_rate = s->fb_Q > 0 ? (double)n / (double)s->fb_Q : 0.0;
        s->fb_pending = false;
    }
    if (k == "fallback_rate") *v = s->fallback_rate;
    else if (k == "surrogate_gate") *v = s->gate ? 1.0 : 0.0;
    else if (k == "surrogate_heldout_max") *v = s->ho_max;
    else if (k == "surrogate_heldout_median") *v = s->ho_median;
    else if (k == "surrogate_heldout_p99") *v = s->ho_p99;
    else if (k == "surrogate_train_ms") *v = s->train_ms;
    else if (k == "surrogate_label_ms") *v = s->label_ms;
    else if (k == "surrogate_gate_ms") *v = s->gate_ms;
    else if (k == "surrogate_loss") *v = s->loss;
    else if (k == "surrogate_r_gate") *v = s->r_gate;
    else if (k == "surrogate_n_params") *v = (double)s->net->n_params;
    else if (k == "launches") *v = s->last_launches;
    else return MF_E_INVAL;
    return MF_OK;
}
}  // namespace mf
