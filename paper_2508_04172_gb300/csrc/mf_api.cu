// C ABI of libmf: handle management, configuration, device column layout,
// weight conversion for each arithmetic form and the lnL launch.
#include "mf_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

namespace mf {
int rbf_build(mf_handle *h, const double *F_host, cudaStream_t st);
int metric_eig(const double *metric, double *R_out);
int svd_compress(const double *z, int N, int M, int rank, double *coef, double *basis, double *sv,
                 cudaStream_t st);
int convert_tc_weights(mf_handle *h, mf_form f);
}  // namespace mf

namespace {

bool supported_mode(int l, int m) {
    return (l == 2 && (m == 2 || m == 1)) || (l == 3 && (m == 3 || m == 2)) || (l == 4 && m == 4);
}

__global__ void convert_fp32_kernel(const double *__restrict__ W64, int rows, int K,
                                    const int *__restrict__ user_of_dev, int Kdev, int Nk,
                                    float *__restrict__ W32) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    int n = blockIdx.y;
    if (c >= Kdev) return;
    int u = user_of_dev[c];
    float v = 0.f;
    if (u >= 0 && n < rows) v = (float)W64[(size_t)n * K + u];
    W32[(size_t)n * Kdev + c] = v;
}

__global__ void prescale_nodes(const double *__restrict__ y, int N, int Nk, double pre,
                               float4 *__restrict__ out) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= Nk) return;
    if (n < N)   // stored negated: kernels form x - y as x + (-y)
        out[n] = make_float4((float)(-pre * y[4 * n]), (float)(-pre * y[4 * n + 1]),
                             (float)(-pre * y[4 * n + 2]), (float)(-pre * y[4 * n + 3]));
    else
        out[n] = make_float4(0.f, 0.f, 0.f, 0.f);
}

void free_form(mf_handle *h) {
    if (h->d_W32) cudaFree(h->d_W32);
    if (h->d_Whi) cudaFree(h->d_Whi);
    if (h->d_Wlo) cudaFree(h->d_Wlo);
    if (h->d_colscale) cudaFree(h->d_colscale);
    if (h->d_user_of_dev) cudaFree(h->d_user_of_dev);
    h->d_W32 = nullptr;
    h->d_Whi = h->d_Wlo = nullptr;
    h->d_colscale = nullptr;
    h->d_user_of_dev = nullptr;
}

}  // namespace

namespace mf {

bool is_tc_form(mf_form f) { return f >= MF_FORM_BF16 && f <= MF_FORM_FP16_3TERM; }

// Split group widths w[0..n) into exactly `count` contiguous non-empty runs
// minimising the widest run (each padded to kPassAlign); start[c] = first
// group of run c.  Returns the widest padded run, or -1 if count > n.
static int split_exact(const std::vector<int> &w, int count, std::vector<int> &start) {
    const int n = (int)w.size();
    if (count < 1 || count > n) return -1;
    auto up = [](int x) { return (x + kPassAlign - 1) / kPassAlign * kPassAlign; };
    std::vector<int> pre(n + 1, 0);
    for (int i = 0; i < n; ++i) pre[i + 1] = pre[i] + w[i];
    const int INF = 1 << 30;
    // best[c][i]: widest run when groups [0, i) form c runs; cut[c][i]: start of the last run
    std::vector<std::vector<int>> best(count + 1, std::vector<int>(n + 1, INF)),
        cut(count + 1, std::vector<int>(n + 1, 0));
    best[0][0] = 0;
    for (int c = 1; c <= count; ++c)
        for (int i = c; i <= n; ++i)
            for (int j = c - 1; j < i; ++j) {
                if (best[c - 1][j] == INF) continue;
                int v = std::max(best[c - 1][j], up(pre[i] - pre[j]));
                if (v < best[c][i]) { best[c][i] = v; cut[c][i] = j; }
            }
    start.assign(count, 0);
    for (int c = count, i = n; c >= 1; --c) {
        start[c - 1] = cut[c][i];
        i = cut[c][i];
    }
    return best[count][n];
}

// Device column layout: per detector, its overlap groups (interleaved Re/Im
// of a run of SVD coefficients, padded to 8 columns) then its cross-term
// group, packed contiguously into passes of at most pass_max columns (each
// padded to 16).  The layout takes the fewest passes that fit (or exactly
// pass_count), balanced by a min-max split.  Every mode may be split into
// 2, 4, ... runs of coefficients (lnL is linear in each coefficient, so a
// mode's contribution may be summed over passes): needed when whole modes
// do not pack into that many passes, and taken when a finer split makes the
// widest pass narrower.
int build_layout(mf_handle *h) {
    const int nd = h->n_det, nm = h->n_modes, l = h->rank;
    auto up = [](int x, int a) { return (x + a - 1) / a * a; };
    struct G { int kind, det, mode, width, i0, ni; };
    auto make = [&](int nsplit) {
        std::vector<G> gs;
        const int chunk = ((l + nsplit - 1) / nsplit + 3) / 4 * 4;   // coefficients per run (a multiple of 4)
        for (int k = 0; k < nd; ++k) {
            for (int mu = 0; mu < nm; ++mu)
                for (int i0 = 0; i0 < l; i0 += chunk) {
                    const int ni = std::min(chunk, l - i0);
                    gs.push_back({0, k, mu, up(2 * ni, kGroupAlign), i0, ni});
                }
            gs.push_back({1, k, 0, up(nm * nm, kGroupAlign), 0, 0});
        }
        return gs;
    };
    const int pmax = h->pass_max;
    std::vector<G> gs;
    std::vector<int> cut_at;
    bool found = false;
    // fewest passes first; among the splits of the modes that fit that many,
    // the one whose widest pass is narrowest (a cluster advances at the pace
    // of its widest pass), the coarsest on ties
    for (int npass = 1; npass <= kMaxPass && !found; ++npass) {
        if (h->pass_count > 0 && npass != h->pass_count) continue;
        int best = pmax + 1;
        for (int nsplit = 1; nsplit <= 32; nsplit *= 2) {
            std::vector<G> cand = make(nsplit);
            if ((int)cand.size() > kMaxGroups) break;
            int total = 0, gmax = 0;
            for (auto &g : cand) { total += g.width; gmax = std::max(gmax, g.width); }
            if (up(gmax, kPassAlign) > pmax) continue;       // a finer split may fit
            if (npass * pmax < total) break;                   // finer splits only add padding
            if (npass > (int)cand.size()) continue;            // a finer split has more groups
            std::vector<int> w;
            for (auto &g : cand) w.push_back(g.width);
            std::vector<int> start;
            const int widest = split_exact(w, npass, start);
            if (widest > 0 && widest < best) {
                best = widest;
                gs = cand;
                cut_at = start;
                found = true;
            }
        }
    }
    if (!found) return MF_E_INVAL;
    h->groups.clear();
    h->passes.clear();
    Pass cur{0, 0, 0, 0};
    int col = 0;
    size_t next_cut = 1;
    for (size_t i = 0; i < gs.size(); ++i) {
        const bool split = next_cut < cut_at.size() && (int)i == cut_at[next_cut];
        if (split) {
            ++next_cut;
            cur.width = up(cur.width, kPassAlign);
            h->passes.push_back(cur);
            col += cur.width;
            cur = Pass{col, 0, (int)h->groups.size(), 0};
        }
        Group g{gs[i].kind, gs[i].det, gs[i].mode, cur.width, gs[i].width, gs[i].i0, gs[i].ni};
        h->groups.push_back(g);
        cur.width += gs[i].width;
        cur.ng++;
    }
    cur.width = up(cur.width, kPassAlign);
    h->passes.push_back(cur);
    col += cur.width;
    if ((int)h->passes.size() > kMaxPass) return MF_E_INVAL;
    h->Kdev = col;
    // device column -> user column (node_values order)
    h->user_of_dev.assign(h->Kdev, -1);
    const int sig0 = nd * nm * 2 * l;
    const int nup = nm * (nm - 1) / 2;
    for (auto &ps : h->passes)
        for (int gi = ps.g0; gi < ps.g0 + ps.ng; ++gi) {
            const Group &g = h->groups[gi];
            int base = ps.col0 + g.col;
            if (g.kind == 0) {
                int ucol = (g.det * nm + g.mode) * 2 * l;
                for (int i = 0; i < g.ni; ++i) {
                    h->user_of_dev[base + 2 * i] = ucol + g.i0 + i;
                    h->user_of_dev[base + 2 * i + 1] = ucol + l + g.i0 + i;
                }
            } else {
                int ucol = sig0 + g.det * nm * nm;
                for (int a = 0; a < nm; ++a) h->user_of_dev[base + a] = ucol + a;
                for (int p = 0; p < nup; ++p) {
                    h->user_of_dev[base + nm + 2 * p] = ucol + nm + p;
                    h->user_of_dev[base + nm + 2 * p + 1] = ucol + nm + nup + p;
                }
            }
        }
    return MF_OK;
}

EpiParams make_epi(const mf_handle *h) {
    EpiParams e;
    memset(&e, 0, sizeof(e));
    e.n_det = h->n_det;
    e.n_modes = h->n_modes;
    e.rank = h->rank;
    e.M = h->M;
    for (int mu = 0; mu < h->n_modes; ++mu) {
        e.ell[mu] = h->ell_m[2 * mu];
        e.em[mu] = h->ell_m[2 * mu + 1];
    }
    // detectors and basis may not be set yet (mf_eval_columns needs only the
    // layout): their fields then stay zero
    const bool det_ok = h->have_det && h->det.size() >= (size_t)3 * h->n_det;
    const bool basis_ok = h->have_basis && h->dt > 0;
    for (int k = 0; k < h->n_det && det_ok && basis_ok; ++k) {
        e.fp0[k] = (float)h->det[3 * k];
        e.fx0[k] = (float)h->det[3 * k + 1];
        double off = (h->det[3 * k + 2] - h->t0) / h->dt;
        double J = std::floor(off);
        e.J[k] = (int)J;
        e.frac[k] = (float)(off - J);
    }
    e.inv_dt = basis_ok ? (float)(1.0 / h->dt) : 0.f;
    e.d_ref = (float)h->d_ref;
    e.cubic = h->d_cubic;
    e.bad = h->d_bad;
    e.err = h->d_err;
    e.n_groups = (int)h->groups.size();
    e.n_pass = (int)h->passes.size();
    for (int g = 0; g < e.n_groups; ++g) e.groups[g] = h->groups[g];
    for (int p = 0; p < e.n_pass; ++p) e.passes[p] = h->passes[p];
    e.sky = h->sky && det_ok ? 1 : 0;
    if (e.sky) {
        for (int k = 0; k < h->n_det; ++k) {
            const double *D = h->sky_tensor.data() + 9 * k;
            e.dten[k][0] = (float)D[0];
            e.dten[k][1] = (float)D[4];
            e.dten[k][2] = (float)D[8];
            e.dten[k][3] = (float)(0.5 * (D[1] + D[3]));
            e.dten[k][4] = (float)(0.5 * (D[2] + D[6]));
            e.dten[k][5] = (float)(0.5 * (D[5] + D[7]));
            for (int i = 0; i < 3; ++i) e.dpos[k][i] = (float)h->sky_pos[3 * k + i];
            // reduced in FP64 so that the FP32 hour angle keeps its precision
            double g = std::fmod(h->gmst0 + h->omega_e * h->sky_tau[k], 2.0 * M_PI);
            if (g < 0) g += 2.0 * M_PI;
            e.gk[k] = (float)g;
        }
        e.omega = (float)h->omega_e;
    }
    return e;
}

RotParams make_rot(const mf_handle *h) {
    RotParams r;
    for (int i = 0; i < 16; ++i) r.R[i] = (float)h->R[i];
    for (int i = 0; i < 4; ++i) r.centre[i] = (float)h->centre[i];
    r.pre = (float)rbf_prescale(h);
    r.rbf = (int)h->rbf;
    return r;
}

int prepare_form(mf_handle *h, mf_form f) {
    if (!h->have_layout) return MF_E_STATE;
    if (f == MF_FORM_MLP) {
        // the surrogate serves through the FP32 layout; its FP32 weights are the fallback
        if (!h->sur) return MF_E_STATE;
        // 128-column passes: the surrogate's final GEMM then allocates 128 TMEM
        // columns per CTA and several CTAs share an SM (its epilogue is
        // latency-bound); the FP32 fallback runs on the same layout
        h->fp32_pass_max = 128;
        int rc = prepare_form(h, MF_FORM_FP32);
        h->fp32_pass_max = 176;
        if (rc) return rc;
        rc = surrogate_prepare(h);
        if (rc) return rc;
        h->form = MF_FORM_MLP;
        return MF_OK;
    }
    // FP16 forms scale Phi by 2^14: only kernels bounded by 1 fit their range
    if ((f == MF_FORM_FP16 || f == MF_FORM_FP16_WSPLIT || f == MF_FORM_FP16_3TERM) &&
        (h->rbf == MF_RBF_PHS3 || h->rbf == MF_RBF_MQ))
        return MF_E_NOTIMPL;
    free_form(h);
    h->pass_count = is_tc_form(f) ? h->pass_count_user : 0;   // exact counts: tcgen05 forms only
    // tcgen05 design: the TMEM design when asked for, or (automatic) when the
    // columns fit in one pass of its width -- measured faster there
    h->tc_tmem = false;
    int rc;
    if (is_tc_form(f) && (h->tc_design == 1 || (h->tc_design == -1 && h->pass_count <= 1))) {
        h->pass_max = h->pass_max_user ? std::min(h->pass_max_user, tc2_pass_max()) : tc2_pass_max();
        rc = build_layout(h);
        if (rc == MF_OK) h->tc_tmem = h->tc_design == 1 || h->passes.size() == 1;
        else if (h->tc_design == 1) return rc;
    }
    if (!h->tc_tmem) {
        h->pass_max = is_tc_form(f) ? (h->pass_max_user ? h->pass_max_user : 256) : h->fp32_pass_max;
        rc = build_layout(h);
        if (rc) return rc;
    }
    MF_CUDA(cudaMalloc((void **)&h->d_user_of_dev, sizeof(int) * h->Kdev));
    MF_CUDA(cudaMemcpy(h->d_user_of_dev, h->user_of_dev.data(), sizeof(int) * h->Kdev,
                       cudaMemcpyHostToDevice));
    if (!is_tc_form(f)) {
        h->Nk = (h->N + h->P + 31) / 32 * 32;
        MF_CUDA(cudaMalloc((void **)&h->d_W32, sizeof(float) * (size_t)h->Nk * h->Kdev));
        dim3 grid((h->Kdev + 127) / 128, h->Nk);
        convert_fp32_kernel<<<grid, 128>>>(h->d_W64, h->N + h->P, h->K, h->d_user_of_dev, h->Kdev,
                                           h->Nk, h->d_W32);
        MF_CUDA(cudaGetLastError());
    } else {
        rc = convert_tc_weights(h, f);
        if (rc) return rc;
    }
    if (h->d_nodes_s) cudaFree(h->d_nodes_s);
    h->d_nodes_s = nullptr;
    MF_CUDA(cudaMalloc((void **)&h->d_nodes_s, sizeof(float4) * (size_t)h->Nk));
    prescale_nodes<<<(h->Nk + 255) / 256, 256>>>(h->d_nodes64, h->N, h->Nk, rbf_prescale(h),
                                                 h->d_nodes_s);
    MF_CUDA(cudaGetLastError());
    MF_CUDA(cudaDeviceSynchronize());
    h->form = f;
    ++h->gen;
    return MF_OK;
}

}  // namespace mf

// ------------------------------------------------------------------ C ABI
extern "C" {

const char *mf_error_string(int s) {
    switch (s) {
        case MF_OK: return "MF_OK";
        case MF_E_INVAL: return "MF_E_INVAL: invalid argument";
        case MF_E_NOMEM: return "MF_E_NOMEM: allocation failed";
        case MF_E_CUDA: return "MF_E_CUDA: CUDA runtime or library error";
        case MF_E_ILLCOND: return "MF_E_ILLCOND: RBF system not positive definite";
        case MF_E_RANGE: return "MF_E_RANGE: queries outside the sampled time window";
        case MF_E_TIMEOUT: return "MF_E_TIMEOUT: bounded device wait gave up";
        case MF_E_NOTIMPL: return "MF_E_NOTIMPL: not implemented";
        case MF_E_STATE: return "MF_E_STATE: handle not configured for this call";
        default: return "unknown status";
    }
}

const char *mf_version(void) { return "mf 0.1 sm_103a"; }

int mf_svd_compress(const double *z, int N, int M, int rank, double *coef, double *basis,
                    double *sv, void *stream) {
    if (!z || !coef || !basis || N < 1 || M < 1 || M > 8192 || rank < 1 || rank > N || rank > M)
        return MF_E_INVAL;
    return mf::svd_compress(z, N, M, rank, coef, basis, sv, (cudaStream_t)stream);
}

int mf_build(const double *nodes, const double *node_values, int N, int K, mf_rbf rbf, double eps,
             int tail_degree, void *stream, mf_handle **out) {
    if (!out) return MF_E_INVAL;
    *out = nullptr;
    if (!nodes || !node_values || N < 1 || N > 65536 || K < 1 || K > 4096 || !(eps > 0) ||
        tail_degree < -1 || tail_degree > 1)
        return MF_E_INVAL;
    if (rbf < MF_RBF_GAUSSIAN || rbf > MF_RBF_IMQ) return MF_E_INVAL;
    if (tail_degree < mf::rbf_min_tail(rbf)) return MF_E_INVAL;   // no unique interpolant
    if (N <= (tail_degree < 0 ? 0 : tail_degree == 0 ? 1 : 5)) return MF_E_INVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return MF_E_CUDA;
    }
    mf_handle *h = new (std::nothrow) mf_handle();
    if (!h) return MF_E_NOMEM;
    cudaGetDevice(&h->dev);
    h->N = N;
    h->K = K;
    h->eps = eps;
    h->rbf = rbf;
    h->tail_degree = tail_degree;
    h->P = tail_degree < 0 ? 0 : (tail_degree == 0 ? 1 : 5);
    h->nodes_h.assign(nodes, nodes + (size_t)N * 4);
    int rc = MF_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMalloc((void **)&h->d_nodes64, sizeof(double) * (size_t)N * 4) != cudaSuccess ||
        cudaMalloc((void **)&h->d_bad, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc((void **)&h->d_err, 16 * sizeof(unsigned int)) != cudaSuccess) {
        cudaGetLastError();
        mf_free(h);
        return MF_E_NOMEM;
    }
    cudaMemcpy(h->d_nodes64, nodes, sizeof(double) * (size_t)N * 4, cudaMemcpyHostToDevice);
    cudaMemset(h->d_bad, 0, sizeof(unsigned long long));
    cudaMemset(h->d_err, 0, 16 * sizeof(unsigned int));
    rc = mf::rbf_build(h, node_values, st);
    if (rc == MF_OK) rc = mf::compute_stencil(h);
    if (rc != MF_OK) {
        mf_free(h);
        return rc;
    }
    *out = h;
    return MF_OK;
}

int mf_set_layout(mf_handle *h, int n_det, int n_modes, const int *ell_m, int rank) {
    if (!h || !ell_m || n_det < 1 || n_det > mf::kMaxDet || n_modes < 1 ||
        n_modes > mf::kMaxModes || rank < 1 || rank > 128)
        return MF_E_INVAL;
    if (h->K != n_det * n_modes * 2 * rank + n_det * n_modes * n_modes) return MF_E_INVAL;
    for (int i = 0; i < n_modes; ++i)
        if (!supported_mode(ell_m[2 * i], ell_m[2 * i + 1])) return MF_E_NOTIMPL;
    h->n_det = n_det;
    h->n_modes = n_modes;
    h->rank = rank;
    h->ell_m.assign(ell_m, ell_m + 2 * n_modes);
    h->have_layout = true;
    h->have_basis = false;
    h->have_det = false;
    h->sky = false;
    return mf::prepare_form(h, h->form);
}

int mf_plan_layout(int n_det, int n_modes, int rank, int pass_max, int pass_count, int *n_pass, int *pass_width,
                   int *Kdev, int *user_of_dev, int cap) {
    if (!n_pass || !pass_width || !Kdev || n_det < 1 || n_det > mf::kMaxDet || n_modes < 1 ||
        n_modes > mf::kMaxModes || rank < 1 || rank > 128 || pass_max < 16 || pass_max > 512 || pass_max % 16 ||
        pass_count < 0 || pass_count > mf::kMaxPass || cap < 0)
        return MF_E_INVAL;
    mf_handle h;   // host fields only: no device memory is touched
    h.n_det = n_det;
    h.n_modes = n_modes;
    h.rank = rank;
    h.pass_max = pass_max;
    h.pass_count = pass_count;
    const int rc = mf::build_layout(&h);
    if (rc) return rc;
    *n_pass = (int)h.passes.size();
    for (int p = 0; p < *n_pass; ++p) pass_width[p] = h.passes[p].width;
    *Kdev = h.Kdev;
    if (user_of_dev) {
        if (cap < h.Kdev) return MF_E_INVAL;
        for (int c = 0; c < h.Kdev; ++c) user_of_dev[c] = h.user_of_dev[c];
    }
    return MF_OK;
}

int mf_set_basis(mf_handle *h, const double *basis, int M, double t0, double dt) {
    if (!h || !basis || M < mf::kStencil || !(dt > 0)) return MF_E_INVAL;
    if (!h->have_layout) return MF_E_STATE;
    h->M = M;
    int rc = mf::build_cubic_table(h, basis);
    if (rc) return rc;
    h->t0 = t0;
    h->dt = dt;
    h->have_basis = true;
    ++h->gen;
    return MF_OK;
}

int mf_set_detectors(mf_handle *h, const double *det, double d_ref) {
    if (!h || !det || !(d_ref > 0)) return MF_E_INVAL;
    if (!h->have_layout) return MF_E_STATE;
    h->det.assign(det, det + 3 * h->n_det);
    h->d_ref = d_ref;
    h->sky = false;
    h->have_det = true;
    ++h->gen;
    return MF_OK;
}

int mf_set_sky(mf_handle *h, const double *tensor, const double *pos, const double *tau, double gmst0,
               double omega, double d_ref) {
    if (!h || !tensor || !pos || !(d_ref > 0) || !std::isfinite(gmst0) || !std::isfinite(omega))
        return MF_E_INVAL;
    if (!h->have_layout) return MF_E_STATE;
    const int nd = h->n_det;
    for (int i = 0; i < 9 * nd; ++i)
        if (!std::isfinite(tensor[i])) return MF_E_INVAL;
    for (int i = 0; i < 3 * nd; ++i)
        if (!std::isfinite(pos[i]) || std::fabs(pos[i]) > 1.0) return MF_E_INVAL;
    for (int k = 0; tau && k < nd; ++k)
        if (!std::isfinite(tau[k]) || std::fabs(tau[k]) > 1e7) return MF_E_INVAL;
    h->sky_tensor.assign(tensor, tensor + 9 * nd);
    h->sky_pos.assign(pos, pos + 3 * nd);
    h->sky_tau.assign(nd, 0.0);
    if (tau) h->sky_tau.assign(tau, tau + nd);
    h->gmst0 = gmst0;
    h->omega_e = omega;
    // the frozen per-detector values are unused; the sample offset of t_c = 0
    // is the same for every channel (its delay is added per query)
    h->det.assign(3 * nd, 0.0);
    h->d_ref = d_ref;
    h->sky = true;
    h->have_det = true;
    ++h->gen;
    return MF_OK;
}

int mf_set_rotation(mf_handle *h, const double *metric, const double *centre) {
    if (!h) return MF_E_INVAL;
    if (metric) {
        double R[16];
        int rc = mf::metric_eig(metric, R);
        if (rc) return rc;
        memcpy(h->R, R, sizeof(R));
    } else {
        for (int i = 0; i < 16; ++i) h->R[i] = (i % 5 == 0) ? 1.0 : 0.0;
    }
    for (int i = 0; i < 4; ++i) h->centre[i] = centre ? centre[i] : 0.0;
    ++h->gen;
    return MF_OK;
}

int mf_set_frame(mf_handle *h, const double *A, const double *centre) {
    if (!h || !A) return MF_E_INVAL;
    for (int i = 0; i < 16; ++i)
        if (!std::isfinite(A[i])) return MF_E_INVAL;
    memcpy(h->R, A, sizeof(h->R));
    for (int i = 0; i < 4; ++i) h->centre[i] = centre ? centre[i] : 0.0;
    ++h->gen;
    return MF_OK;
}

int mf_set_form(mf_handle *h, mf_form f) {
    if (!h || f < MF_FORM_FP32 || f > MF_FORM_MLP) return MF_E_INVAL;
    if (f == MF_FORM_MLP && !h->sur) return MF_E_STATE;   // train the surrogate first
    if (!h->have_layout) {
        h->form = f;
        return MF_OK;
    }
    if (f == h->form && f != MF_FORM_MLP && (h->d_W32 || h->d_Whi)) return MF_OK;
    return mf::prepare_form(h, f);
}

static const int kMaxPassCount = 8;

static int ensure_partial(mf_handle *h, size_t need) {
    if (need <= h->partial_cap) return MF_OK;
    if (h->d_partial) cudaFree(h->d_partial);
    h->d_partial = nullptr;
    h->partial_cap = 0;
    MF_CUDA(cudaMalloc((void **)&h->d_partial, sizeof(float) * need));
    h->partial_cap = need;
    return MF_OK;
}

int mf_loglike(mf_handle *h, const float *intrinsic, const float *extrinsic, int Q, int E,
               float *out_lnL, void *stream) {
    if (!h || Q < 0 || Q > (1 << 26) || E < 5) return MF_E_INVAL;
    if (Q == 0) return MF_OK;
    if (!intrinsic || !extrinsic || !out_lnL) return MF_E_INVAL;
    if ((uintptr_t)intrinsic & 15) return MF_E_INVAL;   // rows are read as float4
    if (!h->have_layout || !h->have_basis || !h->have_det) return MF_E_STATE;
    if (h->sky && E < 7) return MF_E_INVAL;   // (alpha, delta) columns needed
    cudaStream_t st = (cudaStream_t)stream;
    if (h->form == MF_FORM_MLP) {
        if (h->timing) MF_CUDA(cudaEventRecord(h->ev0, st));
        int rc = mf::loglike_surrogate(h, intrinsic, extrinsic, Q, E, out_lnL, st, false);
        if (h->timing) MF_CUDA(cudaEventRecord(h->ev1, st));
        return rc;
    }
    const int np = (int)h->passes.size();
    float *partial = nullptr;
    if (np > 1) {
        int rc = ensure_partial(h, (size_t)np * Q);
        if (rc) return rc;
        partial = h->d_partial;
    }
    if (h->timing) MF_CUDA(cudaEventRecord(h->ev0, st));
    int rc = !mf::is_tc_form(h->form) ? mf::launch_fp32(h, intrinsic, extrinsic, Q, E, out_lnL, st, partial)
             : h->tc_tmem ? mf::launch_tc2(h, intrinsic, extrinsic, Q, E, out_lnL, st, partial)
                            : mf::launch_tc(h, intrinsic, extrinsic, Q, E, out_lnL, st, partial);
    if (rc) return rc;
    if (h->timing) MF_CUDA(cudaEventRecord(h->ev1, st));
    if (np > 1) return mf::launch_combine(partial, np, Q, out_lnL, st, h->d_bad);
    return MF_OK;
}

int mf_eval_columns(mf_handle *h, const float *intrinsic, int Q, float *out, void *stream) {
    if (!h || Q < 0 || Q > (1 << 26)) return MF_E_INVAL;
    if (Q == 0) return MF_OK;
    if (!intrinsic || !out) return MF_E_INVAL;
    if ((uintptr_t)intrinsic & 15) return MF_E_INVAL;
    if (!h->have_layout) return MF_E_STATE;
    cudaStream_t st = (cudaStream_t)stream;
    if (mf::is_tc_form(h->form))
        return h->tc_tmem ? mf::launch_tc2(h, intrinsic, nullptr, Q, 5, nullptr, st, nullptr, out)
                          : mf::launch_tc(h, intrinsic, nullptr, Q, 5, nullptr, st, nullptr, out);
    if (h->form == MF_FORM_MLP) return mf::eval_columns_surrogate(h, intrinsic, Q, out, st);
    if (h->form != MF_FORM_FP32) return MF_E_NOTIMPL;
    return mf::launch_fp32_columns(h, intrinsic, Q, out, st);
}

int mf_set_option(mf_handle *h, const char *key, double value) {
    if (!h || !key) return MF_E_INVAL;
    std::string k(key);
    if (k == "timing") {
        if (value != 0 && !h->ev0) {
            MF_CUDA(cudaEventCreate(&h->ev0));
            MF_CUDA(cudaEventCreate(&h->ev1));
        }
        h->timing = value != 0;
        return MF_OK;
    }
    if (k == "pass_max") {
        int v = (int)value;
        if (v < 16 || v > 512 || v % 16) return MF_E_INVAL;
        h->pass_max_user = v;
        if (h->have_layout && mf::is_tc_form(h->form)) return mf::prepare_form(h, h->form);
        return MF_OK;
    }
    if (k == "pass_count") {
        int v = (int)value;
        if (v < 0 || v > kMaxPassCount || v != value) return MF_E_INVAL;
        const int old = h->pass_count_user;
        h->pass_count_user = v;
        if (h->have_layout && (h->d_W32 || h->d_Whi)) {
            int rc = mf::prepare_form(h, h->form);
            if (rc) {   // keep the previous, still valid layout
                h->pass_count_user = old;
                mf::prepare_form(h, h->form);
                return rc;
            }
        }
        return MF_OK;
    }
    if (k == "tc_design") {
        int v = (int)value;
        if (v < -1 || v > 1) return MF_E_INVAL;
        h->tc_design = v;
        if (h->have_layout && mf::is_tc_form(h->form)) return mf::prepare_form(h, h->form);
        return MF_OK;
    }
    if (k == "tc_pair") {
        if (value != 0 && value != 1) return MF_E_INVAL;
        h->tc_pair = (int)value;
        return MF_OK;
    }
    if (k == "tc_rot") {   // rotate each query tile's node-block order (1, default) or not (0)
        if (value != 0 && value != 1) return MF_E_INVAL;
        h->tc_rot = (int)value;
        return MF_OK;
    }
    if (k == "tc_chunk") {   // passes per cluster launch at most (0: as many as fit)
        if (value < 0 || value > 8 || value != (int)value || value == 1) return MF_E_INVAL;
        h->tc_chunk = (int)value;
        return MF_OK;
    }
    if (k == "tc_nbs") {
        int v = (int)value;
        if (v != 0 && (v < 2 || v > 6)) return MF_E_INVAL;
        h->tc_nbs = v;
        return MF_OK;
    }
    return MF_E_INVAL;
}

int mf_sync_status(mf_handle *h, void *stream, long long *n_bad) {
    if (!h) return MF_E_INVAL;
    MF_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    unsigned long long b = 0;
    unsigned int err = 0;
    MF_CUDA(cudaMemcpy(&b, h->d_bad, sizeof(b), cudaMemcpyDeviceToHost));
    unsigned int ew[16];
    MF_CUDA(cudaMemcpy(ew, h->d_err, sizeof(ew), cudaMemcpyDeviceToHost));
    err = ew[0];
    if (err) {
        mf::log_msg("device status 0x%x; first give-up k-block+1 per site:", err);
        for (int i = 1; i < 9; ++i)
            if (ew[i]) mf::log_msg("  site %d: %u", i - 1, ew[i]);
    }
    MF_CUDA(cudaMemset(h->d_bad, 0, sizeof(b)));
    MF_CUDA(cudaMemset(h->d_err, 0, sizeof(ew)));
    if (n_bad) *n_bad = (long long)b;
    if (err) return MF_E_TIMEOUT;
    return b ? MF_E_RANGE : MF_OK;
}

int mf_query(const mf_handle *h, const char *key, double *value) {
    if (!h || !key || !value) return MF_E_INVAL;
    std::string k(key);
    if (k == "cond") *value = h->cond;
    else if (k == "lambda_min") *value = h->lam_min;
    else if (k == "lambda_max") *value = h->lam_max;
    else if (k == "cancel") *value = h->cancel;
    else if (k == "N") *value = h->N;
    else if (k == "K") *value = h->K;
    else if (k == "n_pass") *value = (double)h->passes.size();
    else if (k == "Kdev") *value = h->Kdev;
    else if (k == "form") *value = (double)h->form;
    else if (k == "tc_design") *value = h->tc_tmem ? 1.0 : 0.0;
    else if (k == "tc_paired") *value = h->tc_paired;
    else if (k == "launches" && h->form == MF_FORM_MLP)
        return mf::surrogate_query(h, k, value);
    else if (k == "launches")
        *value = 1.0 + (h->passes.size() > 1 ? 1.0 : 0.0);
    else if (k.compare(0, 9, "surrogate") == 0 || k == "fallback_rate")
        return mf::surrogate_query(h, k, value);
    else if (k == "kernel_ms") {
        if (!h->timing) return MF_E_STATE;
        float ms = 0.f;
        MF_CUDA(cudaEventSynchronize(h->ev1));
        MF_CUDA(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
        *value = ms;
    }
    else return MF_E_INVAL;
    return MF_OK;
}

int mf_get_weights(const mf_handle *h, double *W_host, size_t count) {
    if (!h || !W_host || count < (size_t)(h->N + h->P) * h->K) return MF_E_INVAL;
    MF_CUDA(cudaMemcpy(W_host, h->d_W64, sizeof(double) * (size_t)(h->N + h->P) * h->K,
                       cudaMemcpyDeviceToHost));
    return MF_OK;
}

void mf_free(mf_handle *h) {
    if (!h) return;
    mf::free_surrogate(h);
    free_form(h);
    if (h->d_nodes64) cudaFree(h->d_nodes64);
    if (h->d_W64) cudaFree(h->d_W64);
    if (h->d_cubic) cudaFree(h->d_cubic);
    if (h->d_nodes_s) cudaFree(h->d_nodes_s);
    if (h->d_bad) cudaFree(h->d_bad);
    if (h->d_err) cudaFree(h->d_err);
    if (h->d_partial) cudaFree(h->d_partial);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    delete h;
}

}  // extern "C"
