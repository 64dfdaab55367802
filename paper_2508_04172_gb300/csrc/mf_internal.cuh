// Internal definitions shared by the libmf translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <cmath>
#include <vector>
#include <string>

#include "../../include/mf.h"

namespace mf {

constexpr int kMaxDet = 8;
constexpr int kMaxModes = 5;
constexpr int kMaxGroups = kMaxDet * (kMaxModes + 1);
constexpr int kMaxPass = kMaxGroups;
constexpr int kStencil = 10;          // spline samples j-4 .. j+5
constexpr int kStencilLo = 4;         // samples before the evaluation interval
constexpr int kTile = 128;            // queries per tile (one TMEM lane each)
constexpr int kGroupAlign = 8;        // every column group padded to 8 columns
constexpr int kPassAlign = 16;        // pass width multiple of 16 (MMA N granularity)

// One column group of the device layout: a detector/mode overlap block
// (interleaved Re/Im of a run of its SVD coefficients) or a detector's
// cross-term block (n_modes diagonals then interleaved Re/Im of the strict
// upper triangle).
struct Group {
    int kind;     // 0 = overlap z_k,mu ; 1 = cross terms sigma_k
    int det;
    int mode;     // overlap groups only
    int col;      // first device column of the group, relative to its pass
    int width;    // padded width (multiple of kGroupAlign)
    int i0, ni;   // overlap groups: SVD coefficients [i0, i0 + ni) of the mode (a mode
                  // may be split over several groups; lnL is linear in each coefficient)
};

struct Pass {
    int col0;     // first device column of the pass (in the device layout)
    int width;    // padded width (multiple of kPassAlign)
    int g0, ng;   // groups [g0, g0+ng)
};

// Everything the per-query epilogue needs; passed by value to kernels.
struct EpiParams {
    int n_det, n_modes, rank, M;
    int ell[kMaxModes], em[kMaxModes];
    float fp0[kMaxDet], fx0[kMaxDet];
    int J[kMaxDet];          // integer part of (dt_k - t0)/dt
    float frac[kMaxDet];     // fractional part of (dt_k - t0)/dt
    float inv_dt;            // 1/dt
    float d_ref;
    // per (detector, mode, sample j, coefficient i): the cubic in u in [0,1)
    // that the not-a-knot spline through samples j-4..j+5 of basis vector i
    // takes on [j, j+1]; two float4 = (c0, c1), (c2, c3) complex
    const float4 *cubic;     // [n_det][n_modes][M][rank][2]
    unsigned long long *bad; // out-of-window counter
    unsigned int *err;       // device status word: bit 0 = bounded wait gave up
    Group groups[kMaxGroups];
    Pass passes[kMaxPass];
    int n_groups, n_pass;
    // sky-dependent patterns (sky != 0): extrinsic columns 5, 6 = (alpha, delta)
    int sky;
    float dten[kMaxDet][6];  // detector tensor (xx, yy, zz, xy, xz, yz), Earth-fixed frame
    float dpos[kMaxDet][3];  // detector position / c (seconds)
    float gk[kMaxDet];       // sidereal angle at t_c = 0 of channel k: gmst0 + omega tau_k (mod 2 pi)
    float omega;             // Earth's rotation rate (rad/s)
};

struct RotParams {
    float R[16];
    float centre[4];
    float pre;               // Gaussian: eps * sqrt(log2 e), exp(-(eps r)^2) = exp2(-|pre (x - y)|^2);
                             // other kernels: eps, s^2 = |pre (x - y)|^2
    int rbf;                 // mf_rbf
};

// phi at s2 = (eps r)^2 for the kernels other than the Gaussian (mf_rbf):
// PHS3 s^3, MQ sqrt(1 + s^2), IMQ 1 / sqrt(1 + s^2)
__device__ __forceinline__ float rbf_other(int kind, float s2) {
    return kind == 1 ? s2 * sqrtf(s2) : kind == 2 ? sqrtf(1.f + s2) : rsqrtf(1.f + s2);
}
// phi at s2 = (eps r)^2 in FP64, every kernel (start-up and labels)
__device__ __forceinline__ double rbf_phi64(int kind, double s2) {
    return kind == 0 ? exp(-s2) : kind == 1 ? s2 * sqrt(s2) : kind == 2 ? sqrt(1.0 + s2) : 1.0 / sqrt(1.0 + s2);
}

// One interpolant as the tcgen05 kernel sees it: everything that does not
// change from call to call.  Passed by value (one event) or as a device
// array (batched launch).
struct TcEvent {
    CUtensorMap tm_hi, tm_lo;   // W_hi / W_lo [Kdev][Nk] K-major, box kKB x nbox
    CUtensorMap tm_hi2, tm_lo2; // the same with half-height boxes (nbox / 2 rows): paired launch
    EpiParams epi;
    RotParams rot;
    const float4 *nodes_s;      // [Nk] nodes * (-pre), padding zero
    const float *colscale;      // [Kdev] per-column scale (FP16 forms) or nullptr
    int N, P;                   // nodes, tail monomials
    int nkb;                    // node blocks of 32 (Nk / 32)
    int nbox;                   // rows of one W tile = widest pass of this event
    int pair_ok;                // half-height maps exist (nbox / 2 a multiple of 8 rows)
    int rot_mul;                // node-block order of tile t starts at rot_mul * (t / 2) mod n_kb (0: at 0)
};

// Per-call arguments of a batched launch (kernel parameter; < 32 KB).
constexpr int kMaxBatch = 128;
struct TcBatchCall {
    int n_ev, n_items, E, np;    // events, work items, extrinsic stride, passes (= cluster size)
    int n_clusters, sb, nbox_max;
    unsigned *err;               // device status words of the batch
    int order[kMaxBatch];        // events by decreasing cost per tile
    int tprefix[kMaxBatch + 1];  // first work item of order[k]
    int qprefix[kMaxBatch + 1];  // first query of event e (event order)
    int Q[kMaxBatch];
    const float *intr[kMaxBatch];
    const float *ext[kMaxBatch];
    float *out[kMaxBatch];
    float *partial[kMaxBatch];   // [np][Q] per event (np > 1)
    unsigned long long *bad[kMaxBatch];
};

}  // namespace mf

struct mf_surrogate;

struct mf_handle {
    int dev = 0;
    int N = 0, K = 0, P = 0, tail_degree = 1;
    double eps = 0.0;
    mf_rbf rbf = MF_RBF_GAUSSIAN;
    // FP64 results of the build
    double *d_nodes64 = nullptr;   // [N][4]
    double *d_W64 = nullptr;       // [(N+P)][K] (user column order)
    double cond = 0, lam_min = 0, lam_max = 0, cancel = 0;
    std::vector<double> nodes_h;   // host copy [N][4]
    // layout
    bool have_layout = false, have_basis = false, have_det = false;
    int n_det = 0, n_modes = 0, rank = 0, M = 0;
    std::vector<int> ell_m;
    double t0 = 0, dt = 0, d_ref = 100.0;
    std::vector<double> det;       // [n_det][3]
    // sky-dependent patterns (mf_set_sky)
    bool sky = false;
    std::vector<double> sky_tensor; // [n_det][3][3]
    std::vector<double> sky_pos;    // [n_det][3] seconds
    std::vector<double> sky_tau;    // [n_det] seconds
    double gmst0 = 0, omega_e = 0;
    float4 *d_cubic = nullptr;      // spline cubic table (see EpiParams::cubic)
    // rotation
    double R[16] = {1,0,0,0, 0,1,0,0, 0,0,1,0, 0,0,0,1};
    double centre[4] = {0, 0, 0, 0};
    // device layout & passes (per form family)
    std::vector<mf::Group> groups;
    std::vector<mf::Pass> passes;
    int Kdev = 0;                   // total device columns (sum of pass widths)
    std::vector<int> user_of_dev;   // device column -> user column (-1: padding)
    int *d_user_of_dev = nullptr;
    int pass_max = 256;
    // weights per form
    mf_form form = MF_FORM_FP32;
    int Nk = 0;                     // N + P padded (node dimension of the weights)
    float *d_W32 = nullptr;         // [Nk][Kdev]
    float4 *d_nodes_s = nullptr;    // nodes * (-pre) [Nk] (negated, prescaled; padding zero)
    void *d_Whi = nullptr, *d_Wlo = nullptr;  // 16-bit K-major [Kdev][Nk]
    float *d_colscale = nullptr;    // per device column scale (FP16 forms)
    mf_form tc_form_built = MF_FORM_FP32;
    // spline constants (device-computed, copied to host params)
    double G4[mf::kStencil], G5[mf::kStencil];
    bool have_stencil = false;
    // instrumentation / tuning
    bool timing = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int tc_nbs = 0;                 // W ring depth of the tcgen05 kernel (0: automatic)
    int tc_design = -1;             // -1: automatic; 0: cluster-shared Phi in smem; 1: Phi in TMEM
    bool tc_tmem = false;           // the current layout runs the TMEM design
    int pass_max_user = 0;          // 0: form default
    int pass_count_user = 0;        // 0: as few passes as pass_max allows; else exactly this many
    int pass_count = 0;             // the value the current layout was built with (tcgen05 forms)
    int fp32_pass_max = 176;        // widest FP32 pass (the surrogate form lays out narrower passes)
    unsigned gen = 0;               // bumped whenever the device layout or weights change
    // tcgen05 forms: tensor maps (opaque 128-byte CUtensorMap) of W_hi / W_lo
    alignas(64) unsigned char tmap_hi[128];
    alignas(64) unsigned char tmap_lo[128];
    alignas(64) unsigned char tmap_hi2[128];   // half-height boxes (paired launch)
    alignas(64) unsigned char tmap_lo2[128];
    bool pair_ok = false;           // the half-height maps exist
    int tc_pair = 1;                // 1: pair two query tiles per cluster when possible, 0: never
    int tc_chunk = 0;               // passes per cluster launch at most (0: as many as fit)
    int tc_paired = 0;              // the last cluster launch paired two query tiles
    int tc_rot = 1;                 // 1: rotate each tile's node-block order (spreads weight reads), 0: no
    int nbox = 0;                   // rows (device columns) per W tile = widest pass
    // scratch
    unsigned long long *d_bad = nullptr;
    unsigned int *d_err = nullptr;
    float *d_partial = nullptr;     // [n_pass][Q] partial lnL
    size_t partial_cap = 0;
    // trained surrogate network (MF_FORM_MLP), or nullptr
    mf_surrogate *sur = nullptr;
};

namespace mf {
// Smallest tail degree giving a unique interpolant for the kernel (the rule
// after Eq. rbfcoeff: conditionally positive definite of order r needs the
// monomials of degree r - 1): PHS3 order 2, MQ order 1, Gaussian / IMQ none.
inline int rbf_min_tail(int rbf) { return rbf == MF_RBF_PHS3 ? 1 : rbf == MF_RBF_MQ ? 0 : -1; }
// Node / query prescale: the Gaussian folds log2 e in (the kernels use exp2).
inline double rbf_prescale(const mf_handle *h) {
    return h->rbf == MF_RBF_GAUSSIAN ? h->eps * std::sqrt(1.0 / std::log(2.0)) : h->eps;
}
int cuda_status(cudaError_t e);
// Diagnostics to stderr when the environment variable MF_LOG is set.
void log_msg(const char *fmt, ...);
int build_layout(mf_handle *h);             // groups/passes/device column map
int prepare_form(mf_handle *h, mf_form f);  // convert weights for a form
int compute_stencil(mf_handle *h);          // spline operator rows on the GPU
int build_cubic_table(mf_handle *h, const double *basis_host);  // spline cubics per interval
EpiParams make_epi(const mf_handle *h);
RotParams make_rot(const mf_handle *h);
// kernels launchers
// dQ != nullptr: the batch size is *dQ (<= Q), read on the device
int launch_fp32(mf_handle *h, const float *intr, const float *ext, int Q, int E, float *out,
                cudaStream_t st, float *partial, const int *dQ = nullptr);
int launch_fp32_columns(mf_handle *h, const float *intr, int Q, float *out, cudaStream_t st);
// cols != nullptr: interpolated columns only, out [Q][K] (mf_eval_columns)
int launch_tc(mf_handle *h, const float *intr, const float *ext, int Q, int E, float *out,
              cudaStream_t st, float *partial, float *cols = nullptr);
int launch_combine(const float *partial, int n_pass, int Q, float *out, cudaStream_t st,
                   unsigned long long *bad, const int *dQ = nullptr);
int launch_tc2(mf_handle *h, const float *intr, const float *ext, int Q, int E, float *out,
               cudaStream_t st, float *partial, float *cols = nullptr);
int tc2_pass_max();
// C[m][n] = A[m][k] B[k][n], row-major FP64 (stream-ordered)
int dgemm_rm(int m, int n, int k, const double *A, int lda, const double *B, int ldb, double *C, int ldc,
             cudaStream_t st);
// batched tcgen05 launch (all events share form and mode count)
int fill_tc_event(const mf_handle *h, TcEvent *out);
size_t tc_smem_bytes(mf_form f, int np, int nbox_max, int sb);   // 0: does not fit
int tc_max_passes(mf_form f, int nbox);   // passes one cluster launch stages
int tc_batch_max_clusters(mf_form f, int n_modes, int np, int nbox_max, int sb, int *max_clusters);
int launch_tc_batch(mf_form f, int n_modes, const TcEvent *d_events, const TcBatchCall &bc,
                    cudaStream_t st);
bool is_tc_form(mf_form f);
// surrogate network (MF_FORM_MLP)
int metric_eig(const double *metric, double *R_out);   // rows = eigenvectors, ascending
int surrogate_prepare(mf_handle *h);
void free_surrogate(mf_handle *h);
int loglike_surrogate(mf_handle *h, const float *intr, const float *ext, int Q, int E, float *out,
                      cudaStream_t st, bool force_net);
int surrogate_query(const mf_handle *h, const std::string &key, double *value);
int eval_columns_surrogate(mf_handle *h, const float *intr, int Q, float *out, cudaStream_t st);
// tensor map of a 16-bit [rows][K] matrix (at: 0 = FP16, 1 = BF16), box K 32 x box_rows
int make_tmap(void *out, void *base, int at, int K, int rows, int box_rows);
}  // namespace mf

#define MF_CUDA(call)                                                              \
    do {                                                                           \
        cudaError_t e__ = (call);                                                  \
        if (e__ != cudaSuccess) {                                                  \
            mf::log_msg("%s:%d %s -> %s", __FILE__, __LINE__, #call,               \
                        cudaGetErrorString(e__));                                  \
            return mf::cuda_status(e__);                                           \
        }                                                                          \
    } while (0)

#define MF_LIBCALL(call)                                                           \
    do {                                                                           \
        int s__ = (int)(call);                                                     \
        if (s__ != 0) {                                                            \
            mf::log_msg("%s:%d %s -> status %d", __FILE__, __LINE__, #call, s__);   \
            return MF_E_CUDA;                                                      \
        }                                                                          \
    } while (0)
