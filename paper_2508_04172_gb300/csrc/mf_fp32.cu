// Plain FP32 form of the fused lnL kernel (SIMT FMAs, no tensor cores).
//
// One CTA evaluates one (query tile of 128, column pass) work item:
//   1. rotate the 128 queries into the metric eigenbasis (Sec. II D, Delta-e),
//   2. per chunk of 32 interpolation nodes: Gaussian RBF values (or the tail
//      monomials 1, x1..x4 for the last P rows) into shared memory, the weight
//      chunk into shared memory, and an 8x12 register-tiled FMA update of the
//      128 x width interpolated columns (Eq. rbfcoeff),
//   3. stage the columns in shared memory and run the per-query epilogue
//      (SVD reconstruction + spline at the detector delay + amplitudes +
//      cross-term form: Eqs. SVD, projected_h_fd, logl_complete).
// Passes of one tile write partial lnL; a combine kernel sums them in a
// fixed order (so results are bitwise reproducible).
#include "mf_epilogue.cuh"

#include <algorithm>

namespace mf {

namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 32;       // nodes per shared-memory chunk
constexpr int kJMax = 11;        // columns per thread (stride 16) -> pass width <= 176
constexpr int kWidthMax = 16 * kJMax;

struct SmemAcc {
    const float *row;
    __device__ void load8(int col, float (&f)[8]) const {
#pragma unroll
        for (int e = 0; e < 8; ++e) f[e] = row[col + e];
    }
};

__device__ __forceinline__ void rotate_query(const RotParams &rot, const float *intr, int q,
                                             float (&xu)[4]) {
    float4 th = *reinterpret_cast<const float4 *>(intr + (size_t)q * 4);
    float d[4] = {th.x - rot.centre[0], th.y - rot.centre[1], th.z - rot.centre[2],
                  th.w - rot.centre[3]};
#pragma unroll
    for (int i = 0; i < 4; ++i)
        xu[i] = rot.R[4 * i] * d[0] + rot.R[4 * i + 1] * d[1] + rot.R[4 * i + 2] * d[2] +
                rot.R[4 * i + 3] * d[3];
}

// One (query tile, column pass) work item.
template <int NM, bool COLUMNS>
__device__ __forceinline__ void fp32_tile(const float *__restrict__ intr, const float *__restrict__ ext, int Q,
                                          int E, int N, int P, int Nk, const float *__restrict__ W, int Kdev,
                                          const float4 *__restrict__ nodes_s, const RotParams &rot,
                                          const EpiParams &epi, float *__restrict__ out,
                                          float *__restrict__ partial, const int *__restrict__ user_of_dev,
                                          const float *__restrict__ colscale, int Kuser, int tile) {
    extern __shared__ __align__(16) float smem[];
    const int tid = threadIdx.x;
    const int pass = blockIdx.y;
    const Pass ps = epi.passes[pass];
    const int width = ps.width;
    const int jw = width >> 4;
    const int q0 = tile * kTile;

    float4 *xs_s = reinterpret_cast<float4 *>(smem);            // [128] prescaled x
    float4 *xu_s = xs_s + kTile;                                 // [128] unscaled x
    float *phi_s = smem + 8 * kTile;                             // [kChunk][128]
    float *w_s = phi_s + kChunk * kTile;                         // [kChunk][width]
    float *F_s = smem + 8 * kTile;                               // [128][width+1] (aliases)

    if (tid < kTile) {
        int q = min(q0 + tid, Q - 1);
        float xu[4];
        rotate_query(rot, intr, q, xu);
        xu_s[tid] = make_float4(xu[0], xu[1], xu[2], xu[3]);
        xs_s[tid] = make_float4(xu[0] * rot.pre, xu[1] * rot.pre, xu[2] * rot.pre, xu[3] * rot.pre);
    }

    const int tq = tid >> 4, tc = tid & 15;
    float2 acc[4][kJMax];      // rows (2h, 2h+1) of this thread, packed for fma.rn.f32x2
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < kJMax; ++j) acc[i][j] = make_float2(0.f, 0.f);

    const int wq = tid & (kTile - 1);          // query handled when filling phi
    const int wn0 = (tid >> 7) * (kChunk / 2); // 16 nodes per thread
    for (int n0 = 0; n0 < Nk; n0 += kChunk) {
        __syncthreads();
        // weights chunk: rows n0..n0+31, columns [ps.col0, ps.col0 + width)
        const int w4 = width >> 2;
        for (int e = tid; e < kChunk * w4; e += kThreads) {
            int r = e / w4, c4 = e - r * w4;
            float4 v = *reinterpret_cast<const float4 *>(W + (size_t)(n0 + r) * Kdev + ps.col0 + 4 * c4);
            *reinterpret_cast<float4 *>(w_s + r * width + 4 * c4) = v;
        }
        // RBF values (Gaussian exp(-eps^2 |x - y|^2) = exp2(-|pre (x - y)|^2),
        // other kernels phi(s^2 = |pre (x - y)|^2)), tail monomials
        {
            float4 xs = xs_s[wq];
            float4 xu = xu_s[wq];
#pragma unroll 4
            for (int t = 0; t < kChunk / 2; ++t) {
                int n = n0 + wn0 + t;
                float v;
                if (n < N) {
                    float4 y = __ldg(nodes_s + n);
                    float d0 = xs.x + y.x, d1 = xs.y + y.y, d2 = xs.z + y.z, d3 = xs.w + y.w;   // y negated
                    float r2 = d0 * d0;
                    r2 = fmaf(d1, d1, r2);
                    r2 = fmaf(d2, d2, r2);
                    r2 = fmaf(d3, d3, r2);
                    v = rot.rbf == 0 ? exp2f(-r2) : rbf_other(rot.rbf, r2);
                } else {
                    int p = n - N;
                    v = (p == 0) ? 1.f : (p == 1) ? xu.x : (p == 2) ? xu.y : (p == 3) ? xu.z
                                                                                 : xu.w;
                    if (p >= P) v = 0.f;
                }
                phi_s[(wn0 + t) * kTile + wq] = v;
            }
        }
        __syncthreads();
#pragma unroll 2
        for (int n = 0; n < kChunk; ++n) {
            float4 p0 = *reinterpret_cast<const float4 *>(phi_s + n * kTile + tq * 8);
            float4 p1 = *reinterpret_cast<const float4 *>(phi_s + n * kTile + tq * 8 + 4);
            const float2 p[4] = {make_float2(p0.x, p0.y), make_float2(p0.z, p0.w), make_float2(p1.x, p1.y),
                                 make_float2(p1.z, p1.w)};
            float wv[kJMax];
#pragma unroll
            for (int j = 0; j < kJMax; ++j) wv[j] = (j < jw) ? w_s[n * width + tc + 16 * j] : 0.f;
#pragma unroll
            for (int j = 0; j < kJMax; ++j) {
                const float2 w2 = make_float2(wv[j], wv[j]);
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[i][j] = __ffma2_rn(p[i], w2, acc[i][j]);
            }
        }
    }
    __syncthreads();
    // stage the tile's columns: F_s[q][col], row stride width+1
    const int ld = width + 1;
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < kJMax; ++j)
            if (j < jw) F_s[(tq * 8 + i) * ld + tc + 16 * j] = (i & 1) ? acc[i >> 1][j].y : acc[i >> 1][j].x;
    __syncthreads();

    if (COLUMNS) {
        // write interpolated columns in the user's column order
        for (int e = tid; e < kTile * width; e += kThreads) {
            int r = e / width, c = e - r * width;
            int q = q0 + r;
            int u = user_of_dev[ps.col0 + c];
            if (q < Q && u >= 0) {
                float s = colscale ? colscale[ps.col0 + c] : 1.f;
                out[(size_t)q * Kuser + u] = F_s[r * ld + c] * s;
            }
        }
        return;
    }
    if (tid < kTile) {
        int q = q0 + tid;
        if (q < Q) {
            QueryExt x = load_ext(epi, ext, E, q);
            SmemAcc a{F_s + tid * ld};
            bool bad = false;
            float l = pass_lnl<NM>(epi, ps, x, a, bad);
            if (bad) l = __int_as_float(0x7fc00000);
            if (epi.n_pass == 1) {
                out[q] = l;
                if (l != l) atomicAdd(epi.bad, 1ull);
            } else {
                partial[(size_t)pass * Q + q] = l;
            }
        }
    }
}

// dQ == nullptr: one tile per CTA (grid.x = tiles of Q).  Otherwise the batch
// size is read on the device (a count another kernel produced, so that the
// host need not wait for it): the CTAs stride over the tiles of *dQ queries.
template <int NM, bool COLUMNS>
__global__ void __launch_bounds__(kThreads, 2)
fp32_kernel(const float *__restrict__ intr, const float *__restrict__ ext, int Q, int E,
            int N, int P, int Nk, const float *__restrict__ W, int Kdev,
            const float4 *__restrict__ nodes_s, RotParams rot, EpiParams epi,
            float *__restrict__ out, float *__restrict__ partial,
            const int *__restrict__ user_of_dev, const float *__restrict__ colscale, int Kuser,
            const int *__restrict__ dQ) {
    if (!dQ) {
        fp32_tile<NM, COLUMNS>(intr, ext, Q, E, N, P, Nk, W, Kdev, nodes_s, rot, epi, out, partial, user_of_dev,
                               colscale, Kuser, blockIdx.x);
        return;
    }
    const int Qd = min(*dQ, Q);
    const int nt = (Qd + kTile - 1) / kTile;
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        fp32_tile<NM, COLUMNS>(intr, ext, Qd, E, N, P, Nk, W, Kdev, nodes_s, rot, epi, out, partial,
                               user_of_dev, colscale, Kuser, t);
        __syncthreads();   // shared memory is reused by the next tile
    }
}

__global__ void combine_kernel(const float *__restrict__ partial, int n_pass, int Q,
                               float *__restrict__ out, unsigned long long *bad, const int *__restrict__ dQ) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (dQ) Q = min(*dQ, Q);
    if (q >= Q) return;
    float s = 0.f;
    for (int p = 0; p < n_pass; ++p) s += partial[(size_t)p * Q + q];
    out[q] = s;
    if (s != s) atomicAdd(bad, 1ull);
}

template <int NM, bool COLUMNS>
int launch_fp32_nm(mf_handle *h, const float *intr, const float *ext, int Q, int E, float *out,
                   cudaStream_t st, float *partial, int Kuser, const int *dQ) {
    EpiParams epi = make_epi(h);
    RotParams rot = make_rot(h);
    int maxw = 0;
    for (auto &p : h->passes) maxw = p.width > maxw ? p.width : maxw;
    if (maxw > kWidthMax) return MF_E_NOTIMPL;
    size_t gemm = (size_t)8 * kTile + (size_t)kChunk * kTile + (size_t)kChunk * maxw;
    size_t epis = (size_t)8 * kTile + (size_t)kTile * (maxw + 1);
    size_t bytes = sizeof(float) * (gemm > epis ? gemm : epis);
    auto kern = fp32_kernel<NM, COLUMNS>;
    MF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    int tiles = (Q + kTile - 1) / kTile;
    if (dQ) {   // at most two resident waves of CTAs stride over the device-counted tiles
        int sms = 0, dev = 0;
        MF_CUDA(cudaGetDevice(&dev));
        MF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        tiles = std::max(1, std::min(tiles, 2 * sms));
    }
    dim3 grid((unsigned)tiles, (unsigned)h->passes.size());
    kern<<<grid, kThreads, bytes, st>>>(intr, ext, Q, E, h->N, h->P, h->Nk, h->d_W32, h->Kdev,
                                        h->d_nodes_s, rot, epi, out, partial, h->d_user_of_dev,
                                        nullptr, Kuser, dQ);
    MF_CUDA(cudaGetLastError());
    return MF_OK;
}

template <bool COLUMNS>
int launch_fp32_any(mf_handle *h, const float *intr, const float *ext, int Q, int E, float *out,
                    cudaStream_t st, float *partial, int Kuser, const int *dQ) {
    switch (h->n_modes) {
        case 1: return launch_fp32_nm<1, COLUMNS>(h, intr, ext, Q, E, out, st, partial, Kuser, dQ);
        case 2: return launch_fp32_nm<2, COLUMNS>(h, intr, ext, Q, E, out, st, partial, Kuser, dQ);
        case 3: return launch_fp32_nm<3, COLUMNS>(h, intr, ext, Q, E, out, st, partial, Kuser, dQ);
        case 4: return launch_fp32_nm<4, COLUMNS>(h, intr, ext, Q, E, out, st, partial, Kuser, dQ);
        case 5: return launch_fp32_nm<5, COLUMNS>(h, intr, ext, Q, E, out, st, partial, Kuser, dQ);
        default: return MF_E_NOTIMPL;
    }
}

}  // namespace

int launch_fp32(mf_handle *h, const float *intr, const float *ext, int Q, int E, float *out,
                cudaStream_t st, float *partial, const int *dQ) {
    return launch_fp32_any<false>(h, intr, ext, Q, E, out, st, partial, 0, dQ);
}

int launch_fp32_columns(mf_handle *h, const float *intr, int Q, float *out, cudaStream_t st) {
    return launch_fp32_any<true>(h, intr, nullptr, Q, 0, out, st, nullptr, h->K, nullptr);
}

int launch_combine(const float *partial, int n_pass, int Q, float *out, cudaStream_t st,
                   unsigned long long *bad, const int *dQ) {
    combine_kernel<<<(Q + 255) / 256, 256, 0, st>>>(partial, n_pass, Q, out, bad, dQ);
    MF_CUDA(cudaGetLastError());
    return MF_OK;
}

}  // namespace mf
