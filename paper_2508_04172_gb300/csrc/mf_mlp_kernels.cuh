// Kernels of the surrogate network (a fully connected SiLU network, BF16
// operands with FP32 accumulation): a tcgen05 GEMM C = A B^T with fused
// epilogues, the first layer (4 inputs: plain FMAs), its weight gradient,
// and the Adam update.  Included by mf_mlp.cu only (network training and
// inference, lnL through the surrogate).
#pragma once

#include "mf_epilogue.cuh"
#include "mf_ptx.cuh"

namespace mf {
namespace {   // kernels and launch plans are private to the including unit

constexpr int kGemmStages = 4;
constexpr int kGemmThreads = 192;          // warp 0 TMA, warp 1 MMA, warps 2..5 epilogue
constexpr int kGemmThreadsLnl = 320;       // lnL epilogue: warps 2..9, two per TMEM lane quadrant
constexpr int kGemmATile = kTile * kRowBytes;
constexpr int kMlpMaxLayers = 8;
constexpr int kMlpMaxIn = 16;

enum : int {
    EPI_SILU = 0,    // h = SiLU(acc + bias) -> bf16 [M][N] (+ transposed, + z FP32)
    EPI_MSE = 1,     // y = acc + bias; dY = gscale (y - t) -> bf16 (+ transposed); loss, column sums
    EPI_DSILU = 2,   // dz = acc * SiLU'(z) -> bf16 (+ transposed, + FP32); column sums
    EPI_F32 = 3,     // C = acc (+ bias) -> FP32 [M][N]
    EPI_LNL = 4      // acc + bias are the interpolated columns of one pass -> lnL (Eq. logl_complete)
};

struct GemmArgs {
    int M, N, K;              // C[M][N] = A[M][K] B[N][K]^T, row-major operands (K contiguous)
    int NT;                   // columns per CTA (B tile rows), multiple of 16, <= 256
    const float *bias;        // [N] or nullptr
    __nv_bfloat16 *out_bf;    // [M][N]
    __nv_bfloat16 *out_t;     // [N][M] or nullptr
    float *out_f;             // [M][N] or nullptr
    const float *aux;         // [M][N]: MSE targets, DSILU pre-activations
    float *colsum;            // [N] accumulated column sums of the result (MSE, DSILU) or nullptr
    float *loss;              // MSE: accumulated sum of squared residuals
    float gscale;             // MSE: 2 / (rows * N) of the loss mean
    unsigned *err;            // device status words
    // EPI_LNL
    const float *ext;
    int E;
    float *lnl_out;           // [M] (one pass)
    float *partial;           // [n_pass][M]
};

// SiLU(z) = z sigmoid(z), sigmoid(z) = 1 / (1 + 2^(-z log2 e)); the fast
// exp2 and division keep ~2^-21 relative accuracy, far below BF16 rounding.
__device__ __forceinline__ float sigmoid_f(float z) { return __fdividef(1.f, 1.f + ex2(-1.4426950408889634f * z)); }
__device__ __forceinline__ float silu_f(float z) { return z * sigmoid_f(z); }
__device__ __forceinline__ float silu_grad_f(float z) {
    const float s = sigmoid_f(z);
    return s * (1.f + z * (1.f - s));
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// tcgen05 GEMM tile: 128 rows x NT columns per CTA, K in blocks of 32 through
// a kGemmStages-deep TMA ring; one thread issues the MMAs (kind::f16, BF16
// inputs, FP32 accumulator in TMEM); four warps read the accumulator rows
// (thread = row) and apply the epilogue.
template <int EPI, int NM>
__global__ void __launch_bounds__(EPI == EPI_LNL ? kGemmThreadsLnl : kGemmThreads)
gemm_kernel(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB,
            const __grid_constant__ GemmArgs g, const __grid_constant__ EpiParams epi) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int NT = g.NT;
    const int stage_bytes = kGemmATile + NT * kRowBytes;
    uint64_t *full = (uint64_t *)(smem + kGemmStages * stage_bytes);
    uint64_t *empty = full + kGemmStages;
    uint64_t *tfull = empty + kGemmStages;
    uint32_t *tslot = (uint32_t *)(tfull + 1);
    float *red = (float *)((uint8_t *)full + 128);            // [128] lnL of the second warp half
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kTile;
    int n0, nw;
    if (EPI == EPI_LNL) {
        n0 = epi.passes[blockIdx.y].col0;
        nw = epi.passes[blockIdx.y].width;
    } else {
        n0 = blockIdx.y * NT;
        nw = NT;
    }
    const int nkb = (g.K + kKB - 1) / kKB;
    uint32_t tcols = 32;
    while (tcols < (uint32_t)NT) tcols <<= 1;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kGemmStages; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        mbar_init(tfull, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                     "r"(tcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        if (lane == 0) {
            int s = 0, issued = 0;
            uint32_t ph = 0;
            for (int kb = 0; kb < nkb; ++kb) {
                if (!mbar_wait(empty + s, ph ^ 1, g.err, 1, kb)) break;
                mbar_expect_tx(full + s, (uint32_t)stage_bytes);
                uint8_t *st = smem + s * stage_bytes;
                tma_load_2d(st, &tA, kb * kKB, m0, full + s);
                tma_load_2d(st + kGemmATile, &tB, kb * kKB, n0, full + s);
                ++issued;
                if (++s == kGemmStages) { s = 0; ph ^= 1; }
            }
            // our last copies must have landed before the CTA may exit
            for (int k = 0; k < kGemmStages && k < issued; ++k) {
                if (--s < 0) { s = kGemmStages - 1; ph ^= 1; }
                mbar_wait(full + s, ph, g.err, 2, 0);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t id = idesc(1, nw);
            int s = 0;
            uint32_t ph = 0;
            for (int kb = 0; kb < nkb; ++kb) {
                if (!mbar_wait(full + s, ph, g.err, 3, kb)) break;
                tc_fence_after();
                const uint32_t base = su32(smem + s * stage_bytes);
                const uint64_t a = sdesc(base), b = sdesc(base + kGemmATile);
#pragma unroll
                for (int k16 = 0; k16 < kKB / 16; ++k16)
                    mma_f16(tmem, a + (uint64_t)(k16 * 2), b + (uint64_t)(k16 * 2), id,
                            (kb > 0 || k16 > 0) ? 1u : 0u);
                mma_commit(empty + s);
                if (++s == kGemmStages) { s = 0; ph ^= 1; }
            }
            mma_commit(tfull);
        }
    } else {
        const int quad = warp & 3;
        const int row = quad * 32 + lane;
        const int m = m0 + row;
        const bool mv = m < g.M;
        bool ok = mbar_wait(tfull, 0, g.err, 7, 0);
        ok = __all_sync(0xffffffffu, ok);
        tc_fence_after();
        const uint32_t tb = tmem + ((uint32_t)(quad * 32) << 16);
        if (EPI == EPI_LNL) {
            // two warps per lane quadrant: each takes one contiguous half of the
            // pass's column groups (lnL is a sum over groups), the halves meet
            // in shared memory
            const int half = (warp - 2) >> 2;
            Pass ps = epi.passes[blockIdx.y];
            const int n_first = (ps.ng + 1) / 2;
            if (half == 0) ps.ng = n_first;
            else { ps.g0 += n_first; ps.ng -= n_first; }
            float l = 0.f;
            if (ok && ps.ng > 0) {
                const QueryExt x = load_ext(epi, g.ext, g.E, min(m, g.M - 1));
                TmemAcc<true> acc{tb, nullptr, g.bias + epi.passes[blockIdx.y].col0};
                bool bad = false;
                l = pass_lnl<NM>(epi, ps, x, acc, bad);
                if (bad) l = __int_as_float(0x7fc00000);
            }
            if (!ok) l = __int_as_float(0x7fc00000);
            if (half == 1) red[row] = l;
            asm volatile("bar.sync 1, 256;" ::: "memory");
            if (half == 0 && mv) {
                l += red[row];
                if (gridDim.y == 1) {
                    g.lnl_out[m] = l;
                    if (l != l) atomicAdd(epi.bad, 1ull);
                } else {
                    g.partial[(size_t)blockIdx.y * g.M + m] = l;
                }
            }
        } else if (ok) {
            float lsum = 0.f;
            for (int c = 0; c < NT && n0 + c < g.N; c += 16) {
                float v[16];
                TmemAcc<false>{tb, nullptr, nullptr}.load16(c, v);
                const int n = n0 + c;
                const bool full16 = mv && n + 16 <= g.N;
                float in[16];     // bias (SILU, MSE, F32) or aux
                if (EPI == EPI_MSE || EPI == EPI_DSILU) {
                    if (full16) {
                        const float4 *ap = reinterpret_cast<const float4 *>(g.aux + (size_t)m * g.N + n);
#pragma unroll
                        for (int q4 = 0; q4 < 4; ++q4) {
                            const float4 t4 = ap[q4];
                            in[4 * q4] = t4.x; in[4 * q4 + 1] = t4.y; in[4 * q4 + 2] = t4.z; in[4 * q4 + 3] = t4.w;
                        }
                    } else {
#pragma unroll
                        for (int e = 0; e < 16; ++e)
                            in[e] = (mv && n + e < g.N) ? g.aux[(size_t)m * g.N + n + e] : 0.f;
                    }
                }
                float bias16[16];
                if (g.bias && n + 16 <= g.N && ((reinterpret_cast<uintptr_t>(g.bias + n) & 15) == 0)) {
                    const float4 *bp = reinterpret_cast<const float4 *>(g.bias + n);
#pragma unroll
                    for (int q4 = 0; q4 < 4; ++q4) {
                        const float4 b4 = __ldg(bp + q4);
                        bias16[4 * q4] = b4.x; bias16[4 * q4 + 1] = b4.y;
                        bias16[4 * q4 + 2] = b4.z; bias16[4 * q4 + 3] = b4.w;
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < 16; ++e) bias16[e] = (g.bias && n + e < g.N) ? __ldg(g.bias + n + e) : 0.f;
                }
                float r[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const bool valid = mv && n + e < g.N;
                    const float bs = bias16[e];
                    float o;
                    if (EPI == EPI_SILU) {
                        o = silu_f(v[e] + bs);
                        if (g.out_f && valid) g.out_f[(size_t)m * g.N + n + e] = v[e] + bs;
                    } else if (EPI == EPI_MSE) {
                        const float res = valid ? v[e] + bs - in[e] : 0.f;
                        lsum = fmaf(res, res, lsum);
                        o = g.gscale * res;
                    } else if (EPI == EPI_DSILU) {
                        o = valid ? v[e] * silu_grad_f(in[e]) : 0.f;
                    } else {
                        o = v[e] + bs;
                    }
                    r[e] = o;
                }
                if (EPI == EPI_F32 || (EPI == EPI_DSILU && g.out_f)) {
                    float *op = g.out_f + (size_t)m * g.N + n;
                    if (full16) {
#pragma unroll
                        for (int q4 = 0; q4 < 4; ++q4)
                            reinterpret_cast<float4 *>(op)[q4] =
                                make_float4(r[4 * q4], r[4 * q4 + 1], r[4 * q4 + 2], r[4 * q4 + 3]);
                    } else {
#pragma unroll
                        for (int e = 0; e < 16; ++e)
                            if (mv && n + e < g.N) op[e] = r[e];
                    }
                }
                if (EPI != EPI_F32 && g.out_bf) {
                    __nv_bfloat16 *op = g.out_bf + (size_t)m * g.N + n;
                    if (full16) {
                        uint4 p0, p1;
                        p0.x = Half2<1>::pack(r[0], r[1]);   p0.y = Half2<1>::pack(r[2], r[3]);
                        p0.z = Half2<1>::pack(r[4], r[5]);   p0.w = Half2<1>::pack(r[6], r[7]);
                        p1.x = Half2<1>::pack(r[8], r[9]);   p1.y = Half2<1>::pack(r[10], r[11]);
                        p1.z = Half2<1>::pack(r[12], r[13]); p1.w = Half2<1>::pack(r[14], r[15]);
                        reinterpret_cast<uint4 *>(op)[0] = p0;
                        reinterpret_cast<uint4 *>(op)[1] = p1;
                    } else {
#pragma unroll
                        for (int e = 0; e < 16; ++e)
                            if (mv && n + e < g.N) op[e] = __float2bfloat16_rn(r[e]);
                    }
                }
                if (EPI != EPI_F32 && g.out_t && mv) {
#pragma unroll
                    for (int e = 0; e < 16; ++e)
                        if (n + e < g.N) g.out_t[(size_t)(n + e) * g.M + m] = __float2bfloat16_rn(r[e]);
                }
                if ((EPI == EPI_MSE || EPI == EPI_DSILU) && g.colsum) {
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const float s = warp_sum(r[e]);   // rows beyond M contribute 0
                        if (lane == 0 && n + e < g.N) atomicAdd(g.colsum + n + e, s);
                    }
                }
            }
            if (EPI == EPI_MSE) {
                lsum = warp_sum(lsum);
                if (lane == 0) atomicAdd(g.loss, lsum);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
    }
}

inline size_t gemm_smem_bytes(int NT) {
    // barriers and the TMEM slot in the first 128 bytes after the ring, then
    // the 128-float exchange of the split lnL epilogue
    static_assert((2 * kGemmStages + 1) * 8 + 4 <= 128, "barriers overflow their 128 bytes");
    return 1024 + (size_t)kGemmStages * (kGemmATile + NT * kRowBytes) + 128 + 128 * sizeof(float);
}

// One GEMM launch, prepared once: operand tensor maps and arguments.
struct GemmPlan {
    CUtensorMap ta, tb;
    GemmArgs g;
    int epi;
    int grid_y;
};

// First layer: z1 = W1 x + b1 (few inputs, plain FMAs), h1 = SiLU(z1).
// Writes H1 bf16 [B][H], optionally H1t bf16 [H][B] and Z1 FP32 [B][H].
__global__ void layer1_kernel(const float *__restrict__ X, int B, int n_in, const float *__restrict__ W1,
                              const float *__restrict__ b1, int H, __nv_bfloat16 *__restrict__ H1,
                              __nv_bfloat16 *__restrict__ H1t, float *__restrict__ Z1) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)B * H) return;
    const int b = (int)(idx / H), o = (int)(idx % H);
    float z = b1[o];
    for (int i = 0; i < n_in; ++i) z = fmaf(W1[o * n_in + i], X[(size_t)b * n_in + i], z);
    const __nv_bfloat16 h = __float2bfloat16_rn(silu_f(z));
    H1[idx] = h;
    if (H1t) H1t[(size_t)o * B + b] = h;
    if (Z1) Z1[idx] = z;
}

// Weight gradient of the first layer: gW1[o][i] = sum_b dZ1[b][o] x[b][i].
__global__ void layer1_wgrad_kernel(const float *__restrict__ dZ1, const float *__restrict__ X, int B,
                                    int n_in, int H, float *__restrict__ gW1) {
    const int o = blockIdx.x;
    float acc[kMlpMaxIn];
#pragma unroll
    for (int i = 0; i < kMlpMaxIn; ++i) acc[i] = 0.f;
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        const float d = dZ1[(size_t)b * H + o];
#pragma unroll
        for (int i = 0; i < kMlpMaxIn; ++i)
            if (i < n_in) acc[i] = fmaf(d, X[(size_t)b * n_in + i], acc[i]);
    }
    __shared__ float red[kMlpMaxIn][8];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < kMlpMaxIn; ++i) {
        const float s = warp_sum(acc[i]);
        if (l == 0) red[i][w] = s;
    }
    __syncthreads();
    if ((int)threadIdx.x < n_in) {
        float s = 0.f;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[threadIdx.x][k];
        gW1[o * n_in + threadIdx.x] = s;
    }
}

// Flat parameter layout: per layer W [out][in] row-major then b [out].
struct LayerTab {
    int n_layers;
    int off[kMlpMaxLayers + 1];
    int in[kMlpMaxLayers], out[kMlpMaxLayers];
    __nv_bfloat16 *W[kMlpMaxLayers];    // [out][in] (nullptr: layer kept in FP32 only)
    __nv_bfloat16 *Wt[kMlpMaxLayers];   // [in][out]
};

// Device-side training state: the step counter drives the learning-rate
// schedule, the minibatch choice and Adam's bias correction, so a whole
// training step can be replayed from a CUDA graph.
struct TrainState {
    int step, total;
    float lr_max, lr_min;
    float beta1, beta2, eps;
    float loss_acc;           // sum of squared residuals of the current step
    float last_loss;          // mean squared residual of the last completed step
    int rows;                 // minibatch rows
    int n_out;
    unsigned long long seed;
};

__device__ __forceinline__ void write_copies(const LayerTab &tab, int idx, float p) {
    int l = 0;
    while (l + 1 < tab.n_layers && idx >= tab.off[l + 1]) ++l;
    const int local = idx - tab.off[l];
    const int nw = tab.in[l] * tab.out[l];
    if (local < nw && tab.W[l]) {
        const int o = local / tab.in[l], i = local % tab.in[l];
        const __nv_bfloat16 h = __float2bfloat16_rn(p);
        tab.W[l][local] = h;
        tab.Wt[l][(size_t)i * tab.out[l] + o] = h;
    }
}

// Adam (Kingma & Ba, Algorithm 1) with bias correction and a cosine
// learning-rate schedule from lr_max to lr_min over `total` steps; zeroes
// the gradient for the next step's accumulation and refreshes the BF16
// copies.  With update = 0 it only refreshes the copies.
__global__ void adam_kernel(float *__restrict__ p, float *__restrict__ grad, float *__restrict__ m1,
                            float *__restrict__ m2, int n, const LayerTab tab, const TrainState *st,
                            int update) {
    float lr = 0.f, c1 = 1.f, c2 = 1.f, b1 = 0.f, b2 = 0.f, eps = 0.f;
    if (update) {
        const int s = st->step;
        const float frac = st->total > 1 ? fminf(1.f, (float)s / (float)(st->total - 1)) : 1.f;
        lr = st->lr_min + 0.5f * (st->lr_max - st->lr_min) * (1.f + cospif(frac));
        b1 = st->beta1;
        b2 = st->beta2;
        eps = st->eps;
        c1 = 1.f - powf(b1, (float)(s + 1));
        c2 = 1.f - powf(b2, (float)(s + 1));
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float w = p[i];
        if (update) {
            const float gi = grad[i];
            const float a = fmaf(b1, m1[i], (1.f - b1) * gi);
            const float v = fmaf(b2, m2[i], (1.f - b2) * gi * gi);
            m1[i] = a;
            m2[i] = v;
            w -= lr * (a / c1) / (sqrtf(v / c2) + eps);
            p[i] = w;
            grad[i] = 0.f;
        }
        write_copies(tab, i, w);
    }
}

// Close a training step: record its loss, advance the step counter.
__global__ void step_end_kernel(TrainState *st) {
    st->last_loss = st->loss_acc / ((float)st->rows * (float)st->n_out);
    st->loss_acc = 0.f;
    st->step += 1;
}

// Minibatch of `rows` rows of the training set: row j = (a + j c) mod n with
// a drawn from the step counter and c a fixed stride coprime to n.
__global__ void gather_kernel(const float *__restrict__ X, const float *__restrict__ T, int n, int n_in,
                              int n_out, const TrainState *st, long long stride, float *__restrict__ Xb,
                              float *__restrict__ Tb) {
    const int rows = st->rows;
    unsigned long long h = st->seed ^ (0x9E3779B97F4A7C15ull * (unsigned long long)(st->step + 1));
    h ^= h >> 31;
    h *= 0xBF58476D1CE4E5B9ull;
    h ^= h >> 29;
    const long long a = (long long)(h % (unsigned long long)n);
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < (long long)rows * (n_in + n_out);
         idx += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(idx / (n_in + n_out)), c = (int)(idx % (n_in + n_out));
        const long long r = (a + (long long)j * stride) % n;
        if (c < n_in) Xb[(size_t)j * n_in + c] = X[(size_t)r * n_in + c];
        else Tb[(size_t)j * n_out + (c - n_in)] = T[(size_t)r * n_out + (c - n_in)];
    }
}

}  // namespace
}  // namespace mf
