// tcgen05 forms of the fused lnL kernel (BF16 / FP16 inputs, FP32 accumulation
// in tensor memory), sm_103a.
//
// One CTA evaluates one (128-query tile, column pass) work item, the same
// decomposition as the FP32 SIMT kernel:
//   warp 0      : TMA producer -- W tiles (device columns x 32 nodes, K-major,
//                 64-byte swizzle) for the 1-2 weight parts (hi, lo),
//   warp 1      : allocates the TMEM accumulator (128 lanes x pass width FP32)
//                 and one elected thread issues tcgen05.mma (kind::f16):
//                 Phi_hi.W_hi [+ Phi_hi.W_lo [+ Phi_lo.W_hi]] per 16-node step,
//   warps 2..5  : one query row per thread (= its TMEM lane): rotate into the
//                 metric eigenbasis, Gaussian RBF values / tail monomials for
//                 32 nodes per stage in registers (Eq. rbfcoeff), split to
//                 16-bit hi (+ lo), store them swizzled as the MMA A operand;
//                 after the last stage the same threads read their row of the
//                 accumulator (tcgen05.ld) and run the epilogue (SVD
//                 reconstruction at each detector delay, amplitudes, cross
//                 terms: Eqs. SVD, projected_h_fd, logl_complete).
// Stages are double-buffered with mbarriers; every wait is bounded and sets a
// status bit instead of hanging.
#include "mf_epilogue.cuh"

#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <cstring>

namespace mf {
namespace {

constexpr int kKB = 32;                 // nodes per stage (64 bytes of 16-bit values per row)
constexpr int kStages = 2;
constexpr int kThreads = 192;           // 6 warps
constexpr int kRowBytes = kKB * 2;      // 64
constexpr int kATile = kTile * kRowBytes;   // 8 KB per 16-bit A part
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s bound on every mbarrier wait

// ------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t su32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t gtimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait: false (and status bit set) if the phase has not completed
// after kWaitNs nanoseconds.
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, unsigned *err) {
    if (mbar_test(b, parity)) return true;
    const uint64_t t0 = gtimer_ns();
    for (uint32_t i = 1;; ++i) {
        if (mbar_test(b, parity)) return true;
        if ((i & 255) == 0 && gtimer_ns() - t0 > kWaitNs) break;
    }
    atomicOr(err, 1u);
    return false;
}
__device__ __forceinline__ void tma_load_2d(void *dst, const void *tmap, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(su32(dst)),
        "l"((uint64_t)tmap), "r"(x), "r"(y), "r"(su32(bar))
        : "memory");
}
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
// Shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row groups
// 512 bytes apart (SBO), version 1 (sm_100 family).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;                 // LBO (unused for swizzled K-major)
    d |= (uint64_t)(512 >> 4) << 32;        // SBO
    d |= (uint64_t)1 << 46;                 // descriptor version
    d |= (uint64_t)4 << 61;                 // SWIZZLE_64B
    return d;
}
// Instruction descriptor, kind::f16: D = F32, A/B = F16 (0) or BF16 (1),
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t idesc(int fmt, int n) {
    return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(kTile >> 4) << 24);
}
__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     su32(bar))
                 : "memory");
}
__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int AT>
struct Half2;
template <>
struct Half2<0> {   // FP16
    static __device__ __forceinline__ uint32_t pack(float a, float b) {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    }
    static __device__ __forceinline__ float2 unpack(uint32_t u) {
        __half2 h = *reinterpret_cast<__half2 *>(&u);
        return __half22float2(h);
    }
};
template <>
struct Half2<1> {   // BF16
    static __device__ __forceinline__ uint32_t pack(float a, float b) {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    }
    static __device__ __forceinline__ float2 unpack(uint32_t u) {
        __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162 *>(&u);
        return __bfloat1622float2(h);
    }
};

struct TmemAcc {
    uint32_t taddr;         // lane quadrant base | column 0 of the accumulator
    const float *scale;     // per-column scale of this pass (FP16 forms), or nullptr
    __device__ __forceinline__ void load8(int col, float (&f)[8]) const {
        uint32_t r0, r1, r2, r3, r4, r5, r6, r7;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
            : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3), "=r"(r4), "=r"(r5), "=r"(r6), "=r"(r7)
            : "r"(taddr + (uint32_t)col));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        uint32_t r[8] = {r0, r1, r2, r3, r4, r5, r6, r7};
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            float v = __uint_as_float(r[e]);
            f[e] = scale ? v * __ldg(scale + col + e) : v;
        }
    }
};

struct TcArgs {
    const float *intr, *ext;
    int Q, E, N, P, Nk, nbox;
    const float4 *nodes_s;
    const float *colscale;  // [Kdev] (FP16 forms: s_c * 2^-14), nullptr for BF16
    float *out, *partial;
    float phi_log2_scale;   // log2 of the A-operand scale (14 for FP16, 0 for BF16)
};

// A-operand byte offset of (row r, 16-byte chunk c) in a 64-byte-swizzled tile.
__device__ __forceinline__ uint32_t a_off(int r, int c) {
    return (uint32_t)((r >> 3) * 512 + (r & 7) * 64 + ((c ^ ((r >> 1) & 3)) << 4));
}

template <int NM, int AT, int TERMS>
__global__ void __launch_bounds__(kThreads, 2)
tc_kernel(const __grid_constant__ CUtensorMap tm_hi, const __grid_constant__ CUtensorMap tm_lo,
          TcArgs args, RotParams rot, EpiParams epi) {
    constexpr int NA = (TERMS == 3) ? 2 : 1;
    constexpr int NB = (TERMS >= 2) ? 2 : 1;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int nbox = args.nbox;
    const int btile = nbox * kRowBytes;
    uint8_t *sA = smem;                                       // [kStages][NA][8 KB]
    uint8_t *sB = sA + kStages * NA * kATile;                 // [kStages][NB][btile]
    float4 *xs_s = (float4 *)(sB + kStages * NB * btile);   // [128] prescaled query coords
    float4 *xu_s = xs_s + kTile;                              // [128] Delta-e query coords
    uint64_t *bars = (uint64_t *)(xu_s + kTile);
    uint64_t *fullA = bars, *fullB = bars + kStages, *empty = bars + 2 * kStages;
    uint64_t *accb = bars + 3 * kStages;
    uint32_t *tslot = (uint32_t *)(bars + 3 * kStages + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int pass = blockIdx.y;
    const Pass ps = epi.passes[pass];
    const int q0 = blockIdx.x * kTile;
    const int nkb = args.Nk / kKB;
    const uint32_t tcols = 256;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(fullA + s, 128);
            mbar_init(fullB + s, 1);
            mbar_init(empty + s, 1);
        }
        mbar_init(accb, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         su32(tslot)),
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
            // ---------------------------------------------------- TMA producer
            const uint32_t bytes = (uint32_t)(NB * btile);
            int issued = 0;
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % kStages;
                const uint32_t ph = (kb / kStages) & 1;
                if (!mbar_wait(empty + s, ph ^ 1, epi.err)) break;
                mbar_expect_tx(fullB + s, bytes);
                tma_load_2d(sB + (s * NB + 0) * btile, &tm_hi, kb * kKB, ps.col0, fullB + s);
                if (NB == 2) tma_load_2d(sB + (s * NB + 1) * btile, &tm_lo, kb * kKB, ps.col0, fullB + s);
                issued = kb + 1;
            }
            // drain: our copies must have landed before the CTA may exit
            for (int kb = max(0, issued - kStages); kb < issued; ++kb)
                mbar_wait(fullB + kb % kStages, (kb / kStages) & 1, epi.err);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------------------------------------------- MMA issuer
            const uint32_t id = idesc(AT, ps.width);
            bool ok = true;
            for (int kb = 0; kb < nkb && ok; ++kb) {
                const int s = kb % kStages;
                const uint32_t ph = (kb / kStages) & 1;
                ok = mbar_wait(fullA + s, ph, epi.err) && mbar_wait(fullB + s, ph, epi.err);
                if (!ok) break;
                tc_fence_after();
                const uint32_t a0 = su32(sA + (s * NA) * kATile);
                const uint32_t b0 = su32(sB + (s * NB) * btile);
#pragma unroll
                for (int k16 = 0; k16 < kKB / 16; ++k16) {
                    const uint32_t koff = k16 * 32;
                    const uint32_t acc0 = (kb > 0 || k16 > 0) ? 1u : 0u;
                    mma_f16(tmem, sdesc(a0 + koff), sdesc(b0 + koff), id, acc0);
                    if (TERMS >= 2) mma_f16(tmem, sdesc(a0 + koff), sdesc(b0 + btile + koff), id, 1u);
                    if (TERMS == 3) mma_f16(tmem, sdesc(a0 + kATile + koff), sdesc(b0 + koff), id, 1u);
                }
                mma_commit(empty + s);
            }
            mma_commit(accb);
            // the accumulator must be complete before warp 1 frees TMEM
            mbar_wait(accb, 0, epi.err);
        }
    } else {
        // ------------------------------------------ Phi producers / epilogue
        const int quad = warp & 3;                  // TMEM lane quadrant of this warp
        const int r = quad * 32 + lane;             // epilogue: query row == TMEM lane
        const int q = q0 + r;
        const int qc = min(q, args.Q - 1);
        {
            // rotate this row's query into the metric eigenbasis (Sec. II E)
            float4 th = *reinterpret_cast<const float4 *>(args.intr + (size_t)qc * 4);
            float d[4] = {th.x - rot.centre[0], th.y - rot.centre[1], th.z - rot.centre[2],
                          th.w - rot.centre[3]};
            float xu[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                xu[i] = rot.R[4 * i] * d[0] + rot.R[4 * i + 1] * d[1] + rot.R[4 * i + 2] * d[2] +
                        rot.R[4 * i + 3] * d[3];
            xu_s[r] = make_float4(xu[0], xu[1], xu[2], xu[3]);
            xs_s[r] = make_float4(xu[0] * rot.pre, xu[1] * rot.pre, xu[2] * rot.pre, xu[3] * rot.pre);
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");   // producer warps only
        // producer mapping: 8 consecutive nodes (one 16-byte chunk) for 4 rows
        const int pidx = threadIdx.x - 64;
        const int c = pidx & 3, rg = pidx >> 2;
        float2 X[2][4];     // rows (rg, rg+32) and (rg+64, rg+96), per coordinate
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
            float4 a = xs_s[rg + 64 * h2], b = xs_s[rg + 64 * h2 + 32];
            X[h2][0] = make_float2(a.x, b.x);
            X[h2][1] = make_float2(a.y, b.y);
            X[h2][2] = make_float2(a.z, b.z);
            X[h2][3] = make_float2(a.w, b.w);
        }
        const float sc = args.phi_log2_scale;
        const float tsc = exp2f(sc);
        bool ok = true;
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % kStages;
            const uint32_t ph = (kb / kStages) & 1;
            if (!mbar_wait(empty + s, ph ^ 1, epi.err)) { ok = false; break; }
            uint8_t *ahi = sA + (s * NA) * kATile;
            const int n0 = kb * kKB + c * 8;
            float v[4][8];   // [row j][node e], rows rg + 32 j
            if (kb * kKB + kKB <= args.N) {
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const float4 y = __ldg(args.nodes_s + n0 + e);
                    const float2 ny0 = make_float2(-y.x, -y.x), ny1 = make_float2(-y.y, -y.y);
                    const float2 ny2 = make_float2(-y.z, -y.z), ny3 = make_float2(-y.w, -y.w);
#pragma unroll
                    for (int h2 = 0; h2 < 2; ++h2) {
                        float2 d = __fadd2_rn(X[h2][0], ny0);
                        float2 r2 = __fmul2_rn(d, d);
                        d = __fadd2_rn(X[h2][1], ny1);
                        r2 = __ffma2_rn(d, d, r2);
                        d = __fadd2_rn(X[h2][2], ny2);
                        r2 = __ffma2_rn(d, d, r2);
                        d = __fadd2_rn(X[h2][3], ny3);
                        r2 = __ffma2_rn(d, d, r2);
                        v[2 * h2][e] = ex2(sc - r2.x);
                        v[2 * h2 + 1][e] = ex2(sc - r2.y);
                    }
                }
            } else {
                // last block: RBF values, tail monomials 1, x1..x4, zero padding
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const int row = rg + 32 * jj;
                    const float4 xs = xs_s[row], xu = xu_s[row];
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int n = n0 + e;
                        float val;
                        if (n < args.N) {
                            float4 y = __ldg(args.nodes_s + n);
                            float d0 = xs.x - y.x, d1 = xs.y - y.y, d2 = xs.z - y.z, d3 = xs.w - y.w;
                            float r2 = d0 * d0;
                            r2 = fmaf(d1, d1, r2);
                            r2 = fmaf(d2, d2, r2);
                            r2 = fmaf(d3, d3, r2);
                            val = ex2(sc - r2);
                        } else {
                            const int p = n - args.N;
                            val = (p == 0) ? 1.f : (p == 1) ? xu.x : (p == 2) ? xu.y : (p == 3) ? xu.z : xu.w;
                            val = (p < args.P) ? val * tsc : 0.f;
                        }
                        v[jj][e] = val;
                    }
                }
            }
            // 16-bit hi (+ lo) parts, 64-byte swizzled A tile (row = rg + 32 jj)
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                const int row = rg + 32 * jj;
                uint4 hi;
                hi.x = Half2<AT>::pack(v[jj][0], v[jj][1]);
                hi.y = Half2<AT>::pack(v[jj][2], v[jj][3]);
                hi.z = Half2<AT>::pack(v[jj][4], v[jj][5]);
                hi.w = Half2<AT>::pack(v[jj][6], v[jj][7]);
                *reinterpret_cast<uint4 *>(ahi + a_off(row, c)) = hi;
                if (TERMS == 3) {
                    float2 h0 = Half2<AT>::unpack(hi.x), h1 = Half2<AT>::unpack(hi.y);
                    float2 h2 = Half2<AT>::unpack(hi.z), h3 = Half2<AT>::unpack(hi.w);
                    uint4 lo;
                    lo.x = Half2<AT>::pack(v[jj][0] - h0.x, v[jj][1] - h0.y);
                    lo.y = Half2<AT>::pack(v[jj][2] - h1.x, v[jj][3] - h1.y);
                    lo.z = Half2<AT>::pack(v[jj][4] - h2.x, v[jj][5] - h2.y);
                    lo.w = Half2<AT>::pack(v[jj][6] - h3.x, v[jj][7] - h3.y);
                    *reinterpret_cast<uint4 *>(ahi + kATile + a_off(row, c)) = lo;
                }
            }
            fence_async_smem();
            mbar_arrive(fullA + s);
        }
        // -------------------------------------------------------- epilogue
        if (ok) ok = mbar_wait(accb, 0, epi.err);
        ok = __all_sync(0xffffffffu, ok);    // tcgen05.ld below is warp-collective
        tc_fence_after();
        float l = __int_as_float(0x7fc00000);
        if (ok) {
            QueryExt x = load_ext(epi, args.ext, args.E, qc);
            TmemAcc acc{tmem + ((uint32_t)(quad * 32) << 16),
                        args.colscale ? args.colscale + ps.col0 : nullptr};
            bool bad = false;
            l = pass_lnl<NM>(epi, ps, x, acc, bad);
            if (bad) l = __int_as_float(0x7fc00000);
        }
        if (q < args.Q) {
            if (epi.n_pass == 1) {
                args.out[q] = l;
                if (l != l) atomicAdd(epi.bad, 1ull);
            } else {
                args.partial[(size_t)pass * args.Q + q] = l;
            }
        }
        tc_fence_before();
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols)
                     : "memory");
    }
}

// ----------------------------------------------------------- host side
__global__ void col_absmax(const double *__restrict__ W64, int rows, int K, double *__restrict__ m) {
    int u = blockIdx.x;
    double best = 0.0;
    for (int n = threadIdx.x; n < rows; n += blockDim.x) best = fmax(best, fabs(W64[(size_t)n * K + u]));
    __shared__ double red[256];
    red[threadIdx.x] = best;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) m[u] = red[0];
}

// W_hi/W_lo [Kdev][Nk] (K-major per device column), 16-bit, with per-column
// power-of-two scale s_c (FP16 forms) so that max |W/s_c| lies in (2^14, 2^15].
template <int AT>
__global__ void convert_tc(const double *__restrict__ W64, int rows, int K,
                           const int *__restrict__ user_of_dev, int Kdev, int Nk,
                           const double *__restrict__ cmax, uint16_t *__restrict__ whi,
                           uint16_t *__restrict__ wlo, float *__restrict__ colscale) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    int c = blockIdx.y;
    if (n >= Nk) return;
    int u = user_of_dev[c];
    double s = 1.0;
    if (AT == 0 && u >= 0 && cmax[u] > 0) s = ldexp(1.0, (int)ceil(log2(cmax[u])) - 15);
    double v = (u >= 0 && n < rows) ? W64[(size_t)n * K + u] / s : 0.0;
    float vf = (float)v;
    uint16_t h, l;
    if (AT == 0) {
        __half hh = __float2half_rn(vf);
        __half ll = __float2half_rn((float)(v - (double)__half2float(hh)));
        h = *reinterpret_cast<uint16_t *>(&hh);
        l = *reinterpret_cast<uint16_t *>(&ll);
    } else {
        __nv_bfloat16 hh = __float2bfloat16_rn(vf);
        __nv_bfloat16 ll = __float2bfloat16_rn((float)(v - (double)__bfloat162float(hh)));
        h = *reinterpret_cast<uint16_t *>(&hh);
        l = *reinterpret_cast<uint16_t *>(&ll);
    }
    whi[(size_t)c * Nk + n] = h;
    wlo[(size_t)c * Nk + n] = l;
    if (n == 0) colscale[c] = (AT == 0) ? (float)(s * ldexp(1.0, -14)) : 1.f;
}

typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int make_tmap(void *out, void *base, int at, int Nk, int Kdev, int nbox) {
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        MF_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                                 cudaEnableDefault, &q));
        if (!p || q != cudaDriverEntryPointSuccess) return MF_E_CUDA;
        fn = (EncodeTiled)p;
    }
    cuuint64_t dims[2] = {(cuuint64_t)Nk, (cuuint64_t)Kdev};
    cuuint64_t strides[1] = {(cuuint64_t)Nk * 2};
    cuuint32_t box[2] = {(cuuint32_t)kKB, (cuuint32_t)nbox};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn((CUtensorMap *)out,
                    at == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                    base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        log_msg("cuTensorMapEncodeTiled failed: %d", (int)r);
        return MF_E_CUDA;
    }
    return MF_OK;
}

int form_type(mf_form f) {   // 0 = FP16, 1 = BF16
    return (f == MF_FORM_BF16 || f == MF_FORM_BF16_WSPLIT || f == MF_FORM_BF16_3TERM) ? 1 : 0;
}
int form_terms(mf_form f) {
    switch (f) {
        case MF_FORM_BF16: case MF_FORM_FP16: return 1;
        case MF_FORM_BF16_WSPLIT: case MF_FORM_FP16_WSPLIT: return 2;
        default: return 3;
    }
}

template <int NM, int AT, int TERMS>
int launch_nm(mf_handle *h, const TcArgs &a, cudaStream_t st) {
    constexpr int NA = (TERMS == 3) ? 2 : 1;
    constexpr int NB = (TERMS >= 2) ? 2 : 1;
    size_t bytes = 1024 + (size_t)kStages * NA * kATile + (size_t)kStages * NB * h->nbox * kRowBytes +
                   2 * kTile * sizeof(float4) + (3 * kStages + 2) * 8;
    bytes = std::max(bytes, (size_t)80 * 1024);   // at most 2 CTAs (2 x 256 TMEM columns) per SM
    auto kern = tc_kernel<NM, AT, TERMS>;
    MF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    dim3 grid((a.Q + kTile - 1) / kTile, (unsigned)h->passes.size());
    CUtensorMap thi, tlo;
    memcpy(&thi, h->tmap_hi, sizeof(thi));
    memcpy(&tlo, h->tmap_lo, sizeof(tlo));
    kern<<<grid, kThreads, bytes, st>>>(thi, tlo, a, make_rot(h), make_epi(h));
    MF_CUDA(cudaGetLastError());
    return MF_OK;
}

template <int NM, int AT>
int launch_terms(mf_handle *h, const TcArgs &a, cudaStream_t st) {
    switch (form_terms(h->form)) {
        case 1: return launch_nm<NM, AT, 1>(h, a, st);
        case 2: return launch_nm<NM, AT, 2>(h, a, st);
        default: return launch_nm<NM, AT, 3>(h, a, st);
    }
}

template <int NM>
int launch_type(mf_handle *h, const TcArgs &a, cudaStream_t st) {
    return form_type(h->form) == 0 ? launch_terms<NM, 0>(h, a, st) : launch_terms<NM, 1>(h, a, st);
}

}  // namespace

int convert_tc_weights(mf_handle *h, mf_form f) {
    const int at = form_type(f);
    h->Nk = (h->N + h->P + 63) / 64 * 64;
    int nbox = 0;
    for (auto &p : h->passes) nbox = std::max(nbox, p.width);
    if (nbox > 256) return MF_E_NOTIMPL;
    h->nbox = nbox;
    double *cmax = nullptr;
    MF_CUDA(cudaMalloc((void **)&cmax, sizeof(double) * h->K));
    col_absmax<<<h->K, 256>>>(h->d_W64, h->N + h->P, h->K, cmax);
    size_t n = (size_t)h->Kdev * h->Nk;
    cudaError_t e1 = cudaMalloc(&h->d_Whi, n * 2);
    cudaError_t e2 = cudaMalloc(&h->d_Wlo, n * 2);
    cudaError_t e3 = cudaMalloc((void **)&h->d_colscale, sizeof(float) * h->Kdev);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
        cudaFree(cmax);
        return MF_E_NOMEM;
    }
    dim3 grid((h->Nk + 255) / 256, h->Kdev);
    if (at == 0)
        convert_tc<0><<<grid, 256>>>(h->d_W64, h->N + h->P, h->K, h->d_user_of_dev, h->Kdev, h->Nk, cmax,
                                     (uint16_t *)h->d_Whi, (uint16_t *)h->d_Wlo, h->d_colscale);
    else
        convert_tc<1><<<grid, 256>>>(h->d_W64, h->N + h->P, h->K, h->d_user_of_dev, h->Kdev, h->Nk, cmax,
                                     (uint16_t *)h->d_Whi, (uint16_t *)h->d_Wlo, h->d_colscale);
    cudaError_t e = cudaGetLastError();
    cudaDeviceSynchronize();
    cudaFree(cmax);
    MF_CUDA(e);
    int rc = make_tmap(h->tmap_hi, h->d_Whi, at, h->Nk, h->Kdev, nbox);
    if (rc) return rc;
    return make_tmap(h->tmap_lo, h->d_Wlo, at, h->Nk, h->Kdev, nbox);
}

int launch_tc(mf_handle *h, const float *intr, const float *ext, int Q, int E, float *out,
              cudaStream_t st, float *partial) {
    if (!h->d_Whi) return MF_E_STATE;
    TcArgs a;
    a.intr = intr;
    a.ext = ext;
    a.Q = Q;
    a.E = E;
    a.N = h->N;
    a.P = h->P;
    a.Nk = h->Nk;
    a.nbox = h->nbox;
    a.nodes_s = h->d_nodes_s;
    a.colscale = form_type(h->form) == 0 ? h->d_colscale : nullptr;
    a.out = out;
    a.partial = partial;
    a.phi_log2_scale = form_type(h->form) == 0 ? 14.f : 0.f;
    switch (h->n_modes) {
        case 1: return launch_type<1>(h, a, st);
        case 2: return launch_type<2>(h, a, st);
        case 3: return launch_type<3>(h, a, st);
        case 4: return launch_type<4>(h, a, st);
        case 5: return launch_type<5>(h, a, st);
        default: return MF_E_NOTIMPL;
    }
}

}  // namespace mf
