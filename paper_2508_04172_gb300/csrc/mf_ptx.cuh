// PTX building blocks shared by the tcgen05 kernels (sm_103a): mbarriers
// with bounded waits, TMA tile loads, tcgen05 MMA / commit / TMEM loads,
// shared-memory matrix descriptors (K-major, 64-byte swizzle), DSMEM copies.
#pragma once

#include "mf_internal.cuh"

namespace mf {

constexpr int kKB = 32;                 // K elements per k-block (16-bit: 64-byte rows)
constexpr int kSwz = kKB * 2;           // swizzle span = row bytes
constexpr int kRowBytes = kKB * 2;      // bytes per A/B row of a k-block
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s bound on every mbarrier wait
constexpr uint32_t kSuspendNs = 20000;          // try_wait suspend-time hint

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
// try_wait with a suspend-time hint: a waiting thread sleeps (up to the hint)
// instead of re-issuing, so waiting warps leave issue slots to working ones.
__device__ __forceinline__ bool mbar_test(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity), "r"(kSuspendNs)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t gtimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait: false if the phase has not completed after kWaitNs
// nanoseconds; then bit 0 of the status word and bit `site` are set, and
// err[1 + site] records (k-block + 1) of the first give-up.
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, unsigned *err, int site = 0,
                                          int kb = 0) {
    if (mbar_test(b, parity)) return true;
    const uint64_t t0 = gtimer_ns();
    for (uint32_t i = 1;; ++i) {
        if (mbar_test(b, parity)) return true;
        if ((i & 7) == 0 && gtimer_ns() - t0 > kWaitNs) break;
    }
    atomicOr(err, 1u | (1u << site));
    atomicCAS(err + 1 + site, 0u, (unsigned)kb + 1u);
    return false;
}
__device__ __forceinline__ void tma_load_2d(void *dst, const void *tmap, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(su32(dst)),
        "l"((uint64_t)tmap), "r"(x), "r"(y), "r"(su32(bar))
        : "memory");
}
// The same tile load delivered to the same shared-memory offset, completing
// as transaction bytes on the same mbarrier offset, in every CTA of `mask`
// (this GPU's own memory; all CTAs of one cluster).
__device__ __forceinline__ void tma_load_2d_mc(void *dst, const void *tmap, int x, int y, uint64_t *bar,
                                               uint16_t mask) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.multicast::cluster"
        " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(su32(dst)),
        "l"((uint64_t)tmap), "r"(x), "r"(y), "r"(su32(bar)), "h"(mask)
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
// Shared-memory matrix descriptor: K-major, rows of kSwz bytes with a
// kSwz-byte swizzle, 8-row groups 8*kSwz bytes apart (SBO), version 1
// (sm_100 family).  Layout codes: 2 = 128-byte swizzle, 4 = 64-byte swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;                 // LBO (unused for swizzled K-major)
    d |= (uint64_t)((8 * kSwz) >> 4) << 32; // SBO
    d |= (uint64_t)1 << 46;                 // descriptor version
    d |= (uint64_t)(kSwz == 128 ? 2 : 4) << 61;
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
__device__ __forceinline__ void mma_commit_mc(uint64_t *bar, uint16_t mask) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
        " [%0], %1;" ::"r"(su32(bar)),
        "h"(mask)
        : "memory");
}
// Shared-memory address of the same location in another CTA of the cluster.
__device__ __forceinline__ uint32_t map_cta(uint32_t addr, int rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
// Bulk copy of `bytes` from this CTA's shared memory into another CTA's
// (cluster address), completing as transaction bytes on that CTA's mbarrier.
__device__ __forceinline__ void bulk_copy_to_cta(uint32_t dst, uint32_t src, uint32_t bytes, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "r"(src), "r"(bytes), "r"(mbar)
        : "memory");
}
// Named barrier 1 over the 256 producer threads that also ANDs a predicate.
__device__ __forceinline__ bool bar_and_256(bool v) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 1, 256, p;\n"
        " selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)v)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
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

template <bool kBias>
struct TmemAcc {
    uint32_t taddr;         // lane quadrant base | column 0 of the accumulator
    const float *scale;     // per-column scale of this pass (FP16 forms), or nullptr
    const float *bias;      // per-column offset added after the scale (kBias)
    __device__ __forceinline__ void load16(int col, float (&f)[16]) const {
        uint32_t r[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
            "%11, %12, %13, %14, %15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
              "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
              "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr + (uint32_t)col));
        // the wait carries the loaded registers so their uses stay after it,
        // while independent global loads may still be hoisted above it
        asm volatile("tcgen05.wait::ld.sync.aligned;"
                     : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                       "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                       "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]));
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            float v = __uint_as_float(r[e]);
            f[e] = scale ? v * __ldg(scale + col + e) : v;
            if (kBias) f[e] += __ldg(bias + col + e);
        }
    }
    __device__ __forceinline__ void load8(int col, float (&f)[8]) const {
        uint32_t r0, r1, r2, r3, r4, r5, r6, r7;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
            : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3), "=r"(r4), "=r"(r5), "=r"(r6), "=r"(r7)
            : "r"(taddr + (uint32_t)col));
        asm volatile("tcgen05.wait::ld.sync.aligned;"
                     : "+r"(r0), "+r"(r1), "+r"(r2), "+r"(r3), "+r"(r4), "+r"(r5), "+r"(r6), "+r"(r7));
        uint32_t r[8] = {r0, r1, r2, r3, r4, r5, r6, r7};
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            float v = __uint_as_float(r[e]);
            f[e] = scale ? v * __ldg(scale + col + e) : v;
            if (kBias) f[e] += __ldg(bias + col + e);
        }
    }
};


}  // namespace mf
