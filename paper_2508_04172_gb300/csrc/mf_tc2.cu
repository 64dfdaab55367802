// tcgen05 forms, second design: the RBF tile Phi lives in tensor memory.
//
// Each CTA owns one column pass of a query tile (work item = (tile, pass)),
// so no Phi is shared between CTAs; instead the producer warps write the
// 16-bit hi (+lo) parts of Phi straight from registers into a TMEM ring
// (tcgen05.st) and the MMAs read the A operand from TMEM.  Shared memory then
// carries only the TMA-staged weight tiles (the B operand), which removes the
// Phi stores, the DSMEM copies and the repeated A-operand reads of the
// cluster design; the price is that every pass recomputes Phi.
//
// TMEM (512 columns): accumulators at columns [0, kAcc2) and [kAcc2, 2 kAcc2)
// (kAcc2 = 192, so passes are at most 192 columns wide), A ring in the rest:
// per stage and part 16 columns = 128 rows x 32 nodes of 16-bit values, two
// per 32-bit column, K-major (node j of a 16-node MMA step in column j/2).
//
//   warp 0        TMA: W tiles (pass columns x 32 nodes, hi / lo) -> smem ring
//   warp 1        TMEM allocation; one thread issues tcgen05.mma kind::f16
//                 with A in TMEM and B in shared memory
//   warps 2..9    Phi producers: warp w serves TMEM lane quadrant w % 4 and
//                 nodes [16 h, 16 h + 16) of each 32-node block, h = (w-2)/4;
//                 thread = query row (Eq. rbfcoeff: Gaussian values, tail)
//
// Measured on GB300 (C1, 3 passes): slower than the cluster design (0.445 vs
// 0.409 ms for bf16 3-term: recomputing Phi per pass with one row per thread
// costs more issue and load latency than the shared-memory traffic it saves);
// faster for single-pass layouts (C0: 0.019 vs 0.023 ms), where no Phi is
// recomputed and no cluster is needed.  The library picks it for those.
//   warps 10..13  epilogue, as in the cluster design (Eqs. SVD,
//                 projected_h_fd, logl_complete)
#include "mf_epilogue.cuh"
#include "mf_ptx.cuh"

#include <algorithm>
#include <cstring>

namespace mf {
namespace {

constexpr int kAcc2 = 192;                       // columns per accumulator (widest pass)
constexpr int kARing0 = 2 * kAcc2;               // first TMEM column of the A ring
constexpr int kACols = 16;                       // TMEM columns per stage and part (32 nodes)
constexpr int kMaxStages2 = 6;
constexpr int kThreads2 = 32 * (2 + 8 + 4);      // 448

__device__ __forceinline__ void mma_f16_tmem_a(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t id,
                                               uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
        "r"(a_tmem), "l"(b), "r"(id), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
        : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

struct Tc2Call {
    const float *intr, *ext;
    float *out, *partial;
    int Q, E;
    int n_tiles, n_pass, n_items;
    int n_ctas;            // persistent CTAs (each loops over items)
    int sb;                // W ring depth
    int sa;                // A ring depth (TMEM stages)
    int nbox;              // W tile rows (widest pass)
    unsigned *err;
    float *cols;           // columns-only launch: out [Q][K] (node_values order)
    const int *umap;       // columns-only launch: device column -> user column
    int K;
};

// COLS = true: columns-only variant (mf_eval_columns), the epilogue writes
// each pass's interpolated columns instead of combining them into lnL.
// Node-block order of tile t: starts at 11 floor(t / 2) mod nkb and wraps
// (the same order as the cluster design, so the two give bitwise equal sums).
__device__ __forceinline__ int tile_rot2(int tile, int nkb, int mul) {
    return (int)(((long long)(tile >> 1) * mul) % nkb);
}

template <int NM, int AT, int TERMS, bool COLS = false>
__global__ void __launch_bounds__(kThreads2, 1)
tc2_kernel(const __grid_constant__ TcEvent ev, const __grid_constant__ Tc2Call c) {
    constexpr int NA = (TERMS == 3) ? 2 : 1;      // A parts in TMEM
    constexpr int NB = (TERMS >= 2) ? 2 : 1;      // W parts in smem
    constexpr float kPhiLog2 = (AT == 0) ? 14.f : 0.f;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int btile = c.nbox * kRowBytes;
    const int SB = c.sb, SA = c.sa;
    uint8_t *sB = smem;                                       // [SB][NB][btile]
    uint64_t *bars = (uint64_t *)(sB + SB * NB * btile);
    uint64_t *fullA = bars, *emptyA = bars + kMaxStages2;
    uint64_t *fullB = emptyA + kMaxStages2, *emptyB = fullB + kMaxStages2;
    uint64_t *tfull = emptyB + kMaxStages2, *tempty = tfull + 2;
    uint64_t *done = tempty + 2;
    uint32_t *tslot = (uint32_t *)(done + 1);                 // barriers + slot fit in 256 bytes
    float4 *sN = (float4 *)((uint8_t *)bars + 256);           // [8 warps][2][16] node blocks
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nkb = ev.nkb;
    unsigned *err = c.err;

    if (threadIdx.x == 0) {
        for (int i = 0; i < SA; ++i) {
            mbar_init(fullA + i, 8);
            mbar_init(emptyA + i, 1);
        }
        for (int i = 0; i < SB; ++i) {
            mbar_init(fullB + i, 1);
            mbar_init(emptyB + i, 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(tfull + i, 1);
            mbar_init(tempty + i, 4);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        if (lane == 0) {
            // ------------------------------------------------------------ TMA
            const uint32_t bytes = (uint32_t)(NB * ev.nbox * kRowBytes);
            int s = 0, issued = 0;
            uint32_t ph = 0;
            bool ok = true;
            for (int it = blockIdx.x; it < c.n_items && ok; it += c.n_ctas) {
                const int col0 = ev.epi.passes[it % c.n_pass].col0;
                const int rot = tile_rot2(it / c.n_pass, nkb, ev.rot_mul);
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!mbar_wait(emptyB + s, ph ^ 1, err, 1, kb)) { ok = false; break; }
                    mbar_expect_tx(fullB + s, bytes);
                    const int kx = (kb + rot < nkb ? kb + rot : kb + rot - nkb) * kKB;
                    tma_load_2d(sB + (s * NB + 0) * btile, &ev.tm_hi, kx, col0, fullB + s);
                    if (NB == 2) tma_load_2d(sB + (s * NB + 1) * btile, &ev.tm_lo, kx, col0, fullB + s);
                    ++issued;
                    if (++s == SB) { s = 0; ph ^= 1; }
                }
            }
            for (int k = 0; k < SB && k < issued; ++k) {
                if (--s < 0) { s = SB - 1; ph ^= 1; }
                mbar_wait(fullB + s, ph, err, 2, 0);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ------------------------------------------------------------ MMA
            int sa = 0, sb = 0;
            uint32_t pa = 0, pb = 0;
            bool ok = true;
            const uint64_t dB0 = sdesc(su32(sB));
            const uint64_t dBstep = (uint64_t)((NB * btile) >> 4), dBlo = (uint64_t)(btile >> 4);
            int i = 0;
            for (int it = blockIdx.x; it < c.n_items && ok; it += c.n_ctas, ++i) {
                const uint32_t id = idesc(AT, ev.epi.passes[it % c.n_pass].width);
                const int acc = i & 1;
                const uint32_t d = tmem + (uint32_t)(acc * kAcc2);
                if (!mbar_wait(tempty + acc, (((uint32_t)i >> 1) & 1) ^ 1, err, 8, i)) break;
                tc_fence_after();
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!mbar_wait(fullA + sa, pa, err, 3, kb)) { ok = false; break; }
                    if (!mbar_wait(fullB + sb, pb, err, 4, kb)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t ahi = tmem + (uint32_t)(kARing0 + sa * NA * kACols);
                    const uint32_t alo = ahi + kACols;
                    const uint64_t b = dB0 + (uint64_t)sb * dBstep;
#pragma unroll
                    for (int k16 = 0; k16 < kKB / 16; ++k16) {
                        const uint32_t ak = (uint32_t)(k16 * 8);       // 16 nodes = 8 columns
                        const uint64_t bk = (uint64_t)(k16 * 2);       // +32 bytes
                        mma_f16_tmem_a(d, ahi + ak, b + bk, id, (kb > 0 || k16 > 0) ? 1u : 0u);
                        if (TERMS >= 2) mma_f16_tmem_a(d, ahi + ak, b + dBlo + bk, id, 1u);
                        if (TERMS == 3) mma_f16_tmem_a(d, alo + ak, b + bk, id, 1u);
                    }
                    mma_commit(emptyB + sb);
                    mma_commit(emptyA + sa);
                    if (++sb == SB) { sb = 0; pb ^= 1; }
                    if (++sa == SA) { sa = 0; pa ^= 1; }
                }
                mma_commit(tfull + acc);
            }
            mma_commit(done);
            mbar_wait(done, 0, err, 5, 0);
        }
    } else if (warp < 10) {
        // --------------------------------------------------- Phi producers
        const int quad = warp & 3;
        const int h = (warp - 2) >> 2;               // node half of each 32-node block
        const int row = quad * 32 + lane;
        const uint32_t tlane = (uint32_t)(quad * 32) << 16;
        const float2 nsc = make_float2(-kPhiLog2, -kPhiLog2);
        const float tsc = exp2f(kPhiLog2);
        float4 *scr = sN + (warp - 2) * 2 * 16;      // this warp's two 16-node buffers
        int sa = 0;
        uint32_t pa = 0;
        int sbuf = 0;
        bool ok = true;
        // lanes 0..15 hold this warp's node of the next block (prefetch FIFO of 1)
        int nit = blockIdx.x, nkb_f = 0;
        float4 ynext = make_float4(0.f, 0.f, 0.f, 0.f);
        auto fetch = [&]() {
            if (nit < c.n_items && lane < 16) {
                const int r = tile_rot2(nit / c.n_pass, nkb, ev.rot_mul);
                const int kd = nkb_f + r < nkb ? nkb_f + r : nkb_f + r - nkb;
                ynext = ldg_keep(ev.nodes_s + kd * kKB + 16 * h + lane);
            }
            if (++nkb_f == nkb) { nkb_f = 0; nit += c.n_ctas; }
        };
        fetch();
        for (int it = blockIdx.x; it < c.n_items && ok; it += c.n_ctas) {
            const int tile = it / c.n_pass;
            float x[4];
            {
                const int q = min(tile * kTile + row, c.Q - 1);
                const float4 th = *reinterpret_cast<const float4 *>(c.intr + (size_t)q * 4);
                const float d0 = th.x - ev.rot.centre[0], d1 = th.y - ev.rot.centre[1];
                const float d2 = th.z - ev.rot.centre[2], d3 = th.w - ev.rot.centre[3];
#pragma unroll
                for (int a = 0; a < 4; ++a)
                    x[a] = ev.rot.R[4 * a] * d0 + ev.rot.R[4 * a + 1] * d1 + ev.rot.R[4 * a + 2] * d2 +
                           ev.rot.R[4 * a + 3] * d3;
            }
            const float pre = ev.rot.pre;
            const int kind = ev.rot.rbf;
            const float2 X0 = make_float2(x[0] * pre, x[0] * pre), X1 = make_float2(x[1] * pre, x[1] * pre);
            const float2 X2 = make_float2(x[2] * pre, x[2] * pre), X3 = make_float2(x[3] * pre, x[3] * pre);
            const int rot = tile_rot2(tile, nkb, ev.rot_mul);
            for (int kb = 0; kb < nkb; ++kb) {
                float4 *buf = scr + sbuf * 16;
                sbuf ^= 1;
                if (lane < 16) buf[lane] = ynext;
                fetch();
                __syncwarp();
                const int n0 = (kb + rot < nkb ? kb + rot : kb + rot - nkb) * kKB + 16 * h;
                float v[16];
                if (n0 + 16 <= ev.N && kind == 0) {
#pragma unroll
                    for (int j = 0; j < 16; j += 2) {
                        const float4 ya = buf[j], yb = buf[j + 1];   // pre-negated, pre-scaled
                        float2 dd = __fadd2_rn(X0, make_float2(ya.x, yb.x));
                        float2 r2 = __ffma2_rn(dd, dd, nsc);
                        dd = __fadd2_rn(X1, make_float2(ya.y, yb.y));
                        r2 = __ffma2_rn(dd, dd, r2);
                        dd = __fadd2_rn(X2, make_float2(ya.z, yb.z));
                        r2 = __ffma2_rn(dd, dd, r2);
                        dd = __fadd2_rn(X3, make_float2(ya.w, yb.w));
                        r2 = __ffma2_rn(dd, dd, r2);
                        v[j] = ex2(-r2.x);
                        v[j + 1] = ex2(-r2.y);
                    }
                } else if (n0 + 16 <= ev.N) {
                    // the other radial kernels, phi(s^2) with s^2 = |pre (x - y)|^2
#pragma unroll
                    for (int j = 0; j < 16; j += 2) {
                        const float4 ya = buf[j], yb = buf[j + 1];
                        float2 dd = __fadd2_rn(X0, make_float2(ya.x, yb.x));
                        float2 r2 = __fmul2_rn(dd, dd);
                        dd = __fadd2_rn(X1, make_float2(ya.y, yb.y));
                        r2 = __ffma2_rn(dd, dd, r2);
                        dd = __fadd2_rn(X2, make_float2(ya.z, yb.z));
                        r2 = __ffma2_rn(dd, dd, r2);
                        dd = __fadd2_rn(X3, make_float2(ya.w, yb.w));
                        r2 = __ffma2_rn(dd, dd, r2);
                        v[j] = rbf_other(kind, r2.x) * tsc;
                        v[j + 1] = rbf_other(kind, r2.y) * tsc;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int n = n0 + j;
                        if (n < ev.N) {
                            const float4 y = buf[j];
                            const float e0 = X0.x + y.x, e1 = X1.x + y.y, e2 = X2.x + y.z, e3 = X3.x + y.w;
                            float r2 = fmaf(e0, e0, kind == 0 ? -kPhiLog2 : 0.f);
                            r2 = fmaf(e1, e1, r2);
                            r2 = fmaf(e2, e2, r2);
                            r2 = fmaf(e3, e3, r2);
                            v[j] = kind == 0 ? ex2(-r2) : rbf_other(kind, r2) * tsc;
                        } else {
                            const int q = n - ev.N;      // tail monomials 1, x1..x4, then padding
                            const float m = (q == 0) ? 1.f : (q == 1) ? x[0] : (q == 2) ? x[1] : (q == 3) ? x[2] : x[3];
                            v[j] = (q < ev.P) ? m * tsc : 0.f;
                        }
                    }
                }
                uint32_t hi[8], lo[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    hi[j] = Half2<AT>::pack(v[2 * j], v[2 * j + 1]);
                    if (TERMS == 3) {
                        const float2 b = Half2<AT>::unpack(hi[j]);
                        lo[j] = Half2<AT>::pack(v[2 * j] - b.x, v[2 * j + 1] - b.y);
                    }
                }
                bool got = true;
                if (lane == 0) got = mbar_wait(emptyA + sa, pa ^ 1, err, 6, kb);
                got = __shfl_sync(0xffffffffu, got, 0);
                if (!got) { ok = false; break; }
                tc_fence_after();
                const uint32_t ta = tmem + tlane + (uint32_t)(kARing0 + sa * NA * kACols + 8 * h);
                tmem_st8(ta, hi);
                if (TERMS == 3) tmem_st8(ta + kACols, lo);
                tmem_wait_st();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(fullA + sa);
                if (++sa == SA) { sa = 0; pa ^= 1; }
            }
        }
    } else {
        // ------------------------------------------------------- epilogue
        const int quad = warp & 3;
        const int r = quad * 32 + lane;
        int i = 0;
        for (int it = blockIdx.x; it < c.n_items; it += c.n_ctas, ++i) {
            const int tile = it / c.n_pass, p = it % c.n_pass;
            const Pass ps = ev.epi.passes[p];
            const int acc = i & 1;
            const int q = tile * kTile + r;
            const int qc = min(q, c.Q - 1);
            QueryExt x{};
            if (!COLS) x = load_ext(ev.epi, c.ext, c.E, qc);
            bool ok = mbar_wait(tfull + acc, ((uint32_t)i >> 1) & 1, err, 7, i);
            ok = __all_sync(0xffffffffu, ok);
            tc_fence_after();
            float l = __int_as_float(0x7fc00000);
            if (ok) {
                TmemAcc<false> tacc{tmem + (uint32_t)(acc * kAcc2) + ((uint32_t)(quad * 32) << 16),
                                    ev.colscale ? ev.colscale + ps.col0 : nullptr, nullptr};
                if (COLS) {
                    pass_columns(ps, tacc, c.umap, q < c.Q ? c.cols + (size_t)q * c.K : nullptr);
                } else {
                    bool bad = false;
                    l = pass_lnl<NM>(ev.epi, ps, x, tacc, bad);
                    if (bad) l = __int_as_float(0x7fc00000);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty + acc);
            if (!COLS && q < c.Q) {
                if (c.n_pass == 1) {
                    c.out[q] = l;
                    if (l != l) atomicAdd(ev.epi.bad, 1ull);
                } else {
                    c.partial[(size_t)p * c.Q + q] = l;
                }
            }
            if (!ok) break;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

size_t smem2(int terms, int nbox, int sb) {
    const int NB = terms >= 2 ? 2 : 1;
    static_assert((4 * kMaxStages2 + 5) * 8 + 4 <= 256, "barriers overflow their 256 bytes");
    return 1024 + (size_t)sb * NB * nbox * kRowBytes + 256 + 8 * 2 * 16 * sizeof(float4);
}

template <int NM, int AT, int TERMS>
void *pick_t() { return (void *)tc2_kernel<NM, AT, TERMS>; }
template <int NM, int AT>
void *pick_a(int terms) { return terms == 1 ? pick_t<NM, AT, 1>() : terms == 2 ? pick_t<NM, AT, 2>() : pick_t<NM, AT, 3>(); }
template <int NM>
void *pick_n(int at, int terms) { return at == 0 ? pick_a<NM, 0>(terms) : pick_a<NM, 1>(terms); }

}  // namespace

int form_terms_of(mf_form f) {
    switch (f) {
        case MF_FORM_BF16: case MF_FORM_FP16: return 1;
        case MF_FORM_BF16_WSPLIT: case MF_FORM_FP16_WSPLIT: return 2;
        default: return 3;
    }
}

// The widest pass this design supports (accumulator width in TMEM).
int tc2_pass_max() { return kAcc2; }

int launch_tc2(mf_handle *h, const float *intr, const float *ext, int Q, int E, float *out, cudaStream_t st,
               float *partial, float *cols) {
    if (!h->d_Whi) return MF_E_STATE;
    if (h->nbox > kAcc2) return MF_E_NOTIMPL;
    const int at = (h->form == MF_FORM_BF16 || h->form == MF_FORM_BF16_WSPLIT || h->form == MF_FORM_BF16_3TERM) ? 1 : 0;
    const int terms = form_terms_of(h->form);
    void *kern = nullptr;
    if (cols) {   // columns only: independent of the mode count
        if (at == 0)
            kern = terms == 1 ? (void *)tc2_kernel<1, 0, 1, true> : terms == 2 ? (void *)tc2_kernel<1, 0, 2, true>
                                                                              : (void *)tc2_kernel<1, 0, 3, true>;
        else
            kern = terms == 1 ? (void *)tc2_kernel<1, 1, 1, true> : terms == 2 ? (void *)tc2_kernel<1, 1, 2, true>
                                                                              : (void *)tc2_kernel<1, 1, 3, true>;
    } else switch (h->n_modes) {
        case 1: kern = pick_n<1>(at, terms); break;
        case 2: kern = pick_n<2>(at, terms); break;
        case 3: kern = pick_n<3>(at, terms); break;
        case 4: kern = pick_n<4>(at, terms); break;
        case 5: kern = pick_n<5>(at, terms); break;
        default: return MF_E_NOTIMPL;
    }
    TcEvent ev;
    int rc = fill_tc_event(h, &ev);
    if (rc) return rc;
    Tc2Call c;
    memset(&c, 0, sizeof(c));
    c.intr = intr;
    c.ext = ext;
    c.out = out;
    c.partial = partial;
    c.Q = Q;
    c.E = E;
    c.n_tiles = (Q + kTile - 1) / kTile;
    c.n_pass = (int)h->passes.size();
    c.n_items = c.n_tiles * c.n_pass;
    c.nbox = h->nbox;
    c.err = h->d_err;
    c.cols = cols;
    c.umap = h->d_user_of_dev;
    c.K = h->K;
    const int NA = terms == 3 ? 2 : 1;
    c.sa = std::min(kMaxStages2, (512 - kARing0) / (NA * kACols));
    c.sb = h->tc_nbs ? h->tc_nbs : kMaxStages2;
    while (smem2(terms, h->nbox, c.sb) > 227 * 1024 && c.sb > 2) --c.sb;
    const size_t bytes = std::max(smem2(terms, h->nbox, c.sb), (size_t)120 * 1024);   // one CTA per SM
    if (bytes > 227 * 1024) return MF_E_NOTIMPL;
    int sms = 0, dev = 0;
    MF_CUDA(cudaGetDevice(&dev));
    MF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    c.n_ctas = std::max(1, std::min(c.n_items, sms));
    MF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    void *args[2] = {(void *)&ev, (void *)&c};
    MF_CUDA(cudaLaunchKernel(kern, dim3((unsigned)c.n_ctas), dim3(kThreads2), args, bytes, st));
    return MF_OK;
}

}  // namespace mf
