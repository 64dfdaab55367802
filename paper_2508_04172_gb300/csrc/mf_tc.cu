// tcgen05 forms of the fused lnL kernel (BF16 / FP16 inputs, FP32 accumulation
// in tensor memory), sm_103a: a persistent, warp-specialised kernel (see
// tc_kernel) with the RBF matrix tile generated in registers as the MMA A
// operand, TMA-staged weight tiles as the B operand, and a double-buffered
// TMEM accumulator so that the per-query epilogue of one work item overlaps
// the contraction of the next.
#include "mf_epilogue.cuh"
#include "mf_ptx.cuh"

#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

namespace mf {
namespace {

constexpr int kMaxStages = 6;           // ring depth bound for the A and W rings
constexpr int kProdWarps = 8;           // Phi producer warps (2 rows x 8 nodes per thread per k-block)
constexpr int kEpiWarps = 4;            // epilogue warps (one accumulator row per thread)
constexpr int kNodeAhead = 4;           // node blocks loaded ahead by each producer warp
constexpr int kMaxCluster = 8;          // passes per tile = CTAs per cluster (portable limit)
constexpr int kSlotsPerProducer = 2;    // A slots owned by each CTA of the cluster (the MMA
                                        // thread's packed per-producer state assumes 2)
constexpr int kThreads = 32 * (2 + kProdWarps + kEpiWarps);   // 448
constexpr int kAccCols = 256;           // TMEM columns per accumulator buffer (2 buffers)
constexpr int kATile = kTile * kRowBytes;   // bytes per 16-bit A part

// Per-call pointers and size of one event.
struct EvIO {
    const float *intr, *ext;
    float *out, *partial;
    int Q;
};

// Per-call arguments of the single-event launch.
struct TcCall {
    const float *intr, *ext;
    float *out, *partial;
    int Q, E;
    int n_tiles;            // query tiles of 128
    int n_items;            // work items: tiles, or pairs of tiles (paired launch)
    int n_clusters;         // clusters launched (each loops over work items)
    int sb;                 // W ring depth
    int nbox_max;           // W ring slot rows
    unsigned *err;          // device status words
    float *cols;            // columns-only launch: out [Q][K] (node_values order)
    const int *umap;        // columns-only launch: device column -> user column
    int K;                  // columns-only launch: row stride of cols
};

// Work source of the single-event kernel: work item = query tile (or pair
// of tiles, `tile` then being the pair index).
struct SingleSrc {
    const TcEvent *ev;
    const TcCall *c;
    __device__ __forceinline__ int n_items() const { return c->n_items; }
    __device__ __forceinline__ void item(int it, int &e, int &tile) const {
        e = 0;
        tile = it;
    }
    __device__ __forceinline__ const TcEvent &event(int) const { return *ev; }
    __device__ __forceinline__ EvIO io(int) const { return EvIO{c->intr, c->ext, c->out, c->partial, c->Q}; }
};

// Work source of the batched kernel: work items are (event, query tile)
// pairs; events are listed in order of decreasing cost per tile and the
// tiles of one event are consecutive.
struct BatchSrc {
    const TcEvent *evs;
    const TcBatchCall *c;
    __device__ __forceinline__ int n_items() const { return c->n_items; }
    __device__ __forceinline__ void item(int it, int &e, int &tile) const {
        int lo = 0, hi = c->n_ev;   // invariant: tprefix[lo] <= it < tprefix[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (c->tprefix[mid] <= it) lo = mid;
            else hi = mid;
        }
        e = c->order[lo];
        tile = it - c->tprefix[lo];
    }
    __device__ __forceinline__ const TcEvent &event(int e) const { return evs[e]; }
    __device__ __forceinline__ EvIO io(int e) const {
        return EvIO{c->intr[e], c->ext[e], c->out[e], c->partial[e], c->Q[e]};
    }
};

// Work item handled by cluster `cid` in round r: snake order (forward in
// even rounds, backward in odd ones), so that with items sorted by
// decreasing cost the clusters' totals stay close.
//
// Node-block order of a tile: the k-loop of tile t starts at block
// rot = 11 floor(t / 2) mod nkb and wraps around, so that the clusters
// (which start together) do not all fetch the same weight tile at the same
// time.  Tiles 2i and 2i+1 share the order (the paired launch gives both the
// same weight tiles); the order depends only on the tile, so a query's sum
// is formed in the same order whatever the launch shape.
__device__ __forceinline__ int tile_rot(int tile, int nkb, int mul) {
    return (int)(((long long)(tile >> 1) * mul) % nkb);
}
__device__ __forceinline__ int rot_kb(int kb, int rot, int nkb) {
    const int k = kb + rot;
    return k >= nkb ? k - nkb : k;
}
__device__ __forceinline__ int item_of(int r, int cid, int nc) {
    return r * nc + ((r & 1) ? nc - 1 - cid : cid);
}

// A-operand byte offset of (row r, 16-byte chunk c) in a swizzled tile: the
// chunk index is XORed with address bits [7, 7 + log2(kSwz/16)).
__device__ __forceinline__ uint32_t a_off(int r, int c) {
    if (kSwz == 128) return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4));
    return (uint32_t)((r >> 3) * 512 + (r & 7) * 64 + ((c ^ ((r >> 1) & 3)) << 4));
}

__device__ __forceinline__ void rotate_row(const RotParams &rot, const float *intr, int q, float (&xu)[4]) {
    float4 th = *reinterpret_cast<const float4 *>(intr + (size_t)q * 4);
    float d[4] = {th.x - rot.centre[0], th.y - rot.centre[1], th.z - rot.centre[2], th.w - rot.centre[3]};
#pragma unroll
    for (int i = 0; i < 4; ++i)
        xu[i] = rot.R[4 * i] * d[0] + rot.R[4 * i + 1] * d[1] + rot.R[4 * i + 2] * d[2] + rot.R[4 * i + 3] * d[3];
}

// Position of a producer warp's node prefetch: the node blocks this CTA makes
// (kb = rank, rank + np, ...) of its cluster's work items, in order.
struct NodeCursor {
    int r;                  // round of the current work item
    int kb, nkb, rot;
    const float4 *nodes;
    bool valid;             // false past the cluster's last work item
};

template <class Src>
__device__ __forceinline__ void cursor_settle(NodeCursor &cu, const Src &src, int cid, int nc, int rank, int pair,
                                              int half) {
    while (cu.valid && cu.kb >= cu.nkb) {
        ++cu.r;
        const int it = item_of(cu.r, cid, nc);
        if (it >= src.n_items()) {
            cu.valid = false;
            break;
        }
        int e, tile;
        src.item(it, e, tile);
        const TcEvent &ev = src.event(e);
        cu.nkb = ev.nkb;
        cu.rot = tile_rot(tile * pair + half, ev.nkb, ev.rot_mul);
        cu.nodes = ev.nodes_s;
        cu.kb = rank;
    }
}

// Persistent, warp-specialised kernel body, one CTA per SM.  A thread-block
// cluster of np CTAs (rank = column pass) walks over work items (a query tile
// of one event); every CTA accumulates its pass's columns for the tile, and
// the RBF tile Phi of node block kb is generated only once, by the CTA of
// rank kb % np, which copies it into the other CTAs' shared memory with bulk
// DSMEM copies.
//   warp 0        TMA: W tiles (pass columns x kKB nodes, K-major, swizzled)
//                 of the 1-2 weight parts into the W ring,
//   warp 1        TMEM allocation (2 accumulators x 256 columns); one thread
//                 issues tcgen05.mma kind::f16 (Phi_hi.W_hi [+ Phi_hi.W_lo
//                 [+ Phi_lo.W_hi]]) per 16-node step into the item's buffer,
//   warps 2..9    Phi producers (this CTA's share of the node blocks): 2-4
//                 rows x 8 nodes per thread; rotation into the metric
//                 eigenbasis, Gaussian RBF values / tail monomials (Eq.
//                 rbfcoeff) in registers, 16-bit hi (+lo) parts stored
//                 swizzled into an A slot owned by this CTA,
//   warps 10..13  epilogue: thread = accumulator row = query; SVD
//                 reconstruction at each detector delay, amplitudes, cross
//                 terms of this pass (Eqs. SVD, projected_h_fd, logl_complete)
//                 while the MMAs of the next item fill the other accumulator.
// Each CTA owns kSlotsPerProducer A slots for the node blocks it makes, so
// every barrier is waited on phase by phase by its waiters.  Every mbarrier
// wait is bounded and sets a status bit instead of hanging.  Every event of
// a batch has exactly np passes.
//
// COLS = true is the columns-only variant (mf_eval_columns): the epilogue
// writes the pass's interpolated columns of each query to cols [Q][K] (user
// column order via umap) instead of combining them into lnL.
//
// PAIR = 2 is the paired launch: a cluster of 2 np CTAs works on two query
// tiles at once (cluster rank = half * np + pass).  The two CTAs of a pass
// read the same weight tiles: each loads half of the tile's rows with a
// multicast TMA into both CTAs' rings, and a ring slot is released when both
// CTAs' MMAs have read it (the emptyB barriers count two commits).  The RBF
// tiles are shared within each half as in the single launch.  Per query the
// arithmetic, and its order, is that of the single launch.
template <int NM, int AT, int TERMS, class Src, bool COLS = false, int PAIR = 1>
__device__ __forceinline__ void tc_body(const Src &src, const int np, const int nbox_max, const int SB,
                                        const int nc, const int E, unsigned *err, float *cols = nullptr,
                                        const int *umap = nullptr, int K = 0) {
    constexpr int NA = (TERMS == 3) ? 2 : 1;
    // How an RBF tile reaches the other CTAs of the cluster: each producer warp
    // copies its own rows as soon as it has written them (single-event, unpaired
    // launches of 4 or more passes: measured 9 % faster on C2), or the eight
    // producer warps meet at a barrier and one thread copies the whole tile
    // (paired launches, where the many small copies slowed C1 / C4 by 15-19 %;
    // 3-pass unpaired launches, 5-8 % slower with them; the batched kernel)
    constexpr bool kWarpCopiesAllowed = PAIR == 1 && std::is_same<Src, SingleSrc>::value;
    const bool warp_copies = kWarpCopiesAllowed && np >= 4;
    constexpr int NB = (TERMS >= 2) ? 2 : 1;
    constexpr int SP = kSlotsPerProducer;
    // FP16 forms carry Phi * 2^14 (W columns are scaled to match)
    constexpr float kPhiLog2 = (AT == 0) ? 14.f : 0.f;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int crank = (int)(blockIdx.x % (unsigned)(PAIR * np));   // == %cluster_ctarank
    const int rank = crank % np;          // column pass of this CTA
    const int half = crank / np;          // tile of the pair
    const int hbase = half * np;          // cluster rank of this half's pass 0
    const uint16_t pairmask = (uint16_t)(PAIR == 2 ? ((1u << rank) | (1u << (np + rank))) : (1u << crank));
    const int cid = (int)(blockIdx.x / (unsigned)(PAIR * np));
    const int btile = nbox_max * kRowBytes;
    const int nslot = np * SP;
    const int n_items = src.n_items();
    uint8_t *sA = smem;                                   // [np][SP][NA][kATile]
    uint8_t *sB = sA + nslot * NA * kATile;               // [SB][NB][btile]
    float4 *sN = (float4 *)(sB + SB * NB * btile);        // [kProdWarps][2][kKB] node blocks
    uint64_t *bars = (uint64_t *)(sN + kProdWarps * 2 * kKB);
    uint64_t *fullA = bars, *emptyA = bars + kMaxCluster * SP;
    uint64_t *fullB = bars + 2 * kMaxCluster * SP, *emptyB = fullB + kMaxStages;
    uint64_t *tfull = emptyB + kMaxStages, *tempty = tfull + 2;
    uint64_t *done = tempty + 2;
    uint32_t *tslot = (uint32_t *)(done + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t tcols = 2 * kAccCols;
    const uint32_t abytes = (uint32_t)(NA * kATile);

    if (threadIdx.x == 0) {
        for (int i = 0; i < nslot; ++i) {
            // own slots: one arrival per producer warp; other CTAs' slots: the
            // arming arrival, completed by their copies' transaction bytes
            mbar_init(fullA + i, warp_copies && i / SP == rank ? (uint32_t)kProdWarps : 1u);
            mbar_init(emptyA + i, (uint32_t)np);
        }
        for (int i = 0; i < SB; ++i) {
            mbar_init(fullB + i, 1);
            mbar_init(emptyB + i, PAIR);   // released by the MMAs of both CTAs of the pass
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(tfull + i, 1);
            mbar_init(tempty + i, kEpiWarps);
        }
        mbar_init(done, 1);
        // slots filled by other CTAs' bulk copies expect their bytes; this CTA
        // arms each for its next use (here the first) -- see the MMA loop
        for (int q = 0; q < np; ++q)
            if (q != rank)
                for (int k = 0; k < SP; ++k) mbar_expect_tx(fullA + q * SP + k, abytes);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                     "r"(tcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncwarp();
    cluster_sync();         // all barriers of the cluster exist before any remote arrive
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        if (lane == 0) {
            // ------------------------------------------------------------ TMA
            int s = 0;              // W ring slot and its phase parity
            uint32_t ph = 0;
            int issued = 0;
            bool ok = true;
            for (int r = 0; ok; ++r) {
                const int it = item_of(r, cid, nc);
                if (it >= n_items) break;
                int e, tile;
                src.item(it, e, tile);
                const TcEvent &ev = src.event(e);
                const int col0 = ev.epi.passes[rank].col0;
                const uint32_t bytes = (uint32_t)(NB * ev.nbox * kRowBytes);   // the whole tile lands here
                const int nkb = ev.nkb;
                const int rot = tile_rot(tile * PAIR + half, nkb, ev.rot_mul);
                const int hrows = ev.nbox / 2;                                  // paired: rows this CTA loads
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!mbar_wait(emptyB + s, ph ^ 1, err, 1, kb)) { ok = false; break; }
                    mbar_expect_tx(fullB + s, bytes);
                    const int kx = rot_kb(kb, rot, nkb) * kKB;
                    if (PAIR == 2) {
                        uint8_t *d0 = sB + (s * NB + 0) * btile + half * hrows * kRowBytes;
                        tma_load_2d_mc(d0, &ev.tm_hi2, kx, col0 + half * hrows, fullB + s, pairmask);
                        if (NB == 2)
                            tma_load_2d_mc(d0 + btile, &ev.tm_lo2, kx, col0 + half * hrows, fullB + s, pairmask);
                    } else {
                        tma_load_2d(sB + (s * NB + 0) * btile, &ev.tm_hi, kx, col0, fullB + s);
                        if (NB == 2) tma_load_2d(sB + (s * NB + 1) * btile, &ev.tm_lo, kx, col0, fullB + s);
                    }
                    ++issued;
                    if (++s == SB) { s = 0; ph ^= 1; }
                }
            }
            // drain: our last copies must have landed before the CTA may exit
            for (int k = 0; k < SB && k < issued; ++k) {
                if (--s < 0) { s = SB - 1; ph ^= 1; }
                mbar_wait(fullB + s, ph, err, 2, 0);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ------------------------------------------------------------ MMA
            // per producer p, bits [2p, 2p+2) = (node blocks consumed from p) mod 4:
            // bit 0 = which of its 2 slots, bit 1 = that slot's phase parity
            uint32_t use = 0;
            int sb = 0;
            uint32_t pb = 0;
            bool ok = true;
            const uint64_t dA0 = sdesc(su32(sA)), dB0 = sdesc(su32(sB));
            const uint64_t dAstep = (uint64_t)(abytes >> 4), dBstep = (uint64_t)((NB * btile) >> 4);
            const uint64_t dAlo = (uint64_t)(kATile >> 4), dBlo = (uint64_t)(btile >> 4);
            for (int r = 0, i = 0; ok; ++r, ++i) {
                const int it = item_of(r, cid, nc);
                if (it >= n_items) break;
                int e, tile;
                src.item(it, e, tile);
                const TcEvent &ev = src.event(e);
                const uint32_t id = idesc(AT, ev.epi.passes[rank].width);
                const int nkb = ev.nkb;
                const int acc = i & 1;
                const uint32_t d = tmem + (uint32_t)(acc * kAccCols);
                if (!mbar_wait(tempty + acc, (((uint32_t)i >> 1) & 1) ^ 1, err, 8, i)) break;
                tc_fence_after();
                int p = 0;          // producer of node block kb = kb % np
                for (int kb = 0; kb < nkb; ++kb) {
                    const uint32_t v = (use >> (2 * p)) & 3u;
                    const int sa = p * SP + (int)(v & 1u);
                    const uint32_t pa = v >> 1;
                    if (!mbar_wait(fullA + sa, pa, err, 3, kb)) { ok = false; break; }
                    if (!mbar_wait(fullB + sb, pb, err, 4, kb)) { ok = false; break; }
                    tc_fence_after();
                    const uint64_t a = dA0 + (uint64_t)sa * dAstep, b = dB0 + (uint64_t)sb * dBstep;
#pragma unroll
                    for (int k16 = 0; k16 < kKB / 16; ++k16) {
                        const uint64_t ko = (uint64_t)(k16 * 2);      // +32 bytes
                        mma_f16(d, a + ko, b + ko, id, (kb > 0 || k16 > 0) ? 1u : 0u);
                        if (TERMS >= 2) mma_f16(d, a + ko, b + dBlo + ko, id, 1u);
                        if (TERMS == 3) mma_f16(d, a + dAlo + ko, b + ko, id, 1u);
                    }
                    if (PAIR == 2) mma_commit_mc(emptyB + sb, pairmask);   // both CTAs' rings
                    else mma_commit(emptyB + sb);
                    mma_commit_mc(emptyA + sa, (uint16_t)(1u << (hbase + p)));   // slot read: tell its producer
                    if (p != rank) mbar_expect_tx(fullA + sa, abytes);   // arm the slot's next fill
                    use = (use & ~(3u << (2 * p))) | (((v + 1u) & 3u) << (2 * p));
                    if (++sb == SB) { sb = 0; pb ^= 1; }
                    if (++p == np) p = 0;
                }
                mma_commit(tfull + acc);
            }
            // every MMA this thread issued must be complete before TMEM is freed
            mma_commit(done);
            mbar_wait(done, 0, err, 5, 0);
        }
    } else if (warp < 2 + kProdWarps) {
        // --------------------------------------------------- Phi producers
        constexpr int CPR = kKB / 8;                // 16-byte chunks per row
        constexpr int RS = 256 / CPR;               // row stride between a thread's rows
        constexpr int RPT = kTile / RS;             // rows per thread (2 or 4)
        static_assert(CPR == 4, "a producer warp's rows must be whole 8-row swizzle atoms");
        const int pt = threadIdx.x - 64;            // 0..255
        const int c = pt % CPR, rg = pt / CPR;      // chunk (8 nodes); rows rg + RS j
        const float2 nsc = make_float2(-kPhiLog2, -kPhiLog2);
        const float tsc = exp2f(kPhiLog2);
        uint32_t aoff[RPT];
#pragma unroll
        for (int j = 0; j < RPT; ++j) aoff[j] = a_off(rg + RS * j, c);
        // scratch slot `lane` holds node nperm of the block: slot e*CPR + c = node c*8 + e
        const int nperm = (lane % CPR) * 8 + lane / CPR;
        int u = 0;              // node blocks produced by this CTA so far
        int sbuf = 0;           // node scratch buffer (double-buffered)
        bool ok = true;
        // this lane's node of the next kNodeAhead node blocks of this CTA (FIFO)
        float4 yq[kNodeAhead];
        NodeCursor cu{-1, 0, 0, 0, nullptr, true};
        cursor_settle(cu, src, cid, nc, rank, PAIR, half);
#pragma unroll
        for (int dd = 0; dd < kNodeAhead; ++dd) {
            yq[dd] = cu.valid ? ldg_keep(cu.nodes + rot_kb(cu.kb, cu.rot, cu.nkb) * kKB + nperm)
                              : make_float4(0.f, 0.f, 0.f, 0.f);
            cu.kb += np;
            cursor_settle(cu, src, cid, nc, rank, PAIR, half);
        }
        for (int r = 0; ok; ++r) {
            const int it = item_of(r, cid, nc);
            if (it >= n_items) break;
            int e, tile;
            src.item(it, e, tile);
            tile = tile * PAIR + half;
            const TcEvent &ev = src.event(e);
            const EvIO io = src.io(e);
            const int N = ev.N, P = ev.P, nkb = ev.nkb;
            const int kind = ev.rot.rbf;
            const int rot = tile_rot(tile, nkb, ev.rot_mul);
            float2 X[RPT / 2][4];   // row pairs (rg + 2h RS, rg + (2h+1) RS), per coordinate
            float4 xu[RPT];
            {
                const RotParams &rot = ev.rot;
                const float pre = rot.pre;
                float a[RPT][4];
#pragma unroll
                for (int j = 0; j < RPT; ++j) {
                    rotate_row(rot, io.intr, min(tile * kTile + rg + RS * j, io.Q - 1), a[j]);
                    xu[j] = make_float4(a[j][0], a[j][1], a[j][2], a[j][3]);
                }
#pragma unroll
                for (int h2 = 0; h2 < RPT / 2; ++h2)
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        X[h2][k] = make_float2(a[2 * h2][k] * pre, a[2 * h2 + 1][k] * pre);
            }
            for (int kb = rank; kb < nkb; kb += np) {
                // node coordinates of this block (pre-negated, pre-scaled): one
                // coalesced 512-byte load per warp issued kNodeAhead blocks ahead,
                // shared through the warp's scratch
                const float4 ycur = yq[0];
#pragma unroll
                for (int dd = 0; dd < kNodeAhead - 1; ++dd) yq[dd] = yq[dd + 1];
                yq[kNodeAhead - 1] = cu.valid ? ldg_keep(cu.nodes + rot_kb(cu.kb, cu.rot, cu.nkb) * kKB + nperm)
                                              : make_float4(0.f, 0.f, 0.f, 0.f);
                cu.kb += np;
                cursor_settle(cu, src, cid, nc, rank, PAIR, half);
                float4 *scr = sN + ((warp - 2) * 2 + sbuf) * kKB;
                sbuf ^= 1;
                scr[lane] = ycur;
                __syncwarp();
                const int kd = rot_kb(kb, rot, nkb);   // node block held by this k-step
                const int n0 = kd * kKB + c * 8;
                float v[RPT][8];   // rows rg + RS j, nodes n0 .. n0+7
                const bool full = (kd * kKB + kKB <= N);
                if (full && kind == 0) {
                    // the common case: 32 nodes, Gaussian kernel
#pragma unroll
                    for (int e8 = 0; e8 < 8; ++e8) {
                        const float4 y = scr[e8 * CPR + c];   // node c*8+e8 (conflict-free broadcast)
                        const float2 ny0 = make_float2(y.x, y.x), ny1 = make_float2(y.y, y.y);
                        const float2 ny2 = make_float2(y.z, y.z), ny3 = make_float2(y.w, y.w);
#pragma unroll
                        for (int h2 = 0; h2 < RPT / 2; ++h2) {
                            // r2 = |x - y|^2 - sc, so Phi * 2^sc = 2^-r2 (two rows at once)
                            float2 dd = __fadd2_rn(X[h2][0], ny0);
                            float2 r2 = __ffma2_rn(dd, dd, nsc);
                            dd = __fadd2_rn(X[h2][1], ny1);
                            r2 = __ffma2_rn(dd, dd, r2);
                            dd = __fadd2_rn(X[h2][2], ny2);
                            r2 = __ffma2_rn(dd, dd, r2);
                            dd = __fadd2_rn(X[h2][3], ny3);
                            r2 = __ffma2_rn(dd, dd, r2);
                            v[2 * h2][e8] = ex2(-r2.x);
                            v[2 * h2 + 1][e8] = ex2(-r2.y);
                        }
                    }
                } else {
                    // the last node block (tail monomials, padding) or another kernel
#pragma unroll
                    for (int e8 = 0; e8 < 8; ++e8) {
                        const int n = n0 + e8;
                        if (full || n < N) {
                            const float4 y = scr[e8 * CPR + c];
                            const float2 ny0 = make_float2(y.x, y.x), ny1 = make_float2(y.y, y.y);
                            const float2 ny2 = make_float2(y.z, y.z), ny3 = make_float2(y.w, y.w);
#pragma unroll
                            for (int h2 = 0; h2 < RPT / 2; ++h2) {
                                // Gaussian: r2 = |x - y|^2 - sc as above; other kernels:
                                // phi(s^2) with s^2 = |pre (x - y)|^2, times 2^sc
                                float2 dd = __fadd2_rn(X[h2][0], ny0);
                                float2 r2 = __ffma2_rn(dd, dd, kind == 0 ? nsc : make_float2(0.f, 0.f));
                                dd = __fadd2_rn(X[h2][1], ny1);
                                r2 = __ffma2_rn(dd, dd, r2);
                                dd = __fadd2_rn(X[h2][2], ny2);
                                r2 = __ffma2_rn(dd, dd, r2);
                                dd = __fadd2_rn(X[h2][3], ny3);
                                r2 = __ffma2_rn(dd, dd, r2);
                                v[2 * h2][e8] = kind == 0 ? ex2(-r2.x) : rbf_other(kind, r2.x) * tsc;
                                v[2 * h2 + 1][e8] = kind == 0 ? ex2(-r2.y) : rbf_other(kind, r2.y) * tsc;
                            }
                        } else {
                            // tail monomials 1, x1..x4 (times 2^sc), then zero padding
                            const int q = n - N;
#pragma unroll
                            for (int j = 0; j < RPT; ++j) {
                                float m = (q == 0) ? 1.f : (q == 1) ? xu[j].x : (q == 2) ? xu[j].y : (q == 3) ? xu[j].z : xu[j].w;
                                v[j][e8] = (q < P) ? m * tsc : 0.f;
                            }
                        }
                    }
                }
                // 16-bit hi (+ lo) parts, computed before waiting for the slot
                uint4 hi[RPT], lo[RPT];
#pragma unroll
                for (int j = 0; j < RPT; ++j) {
                    hi[j].x = Half2<AT>::pack(v[j][0], v[j][1]);
                    hi[j].y = Half2<AT>::pack(v[j][2], v[j][3]);
                    hi[j].z = Half2<AT>::pack(v[j][4], v[j][5]);
                    hi[j].w = Half2<AT>::pack(v[j][6], v[j][7]);
                    if (TERMS == 3) {
                        float2 a = Half2<AT>::unpack(hi[j].x), b = Half2<AT>::unpack(hi[j].y);
                        float2 cc = Half2<AT>::unpack(hi[j].z), dd = Half2<AT>::unpack(hi[j].w);
                        lo[j].x = Half2<AT>::pack(v[j][0] - a.x, v[j][1] - a.y);
                        lo[j].y = Half2<AT>::pack(v[j][2] - b.x, v[j][3] - b.y);
                        lo[j].z = Half2<AT>::pack(v[j][4] - cc.x, v[j][5] - cc.y);
                        lo[j].w = Half2<AT>::pack(v[j][6] - dd.x, v[j][7] - dd.y);
                    }
                }
                const int sa = rank * SP + (u & (SP - 1));
                const uint32_t pa = (uint32_t)((u / SP) & 1);
                bool got = true;
                if (lane == 0) got = mbar_wait(emptyA + sa, pa ^ 1, err, 6, kb);
                got = __shfl_sync(0xffffffffu, got, 0);
                uint8_t *base = sA + sa * abytes;
                if (got) {
#pragma unroll
                    for (int j = 0; j < RPT; ++j) {
                        *reinterpret_cast<uint4 *>(base + aoff[j]) = hi[j];
                        if (TERMS == 3) *reinterpret_cast<uint4 *>(base + kATile + aoff[j]) = lo[j];
                    }
                    fence_async_smem();
                }
                if (!warp_copies) {
                    // all producer warps wrote the slot; and all agree whether to go on
                    if (!bar_and_256(got)) { ok = false; break; }
                    if (pt == 0) {
                        // local slot: plain arrive; other CTAs: bulk copy completing
                        // as transaction bytes on their (pre-armed) fullA barrier
                        const uint32_t src_a = su32(base), fa = su32(fullA + sa);
                        for (int dst = 0; dst < np; ++dst)
                            if (dst != rank)
                                bulk_copy_to_cta(map_cta(src_a, hbase + dst), src_a, abytes,
                                                 map_cta(fa, hbase + dst));
                        mbar_arrive(fullA + sa);
                    }
                    ++u;
                    continue;
                }
                if (!got) { ok = false; break; }   // warp-uniform (broadcast above)
                __syncwarp();
                if (lane == 0) {
                    // this warp's rows are whole 8-row swizzle atoms (rows
                    // 8 w' .. 8 w' + 7 + RS j); each goes to the other CTAs by a
                    // bulk copy completing as transaction bytes on their
                    // (pre-armed) fullA barrier, and this warp arrives on its own
                    const uint32_t fa = su32(fullA + sa);
                    const int wp = warp - 2;
#pragma unroll
                    for (int j = 0; j < RPT; ++j)
#pragma unroll
                        for (int part = 0; part < NA; ++part) {
                            const uint32_t src =
                                su32(base) + (uint32_t)(part * kATile + (wp + (RS >> 3) * j) * 8 * kRowBytes);
                            for (int dst = 0; dst < np; ++dst)
                                if (dst != rank)
                                    bulk_copy_to_cta(map_cta(src, hbase + dst), src, 8 * kRowBytes,
                                                     map_cta(fa, hbase + dst));
                        }
                    mbar_arrive(fullA + sa);
                }
                ++u;
            }
        }
    } else {
        // ------------------------------------------------------- epilogue
        const int quad = warp & 3;                  // TMEM lane quadrant of this warp
        const int row = quad * 32 + lane;           // accumulator row == query in tile
        for (int r = 0, i = 0;; ++r, ++i) {
            const int it = item_of(r, cid, nc);
            if (it >= n_items) break;
            int e, tile;
            src.item(it, e, tile);
            tile = tile * PAIR + half;
            const TcEvent &ev = src.event(e);
            const EvIO io = src.io(e);
            const Pass ps = ev.epi.passes[rank];
            const int acc = i & 1;
            const int q = tile * kTile + row;
            const int qc = min(q, io.Q - 1);
            QueryExt x{};
            if (!COLS) x = load_ext(ev.epi, io.ext, E, qc);
            bool ok = mbar_wait(tfull + acc, ((uint32_t)i >> 1) & 1, err, 7, i);
            ok = __all_sync(0xffffffffu, ok);    // tcgen05.ld below is warp-collective
            tc_fence_after();
            float l = __int_as_float(0x7fc00000);
            if (ok) {
                TmemAcc<false> tacc{tmem + (uint32_t)(acc * kAccCols) + ((uint32_t)(quad * 32) << 16),
                             ev.colscale ? ev.colscale + ps.col0 : nullptr};
                if (COLS) {
                    pass_columns(ps, tacc, umap, q < io.Q ? cols + (size_t)q * K : nullptr);
                } else {
                    bool bad = false;
                    l = pass_lnl<NM>(ev.epi, ps, x, tacc, bad);
                    if (bad) l = __int_as_float(0x7fc00000);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty + acc);
            if (!COLS && q < io.Q) {
                if (np == 1) {
                    io.out[q] = l;
                    if (l != l) atomicAdd(ev.epi.bad, 1ull);
                } else {
                    io.partial[(size_t)rank * io.Q + q] = l;
                }
            }
            if (!ok) break;
        }
    }
    __syncwarp();
    // no CTA may leave while a peer can still copy into it or signal it
    cluster_sync();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
    }
}

template <int NM, int AT, int TERMS, bool COLS = false, int PAIR = 1>
__global__ void __launch_bounds__(kThreads, 1)
tc_kernel(const __grid_constant__ TcEvent ev, const __grid_constant__ TcCall call) {
    SingleSrc src{&ev, &call};
    tc_body<NM, AT, TERMS, SingleSrc, COLS, PAIR>(src, ev.epi.n_pass, call.nbox_max, call.sb, call.n_clusters,
                                                 call.E, call.err, call.cols, call.umap, call.K);
}

template <int NM, int AT, int TERMS>
__global__ void __launch_bounds__(kThreads, 1)
tc_batch_kernel(const TcEvent *__restrict__ evs, const __grid_constant__ TcBatchCall call) {
    BatchSrc src{evs, &call};
    tc_body<NM, AT, TERMS>(src, call.np, call.nbox_max, call.sb, call.n_clusters, call.E, call.err);
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

constexpr size_t kSmemMax = 227 * 1024;

size_t smem_for(int terms, int np, int nbox_max, int sb) {
    const int NA = (terms == 3) ? 2 : 1;
    const int NB = (terms >= 2) ? 2 : 1;
    return (size_t)1024 + (size_t)np * kSlotsPerProducer * NA * kATile + (size_t)sb * NB * nbox_max * kRowBytes +
           (size_t)kProdWarps * 2 * kKB * sizeof(float4) + (2 * kMaxCluster * kSlotsPerProducer + 2 * kMaxStages + 5) * 8 +
           16;
}

// The kernel a (form, mode count) pair runs, single-event or batched.
template <int NM, int AT, int TERMS>
void *pick3(bool batch) {
    return batch ? (void *)tc_batch_kernel<NM, AT, TERMS> : (void *)tc_kernel<NM, AT, TERMS>;
}
template <int NM, int AT>
void *pick2(int terms, bool batch) {
    return terms == 1 ? pick3<NM, AT, 1>(batch) : terms == 2 ? pick3<NM, AT, 2>(batch) : pick3<NM, AT, 3>(batch);
}
template <int NM>
void *pick1(int at, int terms, bool batch) {
    return at == 0 ? pick2<NM, 0>(terms, batch) : pick2<NM, 1>(terms, batch);
}
// Columns-only kernels do not depend on the mode count (no lnL epilogue).
void *pick_cols_kernel(mf_form f) {
    const int at = form_type(f), terms = form_terms(f);
    if (at == 0)
        return terms == 1 ? (void *)tc_kernel<1, 0, 1, true> : terms == 2 ? (void *)tc_kernel<1, 0, 2, true>
                                                                          : (void *)tc_kernel<1, 0, 3, true>;
    return terms == 1 ? (void *)tc_kernel<1, 1, 1, true> : terms == 2 ? (void *)tc_kernel<1, 1, 2, true>
                                                                      : (void *)tc_kernel<1, 1, 3, true>;
}
// Paired launch (3-term forms, lnL kernels only).
template <int NM>
void *pick_pair1(int at) { return at == 0 ? (void *)tc_kernel<NM, 0, 3, false, 2> : (void *)tc_kernel<NM, 1, 3, false, 2>; }
void *pick_pair_kernel(mf_form f, int n_modes) {
    if (form_terms(f) != 3) return nullptr;
    const int at = form_type(f);
    switch (n_modes) {
        case 1: return pick_pair1<1>(at);
        case 2: return pick_pair1<2>(at);
        case 3: return pick_pair1<3>(at);
        case 4: return pick_pair1<4>(at);
        case 5: return pick_pair1<5>(at);
        default: return nullptr;
    }
}
void *pick_kernel(mf_form f, int n_modes, bool batch) {
    const int at = form_type(f), terms = form_terms(f);
    switch (n_modes) {
        case 1: return pick1<1>(at, terms, batch);
        case 2: return pick1<2>(at, terms, batch);
        case 3: return pick1<3>(at, terms, batch);
        case 4: return pick1<4>(at, terms, batch);
        case 5: return pick1<5>(at, terms, batch);
        default: return nullptr;
    }
}

// Launch configuration shared by both kernels: cluster of np CTAs, one CTA
// per SM (it owns all 512 TMEM columns: request > half the SM's shared
// memory), as many clusters as can be resident at once.
int tc_config(void *kern, int np, size_t smem, cudaStream_t st, cudaLaunchConfig_t &cfg,
              cudaLaunchAttribute *attr, int *max_clusters) {
    const size_t bytes = std::max(smem, (size_t)120 * 1024);
    MF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    if (np > 1) MF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 0));
    cfg = cudaLaunchConfig_t{};
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = bytes;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)np;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3((unsigned)np, 1, 1);
    *max_clusters = 0;
    MF_CUDA(cudaOccupancyMaxActiveClusters(max_clusters, kern, &cfg));
    if (*max_clusters < 1) return MF_E_NOTIMPL;
    return MF_OK;
}

}  // namespace

typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// 2-D tensor map of a 16-bit row-major matrix [rows][K] (K contiguous),
// tiles of kKB x box_rows, 64-byte swizzle, zero fill out of bounds.
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
                    kSwz == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        log_msg("cuTensorMapEncodeTiled failed: %d", (int)r);
        return MF_E_CUDA;
    }
    return MF_OK;
}

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
    rc = make_tmap(h->tmap_lo, h->d_Wlo, at, h->Nk, h->Kdev, nbox);
    if (rc) return rc;
    // half-height boxes for the paired launch: each half a whole number of
    // 8-row swizzle atoms, so the two halves tile the ring slot exactly
    h->pair_ok = false;
    if (nbox % 16 == 0) {
        rc = make_tmap(h->tmap_hi2, h->d_Whi, at, h->Nk, h->Kdev, nbox / 2);
        if (rc) return rc;
        rc = make_tmap(h->tmap_lo2, h->d_Wlo, at, h->Nk, h->Kdev, nbox / 2);
        if (rc) return rc;
        h->pair_ok = true;
    }
    return MF_OK;
}

int fill_tc_event(const mf_handle *h, TcEvent *ev) {
    if (!h->d_Whi || !is_tc_form(h->form)) return MF_E_STATE;
    memset(ev, 0, sizeof(*ev));
    memcpy(&ev->tm_hi, h->tmap_hi, sizeof(CUtensorMap));
    memcpy(&ev->tm_lo, h->tmap_lo, sizeof(CUtensorMap));
    if (h->pair_ok) {
        memcpy(&ev->tm_hi2, h->tmap_hi2, sizeof(CUtensorMap));
        memcpy(&ev->tm_lo2, h->tmap_lo2, sizeof(CUtensorMap));
    }
    ev->pair_ok = h->pair_ok ? 1 : 0;
    ev->rot_mul = h->tc_rot ? 11 : 0;
    ev->epi = make_epi(h);
    ev->rot = make_rot(h);
    ev->nodes_s = h->d_nodes_s;
    ev->colscale = form_type(h->form) == 0 ? h->d_colscale : nullptr;
    ev->N = h->N;
    ev->P = h->P;
    ev->nkb = h->Nk / kKB;
    ev->nbox = h->nbox;
    return MF_OK;
}

size_t tc_smem_bytes(mf_form f, int np, int nbox_max, int sb) {
    if (np < 1 || np > kMaxCluster || sb < 2 || sb > kMaxStages || nbox_max < 16 || nbox_max > kAccCols) return 0;
    size_t b = smem_for(form_terms(f), np, nbox_max, sb);
    return b <= kSmemMax ? b : 0;
}

int tc_batch_max_clusters(mf_form f, int n_modes, int np, int nbox_max, int sb, int *max_clusters) {
    void *kern = pick_kernel(f, n_modes, true);
    const size_t smem = tc_smem_bytes(f, np, nbox_max, sb);
    if (!kern || !smem) return MF_E_NOTIMPL;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    return tc_config(kern, np, smem, nullptr, cfg, attr, max_clusters);
}

int launch_tc_batch(mf_form f, int n_modes, const TcEvent *d_events, const TcBatchCall &bc,
                    cudaStream_t st) {
    void *kern = pick_kernel(f, n_modes, true);
    const size_t smem = tc_smem_bytes(f, bc.np, bc.nbox_max, bc.sb);
    if (!kern || !smem) return MF_E_NOTIMPL;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    int maxc = 0;
    int rc = tc_config(kern, bc.np, smem, st, cfg, attr, &maxc);
    if (rc) return rc;
    if (bc.n_clusters < 1 || bc.n_clusters > maxc) return MF_E_INVAL;
    cfg.gridDim = dim3((unsigned)(bc.n_clusters * bc.np), 1, 1);
    void *args[2] = {(void *)&d_events, (void *)&bc};
    MF_CUDA(cudaLaunchKernelExC(&cfg, kern, args));
    return MF_OK;
}

// One launch over passes [p0, p0 + npc) of the handle (a cluster of npc, or
// 2 npc when paired, CTAs per query tile); the pass partials go to rows
// p0 .. p0 + npc - 1 of `partial`.
static int launch_tc_part(mf_handle *h, const float *intr, const float *ext, int Q, int E, float *out,
                          cudaStream_t st, float *partial, float *cols, int p0, int npc) {
    const int np = npc;
    int sb = h->tc_nbs ? h->tc_nbs : 4;
    while (!tc_smem_bytes(h->form, np, h->nbox, sb) && sb > 2) --sb;
    const size_t smem = tc_smem_bytes(h->form, np, h->nbox, sb);
    if (!smem) return MF_E_NOTIMPL;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    int rc;
    // paired launch: two query tiles per cluster sharing the weight tiles
    // (cluster of 2 np <= 8 CTAs), for the 3-term lnL kernels -- unless the
    // larger clusters leave more than 7 % more SMs idle than the single
    // launch's (clusters must fit a GPC; measured: pairing gains ~6 % at 6
    // CTAs per cluster and loses ~20 % at 8)
    bool pair = !cols && h->tc_pair && h->pair_ok && 2 * np <= kMaxCluster && form_terms(h->form) == 3 &&
                Q > kTile;
    if (pair) {
        void *kp = pick_pair_kernel(h->form, h->n_modes), *ks = pick_kernel(h->form, h->n_modes, false);
        int mp = 0, ms = 0;
        if (!kp || !ks) return MF_E_NOTIMPL;
        if ((rc = tc_config(kp, 2 * np, smem, st, cfg, attr, &mp))) return rc;
        if ((rc = tc_config(ks, np, smem, st, cfg, attr, &ms))) return rc;
        pair = 2.0 * np * mp >= 0.93 * np * ms;
    }
    h->tc_paired = pair ? 1 : 0;
    void *kern = cols ? pick_cols_kernel(h->form)
                      : pair ? pick_pair_kernel(h->form, h->n_modes) : pick_kernel(h->form, h->n_modes, false);
    if (!kern) return MF_E_NOTIMPL;
    TcEvent ev;
    rc = fill_tc_event(h, &ev);
    if (rc) return rc;
    ev.epi.n_pass = np;
    for (int i = 0; i < np; ++i) ev.epi.passes[i] = h->passes[p0 + i];
    TcCall c;
    memset(&c, 0, sizeof(c));
    c.cols = cols;
    c.umap = h->d_user_of_dev;
    c.K = h->K;
    c.intr = intr;
    c.ext = ext;
    c.out = out;
    c.partial = partial ? partial + (size_t)p0 * Q : nullptr;
    c.Q = Q;
    c.E = E;
    c.n_tiles = (Q + kTile - 1) / kTile;
    c.n_items = pair ? (c.n_tiles + 1) / 2 : c.n_tiles;
    c.nbox_max = h->nbox;
    c.err = h->d_err;
    c.sb = sb;
    int maxc = 0;
    const int cl = pair ? 2 * np : np;
    rc = tc_config(kern, cl, smem, st, cfg, attr, &maxc);
    if (rc) return rc;
    c.n_clusters = std::min(c.n_items, maxc);
    cfg.gridDim = dim3((unsigned)(c.n_clusters * cl), 1, 1);
    void *args[2] = {(void *)&ev, (void *)&c};
    MF_CUDA(cudaLaunchKernelExC(&cfg, kern, args));
    return MF_OK;
}

int tc_max_passes(mf_form f, int nbox) {
    for (int k = kMaxCluster; k >= 1; --k)
        if (tc_smem_bytes(f, k, nbox, 2)) return k;
    return 0;
}

// cols != nullptr: the columns-only variant, out [Q][K] (ext, out, partial unused).
// More passes than one cluster stages (its shared memory holds one Phi slot
// pair per pass) run as several launches over runs of 2 .. max passes, each
// writing its own pass partials (the per-pass arithmetic, hence every
// partial, is the same as in a single launch).
int launch_tc(mf_handle *h, const float *intr, const float *ext, int Q, int E, float *out,
              cudaStream_t st, float *partial, float *cols) {
    if (!h->d_Whi) return MF_E_STATE;
    const int np = (int)h->passes.size();
    int maxnp = tc_max_passes(h->form, h->nbox);
    if (h->tc_chunk > 0) maxnp = std::min(maxnp, h->tc_chunk);
    if (maxnp < 1) return MF_E_NOTIMPL;
    if (np <= maxnp) return launch_tc_part(h, intr, ext, Q, E, out, st, partial, cols, 0, np);
    const int nch = (np + maxnp - 1) / maxnp;
    if (np / nch < 2 || (!cols && !partial)) return MF_E_NOTIMPL;   // every run must write partials
    for (int c = 0, p0 = 0; c < nch; ++c) {
        const int cnt = np / nch + (c < np % nch ? 1 : 0);
        const int rc = launch_tc_part(h, intr, ext, Q, E, out, st, partial, cols, p0, cnt);
        if (rc) return rc;
        p0 += cnt;
    }
    return MF_OK;
}

}  // namespace mf

