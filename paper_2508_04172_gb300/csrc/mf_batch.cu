// Batched lnL over many events (interpolants) in one persistent tcgen05
// launch, replayed from a CUDA graph, with the launch shape chosen by
// measurement.
//
// Every event of a batch is laid out in exactly np column passes (np = the
// cluster size of the launch), so one cluster of np CTAs handles any work
// item (event, query tile).  The tunable shape is (np, W ring depth): np
// sets the MMA N-tile width of every event (its device columns / np) and
// trades Phi-sharing (larger clusters generate each RBF tile once for more
// columns) against occupancy and shared memory.  The autotuner times every
// shape that fits on synthetic in-window queries of the planned sizes and
// keeps the fastest.
//
// Work items are listed event by event, events in order of decreasing
// modelled cost per tile (node blocks x (widest pass + 64)); clusters take
// them in snake order, so the clusters' totals differ by about one item.
#include "mf_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>

namespace {

using mf::TcBatchCall;
using mf::TcEvent;
using mf::kMaxBatch;

constexpr int kTile = mf::kTile;
constexpr int kMaxClusterSize = 8;

struct TuneEntry {
    int np, sb;
    double ms;
};

// Sum of the np partial lnL of every query of every event, NaN counted per
// event (Eq. logl_complete: the passes' terms add).
__global__ void combine_batch_kernel(const __grid_constant__ TcBatchCall c) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= c.qprefix[c.n_ev]) return;
    int lo = 0, hi = c.n_ev;   // qprefix[lo] <= g < qprefix[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (c.qprefix[mid] <= g) lo = mid;
        else hi = mid;
    }
    const int q = g - c.qprefix[lo];
    const int Q = c.Q[lo];
    const float *p = c.partial[lo];
    float s = 0.f;
    for (int k = 0; k < c.np; ++k) s += p[(size_t)k * Q + q];
    c.out[lo][q] = s;
    if (s != s) atomicAdd(c.bad[lo], 1ull);
}

// Synthetic in-window queries for timing: intrinsic inside the ball of
// radius 0.5, extrinsic (d_L, cos i, psi, phi_c, t_c) in typical ranges.
__global__ void synth_queries(float *intr, float *ext, int Q, unsigned seed) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= Q) return;
    unsigned x = seed ^ (2654435761u * (unsigned)(q + 1));
    auto next = [&x]() {
        x ^= x << 13;
        x ^= x >> 17;
        x ^= x << 5;
        return (float)(x >> 8) * (1.0f / 16777216.0f);
    };
    for (int i = 0; i < 4; ++i) intr[(size_t)q * 4 + i] = 0.5f * (next() - 0.5f);
    ext[(size_t)q * 5 + 0] = 100.f + 300.f * next();
    ext[(size_t)q * 5 + 1] = 2.f * next() - 1.f;
    ext[(size_t)q * 5 + 2] = 3.14159265f * next();
    ext[(size_t)q * 5 + 3] = 6.28318531f * next();
    ext[(size_t)q * 5 + 4] = 0.004f * (next() - 0.5f);
}

}  // namespace

struct mf_batch {
    int dev = 0;
    int n = 0;
    std::vector<mf_handle *> hs;
    std::vector<unsigned> gens;
    mf_form form = MF_FORM_FP32;
    int n_modes = 0;
    int np = 0, sb = 0, nbox_max = 0, max_clusters = 0;
    std::vector<double> cost;         // modelled cost per tile of each event
    TcEvent *d_events = nullptr;
    unsigned *d_err = nullptr;        // 16 status words
    float *d_partial = nullptr;
    size_t partial_cap = 0;
    cudaStream_t cap = nullptr;       // private stream the graph is captured on
    cudaGraphExec_t exec = nullptr;
    TcBatchCall last;
    bool use_graph = true;
    bool timing = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    long long captures = 0, replays = 0, launches = 0;
    int last_items = 0;
    std::vector<TuneEntry> tune;
};

namespace {

int release_graph(mf_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    return MF_OK;
}

// Lay every event out in exactly np passes; the W ring slot holds the widest.
int set_shape(mf_batch *b, int np) {
    int nbox = 0;
    for (mf_handle *h : b->hs) {
        if (h->pass_count_user != np || (int)h->passes.size() != np) {
            h->pass_count_user = np;
            int rc = mf::prepare_form(h, h->form);
            if (rc) return rc;
        }
        nbox = std::max(nbox, h->nbox);
    }
    b->np = np;
    b->nbox_max = nbox;
    b->cost.resize(b->n);
    for (int e = 0; e < b->n; ++e) {
        const mf_handle *h = b->hs[e];
        b->cost[e] = (double)(h->Nk / 32) * (double)(h->nbox + 64);
    }
    return MF_OK;
}

int upload_events(mf_batch *b) {
    std::vector<TcEvent> evs(b->n);
    for (int e = 0; e < b->n; ++e) {
        int rc = mf::fill_tc_event(b->hs[e], &evs[e]);
        if (rc) return rc;
    }
    if (!b->d_events) MF_CUDA(cudaMalloc((void **)&b->d_events, sizeof(TcEvent) * kMaxBatch));
    MF_CUDA(cudaMemcpy(b->d_events, evs.data(), sizeof(TcEvent) * b->n, cudaMemcpyHostToDevice));
    b->gens.resize(b->n);
    for (int e = 0; e < b->n; ++e) b->gens[e] = b->hs[e]->gen;
    release_graph(b);
    return MF_OK;
}

int ensure_partial(mf_batch *b, size_t need, cudaStream_t st) {
    if (need <= b->partial_cap) return MF_OK;
    // the captured graph and work in flight may still use the old buffer
    MF_CUDA(cudaStreamSynchronize(st));
    release_graph(b);
    if (b->d_partial) cudaFree(b->d_partial);
    b->d_partial = nullptr;
    b->partial_cap = 0;
    MF_CUDA(cudaMalloc((void **)&b->d_partial, sizeof(float) * need));
    b->partial_cap = need;
    return MF_OK;
}

// The per-call kernel argument block.
int make_call(mf_batch *b, const float *const *intr, const float *const *ext, const int *Q, int E,
              float *const *out, cudaStream_t st, TcBatchCall &c) {
    memset(&c, 0, sizeof(c));
    c.n_ev = b->n;
    c.E = E;
    c.np = b->np;
    c.sb = b->sb;
    c.nbox_max = b->nbox_max;
    c.err = b->d_err;
    size_t need = 0;
    for (int e = 0; e < b->n; ++e) need += (size_t)b->np * (size_t)Q[e];
    if (b->np > 1) {
        int rc = ensure_partial(b, need, st);
        if (rc) return rc;
    }
    std::vector<int> ord(b->n);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return b->cost[x] > b->cost[y]; });
    int items = 0;
    for (int k = 0; k < b->n; ++k) {
        c.order[k] = ord[k];
        c.tprefix[k] = items;
        items += (Q[ord[k]] + kTile - 1) / kTile;
    }
    c.tprefix[b->n] = items;
    c.n_items = items;
    size_t off = 0;
    int qsum = 0;
    for (int e = 0; e < b->n; ++e) {
        c.qprefix[e] = qsum;
        qsum += Q[e];
        c.Q[e] = Q[e];
        c.intr[e] = intr[e];
        c.ext[e] = ext[e];
        c.out[e] = out[e];
        c.partial[e] = b->np > 1 ? b->d_partial + off : nullptr;
        c.bad[e] = b->hs[e]->d_bad;
        off += (size_t)b->np * (size_t)Q[e];
    }
    c.qprefix[b->n] = qsum;
    c.n_clusters = std::max(1, std::min(items, b->max_clusters));
    return MF_OK;
}

int enqueue(mf_batch *b, const TcBatchCall &c, cudaStream_t st) {
    int rc = mf::launch_tc_batch(b->form, b->n_modes, b->d_events, c, st);
    if (rc) return rc;
    if (b->np > 1 && c.qprefix[c.n_ev] > 0) {
        combine_batch_kernel<<<(c.qprefix[c.n_ev] + 255) / 256, 256, 0, st>>>(c);
        MF_CUDA(cudaGetLastError());
    }
    return MF_OK;
}

// Launch through the graph: replay when the argument block is unchanged,
// otherwise capture the two launches again and update the executable graph.
int run(mf_batch *b, const TcBatchCall &c, cudaStream_t st) {
    b->last_items = c.n_items;
    if (c.n_items == 0) return MF_OK;
    if (!b->use_graph) {
        ++b->launches;
        return enqueue(b, c, st);
    }
    if (!b->exec || memcmp(&c, &b->last, sizeof(c)) != 0) {
        cudaGraph_t g = nullptr;
        MF_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed));
        int rc = enqueue(b, c, b->cap);
        cudaError_t e = cudaStreamEndCapture(b->cap, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        MF_CUDA(e);
        bool updated = false;
        if (b->exec) {
            cudaGraphExecUpdateResultInfo info;
            updated = cudaGraphExecUpdate(b->exec, g, &info) == cudaSuccess;
            if (!updated) {
                cudaGetLastError();
                release_graph(b);
            }
        }
        if (!updated) {
            cudaError_t ei = cudaGraphInstantiate(&b->exec, g, 0);
            if (ei != cudaSuccess) {
                cudaGraphDestroy(g);
                b->exec = nullptr;
                MF_CUDA(ei);
            }
        }
        cudaGraphDestroy(g);
        b->last = c;
        ++b->captures;
    } else {
        ++b->replays;
    }
    MF_CUDA(cudaGraphLaunch(b->exec, st));
    ++b->launches;
    return MF_OK;
}

int check_handles(const mf_batch *b) {
    for (int e = 0; e < b->n; ++e)
        if (b->hs[e]->gen != b->gens[e] || b->hs[e]->form != b->form) return MF_E_STATE;
    return MF_OK;
}

// Time every (np, ring depth) that fits on synthetic queries of the planned
// sizes; leave the batch in the fastest shape.
int autotune(mf_batch *b, int np_min, int np_max, const int *Qp, bool measure, cudaStream_t st) {
    std::vector<float *> bi(b->n), be(b->n), bo(b->n);
    std::vector<const float *> ci(b->n), ce(b->n);
    int rc = MF_OK;
    float *pool = nullptr;
    // every buffer starts on a 256-byte boundary (the kernels read intrinsic rows as float4)
    auto up64 = [](size_t x) { return (x + 63) / 64 * 64; };
    size_t tot = 0;
    for (int e = 0; e < b->n; ++e) tot += up64((size_t)Qp[e] * 4) + up64((size_t)Qp[e] * 5) + up64(Qp[e]);
    if (measure) {
        MF_CUDA(cudaMalloc((void **)&pool, sizeof(float) * std::max<size_t>(tot, 1)));
        size_t off = 0;
        for (int e = 0; e < b->n; ++e) {
            bi[e] = pool + off;
            off += up64((size_t)Qp[e] * 4);
            be[e] = pool + off;
            off += up64((size_t)Qp[e] * 5);
            bo[e] = pool + off;
            off += up64(Qp[e]);
            ci[e] = bi[e];
            ce[e] = be[e];
            if (Qp[e] > 0) synth_queries<<<(Qp[e] + 255) / 256, 256, 0, st>>>(bi[e], be[e], Qp[e], 12345u + e);
        }
        cudaError_t e0 = cudaGetLastError();
        if (e0 != cudaSuccess) {
            cudaFree(pool);
            MF_CUDA(e0);
        }
    }
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (measure) {
        cudaEventCreate(&t0);
        cudaEventCreate(&t1);
    }
    b->tune.clear();
    const bool graph = b->use_graph;
    b->use_graph = false;
    int best_np = 0, best_sb = 0;
    double best = 1e300;
    for (int np = np_min; np <= np_max && rc == MF_OK; ++np) {
        int r2 = set_shape(b, np);
        if (r2) continue;   // this many passes does not fit every event
        for (int sb = 4; sb >= 2; --sb) {
            if (!mf::tc_smem_bytes(b->form, np, b->nbox_max, sb)) continue;
            int maxc = 0;
            if (mf::tc_batch_max_clusters(b->form, b->n_modes, np, b->nbox_max, sb, &maxc)) continue;
            b->sb = sb;
            b->max_clusters = maxc;
            if (!measure) {   // no timing: the deepest ring of the fewest passes
                best_np = np;
                best_sb = sb;
                break;
            }
            rc = upload_events(b);
            if (rc) break;
            TcBatchCall c;
            rc = make_call(b, ci.data(), ce.data(), Qp, 5, bo.data(), st, c);
            if (rc) break;
            float ms_best = 1e30f;
            for (int it = 0; it < 4 && rc == MF_OK; ++it) {
                cudaEventRecord(t0, st);
                rc = enqueue(b, c, st);
                cudaEventRecord(t1, st);
                cudaError_t es = cudaEventSynchronize(t1);
                if (es != cudaSuccess) {
                    mf::log_msg("batch autotune: shape (%d passes, ring %d): %s", np, sb, cudaGetErrorString(es));
                    rc = mf::cuda_status(es);
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, t0, t1);
                if (it > 0) ms_best = std::min(ms_best, ms);   // first run is a warm-up
            }
            unsigned err = 0;
            cudaMemcpy(&err, b->d_err, sizeof(err), cudaMemcpyDeviceToHost);
            if (err) rc = MF_E_TIMEOUT;
            if (rc) break;
            b->tune.push_back({np, sb, (double)ms_best});
            if (ms_best < best) {
                best = ms_best;
                best_np = np;
                best_sb = sb;
            }
        }
        if (!measure && best_np) break;
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (pool) cudaFree(pool);
    b->use_graph = graph;
    // the synthetic runs counted their out-of-window queries: clear them
    for (mf_handle *h : b->hs) cudaMemset(h->d_bad, 0, sizeof(unsigned long long));
    cudaMemset(b->d_err, 0, 16 * sizeof(unsigned));
    if (rc) return rc;
    if (!best_np) return MF_E_NOTIMPL;
    rc = set_shape(b, best_np);
    if (rc) return rc;
    b->sb = best_sb;
    rc = mf::tc_batch_max_clusters(b->form, b->n_modes, best_np, b->nbox_max, best_sb, &b->max_clusters);
    if (rc) return rc;
    return upload_events(b);
}

void destroy(mf_batch *b) {
    if (!b) return;
    release_graph(b);
    if (b->d_events) cudaFree(b->d_events);
    if (b->d_err) cudaFree(b->d_err);
    if (b->d_partial) cudaFree(b->d_partial);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    delete b;
}

}  // namespace

extern "C" {

int mf_batch_create(mf_handle *const *hs, int n_events, const int *Q_plan, int autotune_shape,
                    void *stream, mf_batch **out) {
    if (!out) return MF_E_INVAL;
    *out = nullptr;
    if (!hs || !Q_plan || n_events < 1 || n_events > kMaxBatch) return MF_E_INVAL;
    for (int e = 0; e < n_events; ++e) {
        const mf_handle *h = hs[e];
        if (!h || Q_plan[e] < 0 || Q_plan[e] > (1 << 26)) return MF_E_INVAL;
        if (!h->have_layout || !h->have_basis || !h->have_det) return MF_E_STATE;
        if (!mf::is_tc_form(h->form) || !h->d_Whi) return MF_E_STATE;
        if (h->form != hs[0]->form || h->n_modes != hs[0]->n_modes) return MF_E_INVAL;
    }
    int dev = 0;
    MF_CUDA(cudaGetDevice(&dev));
    mf_batch *b = new (std::nothrow) mf_batch();
    if (!b) return MF_E_NOMEM;
    b->dev = dev;
    b->n = n_events;
    b->hs.assign(hs, hs + n_events);
    b->form = hs[0]->form;
    b->n_modes = hs[0]->n_modes;
    if (cudaMalloc((void **)&b->d_err, 16 * sizeof(unsigned)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        destroy(b);
        return MF_E_NOMEM;
    }
    cudaMemset(b->d_err, 0, 16 * sizeof(unsigned));
    // fewest passes every event fits in (<= 256 columns each), most = groups of the smallest
    int np_min = 1, np_max = kMaxClusterSize;
    for (mf_handle *h : b->hs) {
        int ng = (int)h->groups.size();
        np_max = std::min(np_max, ng);
        np_min = std::max(np_min, (h->Kdev + 255) / 256);
    }
    if (np_min > np_max) {
        destroy(b);
        return MF_E_NOTIMPL;
    }
    std::vector<int> prev(n_events);
    for (int e = 0; e < n_events; ++e) prev[e] = hs[e]->pass_count_user;
    int rc = autotune(b, np_min, np_max, Q_plan, autotune_shape != 0, (cudaStream_t)stream);
    if (rc) {
        // give the handles back their own layout
        for (int e = 0; e < n_events; ++e) {
            hs[e]->pass_count_user = prev[e];
            mf::prepare_form(hs[e], hs[e]->form);
        }
        destroy(b);
        return rc;
    }
    *out = b;
    return MF_OK;
}

int mf_batch_loglike(mf_batch *b, const float *const *intrinsic, const float *const *extrinsic,
                     const int *Q, int E, float *const *out_lnL, void *stream) {
    if (!b || !intrinsic || !extrinsic || !Q || !out_lnL || E < 5) return MF_E_INVAL;
    for (int e = 0; e < b->n; ++e)
        if (b->hs[e]->sky && E < 7) return MF_E_INVAL;   // (alpha, delta) columns needed
    long long qtot = 0;
    for (int e = 0; e < b->n; ++e) {
        if (Q[e] < 0 || Q[e] > (1 << 26)) return MF_E_INVAL;
        if (Q[e] > 0 && (!intrinsic[e] || !extrinsic[e] || !out_lnL[e])) return MF_E_INVAL;
        if (Q[e] > 0 && ((uintptr_t)intrinsic[e] & 15)) return MF_E_INVAL;
        qtot += Q[e];
    }
    if (qtot > (1ll << 30)) return MF_E_INVAL;
    int rc = check_handles(b);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    TcBatchCall c;
    rc = make_call(b, intrinsic, extrinsic, Q, E, out_lnL, st, c);
    if (rc) return rc;
    if (b->timing) MF_CUDA(cudaEventRecord(b->ev0, st));
    rc = run(b, c, st);
    if (rc) return rc;
    if (b->timing) MF_CUDA(cudaEventRecord(b->ev1, st));
    return MF_OK;
}

int mf_batch_set_option(mf_batch *b, const char *key, double value) {
    if (!b || !key) return MF_E_INVAL;
    std::string k(key);
    if (k == "timing") {
        if (value != 0 && !b->ev0) {
            MF_CUDA(cudaEventCreate(&b->ev0));
            MF_CUDA(cudaEventCreate(&b->ev1));
        }
        b->timing = value != 0;
        return MF_OK;
    }
    if (k == "graph") {
        b->use_graph = value != 0;
        return MF_OK;
    }
    return MF_E_INVAL;
}

int mf_batch_query(const mf_batch *b, const char *key, double *value) {
    if (!b || !key || !value) return MF_E_INVAL;
    std::string k(key);
    if (k == "n_events") *value = b->n;
    else if (k == "n_pass") *value = b->np;
    else if (k == "ring") *value = b->sb;
    else if (k == "nbox") *value = b->nbox_max;
    else if (k == "clusters") *value = b->max_clusters;
    else if (k == "n_items") *value = b->last_items;
    else if (k == "captures") *value = (double)b->captures;
    else if (k == "replays") *value = (double)b->replays;
    else if (k == "launches") *value = b->np > 1 ? 2.0 : 1.0;
    else if (k == "n_tuned") *value = (double)b->tune.size();
    else if (k == "kernel_ms") {
        if (!b->timing) return MF_E_STATE;
        float ms = 0.f;
        MF_CUDA(cudaEventSynchronize(b->ev1));
        MF_CUDA(cudaEventElapsedTime(&ms, b->ev0, b->ev1));
        *value = ms;
    } else
        return MF_E_INVAL;
    return MF_OK;
}

int mf_batch_tuning(const mf_batch *b, int i, int *n_pass, int *ring, double *ms) {
    if (!b || i < 0 || i >= (int)b->tune.size()) return MF_E_INVAL;
    if (n_pass) *n_pass = b->tune[i].np;
    if (ring) *ring = b->tune[i].sb;
    if (ms) *ms = b->tune[i].ms;
    return MF_OK;
}

int mf_batch_sync_status(mf_batch *b, void *stream, long long *n_bad) {
    if (!b) return MF_E_INVAL;
    MF_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    unsigned ew[16];
    MF_CUDA(cudaMemcpy(ew, b->d_err, sizeof(ew), cudaMemcpyDeviceToHost));
    if (ew[0]) {
        mf::log_msg("batch device status 0x%x; first give-up k-block+1 per site:", ew[0]);
        for (int i = 1; i < 9; ++i)
            if (ew[i]) mf::log_msg("  site %d: %u", i - 1, ew[i]);
    }
    MF_CUDA(cudaMemset(b->d_err, 0, sizeof(ew)));
    long long tot = 0;
    for (mf_handle *h : b->hs) {
        unsigned long long v = 0;
        MF_CUDA(cudaMemcpy(&v, h->d_bad, sizeof(v), cudaMemcpyDeviceToHost));
        MF_CUDA(cudaMemset(h->d_bad, 0, sizeof(v)));
        tot += (long long)v;
    }
    if (n_bad) *n_bad = tot;
    if (ew[0]) return MF_E_TIMEOUT;
    return tot ? MF_E_RANGE : MF_OK;
}

void mf_batch_free(mf_batch *b) { destroy(b); }

int mf_loglike_batch(mf_handle *const *hs, int n_events, const float *const *intrinsic,
                     const float *const *extrinsic, const int *Q, int E, float *const *out_lnL,
                     void *stream) {
    mf_batch *b = nullptr;
    int rc = mf_batch_create(hs, n_events, Q, 0, stream, &b);
    if (rc) return rc;
    b->use_graph = false;
    rc = mf_batch_loglike(b, intrinsic, extrinsic, Q, E, out_lnL, stream);
    // the launch reads the batch's event table: finish before freeing it
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    destroy(b);
    if (rc) return rc;
    return e == cudaSuccess ? MF_OK : mf::cuda_status(e);
}

}  // extern "C"
