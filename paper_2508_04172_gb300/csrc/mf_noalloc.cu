// mf_loglike_noalloc: the plain FP32 lnL path for callers that must not
// allocate device memory during a call.
//
// Some callers cannot call cudaMalloc on their hot path: callers that hand
// all device memory to a fixed-size pool of their own at start-up, and
// real-time sampler loops that forbid any allocation (and the implicit
// device synchronisation cudaMalloc/cudaFree may bring) once they run.  When
// a handle's columns are split into several passes, mf_loglike needs a
// scratch buffer of n_pass * Q partial sums and grows one with cudaMalloc on
// demand.  This entry point keeps that scratch in a fixed-size array in the
// library's own device memory instead, so the call itself allocates nothing.
//
// The array (kNoallocMaxPartial floats, 16 MiB) is a file-scope __device__
// variable: every GPU that loads the library holds it until the process exits,
// and every call on that device shares it.  A call overwrites every entry it
// later reads, so nothing needs clearing; two calls that overlap on the GPU
// (different streams, or different handles on one device) race on it and must
// be serialised by the caller.
//
// Host code cannot use `g_noalloc_partial` as a device pointer (in host code
// the name is a host-side shadow).  The first call on each device looks up the
// device address with cudaGetSymbolAddress, with that device current, and
// caches it.  The cache belongs to the device's primary context: after a
// cudaDeviceReset in this process the cached address is stale, so a process
// that resets a device must not call this entry point on it again.
#include "mf_internal.cuh"

#include <mutex>

namespace {

constexpr size_t kNoallocMaxPartial = MF_NOALLOC_MAX_PARTIAL;

static __device__ __align__(256) float g_noalloc_partial[kNoallocMaxPartial];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float *g_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (set-up once per
// device, with that device current).
int scratch_address(float **out) {
    int dev = 0;
    MF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return MF_E_INVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partial);
        if (e != cudaSuccess) {
            mf::log_msg("noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return mf::cuda_status(e);
        }
        g_addr[dev] = static_cast<float *>(p);
    }
    *out = g_addr[dev];
    return MF_OK;
}

}  // namespace

extern "C" int mf_loglike_noalloc(mf_handle *h, const float *intrinsic, const float *extrinsic,
                                  int Q, int E, float *out_lnL, void *stream) {
    if (!h || Q < 0 || Q > (1 << 26) || E < 5) return MF_E_INVAL;
    if (Q == 0) return MF_OK;
    if (!intrinsic || !extrinsic || !out_lnL) return MF_E_INVAL;
    if ((uintptr_t)intrinsic & 15) return MF_E_INVAL;   // rows are read as float4
    if (!h->have_layout || !h->have_basis || !h->have_det) return MF_E_STATE;
    if (h->sky && E < 7) return MF_E_INVAL;
    if (h->form != MF_FORM_FP32 || !h->d_W32) return MF_E_STATE;
    // the handle's buffers and the scratch address belong to h->dev
    int cur = -1;
    MF_CUDA(cudaGetDevice(&cur));
    if (cur != h->dev) return MF_E_STATE;
    const size_t np = h->passes.size();
    if (np > 1 && np * (size_t)Q > kNoallocMaxPartial) {
        mf::log_msg("noalloc: n_pass * Q = %zu exceeds the %zu-float scratch", np * (size_t)Q,
                    kNoallocMaxPartial);
        return MF_E_INVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    float *partial = nullptr;
    if (np > 1) {
        int rc = scratch_address(&partial);
        if (rc) return rc;
    }
    int rc = mf::launch_fp32(h, intrinsic, extrinsic, Q, E, out_lnL, st, partial);
    if (rc) return rc;
    if (np > 1) return mf::launch_combine(partial, (int)np, Q, out_lnL, st, h->d_bad);
    return MF_OK;
}
