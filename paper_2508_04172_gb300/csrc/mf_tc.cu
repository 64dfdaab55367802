// tcgen05 forms of the fused lnL kernel (placeholder until implemented).
#include "mf_internal.cuh"

namespace mf {
int convert_tc_weights(mf_handle *, mf_form) { return MF_E_NOTIMPL; }
int launch_tc(mf_handle *, const float *, const float *, int, int, float *, cudaStream_t, float *) {
    return MF_E_NOTIMPL;
}
}  // namespace mf
