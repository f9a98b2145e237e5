// Tensor-core (tcgen05) form of the feature contraction: not yet built.
#include "gsff_internal.cuh"

namespace gsff {

gs_status launch_render_fwd_tc(const CamF&, const int32_t*, const uint32_t*, const float*, const float*,
                               const __nv_bfloat16*, int, float*, int32_t*, cudaStream_t) {
  return GS_ERR_UNSUPPORTED;
}

}  // namespace gsff
