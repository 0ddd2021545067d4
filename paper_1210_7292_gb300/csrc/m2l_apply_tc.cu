// Tensor-core (tcgen05) apply kernels; filled in below.
#include "m2l_internal.cuh"

namespace m2l {
m2l_status launch_tc(const m2l_ops *, const Buckets &, const void *, void *, int, int, double, cudaStream_t)
{
    set_error("tensor-core precisions are not built yet");
    return M2L_EUNSUPPORTED;
}
}  // namespace m2l
