// lgt_stout.cu -- stout smearing (placeholder until the adjoint kernels land)
#include "lgt_internal.h"
#include "lgt_su3.cuh"

namespace lgt {
cudaError_t stout_forward(const double2*, double2*, const Geom&, double, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t stout_backward(const double2*, const double2*, double2*, double2*, const Geom&, double, cudaStream_t) {
    return cudaErrorNotSupported;
}
}  // namespace lgt
