// float instantiation of the connected-configuration engine: GL = 32, MPL = 16,
// all flip-set kinds (Lanczos).
#include "k_eloc.cuh"

namespace nnqs {
template cudaError_t launch_eloc_mode<float, 32, 16, 1>(const DevModel<float> &, const uint64_t *, int64_t, int,
                                                             double *, double *, int, cudaStream_t);
}  // namespace nnqs
