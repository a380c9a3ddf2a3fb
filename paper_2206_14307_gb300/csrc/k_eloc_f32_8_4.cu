// float instantiation of the connected-configuration engine, GL = 8, MPL = 4.
#include "k_eloc.cuh"

namespace nnqs {
template cudaError_t launch_eloc_variant<float, 8, 4>(const DevModel<float> &, const uint64_t *, int64_t, int, int,
                                                          double *, double *, int, cudaStream_t);
}  // namespace nnqs
