// double instantiation of the connected-configuration engine, GL = 32, MPL = 8.
#include "k_eloc.cuh"

namespace nnqs {
template cudaError_t launch_eloc_variant<double, 32, 8>(const DevModel<double> &, const uint64_t *, int64_t, int, int,
                                                          double *, double *, int, cudaStream_t);
}  // namespace nnqs
