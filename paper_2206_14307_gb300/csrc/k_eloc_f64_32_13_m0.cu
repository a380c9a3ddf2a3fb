// double instantiation of the connected-configuration engine: GL = 32, MPL = 13,
// single exchanged bonds (E_loc).
#include "k_eloc.cuh"

namespace nnqs {
template cudaError_t launch_eloc_mode<double, 32, 13, 0>(const DevModel<double> &, const uint64_t *, int64_t, int,
                                                             double *, double *, int, cudaStream_t);
}  // namespace nnqs
