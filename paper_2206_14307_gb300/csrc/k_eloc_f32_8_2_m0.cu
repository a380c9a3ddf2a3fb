// float instantiation of the connected-configuration engine: GL = 8, MPL = 2,
// single exchanged bonds (E_loc).
#include "k_eloc.cuh"

namespace nnqs {
template cudaError_t launch_eloc_mode<float, 8, 2, 0>(const DevModel<float> &, const uint64_t *, int64_t, int,
                                                             double *, double *, int, cudaStream_t);
}  // namespace nnqs
