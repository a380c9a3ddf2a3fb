// Tensor-core log psi with 20 hidden units per epilogue thread and block (one
// translation unit per unit count, so that the variants compile in parallel).
#include "k_logpsi_tc.cuh"

namespace nnqs {
NNQS_TC_INSTANTIATE(20)
}  // namespace nnqs
