// Mixed-batch body of tile shape GL = 16, MPL = 5 (relocatable device code).
#include "k_mixed.cuh"

namespace nnqs {
NNQS_MIXED_DEF(16, 5)
}  // namespace nnqs
