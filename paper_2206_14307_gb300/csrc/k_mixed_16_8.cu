// Mixed-batch body of tile shape GL = 16, MPL = 8 (relocatable device code).
#include "k_mixed.cuh"

namespace nnqs {
NNQS_MIXED_DEF(16, 8)
}  // namespace nnqs
