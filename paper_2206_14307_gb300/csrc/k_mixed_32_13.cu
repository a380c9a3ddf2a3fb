// Mixed-batch body of tile shape GL = 32, MPL = 13 (relocatable device code).
#include "k_mixed.cuh"

namespace nnqs {
NNQS_MIXED_DEF(32, 13)
}  // namespace nnqs
