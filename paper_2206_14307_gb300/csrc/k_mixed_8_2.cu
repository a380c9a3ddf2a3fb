// Mixed-batch body of tile shape GL = 8, MPL = 2 (relocatable device code).
#include "k_mixed.cuh"

namespace nnqs {
NNQS_MIXED_DEF(8, 2)
}  // namespace nnqs
