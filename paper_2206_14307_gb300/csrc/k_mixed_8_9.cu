// Mixed-batch body of tile shape GL = 8, MPL = 9 (relocatable device code).
#include "k_mixed.cuh"

namespace nnqs {
NNQS_MIXED_DEF(8, 9)
}  // namespace nnqs
