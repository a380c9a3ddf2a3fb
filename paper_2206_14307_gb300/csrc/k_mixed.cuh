// k_mixed.cuh -- the per-sample bodies of the mixed-batch launch.
//
// Each tile shape's body is a separately compiled device function (relocatable
// device code, one translation unit per shape, so that they compile in
// parallel); the persistent kernel calls the body of the item's instance.
// The bodies take the instance's device view and the engine's per-CTA state
// from fixed offsets of the dynamic shared memory:
//   [EShared<float>] [DevModel<float>] [entries, accumulators, tiles]
#pragma once
#include "k_eloc.cuh"

namespace nnqs {

constexpr int kMixedChunk = 512;  // entries gathered per pass (Lanczos mode)
constexpr size_t kMixedOffS = 0;
constexpr size_t kMixedOffMd = (sizeof(EShared<float>) + 15) / 16 * 16;
constexpr size_t kMixedOffRest = (kMixedOffMd + sizeof(DevModel<float>) + 15) / 16 * 16;

#define NNQS_MIXED_DECL(GL, MPL) \
    __device__ void mixed_sample_##GL##_##MPL(const uint64_t *row, double *h1o, double *h2o);
NNQS_MIXED_DECL(8, 2)
NNQS_MIXED_DECL(8, 4)
NNQS_MIXED_DECL(16, 2)
NNQS_MIXED_DECL(8, 5)
NNQS_MIXED_DECL(8, 8)
NNQS_MIXED_DECL(16, 4)
NNQS_MIXED_DECL(8, 9)
NNQS_MIXED_DECL(16, 5)
NNQS_MIXED_DECL(16, 7)
NNQS_MIXED_DECL(16, 8)
NNQS_MIXED_DECL(32, 4)
NNQS_MIXED_DECL(16, 9)
NNQS_MIXED_DECL(32, 7)
NNQS_MIXED_DECL(32, 8)
NNQS_MIXED_DECL(32, 13)
NNQS_MIXED_DECL(32, 16)

#define NNQS_MIXED_DEF(GL, MPL)                                                                           \
    __device__ __noinline__ void mixed_sample_##GL##_##MPL(const uint64_t *row, double *h1o, double *h2o) \
    {                                                                                                     \
        extern __shared__ __align__(16) unsigned char smem_mixed[];                                      \
        const DevModel<float> &md = *reinterpret_cast<const DevModel<float> *>(smem_mixed + kMixedOffMd);  \
        EShared<float> &S = *reinterpret_cast<EShared<float> *>(smem_mixed + kMixedOffS);                  \
        eloc_sample<float, GL, MPL, 1>(md, row, kMixedChunk, h1o, h2o, S, smem_mixed + kMixedOffRest);     \
    }

}  // namespace nnqs
