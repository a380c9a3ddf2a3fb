// k_eloc_dispatch.cu -- picks the variant of the connected-configuration engine:
// GL lanes per row and MPL hidden units per lane from the hidden-layer width,
// and the kernel holding only the single-bond path for E_loc.
#include "common.cuh"
#include "kernels.h"

namespace nnqs {

template <typename T, int GL, int MPL, int MODE>
cudaError_t launch_eloc_mode(const DevModel<T> &md, const uint64_t *cfg, int64_t n, int chunk, double *h1, double *h2,
                             int nsm, cudaStream_t st);

template <typename T, int GL, int MPL>
static cudaError_t by_mode(const DevModel<T> &md, const uint64_t *cfg, int64_t n, int mode, int chunk, double *h1,
                           double *h2, int nsm, cudaStream_t st)
{
    return mode == 0 ? launch_eloc_mode<T, GL, MPL, 0>(md, cfg, n, chunk, h1, h2, nsm, st)
                     : launch_eloc_mode<T, GL, MPL, 1>(md, cfg, n, chunk, h1, h2, nsm, st);
}

template <typename T>
cudaError_t launch_ratio_variant(const DevModel<T> &md, int v, const uint64_t *cfg, int64_t n, int mode, double *h1,
                                 double *h2, int nsm, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    if (v < 0 || v >= kNumVariants || variant_width(v) > md.Mp || variant_width(v) < md.M) return cudaErrorInvalidValue;
    const int chunk = mode == 0 ? md.nbonds : 512;
    switch (v) {
    case 0: return by_mode<T, 8, 2>(md, cfg, n, mode, chunk, h1, h2, nsm, st);
    case 1: return by_mode<T, 8, 4>(md, cfg, n, mode, chunk, h1, h2, nsm, st);
    case 2: return by_mode<T, 8, 9>(md, cfg, n, mode, chunk, h1, h2, nsm, st);
    case 3: return by_mode<T, 16, 8>(md, cfg, n, mode, chunk, h1, h2, nsm, st);
    case 4: return by_mode<T, 32, 8>(md, cfg, n, mode, chunk, h1, h2, nsm, st);
    case 5: return by_mode<T, 32, 13>(md, cfg, n, mode, chunk, h1, h2, nsm, st);
    default: return by_mode<T, 32, 16>(md, cfg, n, mode, chunk, h1, h2, nsm, st);
    }
}

template <typename T>
cudaError_t launch_ratio(const DevModel<T> &md, const uint64_t *cfg, int64_t n, int mode, double *h1, double *h2,
                         int nsm, cudaStream_t st)
{
    return launch_ratio_variant(md, default_variant(md.M), cfg, n, mode, h1, h2, nsm, st);
}

template cudaError_t launch_ratio_variant<float>(const DevModel<float> &, int, const uint64_t *, int64_t, int, double *, double *, int, cudaStream_t);
template cudaError_t launch_ratio_variant<double>(const DevModel<double> &, int, const uint64_t *, int64_t, int, double *, double *, int, cudaStream_t);
template cudaError_t launch_ratio<float>(const DevModel<float> &, const uint64_t *, int64_t, int, double *, double *, int, cudaStream_t);
template cudaError_t launch_ratio<double>(const DevModel<double> &, const uint64_t *, int64_t, int, double *, double *, int, cudaStream_t);

}  // namespace nnqs
