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
cudaError_t launch_ratio(const DevModel<T> &md, const uint64_t *cfg, int64_t n, int mode, double *h1, double *h2,
                         int nsm, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int chunk = mode == 0 ? md.nbonds : 512;
    const int M = md.M;
    if (M <= 16) return by_mode<T, 8, 2>(md, cfg, n, mode, chunk, h1, h2, nsm, st);
    if (M <= 32) return by_mode<T, 8, 4>(md, cfg, n, mode, chunk, h1, h2, nsm, st);
    if (M <= 72) return by_mode<T, 8, 9>(md, cfg, n, mode, chunk, h1, h2, nsm, st);
    if (M <= 128) return by_mode<T, 16, 8>(md, cfg, n, mode, chunk, h1, h2, nsm, st);
    if (M <= 256) return by_mode<T, 32, 8>(md, cfg, n, mode, chunk, h1, h2, nsm, st);
    if (M <= 416) return by_mode<T, 32, 13>(md, cfg, n, mode, chunk, h1, h2, nsm, st);
    return by_mode<T, 32, 16>(md, cfg, n, mode, chunk, h1, h2, nsm, st);
}

template cudaError_t launch_ratio<float>(const DevModel<float> &, const uint64_t *, int64_t, int, double *, double *, int, cudaStream_t);
template cudaError_t launch_ratio<double>(const DevModel<double> &, const uint64_t *, int64_t, int, double *, double *, int, cudaStream_t);

}  // namespace nnqs
