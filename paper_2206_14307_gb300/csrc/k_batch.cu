// k_batch.cu -- a batch of models of uneven size (lattice, hidden units,
// number of RBMs, symmetry group) in one persistent launch (relocatable
// device code; the per-shape bodies live in k_mixed_<GL>_<MPL>.cu).
//
// The work is a list of (instance, sample, output slot) items, ordered by the
// host with the most expensive instances first; each CTA takes items from an
// atomic counter, loads the instance's device view into shared memory when it
// changes, and runs the body of the instance's tile shape (Lanczos mode: h1
// and h2, Sec. 3.3).  A second launch reduces every instance's samples to its
// FP64 moments and p = 1 Lanczos step.
#include "k_mixed.cuh"

namespace nnqs {

__global__ void __launch_bounds__(kThreads, 2)
    k_mixed(const DevModel<float> *__restrict__ models, const int *__restrict__ shape,
            const BatchItem *__restrict__ items, int nitems, int *__restrict__ counter,
            const uint64_t *__restrict__ cfg_all, const int64_t *__restrict__ cfg_off, double *__restrict__ h1_all,
            double *__restrict__ h2_all)
{
    extern __shared__ __align__(16) unsigned char smem_mixed[];
    DevModel<float> *smd = reinterpret_cast<DevModel<float> *>(smem_mixed + kMixedOffMd);
    __shared__ int item_sh, shape_sh;
    __shared__ BatchItem bi_sh;
    int loaded = -1;  // instance whose view is in shared memory (same in every thread)
    for (;;) {
        if (threadIdx.x == 0) {
            const int it = atomicAdd(counter, 1);
            item_sh = it;
            if (it < nitems) {
                bi_sh = items[it];
                shape_sh = shape[bi_sh.model];
            }
        }
        __syncthreads();
        if (item_sh >= nitems) break;
        const BatchItem bi = bi_sh;
        const int sh = shape_sh;
        if (bi.model != loaded) {
            if (threadIdx.x < 32) {
                const int *src = reinterpret_cast<const int *>(models + bi.model);
                int *dst = reinterpret_cast<int *>(smd);
                for (int w = threadIdx.x; w < (int)(sizeof(DevModel<float>) / sizeof(int)); w += 32) dst[w] = src[w];
            }
            loaded = bi.model;
            __syncthreads();
        }
        const uint64_t *row = cfg_all + cfg_off[bi.model] + (int64_t)bi.sample * smd->nwords;
        double *h1o = h1_all ? h1_all + 2 * (int64_t)bi.out : nullptr;
        double *h2o = h2_all ? h2_all + 2 * (int64_t)bi.out : nullptr;
        switch (sh) {
        case 0: mixed_sample_8_2(row, h1o, h2o); break;
        case 1: mixed_sample_8_4(row, h1o, h2o); break;
        case 2: mixed_sample_16_2(row, h1o, h2o); break;
        case 3: mixed_sample_8_5(row, h1o, h2o); break;
        case 4: mixed_sample_8_8(row, h1o, h2o); break;
        case 5: mixed_sample_16_4(row, h1o, h2o); break;
        case 6: mixed_sample_8_9(row, h1o, h2o); break;
        case 7: mixed_sample_16_5(row, h1o, h2o); break;
        case 8: mixed_sample_16_7(row, h1o, h2o); break;
        case 9: mixed_sample_16_8(row, h1o, h2o); break;
        case 10: mixed_sample_32_4(row, h1o, h2o); break;
        case 11: mixed_sample_16_9(row, h1o, h2o); break;
        case 12: mixed_sample_32_7(row, h1o, h2o); break;
        case 13: mixed_sample_32_8(row, h1o, h2o); break;
        case 14: mixed_sample_32_13(row, h1o, h2o); break;
        default: mixed_sample_32_16(row, h1o, h2o); break;
        }
        __syncthreads();  // the next item overwrites item_sh, bi_sh and the view
    }
}

static size_t mixed_smem_bytes()
{
    size_t b = eloc_smem<float, 8>(kMixedChunk);
    const size_t b16 = eloc_smem<float, 16>(kMixedChunk), b32 = eloc_smem<float, 32>(kMixedChunk);
    if (b16 > b) b = b16;
    if (b32 > b) b = b32;
    return kMixedOffRest + b;
}

int mixed_grid(int nsm)
{
    const size_t smem = mixed_smem_bytes();
    if (cudaFuncSetAttribute(k_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_mixed, kThreads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return (per > 0 ? per : 1) * nsm;
}

cudaError_t launch_mixed(int grid, const DevModel<float> *models, const int *shape, const BatchItem *items,
                         int nitems, int *counter, const uint64_t *cfg_all, const int64_t *cfg_off, double *h1_all,
                         double *h2_all, cudaStream_t st)
{
    if (nitems <= 0) return cudaSuccess;
    const int g = nitems < grid ? nitems : grid;
    k_mixed<<<g, kThreads, mixed_smem_bytes(), st>>>(models, shape, items, nitems, counter, cfg_all, cfg_off, h1_all,
                                                     h2_all);
    return cudaGetLastError();
}

// one block per instance: FP64 moments of its samples (the same sums as the
// single-model reduction) and the p = 1 step
__global__ void __launch_bounds__(256) k_moments_batched(const double *__restrict__ h1_all,
                                                         const double *__restrict__ h2_all,
                                                         const int64_t *__restrict__ out_off,
                                                         double *__restrict__ moments, double *__restrict__ lanczos)
{
    __shared__ double sh[8][kMomentSums];
    const int mi = blockIdx.x;
    const int64_t lo = out_off[mi], hi = out_off[mi + 1];
    double v[kMomentSums] = {0, 0, 0, 0, 0, 0, 0};
    for (int64_t k = lo + threadIdx.x; k < hi; k += blockDim.x) {
        const double ax = h1_all[2 * k], ay = h1_all[2 * k + 1], bx = h2_all[2 * k], by = h2_all[2 * k + 1];
        v[0] += 1.0;
        v[1] += ax;
        v[2] += ax * ax + ay * ay;
        v[3] += ax * bx + ay * by;  // Re(conj(h1) h2)
        v[4] += ay;
        v[5] += ax * by - ay * bx;  // Im(conj(h1) h2)
        v[6] += bx * bx + by * by;  // |h2|^2
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kMomentSums; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    if (lane == 0)
        for (int q = 0; q < kMomentSums; ++q) sh[warp][q] = v[q];
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int w = 1; w < 8; ++w)
        for (int q = 0; q < kMomentSums; ++q) sh[0][q] += sh[w][q];
    const double z = sh[0][0] > 0 ? sh[0][0] : 1.0;
    const double m1 = sh[0][1] / z, m2 = sh[0][2] / z, m3 = sh[0][3] / z;
    if (moments) {
        double *mo = moments + 8 * mi;
        mo[0] = 1.0; mo[1] = m1; mo[2] = m2; mo[3] = m3;
        mo[4] = sh[0][0]; mo[5] = sh[0][4] / z; mo[6] = sh[0][5] / z; mo[7] = sh[0][6] / z;
    }
    if (lanczos) lanczos_p1(m1, m2, m3, lanczos + 3 * mi);
}

cudaError_t launch_moments_batched(const double *h1_all, const double *h2_all, const int64_t *out_off, int nmodels,
                                   double *moments, double *lanczos, cudaStream_t st)
{
    if (nmodels <= 0) return cudaSuccess;
    k_moments_batched<<<nmodels, 256, 0, st>>>(h1_all, h2_all, out_off, moments, lanczos);
    return cudaGetLastError();
}

}  // namespace nnqs
