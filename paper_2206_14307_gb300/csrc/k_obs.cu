// k_obs.cu -- observables from the samples: the static spin structure factor
// (Sec. 4.1) and the energy variance of the p = 0 and p = 1 states with the
// variance extrapolation (Sec. 3.3 Eq. 16; Sec. 4.3).
#include "common.cuh"
#include "kernels.h"

namespace nnqs {

constexpr int kSqThreads = 256;  // one wave vector per thread (N <= kMaxN = 256)

int sq_grid(int64_t n, int nsm)
{
    const int64_t g = 2 * (int64_t)nsm;
    return (int)(n < g ? n : g);
}

// Stage 1: block b sums w_k |rho_k(q)|^2 over samples k = b, b + grid, ...
// with rho_k(q) = sum_j sz_j e^{i q.r_j}, sz = s/2, q = 2 pi (qx, qy)/L;
// thread t owns q = t.  partial: [grid][N + 1] (the last entry: sum of w).
__global__ void __launch_bounds__(kSqThreads) k_sq_partial(const uint64_t *__restrict__ cfg, int64_t n, int L,
                                                           int nwords, const double *__restrict__ weights,
                                                           double *__restrict__ partial)
{
    __shared__ double cs[kMaxL], sn[kMaxL];
    __shared__ double sz[kMaxN];
    const int N = L * L;
    if (threadIdx.x < L) {
        double s, c;
        sincospi(2.0 * threadIdx.x / L, &s, &c);
        cs[threadIdx.x] = c;
        sn[threadIdx.x] = s;
    }
    const int qx = threadIdx.x % L, qy = threadIdx.x / L;
    double acc = 0.0, wsum = 0.0;
    for (int64_t k = blockIdx.x; k < n; k += gridDim.x) {
        __syncthreads();  // the previous sample's spins are no longer read
        for (int i = threadIdx.x; i < N; i += blockDim.x) sz[i] = 0.5 * spin_of(cfg + k * nwords, i);
        __syncthreads();
        const double w = weights ? weights[k] : 1.0;
        wsum += w;
        if (threadIdx.x < N) {
            double re = 0.0, im = 0.0;
            for (int y = 0; y < L; ++y) {
                int ph = (qy * y) % L;  // phase index (qx x + qy y) mod L
                for (int x = 0; x < L; ++x) {
                    const double v = sz[x + L * y];
                    re += v * cs[ph];
                    im += v * sn[ph];
                    ph += qx;
                    if (ph >= L) ph -= L;
                }
            }
            acc += w * (re * re + im * im);
        }
    }
    if (threadIdx.x < N) partial[(size_t)blockIdx.x * (N + 1) + threadIdx.x] = acc;
    if (threadIdx.x == 0) partial[(size_t)blockIdx.x * (N + 1) + N] = wsum;
}

// Stage 2: fixed-order sum over the blocks; S(q) = sum / (sum w * N^2).
__global__ void __launch_bounds__(kSqThreads) k_sq_final(const double *__restrict__ partial, int grid, int N,
                                                         double *__restrict__ sq)
{
    if (threadIdx.x >= N) return;
    double a = 0.0, z = 0.0;
    for (int b = 0; b < grid; ++b) {
        a += partial[(size_t)b * (N + 1) + threadIdx.x];
        z += partial[(size_t)b * (N + 1) + N];
    }
    sq[threadIdx.x] = a / (z * (double)N * (double)N);
}

cudaError_t launch_structure_factor(const uint64_t *cfg, int64_t n, int L, int nwords, const double *weights,
                                    double *partial, int grid, double *sq_out, cudaStream_t st)
{
    k_sq_partial<<<grid, kSqThreads, 0, st>>>(cfg, n, L, nwords, weights, partial);
    k_sq_final<<<1, kSqThreads, 0, st>>>(partial, grid, L * L, sq_out);
    return cudaGetLastError();
}

// The p = 1 state phi = psi0 + alpha (H - m1) psi0 / v = a psi0 + b H psi0
// (b = alpha / v, a = 1 - alpha m1 / v) has <phi|H^k|phi> = a^2 m_k +
// 2ab m_{k+1} + b^2 m_{k+2}; its energy and variance follow, and the line
// through (var0, m1) and (var1, E1) is taken to zero variance.
__global__ void k_lanczos_variance(const double *__restrict__ mo, const double *__restrict__ lz,
                                   double *__restrict__ out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double m1 = mo[1], m2 = mo[2], m3 = mo[3], m4 = mo[7];
    const double v = lz[1], alpha = lz[2];
    const double var0 = m2 - m1 * m1;
    double a = 1.0, b = 0.0;
    if (v > 0.0) {
        b = alpha / v;
        a = 1.0 - alpha * m1 / v;
    }
    const double n0 = a * a + 2.0 * a * b * m1 + b * b * m2;
    const double n1 = a * a * m1 + 2.0 * a * b * m2 + b * b * m3;
    const double n2 = a * a * m2 + 2.0 * a * b * m3 + b * b * m4;
    const double E1 = n1 / n0, var1 = n2 / n0 - E1 * E1;
    out[0] = var0;
    out[1] = E1;
    out[2] = var1;
    out[3] = var0 != var1 ? E1 - var1 * (m1 - E1) / (var0 - var1) : E1;
}

cudaError_t launch_lanczos_variance(const double *moments, const double *lanczos, double *out, cudaStream_t st)
{
    k_lanczos_variance<<<1, 32, 0, st>>>(moments, lanczos, out);
    return cudaGetLastError();
}

}  // namespace nnqs
