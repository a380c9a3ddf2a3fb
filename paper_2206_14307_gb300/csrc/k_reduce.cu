// k_reduce.cu -- FP64 reductions (moments of Sec. 3.3, E_loc sums, the energy
// gradient and the SR product of Eq. 12) and the parameter-derived tables.
#include "common.cuh"
#include "kernels.h"

namespace nnqs {

constexpr int kRedThreads = 256;

template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double (*sh)[NV])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) sh[warp][q] = v[q];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
#pragma unroll
            for (int q = 0; q < NV; ++q) sh[0][q] += sh[w][q];
#pragma unroll
        for (int q = 0; q < NV; ++q) v[q] = sh[0][q];
    }
}

// stage 1: per-block sums over a contiguous range of samples
__global__ void __launch_bounds__(kRedThreads) k_moments_partial(const double *__restrict__ h1,
                                                                 const double *__restrict__ h2, int64_t n,
                                                                 double *__restrict__ partial)
{
    __shared__ double sh[kRedThreads / 32][kMomentSums];
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t lo = per * blockIdx.x, hi = lo + per < n ? lo + per : n;
    double v[kMomentSums] = {0, 0, 0, 0, 0, 0, 0};
    for (int64_t k = lo + threadIdx.x; k < hi; k += blockDim.x) {
        const double ax = h1[2 * k], ay = h1[2 * k + 1];
        v[0] += 1.0;
        v[1] += ax;
        v[2] += ax * ax + ay * ay;
        v[4] += ay;
        if (h2) {
            const double bx = h2[2 * k], by = h2[2 * k + 1];
            v[3] += ax * bx + ay * by;   // Re(conj(h1) h2)
            v[5] += ax * by - ay * bx;   // Im(conj(h1) h2)
            v[6] += bx * bx + by * by;   // |h2|^2
        }
    }
    block_sum<kMomentSums>(v, sh);
    if (threadIdx.x == 0)
        for (int q = 0; q < kMomentSums; ++q) partial[blockIdx.x * kMomentSums + q] = v[q];
}

// Checked mode of the boundary: the first configuration (lowest index) that is
// not in the Sz = 0 sector (popcount != N/2) or has bits set past site N - 1;
// first_bad must hold UINT64_MAX on entry and keeps it if all are valid.
__global__ void k_check_sz0(const uint64_t *__restrict__ cfg, int64_t n, int nwords, int N,
                            unsigned long long *__restrict__ first_bad)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        int pc = 0;
        bool stray = false;
        for (int w = 0; w < nwords; ++w) {
            const uint64_t x = cfg[k * nwords + w];
            pc += __popcll(x);
            const int lo = 64 * w, valid = N - lo < 64 ? N - lo : 64;   // sites of this word
            if (valid < 64 && (x >> valid) != 0ull) stray = true;
        }
        if (stray || 2 * pc != N) atomicMin(first_bad, (unsigned long long)k);
    }
}

cudaError_t launch_check_sz0(const uint64_t *cfg, int64_t n, int nwords, int N, unsigned long long *first_bad,
                             cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(first_bad, 0xff, sizeof(unsigned long long), st);
    if (e != cudaSuccess || n <= 0) return e;
    const int64_t want = (n + kRedThreads - 1) / kRedThreads;
    const int grid = (int)(want < 1024 ? want : 1024);
    k_check_sz0<<<grid, kRedThreads, 0, st>>>(cfg, n, nwords, N, first_bad);
    return cudaGetLastError();
}

// Configurations whose projected amplitude vanishes identically (Eqs. 4-6): s is
// fixed by an operation g with chi(g) = -1 (T_g s = s), or mapped to -s by g
// where the inverted term's character is -1 (chi_P chi(g) with spin inversion;
// chi(g) for bias-free RBMs without inversion, which are even in s).  Then
// psi(s) = -psi(s) = 0 exactly, whatever the rounding of the sum.  One warp per
// configuration, lanes over g.  mode 0: o1[k] = log psi = (-inf, 0); mode 1
// (E_loc, h1, h2 = 0/0): o1[k], o2[k] = NaN and NNQS_ERANGE in the status word.
template <typename T>
__global__ void k_mark_vanishing(DevModel<T> md, const uint64_t *__restrict__ cfg, int64_t n, int mode,
                                 double *__restrict__ o1, double *__restrict__ o2)
{
    const int lane = threadIdx.x & 31;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int inv_char = md.nsign == 2 ? md.chiP : (md.use_bias ? 0 : 1);
    for (int64_t k = wid; k < n; k += nw) {
        const uint64_t *w = cfg + k * md.nwords;
        bool dead = false;
        for (int g = lane; g < md.G && !dead; g += 32) {
            const T chi = md.chi[g];
            bool fix = chi < T(0), flip = (double)inv_char * (double)chi < 0.0;
            const uint8_t *pg = md.perm + (size_t)g * md.N;
            for (int i = 0; i < md.N && (fix || flip); ++i) {
                const int a = spin_of(w, i), b = spin_of(w, pg[i]);
                if (a != b) fix = false;
                if (a != -b) flip = false;
            }
            dead = fix || flip;
        }
        if (__any_sync(0xffffffffu, dead) && lane == 0) {
            if (mode == 0) {
                o1[2 * k] = -INFINITY;
                o1[2 * k + 1] = 0.0;
            } else {
                flag_range(md.status);
                if (o1) { o1[2 * k] = nan(""); o1[2 * k + 1] = nan(""); }
                if (o2) { o2[2 * k] = nan(""); o2[2 * k + 1] = nan(""); }
            }
        }
    }
}

template <typename T>
cudaError_t launch_mark_vanishing(const DevModel<T> &md, const uint64_t *cfg, int64_t n, int mode, double *o1,
                                  double *o2, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int64_t want = (n + 7) / 8;
    const int grid = (int)(want < 2048 ? want : 2048);
    k_mark_vanishing<T><<<grid, 256, 0, st>>>(md, cfg, n, mode, o1, o2);
    return cudaGetLastError();
}
template cudaError_t launch_mark_vanishing<float>(const DevModel<float> &, const uint64_t *, int64_t, int, double *,
                                                  double *, cudaStream_t);
template cudaError_t launch_mark_vanishing<double>(const DevModel<double> &, const uint64_t *, int64_t, int,
                                                   double *, double *, cudaStream_t);

// stage 2: fixed-order sum of the partials (raw sums to sums_out), moments and
// the p = 1 Lanczos step; with nb = 1 and partial = the all-reduced raw sums of
// several processes it is the finishing step of a distributed Lanczos step
__global__ void __launch_bounds__(32) k_moments_final(const double *__restrict__ partial, int nb,
                                                      double *__restrict__ sums_out, double *__restrict__ moments,
                                                      double *__restrict__ lanczos)
{
    if (threadIdx.x != 0) return;
    double v[kMomentSums] = {0, 0, 0, 0, 0, 0, 0};
    for (int b = 0; b < nb; ++b)
        for (int q = 0; q < kMomentSums; ++q) v[q] += partial[b * kMomentSums + q];
    if (sums_out)
        for (int q = 0; q < kMomentSums; ++q) sums_out[q] = v[q];
    const double z = v[0] > 0 ? v[0] : 1.0;
    const double m1 = v[1] / z, m2 = v[2] / z, m3 = v[3] / z;
    if (moments) {
        moments[0] = 1.0; moments[1] = m1; moments[2] = m2; moments[3] = m3;
        moments[4] = v[0]; moments[5] = v[4] / z; moments[6] = v[5] / z; moments[7] = v[6] / z;
    }
    if (lanczos) lanczos_p1(m1, m2, m3, lanczos);
}

cudaError_t launch_moments(const double *h1, const double *h2, int64_t n, double *partial, int nblocks,
                           double *moments, double *lanczos, cudaStream_t st, double *sums_out)
{
    k_moments_partial<<<nblocks, kRedThreads, 0, st>>>(h1, h2, n, partial);
    k_moments_final<<<1, 32, 0, st>>>(partial, nblocks, sums_out, moments, lanczos);
    return cudaGetLastError();
}

cudaError_t launch_moments_finish(const double *sums, double *moments, double *lanczos, cudaStream_t st)
{
    k_moments_final<<<1, 32, 0, st>>>(sums, 1, nullptr, moments, lanczos);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(32) k_eloc_final(const double *__restrict__ partial, int nb, double *__restrict__ sums)
{
    if (threadIdx.x != 0) return;
    double v[kMomentSums] = {0, 0, 0, 0, 0, 0, 0};
    for (int b = 0; b < nb; ++b)
        for (int q = 0; q < kMomentSums; ++q) v[q] += partial[b * kMomentSums + q];
    sums[0] = v[1]; sums[1] = v[4]; sums[2] = v[2]; sums[3] = v[0];
}

cudaError_t launch_eloc_sums(const double *eloc, int64_t n, double *partial, int nblocks, double *sums, cudaStream_t st)
{
    k_moments_partial<<<nblocks, kRedThreads, 0, st>>>(eloc, nullptr, n, partial);
    k_eloc_final<<<1, 32, 0, st>>>(partial, nblocks, sums);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// parameter-derived tables (computed in FP64, stored in T)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_tables(const double *__restrict__ par, int N, int M, int K, cx<T> *Wt, cx<T> *b, cx<T> *a, cx<T> *logc,
                         cx2<T> *X, cx2<T> *XA)
{
    const int64_t P1 = 1 + N + M + (int64_t)M * N;
    const int64_t tot = (int64_t)K * P1;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < tot; q += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(q / P1);
        const int64_t o = q - r * P1;
        const double vx = par[2 * q], vy = par[2 * q + 1];
        if (o == 0) {
            logc[r] = cx<T>{(T)vx, (T)vy};
        } else if (o < 1 + N) {
            const int k = (int)(o - 1);
            a[(size_t)r * N + k] = cx<T>{(T)vx, (T)vy};
            double s, c;
            sincos(2.0 * vy, &s, &c);
            const double em = exp(-2.0 * vx), ep = exp(2.0 * vx);
            XA[(size_t)r * N + k] = cx2<T>{cx<T>{(T)(em * c), (T)(-em * s)}, cx<T>{(T)(ep * c), (T)(ep * s)}};
        } else if (o < 1 + N + M) {
            b[(size_t)r * M + (o - 1 - N)] = cx<T>{(T)vx, (T)vy};
        } else {
            const int64_t wq = o - 1 - N - M;
            const int m = (int)(wq / N), k = (int)(wq - (int64_t)m * N);
            const size_t t = ((size_t)r * N + k) * M + m;
            Wt[t] = cx<T>{(T)vx, (T)vy};
            double s, c;
            sincos(2.0 * vy, &s, &c);
            const double em = exp(-2.0 * vx), ep = exp(2.0 * vx);
            X[t] = cx2<T>{cx<T>{(T)(em * c), (T)(-em * s)}, cx<T>{(T)(ep * c), (T)(ep * s)}};
        }
    }
}

// e^{z} - 1 without cancellation for small z
__device__ __forceinline__ void cexpm1(double x, double y, double &re, double &im)
{
    double sy, cy;
    sincos(y, &sy, &cy);
    const double sh = sin(0.5 * y);
    re = expm1(x) * cy - 2.0 * sh * sh;
    im = exp(x) * sy;
}

// exp(z) as a scaled number: mantissa * 2^e with |mantissa| in [1, 2)
template <typename T> __device__ __forceinline__ sc<T> exp_scaled(double x, double y)
{
    const double t = x * 1.4426950408889634;
    const double k = floor(t);
    const double m = exp2(t - k);
    double s, c;
    sincos(y, &s, &c);
    return sc<T>{(T)(m * c), (T)(m * s), (int)k};
}

template <typename T>
__global__ void k_tables_conn(const double *__restrict__ par, int N, int M, int Mp, int K, int nb, int use_bias,
                              const int16_t *__restrict__ bi, const int16_t *__restrict__ bj, cx<T> *Tb, cx<T> *Cb,
                              cx<T> *S4, cx<T> *CS, sc<T> *ES)
{
    const int64_t P1 = 1 + N + M + (int64_t)M * N;
    const int64_t n1 = (int64_t)K * nb * Mp, n2 = (int64_t)K * N * Mp, n3 = (int64_t)K * nb, n4 = (int64_t)K * N;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n1 + n2 + n3 + n4;
         q += (int64_t)gridDim.x * blockDim.x) {
        if (q < n1) {
            const int r = (int)(q / ((int64_t)nb * Mp));
            const int64_t rem = q - (int64_t)r * nb * Mp;
            const int b = (int)(rem / Mp), m = (int)(rem - (int64_t)b * Mp);
            double px = 0, py = 0, mx = 0, my = 0;  // padding: T = 0
            if (m < M) {
                const double *W = par + 2 * (r * P1 + 1 + N + M + (int64_t)m * N);
                const int a = bi[b], c = bj[b];
                const double zx = -4.0 * (W[2 * a] - W[2 * c]), zy = -4.0 * (W[2 * a + 1] - W[2 * c + 1]);
                cexpm1(zx, zy, px, py);
                cexpm1(-zx, -zy, mx, my);
            }
            Tb[(((size_t)r * 2 + 0) * nb + b) * Mp + m] = cx<T>{(T)px, (T)py};
            Tb[(((size_t)r * 2 + 1) * nb + b) * Mp + m] = cx<T>{(T)mx, (T)my};
        } else if (q < n1 + n2) {
            const int64_t u = q - n1;
            const int r = (int)(u / ((int64_t)N * Mp));
            const int64_t rem = u - (int64_t)r * N * Mp;
            const int k = (int)(rem / Mp), m = (int)(rem - (int64_t)k * Mp);
            double s = 0, c = 1, em = 1, ep = 1;  // padding: exp(+-4W) = 1
            if (m < M) {
                const double *W = par + 2 * (r * P1 + 1 + N + M + (int64_t)m * N + k);
                sincos(4.0 * W[1], &s, &c);
                em = exp(-4.0 * W[0]);
                ep = exp(4.0 * W[0]);
            }
            S4[(((size_t)r * 2 + 0) * N + k) * Mp + m] = cx<T>{(T)(em * c), (T)(-em * s)};
            S4[(((size_t)r * 2 + 1) * N + k) * Mp + m] = cx<T>{(T)(ep * c), (T)(ep * s)};
        } else if (q < n1 + n2 + n3) {
            const int64_t u = q - n1 - n2;
            const int r = (int)(u / nb), b = (int)(u - (int64_t)r * nb);
            const double *base = par + 2 * r * P1;
            const int a = bi[b], c = bj[b];
            double sx = 0, sy = 0;
            for (int m = 0; m < M; ++m) {
                const double *W = base + 2 * (1 + N + M + (int64_t)m * N);
                sx += W[2 * a] - W[2 * c];
                sy += W[2 * a + 1] - W[2 * c + 1];
            }
            double cx_ = 2.0 * sx, cy_ = 2.0 * sy;
            if (use_bias) {
                cx_ -= 2.0 * (base[2 * (1 + a)] - base[2 * (1 + c)]);
                cy_ -= 2.0 * (base[2 * (1 + a) + 1] - base[2 * (1 + c) + 1]);
            }
            Cb[(size_t)r * nb + b] = cx<T>{(T)cx_, (T)cy_};
        } else {
            const int64_t u = q - n1 - n2 - n3;
            const int r = (int)(u / N), k = (int)(u - (int64_t)r * N);
            const double *base = par + 2 * r * P1;
            double sx = 0, sy = 0;
            for (int m = 0; m < M; ++m) {
                const double *W = base + 2 * (1 + N + M + (int64_t)m * N + k);
                sx += W[0];
                sy += W[1];
            }
            CS[(size_t)r * N + k] = cx<T>{(T)sx, (T)sy};
            // site prefactor exponent Cs_k = 2 sum_m W_mk - 2 a_k
            double cx_ = 2.0 * sx, cy_ = 2.0 * sy;
            if (use_bias) {
                cx_ -= 2.0 * base[2 * (1 + k)];
                cy_ -= 2.0 * base[2 * (1 + k) + 1];
            }
            ES[((size_t)r * 2 + 0) * N + k] = exp_scaled<T>(cx_, cy_);
            ES[((size_t)r * 2 + 1) * N + k] = exp_scaled<T>(-cx_, -cy_);
        }
    }
}

template <typename T>
cudaError_t launch_tables_conn(const double *params, int N, int M, int Mp, int K, int nb, int use_bias,
                               const int16_t *bi, const int16_t *bj, cx<T> *Tb, cx<T> *Cb, cx<T> *S4, cx<T> *CS,
                               sc<T> *ES, cudaStream_t st)
{
    k_tables_conn<T><<<2048, 256, 0, st>>>(params, N, M, Mp, K, nb, use_bias, bi, bj, Tb, Cb, S4, CS, ES);
    return cudaGetLastError();
}

template cudaError_t launch_tables_conn<float>(const double *, int, int, int, int, int, int, const int16_t *, const int16_t *, cx<float> *, cx<float> *, cx<float> *, cx<float> *, sc<float> *, cudaStream_t);
template cudaError_t launch_tables_conn<double>(const double *, int, int, int, int, int, int, const int16_t *, const int16_t *, cx<double> *, cx<double> *, cx<double> *, cx<double> *, sc<double> *, cudaStream_t);

template <typename T>
cudaError_t launch_build_tables(const double *params, int N, int M, int K, cx<T> *Wt, cx<T> *b, cx<T> *a, cx<T> *logc,
                                cx2<T> *X, cx2<T> *XA, cudaStream_t st)
{
    k_tables<T><<<1024, 256, 0, st>>>(params, N, M, K, Wt, b, a, logc, X, XA);
    return cudaGetLastError();
}

template cudaError_t launch_build_tables<float>(const double *, int, int, int, cx<float> *, cx<float> *, cx<float> *, cx<float> *, cx2<float> *, cx2<float> *, cudaStream_t);
template cudaError_t launch_build_tables<double>(const double *, int, int, int, cx<double> *, cx<double> *, cx<double> *, cx<double> *, cx2<double> *, cx2<double> *, cudaStream_t);

}  // namespace nnqs
