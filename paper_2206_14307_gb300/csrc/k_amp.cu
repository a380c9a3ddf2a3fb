// k_amp.cu -- log psi of fresh configurations (Eqs. 2-6), SIMT form.
//
// Layout of the work: one CTA per sample (grid-stride over samples), one warp
// per row (r, g) of the projected sum (Eqs. 4-6), lanes over hidden units m.
// Each row computes theta'_m = sum_i W_r[m][g(i)] s_i once and serves both
// spin-inversion signs.  Amplitudes are kept as scaled complex numbers
// (mantissa * 2^e) so that log psi keeps its absolute accuracy.
#include "common.cuh"
#include "kernels.h"

namespace nnqs {

template <typename T, int MPL>
__device__ __forceinline__ void row_theta(const DevModel<T> &md, int r, int g, const T *s_sm, cx<T> (&th)[MPL],
                                          int lane)
{
#pragma unroll
    for (int j = 0; j < MPL; ++j) th[j] = cx<T>{T(0), T(0)};
    const uint8_t *pg = md.perm + (size_t)g * md.N;
    const cx<T> *Wr = md.Wt + (size_t)r * md.N * md.M;
    for (int i = 0; i < md.N; ++i) {
        const int k = __ldg(pg + i);
        const T si = s_sm[i];
        const cx<T> *wk = Wr + (size_t)k * md.M;
#pragma unroll
        for (int j = 0; j < MPL; ++j) {
            const int m = lane + 32 * j;
            if (m < md.M) {
                cx<T> w = wk[m];
                th[j].x += si * w.x;
                th[j].y += si * w.y;
            }
        }
    }
}

// a_r . T_g s (warp-reduced; all lanes receive it)
template <typename T>
__device__ __forceinline__ cx<T> row_visible(const DevModel<T> &md, int r, int g, const T *s_sm, int lane)
{
    cx<T> acc{T(0), T(0)};
    if (!md.use_bias) return acc;
    const uint8_t *pg = md.perm + (size_t)g * md.N;
    const cx<T> *ar = md.avec + (size_t)r * md.N;
    for (int i = lane; i < md.N; i += 32) {
        cx<T> a = ar[pg[i]];
        acc.x += s_sm[i] * a.x;
        acc.y += s_sm[i] * a.y;
    }
    return warp_sum(acc);
}

// Leading factor c_r chi(g) chi_P^{[sign<0]} exp(sign * a.T_g s) of one term.
template <typename T>
__device__ __forceinline__ sc<T> row_lead(const DevModel<T> &md, int r, int g, int sign, cx<T> at)
{
    cx<T> lc = md.logc[r];
    sc<T> v = sc_exp(cx<T>{lc.x + sign * at.x, lc.y + sign * at.y});
    T c = md.chi[g];
    if (sign < 0 && md.chiP < 0) c = -c;
    v.x *= c;
    v.y *= c;
    return sc_norm(v);
}

// Product over hidden units of 2cosh(theta_m) for one sign, and p_m.
template <typename T, int MPL>
__device__ __forceinline__ sc<T> row_cosh(const DevModel<T> &md, int r, int sign, const cx<T> (&thp)[MPL],
                                          cx<T> (&p)[MPL], int lane)
{
    sc<T> prod{T(1), T(0), 0};
    const cx<T> *br = md.bvec + (size_t)r * md.M;
#pragma unroll
    for (int j = 0; j < MPL; ++j) {
        const int m = lane + 32 * j;
        if (m < md.M) {
            cx<T> th{sign * thp[j].x, sign * thp[j].y};
            if (md.use_bias) { cx<T> b = br[m]; th.x += b.x; th.y += b.y; }
            cx<T> mant;
            int k;
            cosh2_mant(th, mant, k);
            p[j] = cx<T>{T(0), T(0)};
            cx<T> q = cmul(mk(prod.x, prod.y), mant);
            prod = sc<T>{q.x, q.y, prod.e + k};
        } else {
            p[j] = cx<T>{T(0), T(0)};
        }
    }
    return warp_prod(prod);
}


template <typename T>
__device__ __forceinline__ void load_spins(const DevModel<T> &md, const uint64_t *cfg, int64_t smp, T *s_sm, int8_t *s8)
{
    const uint64_t *w = cfg + smp * md.nwords;
    for (int i = threadIdx.x; i < md.N; i += blockDim.x) {
        int s = spin_of(w, i);
        s_sm[i] = T(s);
        s8[i] = (int8_t)s;
    }
}

// ---------------------------------------------------------------------------
// log psi of fresh configurations
// ---------------------------------------------------------------------------
template <typename T, int MPL>
__global__ void __launch_bounds__(kThreads) k_log_psi(DevModel<T> md, const uint64_t *__restrict__ cfg, int64_t n,
                                                      double *__restrict__ out)
{
    __shared__ T s_sm[kMaxN];
    __shared__ int8_t s8[kMaxN];
    __shared__ sc<T> wacc[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rows = md.K * md.G;
    for (int64_t smp = blockIdx.x; smp < n; smp += gridDim.x) {
        load_spins(md, cfg, smp, s_sm, s8);
        __syncthreads();
        sc<T> acc{T(0), T(0), 0};
        for (int row = warp; row < rows; row += kWarps) {
            const int r = row / md.G, g = row - r * md.G;
            cx<T> thp[MPL], p[MPL];
            row_theta<T, MPL>(md, r, g, s_sm, thp, lane);
            cx<T> at = row_visible(md, r, g, s_sm, lane);
            for (int sg = 0; sg < md.nsign; ++sg) {
                const int sign = sg ? -1 : 1;
                sc<T> prod = row_cosh<T, MPL>(md, r, sign, thp, p, lane);
                acc = sc_add(acc, sc_mul(prod, row_lead(md, r, g, sign, at)));
            }
        }
        if (lane == 0) wacc[warp] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            sc<T> tot = wacc[0];
            for (int w = 1; w < kWarps; ++w) tot = sc_add(tot, wacc[w]);
            double re, im;
            if (!sc_finite(tot)) {
                flag_range(md.status);
                re = nan(""); im = nan("");
            } else if (sc_zero(tot)) {
                re = -INFINITY; im = 0.0;
            } else {
                double x = (double)tot.x, y = (double)tot.y;
                re = log(hypot(x, y)) + tot.e * 0.69314718055994530942;
                im = atan2(y, x);
            }
            out[2 * smp] = re;
            out[2 * smp + 1] = im;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
#define NNQS_MPL_DISPATCH(MPLV, ...)                                   \
    switch (mpl_slot(MPLV)) {                                           \
    case 1: { constexpr int MPL = 1; __VA_ARGS__; } break;              \
    case 2: { constexpr int MPL = 2; __VA_ARGS__; } break;              \
    case 3: { constexpr int MPL = 3; __VA_ARGS__; } break;              \
    case 4: { constexpr int MPL = 4; __VA_ARGS__; } break;              \
    case 6: { constexpr int MPL = 6; __VA_ARGS__; } break;              \
    case 8: { constexpr int MPL = 8; __VA_ARGS__; } break;              \
    case 13: { constexpr int MPL = 13; __VA_ARGS__; } break;            \
    default: { constexpr int MPL = 16; __VA_ARGS__; } break;            \
    }

int mpl_slot(int M)
{
    const int need = (M + 31) / 32;
    const int opts[] = {1, 2, 3, 4, 6, 8, 13, 16};
    for (int o : opts)
        if (o >= need) return o;
    return 16;
}

template <typename T>
cudaError_t launch_log_psi(const DevModel<T> &md, const uint64_t *cfg, int64_t n, double *out, int nsm,
                           cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    cudaError_t err = cudaSuccess;
    NNQS_MPL_DISPATCH(md.M, {
        int per = 0;
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_log_psi<T, MPL>, kThreads, 0);
        const int64_t grid = (int64_t)(per > 0 ? per : 1) * nsm;
        const int g = (int)(n < grid ? n : grid);
        if (err == cudaSuccess) k_log_psi<T, MPL><<<g, kThreads, 0, st>>>(md, cfg, n, out);
    });
    if (err != cudaSuccess) return err;
    return cudaGetLastError();
}

template cudaError_t launch_log_psi<float>(const DevModel<float> &, const uint64_t *, int64_t, double *, int, cudaStream_t);
template cudaError_t launch_log_psi<double>(const DevModel<double> &, const uint64_t *, int64_t, double *, int, cudaStream_t);

}  // namespace nnqs
