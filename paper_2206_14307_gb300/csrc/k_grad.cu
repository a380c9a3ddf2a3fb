// k_grad.cu -- log-derivatives O_k = d log psi / d alpha_k (Sec. 3.2, after
// Eq. 12) of the projected sum of RBMs.
//
// With w_t = term_t / psi for the terms t = (r, g, sign) of Eqs. 4-6 and the
// transformed configuration u_t = sign * T_g s:
//   O[log c_r] = sum_{g,sign} w_t
//   O[a_r,k]   = sum_g A_rg (T_g s)_k,            A_rg = sum_sign sign w_t
//   O[b_r,m]   = sum_{g,sign} w_t tanh(theta_tm)
//   O[W_r,m,k] = sum_g U_rgm (T_g s)_k,           U_rgm = sum_sign sign w_t tanh(theta_tm)
// Phase 1 (one warp per row) writes A, C = sum_sign w and the U, V rows to a
// per-CTA scratch; phase 2 contracts them with the +-1 matrix T_g s held in
// shared memory.  tanh(theta) = 2p - 1 with p from the scaled 2cosh.
#include "common.cuh"
#include "kernels.h"

namespace nnqs {

constexpr int kGc = 16;   // rows g per staged chunk of the W-block GEMM

__host__ __device__ __forceinline__ size_t grad_tg_bytes(int G, int N) { return ((size_t)G * N + 15) & ~(size_t)15; }

// units a pass of the W-block GEMM covers (2 per thread slot)
template <typename T> __host__ __device__ __forceinline__ int grad_mpass(int N)
{
    return 2 * (kThreads / ((N + 7) / 8));
}

template <typename T> size_t grad_smem_bytes(const DevModel<T> &md)
{
    const int nkb = (md.N + 7) / 8;
    return grad_tg_bytes(md.G, md.N) + (size_t)kGc * grad_mpass<T>(md.N) * sizeof(cx<T>) +
           (size_t)kGc * nkb * 8 * sizeof(T);
}

template <typename T> size_t grad_scratch_bytes(const DevModel<T> &md)
{
    const size_t rows = (size_t)md.K * md.G;
    const size_t b = rows * md.M * sizeof(cx<T>) * 2 + rows * sizeof(cx<T>) * 2;
    return (b + 255) & ~(size_t)255;
}

template <typename T, int MPL>
__global__ void __launch_bounds__(kThreads, 2) k_grad(DevModel<T> md, const uint64_t *__restrict__ cfg, int64_t n,
                                                   double *__restrict__ O, unsigned char *__restrict__ scratch,
                                                   size_t scratch_stride, const float2 *__restrict__ th)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int8_t *tg = reinterpret_cast<int8_t *>(smem_raw);  // [G][N]  (T_g s)_k
    // staging of the W-block GEMM: kGc rows of U (4 units per thread slot) and
    // of T_g s as floats (sites padded to 8)
    cx<T> *us = reinterpret_cast<cx<T> *>(smem_raw + grad_tg_bytes(md.G, md.N));
    T *ts = reinterpret_cast<T *>(us + (size_t)kGc * grad_mpass<T>(md.N));
    __shared__ T s_sm[kMaxN];
    __shared__ int8_t s8[kMaxN];
    __shared__ sc<T> wacc[kWarps];
    __shared__ sc<T> S0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int N = md.N, M = md.M, G = md.G, K = md.K;
    const int rows = K * G;
    const int64_t P1 = 1 + N + M + (int64_t)M * N;
    cx<T> *U = reinterpret_cast<cx<T> *>(scratch + scratch_stride * blockIdx.x);  // [rows][M]
    cx<T> *V = U + (size_t)rows * M;                                              // [rows][M]
    cx<T> *A = V + (size_t)rows * M;                                              // [rows]
    cx<T> *C = A + rows;                                                          // [rows]

    for (int64_t smp = blockIdx.x; smp < n; smp += gridDim.x) {
        const uint64_t *w = cfg + smp * md.nwords;
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            const int s = spin_of(w, i);
            s_sm[i] = T(s);
            s8[i] = (int8_t)s;
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < G * N; idx += blockDim.x) {
            const int g = idx / N, i = idx - g * N;
            tg[g * N + md.perm[(size_t)g * N + i]] = s8[i];
        }
        // ---- pass A: psi ----
        sc<T> acc{T(0), T(0), 0};
        for (int pass = 0; pass < 2; ++pass) {
            for (int row = warp; row < rows; row += kWarps) {
                const int r = row / G, g = row - r * G;
                const uint8_t *pg = md.perm + (size_t)g * N;
                const cx<T> *Wr = md.Wt + (size_t)r * N * M;
                cx<T> thp[MPL];
#pragma unroll
                for (int j = 0; j < MPL; ++j) thp[j] = cx<T>{T(0), T(0)};
                if (th) {
                    // theta' of the row from the tensor cores
                    const float2 *tr = th + ((smp * K + r) * (int64_t)G + g) * M;
#pragma unroll
                    for (int j = 0; j < MPL; ++j) {
                        const int m = lane + 32 * j;
                        if (m < M) { const float2 v = tr[m]; thp[j] = cx<T>{T(v.x), T(v.y)}; }
                    }
                } else {
                    for (int i = 0; i < N; ++i) {
                        const cx<T> *wk = Wr + (size_t)pg[i] * M;
                        const T si = s_sm[i];
#pragma unroll
                        for (int j = 0; j < MPL; ++j) {
                            const int m = lane + 32 * j;
                            if (m < M) { const cx<T> ww = wk[m]; thp[j].x += si * ww.x; thp[j].y += si * ww.y; }
                        }
                    }
                }
                cx<T> at{T(0), T(0)};
                if (md.use_bias) {
                    const cx<T> *ar = md.avec + (size_t)r * N;
                    for (int i = lane; i < N; i += 32) { const cx<T> a = ar[pg[i]]; at.x += s_sm[i] * a.x; at.y += s_sm[i] * a.y; }
                    at = warp_sum(at);
                }
                // (U and V of the row are summed over the signs in the scratch
                // rows themselves: no per-unit accumulators stay live)
                cx<T> aacc{T(0), T(0)}, cacc{T(0), T(0)};
                cx<T> *Urow = U + (size_t)row * M, *Vrow = V + (size_t)row * M;
                for (int sg = 0; sg < md.nsign; ++sg) {
                    const int sign = sg ? -1 : 1;
                    cx<T> p[MPL];
                    sc<T> prod{T(1), T(0), 0};
                    const cx<T> *br = md.bvec + (size_t)r * M;
#pragma unroll
                    for (int j = 0; j < MPL; ++j) {
                        const int m = lane + 32 * j;
                        if (m < M) {
                            cx<T> th{sign * thp[j].x, sign * thp[j].y};
                            if (md.use_bias) { const cx<T> b = br[m]; th.x += b.x; th.y += b.y; }
                            cx<T> mant; int k;
                            cosh2(th, mant, k, p[j]);
                            const cx<T> q = cmul(mk(prod.x, prod.y), mant);
                            prod = sc<T>{q.x, q.y, prod.e + k};
                        } else {
                            p[j] = cx<T>{T(0), T(0)};
                        }
                    }
                    prod = warp_prod(prod);
                    const cx<T> lc = md.logc[r];
                    sc<T> lead = sc_exp(cx<T>{lc.x + sign * at.x, lc.y + sign * at.y});
                    T c = md.chi[g];
                    if (sign < 0 && md.chiP < 0) c = -c;
                    lead.x *= c; lead.y *= c;
                    const sc<T> term = sc_mul(prod, sc_norm(lead));
                    if (pass == 0) {
                        if (lane == 0) acc = sc_add(acc, term);
                    } else {
                        // w = term / psi
                        const sc<T> s0 = S0;
                        cx<T> wt{T(0), T(0)};
                        if (!sc_zero(term)) {
                            const cx<T> q = cdiv(mk(term.x, term.y), mk(s0.x, s0.y));
                            const T f = pow2i<T>(term.e - s0.e);
                            wt = cx<T>{q.x * f, q.y * f};
                        }
                        cacc = cadd(cacc, wt);
                        aacc = cadd(aacc, cscale(wt, T(sign)));
#pragma unroll
                        for (int j = 0; j < MPL; ++j) {
                            const int m = lane + 32 * j;
                            if (m < M) {
                                const cx<T> th = cx<T>{T(2) * p[j].x - T(1), T(2) * p[j].y};  // tanh
                                const cx<T> wth = cmul(wt, th);
                                const cx<T> uw = cscale(wth, T(sign));
                                if (sg == 0) {
                                    Urow[m] = uw;
                                    Vrow[m] = wth;
                                } else {
                                    Urow[m] = cadd(Urow[m], uw);
                                    Vrow[m] = cadd(Vrow[m], wth);
                                }
                            }
                        }
                    }
                }
                if (pass == 1 && lane == 0) { A[row] = aacc; C[row] = cacc; }
            }
            if (pass == 0) {
                if (lane == 0) wacc[warp] = acc;
                __syncthreads();
                if (threadIdx.x == 0) {
                    sc<T> tot = wacc[0];
                    for (int ww = 1; ww < kWarps; ++ww) tot = sc_add(tot, wacc[ww]);
                    S0 = tot;
                    if (!sc_finite(tot) || sc_zero(tot)) atomicExch(md.status, -6);
                }
            }
            __syncthreads();
        }
        // ---- phase 2: contractions with T_g s ----
        double *Os = O + (size_t)smp * K * P1 * 2;
        for (int r = 0; r < K; ++r) {
            double *Or = Os + (size_t)r * P1 * 2;
            const cx<T> *Ur = U + (size_t)r * G * M, *Vr = V + (size_t)r * G * M;
            const cx<T> *Ar = A + (size_t)r * G, *Cr = C + (size_t)r * G;
            if (warp == 0) {
                cx<T> c{T(0), T(0)};
                for (int g = lane; g < G; g += 32) c = cadd(c, Cr[g]);
                c = warp_sum(c);
                if (lane == 0) { Or[0] = (double)c.x; Or[1] = (double)c.y; }
            }
            for (int k = threadIdx.x; k < N; k += blockDim.x) {
                cx<T> a{T(0), T(0)};
                if (md.use_bias)
                    for (int g = 0; g < G; ++g) a = cadd(a, cscale(Ar[g], T(tg[g * N + k])));
                Or[2 * (1 + k)] = (double)a.x; Or[2 * (1 + k) + 1] = (double)a.y;
            }
            for (int m = threadIdx.x; m < M; m += blockDim.x) {
                cx<T> b{T(0), T(0)};
                if (md.use_bias)
                    for (int g = 0; g < G; ++g) b = cadd(b, Vr[(size_t)g * M + m]);
                Or[2 * (1 + N + m)] = (double)b.x; Or[2 * (1 + N + m) + 1] = (double)b.y;
            }
            // W block, O[W_r,m,k] = sum_g U_rgm (T_g s)_k: a register-tiled
            // GEMM over g.  Thread (mi, ki) owns TM = 2 units x 8 sites (within
            // the two-CTAs-per-SM register budget); a pass covers TM MI units,
            // and chunks of kGc rows of U and of T_g s (as +-1 values) are
            // staged in shared memory.
            {
                constexpr int TM = 2;
                const int nkb = (N + 7) / 8;
                const int MI = kThreads / nkb;
                const int mpass = grad_mpass<T>(N);   // TM MI
                const int mi = (int)threadIdx.x % MI, ki = (int)threadIdx.x / MI;
                const bool act = ki < nkb;
                for (int mp = 0; mp < M; mp += mpass) {
                    cx<T> o[TM][8];
#pragma unroll
                    for (int a = 0; a < TM; ++a)
#pragma unroll
                        for (int q = 0; q < 8; ++q) o[a][q] = cx<T>{T(0), T(0)};
                    for (int g0 = 0; g0 < G; g0 += kGc) {
                        const int gc = G - g0 < kGc ? G - g0 : kGc;
                        __syncthreads();
                        for (int q = threadIdx.x; q < kGc * mpass; q += blockDim.x) {
                            const int gg = q / mpass, mm = q - gg * mpass;
                            cx<T> u{T(0), T(0)};
                            if (gg < gc && mp + mm < M) u = Ur[(size_t)(g0 + gg) * M + mp + mm];
                            us[q] = u;
                        }
                        for (int q = threadIdx.x; q < kGc * nkb * 8; q += blockDim.x) {
                            const int gg = q / (nkb * 8), kk = q - gg * nkb * 8;
                            ts[q] = (gg < gc && kk < N) ? T(tg[(g0 + gg) * N + kk]) : T(0);
                        }
                        __syncthreads();
                        if (act) {
                            for (int gg = 0; gg < gc; ++gg) {
                                const cx<T> *ur = us + gg * mpass + TM * mi;
                                const T *tr = ts + gg * nkb * 8 + 8 * ki;
                                cx<T> u[TM];
                                T tv[8];
#pragma unroll
                                for (int a = 0; a < TM; ++a) u[a] = ur[a];
#pragma unroll
                                for (int q = 0; q < 8; ++q) tv[q] = tr[q];
#pragma unroll
                                for (int a = 0; a < TM; ++a)
#pragma unroll
                                    for (int q = 0; q < 8; ++q) {
                                        o[a][q].x += tv[q] * u[a].x;
                                        o[a][q].y += tv[q] * u[a].y;
                                    }
                            }
                        }
                    }
                    if (act) {
#pragma unroll
                        for (int a = 0; a < TM; ++a) {
                            const int m = mp + TM * mi + a;
                            if (m >= M) continue;
                            double *ow = Or + 2 * (1 + N + M + (size_t)m * N + 8 * ki);
#pragma unroll
                            for (int q = 0; q < 8; ++q)
                                if (8 * ki + q < N) { ow[2 * q] = (double)o[a][q].x; ow[2 * q + 1] = (double)o[a][q].y; }
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
}

template <typename T> int grad_grid(const DevModel<T> &md, int64_t n, int nsm)
{
    const int64_t g = (int64_t)2 * nsm;
    return (int)(n < g ? (n > 0 ? n : 1) : g);
}

template <typename T>
cudaError_t launch_grad(const DevModel<T> &md, const uint64_t *cfg, int64_t n, double *O, void *scratch, int grid,
                        cudaStream_t st, const float2 *th)
{
    if (n <= 0) return cudaSuccess;
    const int g = grid;
    const size_t smem = grad_smem_bytes(md);
    const size_t stride = grad_scratch_bytes(md);
    cudaError_t err = cudaSuccess;
    switch (mpl_slot(md.M)) {
#define NNQS_CASE(V)                                                                                              \
    case V:                                                                                                       \
        err = cudaFuncSetAttribute(k_grad<T, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);         \
        if (err == cudaSuccess) k_grad<T, V><<<g, kThreads, smem, st>>>(md, cfg, n, O, (unsigned char *)scratch, stride, th); \
        break;
        NNQS_CASE(1) NNQS_CASE(2) NNQS_CASE(3) NNQS_CASE(4) NNQS_CASE(6) NNQS_CASE(8) NNQS_CASE(13) NNQS_CASE(16)
#undef NNQS_CASE
    }
    if (err != cudaSuccess) return err;
    return cudaGetLastError();
}

template int grad_grid<float>(const DevModel<float> &, int64_t, int);
template int grad_grid<double>(const DevModel<double> &, int64_t, int);
template size_t grad_scratch_bytes<float>(const DevModel<float> &);
template size_t grad_scratch_bytes<double>(const DevModel<double> &);
template cudaError_t launch_grad<float>(const DevModel<float> &, const uint64_t *, int64_t, double *, void *, int, cudaStream_t, const float2 *);
template cudaError_t launch_grad<double>(const DevModel<double> &, const uint64_t *, int64_t, double *, void *, int, cudaStream_t, const float2 *);

}  // namespace nnqs
