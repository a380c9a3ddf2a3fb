// k_lanczos2.cu -- the p = 2 Lanczos step (Sec. 3.3,
// |Psi_2> = (1 + beta_1 H + beta_2 H^2)|psi0>).
//
// h3 = (H^3 psi)(s)/psi(s) = diag(s) h2(s) + sum_b (J_b/2) R_b h2(s^b) over
// the anti-aligned bonds b of s, with R_b = psi(s^b)/psi(s).  The first-level
// neighbours s^b are expanded into a flat list (count, scan, fill); h2 at
// every neighbour comes from the Lanczos mode of the connected-configuration
// engine and R_b from log psi.  The moments about c = <Re h1> up to order 6
// give the 3x3 Krylov pencil, solved in FP64 by Cholesky and Jacobi.
#include "common.cuh"
#include "kernels.h"

namespace nnqs {

// number of anti-aligned bonds of every configuration
template <typename T>
__global__ void k_count_nb(DevModel<T> md, const uint64_t *__restrict__ cfg, int64_t n, int64_t *__restrict__ cnt)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t *w = cfg + k * md.nwords;
        int c = 0;
        for (int b = 0; b < md.nbonds; ++b) c += spin_of(w, md.bond_i[b]) != spin_of(w, md.bond_j[b]);
        cnt[k] = c;
    }
}

// exclusive prefix sum of cnt[0..n) into off[0..n] (off[n] = total), one block
__global__ void __launch_bounds__(1024) k_scan(const int64_t *__restrict__ cnt, int64_t n, int64_t *__restrict__ off)
{
    __shared__ int64_t part[1024];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < n; base += blockDim.x) {
        const int64_t k = base + threadIdx.x;
        part[threadIdx.x] = k < n ? cnt[k] : 0;
        __syncthreads();
        for (int o = 1; o < (int)blockDim.x; o <<= 1) {  // Hillis-Steele inclusive scan
            const int64_t v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
            __syncthreads();
            part[threadIdx.x] += v;
            __syncthreads();
        }
        if (k < n) off[k] = carry + part[threadIdx.x] - cnt[k];
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += part[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) off[n] = carry;
}

// the neighbours s^b of every configuration in bond order, with J_b / 2
template <typename T>
__global__ void k_fill_nb(DevModel<T> md, const uint64_t *__restrict__ cfg, int64_t n, const int64_t *__restrict__ off,
                          uint64_t *__restrict__ nb_cfg, double *__restrict__ nb_coef)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t *w = cfg + k * md.nwords;
        int64_t o = off[k];
        for (int b = 0; b < md.nbonds; ++b) {
            const int i = md.bond_i[b], j = md.bond_j[b];
            if (spin_of(w, i) == spin_of(w, j)) continue;
            uint64_t *dst = nb_cfg + o * md.nwords;
            for (int q = 0; q < md.nwords; ++q) dst[q] = w[q];
            dst[i >> 6] ^= 1ull << (i & 63);   // exchanging an anti-aligned pair flips both spins
            dst[j >> 6] ^= 1ull << (j & 63);
            nb_coef[o] = 0.5 * (double)bondJ(md, b);
            ++o;
        }
    }
}

// h3 = diag(s) h2(s) + sum_b (J_b/2) exp(log psi(s^b) - log psi(s)) h2(s^b)
template <typename T>
__global__ void k_h3(DevModel<T> md, const uint64_t *__restrict__ cfg, int64_t n, const int64_t *__restrict__ off,
                     const double *__restrict__ nb_coef, const double *__restrict__ lp, const double *__restrict__ lpn,
                     const double *__restrict__ h2, const double *__restrict__ h2n, double *__restrict__ h3)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t *w = cfg + k * md.nwords;
        double diag = 0.0;
        for (int b = 0; b < md.nbonds; ++b)
            diag += 0.25 * (double)bondJ(md, b) * spin_of(w, md.bond_i[b]) * spin_of(w, md.bond_j[b]);
        double ax = diag * h2[2 * k], ay = diag * h2[2 * k + 1];
        for (int64_t q = off[k]; q < off[k + 1]; ++q) {
            const double dr = lpn[2 * q] - lp[2 * k], di = lpn[2 * q + 1] - lp[2 * k + 1];
            double s, c;
            sincos(di, &s, &c);
            const double m = nb_coef[q] * exp(dr);
            const double rx = m * c, ry = m * s;
            ax += rx * h2n[2 * q] - ry * h2n[2 * q + 1];
            ay += rx * h2n[2 * q + 1] + ry * h2n[2 * q];
        }
        h3[2 * k] = ax;
        h3[2 * k + 1] = ay;
    }
}

template <typename T>
cudaError_t launch_expand_nb(const DevModel<T> &md, const uint64_t *cfg, int64_t n, int64_t *cnt, int64_t *off,
                             cudaStream_t st)
{
    const int grid = (int)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
    k_count_nb<T><<<grid, 256, 0, st>>>(md, cfg, n, cnt);
    k_scan<<<1, 1024, 0, st>>>(cnt, n, off);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fill_nb(const DevModel<T> &md, const uint64_t *cfg, int64_t n, const int64_t *off,
                           uint64_t *nb_cfg, double *nb_coef, cudaStream_t st)
{
    const int grid = (int)((n + 127) / 128 < 1024 ? (n + 127) / 128 : 1024);
    k_fill_nb<T><<<grid, 128, 0, st>>>(md, cfg, n, off, nb_cfg, nb_coef);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_h3(const DevModel<T> &md, const uint64_t *cfg, int64_t n, const int64_t *off,
                      const double *nb_coef, const double *lp, const double *lpn, const double *h2,
                      const double *h2n, double *h3, cudaStream_t st)
{
    const int grid = (int)((n + 127) / 128 < 1024 ? (n + 127) / 128 : 1024);
    k_h3<T><<<grid, 128, 0, st>>>(md, cfg, n, off, nb_coef, lp, lpn, h2, h2n, h3);
    return cudaGetLastError();
}

// ---- moments about c (read from c_ptr) up to order 6 -------------------------
constexpr int kShiftSums = 8;  // n, Re a1, |a1|^2, Re(a1* a2), |a2|^2, Re(a2* a3), |a3|^2, n

__global__ void __launch_bounds__(256) k_shifted_partial(const double *__restrict__ h1, const double *__restrict__ h2,
                                                         const double *__restrict__ h3, int64_t n,
                                                         const double *__restrict__ c_ptr,
                                                         double *__restrict__ partial)
{
    __shared__ double sh[8][kShiftSums];
    const double c = *c_ptr;
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t lo = per * blockIdx.x, hi = lo + per < n ? lo + per : n;
    double v[kShiftSums] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t k = lo + threadIdx.x; k < hi; k += blockDim.x) {
        const double x1r = h1[2 * k], x1i = h1[2 * k + 1];
        const double x2r = h2[2 * k], x2i = h2[2 * k + 1];
        const double x3r = h3[2 * k], x3i = h3[2 * k + 1];
        // a_i = ((H - c)^i psi)(s)/psi(s)
        const double a1r = x1r - c, a1i = x1i;
        const double a2r = x2r - 2.0 * c * x1r + c * c, a2i = x2i - 2.0 * c * x1i;
        const double a3r = x3r - 3.0 * c * x2r + 3.0 * c * c * x1r - c * c * c;
        const double a3i = x3i - 3.0 * c * x2i + 3.0 * c * c * x1i;
        v[0] += 1.0;
        v[1] += a1r;
        v[2] += a1r * a1r + a1i * a1i;
        v[3] += a1r * a2r + a1i * a2i;
        v[4] += a2r * a2r + a2i * a2i;
        v[5] += a2r * a3r + a2i * a3i;
        v[6] += a3r * a3r + a3i * a3i;
        v[7] += 1.0;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kShiftSums; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    if (lane == 0)
        for (int q = 0; q < kShiftSums; ++q) sh[warp][q] = v[q];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int q = 0; q < kShiftSums; ++q) {
            double t = 0;
            for (int w = 0; w < 8; ++w) t += sh[w][q];
            partial[blockIdx.x * kShiftSums + q] = t;
        }
}

// Fixed-order sum of the partials -> mu_0..mu_6 and c; then the 3x3 pencil
// A_ij = mu_{i+j+1}, B_ij = mu_{i+j}: B = L L^T, C = L^{-1} A L^{-T}, cyclic
// Jacobi rotations on C, x = L^{-T} y of the lowest eigenvalue lambda (x0 = 1).
// out = {E_p2 = c + lambda, x0, x1, x2, var_p2}.
__global__ void k_krylov2(const double *__restrict__ partial, int nb, const double *__restrict__ c_ptr,
                          double *__restrict__ mu_out, double *__restrict__ out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s[kShiftSums] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = 0; b < nb; ++b)
        for (int q = 0; q < kShiftSums; ++q) s[q] += partial[b * kShiftSums + q];
    const double z = s[0] > 0 ? s[0] : 1.0;
    double mu[7];
    mu[0] = 1.0;
    for (int q = 1; q < 7; ++q) mu[q] = s[q] / z;
    const double c = *c_ptr;
    if (mu_out) {
        for (int q = 0; q < 7; ++q) mu_out[q] = mu[q];
        mu_out[7] = c;
    }
    if (!out) return;
    double A[3][3], B[3][3], Lm[3][3], Li[3][3], T[3][3], C[3][3], V[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            A[i][j] = mu[i + j + 1];
            B[i][j] = mu[i + j];
            Lm[i][j] = 0.0;
            Li[i][j] = 0.0;
            V[i][j] = i == j ? 1.0 : 0.0;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j <= i; ++j) {
            double t = B[i][j];
            for (int k = 0; k < j; ++k) t -= Lm[i][k] * Lm[j][k];
            Lm[i][j] = i == j ? sqrt(t > 0.0 ? t : 0.0) : t / Lm[j][j];
        }
    for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) {
            double t = i == j ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) t -= Lm[i][k] * Li[k][j];
            Li[i][j] = t / Lm[i][i];
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double t = 0.0;
            for (int k = 0; k < 3; ++k) t += Li[i][k] * A[k][j];
            T[i][j] = t;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double t = 0.0;
            for (int k = 0; k < 3; ++k) t += T[i][k] * Li[j][k];
            C[i][j] = t;
        }
    for (int sweep = 0; sweep < 50; ++sweep) {
        if (fabs(C[0][1]) + fabs(C[0][2]) + fabs(C[1][2]) < 1e-300) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (C[p][q] == 0.0) continue;
                const double th = (C[q][q] - C[p][p]) / (2.0 * C[p][q]);
                const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                const double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
                for (int k = 0; k < 3; ++k) {
                    const double ckp = C[k][p], ckq = C[k][q];
                    C[k][p] = cs * ckp - sn * ckq;
                    C[k][q] = sn * ckp + cs * ckq;
                }
                for (int k = 0; k < 3; ++k) {
                    const double cpk = C[p][k], cqk = C[q][k];
                    C[p][k] = cs * cpk - sn * cqk;
                    C[q][k] = sn * cpk + cs * cqk;
                }
                for (int k = 0; k < 3; ++k) {
                    const double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = cs * vkp - sn * vkq;
                    V[k][q] = sn * vkp + cs * vkq;
                }
            }
    }
    int lo = 0;
    for (int i = 1; i < 3; ++i)
        if (C[i][i] < C[lo][lo]) lo = i;
    const double lam = C[lo][lo];
    double x[3];
    for (int i = 0; i < 3; ++i) {
        double t = 0.0;
        for (int k = 0; k < 3; ++k) t += Li[k][i] * V[k][lo];
        x[i] = t;
    }
    const double x0 = x[0];
    for (int i = 0; i < 3; ++i) x[i] /= x0;
    double n0 = 0.0, n2 = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            n0 += x[i] * x[j] * mu[i + j];
            n2 += x[i] * x[j] * mu[i + j + 2];
        }
    out[0] = c + lam;
    out[1] = x[0];
    out[2] = x[1];
    out[3] = x[2];
    out[4] = n2 / n0 - lam * lam;
}

cudaError_t launch_krylov2(const double *h1, const double *h2, const double *h3, int64_t n, const double *c_ptr,
                           double *partial, int nb, double *mu_out, double *out, cudaStream_t st)
{
    k_shifted_partial<<<nb, 256, 0, st>>>(h1, h2, h3, n, c_ptr, partial);
    k_krylov2<<<1, 32, 0, st>>>(partial, nb, c_ptr, mu_out, out);
    return cudaGetLastError();
}

#define NNQS_INST(T)                                                                                               \
    template cudaError_t launch_expand_nb<T>(const DevModel<T> &, const uint64_t *, int64_t, int64_t *, int64_t *,  \
                                             cudaStream_t);                                                        \
    template cudaError_t launch_fill_nb<T>(const DevModel<T> &, const uint64_t *, int64_t, const int64_t *,        \
                                           uint64_t *, double *, cudaStream_t);                                    \
    template cudaError_t launch_h3<T>(const DevModel<T> &, const uint64_t *, int64_t, const int64_t *,             \
                                      const double *, const double *, const double *, const double *,              \
                                      const double *, double *, cudaStream_t);
NNQS_INST(float)
NNQS_INST(double)
#undef NNQS_INST

}  // namespace nnqs
