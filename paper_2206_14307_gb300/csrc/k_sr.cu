// k_sr.cu -- stochastic reconfiguration pieces (Eq. 12), FP64 throughout.
//
//   F_k   = <conj(O_k) (E_loc - <E_loc>)>
//   S x   = <conj(O) (O x)> - <conj(O)> <O x>,    (S + lambda I) x
//   solve (S + lambda I) delta = -dtau F by conjugate gradients (Hermitian
//   positive definite for lambda > 0), matrix-free, with the CG scalars kept
//   in device memory so that a solve needs no host synchronisation; after
//   convergence (|r| <= tol |b|) the remaining iterations do nothing.
// Means are over samples with optional weights w_s (NULL: all 1).
#include "common.cuh"
#include "kernels.h"

namespace nnqs {

constexpr int kSrThreads = 256;
constexpr int kDotBlocks = 128;
constexpr int kSrChunksMax = 128;   // sample chunks of the two-pass S x product and of F
constexpr int kOvSplit = 16;        // blocks per sample of the O x product

// scratch layout (doubles)
//   [0, 16)          CG state: 0 rr, 1 pAp, 2 alpha, 3 beta, 4 |b|^2, 5 done, 6 iterations, 7 W, 8-9 mean
//   [16, 16+2*kDot)  partial sums
//   then z [n][2], r [P][2], p [P][2], Ap [P][2]
enum { S_RR = 0, S_PAP = 1, S_ALPHA = 2, S_BETA = 3, S_B2 = 4, S_DONE = 5, S_IT = 6, S_W = 7, S_MEAN = 8 };
constexpr int kStateDoubles = 16;

size_t sr_scratch_doubles(int64_t n, int64_t P)
{
    // state, dot partials, z [n][2], r, p, Ap [P][2], the matvec's state block,
    // the chunk partials [kSrChunks][P][2] of the S x product, the split
    // partials [n][kOvSplit][2] of O x and zeta [n][2]
    return kStateDoubles + 2 * kDotBlocks + 2 * (size_t)n + 6 * (size_t)P + 64 + (size_t)kSrChunksMax * 2 * (size_t)P +
           2 * (size_t)kOvSplit * (size_t)n + 2 * (size_t)n;
}

template <int NV>
__device__ __forceinline__ void blk_sum(double (&v)[NV], double (*sh)[NV])
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

// weighted mean of a complex vector and the weight total (one block, fixed order)
__global__ void __launch_bounds__(kSrThreads) k_wmean(const double *__restrict__ v, const double *__restrict__ w,
                                                      int64_t n, double *__restrict__ state)
{
    __shared__ double sh[kSrThreads / 32][3];
    double a[3] = {0, 0, 0};
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
        const double wk = w ? w[k] : 1.0;
        a[0] += wk * v[2 * k];
        a[1] += wk * v[2 * k + 1];
        a[2] += wk;
    }
    blk_sum<3>(a, sh);
    if (threadIdx.x == 0) {
        state[S_MEAN] = a[0] / a[2];
        state[S_MEAN + 1] = a[1] / a[2];
        state[S_W] = a[2];
    }
}

// Both F and S x are sums over samples of conj(O_sk) zeta_s with a per-sample
// coefficient zeta (F: w_s (e_s - ebar)/W; S x: w_s (z_s - zbar)/W, which
// folds the <conj O><O x> term in), i.e. 4 FP64 FMAs per complex element of O
// -- on GB300 (FP64 at 1/74 of FP32) that, not HBM, bounds a pass over O.
// Two passes over sample chunks: pass 1 (block (k tile, chunk c)) reads rows
// of O coalesced (16 B per k) into part[c][k], pass 2 adds the chunks in order
// (deterministic) and adds lambda x.
__global__ void __launch_bounds__(256) k_oz_part(const double *__restrict__ O, const double *__restrict__ zeta,
                                                 int64_t n, int64_t P, int64_t chunk, double *__restrict__ part,
                                                 const double *__restrict__ state)
{
    if (state && state[S_DONE] != 0.0) return;
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= P) return;
    const int64_t s0 = blockIdx.y * chunk, s1 = s0 + chunk < n ? s0 + chunk : n;
    double ax = 0, ay = 0, bx = 0, by = 0;
    int64_t s = s0;
    for (; s + 1 < s1; s += 2) {
        const double2 o0 = *reinterpret_cast<const double2 *>(O + (s * P + k) * 2);
        const double2 o1 = *reinterpret_cast<const double2 *>(O + ((s + 1) * P + k) * 2);
        const double2 z0 = *reinterpret_cast<const double2 *>(zeta + 2 * s);
        const double2 z1 = *reinterpret_cast<const double2 *>(zeta + 2 * s + 2);
        ax = fma(o0.x, z0.x, fma(o0.y, z0.y, ax));
        ay = fma(o0.x, z0.y, fma(-o0.y, z0.x, ay));
        bx = fma(o1.x, z1.x, fma(o1.y, z1.y, bx));
        by = fma(o1.x, z1.y, fma(-o1.y, z1.x, by));
    }
    if (s < s1) {
        const double2 o0 = *reinterpret_cast<const double2 *>(O + (s * P + k) * 2);
        const double2 z0 = *reinterpret_cast<const double2 *>(zeta + 2 * s);
        ax = fma(o0.x, z0.x, fma(o0.y, z0.y, ax));
        ay = fma(o0.x, z0.y, fma(-o0.y, z0.x, ay));
    }
    double *pp = part + ((int64_t)blockIdx.y * P + k) * 2;
    pp[0] = ax + bx;
    pp[1] = ay + by;
}

// y_k = sum_c part[c][k] (+ lambda x_k when x is given)
__global__ void k_oz_out(const double *__restrict__ part, int nch, const double *__restrict__ x, double lambda,
                         int64_t P, double *__restrict__ y, const double *__restrict__ state)
{
    if (state && state[S_DONE] != 0.0) return;
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= P) return;
    double ax = 0, ay = 0;
    for (int c = 0; c < nch; ++c) {
        ax += part[((int64_t)c * P + k) * 2];
        ay += part[((int64_t)c * P + k) * 2 + 1];
    }
    if (x) {
        ax += lambda * x[2 * k];
        ay += lambda * x[2 * k + 1];
    }
    y[2 * k] = ax;
    y[2 * k + 1] = ay;
}

// zeta_s = w_s (v_s - vbar) / W from a state block holding vbar and W
__global__ void k_zeta(const double *__restrict__ v, const double *__restrict__ w, int64_t n,
                       const double *__restrict__ vst, double *__restrict__ zeta, const double *__restrict__ state)
{
    if (state && state[S_DONE] != 0.0) return;
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    const double f = (w ? w[s] : 1.0) / vst[S_W];
    zeta[2 * s] = f * (v[2 * s] - vst[S_MEAN]);
    zeta[2 * s + 1] = f * (v[2 * s + 1] - vst[S_MEAN + 1]);
}

static int sr_nch(int64_t n, int64_t &chunk)
{
    chunk = (n + kSrChunksMax - 1) / kSrChunksMax;
    return (int)((n + chunk - 1) / chunk);
}

size_t egrad_scratch_doubles(int64_t n, int64_t P)
{
    int64_t chunk;
    const int nch = sr_nch(n, chunk);
    return kStateDoubles + 2 * (size_t)n + 2 * (size_t)nch * (size_t)P;
}

// F_k = (1/W) sum_s w_s conj(O_sk) (e_s - ebar)
cudaError_t launch_energy_grad(const double *O, const double *eloc, const double *w, int64_t n, int64_t P, double *F,
                               double *scratch, cudaStream_t st)
{
    int64_t chunk;
    const int nch = sr_nch(n, chunk);
    double *zeta = scratch + kStateDoubles;
    double *part = zeta + 2 * n;
    k_wmean<<<1, kSrThreads, 0, st>>>(eloc, w, n, scratch);
    k_zeta<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(eloc, w, n, scratch, zeta, nullptr);
    k_oz_part<<<dim3((unsigned)((P + 255) / 256), (unsigned)nch), 256, 0, st>>>(O, zeta, n, P, chunk, part, nullptr);
    k_oz_out<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(part, nch, nullptr, 0.0, P, F, nullptr);
    return cudaGetLastError();
}

// z_s = sum_k O_sk x_k: kOvSplit blocks per sample, each a contiguous slice of
// the row with two 16-byte loads in flight per thread; the partial sums go to
// zpart [n][kOvSplit] (added in order by k_zsum).  Skipped once the solve
// converged.
__global__ void __launch_bounds__(kSrThreads) k_ov(const double *__restrict__ O, const double *__restrict__ x, int64_t P,
                                                   double *__restrict__ zpart, const double *__restrict__ state)
{
    if (state && state[S_DONE] != 0.0) return;
    __shared__ double sh[kSrThreads / 32][2];
    const int64_t s = blockIdx.x / kOvSplit;
    const int sp = blockIdx.x % kOvSplit;
    const int64_t len = (P + kOvSplit - 1) / kOvSplit;
    const int64_t k0 = sp * len, k1 = k0 + len < P ? k0 + len : P;
    const double2 *Os = reinterpret_cast<const double2 *>(O) + s * P;
    const double2 *xv = reinterpret_cast<const double2 *>(x);
    double a[2] = {0, 0}, b0 = 0, b1 = 0;
    int64_t k = k0 + threadIdx.x;
    for (; k + kSrThreads < k1; k += 2 * kSrThreads) {
        const double2 o0 = Os[k], o1 = Os[k + kSrThreads];
        const double2 x0 = xv[k], x1 = xv[k + kSrThreads];
        a[0] += o0.x * x0.x - o0.y * x0.y;
        a[1] += o0.x * x0.y + o0.y * x0.x;
        b0 += o1.x * x1.x - o1.y * x1.y;
        b1 += o1.x * x1.y + o1.y * x1.x;
    }
    if (k < k1) {
        const double2 o0 = Os[k], x0 = xv[k];
        a[0] += o0.x * x0.x - o0.y * x0.y;
        a[1] += o0.x * x0.y + o0.y * x0.x;
    }
    a[0] += b0;
    a[1] += b1;
    blk_sum<2>(a, sh);
    if (threadIdx.x == 0) {
        zpart[(s * kOvSplit + sp) * 2] = a[0];
        zpart[(s * kOvSplit + sp) * 2 + 1] = a[1];
    }
}

// z_s from its split partials (in order), and the weighted mean of z (one block)
__global__ void __launch_bounds__(kSrThreads) k_zsum(const double *__restrict__ zpart, const double *__restrict__ w,
                                                     int64_t n, double *__restrict__ z, double *__restrict__ zst,
                                                     const double *__restrict__ state)
{
    if (state && state[S_DONE] != 0.0) return;
    __shared__ double sh[kSrThreads / 32][3];
    double a[3] = {0, 0, 0};
    for (int64_t s = threadIdx.x; s < n; s += blockDim.x) {
        double zx = 0, zy = 0;
        for (int q = 0; q < kOvSplit; ++q) {
            zx += zpart[(s * kOvSplit + q) * 2];
            zy += zpart[(s * kOvSplit + q) * 2 + 1];
        }
        z[2 * s] = zx;
        z[2 * s + 1] = zy;
        const double ws = w ? w[s] : 1.0;
        a[0] += ws * zx;
        a[1] += ws * zy;
        a[2] += ws;
    }
    blk_sum<3>(a, sh);
    if (threadIdx.x == 0) {
        zst[S_MEAN] = a[0] / a[2];
        zst[S_MEAN + 1] = a[1] / a[2];
        zst[S_W] = a[2];
    }
}

// (S + lambda) x: z = O x (k_ov, k_zsum: z and its weighted mean), zeta,
// then y = sum_s conj(O_s) zeta_s + lambda x
static void matvec(const double *O, const double *w, int64_t n, int64_t P, const double *x, double lambda, double *y,
                   double *z, double *zst, double *part, const double *state, cudaStream_t st)
{
    int64_t chunk;
    const int nch = sr_nch(n, chunk);
    double *zpart = part + (size_t)kSrChunksMax * 2 * (size_t)P;
    double *zeta = zpart + 2 * (size_t)kOvSplit * (size_t)n;
    k_ov<<<(unsigned)(n * kOvSplit), kSrThreads, 0, st>>>(O, x, P, zpart, state);
    k_zsum<<<1, kSrThreads, 0, st>>>(zpart, w, n, z, zst, state);
    k_zeta<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(z, w, n, zst, zeta, state);
    k_oz_part<<<dim3((unsigned)((P + 255) / 256), (unsigned)nch), 256, 0, st>>>(O, zeta, n, P, chunk, part, state);
    k_oz_out<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(part, nch, x, lambda, P, y, state);
}

cudaError_t launch_sr_matvec(const double *O, const double *w, int64_t n, int64_t P, const double *x, double lambda,
                             double *y, double *scratch, cudaStream_t st)
{
    double *zst = scratch;                                     // its own small state block
    double *z = scratch + kStateDoubles + 2 * kDotBlocks;
    double *part = z + 2 * n + 6 * P + 64;
    matvec(O, w, n, P, x, lambda, y, z, zst, part, nullptr, st);
    return cudaGetLastError();
}

// ---- conjugate gradients --------------------------------------------------
__global__ void __launch_bounds__(kSrThreads) k_dot_partial(const double *__restrict__ a, const double *__restrict__ b,
                                                            int64_t P, double *__restrict__ part)
{
    __shared__ double sh[kSrThreads / 32][1];
    double v[1] = {0};
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x)
        v[0] += a[2 * k] * b[2 * k] + a[2 * k + 1] * b[2 * k + 1];   // Re(conj(a) b)
    blk_sum<1>(v, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = v[0];
}

// mode 0: start (rr = |b|^2), 1: pAp -> alpha, 2: rr_new -> beta, convergence
__global__ void k_dot_final(const double *__restrict__ part, int nb, double *__restrict__ state, int mode, double tol)
{
    if (threadIdx.x != 0) return;
    double s = 0;
    for (int i = 0; i < nb; ++i) s += part[i];
    if (mode == 0) {
        state[S_RR] = s; state[S_B2] = s; state[S_IT] = 0; state[S_ALPHA] = 0; state[S_BETA] = 0;
        state[S_DONE] = (s == 0.0) ? 1.0 : 0.0;
    } else if (mode == 1) {
        state[S_PAP] = s;
        state[S_ALPHA] = (state[S_DONE] != 0.0 || s == 0.0) ? 0.0 : state[S_RR] / s;
    } else {
        if (state[S_DONE] != 0.0) return;
        state[S_BETA] = state[S_RR] > 0 ? s / state[S_RR] : 0.0;
        state[S_RR] = s;
        state[S_IT] += 1.0;
        if (sqrt(s) <= tol * sqrt(state[S_B2])) state[S_DONE] = 1.0;
    }
}

__global__ void k_cg_init(const double *__restrict__ F, double dtau, int64_t P, double *__restrict__ x,
                          double *__restrict__ r, double *__restrict__ p)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= P) return;
    const double bx = -dtau * F[2 * k], by = -dtau * F[2 * k + 1];
    x[2 * k] = 0; x[2 * k + 1] = 0;
    r[2 * k] = bx; r[2 * k + 1] = by;
    p[2 * k] = bx; p[2 * k + 1] = by;
}

__global__ void k_cg_update(int64_t P, double *__restrict__ x, double *__restrict__ r, const double *__restrict__ p,
                            const double *__restrict__ Ap, const double *__restrict__ state)
{
    if (state[S_DONE] != 0.0) return;
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= P) return;
    const double a = state[S_ALPHA];
    x[2 * k] += a * p[2 * k]; x[2 * k + 1] += a * p[2 * k + 1];
    r[2 * k] -= a * Ap[2 * k]; r[2 * k + 1] -= a * Ap[2 * k + 1];
}

__global__ void k_cg_dir(int64_t P, const double *__restrict__ r, double *__restrict__ p, const double *__restrict__ state)
{
    if (state[S_DONE] != 0.0) return;
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= P) return;
    const double b = state[S_BETA];
    p[2 * k] = r[2 * k] + b * p[2 * k];
    p[2 * k + 1] = r[2 * k + 1] + b * p[2 * k + 1];
}

__global__ void k_cg_finish(int64_t P, const double *__restrict__ x, double *__restrict__ params,
                            const double *__restrict__ state, double *__restrict__ info)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (params && k < P) { params[2 * k] += x[2 * k]; params[2 * k + 1] += x[2 * k + 1]; }
    if (info && k == 0) {
        info[0] = state[S_IT];
        info[1] = state[S_B2] > 0 ? sqrt(state[S_RR] / state[S_B2]) : 0.0;
    }
}

cudaError_t launch_sr_solve(const double *O, const double *w, int64_t n, int64_t P, const double *F, double lambda,
                            double dtau, int max_iter, double tol, double *x, double *info, double *params_inout,
                            double *scratch, cudaStream_t st)
{
    double *state = scratch;
    double *part = scratch + kStateDoubles;
    double *z = part + 2 * kDotBlocks;
    double *r = z + 2 * n, *p = r + 2 * P, *Ap = p + 2 * P;
    double *zst = Ap + 2 * P;   // state block of the matvec means (16 doubles)
    double *cpart = zst + 64;   // chunk partials of the S x product
    const unsigned gp = (unsigned)((P + 255) / 256);
    k_cg_init<<<gp, 256, 0, st>>>(F, dtau, P, x, r, p);
    k_dot_partial<<<kDotBlocks, kSrThreads, 0, st>>>(r, r, P, part);
    k_dot_final<<<1, 32, 0, st>>>(part, kDotBlocks, state, 0, tol);
    for (int it = 0; it < max_iter; ++it) {
        matvec(O, w, n, P, p, lambda, Ap, z, zst, cpart, state, st);
        k_dot_partial<<<kDotBlocks, kSrThreads, 0, st>>>(p, Ap, P, part);
        k_dot_final<<<1, 32, 0, st>>>(part, kDotBlocks, state, 1, tol);
        k_cg_update<<<gp, 256, 0, st>>>(P, x, r, p, Ap, state);
        k_dot_partial<<<kDotBlocks, kSrThreads, 0, st>>>(r, r, P, part);
        k_dot_final<<<1, 32, 0, st>>>(part, kDotBlocks, state, 2, tol);
        k_cg_dir<<<gp, 256, 0, st>>>(P, r, p, state);
    }
    k_cg_finish<<<gp, 256, 0, st>>>(P, x, params_inout, state, info);
    return cudaGetLastError();
}

}  // namespace nnqs
