// k_sample.cu -- persistent chain-parallel Metropolis sampler (Sec. 3.2).
//
// Persistent CTAs loop over Markov chains.  A chain keeps in device memory,
// for every row t = (r, g, sign) of the projected sum, its term
// c_r chi(g) chi_P phi_r(+-T_g s) and, per hidden unit, p = e^theta/(2cosh theta).
// A proposed exchange of an up site u and a down site d changes row t by
//   exp(sigma C_ud) prod_m (1 + p_m T_m),  T_m = exp(-4 sigma (W_m,g(u) - W_m,g(d))) - 1,
// with sigma = sign, C_ud the prefactor exponent from the column-sum tables;
// T_m is the product of two per-site table entries.  One pass per step
// computes the ratio and, speculatively, the updated cache
//   p' = p (1 + T) / (1 + p T),   term' = term * ratio
// into the chain's second buffer; an accepted step flips the buffer index.
// Only the active chains' caches are touched, so with one or two resident
// CTAs per SM they stay in L2.  Random numbers: Philox4x32-10 keyed by
// (seed, chain).
#include "common.cuh"
#include "kernels.h"

namespace nnqs {

constexpr int kSGL = 8;          // lanes per row group
constexpr int kSWarps = 16;      // warps per CTA (one chain per CTA at a time)
constexpr int kSThreads = 32 * kSWarps;

// Layout of one chain's cache: [p buffer 0][terms 0][p buffer 1][terms 1],
// every segment padded to 256 bytes so that each starts aligned.
__host__ __device__ __forceinline__ size_t pad256(size_t b) { return (b + 255) & ~(size_t)255; }
// Complex division for the speculative cache update, where the divisor
// f = 1 + p (e^{2 Delta} - 1) stays near 1: the reciprocal of |f|^2 from the
// hardware approximation refined by one Newton-Raphson step (r' = r + r(1 - x r)),
// within an ulp of the correctly rounded one.
__device__ __forceinline__ float rcp_nr(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return fmaf(r, fmaf(-x, r, 1.0f), r);
}
__device__ __forceinline__ double rcp_nr(double x) { return 1.0 / x; }
template <typename T> __device__ __forceinline__ cx<T> cdiv_upd(cx<T> a, cx<T> b)
{
    const T d = rcp_nr(b.x * b.x + b.y * b.y);
    return cx<T>{(a.x * b.x + a.y * b.y) * d, (a.y * b.x - a.x * b.y) * d};
}

template <typename T> __host__ __device__ size_t seg_p(int K, int G, int nsign, int M)
{
    return pad256((size_t)K * G * nsign * M * sizeof(cx<T>));
}
template <typename T> __host__ __device__ size_t seg_t(int K, int G, int nsign)
{
    return pad256((size_t)K * G * nsign * sizeof(sc<T>));
}
template <typename T> __host__ __device__ size_t chain_stride(int K, int G, int nsign, int M)
{
    return 2 * (seg_p<T>(K, G, nsign, M) + seg_t<T>(K, G, nsign));
}

template <typename T> size_t sampler_cache_bytes(const DevModel<T> &md)
{
    return chain_stride<T>(md.K, md.G, md.nsign, md.M);
}

template <typename T> int sampler_grid(const DevModel<T> &md, int n_chains, int nsm);

// k-th set bit (0-based) of a multi-word mask
__device__ __forceinline__ int kth_bit(const uint64_t *w, int nwords, int k)
{
    for (int q = 0; q < nwords; ++q) {
        const int c = __popcll(w[q]);
        if (k < c) {
            const uint32_t lo = (uint32_t)w[q], hi = (uint32_t)(w[q] >> 32);
            const int cl = __popc(lo);
            if (k < cl) return q * 64 + (int)__fns(lo, 0, k + 1);
            return q * 64 + 32 + (int)__fns(hi, 0, k - cl + 1);
        }
        k -= c;
    }
    return -1;
}

template <typename T, int MPL>
__global__ void __launch_bounds__(kSThreads, 1) k_sample(DevModel<T> md, uint64_t seed, int n_chains, int n_per_chain,
                                                     int n_skip, int n_burn, uint64_t *__restrict__ cfg_out,
                                                     float *__restrict__ acc_out, unsigned char *__restrict__ cache)
{
    constexpr int NG = 32 / kSGL;
    __shared__ T s_sm[kMaxN];
    __shared__ uint64_t upm[kMaxWords], dnm[kMaxWords];
    __shared__ sc<T> wold[kSWarps], wnew[kSWarps];
    __shared__ int site_u, site_d, accept, buf;
    __shared__ float u_sh;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane / kSGL, gl = lane % kSGL;
    const int N = md.N, M = md.M;
    const int rows = md.K * md.G;
    const int nrs = rows * md.nsign;
    const int slot = warp * NG + grp, nslots = kSWarps * NG;
    const size_t per_chain = chain_stride<T>(md.K, md.G, md.nsign, M);
    const size_t pbytes = seg_p<T>(md.K, md.G, md.nsign, M), tbytes = seg_t<T>(md.K, md.G, md.nsign);

    for (int chain = blockIdx.x; chain < n_chains; chain += gridDim.x) {
        unsigned char *base = cache + per_chain * chain;
        cx<T> *const pc0 = reinterpret_cast<cx<T> *>(base);
        cx<T> *const pc1 = reinterpret_cast<cx<T> *>(base + pbytes + tbytes);
        sc<T> *const tc0 = reinterpret_cast<sc<T> *>(base + pbytes);
        sc<T> *const tc1 = reinterpret_cast<sc<T> *>(base + 2 * pbytes + tbytes);
        const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32) ^ (uint32_t)chain;

        // ---- initial configuration: Fisher-Yates shuffle of N/2 ups ----
        if (threadIdx.x == 0) {
            int8_t s8[kMaxN];
            for (int i = 0; i < N; ++i) s8[i] = (int8_t)(i < N / 2 ? 1 : -1);
            u32x4 w{};
            for (int j = N - 1, q = 0; j >= 1; --j, ++q) {
                if ((q & 3) == 0) w = philox((uint32_t)(q >> 2), 1u, 0u, 0u, k0, k1);
                const uint32_t x = w.v[q & 3];
                const int r = (int)(((uint64_t)x * (uint64_t)(j + 1)) >> 32);
                const int8_t t = s8[j]; s8[j] = s8[r]; s8[r] = t;
            }
            for (int q = 0; q < md.nwords; ++q) { upm[q] = 0; dnm[q] = 0; }
            for (int i = 0; i < N; ++i) {
                s_sm[i] = T(s8[i]);
                if (s8[i] > 0) upm[i >> 6] |= 1ull << (i & 63);
                else dnm[i >> 6] |= 1ull << (i & 63);
            }
            buf = 0;
        }
        __syncthreads();

        // ---- fresh cache (buffer 0) ----
        // (the trip count is uniform over the warp: the group shuffles below
        // need every lane; groups past the last row compute row 0 and store nothing)
        for (int rbase = 0; rbase < rows; rbase += nslots) {
            const int row0 = rbase + slot;
            const bool active = row0 < rows;
            const int row = active ? row0 : 0;
            const int r = row / md.G, g = row - r * md.G;
            const uint8_t *pg = md.perm + (size_t)g * N;
            const cx<T> *Wr = md.Wt + (size_t)r * N * M;
            cx<T> thp[MPL];
#pragma unroll
            for (int j = 0; j < MPL; ++j) thp[j] = cx<T>{T(0), T(0)};
            for (int i = 0; i < N; ++i) {
                const cx<T> *wk = Wr + (size_t)pg[i] * M;
                const T si = s_sm[i];
#pragma unroll
                for (int j = 0; j < MPL; ++j) {
                    const int m = gl + kSGL * j;
                    if (m < M) { const cx<T> w = wk[m]; thp[j].x += si * w.x; thp[j].y += si * w.y; }
                }
            }
            cx<T> at{T(0), T(0)};
            if (md.use_bias) {
                const cx<T> *ar = md.avec + (size_t)r * N;
                for (int i = gl; i < N; i += kSGL) { const cx<T> a = ar[pg[i]]; at.x += s_sm[i] * a.x; at.y += s_sm[i] * a.y; }
#pragma unroll
                for (int o = kSGL / 2; o > 0; o >>= 1) { at.x += shfl_x(at.x, o); at.y += shfl_x(at.y, o); }
            }
            for (int sg = 0; sg < md.nsign; ++sg) {
                const int sign = sg ? -1 : 1;
                const int t = row * md.nsign + sg;
                sc<T> prod{T(1), T(0), 0};
                const cx<T> *br = md.bvec + (size_t)r * M;
#pragma unroll
                for (int j = 0; j < MPL; ++j) {
                    const int m = gl + kSGL * j;
                    if (m < M) {
                        cx<T> th{sign * thp[j].x, sign * thp[j].y};
                        if (md.use_bias) { const cx<T> b = br[m]; th.x += b.x; th.y += b.y; }
                        cx<T> mant, pv; int k;
                        cosh2(th, mant, k, pv);
                        if (active) pc0[(size_t)t * M + m] = pv;
                        const cx<T> q = cmul(mk(prod.x, prod.y), mant);
                        prod = sc<T>{q.x, q.y, prod.e + k};
                    }
                }
                prod = sc_norm(prod);
#pragma unroll
                for (int o = kSGL / 2; o > 0; o >>= 1) {
                    const sc<T> w{shfl_x(prod.x, o), shfl_x(prod.y, o), __shfl_xor_sync(0xffffffffu, prod.e, o)};
                    prod = sc_mul(prod, w);
                }
                if (gl == 0 && active) {
                    const cx<T> lc = md.logc[r];
                    sc<T> lead = sc_exp(cx<T>{lc.x + sign * at.x, lc.y + sign * at.y});
                    T c = md.chi[g];
                    if (sign < 0 && md.chiP < 0) c = -c;
                    lead.x *= c; lead.y *= c;
                    tc0[t] = sc_mul(prod, sc_norm(lead));
                }
            }
        }
        __syncthreads();

        const int total = n_burn + n_per_chain * n_skip;
        int n_acc = 0;
        for (int step = 0; step < total; ++step) {
            if (threadIdx.x == 0) {
                const u32x4 w = philox((uint32_t)step, 0u, 0u, 0u, k0, k1);
                const int ku = (int)(((uint64_t)w.v[0] * (uint64_t)(N / 2)) >> 32);
                const int kd = (int)(((uint64_t)w.v[1] * (uint64_t)(N / 2)) >> 32);
                site_u = kth_bit(upm, md.nwords, ku);
                site_d = kth_bit(dnm, md.nwords, kd);
                u_sh = (float)(w.v[2] >> 8) * (1.0f / 16777216.0f);
            }
            __syncthreads();
            const int iu = site_u, id = site_d, cb = buf;
            const cx<T> *P0 = cb ? pc1 : pc0;
            cx<T> *P1 = cb ? pc0 : pc1;
            const sc<T> *T0 = cb ? tc1 : tc0;
            sc<T> *T1 = cb ? tc0 : tc1;
            // ---- ratio of the proposal, and the speculative update ----
            sc<T> so{T(0), T(0), 0}, sn{T(0), T(0), 0};
            // one (row, sign) pair per group and iteration: K |G| n_sign pairs
            // divide the groups evenly where K |G| alone does not
            for (int tbase = 0; tbase < nrs; tbase += nslots) {
                const int t0 = tbase + slot;
                const bool active = t0 < nrs;
                const int t = active ? t0 : 0;
                const int row = md.nsign == 2 ? t >> 1 : t;
                const int sg = t - row * md.nsign;
                const int r = row / md.G, g = row - r * md.G;
                const int ku = md.perm[(size_t)g * N + iu], kd = md.perm[(size_t)g * N + id];
                const size_t rs = (size_t)r * 2 * N * md.Mp;
                {
                    // site u holds +1: sigma = sign
                    const cx<T> *Su = md.S4 + rs + ((size_t)sg * N + ku) * md.Mp;         // exp(-4 sigma W_u)
                    const cx<T> *Sd = md.S4 + rs + ((size_t)(sg ^ 1) * N + kd) * md.Mp;   // exp(+4 sigma W_d)
                    const cx<T> *__restrict__ pr_in = P0 + (size_t)t * M;
                    cx<T> *__restrict__ pr_out = P1 + (size_t)t * M;
                    // loads of a block of JB hidden units first (the stores below do
                    // not alias them), then the arithmetic and the stores
                    constexpr int JB = MPL < 10 ? MPL : 8;
                    cx<T> prod{T(1), T(0)};
#pragma unroll
                    for (int j0 = 0; j0 < MPL; j0 += JB) {
                        cx<T> pv_[JB], su_[JB], sd_[JB];
#pragma unroll
                        for (int jj = 0; jj < JB; ++jj) {
                            const int m = gl + kSGL * (j0 + jj);
                            if (j0 + jj < MPL && m < M) { pv_[jj] = pr_in[m]; su_[jj] = Su[m]; sd_[jj] = Sd[m]; }
                        }
#pragma unroll
                        for (int jj = 0; jj < JB; ++jj) {
                            const int m = gl + kSGL * (j0 + jj);
                            if (j0 + jj < MPL && m < M) {
                                const cx<T> e2 = cmul(su_[jj], sd_[jj]);          // e^{2 Delta}
                                const cx<T> tt{e2.x - T(1), e2.y};
                                const cx<T> p = pv_[jj];
                                const cx<T> f{T(1) + p.x * tt.x - p.y * tt.y, p.x * tt.y + p.y * tt.x};
                                prod = cmul(prod, f);
                                if (active) pr_out[m] = cdiv_upd(cmul(p, e2), f);
                            }
                        }
                    }
                    const int ex = expo<T>(prod.x, prod.y);
                    const T scl = pow2i<T>(-ex);
                    sc<T> pv{prod.x * scl, prod.y * scl, ex};
#pragma unroll
                    for (int o = kSGL / 2; o > 0; o >>= 1) {
                        const sc<T> w{shfl_x(pv.x, o), shfl_x(pv.y, o), __shfl_xor_sync(0xffffffffu, pv.e, o)};
                        pv = sc_mul(pv, w);
                    }
                    // the pair's product over m, staged in its next-term slot
                    if (gl == 0 && active) T1[t] = pv;
                }
            }
            __syncthreads();
            // every thread finishes pairs: prefactor exp(sigma (Cs_u - Cs_d)),
            // sigma = sign, the new term, and the old and new sums
            for (int t = threadIdx.x; t < nrs; t += blockDim.x) {
                const int row = md.nsign == 2 ? t >> 1 : t;
                const int sg = t - row * md.nsign;
                const int r = row / md.G, g = row - r * md.G;
                const int ku = md.perm[(size_t)g * N + iu], kd = md.perm[(size_t)g * N + id];
                const sc<T> *ESr = md.ES + (size_t)r * 2 * N;
                const sc<T> pref = sc_mul(ESr[(size_t)sg * N + ku], ESr[(size_t)(sg ^ 1) * N + kd]);
                const sc<T> term = T0[t];
                const sc<T> tn = sc_mul(sc_mul(term, T1[t]), pref);
                T1[t] = tn;
                so = sc_add(so, term);
                sn = sc_add(sn, tn);
            }
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const sc<T> a{shfl_x(so.x, o), shfl_x(so.y, o), __shfl_xor_sync(0xffffffffu, so.e, o)};
                const sc<T> b{shfl_x(sn.x, o), shfl_x(sn.y, o), __shfl_xor_sync(0xffffffffu, sn.e, o)};
                so = sc_add(so, a);
                sn = sc_add(sn, b);
            }
            if (lane == 0) { wold[warp] = so; wnew[warp] = sn; }
            __syncthreads();
            if (warp == 0) {
                sc<T> a = lane < kSWarps ? wold[lane] : sc<T>{T(0), T(0), 0};
                sc<T> b = lane < kSWarps ? wnew[lane] : sc<T>{T(0), T(0), 0};
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const sc<T> x{shfl_x(a.x, o), shfl_x(a.y, o), __shfl_xor_sync(0xffffffffu, a.e, o)};
                    const sc<T> y{shfl_x(b.x, o), shfl_x(b.y, o), __shfl_xor_sync(0xffffffffu, b.e, o)};
                    a = sc_add(a, x);
                    b = sc_add(b, y);
                }
                if (lane == 0) {
                const double ax = a.x, ay = a.y, bx = b.x, by = b.y;
                const double r2 = (bx * bx + by * by) / (ax * ax + ay * ay) * ldexp(1.0, 2 * (b.e - a.e));
                const int acc_now = (double)u_sh < r2;
                if (!isfinite(r2)) flag_range(md.status);
                if (acc_now) {
                    s_sm[iu] = T(-1); s_sm[id] = T(1);
                    upm[iu >> 6] &= ~(1ull << (iu & 63)); dnm[iu >> 6] |= 1ull << (iu & 63);
                    dnm[id >> 6] &= ~(1ull << (id & 63)); upm[id >> 6] |= 1ull << (id & 63);
                    buf = cb ^ 1;
                    if (step >= n_burn) ++n_acc;
                }
                accept = acc_now;
                }
            }
            __syncthreads();
            // ---- keep every n_skip-th state after burn-in ----
            if (step >= n_burn && ((step - n_burn + 1) % n_skip) == 0 && threadIdx.x < md.nwords) {
                const int kept = (step - n_burn + 1) / n_skip - 1;
                cfg_out[((size_t)chain * n_per_chain + kept) * md.nwords + threadIdx.x] = upm[threadIdx.x];
            }
        }
        if (threadIdx.x == 0 && acc_out)
            acc_out[chain] = n_per_chain * n_skip > 0 ? (float)n_acc / (float)(n_per_chain * n_skip) : 0.f;
        __syncthreads();
    }
}

template <typename T> int sampler_grid(const DevModel<T> &md, int n_chains, int nsm)
{
    // one resident CTA per SM keeps the active chains' caches in L2
    const int g = nsm > 0 ? nsm : 1;
    return n_chains < g ? n_chains : g;
}

template <typename T>
cudaError_t launch_sample(const DevModel<T> &md, uint64_t seed, int n_chains, int n_per_chain, int n_skip, int n_burn,
                          uint64_t *cfg_out, float *acc_out, void *cache, int nsm, cudaStream_t st)
{
    if (n_chains <= 0) return cudaSuccess;
    const int grid = sampler_grid(md, n_chains, nsm);
    const int need = (md.M + kSGL - 1) / kSGL;
#define NNQS_CASE(V) \
    if (need <= V) { k_sample<T, V><<<grid, kSThreads, 0, st>>>(md, seed, n_chains, n_per_chain, n_skip, n_burn, cfg_out, acc_out, (unsigned char *)cache); return cudaGetLastError(); }
    NNQS_CASE(2) NNQS_CASE(4) NNQS_CASE(9) NNQS_CASE(16) NNQS_CASE(32) NNQS_CASE(64)
#undef NNQS_CASE
    return cudaErrorInvalidValue;
}

template size_t sampler_cache_bytes<float>(const DevModel<float> &);
template size_t sampler_cache_bytes<double>(const DevModel<double> &);
template int sampler_grid<float>(const DevModel<float> &, int, int);
template int sampler_grid<double>(const DevModel<double> &, int, int);
template cudaError_t launch_sample<float>(const DevModel<float> &, uint64_t, int, int, int, int, uint64_t *, float *, void *, int, cudaStream_t);
template cudaError_t launch_sample<double>(const DevModel<double> &, uint64_t, int, int, int, int, uint64_t *, float *, void *, int, cudaStream_t);

}  // namespace nnqs
