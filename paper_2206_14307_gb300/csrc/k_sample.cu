// k_sample.cu -- persistent chain-parallel Metropolis sampler (Sec. 3.2).
//
// One CTA per Markov chain.  The chain keeps, in device memory, for every row
// (r, g, sign) of the projected sum its term c_r chi(g) chi_P phi_r(+-T_g s)
// and, for every hidden unit, p_m = e^{theta_m}/(2cosh theta_m).  A proposed
// exchange of an up site i and a down site j changes the row by
//   prod_m [p_m e^{Delta_m} + (1-p_m) e^{-Delta_m}] * e^{sign Delta_a},
// evaluated from the exp(+-2W) tables without any transcendental function; on
// acceptance p_m <- p_m e^{Delta_m} / factor_m and the row term is multiplied
// by its factor.  Random numbers: Philox4x32-10 keyed by (seed, chain).
#include "common.cuh"
#include "kernels.h"

namespace nnqs {

// bytes of one chain's cache, padded to 256 so every chain starts aligned
template <typename T> __host__ __device__ size_t chain_stride(int K, int G, int nsign, int M)
{
    const size_t rows = (size_t)K * G * nsign;
    const size_t b = rows * M * sizeof(cx<T>) + rows * sizeof(sc<T>);
    return (b + 255) & ~(size_t)255;
}

template <typename T> size_t sampler_cache_bytes(const DevModel<T> &md)
{
    return chain_stride<T>(md.K, md.G, md.nsign, md.M);
}

template <typename T, int MPL>
__global__ void __launch_bounds__(kThreads) k_sample(DevModel<T> md, uint64_t seed, int n_per_chain, int n_skip,
                                                     int n_burn, uint64_t *__restrict__ cfg_out,
                                                     float *__restrict__ acc_out, unsigned char *__restrict__ cache)
{
    __shared__ T s_sm[kMaxN];
    __shared__ int8_t s8[kMaxN];
    __shared__ sc<T> wold[kWarps], wnew[kWarps];
    __shared__ int site_u, site_d, accept;
    __shared__ float u_sh;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int chain = blockIdx.x;
    const int N = md.N, M = md.M;
    const int rows = md.K * md.G;
    const size_t nrs = (size_t)rows * md.nsign;
    const size_t per_chain = chain_stride<T>(md.K, md.G, md.nsign, M);
    cx<T> *pc = reinterpret_cast<cx<T> *>(cache + per_chain * chain);   // [rows][nsign][M]
    sc<T> *tc = reinterpret_cast<sc<T> *>(cache + per_chain * chain + nrs * M * sizeof(cx<T>));
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32) ^ (uint32_t)chain;

    // ---- initial configuration: Fisher-Yates shuffle of N/2 ups ----
    if (threadIdx.x == 0) {
        for (int i = 0; i < N; ++i) s8[i] = (int8_t)(i < N / 2 ? 1 : -1);
        u32x4 w{};
        for (int j = N - 1, q = 0; j >= 1; --j, ++q) {
            if ((q & 3) == 0) w = philox((uint32_t)(q >> 2), 1u, 0u, 0u, k0, k1);
            const uint32_t x = w.v[q & 3];
            const int r = (int)(((uint64_t)x * (uint64_t)(j + 1)) >> 32);
            const int8_t t = s8[j]; s8[j] = s8[r]; s8[r] = t;
        }
        for (int i = 0; i < N; ++i) s_sm[i] = T(s8[i]);
    }
    __syncthreads();

    // ---- fresh cache ----
    for (int row = warp; row < rows; row += kWarps) {
        const int r = row / md.G, g = row - r * md.G;
        cx<T> thp[MPL], p[MPL];
        cx<T> acc[MPL];
        // theta' = W_r T_g s
#pragma unroll
        for (int j = 0; j < MPL; ++j) acc[j] = cx<T>{T(0), T(0)};
        const uint8_t *pg = md.perm + (size_t)g * N;
        const cx<T> *Wr = md.Wt + (size_t)r * N * M;
        for (int i = 0; i < N; ++i) {
            const cx<T> *wk = Wr + (size_t)pg[i] * M;
            const T si = s_sm[i];
#pragma unroll
            for (int j = 0; j < MPL; ++j) {
                const int m = lane + 32 * j;
                if (m < M) { const cx<T> w = wk[m]; acc[j].x += si * w.x; acc[j].y += si * w.y; }
            }
        }
#pragma unroll
        for (int j = 0; j < MPL; ++j) thp[j] = acc[j];
        cx<T> at{T(0), T(0)};
        if (md.use_bias) {
            const cx<T> *ar = md.avec + (size_t)r * N;
            for (int i = lane; i < N; i += 32) { const cx<T> a = ar[pg[i]]; at.x += s_sm[i] * a.x; at.y += s_sm[i] * a.y; }
            at = warp_sum(at);
        }
        for (int sg = 0; sg < md.nsign; ++sg) {
            const int sign = sg ? -1 : 1;
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
                    pc[((size_t)row * md.nsign + sg) * M + m] = p[j];
                }
            }
            prod = warp_prod(prod);
            if (lane == 0) {
                const cx<T> lc = md.logc[r];
                sc<T> lead = sc_exp(cx<T>{lc.x + sign * at.x, lc.y + sign * at.y});
                T c = md.chi[g];
                if (sign < 0 && md.chiP < 0) c = -c;
                lead.x *= c; lead.y *= c;
                tc[(size_t)row * md.nsign + sg] = sc_mul(prod, sc_norm(lead));
            }
        }
    }
    __syncthreads();

    const int total = n_burn + n_per_chain * n_skip;
    int n_acc = 0;
    for (int t = 0; t < total; ++t) {
        if (threadIdx.x == 0) {
            const u32x4 w = philox((uint32_t)t, 0u, 0u, 0u, k0, k1);
            const int ku = (int)(((uint64_t)w.v[0] * (uint64_t)(N / 2)) >> 32);
            const int kd = (int)(((uint64_t)w.v[1] * (uint64_t)(N / 2)) >> 32);
            int cu = 0, cd = 0, iu = -1, id = -1;
            for (int i = 0; i < N; ++i) {
                if (s8[i] > 0) { if (cu == ku) iu = i; ++cu; }
                else { if (cd == kd) id = i; ++cd; }
            }
            site_u = iu; site_d = id;
            u_sh = (float)(w.v[2] >> 8) * (1.0f / 16777216.0f);
        }
        __syncthreads();
        const int iu = site_u, id = site_d;
        // ---- ratio of the proposal ----
        sc<T> so{T(0), T(0), 0}, sn{T(0), T(0), 0};
        for (int row = warp; row < rows; row += kWarps) {
            const int r = row / md.G, g = row - r * md.G;
            const uint8_t *pg = md.perm + (size_t)g * N;
            const int ku = pg[iu], kd = pg[id];
            const cx2<T> *Xr = md.X + (size_t)r * N * M;
            for (int sg = 0; sg < md.nsign; ++sg) {
                const int sign = sg ? -1 : 1;
                const cx<T> *prow = pc + ((size_t)row * md.nsign + sg) * M;
                sc<T> fp{T(1), T(0), 0};
#pragma unroll
                for (int j = 0; j < MPL; ++j) {
                    const int m = lane + 32 * j;
                    if (m < M) {
                        const cx2<T> xu = Xr[(size_t)ku * M + m], xd = Xr[(size_t)kd * M + m];
                        // site iu holds +1, site id holds -1 in s
                        const cx<T> eD = sign > 0 ? cmul(xu.a, xd.b) : cmul(xu.b, xd.a);
                        const cx<T> eDi = sign > 0 ? cmul(xu.b, xd.a) : cmul(xu.a, xd.b);
                        const cx<T> fac = cadd(eDi, cmul(prow[m], csub(eD, eDi)));
                        const cx<T> q = cmul(mk(fp.x, fp.y), fac);
                        fp.x = q.x; fp.y = q.y;
                    }
                }
                fp = warp_prod(fp);
                if (lane == 0) {
                    const sc<T> term = tc[(size_t)row * md.nsign + sg];
                    cx<T> eA{T(1), T(0)};
                    if (md.use_bias) {
                        const cx2<T> au = md.XA[(size_t)r * N + ku], ad = md.XA[(size_t)r * N + kd];
                        eA = sign > 0 ? cmul(au.a, ad.b) : cmul(au.b, ad.a);
                    }
                    sc<T> tn = sc_mul(term, fp);
                    const cx<T> q = cmul(mk(tn.x, tn.y), eA);
                    tn.x = q.x; tn.y = q.y;
                    so = sc_add(so, term);
                    sn = sc_add(sn, sc_norm(tn));
                }
            }
        }
        if (lane == 0) { wold[warp] = so; wnew[warp] = sn; }
        __syncthreads();
        if (threadIdx.x == 0) {
            sc<T> a = wold[0], b = wnew[0];
            for (int w = 1; w < kWarps; ++w) { a = sc_add(a, wold[w]); b = sc_add(b, wnew[w]); }
            const double ax = a.x, ay = a.y, bx = b.x, by = b.y;
            const double r2 = (bx * bx + by * by) / (ax * ax + ay * ay) * ldexp(1.0, 2 * (b.e - a.e));
            const int acc_now = (double)u_sh < r2;
            accept = acc_now;
            if (!isfinite(r2)) atomicExch(md.status, -6);
            if (acc_now) { s8[iu] = -1; s8[id] = 1; s_sm[iu] = T(-1); s_sm[id] = T(1); }
            if (acc_now && t >= n_burn) ++n_acc;
        }
        __syncthreads();
        if (accept) {
            for (int row = warp; row < rows; row += kWarps) {
                const int r = row / md.G, g = row - r * md.G;
                const uint8_t *pg = md.perm + (size_t)g * N;
                const int ku = pg[iu], kd = pg[id];
                const cx2<T> *Xr = md.X + (size_t)r * N * M;
                for (int sg = 0; sg < md.nsign; ++sg) {
                    const int sign = sg ? -1 : 1;
                    cx<T> *prow = pc + ((size_t)row * md.nsign + sg) * M;
                    sc<T> fp{T(1), T(0), 0};
#pragma unroll
                    for (int j = 0; j < MPL; ++j) {
                        const int m = lane + 32 * j;
                        if (m < M) {
                            const cx2<T> xu = Xr[(size_t)ku * M + m], xd = Xr[(size_t)kd * M + m];
                            const cx<T> eD = sign > 0 ? cmul(xu.a, xd.b) : cmul(xu.b, xd.a);
                            const cx<T> eDi = sign > 0 ? cmul(xu.b, xd.a) : cmul(xu.a, xd.b);
                            const cx<T> p = prow[m];
                            const cx<T> fac = cadd(eDi, cmul(p, csub(eD, eDi)));
                            prow[m] = cdiv(cmul(p, eD), fac);
                            const cx<T> q = cmul(mk(fp.x, fp.y), fac);
                            fp.x = q.x; fp.y = q.y;
                        }
                    }
                    fp = warp_prod(fp);
                    if (lane == 0) {
                        sc<T> &term = tc[(size_t)row * md.nsign + sg];
                        cx<T> eA{T(1), T(0)};
                        if (md.use_bias) {
                            const cx2<T> au = md.XA[(size_t)r * N + ku], ad = md.XA[(size_t)r * N + kd];
                            eA = sign > 0 ? cmul(au.a, ad.b) : cmul(au.b, ad.a);
                        }
                        sc<T> tn = sc_mul(term, fp);
                        const cx<T> q = cmul(mk(tn.x, tn.y), eA);
                        tn.x = q.x; tn.y = q.y;
                        term = sc_norm(tn);
                    }
                }
            }
        }
        // ---- keep every n_skip-th state after burn-in ----
        if (t >= n_burn && ((t - n_burn + 1) % n_skip) == 0) {
            const int kept = (t - n_burn + 1) / n_skip - 1;
            uint64_t *o = cfg_out + ((size_t)chain * n_per_chain + kept) * md.nwords;
            for (int wd = warp; wd < md.nwords; wd += kWarps) {
                uint64_t v = 0;
                for (int b0 = 0; b0 < 64; b0 += 32) {
                    const int i = wd * 64 + b0 + lane;
                    const unsigned bal = __ballot_sync(0xffffffffu, i < N && s8[i] > 0);
                    v |= (uint64_t)bal << b0;
                }
                if (lane == 0) o[wd] = v;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && acc_out)
        acc_out[chain] = n_per_chain * n_skip > 0 ? (float)n_acc / (float)(n_per_chain * n_skip) : 0.f;
}

template <typename T>
cudaError_t launch_sample(const DevModel<T> &md, uint64_t seed, int n_chains, int n_per_chain, int n_skip, int n_burn,
                          uint64_t *cfg_out, float *acc_out, void *cache, cudaStream_t st)
{
    if (n_chains <= 0) return cudaSuccess;
    switch (mpl_slot(md.M)) {
#define NNQS_CASE(V) case V: k_sample<T, V><<<n_chains, kThreads, 0, st>>>(md, seed, n_per_chain, n_skip, n_burn, cfg_out, acc_out, (unsigned char *)cache); break;
        NNQS_CASE(1) NNQS_CASE(2) NNQS_CASE(3) NNQS_CASE(4) NNQS_CASE(6) NNQS_CASE(8) NNQS_CASE(13)
        default: k_sample<T, 16><<<n_chains, kThreads, 0, st>>>(md, seed, n_per_chain, n_skip, n_burn, cfg_out, acc_out, (unsigned char *)cache); break;
#undef NNQS_CASE
    }
    return cudaGetLastError();
}

template size_t sampler_cache_bytes<float>(const DevModel<float> &);
template size_t sampler_cache_bytes<double>(const DevModel<double> &);
template cudaError_t launch_sample<float>(const DevModel<float> &, uint64_t, int, int, int, int, uint64_t *, float *, void *, cudaStream_t);
template cudaError_t launch_sample<double>(const DevModel<double> &, uint64_t, int, int, int, int, uint64_t *, float *, void *, cudaStream_t);

}  // namespace nnqs
