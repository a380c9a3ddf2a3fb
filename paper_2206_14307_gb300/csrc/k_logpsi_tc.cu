// k_logpsi_tc.cu -- log psi of fresh configurations with the theta GEMM on the
// tcgen05 tensor cores (Eqs. 2-6), BF16-split weights, FP32 accumulation.
//
// For RBM r the rows of the GEMM are the transformed configurations T_g s of
// S samples x |G| operations (S chosen so that S |G| is a multiple of 128):
//   theta'[row][n] = sum_k A[row][k] B[n][k],
//   A[row] = [t | t (| t)]   (t = T_g s in +-1, exact in bf16),
//   B[n]   = [W_hi | W_lo (| W_mid)] of Re W_m (n < M8) or Im W_m (n >= M8),
// so theta' = (W_hi + W_lo (+ W_mid)) . t to within the split's error (2^-17
// relative per weight for two terms, 2^-25 for three).  A is built by the
// threads in shared memory in the no-swizzle K-major core-matrix layout; B's
// shared-memory image is laid out on the device once per parameter set and
// brought in with a bulk (TMA) copy; the 128 x 2*MT accumulator lives in TMEM.
// Hidden units are taken MT at a time (one tile when M <= 128; otherwise
// ceil(M/128) tiles, each with its own B image, copied per 128-row tile): the
// epilogue multiplies each tile's factors into the row's running products.
// The epilogue reads each row from TMEM, forms prod_m 2cosh(b_m +- theta'_m)
// as a scaled complex number, multiplies the leading factor
// c_r chi(g) chi_P e^{+-a.t} and sums the rows of every sample (segmented
// warp reduction), giving log psi with an exact binary exponent.
//
// Every wait on an mbarrier has an iteration limit; on expiry the kernel sets
// NNQS_ETIMEOUT in the status word, waits (bounded) for its own MMAs, frees
// its TMEM and returns.
#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

#include <cuda_bf16.h>

namespace nnqs {

struct TcShape {
    int N, M, M8, NS, KD, NC, G, K, S, ntiles, nsign;
    int MT, nmt;                 // hidden units per tile (multiple of 8), tiles; NC = 2 MT columns per tile
    uint32_t a_bytes, b_bytes;   // allocated (with margin) shared bytes of A and B
    uint32_t b_img_bytes;        // bytes of one B image (one tile of one RBM)
};

__host__ __device__ inline int gcd_i(int a, int b) { while (b) { int t = a % b; a = b; b = t; } return a; }

TcShape tc_shape(int N, int M, int G, int K, int nsign, int NS)
{
    TcShape s;
    s.N = N; s.M = M; s.M8 = (M + 7) / 8 * 8; s.NS = NS;
    s.KD = (NS * N + 15) / 16 * 16;
    s.nmt = (s.M8 + 127) / 128;
    s.MT = ((s.M8 + s.nmt - 1) / s.nmt + 7) / 8 * 8;
    s.NC = 2 * s.MT;
    s.G = G; s.K = K; s.nsign = nsign;
    s.S = 128 / gcd_i(G, 128);
    s.ntiles = s.S * G / 128;
    const uint32_t sbo = (uint32_t)(s.KD / 8) * 128;
    const uint32_t a_dense = 16 * sbo;
    const uint32_t b_dense = (uint32_t)(s.NC / 8) * sbo;
    // margin: stay inside the allocation even if the two byte offsets of the
    // descriptor were read the other way round
    const uint32_t a_alt = 15 * 128 + (uint32_t)(s.KD / 8) * sbo;
    const uint32_t b_alt = (uint32_t)(s.NC / 8 - 1) * 128 + (uint32_t)(s.KD / 8) * sbo;
    const uint32_t a_need = a_dense > a_alt + 128 ? a_dense : a_alt + 128;
    const uint32_t b_need = b_dense > b_alt + 128 ? b_dense : b_alt + 128;
    s.a_bytes = (a_need + 1023) / 1024 * 1024;   // rounded up: every region holds its image
    s.b_bytes = (b_need + 1023) / 1024 * 1024;
    s.b_img_bytes = b_dense;
    return s;
}

// byte offset of element (row, k) in the no-swizzle K-major core layout
__host__ __device__ __forceinline__ uint32_t core_off(int row, int k, int KD)
{
    return (uint32_t)(row >> 3) * (uint32_t)(KD / 8) * 128u + (uint32_t)(k >> 3) * 128u + (uint32_t)(row & 7) * 16u +
           (uint32_t)(k & 7) * 2u;
}

// ---------------------------------------------------------------------------
// B images: for every RBM r and hidden-unit tile t, NC = 2 MT rows (Re W_m
// for n < MT, Im W_m after, m = t MT + n mod MT) x KD columns (NS bf16 terms
// of W_m,j), zero-padded (m >= M), in the core layout.
// ---------------------------------------------------------------------------
__global__ void k_bimg(const double *__restrict__ par, int N, int M, int K, int MT, int nmt, int NS, int KD,
                       uint16_t *__restrict__ img)
{
    const int NC = 2 * MT;
    const int64_t P1 = 1 + N + M + (int64_t)M * N;
    const int64_t per = (int64_t)NC * KD;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < per * K * nmt;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int rt = (int)(q / per);           // r * nmt + t
        const int r = rt / nmt, t = rt - r * nmt;
        const int64_t rem = q - rt * per;
        const int n = (int)(rem / KD), k = (int)(rem - (int64_t)n * KD);
        const int m = t * MT + (n < MT ? n : n - MT);
        const int part = n < MT ? 0 : 1;
        const int split = k / N, j = k - split * N;
        float v = 0.f;
        if (m < M && split < NS) {
            const double w = par[2 * (r * P1 + 1 + N + M + (int64_t)m * N + j) + part];
            // successive bf16 terms of w
            double rest = w;
            float term = 0.f;
            for (int u = 0; u <= split; ++u) {
                term = __bfloat162float(__float2bfloat16_rn((float)rest));
                rest -= (double)term;
            }
            v = term;
        }
        const __nv_bfloat16 b = __float2bfloat16_rn(v);
        img[(size_t)rt * per + core_off(n, k, KD) / 2] = *reinterpret_cast<const uint16_t *>(&b);
    }
}

// ---------------------------------------------------------------------------
// the fused GEMM + log-cosh + projection-sum kernel
// ---------------------------------------------------------------------------
constexpr int kTcThreads = 256;
constexpr uint32_t kTmemCols = 256;

struct TcArgs {
    TcShape sh;
    const uint16_t *bimg;     // [K][nmt][NC x KD] core-layout images
    const uint8_t *pinv;      // [G][N] inverse permutations: (T_g s)_j = s_{pinv[g][j]}
};

template <typename T>
__global__ void __launch_bounds__(kTcThreads, 1) k_logpsi_tc(DevModel<T> md, TcArgs ta, const uint64_t *__restrict__ cfg,
                                                             int64_t n, double *__restrict__ out)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const TcShape sh = ta.sh;
    unsigned char *A = smem;
    unsigned char *B = smem + sh.a_bytes;
    int8_t *spins = reinterpret_cast<int8_t *>(B + sh.b_bytes);                        // [S][N]
    sc<float> *acc = reinterpret_cast<sc<float> *>(spins + ((sh.S * sh.N + 15) / 16) * 16);  // [S]
    sc<float> *xbuf = acc + sh.S;                                                       // [128][2]
    sc<float> *wpart = xbuf + 256;                                                      // [4][32]
    int *wkey = reinterpret_cast<int *>(wpart + 128);                                   // [4][32]
    uint64_t *bars = reinterpret_cast<uint64_t *>(wkey + 128 + 2);                      // [2] (8-aligned below)
    bars = reinterpret_cast<uint64_t *>((reinterpret_cast<uintptr_t>(bars) + 7) & ~(uintptr_t)7);
    uint32_t *tmem_base = reinterpret_cast<uint32_t *>(bars + 2);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3, half = warp >> 2;
    const int N = sh.N, M = sh.M, MT = sh.MT, KD = sh.KD, G = sh.G;
    const int nchunk = MT / 8, c0 = (nchunk + 1) / 2;
    const uint32_t sbo = (uint32_t)(KD / 8) * 128u;
    const uint32_t idesc = tc::idesc_bf16(128, sh.NC);

    if (warp == 0) {
        tc::tmem_alloc(tmem_base, kTmemCols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&bars[0], 1);  // B image landed
        tc::mbar_init(&bars[1], 1);  // MMAs of a tile completed
        tc::mbar_fence_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *tmem_base;
    uint32_t ph_b = 0, ph_m = 0;
    bool aborted = false;  // uniform over the CTA (set from __syncthreads_or)
    // this thread's view of work still in flight after a timed-out wait (the
    // phase bits are flipped only on success, so they still name that phase)
    bool mma_pending = false, copy_pending = false;

    const int64_t nsuper = (n + sh.S - 1) / sh.S;
    for (int64_t st = blockIdx.x; st < nsuper; st += gridDim.x) {
        const int64_t s0 = st * sh.S;
        const int nsamp = (int)((n - s0) < sh.S ? (n - s0) : sh.S);
        for (int i = tid; i < sh.S * N; i += kTcThreads) {
            const int sl = i / N, site = i - sl * N;
            spins[i] = sl < nsamp ? (int8_t)spin_of(cfg + (s0 + sl) * md.nwords, site) : (int8_t)1;
        }
        for (int i = tid; i < sh.S; i += kTcThreads) acc[i] = sc<float>{0.f, 0.f, 0};
        __syncthreads();

        for (int r = 0; r < sh.K; ++r) {
            // ---- bring in B of RBM r (one tile: once per RBM) ----
            if (sh.nmt == 1) {
                if (tid == 0) {
                    tc::mbar_expect_tx(&bars[0], sh.b_img_bytes);
                    tc::bulk_g2s(B, ta.bimg + (size_t)r * sh.NC * KD, sh.b_img_bytes, &bars[0]);
                }
                const bool okb = tc::mbar_wait_bounded(&bars[0], ph_b);
                if (okb) ph_b ^= 1; else copy_pending = true;
                if (__syncthreads_or(!okb)) { aborted = true; if (tid == 0) atomicExch(md.status, -4); break; }
            }

            for (int tile = 0; tile < sh.ntiles; ++tile) {
                // ---- A: rows of this tile, K split between two threads per row ----
                {
                    const int row = tid & 127, hk = tid >> 7;
                    const int q = tile * 128 + row;
                    const int sl = q / G, g = q - sl * G;
                    const bool valid = sl < nsamp;
                    const int8_t *sp = spins + sl * N;
                    const uint8_t *pg = ta.pinv + (size_t)g * N;
                    const int nkc = KD / 8, kc_lo = hk ? nkc / 2 : 0, kc_hi = hk ? nkc : nkc / 2;
                    for (int kc = kc_lo; kc < kc_hi; ++kc) {
                        uint32_t w4[4];
#pragma unroll
                        for (int h2 = 0; h2 < 4; ++h2) {
                            uint32_t pair = 0;
#pragma unroll
                            for (int e = 0; e < 2; ++e) {
                                const int k = kc * 8 + h2 * 2 + e;
                                uint32_t bits = 0;
                                if (valid && k < sh.NS * N) {
                                    const int j = k % N;
                                    bits = sp[pg[j]] > 0 ? 0x3F80u : 0xBF80u;   // bf16 +1 / -1
                                }
                                pair |= bits << (16 * e);
                            }
                            w4[h2] = pair;
                        }
                        *reinterpret_cast<uint4 *>(A + core_off(row, kc * 8, KD)) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
                    }
                }
                tc::fence_proxy_async_smem();
                __syncthreads();
                const int row = quad * 32 + lane;
                const int q = tile * 128 + row;
                const int sl = q / G, g = q - sl * G;
                const bool valid = sl < nsamp;
                sc<float> pp{1.f, 0.f, 0}, pm{1.f, 0.f, 0};
                const cx<float> *br = reinterpret_cast<const cx<float> *>(md.bvec) + (size_t)r * M;
                const uint32_t lane_addr = taddr + ((uint32_t)(quad * 32) << 16);
                for (int mt = 0; mt < sh.nmt; ++mt) {
                    if (sh.nmt > 1) {
                        // ---- B of (RBM r, hidden-unit tile mt); the previous tile's MMAs are complete ----
                        if (tid == 0) {
                            tc::mbar_expect_tx(&bars[0], sh.b_img_bytes);
                            tc::bulk_g2s(B, ta.bimg + ((size_t)r * sh.nmt + mt) * sh.NC * KD, sh.b_img_bytes,
                                         &bars[0]);
                        }
                        const bool okb = tc::mbar_wait_bounded(&bars[0], ph_b);
                        if (okb) ph_b ^= 1; else copy_pending = true;
                        if (__syncthreads_or(!okb)) { aborted = true; if (tid == 0) atomicExch(md.status, -4); break; }
                    }
                    // ---- MMAs: K/16 steps into TMEM columns [0, NC) ----
                    if (tid == 0) {
                        tc::fence_after_sync();
                        const uint32_t a0 = tc::smem_u32(A), b0 = tc::smem_u32(B);
                        for (int kk = 0; kk < KD / 16; ++kk) {
                            const uint64_t ad = tc::smem_desc(a0 + kk * 256u, 128u, sbo);
                            const uint64_t bd = tc::smem_desc(b0 + kk * 256u, 128u, sbo);
                            tc::mma_bf16(taddr, ad, bd, idesc, kk > 0 ? 1u : 0u);
                        }
                        tc::mma_commit(&bars[1]);
                    }
                    const bool okm = tc::mbar_wait_bounded(&bars[1], ph_m);
                    if (okm) ph_m ^= 1; else mma_pending = true;
                    if (__syncthreads_or(!okm)) { aborted = true; if (tid == 0) atomicExch(md.status, -4); break; }
                    tc::fence_after_sync();

                    // ---- epilogue: 2cosh products of this thread's half of the tile's hidden units ----
                    const int cb = half ? c0 : 0, ce = half ? nchunk : c0;
                    for (int c = cb; c < ce; ++c) {
                        float re[8], im[8];
                        tc::tmem_ld8(lane_addr + (uint32_t)(c * 8), re);
                        tc::tmem_ld8(lane_addr + (uint32_t)(MT + c * 8), im);
                        tc::tmem_wait_ld();
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const int m = mt * MT + c * 8 + e;
                            if (m < M) {
                                cx<float> b{0.f, 0.f};
                                if (md.use_bias) b = br[m];
                                cx<float> mant;
                                int k;
                                cosh2_mant(cx<float>{b.x + re[e], b.y + im[e]}, mant, k);
                                const cx<float> x = cmul(mk(pp.x, pp.y), mant);
                                pp = sc_norm(sc<float>{x.x, x.y, pp.e + k});
                                if (sh.nsign == 2) {
                                    cosh2_mant(cx<float>{b.x - re[e], b.y - im[e]}, mant, k);
                                    const cx<float> y = cmul(mk(pm.x, pm.y), mant);
                                    pm = sc_norm(sc<float>{y.x, y.y, pm.e + k});
                                }
                            }
                        }
                    }
                    if (sh.nmt > 1) {
                        // the next tile's MMAs overwrite TMEM and its copy overwrites B
                        tc::fence_before_sync();
                        __syncthreads();
                        tc::fence_after_sync();
                    }
                }
                if (aborted) break;
                tc::fence_before_sync();
                if (half == 1) { xbuf[2 * row] = pp; xbuf[2 * row + 1] = pm; }
                __syncthreads();
                if (half == 0) {
                    pp = sc_mul(pp, xbuf[2 * row]);
                    pm = sc_mul(pm, xbuf[2 * row + 1]);
                    // leading factor c_r chi(g) chi_P e^{+-a.t}
                    sc<float> term{0.f, 0.f, 0};
                    if (valid) {
                        cx<float> at{0.f, 0.f};
                        if (md.use_bias) {
                            const cx<float> *ar = reinterpret_cast<const cx<float> *>(md.avec) + (size_t)r * N;
                            const int8_t *sp = spins + sl * N;
                            const uint8_t *pg = ta.pinv + (size_t)g * N;
                            for (int j = 0; j < N; ++j) {
                                const float t = (float)sp[pg[j]];
                                at.x += t * ar[j].x;
                                at.y += t * ar[j].y;
                            }
                        }
                        const cx<float> lc = reinterpret_cast<const cx<float> *>(md.logc)[r];
                        const float chi = ((const float *)md.chi)[g];
                        sc<float> lp = sc_exp(cx<float>{lc.x + at.x, lc.y + at.y});
                        lp.x *= chi; lp.y *= chi;
                        term = sc_mul(pp, sc_norm(lp));
                        if (sh.nsign == 2) {
                            sc<float> lm = sc_exp(cx<float>{lc.x - at.x, lc.y - at.y});
                            const float c2 = md.chiP < 0 ? -chi : chi;
                            lm.x *= c2; lm.y *= c2;
                            term = sc_add(term, sc_mul(pm, sc_norm(lm)));
                        }
                    }
                    // segmented reduction over lanes with the same sample (keys non-decreasing)
                    int key = valid ? sl : -1;
                    sc<float> v = term;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const sc<float> up{__shfl_down_sync(0xffffffffu, v.x, o), __shfl_down_sync(0xffffffffu, v.y, o),
                                           __shfl_down_sync(0xffffffffu, v.e, o)};
                        const int ku = __shfl_down_sync(0xffffffffu, key, o);
                        if (lane + o < 32 && ku == key) v = sc_add(v, up);
                    }
                    const int kprev = __shfl_up_sync(0xffffffffu, key, 1);
                    const bool head = lane == 0 || kprev != key;
                    wpart[quad * 32 + lane] = v;
                    wkey[quad * 32 + lane] = head ? key : -1;
                }
                __syncthreads();
                if (tid == 0) {
                    for (int i = 0; i < 128; ++i) {
                        const int k = wkey[i];
                        if (k >= 0) acc[k] = sc_add(acc[k], wpart[i]);
                    }
                }
                tc::fence_before_sync();
                __syncthreads();
                tc::fence_after_sync();
            }
            if (aborted) break;
        }
        if (aborted) break;
        for (int i = tid; i < nsamp; i += kTcThreads) {
            const sc<float> tot = acc[i];
            double re, im;
            if (!sc_finite(tot)) {
                flag_range(md.status);
                re = nan(""); im = nan("");
            } else if (sc_zero(tot)) {
                re = -INFINITY; im = 0.0;
            } else {
                const double x = (double)tot.x, y = (double)tot.y;
                re = log(hypot(x, y)) + tot.e * 0.69314718055994530942;
                im = atan2(y, x);
            }
            out[2 * (s0 + i)] = re;
            out[2 * (s0 + i) + 1] = im;
        }
        __syncthreads();
    }
    if (aborted && tid == 0) {
        // the issuing thread lets its MMAs and its bulk copy still in flight
        // finish (bounded) before the accumulator is freed and the CTA exits
        if (mma_pending) (void)tc::mbar_wait_bounded(&bars[1], ph_m, 1u << 22);
        if (copy_pending) (void)tc::mbar_wait_bounded(&bars[0], ph_b, 1u << 22);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, kTmemCols);
}

static size_t tc_smem_bytes(const TcShape &s)
{
    size_t b = s.a_bytes + s.b_bytes;
    b += ((size_t)(s.S * s.N + 15) / 16) * 16;
    b += (size_t)(s.S + 256 + 128) * sizeof(sc<float>) + 130 * sizeof(int) + 8 + 16 + 4 + 64;
    b = (b + 1023) / 1024 * 1024;
    // at most two CTAs per SM, so that two 256-column TMEM allocations always fit
    return b < 80 * 1024 ? 80 * 1024 : b;
}

bool tc_supported(int N, int M, int G, int K, int nsign, int NS)
{
    if (M > kMaxM || NS < 2 || NS > 3) return false;
    const TcShape s = tc_shape(N, M, G, K, nsign, NS);
    return tc_smem_bytes(s) <= 220 * 1024 && s.KD <= 4096 && s.S <= 128;
}

size_t tc_bimg_bytes(int N, int M, int K, int NS)
{
    const TcShape s = tc_shape(N, M, 1, K, 1, NS);
    return (size_t)K * s.nmt * s.b_img_bytes;
}

cudaError_t launch_bimg(const double *params, int N, int M, int K, int NS, uint16_t *img, cudaStream_t st)
{
    const TcShape s = tc_shape(N, M, 1, K, 1, NS);
    k_bimg<<<1024, 256, 0, st>>>(params, N, M, K, s.MT, s.nmt, NS, s.KD, img);
    return cudaGetLastError();
}

cudaError_t launch_log_psi_tc(const DevModel<float> &md, const uint16_t *bimg, const uint8_t *pinv, int NS,
                              const uint64_t *cfg, int64_t n, double *out, int nsm, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    TcArgs ta;
    ta.sh = tc_shape(md.N, md.M, md.G, md.K, md.nsign, NS);
    ta.bimg = bimg;
    ta.pinv = pinv;
    const size_t smem = tc_smem_bytes(ta.sh);
    cudaError_t err = cudaFuncSetAttribute(k_logpsi_tc<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    const int64_t nsuper = (n + ta.sh.S - 1) / ta.sh.S;
    const int64_t g = 2 * (int64_t)nsm;
    const int grid = (int)(nsuper < g ? nsuper : g);
    k_logpsi_tc<float><<<grid, kTcThreads, smem, st>>>(md, ta, cfg, n, out);
    return cudaGetLastError();
}

}  // namespace nnqs
