// k_logpsi_tc.cuh -- log psi of fresh configurations with the theta GEMM on the
// tcgen05 tensor cores (Eqs. 2-6), BF16-split weights, FP32 accumulation.
//
// The rows of the GEMM are the transformed configurations t = T_g s of S
// samples x |G| operations (S chosen so that S |G| is a multiple of 128):
//   theta'[row][n] = sum_k A[row][k] B[n][k],   A[row] = t (+-1, exact in bf16),
// once per bf16 term of W (hi, lo (, mid)): B[n] = that term of Re W_m
// (n < MT) or Im W_m (n >= MT), accumulated in one FP32 TMEM accumulator, so
// theta' = W . t to within the split's error (2^-17 relative per weight for
// two terms, 2^-25 for three).  A is the same for every RBM r and hidden-unit
// tile: it is built once per 128-row tile in shared memory (no-swizzle K-major
// core-matrix layout) together with a_r . t of every row.  The image of
// (r, tile) -- its split weights and the tile's bias slice -- is laid out on
// the device once per parameter set and brought in by bulk (TMA) copies: all
// images at once when they fit, else streamed through two buffers.
//
// Pipeline (one CTA per SM, 16 warps): the block sequence of a CTA is
// (supertile, 128-row tile, r, hidden tile).  Two TMEM accumulators alternate:
// one elected thread issues the MMAs of block j + 1 while all warps run the
// epilogue of block j; the A tile of the next row tile is built (into the
// other A buffer when two fit) before that MMA issue.
//
// Epilogue: warp w reads TMEM lanes 32 (w mod 4) .. + 31 (its rows) and a
// quarter (MQ units) of the tile's hidden units (column group w / 4).  Per
// hidden unit one complex exponential: with theta = x + i y,
//   2 cosh(theta) = (e^x + e^-x) cos y + i (e^x - e^-x) sin y.
// When every |x| < 4 and every angle < pi/4 in the warp's group of units (the
// common case at the workloads' parameter scales), e^{+-x} are two hardware
// 2^x and sin, cos the Taylor series; otherwise the general form splits
// |x| log2(e) = k + f (exact exponent k) and reduces the angle by pi/2 (Cody
// and Waite's additive reduction).  With spin inversion the partner row
// b - W.t shares the sine/cosine of Im W.t through the angle-addition formulas
// and per-unit sin/cos of Im b.  Each thread multiplies its factors into
// running products with an exact binary exponent, renormalised every 8
// factors; after the last hidden tile of (tile, r) the four column groups'
// products are combined, multiplied by the leading factor
// c_r chi(g) chi_P e^{+-a.t} and summed over the rows of each sample
// (segmented warp reduction, then one ordered pass per warp).
//
// Every wait on an mbarrier has a time limit; on expiry the kernel sets
// NNQS_ETIMEOUT in the status word, lets the MMAs and copies it issued finish
// (bounded), frees its TMEM and returns.
#pragma once

#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace nnqs {

constexpr int kTcThreads = 512;              // 16 warps: 4 lane quadrants x 4 column groups
constexpr uint32_t kTmemCols = 512;          // two accumulators at columns 0 and 256
constexpr uint32_t kSmemBudget = 227 * 1024; // opt-in dynamic shared memory of one CTA
constexpr uint32_t kSmemFloor = 120 * 1024;  // requested at least: never two CTAs (and TMEM owners) per SM

struct TcPlan {
    int N, M, K, G, nsign, NS;
    int KD1;            // K extent of one split term: N rounded up to 16
    int MT, nmt, NC;    // hidden units per tile (multiple of 8), tiles, accumulator columns 2 MT
    int Mpad;           // nmt * MT
    int S, ntiles;      // samples per supertile, 128-row tiles per supertile
    int resident;       // all K * nmt images in shared memory
    int double_a;       // two A buffers
    uint32_t a_bytes, sub_bytes, img_bytes, img_stride, nimg;
    uint32_t off_a0, off_a1, off_b, off_sl, off_spins, off_at, off_xbuf, off_acc, off_bars, smem;
    uint32_t slice_bytes;   // (MT + 1) float4: bias slice and bounds
    // streaming: weights in two buffers at off_b, the slices of blocks j, j + 1,
    // j + 2 in a ring of three at off_sl (block j's slice is read by its
    // epilogue while block j + 2's image is already landing)
    bool ok;
};

// Image of one (RBM, hidden tile): NS split-term matrices [NC][KD1] bf16 in the
// core layout, then the bias slice [MT] float4 (Re b, Im b, sin Im b, cos Im b)
// and one float4 of bounds (max |Re b|, max |Im b|, 0, 0) over the slice.
__host__ __device__ __forceinline__ uint32_t tc_slice_off(const TcPlan &p) { return (uint32_t)p.NS * p.sub_bytes; }

__host__ __device__ inline int gcd_i(int a, int b) { while (b) { int t = a % b; a = b; b = t; } return a; }

TcPlan tc_plan(int N, int M, int G, int K, int nsign, int NS);

// byte offset of element (row, k) in the no-swizzle K-major core layout of a
// matrix with KD columns: 8-row x 16-byte core matrices, adjacent along K at
// 128 bytes, 8-row groups at KD/8 x 128 bytes
__host__ __device__ __forceinline__ uint32_t core_off(int row, int k, int KD)
{
    return (uint32_t)(row >> 3) * (uint32_t)(KD / 8) * 128u + (uint32_t)(k >> 3) * 128u + (uint32_t)(row & 7) * 16u +
           (uint32_t)(k & 7) * 2u;
}

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
constexpr float kLog2e = 1.44269504088896341f;

// Taylor series of sin and cos on |r| <= pi/4 (truncation below 2e-10)
__device__ __forceinline__ void sincos_taylor(float r, float &s, float &c)
{
    const float r2 = r * r;
    float ps = fmaf(r2, 2.75573192e-6f, -1.98412698e-4f);   // 1/9!, -1/7!
    ps = fmaf(r2, ps, 8.33333333e-3f);                        // 1/5!
    ps = fmaf(r2, ps, -1.66666667e-1f);                       // -1/3!
    s = fmaf(r * r2, ps, r);
    float pc = fmaf(r2, -2.75573192e-7f, 2.48015873e-5f);   // -1/10!, 1/8!
    pc = fmaf(r2, pc, -1.38888889e-3f);                       // -1/6!
    pc = fmaf(r2, pc, 4.16666667e-2f);                        // 1/4!
    pc = fmaf(r2, pc, -0.5f);
    c = fmaf(r2, pc, 1.0f);
}

// sin and cos of any x: x = q pi/2 + r with the quotient q rounded to nearest
// and pi/2 split into two floats (Cody and Waite's additive reduction), the
// Taylor series on r, and the quadrant's swap and signs.
__device__ __forceinline__ void sincos_cw(float x, float &s, float &c)
{
    const float q = rintf(x * 0.63661977236758134f);
    float r = fmaf(q, -1.57079637050628662109375f, x);
    r = fmaf(q, 4.37113900018624283e-8f, r);
    float sr, cr;
    sincos_taylor(r, sr, cr);
    const int qi = (int)q;
    const float ss = (qi & 1) ? cr : sr;
    const float cc = (qi & 1) ? sr : cr;
    s = (qi & 2) ? -ss : ss;
    c = ((qi + 1) & 2) ? -cc : cc;
}

// Running product of 2 cosh factors: value = (x + i y) 2^e (e integer-valued).
struct RP { float x, y, e; };

__device__ __forceinline__ void rp_renorm(RP &p)
{
    const int bits = __float_as_int(fmaxf(fabsf(p.x), fabsf(p.y)));
    const int k = ((bits >> 23) & 0xff) - 127;        // exponent of the larger part (-127 for 0 / denormals)
    const int kk = k < -126 ? -126 : (k > 126 ? 126 : k);
    const float s = __int_as_float((127 - kk) << 23);
    p.x *= s; p.y *= s; p.e += (float)kk;
}

__device__ __forceinline__ void rp_cmul(RP &p, float fr, float fi)
{
    const float nx = fmaf(p.x, fr, -p.y * fi);
    const float ny = fmaf(p.x, fi, p.y * fr);
    p.x = nx; p.y = ny;
}

// p *= 2 cosh(x + i y) given sin y, cos y: any x (exact exponent split)
__device__ __forceinline__ void rp_cosh(RP &p, float x, float sy, float cy)
{
    const float t = fabsf(x) * kLog2e;
    const float kf = floorf(t);
    const float e1 = tc::ex2_approx(t - kf);
    const float e2 = tc::ex2_approx(-t - kf);
    const float a = e1 + e2;
    const float b = copysignf(e1 - e2, x);
    rp_cmul(p, a * cy, b * sy);
    p.e += kf;
}

// p *= 2 cosh(x + i y) for |x| < 4: factor magnitude below 110
__device__ __forceinline__ void rp_cosh_small(RP &p, float x, float sy, float cy)
{
    const float t = x * kLog2e;
    const float e1 = tc::ex2_approx(t);
    const float e2 = tc::ex2_approx(-t);
    rp_cmul(p, (e1 + e2) * cy, (e1 - e2) * sy);
}

__device__ __forceinline__ RP rp_mul(RP a, RP b)
{
    RP c{fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x), a.e + b.e};
    rp_renorm(c);
    return c;
}

// RP times exp(L) as a scaled complex number
__device__ __forceinline__ sc<float> rp_times_exp(RP p, float Lx, float Ly)
{
    const float X = p.e + Lx * kLog2e;
    const float k = floorf(X);
    const float m = tc::ex2_approx(X - k);
    float s, c;
    sincos_cw(Ly, s, c);
    const float ux = m * c, uy = m * s;
    return sc_norm(sc<float>{p.x * ux - p.y * uy, p.x * uy + p.y * ux, (int)k});
}

// Factors of NH hidden units (compile time) of one row into the running
// products; re, im = W.t of the units, bs = their bias slice entries, bnd =
// the slice's bounds.  The fast form is taken when the whole warp qualifies.
template <int NH, int NSIGN>
__device__ __forceinline__ void epi_units(const float (&re)[16], const float (&im)[16], const float4 *bs, float4 bnd,
                                          RP &pp, RP &pm)
{
    float mx = 0.f, my = 0.f;
#pragma unroll
    for (int e = 0; e < NH; ++e) {
        mx = fmaxf(mx, fabsf(re[e]));
        my = fmaxf(my, fabsf(im[e]));
    }
    const bool ok = (mx + bnd.x < 4.0f) && (my + (NSIGN == 2 ? 0.f : bnd.y) < 0.78f);
    if (__all_sync(0xffffffffu, ok)) {
#pragma unroll
        for (int e = 0; e < NH; ++e) {
            const float4 b = bs[e];
            if (NSIGN == 2) {
                float s0, c0;
                sincos_taylor(im[e], s0, c0);
                const float p1 = b.z * c0, p2 = b.w * s0, p3 = b.w * c0, p4 = b.z * s0;
                rp_cosh_small(pp, b.x + re[e], p1 + p2, p3 - p4);
                rp_cosh_small(pm, b.x - re[e], p1 - p2, p3 + p4);
            } else {
                float sy, cy;
                sincos_taylor(b.y + im[e], sy, cy);
                rp_cosh_small(pp, b.x + re[e], sy, cy);
            }
            if ((e & 7) == 7) {
                rp_renorm(pp);
                if (NSIGN == 2) rp_renorm(pm);
            }
        }
    } else {
#pragma unroll
        for (int e = 0; e < NH; ++e) {
            const float4 b = bs[e];
            if (NSIGN == 2) {
                float s0, c0;
                sincos_cw(im[e], s0, c0);
                const float p1 = b.z * c0, p2 = b.w * s0, p3 = b.w * c0, p4 = b.z * s0;
                rp_cosh(pp, b.x + re[e], p1 + p2, p3 - p4);
                rp_cosh(pm, b.x - re[e], p1 - p2, p3 + p4);
            } else {
                float sy, cy;
                sincos_cw(b.y + im[e], sy, cy);
                rp_cosh(pp, b.x + re[e], sy, cy);
            }
            if ((e & 7) == 7) {
                rp_renorm(pp);
                if (NSIGN == 2) rp_renorm(pm);
            }
        }
    }
    rp_renorm(pp);
    if (NSIGN == 2) rp_renorm(pm);
}

// NH units (compile time) starting at column c0 of the accumulator at tb
template <int NH, int NSIGN>
__device__ __forceinline__ void epi_chunk(uint32_t tb, int MT, int c0, const float4 *bs, float4 bnd, RP &pp, RP &pm)
{
    float re[16], im[16];
#pragma unroll
    for (int c = 0; c < NH / 2; ++c) {
        tc::tmem_ld2(tb + (uint32_t)(c0 + 2 * c), re[2 * c], re[2 * c + 1]);
        tc::tmem_ld2(tb + (uint32_t)(MT + c0 + 2 * c), im[2 * c], im[2 * c + 1]);
    }
    tc::tmem_wait_ld();
    epi_units<NH, NSIGN>(re, im, bs, bnd, pp, pm);
}

// The thread's MQ units of the block (MQ > 0: compile time; MQ == 0: any even
// count, in chunks of 2)
template <int MQ, int NSIGN>
__device__ __forceinline__ void epi_block(uint32_t tb, int MT, int m0, const float4 *bs, float4 bnd, RP &pp, RP &pm)
{
    if constexpr (MQ > 0) {
        constexpr int A0 = MQ > 16 ? 16 : MQ;
        epi_chunk<A0, NSIGN>(tb, MT, m0, bs, bnd, pp, pm);
        if constexpr (MQ > 16) epi_chunk<MQ - 16, NSIGN>(tb, MT, m0 + 16, bs + 16, bnd, pp, pm);
    } else {
        const int mq = MT / 4;
        for (int c = 0; c < mq; c += 2) epi_chunk<2, NSIGN>(tb, MT, m0 + c, bs + c, bnd, pp, pm);
    }
}

struct TcArgs {
    TcPlan p;
    const uint16_t *bimg;     // [K][nmt] images (split weights + bias slice)
    const uint16_t *pinv;     // [G][KD1]: (T_g s)_j = s_{pinv[g][j]}; N marks padding
    int skip_first_copy;      // test hook: arm the first image barrier but issue no copy, so
                              // its bounded wait runs out (NNQS_ETIMEOUT) with nothing in flight
    float2 *theta_out;        // non-NULL: write theta' = W.t [n][K][G][M] instead of log psi
};

// theta' = W.t of this thread's row and MT/4 units of the accumulator at tb
// (no bias), to th[m0 .. m0 + MT/4) within the tile's units
__device__ __forceinline__ void theta_store(uint32_t tb, int MT, int m0, int mbase, int M, float2 *th)
{
    for (int c = 0; c < MT / 4; c += 2) {
        float r0, r1, i0, i1;
        tc::tmem_ld2(tb + (uint32_t)(m0 + c), r0, r1);
        tc::tmem_ld2(tb + (uint32_t)(MT + m0 + c), i0, i1);
        tc::tmem_wait_ld();
        const int m = mbase + m0 + c;
        if (th) {
            if (m < M) th[m] = make_float2(r0, i0);
            if (m + 1 < M) th[m + 1] = make_float2(r1, i1);
        }
    }
}

struct Blk {
    int64_t st;
    int t, r, mt;
};

__device__ __forceinline__ bool next_blk(Blk &b, const TcPlan &p, int64_t nsuper)
{
    if (++b.mt < p.nmt) return true;
    b.mt = 0;
    if (++b.r < p.K) return true;
    b.r = 0;
    if (++b.t < p.ntiles) return true;
    b.t = 0;
    b.st += gridDim.x;
    return b.st < nsuper;
}

// ---------------------------------------------------------------------------
// the fused GEMM + log-cosh + projection-sum kernel
// ---------------------------------------------------------------------------
template <int MQ, int NSIGN>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_logpsi_tc(DevModel<float> md, TcArgs ta, const uint64_t *__restrict__ cfg, int64_t n, double *__restrict__ out)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const TcPlan &P = ta.p;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3, cg = warp >> 2;
    const int N = P.N, G = P.G, KD1 = P.KD1, MT = P.MT;
    uint16_t *spins = reinterpret_cast<uint16_t *>(smem + P.off_spins);   // [S][N + 1] bf16 bits of s_j (0 = pad)
    cx<float> *atbuf = reinterpret_cast<cx<float> *>(smem + P.off_at);    // [2][K][128] a_r . t per row
    float *xbuf = reinterpret_cast<float *>(smem + P.off_xbuf);            // [3][128][6]
    sc<float> *accs = reinterpret_cast<sc<float> *>(smem + P.off_acc);     // [S]
    uint64_t *bar_b = reinterpret_cast<uint64_t *>(smem + P.off_bars);     // [2] images landed
    uint64_t *bar_m = bar_b + 2;                                           // [2] MMAs into accumulator i done
    uint32_t *tmem_base = reinterpret_cast<uint32_t *>(bar_b + 4);

    const int64_t nsuper = (n + P.S - 1) / P.S;
    const uint32_t idesc = tc::idesc_bf16(128, P.NC);
    const uint32_t sbo = (uint32_t)(KD1 / 8) * 128u;

    if (warp == 0) {
        tc::tmem_alloc(tmem_base, kTmemCols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&bar_b[0], 1);
        tc::mbar_init(&bar_b[1], 1);
        tc::mbar_init(&bar_m[0], 1);
        tc::mbar_init(&bar_m[1], 1);
        tc::mbar_fence_init();
    }
    for (int i = tid; i < P.S; i += kTcThreads) accs[i] = sc<float>{0.f, 0.f, 0};
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *tmem_base;

    // phases; the issuing thread's view of work in flight (for the abort drain)
    uint32_t ph_m0 = 0, ph_m1 = 0, ph_b0 = 0, ph_b1 = 0;
    bool mma_pend0 = false, mma_pend1 = false, copy_pend0 = false, copy_pend1 = false;
    bool timed_out = false;

    auto load_spins = [&](int64_t st) {
        const int64_t s0 = st * P.S;
        const int nsamp = (int)((n - s0) < P.S ? (n - s0) : P.S);
        for (int i = tid; i < P.S * (N + 1); i += kTcThreads) {
            const int sl = i / (N + 1), j = i - sl * (N + 1);
            uint16_t v = 0;
            if (sl < nsamp && j < N) v = spin_of(cfg + (s0 + sl) * md.nwords, j) > 0 ? 0x3F80 : 0xBF80;
            spins[i] = v;
        }
    };
    // A tile t of the current supertile's samples and a_r . t of its rows
    auto build_a = [&](int abuf, int atb, int t) {
        unsigned char *A = smem + (abuf ? P.off_a1 : P.off_a0);
        const int row = tid >> 2, c4 = tid & 3;
        const int qg = t * 128 + row;
        const int sl = qg / G, g = qg - sl * G;
        const uint16_t *sp = spins + sl * (N + 1);
        const uint16_t *pg = ta.pinv + (size_t)g * KD1;
        float ax[kMaxK], ay[kMaxK];
#pragma unroll
        for (int r = 0; r < kMaxK; ++r) { ax[r] = 0.f; ay[r] = 0.f; }
        for (int kc = c4; kc < KD1 / 8; kc += 4) {
            const uint4 ix = *reinterpret_cast<const uint4 *>(pg + kc * 8);
            const uint32_t iw[4] = {ix.x, ix.y, ix.z, ix.w};
            uint32_t w4[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const uint32_t v0 = sp[iw[h] & 0xffffu], v1 = sp[iw[h] >> 16];
                w4[h] = v0 | (v1 << 16);
                if (md.use_bias) {
                    const float t0 = __uint_as_float(v0 << 16), t1 = __uint_as_float(v1 << 16);
                    const int j0 = kc * 8 + 2 * h;
#pragma unroll
                    for (int r = 0; r < kMaxK; ++r) {
                        if (r < P.K) {
                            const cx<float> *ar = md.avec + (size_t)r * N;
                            if (j0 < N) { ax[r] = fmaf(t0, ar[j0].x, ax[r]); ay[r] = fmaf(t0, ar[j0].y, ay[r]); }
                            if (j0 + 1 < N) { ax[r] = fmaf(t1, ar[j0 + 1].x, ax[r]); ay[r] = fmaf(t1, ar[j0 + 1].y, ay[r]); }
                        }
                    }
                }
            }
            *reinterpret_cast<uint4 *>(A + core_off(row, kc * 8, KD1)) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
        }
#pragma unroll
        for (int r = 0; r < kMaxK; ++r) {
            if (r < P.K) {
                float x = ax[r], y = ay[r];
                x += __shfl_xor_sync(0xffffffffu, x, 1);
                y += __shfl_xor_sync(0xffffffffu, y, 1);
                x += __shfl_xor_sync(0xffffffffu, x, 2);
                y += __shfl_xor_sync(0xffffffffu, y, 2);
                if (c4 == 0) atbuf[(atb * P.K + r) * 128 + row] = cx<float>{x, y};
            }
        }
    };
    // smem address of the image block b uses (in buffer bi when streaming)
    auto img_smem = [&](const Blk &b, int bi) -> unsigned char * {
        const uint32_t img = P.resident ? (uint32_t)(b.r * P.nmt + b.mt) : (uint32_t)bi;
        return smem + P.off_b + img * P.img_stride;
    };
    // one elected thread: MMAs of block b into accumulator ai
    auto issue_mma = [&](const Blk &b, int abuf, int ai) {
        const uint32_t a0 = tc::smem_u32(smem + (abuf ? P.off_a1 : P.off_a0));
        const uint32_t b0 = tc::smem_u32(img_smem(b, ai));
        const uint32_t d = taddr + (uint32_t)ai * 256u;
        tc::fence_after_sync();
        for (int s = 0; s < P.NS; ++s)
            for (int kk = 0; kk < KD1 / 16; ++kk) {
                const uint64_t ad = tc::smem_desc(a0 + kk * 256u, 128u, sbo);
                const uint64_t bd = tc::smem_desc(b0 + s * P.sub_bytes + kk * 256u, 128u, sbo);
                tc::mma_bf16(d, ad, bd, idesc, (s | kk) ? 1u : 0u);
            }
        tc::mma_commit(&bar_m[ai]);
        if (ai) mma_pend1 = true; else mma_pend0 = true;
    };
    // streaming: image of block b (the jb-th block of this CTA) -> weights buffer
    // bi, slice ring entry jb mod 3
    auto issue_copy = [&](const Blk &b, int bi, int jb) {
        const uint16_t *src = ta.bimg + (size_t)(b.r * P.nmt + b.mt) * (P.img_bytes / 2);
        const uint32_t wbytes = tc_slice_off(P);
        tc::mbar_expect_tx(&bar_b[bi], wbytes + P.slice_bytes);
        tc::bulk_g2s(smem + P.off_b + (uint32_t)bi * P.img_stride, src, wbytes, &bar_b[bi]);
        tc::bulk_g2s(smem + P.off_sl + (uint32_t)(jb % 3) * P.slice_bytes, src + wbytes / 2, P.slice_bytes,
                     &bar_b[bi]);
        if (bi) copy_pend1 = true; else copy_pend0 = true;
    };
    auto wait_m = [&](int ai) -> bool {
        const bool ok = tc::mbar_wait_bounded(&bar_m[ai], ai ? ph_m1 : ph_m0);
        if (ok) {
            if (ai) { ph_m1 ^= 1; mma_pend1 = false; } else { ph_m0 ^= 1; mma_pend0 = false; }
        }
        return ok;
    };
    auto wait_b = [&](int bi) -> bool {
        const bool ok = tc::mbar_wait_bounded(&bar_b[bi], bi ? ph_b1 : ph_b0);
        if (ok) {
            if (bi) { ph_b1 ^= 1; copy_pend1 = false; } else { ph_b0 ^= 1; copy_pend0 = false; }
        }
        return ok;
    };

    Blk cur{(int64_t)blockIdx.x, 0, 0, 0};
    if (cur.st < nsuper) {
        // ---- prologue: spins and A of the first tile, images, the first MMAs ----
        load_spins(cur.st);
        __syncthreads();
        build_a(0, 0, 0);
        tc::fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            bool ok = true;
            if (ta.skip_first_copy) {
                tc::mbar_expect_tx(&bar_b[0], P.img_bytes);
                ok = wait_b(0);
            } else if (P.resident) {
                tc::mbar_expect_tx(&bar_b[0], P.nimg * P.img_bytes);
                for (uint32_t i = 0; i < P.nimg; ++i)
                    tc::bulk_g2s(smem + P.off_b + i * P.img_stride, ta.bimg + (size_t)i * (P.img_bytes / 2),
                                 P.img_bytes, &bar_b[0]);
                copy_pend0 = true;
                ok = wait_b(0);
            } else {
                issue_copy(cur, 0, 0);
                Blk b1 = cur;
                if (next_blk(b1, P, nsuper)) issue_copy(b1, 1, 1);
                ok = wait_b(0);
            }
            if (ok) issue_mma(cur, 0, 0);
            else timed_out = true;
        }
        int abuf = 0, atb = 0;
        int j = 0;
        bool aborted = __syncthreads_or(timed_out);
        RP pp{1.f, 0.f, 0.f}, pm{1.f, 0.f, 0.f};
        while (!aborted) {
            Blk nxt = cur;
            const bool has_next = next_blk(nxt, P, nsuper);
            const bool new_tile = has_next && (nxt.t != cur.t || nxt.st != cur.st);
            const int ai = j & 1;
            int abuf_n = abuf, atb_n = atb;
            bool waited = false;
            if (new_tile) {
                abuf_n = P.double_a ? abuf ^ 1 : abuf;
                atb_n = atb ^ 1;
                if (!P.double_a) {
                    // the single A buffer is free once the MMAs of block j are done
                    waited = true;
                    if (!wait_m(ai)) timed_out = true;
                    if (__syncthreads_or(timed_out)) { aborted = true; break; }
                }
                if (nxt.st != cur.st) {
                    load_spins(nxt.st);
                    __syncthreads();
                }
                build_a(abuf_n, atb_n, nxt.t);
                tc::fence_proxy_async_smem();
                // A(next) complete before its MMAs are issued
                __syncthreads();
            }
            // (accumulator (j + 1) & 1 was released by every thread at the end
            // of iteration j - 1)
            if (has_next && tid == 0) {
                bool ok = true;
                if (!P.resident) ok = wait_b((j + 1) & 1);
                if (ok) issue_mma(nxt, abuf_n, (j + 1) & 1);
                else timed_out = true;
            }
            // a thread whose wait runs out skips the epilogue; the barrier at
            // the end of the iteration then aborts the CTA
            const bool ready = __all_sync(0xffffffffu, waited || wait_m(ai));   // warp-uniform
            if (!ready) timed_out = true;
            tc::fence_after_sync();
            if (tid == 0 && !P.resident && has_next && ready) {
                Blk n2 = nxt;
                if (next_blk(n2, P, nsuper)) issue_copy(n2, ai, j + 2);   // buffer ai: block j's MMAs are done
            }

            // ---- epilogue of block j: this thread's row and quarter of the tile's hidden units ----
            if (ready) {
                const int m0 = cg * (MT / 4);
                const uint32_t tb = taddr + (uint32_t)ai * 256u + ((uint32_t)(quad * 32) << 16);
                if (ta.theta_out) {
                    const int qg = cur.t * 128 + quad * 32 + lane;
                    const int sl = qg / G, g = qg - sl * G;
                    const int64_t s = cur.st * P.S + sl;
                    float2 *th = s < n ? ta.theta_out + ((s * P.K + cur.r) * (int64_t)G + g) * P.M : nullptr;
                    theta_store(tb, MT, m0, cur.mt * MT, P.M, th);
                } else {
                    const float4 *slice = reinterpret_cast<const float4 *>(
                        P.resident ? img_smem(cur, ai) + tc_slice_off(P) : smem + P.off_sl + (uint32_t)(j % 3) * P.slice_bytes);
                    epi_block<MQ, NSIGN>(tb, MT, m0, slice + m0, slice[MT], pp, pm);
                }
            }
            tc::fence_before_sync();

            // ---- after the last hidden tile of (tile, r): row terms -> per-sample sums ----
            if (cur.mt == P.nmt - 1 && !ta.theta_out) {
                const int row = quad * 32 + lane;
                if (cg > 0) {
                    float *xb = xbuf + ((cg - 1) * 128 + row) * 6;
                    xb[0] = pp.x; xb[1] = pp.y; xb[2] = pp.e; xb[3] = pm.x; xb[4] = pm.y; xb[5] = pm.e;
                }
                __syncthreads();
                if (cg == 0) {
                    for (int c = 0; c < 3; ++c) {
                        const float *xb = xbuf + (c * 128 + row) * 6;
                        pp = rp_mul(pp, RP{xb[0], xb[1], xb[2]});
                        if (NSIGN == 2) pm = rp_mul(pm, RP{xb[3], xb[4], xb[5]});
                    }
                    // padded hidden units contributed 2cosh(0) = 2 each
                    const float npad = (float)(P.Mpad - P.M);
                    pp.e -= npad;
                    pm.e -= npad;
                    const int64_t s0 = cur.st * P.S;
                    const int nsamp = (int)((n - s0) < P.S ? (n - s0) : P.S);
                    const int qg = cur.t * 128 + row;
                    const int sl = qg / G, g = qg - sl * G;
                    const bool valid = sl < nsamp;
                    sc<float> term{0.f, 0.f, 0};
                    if (valid) {
                        const cx<float> at = atbuf[(atb * P.K + cur.r) * 128 + row];
                        const cx<float> lc = md.logc[cur.r];
                        const float chi = md.chi[g];
                        sc<float> tp = rp_times_exp(pp, lc.x + at.x, lc.y + at.y);
                        tp.x *= chi; tp.y *= chi;
                        term = tp;
                        if (NSIGN == 2) {
                            sc<float> tm = rp_times_exp(pm, lc.x - at.x, lc.y - at.y);
                            const float c2 = md.chiP < 0 ? -chi : chi;
                            tm.x *= c2; tm.y *= c2;
                            term = sc_add(term, tm);
                        }
                    }
                    // segmented reduction over lanes of the same sample (keys non-decreasing)
                    const int key = valid ? sl : -1;
                    sc<float> v = term;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const sc<float> w{__shfl_down_sync(0xffffffffu, v.x, o), __shfl_down_sync(0xffffffffu, v.y, o),
                                          __shfl_down_sync(0xffffffffu, v.e, o)};
                        const int kw = __shfl_down_sync(0xffffffffu, key, o);
                        if (lane + o < 32 && kw == key) v = sc_add(v, w);
                    }
                    const int kprev = __shfl_up_sync(0xffffffffu, key, 1);
                    const bool head = key >= 0 && (lane == 0 || kprev != key);
                    // one warp at a time adds its segment heads (distinct keys within a warp)
                    for (int w = 0; w < 4; ++w) {
                        if (quad == w && head) accs[key] = sc_add(accs[key], v);
                        tc::named_sync(1, 128);
                    }
                    // last block of the supertile: log of every sample's sum
                    if (!has_next || nxt.st != cur.st) {
                        for (int i = row; i < nsamp; i += 128) {
                            const sc<float> tot = accs[i];
                            double lre, lim;
                            if (!sc_finite(tot)) {
                                flag_range(md.status);
                                lre = nan(""); lim = nan("");
                            } else if (sc_zero(tot)) {
                                lre = -INFINITY; lim = 0.0;
                            } else {
                                const double x = (double)tot.x, y = (double)tot.y;
                                lre = log(hypot(x, y)) + tot.e * 0.69314718055994530942;
                                lim = atan2(y, x);
                            }
                            out[2 * (s0 + i)] = lre;
                            out[2 * (s0 + i) + 1] = lim;
                        }
                        for (int i = row; i < P.S; i += 128) accs[i] = sc<float>{0.f, 0.f, 0};
                    }
                }
                pp = RP{1.f, 0.f, 0.f};
                pm = RP{1.f, 0.f, 0.f};
            }
            if (__syncthreads_or(timed_out)) { aborted = true; break; }
            if (!has_next) break;
            cur = nxt;
            if (new_tile) { abuf = abuf_n; atb = atb_n; }
            ++j;
        }
        if (aborted) {
            if (tid == 0) {
                atomicExch(md.status, -4);
                // let the MMAs and copies this thread issued finish (bounded)
                if (mma_pend0) (void)tc::mbar_wait_bounded(&bar_m[0], ph_m0);
                if (mma_pend1) (void)tc::mbar_wait_bounded(&bar_m[1], ph_m1);
                if (copy_pend0) (void)tc::mbar_wait_bounded(&bar_b[0], ph_b0);
                if (copy_pend1) (void)tc::mbar_wait_bounded(&bar_b[1], ph_b1);
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, kTmemCols);
}

// Launch of one (MQ, NSIGN) instantiation (each in its own translation unit).
template <int MQ, int NSIGN>
cudaError_t launch_tc_variant(const DevModel<float> &md, const TcArgs &ta, const uint64_t *cfg, int64_t n,
                              double *out, int grid, cudaStream_t st)
{
    cudaError_t err =
        cudaFuncSetAttribute(k_logpsi_tc<MQ, NSIGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ta.p.smem);
    if (err != cudaSuccess) return err;
    k_logpsi_tc<MQ, NSIGN><<<grid, kTcThreads, ta.p.smem, st>>>(md, ta, cfg, n, out);
    return cudaGetLastError();
}

#define NNQS_TC_INSTANTIATE(MQ)                                                                                    \
    template cudaError_t launch_tc_variant<MQ, 1>(const DevModel<float> &, const TcArgs &, const uint64_t *, int64_t, \
                                                  double *, int, cudaStream_t);                                      \
    template cudaError_t launch_tc_variant<MQ, 2>(const DevModel<float> &, const TcArgs &, const uint64_t *, int64_t, \
                                                  double *, int, cudaStream_t);

}  // namespace nnqs
