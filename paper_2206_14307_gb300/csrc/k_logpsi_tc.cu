// k_logpsi_tc.cu -- host side of the tensor-core log psi (see k_logpsi_tc.cuh):
// the tiling plan, the device images of the split weights and bias slices,
// and the choice of the compiled epilogue variant.
#include "k_logpsi_tc.cuh"

#include <cuda_bf16.h>
#include <cstdlib>

namespace nnqs {

static uint32_t up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

TcPlan tc_plan(int N, int M, int G, int K, int nsign, int NS)
{
    TcPlan p{};
    p.N = N; p.M = M; p.K = K; p.G = G; p.nsign = nsign; p.NS = NS;
    p.KD1 = (N + 15) / 16 * 16;
    p.S = 128 / gcd_i(G, 128);
    p.ntiles = p.S * G / 128;
    p.a_bytes = 128u * p.KD1 * 2u;
    const int M8 = (M + 7) / 8 * 8;
    p.ok = false;
    for (int nmt = (M8 + 127) / 128; nmt <= M8 / 8 && !p.ok; ++nmt) {
        const int MT = ((M8 + nmt - 1) / nmt + 7) / 8 * 8;
        if (MT > 128) continue;
        p.nmt = nmt; p.MT = MT; p.NC = 2 * MT; p.Mpad = nmt * MT;
        p.sub_bytes = (uint32_t)p.NC * p.KD1 * 2u;
        p.img_bytes = (uint32_t)NS * p.sub_bytes + (uint32_t)(MT + 1) * 16u;   // + bias slice and bounds
        p.nimg = (uint32_t)K * nmt;
        const uint32_t misc = up((uint32_t)p.S * (N + 1) * 2u, 16) + 2u * K * 128u * 8u + 3u * 128u * 24u +
                              up((uint32_t)p.S * 12u, 16) + 128u + 4096u;
        const uint32_t a1 = up(p.a_bytes, 1024), b1 = up(p.img_bytes, 1024);
        p.img_stride = b1;
        p.slice_bytes = (uint32_t)(MT + 1) * 16u;
        const uint32_t ring = 3u * p.slice_bytes;
        const uint32_t cand[3][3] = {{1, 1, 2 * a1 + p.nimg * b1},
                                     {0, 1, 2 * a1 + 2 * b1 + ring},
                                     {0, 0, a1 + 2 * b1 + ring}};
        for (int c = 0; c < 3 && !p.ok; ++c) {
            if (cand[c][2] + misc <= kSmemBudget) {
                p.resident = (int)cand[c][0];
                p.double_a = (int)cand[c][1];
                p.ok = true;
            }
        }
    }
    if (!p.ok) return p;
    uint32_t o = 0;
    p.off_a0 = o; o += up(p.a_bytes, 1024);
    p.off_a1 = p.double_a ? o : p.off_a0; if (p.double_a) o += up(p.a_bytes, 1024);
    p.off_b = o; o += (p.resident ? p.nimg : 2u) * p.img_stride;
    p.off_sl = o; o += p.resident ? 0u : 3u * p.slice_bytes;
    p.off_spins = o; o += up((uint32_t)p.S * (N + 1) * 2u, 16);
    p.off_at = o; o += 2u * K * 128u * 8u;
    p.off_xbuf = o; o += 3u * 128u * 24u;
    p.off_acc = o; o += up((uint32_t)p.S * 12u, 16);
    p.off_bars = o; o += 128;
    p.smem = up(o, 1024) < kSmemFloor ? kSmemFloor : up(o, 1024);
    p.ok = p.smem <= kSmemBudget && p.KD1 <= 256 && p.S <= 128;
    return p;
}

// ---------------------------------------------------------------------------
// Images [K][nmt], each: NS split-term matrices [NC][KD1] (core layout; row
// n < MT is Re W_m, row MT + n' is Im W_m, m = tile MT + n mod MT; zero past M
// and past N), then the bias slice [MT] float4 (Re b, Im b, sin Im b, cos Im b;
// zero bias past M) and the slice's bounds (max |Re b|, max |Im b|, 0, 0).
// ---------------------------------------------------------------------------
__global__ void k_bimg(const double *__restrict__ par, TcPlan p, uint16_t *__restrict__ img, int use_bias)
{
    const int N = p.N, M = p.M, NC = p.NC, KD1 = p.KD1, MT = p.MT;
    const int64_t P1 = 1 + N + M + (int64_t)M * N;
    const int64_t per_sub = (int64_t)NC * KD1;
    const int64_t img_el = p.img_bytes / 2;   // uint16 elements per image
    const int64_t total = per_sub * p.NS * p.nimg;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t sub = q / per_sub;                 // (r * nmt + t) * NS + split
        const int split = (int)(sub % p.NS);
        const int rt = (int)(sub / p.NS);
        const int r = rt / p.nmt, t = rt - r * p.nmt;
        const int64_t rem = q - sub * per_sub;
        const int n = (int)(rem / KD1), k = (int)(rem - (int64_t)n * KD1);
        const int m = t * MT + (n < MT ? n : n - MT);
        const int part = n < MT ? 0 : 1;
        float v = 0.f;
        if (m < M && k < N) {
            const double w = par[2 * (r * P1 + 1 + N + M + (int64_t)m * N + k) + part];
            double rest = w;  // successive bf16 terms of w
            float term = 0.f;
            for (int u = 0; u <= split; ++u) {
                term = __bfloat162float(__float2bfloat16_rn((float)rest));
                rest -= (double)term;
            }
            v = term;
        }
        const __nv_bfloat16 b = __float2bfloat16_rn(v);
        img[rt * img_el + (int64_t)split * per_sub + core_off(n, k, KD1) / 2] = *reinterpret_cast<const uint16_t *>(&b);
    }
    // bias slices: one thread per (image, unit); the bounds by the image's last thread
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < (int64_t)p.nimg * (MT + 1);
         q += (int64_t)gridDim.x * blockDim.x) {
        const int rt = (int)(q / (MT + 1)), u = (int)(q - (int64_t)rt * (MT + 1));
        const int r = rt / p.nmt, t = rt - r * p.nmt;
        float4 *slice = reinterpret_cast<float4 *>(img + rt * img_el + (int64_t)p.NS * per_sub);
        if (u < MT) {
            const int m = t * MT + u;
            float4 v = make_float4(0.f, 0.f, 0.f, 1.f);
            if (m < M && use_bias) {
                const double bx = par[2 * (r * P1 + 1 + N + m)], by = par[2 * (r * P1 + 1 + N + m) + 1];
                v = make_float4((float)bx, (float)by, (float)sin(by), (float)cos(by));
            }
            slice[u] = v;
        } else {
            float mx = 0.f, my = 0.f;
            if (use_bias)
                for (int uu = 0; uu < MT; ++uu) {
                    const int m = t * MT + uu;
                    if (m < M) {
                        mx = fmaxf(mx, fabsf((float)par[2 * (r * P1 + 1 + N + m)]));
                        my = fmaxf(my, fabsf((float)par[2 * (r * P1 + 1 + N + m) + 1]));
                    }
                }
            slice[MT] = make_float4(mx, my, 0.f, 0.f);
        }
    }
}

// Test hook: an environment variable set to 1 (read at every launch; unset in
// normal use).
static int test_hook_enabled(const char *name)
{
    const char *v = getenv(name);
    return v && v[0] == '1' && v[1] == 0;
}

bool tc_supported(int N, int M, int G, int K, int nsign, int NS)
{
    if (M > kMaxM || NS < 2 || NS > 3 || K > kMaxK) return false;
    return tc_plan(N, M, G, K, nsign, NS).ok;
}

size_t tc_bimg_bytes(int N, int M, int G, int K, int nsign, int NS)
{
    const TcPlan p = tc_plan(N, M, G, K, nsign, NS);
    return (size_t)p.nimg * p.img_bytes;
}

size_t tc_pinv_bytes(int N, int G) { return (size_t)G * ((N + 15) / 16 * 16) * sizeof(uint16_t); }

void tc_pinv_table(const uint8_t *perm, int N, int G, uint16_t *out)
{
    const int KD1 = (N + 15) / 16 * 16;
    for (int g = 0; g < G; ++g) {
        for (int j = 0; j < KD1; ++j) out[(size_t)g * KD1 + j] = (uint16_t)N;
        for (int i = 0; i < N; ++i) out[(size_t)g * KD1 + perm[(size_t)g * N + i]] = (uint16_t)i;
    }
}

cudaError_t launch_bimg(const double *params, int N, int M, int G, int K, int nsign, int NS, int use_bias,
                        uint16_t *img, cudaStream_t st)
{
    const TcPlan p = tc_plan(N, M, G, K, nsign, NS);
    k_bimg<<<1024, 256, 0, st>>>(params, p, img, use_bias);
    return cudaGetLastError();
}

// the epilogue variants compiled with a fixed unit count per thread (one
// translation unit each); other counts use the generic MQ = 0 variant
template <int MQ, int NSIGN>
cudaError_t launch_tc_variant(const DevModel<float> &md, const TcArgs &ta, const uint64_t *cfg, int64_t n,
                              double *out, int grid, cudaStream_t st);

template <int NSIGN>
static cudaError_t launch_by_mq(int mq, const DevModel<float> &md, const TcArgs &ta, const uint64_t *cfg, int64_t n,
                                double *out, int grid, cudaStream_t st)
{
    switch (mq) {
    case 4: return launch_tc_variant<4, NSIGN>(md, ta, cfg, n, out, grid, st);
    case 8: return launch_tc_variant<8, NSIGN>(md, ta, cfg, n, out, grid, st);
    case 10: return launch_tc_variant<10, NSIGN>(md, ta, cfg, n, out, grid, st);
    case 16: return launch_tc_variant<16, NSIGN>(md, ta, cfg, n, out, grid, st);
    case 18: return launch_tc_variant<18, NSIGN>(md, ta, cfg, n, out, grid, st);
    case 20: return launch_tc_variant<20, NSIGN>(md, ta, cfg, n, out, grid, st);
    case 26: return launch_tc_variant<26, NSIGN>(md, ta, cfg, n, out, grid, st);
    case 32: return launch_tc_variant<32, NSIGN>(md, ta, cfg, n, out, grid, st);
    default: return launch_tc_variant<0, NSIGN>(md, ta, cfg, n, out, grid, st);
    }
}

cudaError_t launch_log_psi_tc(const DevModel<float> &md, const uint16_t *bimg, const uint16_t *pinv, int NS,
                              const uint64_t *cfg, int64_t n, double *out, int nsm, cudaStream_t st,
                              float2 *theta_out)
{
    if (n <= 0) return cudaSuccess;
    TcArgs ta;
    ta.p = tc_plan(md.N, md.M, md.G, md.K, md.nsign, NS);
    if (!ta.p.ok) return cudaErrorInvalidValue;
    ta.bimg = bimg;
    ta.pinv = pinv;
    ta.theta_out = theta_out;
    ta.skip_first_copy = test_hook_enabled("NNQS_TEST_SKIP_TC_COPY");
    const int64_t nsuper = (n + ta.p.S - 1) / ta.p.S;
    const int grid = (int)(nsuper < nsm ? nsuper : nsm);
    const int mq = ta.p.MT / 4;
    return md.nsign == 2 ? launch_by_mq<2>(mq, md, ta, cfg, n, out, grid, st)
                         : launch_by_mq<1>(mq, md, ta, cfg, n, out, grid, st);
}

NNQS_TC_INSTANTIATE(0)

}  // namespace nnqs
