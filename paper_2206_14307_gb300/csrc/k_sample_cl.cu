// k_sample_cl.cu -- Metropolis sampler (Sec. 3.2) with each chain's cache in the
// shared memory of a thread-block cluster (FP32).
//
// Same chain, proposals, acceptance rule and cache arithmetic as k_sample.cu:
// for every (row, sign) pair t of the projected sum the chain keeps
// p_m = e^theta/(2cosh theta) per hidden unit and the pair's term; a proposed
// exchange of an up site u and a down site d changes pair t by
// exp(sigma C_ud) prod_m (1 + p_m T_m), T_m = exp(-4 sigma (W_m,g(u) - W_m,g(d))) - 1.
//
// Here the pairs of one chain are split over the CL CTAs of a cluster (one
// CTA per SM), each holding its pairs' p and the per-site tables exp(-+4W)
// in shared memory (no L1/L2 round trip per proposal).  A step is: the proposal (every CTA draws the same Philox
// words), one pass over the CTA's pairs, the CTA's sums of old and new terms,
// an exchange of those sums through distributed shared memory and one cluster
// barrier, and the acceptance decision (every CTA adds the CL partial sums in
// rank order and reaches the same decision).  An accepted exchange is applied
// in place -- p' = p (1 + T)/(1 + p T), term' = term * ratio -- at the start of
// the next step's pass, so no speculative second buffer is needed and p is
// read once per step.
#include "common.cuh"
#include "f2.cuh"
#include "kernels.h"

namespace nnqs {

constexpr int kCGL = 8;              // lanes per pair group
constexpr int kClMaxThreads = 640;   // at most 20 warps

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_id_x()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_count_x()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// store to the shared memory of CTA `rank` of the cluster at the address that
// `local` has in this CTA
__device__ __forceinline__ void st_cluster_f32(const void *local, uint32_t rank, float v)
{
    uint32_t a = (uint32_t)__cvta_generic_to_shared(local), ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(ra), "f"(v) : "memory");
}

__device__ __forceinline__ float rcp_nr_f(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return fmaf(r, fmaf(-x, r, 1.0f), r);
}

// k-th set bit (0-based) of a multi-word mask
__device__ __forceinline__ int kth_set(const uint64_t *w, int nwords, int k)
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

struct ClPlan {
    int CL;        // CTAs per cluster (1, 2, 4, 8)
    int TP;        // pairs per CTA
    int threads;   // threads per CTA (multiple of 32)
    size_t smem;   // dynamic shared memory per CTA
};

// Shared memory of one CTA: site factor rows u = exp(-+4W) [K][2][N] and the
// chain's q rows [TP] (64 MPL bytes a row, see below), per pair the term,
// term x prod_m p_m and their values after an accepted proposal, site
// prefactors e^{+-Cs} and the products of u over the units e^{-+4 CS}
// [K][2][N] each, exchange slots [2][CL][8], a flag byte per pair.
static size_t cl_smem(const DevModel<float> &md, int TP, int CL, int MPL)
{
    return (size_t)(md.K * 2 * md.N + TP) * 64 * MPL + 4 * (size_t)TP * sizeof(sc<float>) +
           2 * (size_t)md.K * 2 * md.N * sizeof(sc<float>) + 2 * (size_t)CL * 8 * sizeof(float) + (size_t)TP;
}

// Sums over the warp of two scaled complex numbers: v = (sum a, sum b) as plain
// FP32 numbers times 2^e, e the largest exponent in the warp (zeros ignored).
__device__ __forceinline__ int warp_scaled(sc<float> a, sc<float> b, float (&v)[4])
{
    const int ea = sc_zero(a) ? -(1 << 28) : a.e, eb = sc_zero(b) ? -(1 << 28) : b.e;
    const int e = __reduce_max_sync(0xffffffffu, ea > eb ? ea : eb);
    const float fa = pow2i<float>(a.e - e), fb = pow2i<float>(b.e - e);
    v[0] = a.x * fa; v[1] = a.y * fa; v[2] = b.x * fb; v[3] = b.y * fb;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    return e;
}

// units per lane of a width M (the kernel's variants)
static int cl_mpl(int M)
{
    const int need = (M + kCGL - 1) / kCGL;
    return need <= 2 ? 2 : need <= 4 ? 4 : need <= 9 ? 9 : 16;
}

constexpr size_t kClSmemLimit = 224 * 1024;   // dynamic shared memory of one CTA (static part below 3 KB)

// The smallest cluster whose CTAs hold the chain's cache; CL = 0 if none does.
static ClPlan cl_plan(const DevModel<float> &md, int force_cl)
{
    ClPlan p{0, 0, 0, 0};
    const int nrs = md.K * md.G * md.nsign;
    for (int CL = 1; CL <= 8; CL *= 2) {
        if (force_cl > 0 && CL != force_cl) continue;
        const int TP = (nrs + CL - 1) / CL;
        const size_t s = cl_smem(md, TP, CL, cl_mpl(md.M));
        if (s <= kClSmemLimit) {
            p.CL = CL; p.TP = TP; p.smem = s;
            break;
        }
    }
    if (!p.CL) return p;
    // warps: the count in 8..20 that leaves the fewest idle pair groups
    int best_w = 16, best_waste = 1 << 30;
    for (int w = 20; w >= 8; --w) {
        const int slots = 4 * w;
        const int waste = (p.TP + slots - 1) / slots * slots - p.TP;
        if (waste < best_waste) { best_waste = waste; best_w = w; }
    }
    p.threads = 32 * best_w;
    return p;
}

// Row layout of the site factor rows and the chain's q rows: lane gl of a
// pair group owns the units m = gl + 8 j (j < MPL); the units (j, j + 1) of
// even j < MPL - 1 sit in one float4 (x_j, x_j+1, y_j, y_j+1) at float4 index
// (j / 2) 8 + gl, so that a group reads 128 contiguous bytes per step; for odd
// MPL the last unit is a float2 at float2 index (MPL - 1) 8 + gl.  A row is
// 8 MPL complex numbers (64 MPL bytes).
template <int MPL> __device__ __forceinline__ void row_offsets(int j, int gl, int &ore, int &oim)
{
    if (j < MPL - (MPL & 1)) {
        const int base = ((j >> 1) * 8 + gl) * 4;
        ore = base + (j & 1);
        oim = base + 2 + (j & 1);
    } else {
        const int base = ((MPL - 1) * 8 + gl) * 2;
        ore = base;
        oim = base + 1;
    }
}

__device__ __forceinline__ void lds64(const void *p, float &x, float &y)
{
    const uint32_t addr = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(x), "=f"(y) : "r"(addr));
}
__device__ __forceinline__ void sts128(void *p, f2 a, f2 b)
{
    const uint32_t addr = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("st.shared.v2.u64 [%0], {%1, %2};" ::"r"(addr), "l"(a), "l"(b) : "memory");
}

template <int MPL>
__global__ void __launch_bounds__(kClMaxThreads, 1)
    k_sample_cl(DevModel<float> md, uint64_t seed, int n_chains, int n_per_chain, int n_skip, int n_burn,
                uint64_t *__restrict__ cfg_out, float *__restrict__ acc_out, int CL, int TP)
{
    constexpr int NG = 32 / kCGL;
    constexpr int NPAIR = MPL / 2, SGL = MPL & 1;
    constexpr int RF4 = 4 * MPL;   // float4 per row
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ float s_sm[kMaxN];
    __shared__ uint64_t upm[kMaxWords], dnm[kMaxWords];
    __shared__ sc<float> wold[32], wnew[32];
    __shared__ int site_u, site_d, pend, pend_u, pend_d;
    __shared__ uint32_t wnext[3];
    __shared__ float u_sh;

    const int M = md.M, N = md.N;
    float4 *s4 = reinterpret_cast<float4 *>(smem);                              // [K][2][N] rows of u = exp(-+4W)
    float4 *qc = s4 + (size_t)md.K * 2 * N * RF4;                               // [TP] rows of q = (1 - p)/p
    sc<float> *term = reinterpret_cast<sc<float> *>(qc + (size_t)TP * RF4);     // [TP] the pair's term
    sc<float> *tpr = term + TP;                                                 // [TP] term x prod_m p_m
    sc<float> *nterm = tpr + TP;                                                // [TP] prod (q + U), then the new term
    sc<float> *ntpr = nterm + TP;                                               // [TP] tpr after an accepted proposal
    sc<float> *es = ntpr + TP;                                                  // [K][2][N] site prefactors e^{+-Cs}
    sc<float> *ec = es + (size_t)md.K * 2 * N;                                  // [K][2][N] prod_m u_m = e^{-+4 CS}
    float *xch = reinterpret_cast<float *>(ec + (size_t)md.K * 2 * N);          // [2][CL][8]
    // [TP] per pair: some |q| of the pair may exceed 2^12, so that its running
    // products are renormalised after every unit pair
    uint8_t *bigf = reinterpret_cast<uint8_t *>(xch + 2 * CL * 8);

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int grp = lane / kCGL, gl = lane % kCGL, gbase = grp * kCGL;
    const int slot = warp * NG + grp, nslots = nwarps * NG;
    const int nrs = md.K * md.G * md.nsign;
    const uint32_t rank = cluster_rank();
    const int t0 = (int)rank * TP;
    const int ntp = t0 >= nrs ? 0 : (nrs - t0 < TP ? nrs - t0 : TP);
    uint32_t gstep = 0;   // steps of this cluster over all its chains (parity of the exchange slots)
    {
        float *s4f = reinterpret_cast<float *>(s4);
        for (int q = threadIdx.x; q < md.K * 2 * N * 8 * MPL; q += blockDim.x) {
            const int row = q / (8 * MPL), w = q - row * 8 * MPL;   // row = (r * 2 + half) * N + k
            const int l = w % 8, j = w / 8, m = l + 8 * j;
            const cx<float> v = m < M ? md.S4[(size_t)row * md.Mp + m] : cx<float>{1.f, 0.f};
            int ore, oim;
            row_offsets<MPL>(j, l, ore, oim);
            s4f[(size_t)row * 8 * MPL * 2 + ore] = v.x;
            s4f[(size_t)row * 8 * MPL * 2 + oim] = v.y;
        }
        for (int q = threadIdx.x; q < md.K * 2 * N; q += blockDim.x) {
            es[q] = md.ES[q];
            const int rk = q / (2 * N), o = (q / N) & 1, k = q % N;
            const cx<float> c = md.CS[(size_t)rk * N + k];
            const float f = o ? 4.f : -4.f;
            ec[q] = sc_norm(sc_exp(cx<float>{f * c.x, f * c.y}));
        }
    }
    __syncthreads();

    for (int chain = (int)cluster_id_x(); chain < n_chains; chain += (int)cluster_count_x()) {
        const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32) ^ (uint32_t)chain;

        // ---- initial configuration: Fisher-Yates shuffle of N/2 ups (same in every CTA) ----
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
                s_sm[i] = (float)s8[i];
                if (s8[i] > 0) upm[i >> 6] |= 1ull << (i & 63);
                else dnm[i >> 6] |= 1ull << (i & 63);
            }
        }
        __syncthreads();

        // ---- fresh cache of this CTA's pairs: q = 1/p - 1 per unit, the term
        //      and term x prod_m p_m per pair ----
        for (int tb = 0; tb < ntp; tb += nslots) {
            const int tl0 = tb + slot;
            const bool active = tl0 < ntp;
            const int tl = active ? tl0 : 0;
            const int t = t0 + tl;
            const int row = md.nsign == 2 ? t >> 1 : t;
            const int sg = t - row * md.nsign;
            const int sign = sg ? -1 : 1;
            const int r = row / md.G, g = row - r * md.G;
            const uint8_t *pg = md.perm + (size_t)g * N;
            const cx<float> *Wr = md.Wt + (size_t)r * N * M;
            cx<float> thp[MPL];
#pragma unroll
            for (int j = 0; j < MPL; ++j) thp[j] = cx<float>{0.f, 0.f};
            for (int i = 0; i < N; ++i) {
                const cx<float> *wk = Wr + (size_t)pg[i] * M;
                const float si = s_sm[i];
#pragma unroll
                for (int j = 0; j < MPL; ++j) {
                    const int m = gl + kCGL * j;
                    if (m < M) { const cx<float> w = wk[m]; thp[j].x += si * w.x; thp[j].y += si * w.y; }
                }
            }
            cx<float> at{0.f, 0.f};
            if (md.use_bias) {
                const cx<float> *ar = md.avec + (size_t)r * N;
                for (int i = gl; i < N; i += kCGL) { const cx<float> a = ar[pg[i]]; at.x += s_sm[i] * a.x; at.y += s_sm[i] * a.y; }
#pragma unroll
                for (int o = kCGL / 2; o > 0; o >>= 1) { at.x += shfl_x(at.x, o); at.y += shfl_x(at.y, o); }
            }
            sc<float> prod{1.f, 0.f, 0}, pp{1.f, 0.f, 0};
            bool big = false;
            float *qf = reinterpret_cast<float *>(qc + (size_t)tl * RF4);
            const cx<float> *br = md.bvec + (size_t)r * M;
#pragma unroll
            for (int j = 0; j < MPL; ++j) {
                const int m = gl + kCGL * j;
                cx<float> q{0.f, 0.f};
                if (m < M) {
                    cx<float> th{sign * thp[j].x, sign * thp[j].y};
                    if (md.use_bias) { const cx<float> b = br[m]; th.x += b.x; th.y += b.y; }
                    cx<float> mant, pv;
                    int k;
                    cosh2(th, mant, k, pv);
                    const cx<float> c = cmul(mk(prod.x, prod.y), mant);
                    prod = sc_norm(sc<float>{c.x, c.y, prod.e + k});
                    pp = sc_mul(pp, sc<float>{pv.x, pv.y, 0});
                    const float d = pv.x * pv.x + pv.y * pv.y;
                    if (d > 0.f) {
                        const float id = 1.f / d;
                        q = cx<float>{pv.x * id - 1.f, -pv.y * id};
                    } else {
                        q = cx<float>{0x1p60f, 0.f};   // p = 0 (the unit's factor is 1 - p: q is not used)
                    }
                    big = big || !(q.x * q.x + q.y * q.y <= 0x1p24f);
                }
                int ore, oim;
                row_offsets<MPL>(j, gl, ore, oim);
                if (active) { qf[ore] = q.x; qf[oim] = q.y; }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, big);
            prod = group_prod<kCGL>(prod);
            pp = group_prod<kCGL>(pp);
            if (gl == 0 && active) {
                const cx<float> lc = md.logc[r];
                sc<float> lead = sc_exp(cx<float>{lc.x + sign * at.x, lc.y + sign * at.y});
                float c = md.chi[g];
                if (sign < 0 && md.chiP < 0) c = -c;
                lead.x *= c; lead.y *= c;
                const sc<float> tm = sc_mul(prod, sc_norm(lead));
                term[tl] = tm;
                tpr[tl] = sc_mul(tm, pp);
                bigf[tl] = ((bal >> gbase) & 0xffu) != 0;
            }
        }
        __syncthreads();

        const int total = n_burn + n_per_chain * n_skip;
        int n_acc = 0;
        if (threadIdx.x == 0) {
            const u32x4 w = philox(0u, 0u, 0u, 0u, k0, k1);
            site_u = kth_set(upm, md.nwords, (int)(((uint64_t)w.v[0] * (uint64_t)(N / 2)) >> 32));
            site_d = kth_set(dnm, md.nwords, (int)(((uint64_t)w.v[1] * (uint64_t)(N / 2)) >> 32));
            u_sh = (float)(w.v[2] >> 8) * (1.0f / 16777216.0f);
            pend = 0; pend_u = 0; pend_d = 0;   // no exchange to apply before the first step
        }
        __syncthreads();
        for (int step = 0; step < total; ++step, ++gstep) {
            const int iu = site_u, id = site_d;
            // the previous step's exchange, if accepted, is applied to q in this pass
            const int pending = pend, pu = pend_u, pd = pend_d;
            if (threadIdx.x == 32 && step + 1 < total) {
                // the next step's Philox words, ahead of this step's decision
                const u32x4 w = philox((uint32_t)(step + 1), 0u, 0u, 0u, k0, k1);
                wnext[0] = w.v[0]; wnext[1] = w.v[1]; wnext[2] = w.v[2];
            }
            // ---- one pass: q <- q / U' for a pending exchange (U' its factors),
            //      then prod_m (q_m + U_m) of this proposal per pair ----
            for (int tb = 0; tb < ntp; tb += nslots) {
                const int tl0 = tb + slot;
                const bool active = tl0 < ntp;
                const int tl = active ? tl0 : 0;
                const int t = t0 + tl;
                const int row = md.nsign == 2 ? t >> 1 : t;
                const int sg = t - row * md.nsign;
                const int r = md.K == 1 ? 0 : row / md.G, g = row - r * md.G;
                const uint8_t *pg = md.perm + (size_t)g * N;
                const int rs = r * 2 * N;
                const float4 *Su = s4 + (size_t)(rs + sg * N + pg[iu]) * RF4 + gl;          // exp(-4 sigma W_u)
                const float4 *Sd = s4 + (size_t)(rs + (sg ^ 1) * N + pg[id]) * RF4 + gl;    // exp(+4 sigma W_d)
                // 1/U' of the pending exchange: the factors of the opposite orientation
                const float4 *Vu = s4 + (size_t)(rs + (sg ^ 1) * N + pg[pu]) * RF4 + gl;
                const float4 *Vd = s4 + (size_t)(rs + sg * N + pg[pd]) * RF4 + gl;
                float4 *qr = qc + (size_t)tl * RF4 + gl;
                bool big = bigf[tl] != 0;
                f2 Rx = 0, Ry = 0;
                int elo = 0, ehi = 0;
#pragma unroll
                for (int i = 0; i < NPAIR; ++i) {
                    f2 qx, qy;
                    lds128(qr + 8 * i, qx, qy);
                    if (pending) {
                        f2 ax, ay, bx, by;
                        lds128(Vu + 8 * i, ax, ay);
                        lds128(Vd + 8 * i, bx, by);
                        const f2 vx = sub2(mul2(ax, bx), mul2(ay, by)), vy = fma2(ax, by, mul2(ay, bx));
                        const f2 nx = sub2(mul2(qx, vx), mul2(qy, vy));
                        qy = fma2(qx, vy, mul2(qy, vx));
                        qx = nx;
                        if (active) sts128(qr + 8 * i, qx, qy);
                        const f2 qq = fma2(qx, qx, mul2(qy, qy));
                        big = big || !(f2_lo(qq) <= 0x1p24f) || !(f2_hi(qq) <= 0x1p24f);
                    }
                    f2 ux, uy, dx, dy;
                    lds128(Su + 8 * i, ux, uy);
                    lds128(Sd + 8 * i, dx, dy);
                    const f2 wx = sub2(fma2(ux, dx, qx), mul2(uy, dy));   // q + U
                    const f2 wy = fma2(ux, dy, fma2(uy, dx, qy));
                    if (i == 0) {
                        Rx = wx; Ry = wy;
                    } else {
                        const f2 nx = sub2(mul2(Rx, wx), mul2(Ry, wy));
                        Ry = fma2(Rx, wy, mul2(Ry, wx));
                        Rx = nx;
                    }
                    if (big) {   // renormalise the even and the odd units' products
                        float xl = f2_lo(Rx), yl = f2_lo(Ry), xh = f2_hi(Rx), yh = f2_hi(Ry);
                        elo += nrm(xl, yl);
                        ehi += nrm(xh, yh);
                        Rx = f2_pack(xl, xh);
                        Ry = f2_pack(yl, yh);
                    }
                }
                float x, y;
                int ex;
                {
                    float xl = f2_lo(Rx), yl = f2_lo(Ry), xh = f2_hi(Rx), yh = f2_hi(Ry);
                    elo += nrm(xl, yl);
                    ehi += nrm(xh, yh);
                    x = xl * xh - yl * yh;
                    y = xl * yh + yl * xh;
                    ex = elo + ehi;
                }
                if (SGL) {
                    const int o2 = (MPL - 1) * 8;   // float2 index of lane 0's single unit
                    float2 *qs = reinterpret_cast<float2 *>(qc + (size_t)tl * RF4) + o2 + gl;
                    float qx = qs->x, qy = qs->y;
                    if (pending) {
                        float ax, ay, bx, by;
                        lds64(reinterpret_cast<const float2 *>(Vu - gl) + o2 + gl, ax, ay);
                        lds64(reinterpret_cast<const float2 *>(Vd - gl) + o2 + gl, bx, by);
                        const float vx = ax * bx - ay * by, vy = ax * by + ay * bx;
                        const float nx = qx * vx - qy * vy;
                        qy = qx * vy + qy * vx;
                        qx = nx;
                        if (active) *qs = make_float2(qx, qy);
                        big = big || !(qx * qx + qy * qy <= 0x1p24f);
                    }
                    float ux, uy, dx, dy;
                    lds64(reinterpret_cast<const float2 *>(Su - gl) + o2 + gl, ux, uy);
                    lds64(reinterpret_cast<const float2 *>(Sd - gl) + o2 + gl, dx, dy);
                    const float wx = qx + ux * dx - uy * dy, wy = qy + ux * dy + uy * dx;
                    const float nx = x * wx - y * wy;
                    y = x * wy + y * wx;
                    x = nx;
                }
                ex += nrm(x, y);
                const unsigned bal = __ballot_sync(0xffffffffu, big);
                // product over the group's 8 lanes: the mantissas are in [1, 2), so
                // the product's stays below 2^8 with no renormalisation (the term
                // pass normalises it)
#pragma unroll
                for (int o = kCGL / 2; o > 0; o >>= 1) {
                    const float ox = shfl_x(x, o), oy = shfl_x(y, o);
                    const int oe = __shfl_xor_sync(0xffffffffu, ex, o);
                    const float nx = x * ox - y * oy;
                    y = x * oy + y * ox;
                    x = nx;
                    ex += oe;
                }
                const sc<float> gq{x, y, ex};
                if (gl == 0 && active) {
                    if (pending) { term[tl] = nterm[tl]; tpr[tl] = ntpr[tl]; }
                    if ((bal >> gbase) & 0xffu) bigf[tl] = 1;
                    nterm[tl] = gq;   // prod_m (q_m + U_m) of this proposal, for the term pass
                }
            }
            __syncthreads();
            // ---- new terms: term x prod_m p_m x prod_m (q_m + U_m) x prefactor;
            //      this CTA's sums of old and new terms ----
            sc<float> so{0.f, 0.f, 0}, sn{0.f, 0.f, 0};
            for (int tl = threadIdx.x; tl < ntp; tl += blockDim.x) {
                const int t = t0 + tl;
                const int row = md.nsign == 2 ? t >> 1 : t;
                const int sg = t - row * md.nsign;
                const int r = md.K == 1 ? 0 : row / md.G, g = row - r * md.G;
                const int ku = md.perm[(size_t)g * N + iu], kd = md.perm[(size_t)g * N + id];
                const int rs = r * 2 * N;
                const sc<float> a = es[rs + sg * N + ku], b = es[rs + (sg ^ 1) * N + kd];
                const sc<float> ca = ec[rs + sg * N + ku], cb = ec[rs + (sg ^ 1) * N + kd];
                const sc<float> gq = nterm[tl], old = term[tl];
                const sc<float> tp = tpr[tl];
                const cx<float> pre = cmul(mk(a.x, a.y), mk(b.x, b.y));
                // the new term, and term x prod p after acceptance (tpr x prefactor x prod_m U_m)
                cx<float> mn = cmul(cmul(mk(tp.x, tp.y), mk(gq.x, gq.y)), pre);
                const int en = tp.e + gq.e + a.e + b.e + nrm(mn.x, mn.y);
                cx<float> mp = cmul(cmul(mk(tp.x, tp.y), pre), cmul(mk(ca.x, ca.y), mk(cb.x, cb.y)));
                const int ep = tp.e + a.e + b.e + ca.e + cb.e + nrm(mp.x, mp.y);
                const sc<float> tn{mn.x, mn.y, en};
                nterm[tl] = tn;
                ntpr[tl] = sc<float>{mp.x, mp.y, ep};
                so = sc_add(so, old);
                sn = sc_add(sn, tn);
            }
            // warp sums: scaled to the warp's largest exponent, then plain FP32
            {
                float v[4];
                const int e = warp_scaled(so, sn, v);
                if (lane == 0) { wold[warp] = sc<float>{v[0], v[1], e}; wnew[warp] = sc<float>{v[2], v[3], e}; }
            }
            __syncthreads();
            float *slots = xch + (size_t)(gstep & 1) * CL * 8;
            if (warp == 0) {
                const sc<float> zero{0.f, 0.f, 0};
                float v[4];
                const int e = warp_scaled(lane < nwarps ? wold[lane] : zero, lane < nwarps ? wnew[lane] : zero, v);
                const sc<float> a = sc_norm(sc<float>{v[0], v[1], e}), b = sc_norm(sc<float>{v[2], v[3], e});
                // lanes q < CL send this CTA's sums to CTA q's slot [rank]
                if (lane < CL) {
                    const float x[6] = {a.x, a.y, __int_as_float(a.e), b.x, b.y, __int_as_float(b.e)};
                    for (int k = 0; k < 6; ++k) st_cluster_f32(slots + rank * 8 + k, (uint32_t)lane, x[k]);
                }
            }
            cluster_sync();
            if (threadIdx.x == 0) {
                // every CTA adds the partial sums in rank order: the same decision everywhere
                sc<float> a{0.f, 0.f, 0}, b{0.f, 0.f, 0};
                for (int q = 0; q < CL; ++q) {
                    const float *sl = slots + q * 8;
                    a = sc_add(a, sc<float>{sl[0], sl[1], __float_as_int(sl[2])});
                    b = sc_add(b, sc<float>{sl[3], sl[4], __float_as_int(sl[5])});
                }
                // |new / old|^2 from the normalised mantissas (in [1, 2)) and the exponents
                const float q = (b.x * b.x + b.y * b.y) / (a.x * a.x + a.y * a.y);
                const int de = 2 * (b.e - a.e);
                const float r2 = de > 60 ? INFINITY : (de < -60 ? 0.f : ldexpf(q, de));
                const int acc_now = u_sh < r2;
                if (!isfinite(r2) && rank == 0) flag_range(md.status);
                if (acc_now) {
                    s_sm[iu] = -1.f; s_sm[id] = 1.f;
                    upm[iu >> 6] &= ~(1ull << (iu & 63)); dnm[iu >> 6] |= 1ull << (iu & 63);
                    dnm[id >> 6] &= ~(1ull << (id & 63)); upm[id >> 6] |= 1ull << (id & 63);
                    if (step >= n_burn) ++n_acc;
                }
                pend = acc_now; pend_u = iu; pend_d = id;
                // the next proposal, in the configuration after this step
                if (step + 1 < total) {
                    site_u = kth_set(upm, md.nwords, (int)(((uint64_t)wnext[0] * (uint64_t)(N / 2)) >> 32));
                    site_d = kth_set(dnm, md.nwords, (int)(((uint64_t)wnext[1] * (uint64_t)(N / 2)) >> 32));
                    u_sh = (float)(wnext[2] >> 8) * (1.0f / 16777216.0f);
                }
            }
            __syncthreads();
            // ---- keep every n_skip-th state after burn-in ----
            if (rank == 0 && step >= n_burn && ((step - n_burn + 1) % n_skip) == 0 && threadIdx.x < md.nwords) {
                const int kept = (step - n_burn + 1) / n_skip - 1;
                cfg_out[((size_t)chain * n_per_chain + kept) * md.nwords + threadIdx.x] = upm[threadIdx.x];
            }
        }
        if (threadIdx.x == 0 && rank == 0 && acc_out)
            acc_out[chain] = n_per_chain * n_skip > 0 ? (float)n_acc / (float)(n_per_chain * n_skip) : 0.f;
        __syncthreads();
    }
    // no CTA leaves while a peer may still write into its shared memory
    cluster_sync();
}

static int forced_cluster()
{
    const char *v = getenv("NNQS_TEST_SAMPLER_CLUSTER");   // test hook: "old", or 1 / 2 / 4 / 8
    if (!v || !*v) return 0;
    if (v[0] == 'o') return -1;
    return atoi(v);
}

// Runs the cluster sampler if the model's cache fits a cluster of at most 8
// CTAs (and it is not switched off by the test hook); returns false
// (launching nothing) otherwise.
bool launch_sample_cl(const DevModel<float> &md, uint64_t seed, int n_chains, int n_per_chain, int n_skip, int n_burn,
                      uint64_t *cfg_out, float *acc_out, int nsm, cudaStream_t st, cudaError_t *err)
{
    const int force = forced_cluster();
    if (force < 0) return false;
    const int need = (md.M + kCGL - 1) / kCGL;
    if (need > 16) return false;
    const ClPlan p = cl_plan(md, force);
    if (!p.CL) return false;
    void (*kern)(DevModel<float>, uint64_t, int, int, int, int, uint64_t *, float *, int, int) = nullptr;
    if (need <= 2) kern = k_sample_cl<2>;
    else if (need <= 4) kern = k_sample_cl<4>;
    else if (need <= 9) kern = k_sample_cl<9>;
    else kern = k_sample_cl<16>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) { *err = e; return true; }
    int nclusters = nsm / p.CL;
    if (nclusters > n_chains) nclusters = n_chains;
    if (nclusters < 1) nclusters = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nclusters * p.CL));
    cfg.blockDim = dim3((unsigned)p.threads);
    cfg.dynamicSmemBytes = p.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)p.CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, md, seed, n_chains, n_per_chain, n_skip, n_burn, cfg_out, acc_out, p.CL, p.TP);
    *err = e == cudaSuccess ? cudaGetLastError() : e;
    return true;
}

}  // namespace nnqs
