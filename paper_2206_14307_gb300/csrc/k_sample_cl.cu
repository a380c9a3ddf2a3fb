// k_sample_cl.cu -- Metropolis sampler (Sec. 3.2) with each chain's cache in the
// shared memory of a thread-block cluster (FP32).
//
// Same chain, proposals and acceptance rule as k_sample.cu.  A proposed
// exchange of an up site u and a down site d changes the hidden angle of unit m
// of the (row, sign) pair (r, g, sigma) by sigma delta_m, and the pair's term by
// exp(sigma C_ud) prod_m cosh(theta_m + sigma delta_m) / cosh(theta_m), with
// U_m = e^{2 delta_m} = exp(-4 (W_m,g(u) - W_m,g(d))) the same for both signs.
//
// Cache.  Per pair the chain keeps, per unit, c_m = e^{-2 theta'_m} with
// theta' = -theta for sigma = +1 and theta' = theta for sigma = -1, and the
// scalar tc = term x prod_m p(theta'_m), p(x) = e^x / (2 cosh x).  With
// theta = sigma x + b, c(-1) = e^{2x - 2b} = c(+1) e^{-4b}: a row keeps c of
// sign +1 only.  In this form
// the unit factor of both signs is (1 + c_m U_m) -- for sigma = +1 it is
// 1 + p(theta)(U - 1) = p(theta') (1 + c U), for sigma = -1 it is
// p(theta')(1 + c U) / U -- so
//   new term = tc x e^{sigma C_ud} x prod_m (1 + c_m U_m) x X,
//   X = 1 (sigma = +1) or prod_m 1/U_m = e^{4 (CS_g(u) - CS_g(d))} (sigma = -1),
// and an accepted exchange multiplies every c_m of both signs by U_m and tc by
// e^{sigma C_ud} X.  The two signs of a row read the same site factors.  The
// pass stores c_m U_m in place, the cache after an acceptance; after a
// rejection the next pass takes it back with 1/U_m, read from the site rows
// of the opposite orientation.  tc keeps two buffers, the current one and the
// one after an acceptance.
//
// Layout.  The rows of the chain are split over the CL CTAs of a cluster (one
// CTA per SM); each CTA holds its rows' c, the per-site factors exp(-+4W) and
// the per-pair scalars in shared memory.  A group of 8 lanes takes a row: one
// pass reads the row's c and the site factors of the proposal (and, after a
// rejection, those of the rejected exchange), forms prod_m (1 + c_m U_m) of
// both signs and the row's new terms.  The CTA's sum of new terms goes to
// every CTA of the cluster through distributed shared memory; after one
// cluster barrier every CTA adds the CL partial sums in rank order and reaches
// the same decision against the chain's sum of current terms.
#include "common.cuh"
#include "f2.cuh"
#include "kernels.h"

namespace nnqs {

constexpr int kCGL = 8;              // lanes per pair group
constexpr int kClMaxThreads = 576;   // at most 18 warps

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
    int TR;        // rows per CTA (each with its nsign pairs)
    int threads;   // threads per CTA (multiple of 32)
    size_t smem;   // dynamic shared memory per CTA
};

// Shared memory of one CTA: site factor rows u = exp(-+4W) [K][2][N], the
// chain's c rows of sign +1 [TR] and, for models with spin inversion, the
// rows e^{-4 b} [K] (64 MPL bytes a row, see below); per pair tc, in two
// buffers (the current one and its value after an acceptance); site
// prefactors e^{+-Cs} and the products of u over the units e^{-+4 CS}
// [K][2][N] each, exchange slots [2][CL][4], a flag byte per row.
static size_t cl_smem(const DevModel<float> &md, int TR, int CL, int MPL)
{
    const size_t rows = (size_t)md.K * 2 * md.N + TR + (md.nsign == 2 ? md.K : 0);
    return rows * 64 * MPL + 2 * (size_t)TR * md.nsign * sizeof(sc<float>) +
           2 * (size_t)md.K * 2 * md.N * sizeof(sc<float>) + 2 * (size_t)CL * 4 * sizeof(float) + (size_t)TR;
}

// Sum over the warp of a scaled complex number: v = sum a as a plain FP32
// number times 2^e, e the largest exponent in the warp (zeros ignored).
__device__ __forceinline__ int warp_scaled(sc<float> a, float (&v)[2])
{
    const int e = __reduce_max_sync(0xffffffffu, sc_zero(a) ? -(1 << 28) : a.e);
    const float f = pow2i<float>(a.e - e);
    v[0] = a.x * f; v[1] = a.y * f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
        v[1] += __shfl_xor_sync(0xffffffffu, v[1], o);
    }
    return e;
}

// The sum of v over every thread of the cluster's CTAs (called by all
// threads; the result is valid in thread 0).  Warp sums, one sum per CTA,
// sent to every CTA's slot [rank] through distributed shared memory, one
// cluster barrier, and the CL partial sums added in rank order, so that every
// CTA gets the same number.
__device__ __forceinline__ sc<float> cluster_sum(sc<float> v, sc<float> *wsum, float *slots, int CL, uint32_t rank)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    {
        float w[2];
        const int e = warp_scaled(v, w);
        if (lane == 0) wsum[warp] = sc<float>{w[0], w[1], e};
    }
    __syncthreads();
    sc<float> t{0.f, 0.f, 0};
    if (CL == 1) {   // one CTA: warp 0's sum is the total (thread 0 is in warp 0)
        if (warp == 0) {
            float w[2];
            const int e = warp_scaled(lane < nwarps ? wsum[lane] : sc<float>{0.f, 0.f, 0}, w);
            t = sc_norm(sc<float>{w[0], w[1], e});
        }
        return t;
    }
    if (warp == 0) {
        float w[2];
        const int e = warp_scaled(lane < nwarps ? wsum[lane] : sc<float>{0.f, 0.f, 0}, w);
        const sc<float> a = sc_norm(sc<float>{w[0], w[1], e});
        if (lane < CL) {   // lane q writes into CTA q's slot [rank]
            st_cluster_f32(slots + rank * 4 + 0, (uint32_t)lane, a.x);
            st_cluster_f32(slots + rank * 4 + 1, (uint32_t)lane, a.y);
            st_cluster_f32(slots + rank * 4 + 2, (uint32_t)lane, __int_as_float(a.e));
        }
    }
    cluster_sync();
    if (threadIdx.x == 0)
        for (int q = 0; q < CL; ++q) t = sc_add(t, sc<float>{slots[q * 4], slots[q * 4 + 1], __float_as_int(slots[q * 4 + 2])});
    return t;
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
    const int nrows = md.K * md.G;
    for (int CL = 1; CL <= 8; CL *= 2) {
        if (force_cl > 0 && CL != force_cl) continue;
        const int TR = (nrows + CL - 1) / CL;
        const size_t s = cl_smem(md, TR, CL, cl_mpl(md.M));
        if (s <= kClSmemLimit) {
            p.CL = CL; p.TR = TR; p.smem = s;
            break;
        }
    }
    if (!p.CL) return p;
    // warps: the count in 8..18 that leaves the fewest idle row groups
    int best_w = 16, best_waste = 1 << 30;
    for (int w = kClMaxThreads / 32; w >= 8; --w) {
        const int slots = 4 * w;
        const int waste = (p.TR + slots - 1) / slots * slots - p.TR;
        if (waste < best_waste) { best_waste = waste; best_w = w; }
    }
    p.threads = 32 * best_w;
    return p;
}

// Row layout of the site factor rows and the chain's c rows: lane gl of a
// row group owns the units m = gl + 8 j (j < MPL); the units (j, j + 1) of
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

__device__ __forceinline__ void lds64(uint32_t addr, float &x, float &y)
{
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(x), "=f"(y) : "r"(addr));
}
__device__ __forceinline__ void sts128(uint32_t addr, f2 a, f2 b)
{
    asm volatile("st.shared.v2.u64 [%0], {%1, %2};" ::"r"(addr), "l"(a), "l"(b) : "memory");
}
__device__ __forceinline__ void sts64(uint32_t addr, float x, float y)
{
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(x), "f"(y) : "memory");
}

// One row's pass for the lane's units: c <- c / U' after a rejection (UNDO),
// c U stored in place, and the lane's share of prod_m (1 + c_m U_m) of each
// sign as a mantissa (x, y) in [1, 2) and an exponent ex; cm = max_m |c_m U_m|^2.
// BIG renormalises the even and the odd units' products after every unit pair
// (rows where some |c| may exceed 2^12).  Addresses are shared-memory byte
// addresses of the lane's first float4 in each row; o2 leads from there to the
// lane's single unit (odd MPL).  bx, by (and bsx, -nbsy) hold Re e^{-4b} and
// Im e^{-4b} of the lane's units when BREG.
template <int MPL, int NS, bool BREG, bool UNDO, bool BIG>
__device__ __forceinline__ void cl_row(uint32_t Su, uint32_t Sd, uint32_t Vu, uint32_t Vd, uint32_t Br, uint32_t cr,
                                       uint32_t o2, bool active, const f2 *bx, const f2 *by, float bsx, float nbsy,
                                       float (&x)[NS], float (&y)[NS], int (&ex)[NS], float &cm)
{
    constexpr int NPAIR = MPL / 2, SGL = MPL & 1;
    const f2 one2 = f2_pack(1.f, 1.f);
    f2 Rx[NS], Ry[NS];
    int elo[NS], ehi[NS];
#pragma unroll
    for (int sg = 0; sg < NS; ++sg) { elo[sg] = 0; ehi[sg] = 0; }
#pragma unroll
    for (int i = 0; i < NPAIR; ++i) {
        f2 ux, uy, dx, dy;
        lds128(Su + 128 * i, ux, uy);
        lds128(Sd + 128 * i, dx, dy);
        const f2 Ux = sub2(mul2(ux, dx), mul2(uy, dy)), Uy = fma2(ux, dy, mul2(uy, dx));
        f2 cx0, cy0;
        lds128(cr + 128 * i, cx0, cy0);
        if (UNDO) {
            f2 ax, ay, vx, vy;
            lds128(Vu + 128 * i, ax, ay);
            lds128(Vd + 128 * i, vx, vy);
            const f2 Vx = sub2(mul2(ax, vx), mul2(ay, vy)), Vy = fma2(ax, vy, mul2(ay, vx));
            const f2 nx = sub2(mul2(cx0, Vx), mul2(cy0, Vy));
            cy0 = fma2(cx0, Vy, mul2(cy0, Vx));
            cx0 = nx;
        }
        // c U: the cache after an acceptance, and the factor 1 + c U of sign +1
        const f2 qx = sub2(mul2(cx0, Ux), mul2(cy0, Uy)), qy = fma2(cx0, Uy, mul2(cy0, Ux));
        if (active) sts128(cr + 128 * i, qx, qy);
        {
            const f2 cq = fma2(qx, qx, mul2(qy, qy));
            cm = fmaxf(cm, fmaxf(f2_lo(cq), f2_hi(cq)));
        }
#pragma unroll
        for (int sg = 0; sg < NS; ++sg) {
            f2 wx, wy;
            if (sg) {   // sign -1: 1 + c e^{-4b} U
                f2 b_x, b_y;
                if (BREG) {
                    b_x = bx[i]; b_y = by[i];
                } else {
                    lds128(Br + 128 * i, b_x, b_y);
                }
                wx = sub2(fma2(b_x, qx, one2), mul2(b_y, qy));
                wy = fma2(b_x, qy, mul2(b_y, qx));
            } else {
                wx = add2(qx, one2);
                wy = qy;
            }
            if (i == 0) {
                Rx[sg] = wx; Ry[sg] = wy;
            } else {
                const f2 nx = sub2(mul2(Rx[sg], wx), mul2(Ry[sg], wy));
                Ry[sg] = fma2(Rx[sg], wy, mul2(Ry[sg], wx));
                Rx[sg] = nx;
            }
            if (BIG) {   // renormalise the even and the odd units' products
                float xl = f2_lo(Rx[sg]), yl = f2_lo(Ry[sg]), xh = f2_hi(Rx[sg]), yh = f2_hi(Ry[sg]);
                elo[sg] += nrm(xl, yl);
                ehi[sg] += nrm(xh, yh);
                Rx[sg] = f2_pack(xl, xh);
                Ry[sg] = f2_pack(yl, yh);
            }
        }
    }
#pragma unroll
    for (int sg = 0; sg < NS; ++sg) {
        float xl = f2_lo(Rx[sg]), yl = f2_lo(Ry[sg]), xh = f2_hi(Rx[sg]), yh = f2_hi(Ry[sg]);
        elo[sg] += nrm(xl, yl);
        ehi[sg] += nrm(xh, yh);
        x[sg] = xl * xh - yl * yh;
        y[sg] = xl * yh + yl * xh;
        ex[sg] = elo[sg] + ehi[sg];
    }
    if (SGL) {
        float ux, uy, dx, dy;
        lds64(Su + o2, ux, uy);
        lds64(Sd + o2, dx, dy);
        const float Ux = ux * dx - uy * dy, Uy = ux * dy + uy * dx;
        float c0x, c0y;
        lds64(cr + o2, c0x, c0y);
        if (UNDO) {
            float ax, ay, vx, vy;
            lds64(Vu + o2, ax, ay);
            lds64(Vd + o2, vx, vy);
            const float Vx = ax * vx - ay * vy, Vy = ax * vy + ay * vx;
            const float nx = c0x * Vx - c0y * Vy;
            c0y = c0x * Vy + c0y * Vx;
            c0x = nx;
        }
        const float qx = c0x * Ux - c0y * Uy, qy = c0x * Uy + c0y * Ux;
        if (active) sts64(cr + o2, qx, qy);
        cm = fmaxf(cm, qx * qx + qy * qy);
#pragma unroll
        for (int sg = 0; sg < NS; ++sg) {
            float wx = 1.f + qx, wy = qy;
            if (sg) {
                float b_x = bsx, nb_y = nbsy;
                if (!BREG) {
                    float b_y;
                    lds64(Br + o2, b_x, b_y);
                    nb_y = -b_y;
                }
                wx = 1.f + b_x * qx + nb_y * qy;
                wy = b_x * qy - nb_y * qx;
            }
            const float nx = x[sg] * wx - y[sg] * wy;
            y[sg] = x[sg] * wy + y[sg] * wx;
            x[sg] = nx;
        }
    }
#pragma unroll
    for (int sg = 0; sg < NS; ++sg) ex[sg] += nrm(x[sg], y[sg]);
}

template <int MPL, int NS>
__global__ void __launch_bounds__(kClMaxThreads, 1)
    k_sample_cl(DevModel<float> md, uint64_t seed, int n_chains, int n_per_chain, int n_skip, int n_burn,
                uint64_t *__restrict__ cfg_out, float *__restrict__ acc_out, int CL, int TR)
{
    constexpr int NG = 32 / kCGL;
    constexpr int NPAIR = MPL / 2, SGL = MPL & 1;
    constexpr int RF4 = 4 * MPL;                   // float4 per row
    constexpr bool BREG = NS == 2 && MPL <= 9;     // e^{-4b} of the lane's units kept in registers
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ float s_sm[kMaxN];
    __shared__ uint64_t upm[kMaxWords], dnm[kMaxWords];
    __shared__ sc<float> wsum[32];
    __shared__ sc<float> s_cur;      // the sum of the current terms (thread 0)
    __shared__ int pend, pend_u, pend_d, tsel;
    __shared__ int cand[4];          // the next proposal (u, d) if this one is rejected, then if accepted
    __shared__ uint32_t wnx[2][3];   // Philox words of the steps, by parity
    __shared__ int s_b2;             // max(1, max_m |e^{-4b_m}|^2), FP32 bits

    const int M = md.M, N = md.N;
    const int TP = TR * NS;
    float4 *s4 = reinterpret_cast<float4 *>(smem);                               // [K][2][N] rows of u = exp(-+4W)
    float4 *cc = s4 + (size_t)md.K * 2 * N * RF4;                                // [TR] rows of c (sign +1)
    float4 *bt = cc + (size_t)TR * RF4;                                          // [K] rows of e^{-4b} (NS = 2)
    sc<float> *tcb = reinterpret_cast<sc<float> *>(bt + (NS == 2 ? (size_t)md.K * RF4 : 0));   // [2][TP] tc
    sc<float> *es = tcb + 2 * TP;                                                // [K][2][N] site prefactors e^{+-Cs}
    sc<float> *ec = es + (size_t)md.K * 2 * N;                                   // [K][2][N] prod_m u_m = e^{-+4 CS}
    float *xch = reinterpret_cast<float *>(ec + (size_t)md.K * 2 * N);           // [2][CL][4]
    // [TR] per row: some |c| of the row may exceed 2^12, so that its running
    // products are renormalised after every unit pair
    uint8_t *bigf = reinterpret_cast<uint8_t *>(xch + 2 * CL * 4);

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int grp = lane / kCGL, gl = lane % kCGL, gbase = grp * kCGL;
    const int slot = warp * NG + grp, nslots = nwarps * NG;
    const int nrows = md.K * md.G;
    const uint32_t rank = cluster_rank();
    const int r0 = (int)rank * TR;
    const int ntr = r0 >= nrows ? 0 : (nrows - r0 < TR ? nrows - r0 : TR);
    const f2 one2 = f2_pack(1.f, 1.f);
    const uint32_t a_s4 = (uint32_t)__cvta_generic_to_shared(s4), a_cc = (uint32_t)__cvta_generic_to_shared(cc),
                   a_bt = (uint32_t)__cvta_generic_to_shared(bt);
    uint32_t gstep = 0;   // exchanges of this cluster (parity of the exchange slots)
    if (threadIdx.x == 0) s_b2 = __float_as_int(1.f);
    __syncthreads();
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
        if (NS == 2) {
            float *btf = reinterpret_cast<float *>(bt);
            for (int q = threadIdx.x; q < md.K * 8 * MPL; q += blockDim.x) {
                const int r = q / (8 * MPL), w = q - r * 8 * MPL;
                const int l = w % 8, j = w / 8, m = l + 8 * j;
                cx<float> v{1.f, 0.f};
                if (m < M && md.use_bias) {
                    const cx<float> b = md.bvec[(size_t)r * M + m];
                    // |e^{-4b}| must stay a normal FP32 number
                    if (!(fabsf(b.x) <= 20.f)) flag_range(md.status);
                    float sn, cs;
                    sincosf(-4.f * b.y, &sn, &cs);
                    const float mg = expf(-4.f * b.x);
                    v = cx<float>{mg * cs, mg * sn};
                    atomicMax(&s_b2, __float_as_int(v.x * v.x + v.y * v.y));   // non-negative: ordered as integers
                }
                int ore, oim;
                row_offsets<MPL>(j, l, ore, oim);
                btf[(size_t)r * 8 * MPL * 2 + ore] = v.x;
                btf[(size_t)r * 8 * MPL * 2 + oim] = v.y;
            }
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
    // a row is flagged big when some |c| of sign +1 or -1 exceeds 2^12, i.e.
    // when some |c(+1)|^2 exceeds c0lim
    const float c0lim = 0x1p24f / __int_as_float(s_b2);
    // e^{-4b} of the lane's units for the RBM rcur (loaded when a row of another RBM comes)
    int rcur = -1;
    f2 bx[BREG ? NPAIR : 1], by[BREG ? NPAIR : 1];   // e^{-4b}
    float bsx = 1.f, nbsy = 0.f;                       // the single unit's Re e^{-4b}, -Im e^{-4b}
#pragma unroll
    for (int i = 0; i < (BREG ? NPAIR : 1); ++i) { bx[i] = one2; by[i] = 0; }

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
            // the first proposal, in the initial configuration
            const u32x4 w0 = philox(0u, 0u, 0u, 0u, k0, k1);
            wnx[0][0] = w0.v[0]; wnx[0][1] = w0.v[1]; wnx[0][2] = w0.v[2];
            cand[0] = kth_set(upm, md.nwords, (int)(((uint64_t)w0.v[0] * (uint64_t)(N / 2)) >> 32));
            cand[1] = kth_set(dnm, md.nwords, (int)(((uint64_t)w0.v[1] * (uint64_t)(N / 2)) >> 32));
            pend = 2; pend_u = 0; pend_d = 0;   // no previous step
            tsel = 0;
        }
        __syncthreads();

        // ---- fresh cache of this CTA's rows: c = e^{-2 theta'} = 1/p(theta') - 1
        //      per unit of sign +1, tc per pair, and the chain's sum of terms ----
        sc<float> so{0.f, 0.f, 0};
        for (int tb = 0; tb < ntr; tb += nslots) {
            const int rl0 = tb + slot;
            const bool active = rl0 < ntr;
            const int rl = active ? rl0 : 0;
            const int row = r0 + rl;
            const int r = row / md.G, g = row - r * md.G;
            const uint8_t *pg = md.perm + (size_t)g * N;
            const cx<float> *Wr = md.Wt + (size_t)r * N * M;
            cx<float> xs[MPL];   // sum_i W_m,g(i) s_i of the lane's units
#pragma unroll
            for (int j = 0; j < MPL; ++j) xs[j] = cx<float>{0.f, 0.f};
#pragma unroll 2
            for (int i = 0; i < N; ++i) {
                const cx<float> *wk = Wr + (size_t)pg[i] * M;
                const float si = s_sm[i];
#pragma unroll
                for (int j = 0; j < MPL; ++j) {
                    const int m = gl + kCGL * j;
                    if (m < M) { const cx<float> w = wk[m]; xs[j].x += si * w.x; xs[j].y += si * w.y; }
                }
            }
            cx<float> at{0.f, 0.f};
            if (md.use_bias) {
                const cx<float> *ar = md.avec + (size_t)r * N;
                for (int i = gl; i < N; i += kCGL) { const cx<float> a = ar[pg[i]]; at.x += s_sm[i] * a.x; at.y += s_sm[i] * a.y; }
#pragma unroll
                for (int o = kCGL / 2; o > 0; o >>= 1) { at.x += shfl_x(at.x, o); at.y += shfl_x(at.y, o); }
            }
            const cx<float> *br = md.bvec + (size_t)r * M;
            bool big = false;
            float *cf = reinterpret_cast<float *>(cc + (size_t)rl * RF4);
#pragma unroll
            for (int sg = 0; sg < NS; ++sg) {
                const float sign = sg ? -1.f : 1.f;
                // c = e^{-2 theta'} directly (no cancellation where p(theta') is near 1);
                // 2 cosh(theta') p(theta') = e^{theta'}, so tc = lead e^{sum theta'} and
                // the term is tc prod_m (1 + c_m)
                float stx = 0.f, sty = 0.f;
                sc<float> qp{1.f, 0.f, 0};
#pragma unroll
                for (int j = 0; j < MPL; ++j) {
                    const int m = gl + kCGL * j;
                    cx<float> c{0.f, 0.f};
                    if (m < M) {
                        // theta' = -(x + b) for sigma = +1, -x + b for sigma = -1
                        cx<float> th{-xs[j].x, -xs[j].y};
                        if (md.use_bias) { const cx<float> b = br[m]; th.x -= sign * b.x; th.y -= sign * b.y; }
                        stx += th.x;
                        sty += th.y;
                        float a2 = -2.8853900817779268f * th.x;   // log2 |c|
                        if (!(a2 <= 100.f)) {   // |c| beyond 2^100: outside the cache's FP32 range
                            flag_range(md.status);
                            a2 = 100.f;
                        }
                        const float e = exp2f(a2);
                        float sn, cs;
                        sincosf(-2.f * th.y, &sn, &cs);
                        c = cx<float>{e * cs, e * sn};
                        qp = sc_mul(qp, sc<float>{1.f + c.x, c.y, 0});
                        big = big || !(c.x * c.x + c.y * c.y <= 0x1p24f);
                    }
                    if (sg == 0) {   // the row keeps c of sign +1 only: c(-1) = c(+1) e^{-4b}
                        int ore, oim;
                        row_offsets<MPL>(j, gl, ore, oim);
                        if (active) { cf[ore] = c.x; cf[oim] = c.y; }
                    }
                }
#pragma unroll
                for (int o = kCGL / 2; o > 0; o >>= 1) {
                    stx += shfl_x(stx, o);
                    sty += shfl_x(sty, o);
                }
                qp = group_prod<kCGL>(qp);
                if (gl == 0 && active) {
                    const cx<float> lc = md.logc[r];
                    sc<float> lead = sc_exp(cx<float>{lc.x + sign * at.x + stx, lc.y + sign * at.y + sty});
                    float ch = md.chi[g];
                    if (sg && md.chiP < 0) ch = -ch;
                    lead.x *= ch; lead.y *= ch;
                    lead = sc_norm(lead);
                    tcb[rl * NS + sg] = lead;
                    so = sc_add(so, sc_mul(lead, qp));
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, big);
            if (gl == 0 && active) bigf[rl] = ((bal >> gbase) & 0xffu) != 0;
        }
        {
            const sc<float> t = cluster_sum(so, wsum, xch + (size_t)(gstep & 1) * CL * 4, CL, rank);
            ++gstep;
            if (threadIdx.x == 0) s_cur = t;
        }
        __syncthreads();

        const int total = n_burn + n_per_chain * n_skip;
        int n_acc = 0;
        for (int step = 0; step < total; ++step, ++gstep) {
            // this step's proposal: the candidate for the previous step's outcome
            // the c rows hold the values after an acceptance of the previous
            // proposal; if it was rejected, this pass divides its factors out again
            const bool undo = pend == 0;
            const int iu = pend == 1 ? cand[2] : cand[0], id = pend == 1 ? cand[3] : cand[1];
            const int pu = pend_u, pd = pend_d;
            const sc<float> *tcur = tcb + tsel * TP;
            sc<float> *tnxt = tcb + (tsel ^ 1) * TP;
            if (threadIdx.x == 32 && step + 1 < total) {
                // the next step's Philox words, ahead of this step's decision
                const u32x4 w = philox((uint32_t)(step + 1), 0u, 0u, 0u, k0, k1);
                uint32_t *wn = wnx[(step + 1) & 1];
                wn[0] = w.v[0]; wn[1] = w.v[1]; wn[2] = w.v[2];
            }
            // ---- one pass per row: c <- c / U' after a rejected exchange (U' its
            //      factors), prod_m (1 + c_m U_m) of this proposal for each sign,
            //      and c <- c U in place (the cache if it is accepted); then per
            //      pair the new term and tc after an acceptance ----
            sc<float> sn{0.f, 0.f, 0};
            // The rows of a group come in chunks of CH: the chunk's 8 pairs
            // k = it NS + sg have their lane products combined by a
            // reduce-scatter over the group's 8 lanes (levels xor 4, 2, 1), after
            // which lane gl holds pair k = 4 bit0(gl) + 2 bit1(gl) + bit2(gl)
            // and computes that pair's new term.
            constexpr int CH = 8 / NS;
            const int my_k = ((gl & 1) << 2) | (gl & 2) | ((gl >> 2) & 1);
            const int my_it = my_k / NS, my_sg = my_k % NS;
            for (int tb = 0; tb < ntr; tb += CH * nslots) {
                float h0x = 1.f, h0y = 0.f, h1x = 1.f, h1y = 0.f, h2x = 1.f, h2y = 0.f;
                int h0e = 0, h1e = 0, h2e = 0;
                float fx = 1.f, fy = 0.f;   // the lane's pair after the last level
                int fe = 0;
#pragma unroll 1
                for (int it = 0; it < CH; ++it) {
                    const int rl0 = tb + it * nslots + slot;
                    const bool active = rl0 < ntr;
                    float x[NS], y[NS];
                    int ex[NS];
#pragma unroll
                    for (int sg = 0; sg < NS; ++sg) { x[sg] = 1.f; y[sg] = 0.f; ex[sg] = 0; }
                    if (tb + it * nslots < ntr) {   // some group of the CTA has a row
                        const int rl = active ? rl0 : 0;
                        const int row = r0 + rl;
                        const int r = md.K == 1 ? 0 : row / md.G, g = row - r * md.G;
                        const uint8_t *pg = md.perm + (size_t)g * N;
                        const int rs = r * 2 * N;
                        const int ku = pg[iu], kd = pg[id];
                        // shared-memory addresses of the lane's first float4 in the rows
                        const uint32_t Su = a_s4 + (uint32_t)(((rs + ku) * RF4 + gl) * 16);         // exp(-4 W_u)
                        const uint32_t Sd = a_s4 + (uint32_t)(((rs + N + kd) * RF4 + gl) * 16);     // exp(+4 W_d)
                        const uint32_t Vu = a_s4 + (uint32_t)(((rs + N + pg[pu]) * RF4 + gl) * 16); // 1/U' of the
                        const uint32_t Vd = a_s4 + (uint32_t)(((rs + pg[pd]) * RF4 + gl) * 16);     // rejected exchange
                        const uint32_t Br = a_bt + (uint32_t)((r * RF4 + gl) * 16);
                        const uint32_t cr = a_cc + (uint32_t)((rl * RF4 + gl) * 16);
                        // float2 offset from a lane's first float4 to its single unit
                        constexpr uint32_t o2b = (uint32_t)((MPL - 1) * 8 * 8);
                        const uint32_t o2 = o2b - (uint32_t)(gl * 8);
                        if (BREG && r != rcur) {
                            rcur = r;
#pragma unroll
                            for (int i = 0; i < NPAIR; ++i) lds128(Br + 128 * i, bx[i], by[i]);
                            if (SGL) {
                                float b_y;
                                lds64(Br + o2, bsx, b_y);
                                nbsy = -b_y;
                            }
                        }
                        const bool big = bigf[rl] != 0;
                        float cm = 0.f;   // max_m |c_m U_m|^2
                        // the row's product: uniform branches to the variant without the
                        // undo and the per-pair renormalisation where none is needed
                        const bool anybig = __any_sync(0xffffffffu, big);
                        if (undo) {
                            if (anybig) cl_row<MPL, NS, BREG, true, true>(Su, Sd, Vu, Vd, Br, cr, o2, active, bx, by, bsx, nbsy, x, y, ex, cm);
                            else cl_row<MPL, NS, BREG, true, false>(Su, Sd, Vu, Vd, Br, cr, o2, active, bx, by, bsx, nbsy, x, y, ex, cm);
                        } else {
                            if (anybig) cl_row<MPL, NS, BREG, false, true>(Su, Sd, Vu, Vd, Br, cr, o2, active, bx, by, bsx, nbsy, x, y, ex, cm);
                            else cl_row<MPL, NS, BREG, false, false>(Su, Sd, Vu, Vd, Br, cr, o2, active, bx, by, bsx, nbsy, x, y, ex, cm);
                        }
                        const unsigned bal = __ballot_sync(0xffffffffu, !(cm <= c0lim));
                        if (gl == 0 && active && ((bal >> gbase) & 0xffu)) bigf[rl] = 1;
                    }
                    // reduce-scatter step for the pairs k = it NS + sg; the lane
                    // mantissas are in [1, 2), so no product of at most 8 of them
                    // needs renormalising
#pragma unroll
                    for (int sg = 0; sg < NS; ++sg) {
                        const int k = it * NS + sg;
                        if ((k & 1) == 0) { h0x = x[sg]; h0y = y[sg]; h0e = ex[sg]; continue; }
                        const bool b2 = (gl >> 2) & 1;   // keeps the odd pair
                        float kx = b2 ? x[sg] : h0x, ky = b2 ? y[sg] : h0y;
                        int ke = b2 ? ex[sg] : h0e;
                        float sx = b2 ? h0x : x[sg], sy = b2 ? h0y : y[sg];
                        int se = b2 ? h0e : ex[sg];
                        float ox = shfl_x(sx, 4), oy = shfl_x(sy, 4);
                        int oe = __shfl_xor_sync(0xffffffffu, se, 4);
                        float vx = kx * ox - ky * oy, vy = kx * oy + ky * ox;
                        int ve = ke + oe;
                        if (((k >> 1) & 1) == 0) { h1x = vx; h1y = vy; h1e = ve; continue; }
                        const bool b1 = (gl >> 1) & 1;
                        kx = b1 ? vx : h1x; ky = b1 ? vy : h1y; ke = b1 ? ve : h1e;
                        sx = b1 ? h1x : vx; sy = b1 ? h1y : vy; se = b1 ? h1e : ve;
                        ox = shfl_x(sx, 2); oy = shfl_x(sy, 2);
                        oe = __shfl_xor_sync(0xffffffffu, se, 2);
                        vx = kx * ox - ky * oy; vy = kx * oy + ky * ox;
                        ve = ke + oe;
                        if (((k >> 2) & 1) == 0) { h2x = vx; h2y = vy; h2e = ve; continue; }
                        const bool b0 = gl & 1;
                        kx = b0 ? vx : h2x; ky = b0 ? vy : h2y; ke = b0 ? ve : h2e;
                        sx = b0 ? h2x : vx; sy = b0 ? h2y : vy; se = b0 ? h2e : ve;
                        ox = shfl_x(sx, 1); oy = shfl_x(sy, 1);
                        oe = __shfl_xor_sync(0xffffffffu, se, 1);
                        fx = kx * ox - ky * oy; fy = kx * oy + ky * ox;
                        fe = ke + oe;
                    }
                }
                // the lane's pair: new term tc x prefactor x prod_m (1 + c_m U_m) x X
                // and tc after an acceptance, tc x prefactor x X
                const int m_rl = tb + my_it * nslots + slot;
                if (m_rl < ntr) {
                    const int row = r0 + m_rl;
                    const int r = md.K == 1 ? 0 : row / md.G, g = row - r * md.G;
                    const int m_ku = md.perm[(size_t)g * N + iu], m_kd = md.perm[(size_t)g * N + id];
                    const int sg = my_sg, tp = m_rl * NS + sg, rs = r * 2 * N;
                    const sc<float> tc = tcur[tp];
                    const sc<float> a = es[rs + sg * N + m_ku], b = es[rs + (sg ^ 1) * N + m_kd];
                    cx<float> base = cmul(cmul(mk(tc.x, tc.y), mk(a.x, a.y)), mk(b.x, b.y));
                    int eb = tc.e + a.e + b.e;
                    if (sg) {   // X = prod_m 1/U_m
                        const sc<float> ca = ec[rs + N + m_ku], cb = ec[rs + m_kd];
                        base = cmul(base, cmul(mk(ca.x, ca.y), mk(cb.x, cb.y)));
                        eb += ca.e + cb.e;
                    }
                    eb += nrm(base.x, base.y);
                    cx<float> mn = cmul(base, mk(fx, fy));
                    const int en = eb + fe + nrm(mn.x, mn.y);
                    tnxt[tp] = sc<float>{base.x, base.y, eb};
                    sn = sc_add(sn, sc<float>{mn.x, mn.y, en});
                }
            }
            const sc<float> snew = cluster_sum(sn, wsum, xch + (size_t)(gstep & 1) * CL * 4, CL, rank);
            const bool more = step + 1 < total;
            if (threadIdx.x == 0) {
                // |new / old|^2 from the normalised mantissas (in [1, 2)) and the exponents
                const sc<float> a = s_cur, b = snew;
                const float q = (b.x * b.x + b.y * b.y) / (a.x * a.x + a.y * a.y);
                const int de = 2 * (b.e - a.e);
                const float r2 = de > 60 ? INFINITY : (de < -60 ? 0.f : q * pow2i<float>(de));
                const float u = (float)(wnx[step & 1][2] >> 8) * (1.0f / 16777216.0f);
                const int acc_now = u < r2;
                if (!isfinite(r2) && rank == 0) flag_range(md.status);
                if (acc_now) {
                    if (step >= n_burn) ++n_acc;
                    s_cur = b;
                    tsel ^= 1;
                }
                pend = acc_now; pend_u = iu; pend_d = id;   // 1 accepted, 0 rejected
            } else if (threadIdx.x == 32 && more) {
                // the next proposal if this one is rejected: the configuration stays
                const uint32_t *wn = wnx[(step + 1) & 1];
                cand[0] = kth_set(upm, md.nwords, (int)(((uint64_t)wn[0] * (uint64_t)(N / 2)) >> 32));
                cand[1] = kth_set(dnm, md.nwords, (int)(((uint64_t)wn[1] * (uint64_t)(N / 2)) >> 32));
            } else if (threadIdx.x == 64 && more) {
                // ... and if it is accepted: iu goes down, id goes up
                uint64_t um[kMaxWords], dm[kMaxWords];
                for (int q = 0; q < md.nwords; ++q) { um[q] = upm[q]; dm[q] = dnm[q]; }
                um[iu >> 6] &= ~(1ull << (iu & 63)); dm[iu >> 6] |= 1ull << (iu & 63);
                dm[id >> 6] &= ~(1ull << (id & 63)); um[id >> 6] |= 1ull << (id & 63);
                const uint32_t *wn = wnx[(step + 1) & 1];
                cand[2] = kth_set(um, md.nwords, (int)(((uint64_t)wn[0] * (uint64_t)(N / 2)) >> 32));
                cand[3] = kth_set(dm, md.nwords, (int)(((uint64_t)wn[1] * (uint64_t)(N / 2)) >> 32));
            }
            __syncthreads();
            // ---- the configuration after this step (one mask word per thread);
            //      keep every n_skip-th state after burn-in ----
            if (threadIdx.x < md.nwords) {
                const int q = threadIdx.x;
                uint64_t um = upm[q], dm = dnm[q];
                if (pend == 1) {
                    if ((iu >> 6) == q) { um &= ~(1ull << (iu & 63)); dm |= 1ull << (iu & 63); }
                    if ((id >> 6) == q) { dm &= ~(1ull << (id & 63)); um |= 1ull << (id & 63); }
                    upm[q] = um; dnm[q] = dm;
                    if (q == 0) { s_sm[iu] = -1.f; s_sm[id] = 1.f; }
                }
                if (rank == 0 && step >= n_burn && ((step - n_burn + 1) % n_skip) == 0) {
                    const int kept = (step - n_burn + 1) / n_skip - 1;
                    cfg_out[((size_t)chain * n_per_chain + kept) * md.nwords + q] = um;
                }
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
    const bool two = md.nsign == 2;
    if (need <= 2) kern = two ? k_sample_cl<2, 2> : k_sample_cl<2, 1>;
    else if (need <= 4) kern = two ? k_sample_cl<4, 2> : k_sample_cl<4, 1>;
    else if (need <= 9) kern = two ? k_sample_cl<9, 2> : k_sample_cl<9, 1>;
    else kern = two ? k_sample_cl<16, 2> : k_sample_cl<16, 1>;
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
    e = cudaLaunchKernelEx(&cfg, kern, md, seed, n_chains, n_per_chain, n_skip, n_burn, cfg_out, acc_out, p.CL, p.TR);
    *err = e == cudaSuccess ? cudaGetLastError() : e;
    return true;
}

}  // namespace nnqs
