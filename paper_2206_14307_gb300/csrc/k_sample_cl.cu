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

// rows (r, g) of the projected sum that a CTA's TP pairs touch
__host__ __device__ __forceinline__ int cl_rows(const DevModel<float> &md, int TP) { return TP / md.nsign + 2; }

// shared memory of one CTA: site tables [K][2][N][M], p [TP][M], terms, new
// terms and pair products [TP], site prefactors [K][2][N], exchange slots
// [2][CL][8], images of the sites under the CTA's rows [rows][N]
static size_t cl_smem(const DevModel<float> &md, int TP, int CL)
{
    return (size_t)md.K * 2 * md.N * md.M * sizeof(cx<float>) + (size_t)TP * md.M * sizeof(cx<float>) +
           3 * (size_t)TP * sizeof(sc<float>) + (size_t)md.K * 2 * md.N * sizeof(sc<float>) +
           2 * (size_t)CL * 8 * sizeof(float) + (size_t)cl_rows(md, TP) * md.N;
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

// The smallest cluster whose CTAs hold the chain's cache; CL = 0 if none does.
static ClPlan cl_plan(const DevModel<float> &md, int force_cl)
{
    ClPlan p{0, 0, 0, 0};
    const int nrs = md.K * md.G * md.nsign;
    for (int CL = 1; CL <= 8; CL *= 2) {
        if (force_cl > 0 && CL != force_cl) continue;
        const int TP = (nrs + CL - 1) / CL;
        const size_t s = cl_smem(md, TP, CL);
        if (s <= 220 * 1024) {
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

template <int MPL>
__global__ void __launch_bounds__(kClMaxThreads, 1)
    k_sample_cl(DevModel<float> md, uint64_t seed, int n_chains, int n_per_chain, int n_skip, int n_burn,
                uint64_t *__restrict__ cfg_out, float *__restrict__ acc_out, int CL, int TP)
{
    constexpr int NG = 32 / kCGL;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ float s_sm[kMaxN];
    __shared__ uint64_t upm[kMaxWords], dnm[kMaxWords];
    __shared__ sc<float> wold[32], wnew[32];
    __shared__ int site_u, site_d, pend, pend_u, pend_d;
    __shared__ uint32_t wnext[3];
    __shared__ float u_sh;

    const int M = md.M, N = md.N;
    cx<float> *s4 = reinterpret_cast<cx<float> *>(smem);                        // [K][2][N][M] exp(-+4W)
    cx<float> *pc = s4 + (size_t)md.K * 2 * N * M;                              // [TP][M]
    sc<float> *term = reinterpret_cast<sc<float> *>(pc + (size_t)TP * M);        // [TP]
    sc<float> *nterm = term + TP;                                               // [TP] new terms of the last proposal
    sc<float> *gprod = nterm + TP;                                              // [TP] pair products of the proposal
    sc<float> *es = gprod + TP;                                                 // [K][2][N] site prefactors
    float *xch = reinterpret_cast<float *>(es + (size_t)md.K * 2 * N);           // [2][CL][8]
    uint8_t *prow = reinterpret_cast<uint8_t *>(xch + 2 * CL * 8);              // [rows][N] images of the sites

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int grp = lane / kCGL, gl = lane % kCGL;
    const int slot = warp * NG + grp, nslots = nwarps * NG;
    const int nrs = md.K * md.G * md.nsign;
    const uint32_t rank = cluster_rank();
    const int t0 = (int)rank * TP;
    const int ntp = t0 >= nrs ? 0 : (nrs - t0 < TP ? nrs - t0 : TP);
    uint32_t gstep = 0;   // steps of this cluster over all its chains (parity of the exchange slots)
    const int row0 = t0 / md.nsign;   // first row (r, g) of this CTA's pairs
    for (int q = threadIdx.x; q < md.K * 2 * N * M; q += blockDim.x) {
        const int m = q % M, row = q / M;   // row = (r * 2 + half) * N + k
        s4[q] = md.S4[(size_t)row * md.Mp + m];
    }
    for (int q = threadIdx.x; q < md.K * 2 * N; q += blockDim.x) es[q] = md.ES[q];
    for (int q = threadIdx.x; q < cl_rows(md, TP) * N; q += blockDim.x) {
        const int rw = row0 + q / N, i = q - (q / N) * N;
        if (rw < md.K * md.G) prow[q] = md.perm[(size_t)(rw % md.G) * N + i];
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

        // ---- fresh cache of this CTA's pairs ----
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
            sc<float> prod{1.f, 0.f, 0};
            const cx<float> *br = md.bvec + (size_t)r * M;
#pragma unroll
            for (int j = 0; j < MPL; ++j) {
                const int m = gl + kCGL * j;
                if (m < M) {
                    cx<float> th{sign * thp[j].x, sign * thp[j].y};
                    if (md.use_bias) { const cx<float> b = br[m]; th.x += b.x; th.y += b.y; }
                    cx<float> mant, pv;
                    int k;
                    cosh2(th, mant, k, pv);
                    if (active) pc[(size_t)tl * M + m] = pv;
                    const cx<float> q = cmul(mk(prod.x, prod.y), mant);
                    prod = sc<float>{q.x, q.y, prod.e + k};
                }
            }
            prod = sc_norm(prod);
#pragma unroll
            for (int o = kCGL / 2; o > 0; o >>= 1) {
                const sc<float> w{shfl_x(prod.x, o), shfl_x(prod.y, o), __shfl_xor_sync(0xffffffffu, prod.e, o)};
                prod = sc_mul(prod, w);
            }
            if (gl == 0 && active) {
                const cx<float> lc = md.logc[r];
                sc<float> lead = sc_exp(cx<float>{lc.x + sign * at.x, lc.y + sign * at.y});
                float c = md.chi[g];
                if (sign < 0 && md.chiP < 0) c = -c;
                lead.x *= c; lead.y *= c;
                term[tl] = sc_mul(prod, sc_norm(lead));
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
            // the previous step's exchange, if accepted, is applied to p in this pass
            const int pending = pend, pu = pend_u, pd = pend_d;
            if (threadIdx.x == 32 && step + 1 < total) {
                // the next step's Philox words, ahead of this step's decision
                const u32x4 w = philox((uint32_t)(step + 1), 0u, 0u, 0u, k0, k1);
                wnext[0] = w.v[0]; wnext[1] = w.v[1]; wnext[2] = w.v[2];
            }
            // ---- one pass: p <- p (1 + T') / (1 + p T') for a pending exchange, then
            //      the factors 1 + p T of this proposal; each pair group's product ----
            for (int tb = 0; tb < ntp; tb += nslots) {
                const int tl0 = tb + slot;
                const bool active = tl0 < ntp;
                const int tl = active ? tl0 : 0;
                const int t = t0 + tl;
                const int row = md.nsign == 2 ? t >> 1 : t;
                const int sg = t - row * md.nsign;
                const int r = row / md.G;
                const uint8_t *pg = prow + (size_t)(row - row0) * N;
                const int ku = pg[iu], kd = pg[id];
                const size_t rs = (size_t)r * 2 * N * M;
                const cx<float> *Su = s4 + rs + ((size_t)sg * N + ku) * M;         // exp(-4 sigma W_u)
                const cx<float> *Sd = s4 + rs + ((size_t)(sg ^ 1) * N + kd) * M;   // exp(+4 sigma W_d)
                const cx<float> *Pu = s4 + rs + ((size_t)sg * N + pg[pu]) * M;
                const cx<float> *Pd = s4 + rs + ((size_t)(sg ^ 1) * N + pg[pd]) * M;
                cx<float> *pr = pc + (size_t)tl * M;
                cx<float> prod{1.f, 0.f};
#pragma unroll
                for (int j = 0; j < MPL; ++j) {
                    const int m = gl + kCGL * j;
                    if (m < M) {
                        cx<float> p = pr[m];
                        if (pending) {
                            const cx<float> e2 = cmul(Pu[m], Pd[m]);
                            const cx<float> tt{e2.x - 1.f, e2.y};
                            const cx<float> f{1.f + p.x * tt.x - p.y * tt.y, p.x * tt.y + p.y * tt.x};
                            const cx<float> num = cmul(p, e2);
                            const float d = rcp_nr_f(f.x * f.x + f.y * f.y);
                            p = cx<float>{(num.x * f.x + num.y * f.y) * d, (num.y * f.x - num.x * f.y) * d};
                            if (active) pr[m] = p;
                        }
                        const cx<float> e2 = cmul(Su[m], Sd[m]);   // e^{2 Delta}
                        const cx<float> tt{e2.x - 1.f, e2.y};
                        const cx<float> f{1.f + p.x * tt.x - p.y * tt.y, p.x * tt.y + p.y * tt.x};
                        prod = cmul(prod, f);
                    }
                }
                const int ex = expo<float>(prod.x, prod.y);
                const float scl = pow2i<float>(-ex);
                sc<float> pv{prod.x * scl, prod.y * scl, ex};
#pragma unroll
                for (int o = kCGL / 2; o > 0; o >>= 1) {
                    const sc<float> w{shfl_x(pv.x, o), shfl_x(pv.y, o), __shfl_xor_sync(0xffffffffu, pv.e, o)};
                    pv = sc_mul(pv, w);
                }
                if (gl == 0 && active) gprod[tl] = pv;
            }
            __syncthreads();
            // ---- prefactor, new terms, and this CTA's sums of old and new terms ----
            sc<float> so{0.f, 0.f, 0}, sn{0.f, 0.f, 0};
            for (int tl = threadIdx.x; tl < ntp; tl += blockDim.x) {
                const int t = t0 + tl;
                const int row = md.nsign == 2 ? t >> 1 : t;
                const int sg = t - row * md.nsign;
                const int r = row / md.G;
                const uint8_t *pg = prow + (size_t)(row - row0) * N;
                const sc<float> *ESr = es + (size_t)r * 2 * N;
                const sc<float> a = ESr[(size_t)sg * N + pg[iu]], b = ESr[(size_t)(sg ^ 1) * N + pg[id]];
                const sc<float> gp = gprod[tl];
                sc<float> old = term[tl];
                if (pending) { old = nterm[tl]; term[tl] = old; }
                // new term = old x pair product x prefactor (mantissas in [1, 2): one normalisation)
                cx<float> m = cmul(cmul(mk(old.x, old.y), mk(gp.x, gp.y)), cmul(mk(a.x, a.y), mk(b.x, b.y)));
                const int e = old.e + gp.e + a.e + b.e + nrm(m.x, m.y);
                const sc<float> tn{m.x, m.y, e};
                nterm[tl] = tn;
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
