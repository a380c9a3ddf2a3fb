// k_amp.cu -- amplitude kernels: log psi of fresh configurations and the
// connected-configuration ratio engine behind E_loc (Eq. 10) and the Lanczos
// quantities (H psi)/psi, (H^2 psi)/psi (Sec. 3.3).
//
// Layout of the work: one CTA per sample (grid-stride over samples), one warp
// per row (r, g) of the projected sum (Eqs. 4-6), lanes over hidden units m.
// Each row computes theta'_m = sum_i W_r[m][g(i)] s_i once and serves both
// spin-inversion signs.  Amplitudes are kept as scaled complex numbers
// (mantissa * 2^e) so that log psi keeps its absolute accuracy.
//
// For a flip set D (the sites whose spins differ between s and s'), the row
// factor of psi(s')/psi(s) is
//   prod_m cosh(theta_m + Delta_m) / cosh(theta_m)
//     = prod_m [ p_m e^{Delta_m} + (1 - p_m) e^{-Delta_m} ],
//   p_m = e^{theta_m} / (2 cosh theta_m),
//   e^{+-Delta_m} = prod_{f in D} exp(-+2 sign s_f W_r[m][g(f)])   (tables),
// so that no transcendental function is evaluated per connected element.
#include "common.cuh"
#include "kernels.h"

namespace nnqs {

template <typename T, int MPL>
__device__ __forceinline__ void row_theta(const DevModel<T> &md, int r, int g, const T *s_sm, cx<T> (&th)[MPL],
                                          int lane)
{
#pragma unroll
    for (int j = 0; j < MPL; ++j) th[j] = cx<T>{T(0), T(0)};
    const uint8_t *pg = md.perm + (size_t)g * md.N;
    const cx<T> *Wr = md.Wt + (size_t)r * md.N * md.M;
    for (int i = 0; i < md.N; ++i) {
        const int k = __ldg(pg + i);
        const T si = s_sm[i];
        const cx<T> *wk = Wr + (size_t)k * md.M;
#pragma unroll
        for (int j = 0; j < MPL; ++j) {
            const int m = lane + 32 * j;
            if (m < md.M) {
                cx<T> w = wk[m];
                th[j].x += si * w.x;
                th[j].y += si * w.y;
            }
        }
    }
}

// a_r . T_g s (warp-reduced; all lanes receive it)
template <typename T>
__device__ __forceinline__ cx<T> row_visible(const DevModel<T> &md, int r, int g, const T *s_sm, int lane)
{
    cx<T> acc{T(0), T(0)};
    if (!md.use_bias) return acc;
    const uint8_t *pg = md.perm + (size_t)g * md.N;
    const cx<T> *ar = md.avec + (size_t)r * md.N;
    for (int i = lane; i < md.N; i += 32) {
        cx<T> a = ar[pg[i]];
        acc.x += s_sm[i] * a.x;
        acc.y += s_sm[i] * a.y;
    }
    return warp_sum(acc);
}

// Leading factor c_r chi(g) chi_P^{[sign<0]} exp(sign * a.T_g s) of one term.
template <typename T>
__device__ __forceinline__ sc<T> row_lead(const DevModel<T> &md, int r, int g, int sign, cx<T> at)
{
    cx<T> lc = md.logc[r];
    sc<T> v = sc_exp(cx<T>{lc.x + sign * at.x, lc.y + sign * at.y});
    T c = md.chi[g];
    if (sign < 0 && md.chiP < 0) c = -c;
    v.x *= c;
    v.y *= c;
    return sc_norm(v);
}

// Product over hidden units of 2cosh(theta_m) for one sign, and p_m.
template <typename T, int MPL>
__device__ __forceinline__ sc<T> row_cosh(const DevModel<T> &md, int r, int sign, const cx<T> (&thp)[MPL],
                                          cx<T> (&p)[MPL], int lane)
{
    sc<T> prod{T(1), T(0), 0};
    const cx<T> *br = md.bvec + (size_t)r * md.M;
#pragma unroll
    for (int j = 0; j < MPL; ++j) {
        const int m = lane + 32 * j;
        if (m < md.M) {
            cx<T> th{sign * thp[j].x, sign * thp[j].y};
            if (md.use_bias) { cx<T> b = br[m]; th.x += b.x; th.y += b.y; }
            cx<T> mant;
            int k;
            cosh2(th, mant, k, p[j]);
            cx<T> q = cmul(mk(prod.x, prod.y), mant);
            prod = sc<T>{q.x, q.y, prod.e + k};
        } else {
            p[j] = cx<T>{T(0), T(0)};
        }
    }
    return warp_prod(prod);
}


template <typename T>
__device__ __forceinline__ void load_spins(const DevModel<T> &md, const uint64_t *cfg, int64_t smp, T *s_sm, int8_t *s8)
{
    const uint64_t *w = cfg + smp * md.nwords;
    for (int i = threadIdx.x; i < md.N; i += blockDim.x) {
        int s = spin_of(w, i);
        s_sm[i] = T(s);
        s8[i] = (int8_t)s;
    }
}

// ---------------------------------------------------------------------------
// log psi of fresh configurations
// ---------------------------------------------------------------------------
template <typename T, int MPL>
__global__ void __launch_bounds__(kThreads) k_log_psi(DevModel<T> md, const uint64_t *__restrict__ cfg, int64_t n,
                                                      double *__restrict__ out)
{
    __shared__ T s_sm[kMaxN];
    __shared__ int8_t s8[kMaxN];
    __shared__ sc<T> wacc[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rows = md.K * md.G;
    for (int64_t smp = blockIdx.x; smp < n; smp += gridDim.x) {
        load_spins(md, cfg, smp, s_sm, s8);
        __syncthreads();
        sc<T> acc{T(0), T(0), 0};
        for (int row = warp; row < rows; row += kWarps) {
            const int r = row / md.G, g = row - r * md.G;
            cx<T> thp[MPL], p[MPL];
            row_theta<T, MPL>(md, r, g, s_sm, thp, lane);
            cx<T> at = row_visible(md, r, g, s_sm, lane);
            for (int sg = 0; sg < md.nsign; ++sg) {
                const int sign = sg ? -1 : 1;
                sc<T> prod = row_cosh<T, MPL>(md, r, sign, thp, p, lane);
                acc = sc_add(acc, sc_mul(prod, row_lead(md, r, g, sign, at)));
            }
        }
        if (lane == 0) wacc[warp] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            sc<T> tot = wacc[0];
            for (int w = 1; w < kWarps; ++w) tot = sc_add(tot, wacc[w]);
            double re, im;
            if (!sc_finite(tot)) {
                flag_range(md.status);
                re = nan(""); im = nan("");
            } else if (sc_zero(tot)) {
                re = -INFINITY; im = 0.0;
            } else {
                double x = (double)tot.x, y = (double)tot.y;
                re = log(hypot(x, y)) + tot.e * 0.69314718055994530942;
                im = atan2(y, x);
            }
            out[2 * smp] = re;
            out[2 * smp + 1] = im;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Ratio engine: psi(s^D)/psi(s) for lists of flip sets D, accumulated into
// h1 = (H psi)/psi and h2 = (H^2 psi)/psi.
// ---------------------------------------------------------------------------
template <typename T> struct Entry {
    uint32_t sites;  // up to four site indices, one byte each, 0xFF = unused
    T c1, c2;        // coefficient of the ratio in h1 and in h2
};

// Candidates of the flip-set enumeration, in a fixed order.
//   mode 0 (E_loc): candidate q = bond q; valid if anti-aligned.
//   mode 1 (Lanczos): q = a * (4N + 1) + slot over the anti-aligned bonds
//     b1 = aa[a]; slot 0 = first-level exchange of b1; slot 1 + b2 = the
//     second-level configuration reached by exchanging b2 in s^{b1}:
//       b2 sharing one site with b1 (anti-aligned in s^{b1}) -> two flips,
//       b2 disjoint, anti-aligned and b2 > b1                  -> four flips,
//         counted twice (the order b2, b1 reaches the same configuration).
template <typename T>
__device__ __forceinline__ bool candidate(const DevModel<T> &md, int mode, int q, const int8_t *s8, const int16_t *aa,
                                          T diag, Entry<T> &e)
{
    const int nb = md.nbonds;
    if (mode == 0) {
        const int i = md.bond_i[q], j = md.bond_j[q];
        if (s8[i] == s8[j]) return false;
        e.sites = (uint32_t)i | ((uint32_t)j << 8) | 0xFFFF0000u;
        e.c1 = T(0.5) * bondJ(md, q);
        e.c2 = T(0);
        return true;
    }
    const int a = q / (nb + 1), slot = q - a * (nb + 1);
    const int b1 = aa[a];
    const int i1 = md.bond_i[b1], j1 = md.bond_j[b1];
    const T J1b = bondJ(md, b1);
    if (slot == 0) {
        // diagonal energy of s^{b1}
        T d = diag;
        for (int b = 0; b < nb; ++b) {
            const int i = md.bond_i[b], j = md.bond_j[b];
            const bool ti = (i == i1 || i == j1), tj = (j == i1 || j == j1);
            if (ti == tj) continue;  // untouched, or b1 itself
            const int si = s8[i], sj = s8[j];
            const int si2 = (i == i1) ? s8[j1] : (i == j1) ? s8[i1] : si;
            const int sj2 = (j == i1) ? s8[j1] : (j == j1) ? s8[i1] : sj;
            d += T(0.25) * bondJ(md, b) * T(si2 * sj2 - si * sj);
        }
        e.sites = (uint32_t)i1 | ((uint32_t)j1 << 8) | 0xFFFF0000u;
        e.c1 = T(0.5) * J1b;
        e.c2 = T(0.5) * J1b * d;
        return true;
    }
    const int b2 = slot - 1;
    if (b2 == b1) return false;
    const int i2 = md.bond_i[b2], j2 = md.bond_j[b2];
    const int shared = (i2 == i1) + (i2 == j1) + (j2 == i1) + (j2 == j1);
    const T J2b = bondJ(md, b2);
    if (shared == 0) {
        if (b2 < b1 || s8[i2] == s8[j2]) return false;
        e.sites = (uint32_t)i1 | ((uint32_t)j1 << 8) | ((uint32_t)i2 << 16) | ((uint32_t)j2 << 24);
        e.c1 = T(0);
        e.c2 = T(0.5) * J1b * J2b;
        return true;
    }
    // one shared site: spins of s^{b1} at the ends of b2
    auto sp = [&](int x) { return x == i1 ? s8[j1] : x == j1 ? s8[i1] : s8[x]; };
    if (sp(i2) == sp(j2)) return false;
    // symmetric difference of {i1,j1} and {i2,j2}
    int u = -1, v = -1;
    if (i1 != i2 && i1 != j2) u = i1; else u = j1;
    if (i2 != i1 && i2 != j1) v = i2; else v = j2;
    e.sites = (uint32_t)u | ((uint32_t)v << 8) | 0xFFFF0000u;
    e.c1 = T(0);
    e.c2 = T(0.25) * J1b * J2b;
    return true;
}

template <typename T, int MPL>
__global__ void __launch_bounds__(kThreads) k_ratio(DevModel<T> md, const uint64_t *__restrict__ cfg, int64_t n,
                                                    int mode, int chunk, double *__restrict__ h1_out,
                                                    double *__restrict__ h2_out)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T s_sm[kMaxN];
    __shared__ int8_t s8[kMaxN];
    __shared__ int16_t aa[4 * kMaxN];
    __shared__ int n_aa;
    __shared__ int n_ent, cursor, first_over;
    __shared__ int wcount[kWarps];
    __shared__ sc<T> wacc0[kWarps];
    __shared__ sc<T> S0;
    __shared__ double red[kWarps][4];
    __shared__ T diag_sh, cst_sh;
    __shared__ double Hs[4];  // running sums of c1 R (re, im) and c2 R (re, im)

    Entry<T> *ent = reinterpret_cast<Entry<T> *>(smem_raw);
    sc<T> *acc = reinterpret_cast<sc<T> *>(smem_raw + sizeof(Entry<T>) * chunk);  // [kWarps][chunk]

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rows = md.K * md.G;
    const int nb = md.nbonds;

    for (int64_t smp = blockIdx.x; smp < n; smp += gridDim.x) {
        load_spins(md, cfg, smp, s_sm, s8);
        __syncthreads();
        if (warp == 0) {
            // diagonal energy, anti-aligned bond list (ordered), and the sum of
            // J_b^2/4 over anti-aligned bonds (second-level returns to s)
            T d = T(0), c = T(0);
            int base = 0;
            for (int b0 = 0; b0 < nb; b0 += 32) {
                const int b = b0 + lane;
                bool isaa = false;
                if (b < nb) {
                    const int si = s8[md.bond_i[b]], sj = s8[md.bond_j[b]];
                    const T J = bondJ(md, b);
                    d += T(0.25) * J * T(si * sj);
                    isaa = si != sj;
                    if (isaa) c += T(0.25) * J * J;
                }
                const unsigned m = __ballot_sync(0xffffffffu, isaa);
                if (isaa) aa[base + __popc(m & ((1u << lane) - 1u))] = (int16_t)b;
                base += __popc(m);
            }
            for (int o = 16; o > 0; o >>= 1) {
                d += __shfl_xor_sync(0xffffffffu, d, o);
                c += __shfl_xor_sync(0xffffffffu, c, o);
            }
            if (lane == 0) { diag_sh = d; cst_sh = c; n_aa = base; cursor = 0; }
        }
        __syncthreads();
        const int ncand = mode == 0 ? nb : n_aa * (nb + 1);
        bool first_chunk = true;
        while (true) {
            // ---- gather up to `chunk` valid entries, in candidate order ----
            if (threadIdx.x == 0) n_ent = 0;
            __syncthreads();
            while (true) {
                const int cur = cursor;
                if (cur >= ncand || n_ent >= chunk) break;
                const int q = cur + threadIdx.x;
                Entry<T> e;
                const bool valid = q < ncand && candidate(md, mode, q, s8, aa, diag_sh, e);
                const unsigned bm = __ballot_sync(0xffffffffu, valid);
                if (lane == 0) wcount[warp] = __popc(bm);
                if (threadIdx.x == 0) first_over = INT_MAX;
                __syncthreads();
                int pos = __popc(bm & ((1u << lane) - 1u));
                for (int w = 0; w < warp; ++w) pos += wcount[w];
                const int room = chunk - n_ent;
                if (valid) {
                    if (pos < room) ent[n_ent + pos] = e;
                    else atomicMin(&first_over, q);
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    int tot = 0;
                    for (int w = 0; w < kWarps; ++w) tot += wcount[w];
                    n_ent += tot < room ? tot : room;
                    cursor = first_over != INT_MAX ? first_over : cur + blockDim.x;
                }
                __syncthreads();
            }
            const int ne = n_ent;
            if (ne == 0 && !first_chunk) break;
            // ---- accumulate every row's contribution to every entry ----
            for (int idx = threadIdx.x; idx < kWarps * ne; idx += blockDim.x) {
                const int w = idx / ne, e = idx - w * ne;
                acc[w * chunk + e] = sc<T>{T(0), T(0), 0};
            }
            __syncthreads();
            sc<T> a0{T(0), T(0), 0};
            for (int row = warp; row < rows; row += kWarps) {
                const int r = row / md.G, g = row - r * md.G;
                const uint8_t *pg = md.perm + (size_t)g * md.N;
                cx<T> thp[MPL], p[MPL];
                row_theta<T, MPL>(md, r, g, s_sm, thp, lane);
                const cx<T> at = row_visible(md, r, g, s_sm, lane);
                const cx2<T> *Xr = md.X + (size_t)r * md.N * md.M;
                const cx2<T> *XAr = md.XA + (size_t)r * md.N;
                for (int sg = 0; sg < md.nsign; ++sg) {
                    const int sign = sg ? -1 : 1;
                    const sc<T> prod = row_cosh<T, MPL>(md, r, sign, thp, p, lane);
                    const sc<T> term = sc_mul(prod, row_lead(md, r, g, sign, at));
                    if (first_chunk) a0 = sc_add(a0, term);
                    for (int e = 0; e < ne; ++e) {
                        const uint32_t st = ent[e].sites;
                        int kk[4], sf[4], nf = 0;
#pragma unroll
                        for (int f = 0; f < 4; ++f) {
                            const int site = (st >> (8 * f)) & 0xFF;
                            kk[f] = site != 0xFF ? pg[site] : 0;
                            sf[f] = site != 0xFF ? sign * s8[site] : 0;
                            nf += site != 0xFF;
                        }
                        sc<T> fp{T(1), T(0), 0};
#pragma unroll
                        for (int j = 0; j < MPL; ++j) {
                            const int m = lane + 32 * j;
                            if (m < md.M) {
                                cx<T> eD{T(1), T(0)}, eDi{T(1), T(0)};
#pragma unroll
                                for (int f = 0; f < 4; ++f) {
                                    if (f < nf) {
                                        const cx2<T> x = Xr[(size_t)kk[f] * md.M + m];
                                        if (sf[f] > 0) { eD = cmul(eD, x.a); eDi = cmul(eDi, x.b); }
                                        else { eD = cmul(eD, x.b); eDi = cmul(eDi, x.a); }
                                    }
                                }
                                const cx<T> d = csub(eD, eDi);
                                const cx<T> fac = cadd(eDi, cmul(p[j], d));
                                const cx<T> q = cmul(mk(fp.x, fp.y), fac);
                                fp.x = q.x;
                                fp.y = q.y;
                            }
                        }
                        fp = warp_prod(fp);
                        if (lane == 0) {
                            cx<T> eA{T(1), T(0)};
                            if (md.use_bias) {
#pragma unroll
                                for (int f = 0; f < 4; ++f)
                                    if (f < nf) {
                                        const cx2<T> x = XAr[kk[f]];
                                        eA = cmul(eA, sf[f] > 0 ? x.a : x.b);
                                    }
                            }
                            sc<T> t = sc_mul(term, fp);
                            const cx<T> tt = cmul(mk(t.x, t.y), eA);
                            t.x = tt.x;
                            t.y = tt.y;
                            acc[warp * chunk + e] = sc_add(acc[warp * chunk + e], sc_norm(t));
                        }
                    }
                }
            }
            if (first_chunk && lane == 0) wacc0[warp] = a0;
            __syncthreads();
            if (first_chunk && threadIdx.x == 0) {
                sc<T> tot = wacc0[0];
                for (int w = 1; w < kWarps; ++w) tot = sc_add(tot, wacc0[w]);
                S0 = tot;
            }
            __syncthreads();
            // ---- ratios R_e = S_e / S0 and their weighted sums ----
            double p1x = 0, p1y = 0, p2x = 0, p2y = 0;
            for (int e = threadIdx.x; e < ne; e += blockDim.x) {
                sc<T> se = acc[e];
                for (int w = 1; w < kWarps; ++w) se = sc_add(se, acc[w * chunk + e]);
                const sc<T> s0 = S0;
                double Rx = 0, Ry = 0;
                if (!sc_zero(se)) {
                    const double sc2 = ldexp(1.0, se.e - s0.e);
                    const double ax = (double)se.x, ay = (double)se.y, bx = (double)s0.x, by = (double)s0.y;
                    const double den = bx * bx + by * by;
                    Rx = (ax * bx + ay * by) / den * sc2;
                    Ry = (ay * bx - ax * by) / den * sc2;
                }
                const double c1 = (double)ent[e].c1, c2 = (double)ent[e].c2;
                p1x += c1 * Rx; p1y += c1 * Ry;
                p2x += c2 * Rx; p2y += c2 * Ry;
            }
            for (int o = 16; o > 0; o >>= 1) {
                p1x += __shfl_xor_sync(0xffffffffu, p1x, o);
                p1y += __shfl_xor_sync(0xffffffffu, p1y, o);
                p2x += __shfl_xor_sync(0xffffffffu, p2x, o);
                p2y += __shfl_xor_sync(0xffffffffu, p2y, o);
            }
            if (lane == 0) { red[warp][0] = p1x; red[warp][1] = p1y; red[warp][2] = p2x; red[warp][3] = p2y; }
            __syncthreads();
            if (threadIdx.x == 0) {
                if (first_chunk) { Hs[0] = Hs[1] = Hs[2] = Hs[3] = 0.0; }
                for (int w = 0; w < kWarps; ++w)
                    for (int c = 0; c < 4; ++c) Hs[c] += red[w][c];
            }
            first_chunk = false;
            __syncthreads();
            if (cursor >= ncand) break;
        }
        if (threadIdx.x == 0) {
            const sc<T> s0 = S0;
            const double diag = (double)diag_sh;
            const double h1x = diag + Hs[0], h1y = Hs[1];
            if (!sc_finite(s0) || sc_zero(s0) || !isfinite(h1x) || !isfinite(h1y)) flag_range(md.status);
            if (h1_out) { h1_out[2 * smp] = h1x; h1_out[2 * smp + 1] = h1y; }
            if (mode == 1 && h2_out) {
                h2_out[2 * smp] = diag * h1x + Hs[2] + (double)cst_sh;
                h2_out[2 * smp + 1] = diag * h1y + Hs[3];
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
#define NNQS_MPL_DISPATCH(MPLV, ...)                                   \
    switch (mpl_slot(MPLV)) {                                           \
    case 1: { constexpr int MPL = 1; __VA_ARGS__; } break;              \
    case 2: { constexpr int MPL = 2; __VA_ARGS__; } break;              \
    case 3: { constexpr int MPL = 3; __VA_ARGS__; } break;              \
    case 4: { constexpr int MPL = 4; __VA_ARGS__; } break;              \
    case 6: { constexpr int MPL = 6; __VA_ARGS__; } break;              \
    case 8: { constexpr int MPL = 8; __VA_ARGS__; } break;              \
    case 13: { constexpr int MPL = 13; __VA_ARGS__; } break;            \
    default: { constexpr int MPL = 16; __VA_ARGS__; } break;            \
    }

int mpl_slot(int M)
{
    const int need = (M + 31) / 32;
    const int opts[] = {1, 2, 3, 4, 6, 8, 13, 16};
    for (int o : opts)
        if (o >= need) return o;
    return 16;
}

template <typename T>
cudaError_t launch_log_psi(const DevModel<T> &md, const uint64_t *cfg, int64_t n, double *out, int nsm,
                           cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    cudaError_t err = cudaSuccess;
    NNQS_MPL_DISPATCH(md.M, {
        int per = 0;
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_log_psi<T, MPL>, kThreads, 0);
        const int64_t grid = (int64_t)(per > 0 ? per : 1) * nsm;
        const int g = (int)(n < grid ? n : grid);
        if (err == cudaSuccess) k_log_psi<T, MPL><<<g, kThreads, 0, st>>>(md, cfg, n, out);
    });
    if (err != cudaSuccess) return err;
    return cudaGetLastError();
}

template <typename T> size_t ratio_smem(int chunk) { return (sizeof(Entry<T>) + kWarps * sizeof(sc<T>)) * (size_t)chunk; }

template <typename T>
cudaError_t launch_ratio(const DevModel<T> &md, const uint64_t *cfg, int64_t n, int mode, double *h1, double *h2,
                         int nsm, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int chunk = mode == 0 ? md.nbonds : 512;
    const size_t smem = ratio_smem<T>(chunk);
    cudaError_t err = cudaSuccess;
    NNQS_MPL_DISPATCH(md.M, {
        err = cudaFuncSetAttribute(k_ratio<T, MPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per = 0;
        if (err == cudaSuccess)
            err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_ratio<T, MPL>, kThreads, smem);
        const int64_t grid = (int64_t)(per > 0 ? per : 1) * nsm;
        const int g = (int)(n < grid ? n : grid);
        if (err == cudaSuccess) k_ratio<T, MPL><<<g, kThreads, smem, st>>>(md, cfg, n, mode, chunk, h1, h2);
    });
    if (err != cudaSuccess) return err;
    return cudaGetLastError();
}

template cudaError_t launch_log_psi<float>(const DevModel<float> &, const uint64_t *, int64_t, double *, int, cudaStream_t);
template cudaError_t launch_log_psi<double>(const DevModel<double> &, const uint64_t *, int64_t, double *, int, cudaStream_t);
template cudaError_t launch_ratio<float>(const DevModel<float> &, const uint64_t *, int64_t, int, double *, double *, int, cudaStream_t);
template cudaError_t launch_ratio<double>(const DevModel<double> &, const uint64_t *, int64_t, int, double *, double *, int, cudaStream_t);

}  // namespace nnqs
