// k_eloc_fast.cu -- E_loc (Eq. 10) in FP32 with the per-bond tables in shared
// memory and packed f32x2 arithmetic.
//
// For a sample s, a row t = (r, g, sign) of the projected sum (Eqs. 4-6) with
// p_m = e^{theta_m}/(2cosh theta_m), and an anti-aligned bond b, the row's ratio
// is e^{C} prod_m (1 + p_m (U_m - 1)): U = e^{2 Delta} and the prefactor
// exponent C belong to the bond's image b' = g(b) and its orientation (the
// tables of the connected-configuration engine).  With q_m = (1 - p_m)/p_m
// the factor is p_m (q_m + U_m); the product of the p_m is the row's, so per
// element the work is q + U (two packed adds) and the running product.  Then
//   E_loc = diag(s) + [sum_t w_t P_t sum_b (J_b/2) e^{C_b} prod_m (q_m + U_m)]
//                     / [sum_t w_t],
// w_t = c_r chi(g) chi_P e^{+-a.T_g s} prod_m 2cosh(theta_m) the row's term and
// P_t = prod_m p_m.  q = e^{-2 theta} is formed directly (1/p - 1 would lose
// its relative precision where p is near 1), and as 2cosh(theta) p = e^theta,
// w_t P_t = c_r chi(g) chi_P e^{+-a.T_g s + sum_m theta_m} and w_t is that
// times prod_m (1 + q_m): no cosh or division on this path.  A row whose group
// has some |p_m| < 2^-12 (|1 + q| above 2^12) takes the plain factors
// 1 + p_m (U_m - 1) instead, with p from cosh2.
//
// Layout: one CTA per SM (the tables of one model, 2 x 4N rows per RBM, are
// copied into its shared memory once), one sample at a time.  A group of 8
// lanes owns a row; lane l owns the unit pairs k = l + 8 j (units 2k, 2k + 1),
// whose q sit in registers as packed pairs.  The table row of a bond image is
// stored as float4 (Ux_2k, Ux_2k+1, Uy_2k, Uy_2k+1) per pair, so a group reads
// one contiguous 128-byte row segment per step (conflict-free).  Entries
// (anti-aligned bonds) go 8 at a time: lane l decodes entry l (image bond,
// orientation, prefactor) and the group shares the table offsets by shuffle; a
// butterfly product-reduce-scatter over the group leaves lane l with entry l's
// full product, which it weights and adds into its FP32 sum for the row.
#include <cstdlib>

#include "common.cuh"
#include "f2.cuh"
#include "kernels.h"

namespace nnqs {

constexpr int kEfGL = 8;             // lanes per row group
constexpr int kEfMaxThreads = 512;   // at most 16 warps (128 registers per thread)

struct EfArgs {
    const float4 *tp;     // [K][2] blocks of BS float4: [NB][MH] paired per-bond tables U = 1 + T
    const sc<float> *ep;  // [K][2][NB] e^{+C}, e^{-C}
    int MH;               // unit pairs per table row
    int BS;               // float4 per (r, orientation) block: NB MH + padding
    int warps;
    int plain;            // 1: every row takes the plain factors (test hook)
    int w_smem;           // 1: the weights W are staged in shared memory (sign-paired variant)
};

// The entries of one row and sign, 8 at a time: sum over the anti-aligned
// bonds of (J_b/2) e^{C_b} prod_m f_m into the owner lanes' (accx, accy)
// (FP32, scaled by 2^eref) or, outside the FP32 window, (Ox, Oy).
// QF: f = q + U (ca, cb = q); else f = 1 + p (U - 1) (ca, cb, cc = Re p,
// Im p, -Im p).
template <int NP, bool QF>
__device__ __forceinline__ void ef_entries(const DevModel<float> &md, const float4 *tps, const sc<float> *eps,
                                           const uint16_t *aa, const uint16_t *bps, int naa, int ntrip, int r, int sg,
                                           int MH, const f2 (&ca)[NP], const f2 (&cb)[NP], const f2 (&cc)[NP],
                                           int eref, int gl, int gbase, float &accx, float &accy, double &Ox,
                                           double &Oy)
{
    const int NB = md.nbonds;
    const f2 one2 = f2_pack(1.f, 1.f);
    // ntrip >= naa is the same in every group of the warp (the shuffles below
    // take all 32 lanes)
    for (int e0 = 0; e0 < ntrip; e0 += kEfGL) {
        // lane gl: table offset and weighted prefactor of entry e0 + gl
        const int e = e0 + gl;
        int off = 0;
        sc<float> pre{0.f, 0.f, 0};
        if (e < naa) {
            const uint16_t code = aa[e];
            const int b = code & 0x7fff;
            const uint16_t bp = bps[b];
            const int bb = bp & 0x7fff;
            // orientation of the exchange on the image bond, for this sign
            const bool pos = ((code >> 15) != 0) != ((bp >> 15) != 0);   // s_i flip-corrected
            const int o = (pos != (sg != 0)) ? 0 : 1;
            off = ((r * 2 + o) * NB + bb) * MH;
            pre = eps[(r * 2 + o) * NB + bb];   // (J_b / 2) e^{+-C}
        }
        float rx[kEfGL], ry[kEfGL];
        int re[kEfGL];
#pragma unroll
        for (int q = 0; q < kEfGL; ++q) {
            const float4 *trow = tps + __shfl_sync(0xffffffffu, off, gbase + q) + gl;
            // running products of the even and odd units (packed)
            f2 Rx = one2, Ry = 0;
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                f2 ux, uy;
                lds128(trow + kEfGL * j, ux, uy);
                f2 fx, fy;
                if constexpr (QF) {
                    fx = add2(ux, ca[j]);
                    fy = add2(uy, cb[j]);
                } else {
                    const f2 tx = sub2(ux, one2);
                    fx = fma2(cc[j], uy, fma2(ca[j], tx, one2));   // 1 + px tx - py ty
                    fy = fma2(ca[j], uy, mul2(cb[j], tx));         // px ty + py tx
                }
                if (j == 0) {
                    Rx = fx; Ry = fy;
                } else {
                    const f2 nx = sub2(mul2(Rx, fx), mul2(Ry, fy));
                    Ry = fma2(Rx, fy, mul2(Ry, fx));
                    Rx = nx;
                }
            }
            // even x odd, then mantissa / exponent
            float x = f2_lo(Rx) * f2_hi(Rx) - f2_lo(Ry) * f2_hi(Ry);
            float y = f2_lo(Rx) * f2_hi(Ry) + f2_lo(Ry) * f2_hi(Rx);
            re[q] = nrm(x, y);
            rx[q] = x;
            ry[q] = y;
        }
        // butterfly product-reduce-scatter: lane gl ends with entry gl's product
#pragma unroll
        for (int lev = 0; lev < 3; ++lev) {
            const int o = 4 >> lev;          // lane distance 4, 2, 1
            const int cnt = 4 >> lev;        // entries exchanged
            const bool upper = (gl & o) != 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (q < cnt) {
                    // keep slot q (lower lanes keep the low half), send the other
                    const float sx = upper ? rx[q] : rx[q + cnt];
                    const float sy = upper ? ry[q] : ry[q + cnt];
                    const int se = upper ? re[q] : re[q + cnt];
                    const float kx = upper ? rx[q + cnt] : rx[q];
                    const float ky = upper ? ry[q + cnt] : ry[q];
                    const int ke = upper ? re[q + cnt] : re[q];
                    const float gx = __shfl_xor_sync(0xffffffffu, sx, o);
                    const float gy = __shfl_xor_sync(0xffffffffu, sy, o);
                    const int ge = __shfl_xor_sync(0xffffffffu, se, o);
                    rx[q] = kx * gx - ky * gy;
                    ry[q] = kx * gy + ky * gx;
                    re[q] = ke + ge;
                }
            }
        }
        if (e < naa) {
            const float vx = rx[0] * pre.x - ry[0] * pre.y, vy = rx[0] * pre.y + ry[0] * pre.x;
            const int d = re[0] + pre.e + eref;
            if (d > -100 && d < 100) {
                const float f = __uint_as_float((uint32_t)(d + 127) << 23);
                accx = fmaf(f, vx, accx);
                accy = fmaf(f, vy, accy);
            } else {
                const double f = pow2i<double>(d);
                Ox += f * (double)vx;
                Oy += f * (double)vy;
            }
        }
    }
}

template <int NP>
__global__ void __launch_bounds__(kEfMaxThreads, 1)
    k_eloc_fast(DevModel<float> md, EfArgs ea, const uint64_t *__restrict__ cfg, int64_t n, double *__restrict__ h1_out)
{
    constexpr int NG = 32 / kEfGL;
    extern __shared__ __align__(16) unsigned char smem[];
    const int NB = md.nbonds, K = md.K, MH = ea.MH, N = md.N, M = md.M;
    float4 *tps = reinterpret_cast<float4 *>(smem);                                      // [K][2][NB][MH]
    sc<float> *eps = reinterpret_cast<sc<float> *>(tps + (size_t)K * 2 * NB * MH);      // [K][2][NB]
    uint16_t *gbp = reinterpret_cast<uint16_t *>(eps + (size_t)K * 2 * NB);            // [groups][NB]
    uint8_t *gperm = reinterpret_cast<uint8_t *>(gbp + (size_t)(blockDim.x / kEfGL) * NB);   // [groups][N]
    __shared__ float s_sm[kMaxN];
    __shared__ int8_t s8[kMaxN];
    __shared__ uint16_t aa[4 * kMaxN];   // anti-aligned bond | (s_i > 0) << 15
    __shared__ int n_aa;
    __shared__ float diag_sh;
    __shared__ sc<double> gsum[2][kEfMaxThreads / kEfGL];   // per row group: sum of w_t P_t A_t, sum of w_t

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int grp = lane / kEfGL, gl = lane % kEfGL, gbase = grp * kEfGL;
    const int gidx = warp * NG + grp, ngroups = nwarps * NG;
    uint8_t *pgs = gperm + (size_t)gidx * N;
    uint16_t *bps = gbp + (size_t)gidx * NB;

    // tables into shared memory (once per CTA)
    {
        const int4 *src = reinterpret_cast<const int4 *>(ea.tp);
        int4 *dst = reinterpret_cast<int4 *>(tps);
        for (int q = threadIdx.x; q < K * 2 * NB * MH; q += blockDim.x) dst[q] = src[q];
        for (int q = threadIdx.x; q < K * 2 * NB; q += blockDim.x) eps[q] = ea.ep[q];
    }

    for (int64_t smp = blockIdx.x; smp < n; smp += gridDim.x) {
        const uint64_t *w = cfg + smp * md.nwords;
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            const int sv = spin_of(w, i);
            s_sm[i] = (float)sv;
            s8[i] = (int8_t)sv;
        }
        for (int q = threadIdx.x; q < 2 * ngroups; q += blockDim.x) gsum[q / ngroups][q % ngroups] = sc<double>{0.0, 0.0, 0};
        __syncthreads();
        if (warp == 0) {
            float d = 0.f;
            int base = 0;
            for (int b0 = 0; b0 < NB; b0 += 32) {
                const int b = b0 + lane;
                bool isaa = false;
                int si = 0;
                if (b < NB) {
                    si = s8[md.bond_i[b]];
                    const int sj = s8[md.bond_j[b]];
                    d += 0.25f * bondJ(md, b) * (float)(si * sj);
                    isaa = si != sj;
                }
                const unsigned bm = __ballot_sync(0xffffffffu, isaa);
                if (isaa) aa[base + __popc(bm & ((1u << lane) - 1u))] = (uint16_t)(b | (si > 0 ? 0x8000 : 0));
                base += __popc(bm);
            }
            for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
            if (lane == 0) { n_aa = base; diag_sh = d; }
        }
        __syncthreads();
        const int naa = n_aa;

        // (every group of a warp runs the same trip counts, so that the warp's
        // shuffles see all lanes; groups past the last row run row 0 and add
        // nothing).  A last wave of at most ngroups / 2 (ngroups / 4) rows
        // gives each row 2 (4) groups, each with its share of the entries.
        for (int rbase = 0; rbase < K * md.G;) {
            const int left = K * md.G - rbase;
            const int split = 4 * left <= ngroups ? 4 : 2 * left <= ngroups ? 2 : 1;
            const int part = gidx % split;
            const bool active = rbase + gidx / split < K * md.G;
            const int row = active ? rbase + gidx / split : 0;
            const int e_lo = part * naa / split, e_n = (part + 1) * naa / split - e_lo;
            const int e_max = (naa + split - 1) / split;   // the largest share: the same trip count in every group
            rbase += ngroups / split;
            const int r = row / md.G, g = row - r * md.G;
            __syncwarp();
            for (int i = gl; i < N; i += kEfGL) pgs[i] = md.perm[(size_t)g * N + i];
            for (int b = gl; b < NB; b += kEfGL) bps[b] = md.bperm[(size_t)g * NB + b];
            __syncwarp();
            // ---- theta' = W_r T_g s for the lane's units (pairs k = gl + 8 j) ----
            float tx[2 * NP], ty[2 * NP];
#pragma unroll
            for (int u = 0; u < 2 * NP; ++u) { tx[u] = 0.f; ty[u] = 0.f; }
            const cx<float> *Wr = md.Wt + (size_t)r * N * M;
            for (int i = 0; i < N; ++i) {
                const cx<float> *wk = Wr + (size_t)pgs[i] * M;
                const float si = s_sm[i];
#pragma unroll
                for (int j = 0; j < NP; ++j) {
                    const int m = 2 * (gl + kEfGL * j);
                    if ((M & 1) == 0 && m + 1 < M) {   // M even: both units of the pair, one aligned 16-byte load
                        const float4 a = *reinterpret_cast<const float4 *>(wk + m);
                        tx[2 * j] = fmaf(si, a.x, tx[2 * j]); ty[2 * j] = fmaf(si, a.y, ty[2 * j]);
                        tx[2 * j + 1] = fmaf(si, a.z, tx[2 * j + 1]); ty[2 * j + 1] = fmaf(si, a.w, ty[2 * j + 1]);
                    } else {
                        if (m < M) { const cx<float> a = wk[m]; tx[2 * j] = fmaf(si, a.x, tx[2 * j]); ty[2 * j] = fmaf(si, a.y, ty[2 * j]); }
                        if (m + 1 < M) { const cx<float> a = wk[m + 1]; tx[2 * j + 1] = fmaf(si, a.x, tx[2 * j + 1]); ty[2 * j + 1] = fmaf(si, a.y, ty[2 * j + 1]); }
                    }
                }
            }
            cx<float> at{0.f, 0.f};
            if (md.use_bias) {
                const cx<float> *ar = md.avec + (size_t)r * N;
                for (int i = gl; i < N; i += kEfGL) { const cx<float> a = ar[pgs[i]]; at.x += s_sm[i] * a.x; at.y += s_sm[i] * a.y; }
#pragma unroll
                for (int o = kEfGL / 2; o > 0; o >>= 1) {
                    at.x += __shfl_xor_sync(0xffffffffu, at.x, o);
                    at.y += __shfl_xor_sync(0xffffffffu, at.y, o);
                }
            }
            for (int sg = 0; sg < md.nsign; ++sg) {
                const float sign = sg ? -1.f : 1.f;
                // ---- q_m = e^{-2 theta_m} = (1 - p_m)/p_m of the lane's units; the row's
                //      term x prod_m p_m is lead e^{sum_m theta_m} (2 cosh(theta) p = e^theta)
                //      and its term that times prod_m (1 + q_m) ----
                f2 ca[NP], cb[NP];
                float stx = 0.f, sty = 0.f;
                f2 Qx = f2_pack(1.f, 1.f), Qy = 0;
                int qlo = 0, qhi = 0;
                bool small = ea.plain != 0;   // some |p| < 2^-12 (|1 + q| > 2^12): the plain factors
                const cx<float> *br = md.bvec + (size_t)r * M;
#pragma unroll
                for (int j = 0; j < NP; ++j) {
                    float qxv[2], qyv[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int m = 2 * (gl + kEfGL * j) + h;
                        qxv[h] = 0.f; qyv[h] = 0.f;   // units past M: q = 0 (their U is 1)
                        if (m < M) {
                            cx<float> th{sign * tx[2 * j + h], sign * ty[2 * j + h]};
                            if (md.use_bias) { const cx<float> b = br[m]; th.x += b.x; th.y += b.y; }
                            stx += th.x;
                            sty += th.y;
                            const float e = exp2f(-2.8853900817779268f * th.x);   // e^{-2 Re theta}
                            float sn, cs;
                            sincosf(2.f * th.y, &sn, &cs);
                            qxv[h] = e * cs;
                            qyv[h] = -e * sn;
                            const float ax = 1.f + qxv[h];
                            small = small || !(ax * ax + qyv[h] * qyv[h] <= 0x1p24f);
                        }
                    }
                    ca[j] = f2_pack(qxv[0], qxv[1]);
                    cb[j] = f2_pack(qyv[0], qyv[1]);
                    const f2 fx = add2(ca[j], f2_pack(1.f, 1.f));
                    const f2 nx = sub2(mul2(Qx, fx), mul2(Qy, cb[j]));
                    Qy = fma2(Qx, cb[j], mul2(Qy, fx));
                    Qx = nx;
                    if ((j % 3) == 2 || j == NP - 1) {
                        float xl = f2_lo(Qx), yl = f2_lo(Qy), xh = f2_hi(Qx), yh = f2_hi(Qy);
                        qlo += nrm(xl, yl);
                        qhi += nrm(xh, yh);
                        Qx = f2_pack(xl, xh);
                        Qy = f2_pack(yl, yh);
                    }
                }
                const cx<float> lc = md.logc[r];
                float chg = md.chi[g];
                if (sg && md.chiP < 0) chg = -chg;

                float accx = 0.f, accy = 0.f;
                double Ox = 0.0, Oy = 0.0;
                sc<float> mult;
                if (!__any_sync(0xffffffffu, small)) {
#pragma unroll
                    for (int o = 1; o < kEfGL; o <<= 1) {
                        stx += __shfl_xor_sync(0xffffffffu, stx, o);
                        sty += __shfl_xor_sync(0xffffffffu, sty, o);
                    }
                    float u = f2_lo(Qx) * f2_hi(Qx) - f2_lo(Qy) * f2_hi(Qy);
                    float v = f2_lo(Qx) * f2_hi(Qy) + f2_lo(Qy) * f2_hi(Qx);
                    const int qe = qlo + qhi + nrm(u, v);
                    const sc<float> Q = group_prod<kEfGL>(sc<float>{u, v, qe});
                    // lead e^{sum theta} = term x prod p, as mantissa x 2^(e + Q.e), with the
                    // entries scaled by 2^-Q.e (near 2^0, as prod (q + U) ~ prod (1 + q))
                    sc<float> lead = sc_exp(cx<float>{lc.x + sign * at.x + stx, lc.y + sign * at.y + sty});
                    lead.x *= chg; lead.y *= chg;
                    lead = sc_norm(lead);
                    const sc<float> wt = sc_mul(lead, Q);   // the row term
                    if (gl == 0 && active && part == 0)
                        gsum[1][gidx] = sc_add(gsum[1][gidx], sc<double>{(double)wt.x, (double)wt.y, wt.e});
                    ef_entries<NP, true>(md, tps, eps, aa + e_lo, bps, e_n, e_max, r, sg, MH, ca, cb, cb, -Q.e, gl,
                                         gbase, accx, accy, Ox, Oy);
                    mult = sc<float>{lead.x, lead.y, lead.e + Q.e};
                } else {
                    // the plain factors 1 + p (U - 1) with p and prod 2 cosh(theta) from cosh2
                    f2 cc[NP];
                    sc<float> prod{1.f, 0.f, 0};
#pragma unroll
                    for (int j = 0; j < NP; ++j) {
                        float pxv[2], pyv[2];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int m = 2 * (gl + kEfGL * j) + h;
                            pxv[h] = 1.f; pyv[h] = 0.f;   // units past M: p = 1 (their U is 1)
                            if (m < M) {
                                cx<float> th{sign * tx[2 * j + h], sign * ty[2 * j + h]};
                                if (md.use_bias) { const cx<float> b = br[m]; th.x += b.x; th.y += b.y; }
                                cx<float> mant, pv;
                                int k;
                                cosh2(th, mant, k, pv);
                                pxv[h] = pv.x; pyv[h] = pv.y;
                                const cx<float> z = cmul(mk(prod.x, prod.y), mant);
                                prod = sc_norm(sc<float>{z.x, z.y, prod.e + k});
                            }
                        }
                        ca[j] = f2_pack(pxv[0], pxv[1]);
                        cb[j] = f2_pack(pyv[0], pyv[1]);
                        cc[j] = f2_pack(-pyv[0], -pyv[1]);
                    }
                    prod = group_prod<kEfGL>(prod);
                    sc<float> lead = sc_exp(cx<float>{lc.x + sign * at.x, lc.y + sign * at.y});
                    lead.x *= chg; lead.y *= chg;
                    const sc<float> wt = sc_mul(prod, sc_norm(lead));
                    if (gl == 0 && active && part == 0)
                        gsum[1][gidx] = sc_add(gsum[1][gidx], sc<double>{(double)wt.x, (double)wt.y, wt.e});
                    ef_entries<NP, false>(md, tps, eps, aa + e_lo, bps, e_n, e_max, r, sg, MH, ca, cb, cc, 0, gl,
                                          gbase, accx, accy, Ox, Oy);
                    mult = wt;
                }
                double ax = (double)accx + Ox, ay = (double)accy + Oy;
#pragma unroll
                for (int o = kEfGL / 2; o > 0; o >>= 1) {
                    ax += __shfl_xor_sync(0xffffffffu, ax, o);
                    ay += __shfl_xor_sync(0xffffffffu, ay, o);
                }
                if (gl == 0 && active) gsum[0][gidx] = sc_add(gsum[0][gidx], sd_mul(mult, ax, ay));
            }
        }
        __syncthreads();
        if (warp == 0) {   // the groups' sums, a tree over the lanes of warp 0
            sc<double> t1{0.0, 0.0, 0}, t0{0.0, 0.0, 0};
            for (int q = lane; q < ngroups; q += 32) { t1 = sc_add(t1, gsum[0][q]); t0 = sc_add(t0, gsum[1][q]); }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const sc<double> u1{__shfl_xor_sync(0xffffffffu, t1.x, o), __shfl_xor_sync(0xffffffffu, t1.y, o),
                                    __shfl_xor_sync(0xffffffffu, t1.e, o)};
                const sc<double> u0{__shfl_xor_sync(0xffffffffu, t0.x, o), __shfl_xor_sync(0xffffffffu, t0.y, o),
                                    __shfl_xor_sync(0xffffffffu, t0.e, o)};
                t1 = sc_add(t1, u1);
                t0 = sc_add(t0, u0);
            }
            if (lane == 0) {
                const double den = t0.x * t0.x + t0.y * t0.y;
                const double f = ldexp(1.0, t1.e - t0.e);
                const double rx = (t1.x * t0.x + t1.y * t0.y) / den * f, ry = (t1.y * t0.x - t1.x * t0.y) / den * f;
                const double h1x = (double)diag_sh + rx;
                if (sc_zero(t0) || !isfinite(h1x) || !isfinite(ry)) flag_range(md.status);
                h1_out[2 * smp] = h1x;
                h1_out[2 * smp + 1] = ry;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Sign-paired variant (models with spin inversion): two groups of 4 lanes take
// the two signs of one row.  They share the row's theta' (each lane computes
// the unit pairs of one parity and swaps the other parity with its partner
// lane), its images and the entry list; lane l owns the unit pairs
// k = l + 4 j (j < NP), so that a row of 8 NP units has no padding when
// M = 8 NP.  The (r, orientation) blocks of the tables are BS float4 apart,
// an odd multiple of 64 bytes past NB MH, so that the pair's two 64-byte reads
// of one entry (the same image bond in opposite orientations) fall in
// different bank halves.
// ---------------------------------------------------------------------------
constexpr int kEpGL = 4;
constexpr int kEpQI = 2;   // entries whose running products interleave

template <int NP, bool QF>
__device__ __forceinline__ void ep_entries(const DevModel<float> &md, const float4 *tps, const sc<float> *eps,
                                           const uint16_t *aa, const uint16_t *bps, int naa, int ntrip, int r, int sg,
                                           int MH, int BS, const f2 (&ca)[NP], const f2 (&cb)[NP],
                                           const f2 (&cc)[NP], int eref, int gl, int gbase, float &accx, float &accy,
                                           double &Ox, double &Oy)
{
    const int NB = md.nbonds;
    const f2 one2 = f2_pack(1.f, 1.f);
    // shared-memory address of the lane's first float4 in table row 0
    const uint32_t a_tps = (uint32_t)__cvta_generic_to_shared(tps) + (uint32_t)gl * 16u;
    // ntrip >= naa is the same in every group of the warp (the shuffles below
    // take all 32 lanes)
    for (int e0 = 0; e0 < ntrip; e0 += kEpGL) {
        const int e = e0 + gl;
        int off = 0;
        sc<float> pre{0.f, 0.f, 0};
        if (e < naa) {
            const uint16_t code = aa[e];
            const int b = code & 0x7fff;
            const uint16_t bp = bps[b];
            const int bb = bp & 0x7fff;
            const bool pos = ((code >> 15) != 0) != ((bp >> 15) != 0);
            const int o = (pos != (sg != 0)) ? 0 : 1;
            off = (r * 2 + o) * BS + bb * MH;
            pre = eps[(r * 2 + o) * NB + bb];   // (J_b / 2) e^{+-C}
        }
        float rx[kEpGL], ry[kEpGL];
        int re[kEpGL];
        // the group's entries kEpQI at a time side by side (independent running products)
        uint32_t ta[kEpGL];
#pragma unroll
        for (int q = 0; q < kEpGL; ++q) ta[q] = a_tps + (uint32_t)__shfl_sync(0xffffffffu, off, gbase + q) * 16u;
#pragma unroll
        for (int q0 = 0; q0 < kEpGL; q0 += kEpQI) {
            f2 Rx[kEpQI], Ry[kEpQI];
#pragma unroll
            for (int j = 0; j < NP; ++j) {
#pragma unroll
                for (int qi = 0; qi < kEpQI; ++qi) {
                    f2 ux, uy;
                    lds128(ta[q0 + qi] + 64u * j, ux, uy);
                    f2 fx, fy;
                    if constexpr (QF) {
                        fx = add2(ux, ca[j]);
                        fy = add2(uy, cb[j]);
                    } else {
                        const f2 tx = sub2(ux, one2);
                        fx = fma2(cc[j], uy, fma2(ca[j], tx, one2));
                        fy = fma2(ca[j], uy, mul2(cb[j], tx));
                    }
                    if (j == 0) {
                        Rx[qi] = fx; Ry[qi] = fy;
                    } else {
                        const f2 nx = sub2(mul2(Rx[qi], fx), mul2(Ry[qi], fy));
                        Ry[qi] = fma2(Rx[qi], fy, mul2(Ry[qi], fx));
                        Rx[qi] = nx;
                    }
                }
            }
#pragma unroll
            for (int qi = 0; qi < kEpQI; ++qi) {
                float x = f2_lo(Rx[qi]) * f2_hi(Rx[qi]) - f2_lo(Ry[qi]) * f2_hi(Ry[qi]);
                float y = f2_lo(Rx[qi]) * f2_hi(Ry[qi]) + f2_lo(Ry[qi]) * f2_hi(Rx[qi]);
                re[q0 + qi] = nrm(x, y);
                rx[q0 + qi] = x;
                ry[q0 + qi] = y;
            }
        }
        // butterfly product-reduce-scatter over the group's 4 lanes
#pragma unroll
        for (int lev = 0; lev < 2; ++lev) {
            const int o = 2 >> lev, cnt = 2 >> lev;
            const bool upper = (gl & o) != 0;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (q < cnt) {
                    const float sx = upper ? rx[q] : rx[q + cnt];
                    const float sy = upper ? ry[q] : ry[q + cnt];
                    const int se = upper ? re[q] : re[q + cnt];
                    const float kx = upper ? rx[q + cnt] : rx[q];
                    const float ky = upper ? ry[q + cnt] : ry[q];
                    const int ke = upper ? re[q + cnt] : re[q];
                    const float gx = __shfl_xor_sync(0xffffffffu, sx, o);
                    const float gy = __shfl_xor_sync(0xffffffffu, sy, o);
                    const int ge = __shfl_xor_sync(0xffffffffu, se, o);
                    rx[q] = kx * gx - ky * gy;
                    ry[q] = kx * gy + ky * gx;
                    re[q] = ke + ge;
                }
            }
        }
        if (e < naa) {
            const float vx = rx[0] * pre.x - ry[0] * pre.y, vy = rx[0] * pre.y + ry[0] * pre.x;
            const int d = re[0] + pre.e + eref;
            if (d > -100 && d < 100) {
                const float f = __uint_as_float((uint32_t)(d + 127) << 23);
                accx = fmaf(f, vx, accx);
                accy = fmaf(f, vy, accy);
            } else {
                const double f = pow2i<double>(d);
                Ox += f * (double)vx;
                Oy += f * (double)vy;
            }
        }
    }
}

template <int NP>
__global__ void __launch_bounds__(kEfMaxThreads, 1)
    k_eloc_pair(DevModel<float> md, EfArgs ea, const uint64_t *__restrict__ cfg, int64_t n, double *__restrict__ h1_out)
{
    constexpr int NH = (NP + 1) / 2;   // unit pairs of one parity per lane
    extern __shared__ __align__(16) unsigned char smem[];
    const int NB = md.nbonds, K = md.K, MH = ea.MH, BS = ea.BS, N = md.N, M = md.M;
    const int nwarps = blockDim.x >> 5, nrs = nwarps * 4;   // row slots: 4 per warp
    float4 *tps = reinterpret_cast<float4 *>(smem);                                        // [K][2] x BS
    float4 *wsv = tps + (size_t)K * 2 * BS;                                                // [K][N][M] W (if staged)
    sc<float> *eps = reinterpret_cast<sc<float> *>(wsv + (ea.w_smem ? ((size_t)K * N * M + 1) / 2 : 0));   // [K][2][NB]
    cx<float> *csum = reinterpret_cast<cx<float> *>(eps + (size_t)K * 2 * NB);          // [K][M] sum_k W_mk
    uint16_t *gbp = reinterpret_cast<uint16_t *>(csum + (size_t)K * M);                  // [nrs][NB]
    uint8_t *gperm = reinterpret_cast<uint8_t *>(gbp + (size_t)nrs * NB);                 // [nrs][N]
    __shared__ float s_sm[kMaxN];
    __shared__ int8_t s8[kMaxN];
    __shared__ uint16_t aa[4 * kMaxN];
    __shared__ uint8_t ups[kMaxN];   // the up sites of the sample
    __shared__ int n_aa, n_up;
    __shared__ float diag_sh;
    __shared__ sc<double> gsum[2][2 * 4 * (kEfMaxThreads / 32)];   // per (row slot, sign)

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane >> 2, gl = lane & 3, gbase = grp * 4;
    const int pi = grp >> 1, sg = grp & 1, l8 = lane & 7;
    const int rslot = warp * 4 + pi, gslot = rslot * 2 + sg;
    uint8_t *pgs = gperm + (size_t)rslot * N;
    uint16_t *bps = gbp + (size_t)rslot * NB;
    const cx<float> *Wsrc = ea.w_smem ? reinterpret_cast<const cx<float> *>(wsv) : md.Wt;
    const float sign = sg ? -1.f : 1.f;

    {
        const int4 *src = reinterpret_cast<const int4 *>(ea.tp);
        int4 *dst = reinterpret_cast<int4 *>(tps);
        for (int q = threadIdx.x; q < K * 2 * BS; q += blockDim.x) dst[q] = src[q];
        for (int q = threadIdx.x; q < K * 2 * NB; q += blockDim.x) eps[q] = ea.ep[q];
        if (ea.w_smem) {
            cx<float> *wd = reinterpret_cast<cx<float> *>(wsv);
            for (int q = threadIdx.x; q < K * N * M; q += blockDim.x) wd[q] = md.Wt[q];
        }
        for (int q = threadIdx.x; q < K * M; q += blockDim.x) {
            const int rr = q / M, m = q - rr * M;
            cx<float> a{0.f, 0.f};
            for (int k = 0; k < N; ++k) {
                const cx<float> w = md.Wt[((size_t)rr * N + k) * M + m];
                a.x += w.x;
                a.y += w.y;
            }
            csum[q] = a;
        }
    }

    for (int64_t smp = blockIdx.x; smp < n; smp += gridDim.x) {
        const uint64_t *w = cfg + smp * md.nwords;
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            const int sv = spin_of(w, i);
            s_sm[i] = (float)sv;
            s8[i] = (int8_t)sv;
        }
        for (int q = threadIdx.x; q < 2 * 2 * nrs; q += blockDim.x) gsum[q / (2 * nrs)][q % (2 * nrs)] = sc<double>{0.0, 0.0, 0};
        __syncthreads();
        if (warp == 0) {
            float d = 0.f;
            int base = 0;
            for (int b0 = 0; b0 < NB; b0 += 32) {
                const int b = b0 + lane;
                bool isaa = false;
                int si = 0;
                if (b < NB) {
                    si = s8[md.bond_i[b]];
                    const int sj = s8[md.bond_j[b]];
                    d += 0.25f * bondJ(md, b) * (float)(si * sj);
                    isaa = si != sj;
                }
                const unsigned bm = __ballot_sync(0xffffffffu, isaa);
                if (isaa) aa[base + __popc(bm & ((1u << lane) - 1u))] = (uint16_t)(b | (si > 0 ? 0x8000 : 0));
                base += __popc(bm);
            }
            for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
            if (lane == 0) { n_aa = base; diag_sh = d; }
        } else if (warp == 1) {
            int base = 0;
            for (int i0 = 0; i0 < N; i0 += 32) {
                const int i = i0 + lane;
                const bool up = i < N && s8[i] > 0;
                const unsigned bm = __ballot_sync(0xffffffffu, up);
                if (up) ups[base + __popc(bm & ((1u << lane) - 1u))] = (uint8_t)i;
                base += __popc(bm);
            }
            if (lane == 0) n_up = base;
        }
        __syncthreads();
        const int naa = n_aa, nup = n_up;

        // waves of nrs rows; a last wave of at most nrs / 2 (nrs / 4) rows
        // gives each row 2 (4) slots, each with its share of the entries
        for (int rbase = 0; rbase < K * md.G;) {
            const int left = K * md.G - rbase;
            const int split = 4 * left <= nrs ? 4 : 2 * left <= nrs ? 2 : 1;
            const int part = rslot % split;
            const bool active = rbase + rslot / split < K * md.G;
            const int row = active ? rbase + rslot / split : 0;
            const int e_lo = part * naa / split, e_n = (part + 1) * naa / split - e_lo;
            const int e_max = (naa + split - 1) / split;   // the largest share: the same trip count in every group
            rbase += nrs / split;
            const int r = K == 1 ? 0 : row / md.G, g = row - r * md.G;
            __syncwarp();
            for (int i = l8; i < N; i += 8) pgs[i] = md.perm[(size_t)g * N + i];
            for (int b = l8; b < NB; b += 8) bps[b] = md.bperm[(size_t)g * NB + b];
            __syncwarp();
            // ---- theta': this lane's parity of unit pairs, then the partner's;
            //      with s_i = +-1, theta'_m = 2 sum_{s_i = +1} W_m,g(i) - sum_k W_mk ----
            float ox[2 * NH], oy[2 * NH];
#pragma unroll
            for (int u = 0; u < 2 * NH; ++u) { ox[u] = 0.f; oy[u] = 0.f; }
            const cx<float> *Wr = Wsrc + (size_t)r * N * M;
            for (int t = 0; t < nup; ++t) {
                const cx<float> *wk = Wr + (size_t)pgs[ups[t]] * M;
#pragma unroll
                for (int h = 0; h < NH; ++h) {
                    const int jj = 2 * h + sg;
                    const int m = 2 * (gl + kEpGL * jj);
                    if ((M & 1) == 0 && m + 1 < M) {
                        const float4 a = *reinterpret_cast<const float4 *>(wk + m);
                        ox[2 * h] += a.x; oy[2 * h] += a.y;
                        ox[2 * h + 1] += a.z; oy[2 * h + 1] += a.w;
                    } else {
                        if (m < M) { const cx<float> a = wk[m]; ox[2 * h] += a.x; oy[2 * h] += a.y; }
                        if (m + 1 < M) { const cx<float> a = wk[m + 1]; ox[2 * h + 1] += a.x; oy[2 * h + 1] += a.y; }
                    }
                }
            }
#pragma unroll
            for (int h = 0; h < NH; ++h) {
                const int m = 2 * (gl + kEpGL * (2 * h + sg));
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    if (m + u < M) {
                        const cx<float> c = csum[(size_t)r * M + m + u];
                        ox[2 * h + u] = fmaf(2.f, ox[2 * h + u], -c.x);
                        oy[2 * h + u] = fmaf(2.f, oy[2 * h + u], -c.y);
                    }
                }
            }
            float tx[2 * NP], ty[2 * NP];
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                const int h = j >> 1;
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const float vx = __shfl_xor_sync(0xffffffffu, ox[2 * h + u], 4);
                    const float vy = __shfl_xor_sync(0xffffffffu, oy[2 * h + u], 4);
                    const bool own = (j & 1) == sg;
                    tx[2 * j + u] = own ? ox[2 * h + u] : vx;
                    ty[2 * j + u] = own ? oy[2 * h + u] : vy;
                }
            }
            cx<float> at{0.f, 0.f};
            if (md.use_bias) {
                const cx<float> *ar = md.avec + (size_t)r * N;
                for (int i = l8; i < N; i += 8) { const cx<float> a = ar[pgs[i]]; at.x += s_sm[i] * a.x; at.y += s_sm[i] * a.y; }
#pragma unroll
                for (int o = 4; o > 0; o >>= 1) {
                    at.x += __shfl_xor_sync(0xffffffffu, at.x, o);
                    at.y += __shfl_xor_sync(0xffffffffu, at.y, o);
                }
            }
            // ---- this group's sign.  With q_m = e^{-2 theta_m} = (1 - p_m)/p_m the
            //      unit factor is p_m (q_m + U_m), and 2 cosh(theta_m) p_m = e^{theta_m}:
            //      the row's term times prod_m p_m is lead e^{sum_m theta_m}, and its
            //      term is that times prod_m (1 + q_m) ----
            f2 ca[NP], cb[NP];
            float stx = 0.f, sty = 0.f;   // sum of theta over the lane's units
            f2 Qx = f2_pack(1.f, 1.f), Qy = 0;
            int qlo = 0, qhi = 0;         // exponents of the even and odd units' products of 1 + q
            bool small = ea.plain != 0;   // some |p| < 2^-12 (|1 + q| > 2^12): the plain factors
            const cx<float> *br = md.bvec + (size_t)r * M;
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                float qxv[2], qyv[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int m = 2 * (gl + kEpGL * j) + h;
                    qxv[h] = 0.f; qyv[h] = 0.f;   // units past M: q = 0 (their U is 1)
                    if (m < M) {
                        cx<float> th{sign * tx[2 * j + h], sign * ty[2 * j + h]};
                        if (md.use_bias) { const cx<float> b = br[m]; th.x += b.x; th.y += b.y; }
                        stx += th.x;
                        sty += th.y;
                        const float e = exp2f(-2.8853900817779268f * th.x);   // e^{-2 Re theta}
                        float sn, cs;
                        sincosf(2.f * th.y, &sn, &cs);
                        qxv[h] = e * cs;
                        qyv[h] = -e * sn;
                        const float ax = 1.f + qxv[h];
                        small = small || !(ax * ax + qyv[h] * qyv[h] <= 0x1p24f);
                    }
                }
                ca[j] = f2_pack(qxv[0], qxv[1]);
                cb[j] = f2_pack(qyv[0], qyv[1]);
                const f2 fx = add2(ca[j], f2_pack(1.f, 1.f));
                const f2 nx = sub2(mul2(Qx, fx), mul2(Qy, cb[j]));
                Qy = fma2(Qx, cb[j], mul2(Qy, fx));
                Qx = nx;
                if ((j % 3) == 2 || j == NP - 1) {
                    float xl = f2_lo(Qx), yl = f2_lo(Qy), xh = f2_hi(Qx), yh = f2_hi(Qy);
                    qlo += nrm(xl, yl);
                    qhi += nrm(xh, yh);
                    Qx = f2_pack(xl, xh);
                    Qy = f2_pack(yl, yh);
                }
            }
            const cx<float> lc = md.logc[r];
            float chg = md.chi[g];
            if (sg && md.chiP < 0) chg = -chg;

            float accx = 0.f, accy = 0.f;
            double Ox = 0.0, Oy = 0.0;
            sc<float> mult;
            if (!__any_sync(0xffffffffu, small)) {
                // sum of theta and prod (1 + q) over the group's 4 lanes
#pragma unroll
                for (int o = 1; o < kEpGL; o <<= 1) {
                    stx += __shfl_xor_sync(0xffffffffu, stx, o);
                    sty += __shfl_xor_sync(0xffffffffu, sty, o);
                }
                float u = f2_lo(Qx) * f2_hi(Qx) - f2_lo(Qy) * f2_hi(Qy);
                float v = f2_lo(Qx) * f2_hi(Qy) + f2_lo(Qy) * f2_hi(Qx);
                const int qe = qlo + qhi + nrm(u, v);
                const sc<float> Q = group_prod<kEpGL>(sc<float>{u, v, qe});
                // lead e^{sum theta} = term x prod p, kept as mantissa x 2^(e + Q.e) and
                // the entries scaled by 2^-Q.e (near 2^0, as prod (q + U) ~ prod (1 + q))
                sc<float> lead = sc_exp(cx<float>{lc.x + sign * at.x + stx, lc.y + sign * at.y + sty});
                lead.x *= chg; lead.y *= chg;
                lead = sc_norm(lead);
                const sc<float> wt = sc_mul(lead, Q);   // the row term
                if (gl == 0 && active && part == 0)
                    gsum[1][gslot] = sc_add(gsum[1][gslot], sc<double>{(double)wt.x, (double)wt.y, wt.e});
                ep_entries<NP, true>(md, tps, eps, aa + e_lo, bps, e_n, e_max, r, sg, MH, BS, ca, cb, cb, -Q.e, gl,
                                     gbase, accx, accy, Ox, Oy);
                mult = sc<float>{lead.x, lead.y, lead.e + Q.e};
            } else {
                // the plain factors 1 + p (U - 1) with p and prod 2 cosh(theta) from cosh2
                f2 cc[NP];
                sc<float> prod{1.f, 0.f, 0};
#pragma unroll
                for (int j = 0; j < NP; ++j) {
                    float pxv[2], pyv[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int m = 2 * (gl + kEpGL * j) + h;
                        pxv[h] = 1.f; pyv[h] = 0.f;   // units past M: p = 1 (their U is 1)
                        if (m < M) {
                            cx<float> th{sign * tx[2 * j + h], sign * ty[2 * j + h]};
                            if (md.use_bias) { const cx<float> b = br[m]; th.x += b.x; th.y += b.y; }
                            cx<float> mant, pv;
                            int k;
                            cosh2(th, mant, k, pv);
                            pxv[h] = pv.x; pyv[h] = pv.y;
                            const cx<float> z = cmul(mk(prod.x, prod.y), mant);
                            prod = sc_norm(sc<float>{z.x, z.y, prod.e + k});
                        }
                    }
                    ca[j] = f2_pack(pxv[0], pxv[1]);
                    cb[j] = f2_pack(pyv[0], pyv[1]);
                    cc[j] = f2_pack(-pyv[0], -pyv[1]);
                }
                prod = group_prod<kEpGL>(prod);
                sc<float> lead = sc_exp(cx<float>{lc.x + sign * at.x, lc.y + sign * at.y});
                lead.x *= chg; lead.y *= chg;
                const sc<float> wt = sc_mul(prod, sc_norm(lead));
                if (gl == 0 && active && part == 0)
                    gsum[1][gslot] = sc_add(gsum[1][gslot], sc<double>{(double)wt.x, (double)wt.y, wt.e});
                ep_entries<NP, false>(md, tps, eps, aa + e_lo, bps, e_n, e_max, r, sg, MH, BS, ca, cb, cc, 0, gl,
                                      gbase, accx, accy, Ox, Oy);
                mult = wt;
            }
            double ax = (double)accx + Ox, ay = (double)accy + Oy;
#pragma unroll
            for (int o = kEpGL / 2; o > 0; o >>= 1) {
                ax += __shfl_xor_sync(0xffffffffu, ax, o);
                ay += __shfl_xor_sync(0xffffffffu, ay, o);
            }
            if (gl == 0 && active) gsum[0][gslot] = sc_add(gsum[0][gslot], sd_mul(mult, ax, ay));
        }
        __syncthreads();
        if (warp == 0) {
            sc<double> t1{0.0, 0.0, 0}, t0{0.0, 0.0, 0};
            for (int q = lane; q < 2 * nrs; q += 32) { t1 = sc_add(t1, gsum[0][q]); t0 = sc_add(t0, gsum[1][q]); }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const sc<double> u1{__shfl_xor_sync(0xffffffffu, t1.x, o), __shfl_xor_sync(0xffffffffu, t1.y, o),
                                    __shfl_xor_sync(0xffffffffu, t1.e, o)};
                const sc<double> u0{__shfl_xor_sync(0xffffffffu, t0.x, o), __shfl_xor_sync(0xffffffffu, t0.y, o),
                                    __shfl_xor_sync(0xffffffffu, t0.e, o)};
                t1 = sc_add(t1, u1);
                t0 = sc_add(t0, u0);
            }
            if (lane == 0) {
                const double den = t0.x * t0.x + t0.y * t0.y;
                const double f = ldexp(1.0, t1.e - t0.e);
                const double rx = (t1.x * t0.x + t1.y * t0.y) / den * f, ry = (t1.y * t0.x - t1.x * t0.y) / den * f;
                const double h1x = (double)diag_sh + rx;
                if (sc_zero(t0) || !isfinite(h1x) || !isfinite(ry)) flag_range(md.status);
                h1_out[2 * smp] = h1x;
                h1_out[2 * smp + 1] = ry;
            }
        }
        __syncthreads();
    }
}

// Paired tables from the connection tables of the model: tp[(r 2 + o) BS + b MH
// + k] = (Ux_2k, Ux_2k+1, Uy_2k, Uy_2k+1), U = 1 + T, for unit pairs k < MH
// (U = 1 past M), and ep = (J_b / 2) e^{(1 - 2 o) C_b} as scaled numbers.
__global__ void k_tables_paired(DevModel<float> md, int MH, int BS, float4 *__restrict__ tp, sc<float> *__restrict__ ep)
{
    const int NB = md.nbonds;
    const int64_t tot = (int64_t)md.K * 2 * NB * MH;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < tot; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t rowi = q / MH;                 // (r 2 + o) NB + b
        const int k = (int)(q - rowi * MH);
        const int64_t blk = rowi / NB, b = rowi - blk * NB;
        const cx<float> *src = md.Tb + rowi * md.Mp;
        const int m0 = 2 * k, m1 = 2 * k + 1;
        const cx<float> a = m0 < md.M ? src[m0] : cx<float>{0.f, 0.f};
        const cx<float> c = m1 < md.M ? src[m1] : cx<float>{0.f, 0.f};
        tp[blk * BS + b * MH + k] = make_float4(1.f + a.x, 1.f + c.x, a.y, c.y);
    }
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < (int64_t)md.K * 2 * NB;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int rb = (int)(q / NB);            // r * 2 + o
        const int b = (int)(q - (int64_t)rb * NB);
        const int r = rb >> 1, o = rb & 1;
        const cx<float> c = md.Cb[(size_t)r * NB + b];
        const sc<float> v = sc_exp(o ? cx<float>{-c.x, -c.y} : c);
        const float hj = 0.5f * bondJ(md, b);   // the symmetry images of a bond have its coupling
        ep[q] = sc_norm(sc<float>{v.x * hj, v.y * hj, v.e});
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int ef_np(int M) { return (M + 2 * kEfGL - 1) / (2 * kEfGL); }   // unit pairs per lane (8 lanes)

struct EfLayout {
    bool pair;      // the sign-paired 4-lane kernel
    int NP, MH, BS;
    bool w_smem;    // W staged in shared memory (sign-paired kernel)
};

static int ef_warps(const DevModel<float> &md)
{
    // the most warps (latency hiding) whose row slots idle at most 1/8 of the
    // time, else the count in 8..16 that idles least (4 row slots a warp)
    const int rows = md.K * md.G;
    int best = 16, waste = 1 << 30;
    for (int w = 16; w >= 8; --w) {
        const int slots = 4 * w;
        const int pad = (rows + slots - 1) / slots * slots;
        if (8 * (pad - rows) <= pad) return w;
        if (pad - rows < waste) { waste = pad - rows; best = w; }
    }
    return best;
}

// dynamic shared memory: tables, W (if staged), prefactors, the row slots'
// images of the bonds and sites
static size_t ef_smem(const DevModel<float> &md, const EfLayout &L, int warps)
{
    const size_t tab = (size_t)md.K * 2 * L.BS * sizeof(float4);
    const size_t wst = L.w_smem ? ((size_t)md.K * md.N * md.M + 1) / 2 * sizeof(float4) : 0;
    const size_t cs = L.pair ? (size_t)md.K * md.M * sizeof(cx<float>) : 0;   // column sums of W
    return tab + wst + (size_t)md.K * 2 * md.nbonds * sizeof(sc<float>) + cs +
           (size_t)warps * 4 * (md.nbonds * sizeof(uint16_t) + md.N);
}

constexpr size_t kEfSmemLimit = 212 * 1024;   // dynamic part; the static part stays below 12 KB

static EfLayout ef_layout(const DevModel<float> &md)
{
    EfLayout L{};
    const int NB = md.nbonds;
    const int npp = (md.M + 2 * kEpGL - 1) / (2 * kEpGL);
    if (md.nsign == 2 && npp >= 1 && npp <= 10) {
        L.pair = true;
        L.NP = npp;
        L.MH = kEpGL * npp;
        const int64_t B = (int64_t)NB * L.MH;
        const int res = (int)((4 * B) % 32);                 // 32-bit words mod the banks
        L.BS = (int)(B + (((16 - res) % 32 + 32) % 32) / 4);  // blocks 16 words apart mod 32
        L.w_smem = true;
        if (ef_smem(md, L, ef_warps(md)) <= kEfSmemLimit) return L;
        L.w_smem = false;
        if (ef_smem(md, L, ef_warps(md)) <= kEfSmemLimit) return L;
    }
    L = EfLayout{};
    L.NP = ef_np(md.M);
    L.MH = kEfGL * L.NP;
    L.BS = NB * L.MH;
    return L;
}

bool eloc_fast_supported(const DevModel<float> &md)
{
    const EfLayout L = ef_layout(md);
    if (L.pair) return true;
    if (L.NP < 1 || L.NP > 8) return false;
    return ef_smem(md, L, ef_warps(md)) <= kEfSmemLimit;
}

size_t eloc_fast_table_bytes(const DevModel<float> &md)
{
    const EfLayout L = ef_layout(md);
    return (size_t)md.K * 2 * L.BS * sizeof(float4) + (size_t)md.K * 2 * md.nbonds * sizeof(sc<float>) + 256;
}

cudaError_t launch_tables_paired(const DevModel<float> &md, void *tables, cudaStream_t st)
{
    const EfLayout L = ef_layout(md);
    float4 *tp = reinterpret_cast<float4 *>(tables);
    sc<float> *ep = reinterpret_cast<sc<float> *>(tp + (size_t)md.K * 2 * L.BS);
    if (L.BS != md.nbonds * L.MH) cudaMemsetAsync(tp, 0, (size_t)md.K * 2 * L.BS * sizeof(float4), st);
    k_tables_paired<<<256, 256, 0, st>>>(md, L.MH, L.BS, tp, ep);
    return cudaGetLastError();
}

cudaError_t launch_eloc_fast(const DevModel<float> &md, const void *tables, const uint64_t *cfg, int64_t n,
                             double *h1, int nsm, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const EfLayout L = ef_layout(md);
    EfArgs ea;
    ea.MH = L.MH;
    ea.BS = L.BS;
    ea.w_smem = L.w_smem;
    ea.tp = reinterpret_cast<const float4 *>(tables);
    ea.ep = reinterpret_cast<const sc<float> *>(ea.tp + (size_t)md.K * 2 * L.BS);
    ea.warps = ef_warps(md);
    // Test hooks (unset in normal use): NNQS_TEST_ELOC_PLAIN=1 takes the plain
    // factors 1 + p (U - 1) in every row.
    const char *hook = getenv("NNQS_TEST_ELOC_PLAIN");
    ea.plain = hook && hook[0] == '1';
    const size_t smem = ef_smem(md, L, ea.warps);
    const int grid = (int)(n < nsm ? n : nsm);
    void (*kern)(DevModel<float>, EfArgs, const uint64_t *, int64_t, double *) = nullptr;
    if (L.pair) {
        switch (L.NP) {
        case 1: kern = k_eloc_pair<1>; break;
        case 2: kern = k_eloc_pair<2>; break;
        case 3: kern = k_eloc_pair<3>; break;
        case 4: kern = k_eloc_pair<4>; break;
        case 5: kern = k_eloc_pair<5>; break;
        case 6: kern = k_eloc_pair<6>; break;
        case 7: kern = k_eloc_pair<7>; break;
        case 8: kern = k_eloc_pair<8>; break;
        case 9: kern = k_eloc_pair<9>; break;
        default: kern = k_eloc_pair<10>; break;
        }
    } else {
        switch (L.NP) {
        case 1: kern = k_eloc_fast<1>; break;
        case 2: kern = k_eloc_fast<2>; break;
        case 3: kern = k_eloc_fast<3>; break;
        case 4: kern = k_eloc_fast<4>; break;
        case 5: kern = k_eloc_fast<5>; break;
        case 6: kern = k_eloc_fast<6>; break;
        case 7: kern = k_eloc_fast<7>; break;
        default: kern = k_eloc_fast<8>; break;
        }
    }
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, 32 * ea.warps, smem, st>>>(md, ea, cfg, n, h1);
    return cudaGetLastError();
}

}  // namespace nnqs
