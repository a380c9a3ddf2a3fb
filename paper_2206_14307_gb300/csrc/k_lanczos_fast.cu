// k_lanczos_fast.cu -- h1 = (H psi)/psi and h2 = (H^2 psi)/psi (Sec. 3.3, the
// per-sample quantities behind the moments of Eqs. 13-18) in FP32 with the
// per-site factor tables in shared memory.
//
// Flipping site k in a row (r, g, sign) of the projected sum (Eqs. 4-6)
// changes theta_m by Delta_m = -2 sign s_k W_{m, g(k)}, i.e. multiplies
// e^{2 theta_m} by u_m = e^{-+4 W_{m, g(k)}} (sign * s_k = +1 picks e^{-4W}).
// With p_m = e^{theta_m}/(2cosh theta_m), a flip set D gives the row's ratio
//   e^{C_D} prod_m (1 + p_m (U_m - 1)),   U = prod_{k in D} u_k,
// C_D the sum of the flipped sites' prefactor exponents
// sign s_k (2 sum_m W_{m g(k)} - 2 a_{g(k)}).
// The second-level flip sets of h2 are exchanges of a bond b2 in the
// configuration s^{b1} that the exchange of b1 reached, so per row
//   psi(s^{b1 b2})/psi(s) = R1 e^{C_{b2}} prod_m (1 + p'_m (U2_m - 1)),
// R1 = psi(s^{b1})/psi(s) and p'_m = p_m U1_m / (1 + p_m (U1_m - 1)) the p of
// s^{b1}.  Per element: two 128-bit shared-memory reads (two units each) and
// 14 packed FP32x2 operations per unit pair.
//
// Layout: one CTA per SM with the model's site tables copied into its shared
// memory once; one sample per CTA at a time.  Per sample the CTA lists, for
// every anti-aligned bond b1, the bonds b2 anti-aligned in s^{b1} (b2 = b1
// left out: it returns to s, the constant sum_b (J_b/2)^2; a b2 disjoint from
// b1 only for b2 > b1, weighted twice for the two orders) as 32-bit codes.  A
// group of GL lanes owns a row; lane l owns the unit pairs k = l + GL j.  Per
// b1 the group forms p' and R1, then takes b1's list 8 entries at a time; a
// butterfly product-reduce-scatter over the group leaves each entry's product
// with one lane.  Sums: FP32 within one b1 list (relative to R1), FP64 across
// the b1 of a row, scaled FP64 across rows.
#include <algorithm>
#include <cstdlib>

#include "common.cuh"
#include "f2.cuh"
#include "kernels.h"

namespace nnqs {

namespace {

constexpr int kLfNE = 8;         // entries per batch
constexpr int kLfThreads = 384;  // 12 warps, up to 168 registers per thread

struct LfArgs {
    const float4 *up;   // [K][2][N][MH] paired site factors (ux_2k, ux_2k+1, uy_2k, uy_2k+1)
    int MH;             // unit pairs per table row (GL NP)
    int cap;            // entries the shared list holds
    int plain;          // 1: every b1 takes the plain form 1 + p'(U - 1) (test hook)
};

// Entry code: c | d << 8 | (s^{b1}_c > 0) << 16 | (b2 is a J2 bond) << 17 |
// (b2 shares a site with b1) << 18, where b2 = (c, d).
__device__ __forceinline__ bool second_level(const DevModel<float> &md, int b1, int i1, int j1, int b2,
                                             const int8_t *s8, uint32_t &code)
{
    if (b2 == b1) return false;
    const int c = md.bond_i[b2], d = md.bond_j[b2];
    const bool shared = c == i1 || c == j1 || d == i1 || d == j1;
    if (!shared && b2 < b1) return false;
    // spins in s^{b1}: the sites of b1 exchanged
    const int sc_ = c == i1 ? s8[j1] : c == j1 ? s8[i1] : s8[c];
    const int sd_ = d == i1 ? s8[j1] : d == j1 ? s8[i1] : s8[d];
    if (sc_ == sd_) return false;
    code = (uint32_t)c | ((uint32_t)d << 8) | ((uint32_t)(sc_ > 0) << 16) | ((uint32_t)(md.bond_t[b2] == 2) << 17) |
           ((uint32_t)shared << 18);
    return true;
}

// One b1 list of one row: for each entry (b2 = (c, d) exchanged in s^{b1})
// the product over the lane's units of the entry's factors, reduced over the
// group by a butterfly, times its prefactor and weight c2, summed into the
// owner lanes' (accx, accy) (FP32, scaled by 2^eref) or, outside the FP32
// window, (Ox, Oy).  QF: factors q + U with q = (1 - p')/p' (ca, cb = q; the
// product of p' is taken out by the caller, eref = its exponent); otherwise
// 1 + p'(U - 1) (ca, cb, cc = Re p', Im p', -Im p').
template <int GL, int NP, bool QF>
__device__ __forceinline__ void b1_list(const float4 *ups, const sc<float> *eps, const uint32_t *le, int cnt,
                                        const uint8_t *pgs, int N, int MH, int rb, int sg, float J1b, float J1,
                                        float J2, const f2 (&ca)[NP], const f2 (&cb)[NP], const f2 (&cc)[NP],
                                        int eref, int gl, int gbase, int eq, bool owner, float &accx, float &accy,
                                        double &Ox, double &Oy)
{
    constexpr int kRep = GL / kLfNE;
    const f2 one2 = f2_pack(1.f, 1.f), mone2 = f2_pack(-1.f, -1.f);
    for (int e0 = 0; e0 < cnt; e0 += kLfNE) {
        const int e = e0 + eq;
        int offc = 0, offd = 0;
        sc<float> pre{0.f, 0.f, 0};
        if (e < cnt) {
            const uint32_t code = le[e];
            const int c = code & 0xff, d = (code >> 8) & 0xff;
            const int oc = ((((code >> 16) & 1u) != 0) == (sg == 0)) ? 0 : 1;   // sign s_c = +1 -> e^{-4W}
            const int kc = pgs[c], kd = pgs[d];
            offc = ((rb + oc) * N + kc) * MH;
            offd = ((rb + 1 - oc) * N + kd) * MH;
            const float c2 = (((code >> 18) & 1u) ? 0.25f : 0.5f) * J1b * (((code >> 17) & 1u) ? J2 : J1);
            pre = sc_mul(eps[(rb + oc) * N + kc], eps[(rb + 1 - oc) * N + kd]);
            pre.x *= c2;
            pre.y *= c2;
        }
        float rx[kLfNE], ry[kLfNE];
        int re[kLfNE];
#pragma unroll
        for (int q = 0; q < kLfNE; ++q) {
            const int src = gbase + q * kRep;
            const float4 *tc = ups + __shfl_sync(0xffffffffu, offc, src) + gl;
            const float4 *td = ups + __shfl_sync(0xffffffffu, offd, src) + gl;
            f2 Rx = one2, Ry = 0;
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                f2 ucx, ucy, udx, udy;
                lds128(tc + GL * j, ucx, ucy);
                lds128(td + GL * j, udx, udy);
                f2 fx, fy;
                if constexpr (QF) {
                    fx = sub2(fma2(ucx, udx, ca[j]), mul2(ucy, udy));   // q + U
                    fy = fma2(ucx, udy, fma2(ucy, udx, cb[j]));
                } else {
                    const f2 Tx = sub2(fma2(ucx, udx, mone2), mul2(ucy, udy));   // U - 1
                    const f2 Ty = fma2(ucx, udy, mul2(ucy, udx));
                    fx = fma2(cc[j], Ty, fma2(ca[j], Tx, one2));
                    fy = fma2(ca[j], Ty, mul2(cb[j], Tx));
                }
                if (j == 0) {
                    Rx = fx; Ry = fy;
                } else {
                    const f2 nx = sub2(mul2(Rx, fx), mul2(Ry, fy));
                    Ry = fma2(Rx, fy, mul2(Ry, fx));
                    Rx = nx;
                }
            }
            // even units x odd units, then mantissa / exponent
            float x = f2_lo(Rx) * f2_hi(Rx) - f2_lo(Ry) * f2_hi(Ry);
            float y = f2_lo(Rx) * f2_hi(Ry) + f2_lo(Ry) * f2_hi(Rx);
            re[q] = nrm(x, y);
            rx[q] = x;
            ry[q] = y;
        }
        // butterfly product-reduce-scatter over the group's GL lanes
#pragma unroll
        for (int lev = 0; (GL >> (lev + 1)) >= 1; ++lev) {
            const int o = GL >> (lev + 1);
            const int half = kLfNE >> (lev + 1);
            const bool upper = (gl & o) != 0;
            if (half >= 1) {
#pragma unroll
                for (int q = 0; q < kLfNE / 2; ++q) {
                    if (q < half) {
                        const float sx = upper ? rx[q] : rx[q + half];
                        const float sy = upper ? ry[q] : ry[q + half];
                        const int se = upper ? re[q] : re[q + half];
                        const float kx = upper ? rx[q + half] : rx[q];
                        const float ky = upper ? ry[q + half] : ry[q];
                        const int ke = upper ? re[q + half] : re[q];
                        const float gx = __shfl_xor_sync(0xffffffffu, sx, o);
                        const float gy = __shfl_xor_sync(0xffffffffu, sy, o);
                        const int ge = __shfl_xor_sync(0xffffffffu, se, o);
                        rx[q] = kx * gx - ky * gy;
                        ry[q] = kx * gy + ky * gx;
                        re[q] = ke + ge;
                    }
                }
            } else {
                const float gx = __shfl_xor_sync(0xffffffffu, rx[0], o);
                const float gy = __shfl_xor_sync(0xffffffffu, ry[0], o);
                const int ge = __shfl_xor_sync(0xffffffffu, re[0], o);
                const float nx = rx[0] * gx - ry[0] * gy;
                ry[0] = rx[0] * gy + ry[0] * gx;
                rx[0] = nx;
                re[0] += ge;
            }
        }
        if (owner && e < cnt) {
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

template <int GL, int NP>
__global__ void __launch_bounds__(kLfThreads, 1)
    k_lanczos_fast(DevModel<float> md, LfArgs la, const uint64_t *__restrict__ cfg, int64_t n,
                   double *__restrict__ h1_out, double *__restrict__ h2_out)
{
    constexpr int NG = 32 / GL;
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = md.N, K = md.K, M = md.M, G = md.G, NB = md.nbonds, MH = la.MH;
    float4 *ups = reinterpret_cast<float4 *>(smem);                                  // [K][2][N][MH]
    sc<float> *eps = reinterpret_cast<sc<float> *>(ups + (size_t)K * 2 * N * MH);   // [K][2][N]
    uint32_t *ent = reinterpret_cast<uint32_t *>(eps + (size_t)K * 2 * N);           // [cap]
    __shared__ int8_t s8[kMaxN];
    __shared__ float s_sm[kMaxN];
    __shared__ uint16_t aa[4 * kMaxN];   // anti-aligned bond | (s_i > 0) << 15
    __shared__ int hb[4 * kMaxN + 1];    // list offsets over aa; hb[n_aa] = total
    __shared__ float hd[4 * kMaxN];      // (J_b1 / 2) x diagonal energy of s^{b1}
    __shared__ int n_aa, a_end;
    __shared__ float diag_sh, cst_sh;
    __shared__ sc<double> gsum[3][kLfThreads / 16];   // per row group: sums of wt h1-part, wt h2-part, wt
    __shared__ uint8_t gperm[kLfThreads / 16][kMaxN]; // per row group: image of each site under its row's g

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int grp = lane / GL, gl = lane % GL, gbase = grp * GL;
    const int gidx = warp * NG + grp, ngroups = nwarps * NG;
    // after the butterfly, lanes gl with equal gl / (GL / 8) hold the same
    // entry, eq = gl / (GL / 8); the first of them adds it
    constexpr int kRep = GL / kLfNE;
    const int eq = gl / kRep;
    const bool owner = (gl % kRep) == 0;
    const f2 one2 = f2_pack(1.f, 1.f), zero2 = 0, mone2 = f2_pack(-1.f, -1.f);
    uint8_t *pgs = gperm[gidx];

    {
        const int4 *src = reinterpret_cast<const int4 *>(la.up);
        int4 *dst = reinterpret_cast<int4 *>(ups);
        for (int q = threadIdx.x; q < K * 2 * N * MH; q += blockDim.x) dst[q] = src[q];
        for (int q = threadIdx.x; q < K * 2 * N; q += blockDim.x) eps[q] = md.ES[q];
    }

    for (int64_t smp = blockIdx.x; smp < n; smp += gridDim.x) {
        const uint64_t *w = cfg + smp * md.nwords;
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            const int sv = spin_of(w, i);
            s8[i] = (int8_t)sv;
            s_sm[i] = (float)sv;
        }
        for (int q = threadIdx.x; q < 3 * ngroups; q += blockDim.x) gsum[q / ngroups][q % ngroups] = sc<double>{0.0, 0.0, 0};
        __syncthreads();
        if (warp == 0) {
            float d = 0.f, c = 0.f;
            int base = 0;
            for (int b0 = 0; b0 < NB; b0 += 32) {
                const int b = b0 + lane;
                bool isaa = false;
                int si = 0;
                if (b < NB) {
                    si = s8[md.bond_i[b]];
                    const int sj = s8[md.bond_j[b]];
                    const float J = bondJ(md, b);
                    d += 0.25f * J * (float)(si * sj);
                    isaa = si != sj;
                    if (isaa) c += 0.25f * J * J;
                }
                const unsigned bm = __ballot_sync(0xffffffffu, isaa);
                if (isaa) aa[base + __popc(bm & ((1u << lane) - 1u))] = (uint16_t)(b | (si > 0 ? 0x8000 : 0));
                base += __popc(bm);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                d += __shfl_xor_sync(0xffffffffu, d, o);
                c += __shfl_xor_sync(0xffffffffu, c, o);
            }
            if (lane == 0) { n_aa = base; diag_sh = d; cst_sh = c; }
        }
        __syncthreads();
        const int naa = n_aa;
        // list sizes and the diagonal energy of every s^{b1}
        for (int a = warp; a < naa; a += nwarps) {
            const int b1 = aa[a] & 0x7fff;
            const int i1 = md.bond_i[b1], j1 = md.bond_j[b1];
            int cnt = 0;
            float dd = 0.f;
            for (int b0 = 0; b0 < NB; b0 += 32) {
                const int b2 = b0 + lane;
                bool ok = false;
                if (b2 < NB) {
                    uint32_t code;
                    ok = second_level(md, b1, i1, j1, b2, s8, code);
                    const int i = md.bond_i[b2], j = md.bond_j[b2];
                    const bool ti = i == i1 || i == j1, tj = j == i1 || j == j1;
                    if (ti != tj) dd -= 0.5f * bondJ(md, b2) * (float)(s8[i] * s8[j]);
                }
                cnt += __popc(__ballot_sync(0xffffffffu, ok));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dd += __shfl_xor_sync(0xffffffffu, dd, o);
            if (lane == 0) {
                hb[a] = cnt;
                hd[a] = 0.5f * bondJ(md, b1) * (diag_sh + dd);
            }
        }
        __syncthreads();
        if (warp == 0) {   // exclusive prefix of the sizes
            int run = 0;
            for (int a0 = 0; a0 < naa; a0 += 32) {
                const int a = a0 + lane;
                const int v = a < naa ? hb[a] : 0;
                int x = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += y;
                }
                if (a < naa) hb[a] = run + x - v;
                run += __shfl_sync(0xffffffffu, x, 31);
            }
            if (lane == 0) hb[naa] = run;
        }
        __syncthreads();

        // passes over ranges of b1 whose lists fit the shared list (one pass
        // unless a sample has more second-level flip sets than the capacity)
        for (int a0 = 0, pass = 0; pass == 0 || a0 < naa; ++pass) {
            if (threadIdx.x == 0) {
                int a1 = a0;
                while (a1 < naa && hb[a1 + 1] - hb[a0] <= la.cap) ++a1;
                // -1: one list above the capacity (the launch rules it out: cap >= nbonds)
                a_end = (a1 == a0 && a0 < naa) ? -1 : a1;
            }
            __syncthreads();
            const int a1 = a_end;
            if (a1 < 0) {
                if (threadIdx.x == 0) flag_range(md.status);
                break;
            }
            const int ebase = hb[a0];
            for (int a = a0 + warp; a < a1; a += nwarps) {
                const int b1 = aa[a] & 0x7fff;
                const int i1 = md.bond_i[b1], j1 = md.bond_j[b1];
                int pos = hb[a] - ebase;
                for (int b0 = 0; b0 < NB; b0 += 32) {
                    const int b2 = b0 + lane;
                    uint32_t code = 0;
                    const bool ok = b2 < NB && second_level(md, b1, i1, j1, b2, s8, code);
                    const unsigned bm = __ballot_sync(0xffffffffu, ok);
                    if (ok) ent[pos + __popc(bm & ((1u << lane) - 1u))] = code;
                    pos += __popc(bm);
                }
            }
            __syncthreads();

            // (every group of a warp runs the same loop trip counts, so that
            // the warp's shuffles see all lanes; groups past the last row run
            // row 0 and add nothing)
            for (int rbase = 0; rbase < K * G; rbase += ngroups) {
                const bool active = rbase + gidx < K * G;
                const int row = active ? rbase + gidx : 0;
                const int r = row / G, g = row - r * G;
                __syncwarp();
                for (int i = gl; i < N; i += GL) pgs[i] = md.perm[(size_t)g * N + i];
                __syncwarp();
                float tx[2 * NP], ty[2 * NP];
#pragma unroll
                for (int u = 0; u < 2 * NP; ++u) { tx[u] = 0.f; ty[u] = 0.f; }
                const cx<float> *Wr = md.Wt + (size_t)r * N * M;
                for (int i = 0; i < N; ++i) {
                    const cx<float> *wk = Wr + (size_t)pgs[i] * M;
                    const float si = s_sm[i];
#pragma unroll
                    for (int j = 0; j < NP; ++j) {
                        const int m = 2 * (gl + GL * j);
                        if ((M & 1) == 0 && m + 1 < M) {
                            const float4 v = *reinterpret_cast<const float4 *>(wk + m);
                            tx[2 * j] = fmaf(si, v.x, tx[2 * j]); ty[2 * j] = fmaf(si, v.y, ty[2 * j]);
                            tx[2 * j + 1] = fmaf(si, v.z, tx[2 * j + 1]); ty[2 * j + 1] = fmaf(si, v.w, ty[2 * j + 1]);
                        } else {
                            if (m < M) { const cx<float> v = wk[m]; tx[2 * j] = fmaf(si, v.x, tx[2 * j]); ty[2 * j] = fmaf(si, v.y, ty[2 * j]); }
                            if (m + 1 < M) { const cx<float> v = wk[m + 1]; tx[2 * j + 1] = fmaf(si, v.x, tx[2 * j + 1]); ty[2 * j + 1] = fmaf(si, v.y, ty[2 * j + 1]); }
                        }
                    }
                }
                cx<float> at{0.f, 0.f};
                if (md.use_bias) {
                    const cx<float> *ar = md.avec + (size_t)r * N;
                    for (int i = gl; i < N; i += GL) { const cx<float> v = ar[pgs[i]]; at.x += s_sm[i] * v.x; at.y += s_sm[i] * v.y; }
#pragma unroll
                    for (int o = GL / 2; o > 0; o >>= 1) {
                        at.x += __shfl_xor_sync(0xffffffffu, at.x, o);
                        at.y += __shfl_xor_sync(0xffffffffu, at.y, o);
                    }
                }
                for (int sg = 0; sg < md.nsign; ++sg) {
                    const float sign = sg ? -1.f : 1.f;
                    // ---- p of the lane's units and the row term ----
                    f2 px[NP], py[NP];
                    sc<float> prod{1.f, 0.f, 0};
                    const cx<float> *br = md.bvec + (size_t)r * M;
#pragma unroll
                    for (int j = 0; j < NP; ++j) {
                        float pxv[2], pyv[2];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int m = 2 * (gl + GL * j) + h;
                            pxv[h] = 0.f; pyv[h] = 0.f;
                            if (m < M) {
                                cx<float> th{sign * tx[2 * j + h], sign * ty[2 * j + h]};
                                if (md.use_bias) { const cx<float> b = br[m]; th.x += b.x; th.y += b.y; }
                                cx<float> mant, pv;
                                int k;
                                cosh2(th, mant, k, pv);
                                pxv[h] = pv.x; pyv[h] = pv.y;
                                const cx<float> q = cmul(mk(prod.x, prod.y), mant);
                                prod = sc<float>{q.x, q.y, prod.e + k};
                            }
                        }
                        px[j] = f2_pack(pxv[0], pxv[1]);
                        py[j] = f2_pack(pyv[0], pyv[1]);
                    }
                    prod = group_prod<GL>(prod);
                    const cx<float> lc = md.logc[r];
                    sc<float> lead = sc_exp(cx<float>{lc.x + sign * at.x, lc.y + sign * at.y});
                    float chg = md.chi[g];
                    if (sg && md.chiP < 0) chg = -chg;
                    lead.x *= chg; lead.y *= chg;
                    const sc<float> wt = sc_mul(prod, sc_norm(lead));   // the row term (every lane of the group)
                    if (pass == 0 && gl == 0 && active) gsum[2][gidx] = sc_add(gsum[2][gidx], sc<double>{(double)wt.x, (double)wt.y, wt.e});

                    double A1x = 0.0, A1y = 0.0, A2x = 0.0, A2y = 0.0;
                    const int rb = r * 2;
                    for (int a = a0; a < a1; ++a) {
                        const uint16_t c1code = aa[a];
                        const int b1 = c1code & 0x7fff;
                        const float J1b = bondJ(md, b1);
                        const int oi = (((c1code >> 15) != 0) == (sg == 0)) ? 0 : 1;   // sign s_i1 = +1 -> e^{-4W}
                        const int ki = pgs[md.bond_i[b1]], kj = pgs[md.bond_j[b1]];
                        const float4 *ri = ups + ((size_t)(rb + oi) * N + ki) * MH + gl;
                        const float4 *rj = ups + ((size_t)(rb + 1 - oi) * N + kj) * MH + gl;
                        // ---- first level: prod (1 + p (U1 - 1)) over the lane's units, p' and q ----
                        f2 ca[NP], cb[NP], cc[NP];
                        f2 Qx = one2, Qy = zero2, Px = one2, Py = zero2;
                        bool small = la.plain != 0;   // some |p'| < 2^-12: the plain form for this b1
#pragma unroll
                        for (int j = 0; j < NP; ++j) {
                            f2 uix, uiy, ujx, ujy;
                            lds128(ri + GL * j, uix, uiy);
                            lds128(rj + GL * j, ujx, ujy);
                            const f2 Ux = sub2(mul2(uix, ujx), mul2(uiy, ujy));
                            const f2 Uy = fma2(uix, ujy, mul2(uiy, ujx));
                            const f2 Tx = sub2(Ux, one2);
                            const f2 fx = sub2(fma2(px[j], Tx, one2), mul2(py[j], Uy));
                            const f2 fy = fma2(px[j], Uy, mul2(py[j], Tx));
                            const f2 nx = sub2(mul2(px[j], Ux), mul2(py[j], Uy));   // p U
                            const f2 ny = fma2(px[j], Uy, mul2(py[j], Ux));
                            const f2 den = fma2(fx, fx, mul2(fy, fy));
                            const f2 inv = f2_pack(__frcp_rn(f2_lo(den)), __frcp_rn(f2_hi(den)));
                            f2 ppx = mul2(fma2(nx, fx, mul2(ny, fy)), inv);          // p' = p U / f
                            f2 ppy = mul2(sub2(mul2(ny, fx), mul2(nx, fy)), inv);
                            const f2 pden = fma2(ppx, ppx, mul2(ppy, ppy));
                            const f2 pinv = f2_pack(__frcp_rn(f2_lo(pden)), __frcp_rn(f2_hi(pden)));
                            f2 qx = fma2(ppx, pinv, mone2);                           // q = 1/p' - 1
                            f2 qy = mul2(sub2(zero2, ppy), pinv);
                            const int m = 2 * (gl + GL * j);
                            if (m + 1 >= M) {   // padding units: f = U = 1 as p' = 1, q = 0
                                if (m >= M) { ppx = one2; ppy = zero2; qx = zero2; qy = zero2; }
                                else {
                                    ppx = f2_pack(f2_lo(ppx), 1.f); ppy = f2_pack(f2_lo(ppy), 0.f);
                                    qx = f2_pack(f2_lo(qx), 0.f); qy = f2_pack(f2_lo(qy), 0.f);
                                }
                            }
                            small = small || (m < M && !(f2_lo(pden) >= 0x1p-24f)) || (m + 1 < M && !(f2_hi(pden) >= 0x1p-24f));
                            ca[j] = qx; cb[j] = qy;
                            if (j == 0) {
                                Qx = fx; Qy = fy; Px = ppx; Py = ppy;
                            } else {
                                const f2 n1 = sub2(mul2(Qx, fx), mul2(Qy, fy));
                                Qy = fma2(Qx, fy, mul2(Qy, fx));
                                Qx = n1;
                                const f2 n2 = sub2(mul2(Px, ppx), mul2(Py, ppy));
                                Py = fma2(Px, ppy, mul2(Py, ppx));
                                Px = n2;
                            }
                        }
                        sc<float> R1, Pp;
                        {
                            const float x = f2_lo(Qx) * f2_hi(Qx) - f2_lo(Qy) * f2_hi(Qy);
                            const float y = f2_lo(Qx) * f2_hi(Qy) + f2_lo(Qy) * f2_hi(Qx);
                            R1 = group_prod<GL>(sc<float>{x, y, 0});
                            R1 = sc_mul(R1, sc_mul(eps[(rb + oi) * N + ki], eps[(rb + 1 - oi) * N + kj]));
                            const float u = f2_lo(Px) * f2_hi(Px) - f2_lo(Py) * f2_hi(Py);
                            const float v = f2_lo(Px) * f2_hi(Py) + f2_lo(Py) * f2_hi(Px);
                            Pp = group_prod<GL>(sc<float>{u, v, 0});
                        }
                        // ---- second level: b1's list ----
                        const uint32_t *le = ent + (hb[a] - ebase);
                        const int cnt = hb[a + 1] - hb[a];
                        float accx = 0.f, accy = 0.f;
                        double Ox = 0.0, Oy = 0.0;
                        sc<float> mult;
                        if (!__any_sync(0xffffffffu, small)) {
                            b1_list<GL, NP, true>(ups, eps, le, cnt, pgs, N, MH, rb, sg, J1b, md.J1, md.J2, ca, cb, cc,
                                                  Pp.e, gl, gbase, eq, owner, accx, accy, Ox, Oy);
                            mult = sc_mul(R1, sc<float>{Pp.x, Pp.y, 0});
                        } else {
                            // p' again (the plain form: no division by p')
#pragma unroll
                            for (int j = 0; j < NP; ++j) {
                                f2 uix, uiy, ujx, ujy;
                                lds128(ri + GL * j, uix, uiy);
                                lds128(rj + GL * j, ujx, ujy);
                                const f2 Ux = sub2(mul2(uix, ujx), mul2(uiy, ujy));
                                const f2 Uy = fma2(uix, ujy, mul2(uiy, ujx));
                                const f2 Tx = sub2(Ux, one2);
                                const f2 fx = sub2(fma2(px[j], Tx, one2), mul2(py[j], Uy));
                                const f2 fy = fma2(px[j], Uy, mul2(py[j], Tx));
                                const f2 nx = sub2(mul2(px[j], Ux), mul2(py[j], Uy));
                                const f2 ny = fma2(px[j], Uy, mul2(py[j], Ux));
                                const f2 den = fma2(fx, fx, mul2(fy, fy));
                                const f2 inv = f2_pack(__frcp_rn(f2_lo(den)), __frcp_rn(f2_hi(den)));
                                ca[j] = mul2(fma2(nx, fx, mul2(ny, fy)), inv);
                                cb[j] = mul2(sub2(mul2(ny, fx), mul2(nx, fy)), inv);
                                cc[j] = sub2(zero2, cb[j]);
                            }
                            b1_list<GL, NP, false>(ups, eps, le, cnt, pgs, N, MH, rb, sg, J1b, md.J1, md.J2, ca, cb,
                                                   cc, 0, gl, gbase, eq, owner, accx, accy, Ox, Oy);
                            mult = R1;
                        }
                        // ---- into the row's sums: R1 (c1 + c2_1) + mult x (the list's sum) ----
                        double mx, my, r1x, r1y;
                        sc_to_d(mult, mx, my);
                        sc_to_d(R1, r1x, r1y);
                        const double vx = (double)accx + Ox, vy = (double)accy + Oy;
                        A2x += mx * vx - my * vy;
                        A2y += mx * vy + my * vx;
                        if (gl == 0) {
                            const double c1 = 0.5 * (double)J1b, c21 = (double)hd[a];
                            A1x += c1 * r1x; A1y += c1 * r1y;
                            A2x += c21 * r1x; A2y += c21 * r1y;
                        }
                    }
#pragma unroll
                    for (int o = GL / 2; o > 0; o >>= 1) {
                        A1x += __shfl_xor_sync(0xffffffffu, A1x, o);
                        A1y += __shfl_xor_sync(0xffffffffu, A1y, o);
                        A2x += __shfl_xor_sync(0xffffffffu, A2x, o);
                        A2y += __shfl_xor_sync(0xffffffffu, A2y, o);
                    }
                    if (active && gl == 0) {
                        gsum[0][gidx] = sc_add(gsum[0][gidx], sd_mul(wt, A1x, A1y));
                        gsum[1][gidx] = sc_add(gsum[1][gidx], sd_mul(wt, A2x, A2y));
                    }
                }
            }
            __syncthreads();   // the lists of the next pass overwrite these
            a0 = a1;
        }
        // ---- sums over the CTA ----
        __syncthreads();
        if (threadIdx.x == 0) {
            sc<double> t1 = gsum[0][0], t2 = gsum[1][0], t0 = gsum[2][0];
            for (int q = 1; q < ngroups; ++q) { t1 = sc_add(t1, gsum[0][q]); t2 = sc_add(t2, gsum[1][q]); t0 = sc_add(t0, gsum[2][q]); }
            const double den = t0.x * t0.x + t0.y * t0.y;
            const double f1 = ldexp(1.0, t1.e - t0.e), f2v = ldexp(1.0, t2.e - t0.e);
            const double r1x = (t1.x * t0.x + t1.y * t0.y) / den * f1, r1y = (t1.y * t0.x - t1.x * t0.y) / den * f1;
            const double r2x = (t2.x * t0.x + t2.y * t0.y) / den * f2v, r2y = (t2.y * t0.x - t2.x * t0.y) / den * f2v;
            const double diag = (double)diag_sh;
            const double h1x = diag + r1x, h1y = r1y;
            const double h2x = diag * h1x + r2x + (double)cst_sh, h2y = diag * h1y + r2y;
            if (sc_zero(t0) || !isfinite(h1x) || !isfinite(h1y) || !isfinite(h2x) || !isfinite(h2y))
                flag_range(md.status);
            if (h1_out) { h1_out[2 * smp] = h1x; h1_out[2 * smp + 1] = h1y; }
            if (h2_out) { h2_out[2 * smp] = h2x; h2_out[2 * smp + 1] = h2y; }
        }
        __syncthreads();
    }
}

// Paired site factors: up[((r 2 + o) N + k) MH + kk] = (ux_2kk, ux_2kk+1,
// uy_2kk, uy_2kk+1), u = e^{-4W} (o = 0) or e^{+4W} (o = 1) from the model's
// per-site table, u = 1 past M.
__global__ void k_tables_site_paired(DevModel<float> md, int MH, float4 *__restrict__ up)
{
    const int64_t tot = (int64_t)md.K * 2 * md.N * MH;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < tot; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t rowi = q / MH;
        const int kk = (int)(q - rowi * MH);
        const cx<float> *src = md.S4 + rowi * md.Mp;
        const int m0 = 2 * kk, m1 = 2 * kk + 1;
        const cx<float> a = m0 < md.M ? src[m0] : cx<float>{1.f, 0.f};
        const cx<float> b = m1 < md.M ? src[m1] : cx<float>{1.f, 0.f};
        up[q] = make_float4(a.x, b.x, a.y, b.y);
    }
}

// variant: GL lanes per row, NP unit pairs per lane (GL = 0: unsupported)
void lf_variant(int M, int &GL, int &NP)
{
    if (M <= 128) { GL = 16; NP = (M + 31) / 32; }
    else if (M <= 256) { GL = 32; NP = (M + 63) / 64; }
    else { GL = 0; NP = 0; }
}

size_t lf_table_bytes(const DevModel<float> &md, int MH)
{
    return (size_t)md.K * 2 * md.N * MH * sizeof(float4) + (size_t)md.K * 2 * md.N * sizeof(sc<float>);
}

constexpr size_t kLfSmemLimit = 226 * 1024;   // dynamic + static shared memory of one CTA
constexpr size_t kLfStaticBytes = 24 * 1024;  // bound on the kernel's static shared memory

template <int GL, int NP>
cudaError_t lf_launch(const DevModel<float> &md, LfArgs la, const uint64_t *cfg, int64_t n, double *h1, double *h2,
                      int nsm, cudaStream_t st)
{
    auto kern = k_lanczos_fast<GL, NP>;
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    const size_t tables = lf_table_bytes(md, la.MH);
    if (fa.sharedSizeBytes + tables + 4 * (size_t)md.nbonds > kLfSmemLimit) return cudaErrorInvalidValue;
    size_t list = kLfSmemLimit - fa.sharedSizeBytes - tables;
    list &= ~(size_t)15;
    la.cap = (int)(list / sizeof(uint32_t));
    // Test hooks (unset in normal use): NNQS_TEST_LANCZOS_LIST=<entries> caps
    // the shared flip-set list (at least nbonds entries), so that samples take
    // several passes over b1; NNQS_TEST_LANCZOS_PLAIN=1 takes the plain form
    // of the second-level factors for every b1.
    if (const char *v = getenv("NNQS_TEST_LANCZOS_LIST")) {
        const long c = atol(v);
        if (c > 0) la.cap = (int)std::max<long>(md.nbonds, std::min<long>(la.cap, c));
    }
    if (const char *v = getenv("NNQS_TEST_LANCZOS_PLAIN")) la.plain = v[0] == '1';
    const size_t smem = tables + list;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int threads = kLfThreads;
    const int grid = (int)(n < nsm ? n : nsm);
    kern<<<grid, threads, smem, st>>>(md, la, cfg, n, h1, h2);
    return cudaGetLastError();
}

}  // namespace

bool lanczos_fast_supported(const DevModel<float> &md)
{
    int GL, NP;
    lf_variant(md.M, GL, NP);
    if (GL == 0 || md.N > 256 || md.nbonds > 4 * kMaxN) return false;
    // tables, a list of at least 4 nbonds entries and the static shared memory within one CTA
    return lf_table_bytes(md, GL * NP) + 16 * (size_t)md.nbonds + kLfStaticBytes <= kLfSmemLimit;
}

size_t lanczos_fast_table_bytes(const DevModel<float> &md)
{
    int GL, NP;
    lf_variant(md.M, GL, NP);
    return (size_t)md.K * 2 * md.N * (GL * NP) * sizeof(float4) + 256;
}

cudaError_t launch_tables_site_paired(const DevModel<float> &md, void *tables, cudaStream_t st)
{
    int GL, NP;
    lf_variant(md.M, GL, NP);
    k_tables_site_paired<<<256, 256, 0, st>>>(md, GL * NP, reinterpret_cast<float4 *>(tables));
    return cudaGetLastError();
}

cudaError_t launch_lanczos_fast(const DevModel<float> &md, const void *tables, const uint64_t *cfg, int64_t n,
                                double *h1, double *h2, int nsm, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    int GL, NP;
    lf_variant(md.M, GL, NP);
    LfArgs la;
    la.up = reinterpret_cast<const float4 *>(tables);
    la.MH = GL * NP;
    la.cap = 0;
    la.plain = 0;
    if (GL == 16) {
        switch (NP) {
        case 1: return lf_launch<16, 1>(md, la, cfg, n, h1, h2, nsm, st);
        case 2: return lf_launch<16, 2>(md, la, cfg, n, h1, h2, nsm, st);
        case 3: return lf_launch<16, 3>(md, la, cfg, n, h1, h2, nsm, st);
        default: return lf_launch<16, 4>(md, la, cfg, n, h1, h2, nsm, st);
        }
    }
    return NP <= 3 ? lf_launch<32, 3>(md, la, cfg, n, h1, h2, nsm, st) : lf_launch<32, 4>(md, la, cfg, n, h1, h2, nsm, st);
}

}  // namespace nnqs
