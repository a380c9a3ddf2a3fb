// k_eloc.cuh -- connected-configuration engine behind E_loc (Eq. 10) and the
// Lanczos quantities h1 = (H psi)/psi, h2 = (H^2 psi)/psi (Sec. 3.3).
//
// For a flip set D and a row (r, g, sign) of the projected sum (Eqs. 4-6),
// with p_m = e^{theta_m}/(2cosh theta_m):
//   cosh(theta_m + Delta_m)/cosh(theta_m) = e^{-Delta_m} (1 + p_m T_m),
//   T_m = e^{2 Delta_m} - 1,
// so the row's ratio is  exp(Delta_a - sum_m Delta_m) * prod_m (1 + p_m T_m).
// For an exchanged bond the T_m and the prefactor's exponent are read from
// per-bond tables (the bond's image under g and its orientation select the
// row of the table); two disjoint bonds multiply their (1 + T); a non-bond
// pair uses per-site tables exp(-+4W).  Per element: one 8-byte table load
// and two complex multiply-adds.
//
// Work layout: a CTA owns one sample at a time; each warp is split into
// 32/GL groups of GL lanes; a group owns one row (r, g) and its lanes own the
// hidden units m = gl + GL*j.  Entries are taken GL at a time; a butterfly
// reduce-scatter over the group leaves lane gl with the full product of entry
// gl, which it weights by the row term and accumulates.
#pragma once
#include "common.cuh"
#include "kernels.h"

namespace nnqs {

template <typename T> struct Entry2 {
    uint32_t code;  // bits 0-14 idx0, 15-29 idx1, 30-31 type
    T c1, c2;       // weight of the ratio in h1 and in h2
};
enum { kOneBond = 0, kTwoBonds = 1, kSitePair = 2 };

// E_loc mode of the narrow FP32 variants (GL = 8, M <= 72) reads the per-site
// tables exp(-+4W) ([K][2][N][Mp], small enough to stay in L1) and forms
// 1 + T = e^{-4 s_u W_u} e^{+4 s_u W_v} per element, instead of the per-bond
// tables T ([K][2][4N][Mp], four times larger); the wider variants keep the
// per-bond tables (the second table stream costs them registers), and so does
// FP64, where the extra complex multiply costs more than the cache misses.
template <typename T, int GL, int MPL> __host__ __device__ constexpr bool eloc_site_pairs()
{
    return sizeof(T) == 4 && GL == 8 && MPL <= 9;
}

__device__ __forceinline__ uint32_t ecode(int type, int i0, int i1)
{
    return (uint32_t)i0 | ((uint32_t)i1 << 15) | ((uint32_t)type << 30);
}

// Candidates in a fixed order (see the header of the kernel):
//   mode 0: q = bond q, valid if anti-aligned.
//   mode 1: q = a * (4N + 1) + slot over the anti-aligned bonds b1 = aa[a]:
//     slot 0      -> first-level exchange of b1,
//     slot 1 + b2 -> second-level configuration after exchanging b2 in s^{b1}:
//       one shared site (b2 anti-aligned in s^{b1}) -> pair of flipped sites,
//       disjoint, anti-aligned, b2 > b1             -> both bonds, counted twice.
template <bool SITE, typename T>
__device__ __forceinline__ bool candidate2(const DevModel<T> &md, int mode, int q, const int8_t *s8,
                                           const int16_t *aa, T diag, Entry2<T> &e)
{
    const int nb = md.nbonds;
    if (mode == 0) {
        const int i = md.bond_i[q], j = md.bond_j[q];
        if (s8[i] == s8[j]) return false;
        // exchanging an anti-aligned bond flips its two sites
        e.code = SITE ? ecode(kSitePair, i, j) : ecode(kOneBond, q, s8[i] > 0);
        e.c1 = T(0.5) * bondJ(md, q);
        e.c2 = T(0);
        return true;
    }
    const int a = q / (nb + 1), slot = q - a * (nb + 1);
    const int b1 = aa[a];
    const int i1 = md.bond_i[b1], j1 = md.bond_j[b1];
    const T J1b = bondJ(md, b1);
    if (slot == 0) {
        T d = diag;  // diagonal energy of s^{b1}
        for (int b = 0; b < nb; ++b) {
            const int i = md.bond_i[b], j = md.bond_j[b];
            const bool ti = (i == i1 || i == j1), tj = (j == i1 || j == j1);
            if (ti == tj) continue;
            const int si = s8[i], sj = s8[j];
            const int si2 = (i == i1) ? s8[j1] : (i == j1) ? s8[i1] : si;
            const int sj2 = (j == i1) ? s8[j1] : (j == j1) ? s8[i1] : sj;
            d += T(0.25) * bondJ(md, b) * T(si2 * sj2 - si * sj);
        }
        e.code = ecode(kOneBond, b1, s8[i1] > 0);
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
        e.code = ecode(kTwoBonds, b1, b2);
        e.c1 = T(0);
        e.c2 = T(0.5) * J1b * J2b;
        return true;
    }
    auto sp = [&](int x) { return x == i1 ? s8[j1] : x == j1 ? s8[i1] : s8[x]; };
    if (sp(i2) == sp(j2)) return false;
    const int u = (i1 != i2 && i1 != j2) ? i1 : j1;
    const int v = (i2 != i1 && i2 != j1) ? i2 : j2;
    e.code = ecode(kSitePair, u, v);
    e.c1 = T(0);
    e.c2 = T(0.25) * J1b * J2b;
    return true;
}

// Per (row, entry) decode: table offsets of sign +1 and the prefactor exponent.
template <typename T> struct Dec {
    int type;
    int o0, o1;      // element offsets (m = 0) into Tb (types 0, 1) or S4 (type 2), sign +1
    int d0, d1;      // offset deltas that select the opposite orientation
    cx<T> E;         // prefactor exponent for sign +1 (sign -1 uses -E)
};

template <typename T, bool WITH_E>
__device__ __forceinline__ Dec<T> decode(const DevModel<T> &md, uint32_t code, int r, int g, const int8_t *s8)
{
    Dec<T> d;
    const int nb = md.nbonds, Mp = md.Mp, N = md.N;
    d.type = (int)(code >> 30);
    const int i0 = code & 0x7fff, i1 = (code >> 15) & 0x7fff;
    const int rb = r * 2 * nb * Mp;   // Tb block of RBM r
    d.E = cx<T>{T(0), T(0)};
    if (d.type != kSitePair) {
        const uint16_t bp0 = md.bperm[(size_t)g * nb + i0];
        const int bb0 = bp0 & 0x7fff;
        const int si0 = d.type == kOneBond ? (i1 ? 1 : -1) : s8[md.bond_i[i0]];
        const int s0 = si0 * ((bp0 >> 15) ? -1 : 1);
        d.o0 = rb + ((s0 > 0 ? 0 : 1) * nb + bb0) * Mp;
        d.d0 = s0 > 0 ? nb * Mp : -nb * Mp;
        if (WITH_E) {
            const cx<T> c0 = md.Cb[(size_t)r * nb + bb0];
            d.E = cx<T>{T(s0) * c0.x, T(s0) * c0.y};
        }
        d.o1 = 0; d.d1 = 0;
        if (d.type == kTwoBonds) {
            const uint16_t bp1 = md.bperm[(size_t)g * nb + i1];
            const int bb1 = bp1 & 0x7fff;
            const int s1 = s8[md.bond_i[i1]] * ((bp1 >> 15) ? -1 : 1);
            d.o1 = rb + ((s1 > 0 ? 0 : 1) * nb + bb1) * Mp;
            d.d1 = s1 > 0 ? nb * Mp : -nb * Mp;
            if (WITH_E) {
                const cx<T> c1 = md.Cb[(size_t)r * nb + bb1];
                d.E.x += T(s1) * c1.x;
                d.E.y += T(s1) * c1.y;
            }
        }
    } else {
        // sites u (spin s_u) and v (spin -s_u) flipped
        const int ku = md.perm[(size_t)g * N + i0], kv = md.perm[(size_t)g * N + i1];
        const int su = s8[i0];
        const int rs = r * 2 * N * Mp;
        d.o0 = rs + ((su > 0 ? 0 : 1) * N + ku) * Mp;
        d.d0 = su > 0 ? N * Mp : -N * Mp;
        d.o1 = rs + ((su > 0 ? 1 : 0) * N + kv) * Mp;
        d.d1 = su > 0 ? -N * Mp : N * Mp;
        if (WITH_E) {
            cx<T> ca{T(0), T(0)};
            if (md.use_bias) {
                const cx<T> au = md.avec[(size_t)r * N + ku], av = md.avec[(size_t)r * N + kv];
                ca = cx<T>{T(-2) * (au.x - av.x), T(-2) * (au.y - av.y)};
            }
            const cx<T> cu = md.CS[(size_t)r * N + ku], cv = md.CS[(size_t)r * N + kv];
            const cx<T> c{ca.x + T(2) * (cu.x - cv.x), ca.y + T(2) * (cu.y - cv.y)};
            d.E = cx<T>{T(su) * c.x, T(su) * c.y};
        }
    }
    return d;
}

// prod over the lane's hidden units m = gl + GL j of (1 + p_m T_m) for one
// entry and one sign.  The tables are padded to GL * MPL with neutral entries
// (and p_m = 0 past M), so no bound check is needed.
// Per-lane state of the Lanczos mode for pairs of disjoint exchanged bonds
// (b1, b2), which the candidate order keeps consecutive for a fixed b1: after
// the first exchange p_m becomes p'_m = p_m (1 + T1_m) / (1 + p_m T1_m) (the
// p of the configuration with b1 exchanged), so that
//   prod_m (1 + p_m T12_m) = prod_m (1 + p_m T1_m) * prod_m (1 + p'_m T2_m),
// one table row per element instead of two.  key identifies (T1 row, sign)
// within one row (r, g) of the projected sum; -1 = empty.
template <typename T, int MPL> struct PairCache {
    int key;
    cx<T> q1;        // prod over the lane's units of (1 + p T1)
    cx<T> pp[MPL];   // p' of the lane's units
};

template <typename T, int GL, int MPL, bool ONLY1, bool ONLYSITE = false>
__device__ __forceinline__ cx<T> entry_partial(const DevModel<T> &md, const Dec<T> &d, int sg, const cx<T> (&p)[MPL],
                                               int gl, PairCache<T, MPL> *pc = nullptr)
{
    const int o0 = (sg ? d.o0 + d.d0 : d.o0) + gl;
    const int o1 = (sg ? d.o1 + d.d1 : d.o1) + gl;
    cx<T> pr{T(1), T(0)};
    if constexpr (ONLYSITE) {
        const cx<T> *__restrict__ t0p = md.S4 + o0;
        const cx<T> *__restrict__ t1p = md.S4 + o1;
#pragma unroll
        for (int j = 0; j < MPL; ++j) {
            const cx<T> x = cmul(t0p[GL * j], t1p[GL * j]);
            const cx<T> t{x.x - T(1), x.y};
            const cx<T> f{T(1) + p[j].x * t.x - p[j].y * t.y, p[j].x * t.y + p[j].y * t.x};
            pr = cmul(pr, f);
        }
        return pr;
    }
    if (ONLY1 || d.type == kOneBond) {
        const cx<T> *__restrict__ tb = md.Tb + o0;
#pragma unroll
        for (int j = 0; j < MPL; ++j) {
            const cx<T> t = tb[GL * j];
            const cx<T> f{T(1) + p[j].x * t.x - p[j].y * t.y, p[j].x * t.y + p[j].y * t.x};
            pr = cmul(pr, f);
        }
    } else if constexpr (!ONLY1) {
        if (pc && d.type == kTwoBonds) {
            const int key = 2 * o0 + sg;
            if (key != pc->key) {
                pc->key = key;
                const cx<T> *__restrict__ t1p = md.Tb + o0;
                cx<T> q{T(1), T(0)};
#pragma unroll
                for (int j = 0; j < MPL; ++j) {
                    const cx<T> t = t1p[GL * j];
                    const cx<T> f{T(1) + p[j].x * t.x - p[j].y * t.y, p[j].x * t.y + p[j].y * t.x};
                    q = cmul(q, f);
                    pc->pp[j] = cdiv(cmul(p[j], cx<T>{T(1) + t.x, t.y}), f);
                }
                pc->q1 = q;
            }
            const cx<T> *__restrict__ t2p = md.Tb + o1;
            pr = pc->q1;
#pragma unroll
            for (int j = 0; j < MPL; ++j) {
                const cx<T> t = t2p[GL * j];
                const cx<T> q = pc->pp[j];
                const cx<T> f{T(1) + q.x * t.x - q.y * t.y, q.x * t.y + q.y * t.x};
                pr = cmul(pr, f);
            }
            return pr;
        }
        const cx<T> *__restrict__ tab = d.type == kTwoBonds ? md.Tb : md.S4;
        const cx<T> *__restrict__ t0p = tab + o0;
        const cx<T> *__restrict__ t1p = tab + o1;
#pragma unroll
        for (int j = 0; j < MPL; ++j) {
            const cx<T> t0 = t0p[GL * j], t1 = t1p[GL * j];
            cx<T> t;
            if (d.type == kTwoBonds) {
                t = cadd(cadd(t0, t1), cmul(t0, t1));  // (1 + t0)(1 + t1) - 1
            } else {
                const cx<T> x = cmul(t0, t1);
                t = cx<T>{x.x - T(1), x.y};
            }
            const cx<T> f{T(1) + p[j].x * t.x - p[j].y * t.y, p[j].x * t.y + p[j].y * t.x};
            pr = cmul(pr, f);
        }
    }
    return pr;
}

// mantissa / exponent split of a partial product, skipped in the common range
template <typename T> __device__ __forceinline__ void split(cx<T> pr, T &x, T &y, int &e)
{
    const T mx = fmax(fabs(pr.x), fabs(pr.y));
    if (mx > T(9.094947017729282e-13) && mx < T(1.099511627776e12)) {  // 2^-40 .. 2^40
        x = pr.x; y = pr.y; e = 0;
    } else {
        e = expo<T>(pr.x, pr.y);
        const T scl = pow2i<T>(-e);
        x = pr.x * scl; y = pr.y * scl;
    }
}

// Per-CTA state of the connected-configuration engine for one sample.
template <typename T> struct EShared {
    T s_sm[kMaxN];
    int8_t s8[kMaxN];
    int16_t aa[4 * kMaxN];
    int n_aa, n_ent, cursor, first_over;
    int wcount[kWarps];
    sc<T> wacc0[kWarps];
    sc<T> S0;
    double red[kWarps][4];
    double Hs[4];
    T diag_sh, cst_sh;
};

// h1 (and, for MODE 1, h2) of one sample: cfg_row = its configuration words,
// h1o / h2o = its two output doubles (may be NULL).  Called by every thread of
// the CTA; smem_raw holds the entries, the accumulators and the tiles.
template <typename T, int GL, int MPL, int MODE>
__device__ __forceinline__ void eloc_sample(const DevModel<T> &md, const uint64_t *__restrict__ cfg_row, int chunk,
                                            double *h1o, double *h2o, EShared<T> &S, unsigned char *smem_raw)
{
    constexpr int mode = MODE;
    constexpr int NG = 32 / GL;
    Entry2<T> *ent = reinterpret_cast<Entry2<T> *>(smem_raw);
    sc<T> *acc = reinterpret_cast<sc<T> *>(smem_raw + sizeof(Entry2<T>) * chunk);  // [kWarps][chunk]
    // transpose tiles of the partial products: [kWarps][TQ][33], TQ = GL (8 for GL = 32)
    constexpr int TQ = GL < 32 ? GL : 8;
    T *tx = reinterpret_cast<T *>(smem_raw + (sizeof(Entry2<T>) + kWarps * sizeof(sc<T>)) * chunk);
    T *ty = tx + kWarps * TQ * 33;
    int *te = reinterpret_cast<int *>(ty + kWarps * TQ * 33);

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane / GL, gl = lane % GL;
    const int rows = md.K * md.G;
    const int nb = md.nbonds, N = md.N, M = md.M;
    const int slot = warp * NG + grp, nslots = kWarps * NG;
    {
        const uint64_t *w = cfg_row;
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            const int sv = spin_of(w, i);
            S.s_sm[i] = T(sv);
            S.s8[i] = (int8_t)sv;
        }
    }
    __syncthreads();
    if (warp == 0) {
        T d = T(0), c = T(0);
        int base = 0;
        for (int b0 = 0; b0 < nb; b0 += 32) {
            const int b = b0 + lane;
            bool isaa = false;
            if (b < nb) {
                const int si = S.s8[md.bond_i[b]], sj = S.s8[md.bond_j[b]];
                const T J = bondJ(md, b);
                d += T(0.25) * J * T(si * sj);
                isaa = si != sj;
                if (isaa) c += T(0.25) * J * J;
            }
            const unsigned bm = __ballot_sync(0xffffffffu, isaa);
            if (isaa) S.aa[base + __popc(bm & ((1u << lane) - 1u))] = (int16_t)b;
            base += __popc(bm);
        }
        for (int o = 16; o > 0; o >>= 1) {
            d += __shfl_xor_sync(0xffffffffu, d, o);
            c += __shfl_xor_sync(0xffffffffu, c, o);
        }
        if (lane == 0) { S.diag_sh = d; S.cst_sh = c; S.n_aa = base; S.cursor = 0; }
    }
    __syncthreads();
    const int ncand = mode == 0 ? nb : S.n_aa * (nb + 1);
    bool first_chunk = true;
    while (true) {
        // ---- gather up to `chunk` entries in candidate order ----
        if (threadIdx.x == 0) S.n_ent = 0;
        __syncthreads();
        while (true) {
            const int cur = S.cursor;
            if (cur >= ncand || S.n_ent >= chunk) break;
            const int q = cur + threadIdx.x;
            Entry2<T> e;
            const bool valid = q < ncand && candidate2<eloc_site_pairs<T, GL, MPL>()>(md, mode, q, S.s8, S.aa, S.diag_sh, e);
            const unsigned bm = __ballot_sync(0xffffffffu, valid);
            if (lane == 0) S.wcount[warp] = __popc(bm);
            if (threadIdx.x == 0) S.first_over = INT_MAX;
            __syncthreads();
            int pos = __popc(bm & ((1u << lane) - 1u));
            for (int w = 0; w < warp; ++w) pos += S.wcount[w];
            const int room = chunk - S.n_ent;
            if (valid) {
                if (pos < room) ent[S.n_ent + pos] = e;
                else atomicMin(&S.first_over, q);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                int tot = 0;
                for (int w = 0; w < kWarps; ++w) tot += S.wcount[w];
                S.n_ent += tot < room ? tot : room;
                S.cursor = S.first_over != INT_MAX ? S.first_over : cur + blockDim.x;
            }
            __syncthreads();
        }
        const int ne = S.n_ent;
        if (ne == 0 && !first_chunk) break;
        for (int idx = threadIdx.x; idx < kWarps * ne; idx += blockDim.x) {
            const int w = idx / ne, e = idx - w * ne;
            acc[w * chunk + e] = sc<T>{T(0), T(0), 0};
        }
        __syncthreads();

        sc<T> a0{T(0), T(0), 0};
        for (int rbase = 0; rbase < rows; rbase += nslots) {
            PairCache<T, MPL> pcache;
            pcache.key = -1;
            const int row = rbase + slot;
            const bool active = row < rows;
            const int r = active ? row / md.G : 0, g = active ? row - (row / md.G) * md.G : 0;
            // ---- theta' = W_r T_g s for the lane's hidden units ----
            cx<T> thp[MPL];
#pragma unroll
            for (int j = 0; j < MPL; ++j) thp[j] = cx<T>{T(0), T(0)};
            const uint8_t *pg = md.perm + (size_t)g * N;
            const cx<T> *Wr = md.Wt + (size_t)r * N * M;
            for (int i = 0; i < N; ++i) {
                const cx<T> *wk = Wr + (size_t)pg[i] * M;
                const T si = S.s_sm[i];
#pragma unroll
                for (int j = 0; j < MPL; ++j) {
                    const int m = gl + GL * j;
                    if (m < M) { const cx<T> w = wk[m]; thp[j].x += si * w.x; thp[j].y += si * w.y; }
                }
            }
            cx<T> at{T(0), T(0)};
            if (md.use_bias) {
                const cx<T> *ar = md.avec + (size_t)r * N;
                for (int i = gl; i < N; i += GL) { const cx<T> a = ar[pg[i]]; at.x += S.s_sm[i] * a.x; at.y += S.s_sm[i] * a.y; }
#pragma unroll
                for (int o = GL / 2; o > 0; o >>= 1) { at.x += shfl_x(at.x, o); at.y += shfl_x(at.y, o); }
            }
            // ---- p_m and the row terms of both signs ----
            cx<T> p[2][MPL];
            sc<T> term[2];
#pragma unroll
            for (int sg = 0; sg < 2; ++sg) {
                const int sign = sg ? -1 : 1;
                sc<T> prod{T(1), T(0), 0};
                const cx<T> *br = md.bvec + (size_t)r * M;
#pragma unroll
                for (int j = 0; j < MPL; ++j) {
                    const int m = gl + GL * j;
                    if (m < M && sg < md.nsign) {
                        cx<T> th{sign * thp[j].x, sign * thp[j].y};
                        if (md.use_bias) { const cx<T> b = br[m]; th.x += b.x; th.y += b.y; }
                        cx<T> mant; int k;
                        cosh2(th, mant, k, p[sg][j]);
                        const cx<T> q = cmul(mk(prod.x, prod.y), mant);
                        prod = sc<T>{q.x, q.y, prod.e + k};
                    } else {
                        p[sg][j] = cx<T>{T(0), T(0)};
                    }
                }
                prod = sc_norm(prod);
#pragma unroll
                for (int o = GL / 2; o > 0; o >>= 1) {
                    sc<T> w{shfl_x(prod.x, o), shfl_x(prod.y, o), __shfl_xor_sync(0xffffffffu, prod.e, o)};
                    prod = sc_mul(prod, w);
                }
                if (sg < md.nsign && active) {
                    const cx<T> lc = md.logc[r];
                    sc<T> lead = sc_exp(cx<T>{lc.x + sign * at.x, lc.y + sign * at.y});
                    T c = md.chi[g];
                    if (sign < 0 && md.chiP < 0) c = -c;
                    lead.x *= c; lead.y *= c;
                    term[sg] = sc_mul(prod, sc_norm(lead));
                } else {
                    term[sg] = sc<T>{T(0), T(0), 0};
                }
            }
            if (first_chunk && gl == 0) a0 = sc_add(a0, sc_add(term[0], term[1]));

            // ---- entries, GL at a time ----
            if constexpr (GL < 32) {
                // Rolled loop over the GL entries of a batch: each lane writes its
                // partial product (over its hidden units) of entry e0 + q into the
                // group's tile; lane gl then multiplies the GL partials of entry
                // e0 + gl.  Tile [warp][q][lane], row stride 33 words.
                T *bx = tx + warp * GL * 33, *by = ty + warp * GL * 33;
                int *be = te + warp * GL * 33;
                for (int e0 = 0; e0 < ne; e0 += GL) {
                    sc<T> mine{T(0), T(0), 0};  // lane gl: contribution of entry e0 + gl
#pragma unroll
                    for (int sg = 0; sg < 2; ++sg) {
                        if (sg >= md.nsign) break;
#pragma unroll 1
                        for (int q = 0; q < GL; ++q) {
                            const int e = e0 + q;
                            cx<T> pr{T(1), T(0)};
                            if (e < ne) {
                                const Dec<T> d = decode<T, false>(md, ent[e].code, r, g, S.s8);
                                pr = entry_partial<T, GL, MPL, MODE == 0 && !eloc_site_pairs<T, GL, MPL>(), MODE == 0 && eloc_site_pairs<T, GL, MPL>()>(md, d, sg, p[sg], gl, (MODE == 1 && MPL <= 13) ? &pcache : nullptr);
                            }
                            T sx, sy;
                            int ex;
                            split(pr, sx, sy, ex);
                            bx[q * 33 + lane] = sx;
                            by[q * 33 + lane] = sy;
                            be[q * 33 + lane] = ex;
                        }
                        __syncwarp();
                        cx<T> pr{T(1), T(0)};
                        int pe = 0;
#pragma unroll
                        for (int k = 0; k < GL; ++k) {
                            const int idx = gl * 33 + grp * GL + k;
                            pr = cmul(pr, cx<T>{bx[idx], by[idx]});
                            pe += be[idx];
                            if ((k & 1) == 1) {   // values are below 2^40: renormalise every two
                                T sx, sy;
                                int ex;
                                split(pr, sx, sy, ex);
                                pr = cx<T>{sx, sy};
                                pe += ex;
                            }
                        }
                        __syncwarp();
                        const int e = e0 + gl;
                        if (e < ne && active) {
                            const Dec<T> d = decode<T, true>(md, ent[e].code, r, g, S.s8);
                            const cx<T> E = sg ? cx<T>{-d.E.x, -d.E.y} : d.E;
                            const sc<T> c = sc_mul(sc_norm(sc<T>{pr.x, pr.y, pe}), sc_exp(E));
                            mine = sc_add(mine, sc_mul(c, term[sg]));
                        }
                    }
                    // sum over the warp's groups (they hold the same entry index)
#pragma unroll
                    for (int o = GL; o < 32; o <<= 1) {
                        const sc<T> w{shfl_x(mine.x, o), shfl_x(mine.y, o), __shfl_xor_sync(0xffffffffu, mine.e, o)};
                        mine = sc_add(mine, w);
                    }
                    if (grp == 0 && e0 + gl < ne)
                        acc[warp * chunk + e0 + gl] = sc_add(acc[warp * chunk + e0 + gl], mine);
                }
            } else {
                // One row per warp: transpose the lanes' partial products of 8
                // entries through shared memory; lane (e, part) multiplies 8 of
                // the 32 partials of entry e, two shuffle stages combine the parts.
                T *bx = tx + warp * TQ * 33, *by = ty + warp * TQ * 33;
                int *be = te + warp * TQ * 33;
                const int el = lane & 7, part = lane >> 3;
                for (int e0 = 0; e0 < ne; e0 += 8) {
#pragma unroll
                    for (int sg = 0; sg < 2; ++sg) {
                        if (sg >= md.nsign) break;
#pragma unroll 1
                        for (int q = 0; q < 8; ++q) {
                            const int e = e0 + q;
                            cx<T> pr{T(1), T(0)};
                            if (e < ne) {
                                const Dec<T> d = decode<T, false>(md, ent[e].code, r, g, S.s8);
                                pr = entry_partial<T, GL, MPL, MODE == 0 && !eloc_site_pairs<T, GL, MPL>(), MODE == 0 && eloc_site_pairs<T, GL, MPL>()>(md, d, sg, p[sg], gl, (MODE == 1 && MPL <= 13) ? &pcache : nullptr);
                            }
                            T sx, sy;
                            int ex;
                            split(pr, sx, sy, ex);
                            bx[q * 33 + lane] = sx;
                            by[q * 33 + lane] = sy;
                            be[q * 33 + lane] = ex;
                        }
                        __syncwarp();
                        cx<T> pr{T(1), T(0)};
                        int pe = 0;
#pragma unroll
                        for (int l = 0; l < 8; ++l) {
                            const int idx = el * 33 + part * 8 + l;
                            pr = cmul(pr, cx<T>{bx[idx], by[idx]});
                            pe += be[idx];
                            if ((l & 1) == 1) {   // values are below 2^40: renormalise every two
                                T sx, sy;
                                int ex;
                                split(pr, sx, sy, ex);
                                pr = cx<T>{sx, sy};
                                pe += ex;
                            }
                        }
                        __syncwarp();
#pragma unroll
                        for (int o = 8; o < 32; o <<= 1) {
                            const cx<T> w{shfl_x(pr.x, o), shfl_x(pr.y, o)};
                            pe += __shfl_xor_sync(0xffffffffu, pe, o);
                            pr = cmul(pr, w);
                            T sx, sy;
                            int ex;
                            split(pr, sx, sy, ex);
                            pr = cx<T>{sx, sy};
                            pe += ex;
                        }
                        const int e = e0 + el;
                        if (part == 0 && e < ne && active) {
                            const Dec<T> d = decode<T, true>(md, ent[e].code, r, g, S.s8);
                            const cx<T> E = sg ? cx<T>{-d.E.x, -d.E.y} : d.E;
                            const sc<T> c = sc_mul(sc_norm(sc<T>{pr.x, pr.y, pe}), sc_exp(E));
                            acc[warp * chunk + e] = sc_add(acc[warp * chunk + e], sc_mul(c, term[sg]));
                        }
                    }
                }
            }
        }
        if (first_chunk) {
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const sc<T> w{shfl_x(a0.x, o), shfl_x(a0.y, o), __shfl_xor_sync(0xffffffffu, a0.e, o)};
                a0 = sc_add(a0, w);
            }
            if (lane == 0) S.wacc0[warp] = a0;
        }
        __syncthreads();
        if (first_chunk && threadIdx.x == 0) {
            sc<T> tot = S.wacc0[0];
            for (int w = 1; w < kWarps; ++w) tot = sc_add(tot, S.wacc0[w]);
            S.S0 = tot;
        }
        __syncthreads();
        double p1x = 0, p1y = 0, p2x = 0, p2y = 0;
        for (int e = threadIdx.x; e < ne; e += blockDim.x) {
            sc<T> se = acc[e];
            for (int w = 1; w < kWarps; ++w) se = sc_add(se, acc[w * chunk + e]);
            const sc<T> s0 = S.S0;
            double Rx = 0, Ry = 0;
            if (!sc_zero(se)) {
                const double f = ldexp(1.0, se.e - s0.e);
                const double ax = (double)se.x, ay = (double)se.y, bx = (double)s0.x, by = (double)s0.y;
                const double den = bx * bx + by * by;
                Rx = (ax * bx + ay * by) / den * f;
                Ry = (ay * bx - ax * by) / den * f;
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
        if (lane == 0) { S.red[warp][0] = p1x; S.red[warp][1] = p1y; S.red[warp][2] = p2x; S.red[warp][3] = p2y; }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (first_chunk) { S.Hs[0] = S.Hs[1] = S.Hs[2] = S.Hs[3] = 0.0; }
            for (int w = 0; w < kWarps; ++w)
                for (int c = 0; c < 4; ++c) S.Hs[c] += S.red[w][c];
        }
        first_chunk = false;
        __syncthreads();
        if (S.cursor >= ncand) break;
    }
    if (threadIdx.x == 0) {
        const sc<T> s0 = S.S0;
        const double diag = (double)S.diag_sh;
        const double h1x = diag + S.Hs[0], h1y = S.Hs[1];
        if (!sc_finite(s0) || sc_zero(s0) || !isfinite(h1x) || !isfinite(h1y)) flag_range(md.status);
        if (h1o) { h1o[0] = h1x; h1o[1] = h1y; }
        if (mode == 1 && h2o) {
            h2o[0] = diag * h1x + S.Hs[2] + (double)S.cst_sh;
            h2o[1] = diag * h1y + S.Hs[3];
        }
    }
    __syncthreads();
}

// CTAs per SM the register budget is sized for: three (80 registers) where
// the FP32 variant needs no spill at that budget, else two (128 registers);
// FP64 is left to the compiler.
template <typename T, int GL, int MPL, int MODE> constexpr int eloc_min_blocks()
{
    if (sizeof(T) != 4) return 1;
    if (MODE == 1) return (GL == 8 && MPL <= 4) ? 3 : 2;   // the pair cache needs registers
    if (GL == 8) return 3;
    return MPL == 8 ? 3 : 2;
}

template <typename T, int GL, int MPL, int MODE>
__global__ void __launch_bounds__(kThreads, eloc_min_blocks<T, GL, MPL, MODE>()) k_eloc(DevModel<T> md, const uint64_t *__restrict__ cfg, int64_t n,
                                                   int chunk, double *__restrict__ h1_out, double *__restrict__ h2_out)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ EShared<T> S;
    for (int64_t smp = blockIdx.x; smp < n; smp += gridDim.x)
        eloc_sample<T, GL, MPL, MODE>(md, cfg + smp * md.nwords, chunk, h1_out ? h1_out + 2 * smp : nullptr,
                                      h2_out ? h2_out + 2 * smp : nullptr, S, smem_raw);
}

// Launcher of one (T, GL, MPL) variant; each variant is instantiated in its
// own translation unit (k_eloc_<type>_<GL>_<MPL>.cu) so they compile in parallel.
template <typename T, int GL> size_t eloc_smem(int chunk)
{
    const size_t tiles = (size_t)kWarps * (GL < 32 ? GL : 8) * 33 * (2 * sizeof(T) + sizeof(int));
    return (sizeof(Entry2<T>) + kWarps * sizeof(sc<T>)) * (size_t)chunk + tiles;
}

// Entries gathered per pass in the Lanczos mode: small enough that the
// shared memory of three CTAs fits an SM where the registers allow three, and
// at two CTAs small enough to leave L1 room for the per-bond table rows.
template <typename T, int GL, int MPL> constexpr int eloc_lanczos_chunk()
{
    return eloc_min_blocks<T, GL, MPL, 1>() < 3 ? 256 : (GL == 16 ? 160 : 384);
}

template <typename T, int GL, int MPL, int MODE>
cudaError_t launch_eloc_mode(const DevModel<T> &md, const uint64_t *cfg, int64_t n, int chunk, double *h1, double *h2,
                             int nsm, cudaStream_t st)
{
    if (MODE == 1) chunk = eloc_lanczos_chunk<T, GL, MPL>();
    const size_t smem = eloc_smem<T, GL>(chunk);
    cudaError_t err =
        cudaFuncSetAttribute(k_eloc<T, GL, MPL, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per = 0;
    if (err == cudaSuccess)
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_eloc<T, GL, MPL, MODE>, kThreads, smem);
    if (err != cudaSuccess) return err;
    const int64_t grid = (int64_t)(per > 0 ? per : 1) * nsm;
    const int gsz = (int)(n < grid ? n : grid);
    k_eloc<T, GL, MPL, MODE><<<gsz, kThreads, smem, st>>>(md, cfg, n, chunk, h1, h2);
    return cudaGetLastError();
}

}  // namespace nnqs
