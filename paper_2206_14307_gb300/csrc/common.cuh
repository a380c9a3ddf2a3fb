// common.cuh -- device-side types and arithmetic shared by the kernels of the
// projected-RBM VMC library (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace nnqs {

constexpr int kMaxL = 16;
constexpr int kMaxN = kMaxL * kMaxL;
constexpr int kMaxWords = (kMaxN + 63) / 64;
constexpr int kMaxM = 512;
constexpr int kMaxK = 8;
constexpr int kWarps = 8;           // warps per CTA of the amplitude kernels
constexpr int kThreads = kWarps * 32;

// ---------------------------------------------------------------------------
// Complex numbers
// ---------------------------------------------------------------------------
template <typename T> struct alignas(2 * sizeof(T)) cx { T x, y; };
template <typename T> struct alignas(4 * sizeof(T) > 16 ? 16 : 4 * sizeof(T)) cx2 { cx<T> a, b; };

template <typename T> __host__ __device__ __forceinline__ cx<T> mk(T x, T y) { return cx<T>{x, y}; }
template <typename T> __device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b)
{
    return cx<T>{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T> __device__ __forceinline__ cx<T> cadd(cx<T> a, cx<T> b) { return cx<T>{a.x + b.x, a.y + b.y}; }
template <typename T> __device__ __forceinline__ cx<T> csub(cx<T> a, cx<T> b) { return cx<T>{a.x - b.x, a.y - b.y}; }
template <typename T> __device__ __forceinline__ cx<T> cscale(cx<T> a, T s) { return cx<T>{a.x * s, a.y * s}; }
template <typename T> __device__ __forceinline__ T recip(T x) { return T(1) / x; }
template <> __device__ __forceinline__ float recip<float>(float x) { return __frcp_rn(x); }
template <typename T> __device__ __forceinline__ cx<T> cdiv(cx<T> a, cx<T> b)
{
    T d = recip<T>(b.x * b.x + b.y * b.y);
    return cx<T>{(a.x * b.x + a.y * b.y) * d, (a.y * b.x - a.x * b.y) * d};
}

// ---------------------------------------------------------------------------
// Scaled complex numbers: value = (x + i y) * 2^e with an exact integer
// binary exponent, so that products of hundreds of hidden-unit factors and
// sums over thousands of symmetry terms never leave the FP32 range and lose
// no absolute accuracy in log psi.
// ---------------------------------------------------------------------------
template <typename T> struct sc { T x, y; int e; };

template <typename T> __device__ __forceinline__ T pow2i(int k);
template <> __device__ __forceinline__ float pow2i<float>(int k)
{
    if (k < -126) return 0.f;
    if (k > 127) k = 127;
    return __int_as_float((127 + k) << 23);
}
template <> __device__ __forceinline__ double pow2i<double>(int k)
{
    if (k < -1022) return 0.0;
    if (k > 1023) k = 1023;
    return __longlong_as_double((long long)(1023 + k) << 52);
}

// binary exponent of max(|x|,|y|) (0 for zero / non-finite inputs)
template <typename T> __device__ __forceinline__ int expo(T x, T y);
template <> __device__ __forceinline__ int expo<float>(float x, float y)
{
    float m = fmaxf(fabsf(x), fabsf(y));
    int b = (__float_as_int(m) >> 23) & 0xff;
    return (b == 0 || b == 0xff) ? 0 : b - 127;
}
template <> __device__ __forceinline__ int expo<double>(double x, double y)
{
    double m = fmax(fabs(x), fabs(y));
    int b = (int)((__double_as_longlong(m) >> 52) & 0x7ff);
    return (b == 0 || b == 0x7ff) ? 0 : b - 1023;
}

template <typename T> __device__ __forceinline__ sc<T> sc_norm(sc<T> v)
{
    int k = expo<T>(v.x, v.y);
    T s = pow2i<T>(-k);
    return sc<T>{v.x * s, v.y * s, v.e + k};
}
template <typename T> __device__ __forceinline__ sc<T> sc_mul(sc<T> a, sc<T> b)
{
    cx<T> p = cmul(mk(a.x, a.y), mk(b.x, b.y));
    return sc_norm(sc<T>{p.x, p.y, a.e + b.e});
}
template <typename T> __device__ __forceinline__ bool sc_zero(sc<T> a) { return a.x == T(0) && a.y == T(0); }
template <typename T> __device__ __forceinline__ bool sc_finite(sc<T> v) { return isfinite(v.x) && isfinite(v.y); }
__device__ __forceinline__ void flag_range(int *status) { atomicExch(status, -6); }

template <typename T> __device__ __forceinline__ sc<T> sc_add(sc<T> a, sc<T> b)
{
    if (sc_zero(b)) return a;
    if (sc_zero(a)) return b;
    if (b.e > a.e) { sc<T> t = a; a = b; b = t; }
    T s = pow2i<T>(b.e - a.e);
    return sc_norm(sc<T>{a.x + b.x * s, a.y + b.y * s, a.e});
}

template <typename T> __device__ __forceinline__ T shfl_x(T v, int lane_mask)
{
    return __shfl_xor_sync(0xffffffffu, v, lane_mask);
}
// product over the 32 lanes of a warp (every lane receives it)
template <typename T> __device__ __forceinline__ sc<T> warp_prod(sc<T> v)
{
    v = sc_norm(v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sc<T> w{shfl_x(v.x, o), shfl_x(v.y, o), __shfl_xor_sync(0xffffffffu, v.e, o)};
        v = sc_mul(v, w);
    }
    return v;
}
template <typename T> __device__ __forceinline__ sc<T> warp_sum_sc(sc<T> v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sc<T> w{shfl_x(v.x, o), shfl_x(v.y, o), __shfl_xor_sync(0xffffffffu, v.e, o)};
        v = sc_add(v, w);
    }
    return v;
}
template <typename T> __device__ __forceinline__ cx<T> warp_sum(cx<T> v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) { v.x += shfl_x(v.x, o); v.y += shfl_x(v.y, o); }
    return v;
}

// product of a scaled number and a double complex, as a scaled double
__device__ __forceinline__ sc<double> sd_mul(sc<float> a, double bx, double by)
{
    const double x = (double)a.x * bx - (double)a.y * by, y = (double)a.x * by + (double)a.y * bx;
    return sc_norm(sc<double>{x, y, a.e});
}

// a scaled number as a double complex
__device__ __forceinline__ void sc_to_d(sc<float> a, double &x, double &y)
{
    const double f = pow2i<double>(a.e);
    x = (double)a.x * f;
    y = (double)a.y * f;
}

// product over the GL lanes of an aligned lane group (every lane receives it)
template <int GL> __device__ __forceinline__ sc<float> group_prod(sc<float> v)
{
    v = sc_norm(v);
#pragma unroll
    for (int o = GL / 2; o > 0; o >>= 1) {
        const sc<float> w{shfl_x(v.x, o), shfl_x(v.y, o), __shfl_xor_sync(0xffffffffu, v.e, o)};
        v = sc_mul(v, w);
    }
    return v;
}

// (x, y) <- mantissa of max(|x|, |y|) in [1, 2); returns the binary exponent.
// Exponent bits only: zero stays zero (exponent -127), a non-finite input
// stays non-finite.
__device__ __forceinline__ int nrm(float &x, float &y)
{
    const uint32_t bits = __float_as_uint(fmaxf(fabsf(x), fabsf(y))) & 0x7f800000u;
    const float s = __uint_as_float(0x7f000000u - bits);
    x *= s;
    y *= s;
    return (int)(bits >> 23) - 127;
}

// exp(z) as a scaled number (exact exponent split of Re z)
template <typename T> __device__ __forceinline__ sc<T> sc_exp(cx<T> z)
{
    const T l2e = T(1.4426950408889634);
    T t = z.x * l2e;
    T k = floor(t);
    T m = exp2(t - k);
    T s, c;
    sincos(z.y, &s, &c);
    return sc<T>{m * c, m * s, (int)k};
}

// 2 cosh(theta) = mant * 2^k  together with  p = e^theta / (2 cosh theta).
// With u = |Re theta| and v = sign(Re theta) Im theta (cosh is even):
//   2 cosh = e^u [e^{iv} + e^{-2u} e^{-iv}] = 2^k e^f [cos v (1+q) + i sin v (1-q)]
// where u log2(e) = k + f, q = e^{-2u} <= 1; and e^{theta'}/(2cosh) =
// e^f e^{iv} / mant for theta' = sign(Re theta) theta, p(theta) = 1 - p(-theta).
template <typename T>
__device__ __forceinline__ void cosh2(cx<T> th, cx<T> &mant, int &k, cx<T> &p)
{
    const T l2e = T(1.4426950408889634);
    bool neg = th.x < T(0);
    T u = fabs(th.x);
    T v = neg ? -th.y : th.y;
    T t = u * l2e;
    T kf = floor(t);
    T ef = exp2(t - kf);
    T q = exp2(T(-2) * t);
    T sv, cv;
    sincos(v, &sv, &cv);
    mant = cx<T>{ef * cv * (T(1) + q), ef * sv * (T(1) - q)};
    k = (int)kf;
    cx<T> pp = cdiv(cx<T>{ef * cv, ef * sv}, mant);
    p = neg ? cx<T>{T(1) - pp.x, -pp.y} : pp;
}

// 2 cosh(theta) = mant * 2^k only (no p)
template <typename T> __device__ __forceinline__ void cosh2_mant(cx<T> th, cx<T> &mant, int &k)
{
    const T l2e = T(1.4426950408889634);
    const bool neg = th.x < T(0);
    const T u = fabs(th.x);
    const T v = neg ? -th.y : th.y;
    const T t = u * l2e;
    const T kf = floor(t);
    const T ef = exp2(t - kf);
    const T q = exp2(T(-2) * t);
    T sv, cv;
    sincos(v, &sv, &cv);
    mant = cx<T>{ef * cv * (T(1) + q), ef * sv * (T(1) - q)};
    k = (int)kf;
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)
struct u32x4 { uint32_t v[4]; };
__device__ __forceinline__ u32x4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    return u32x4{{c0, c1, c2, c3}};
}

// ---------------------------------------------------------------------------
// Device view of a model (passed by value to kernels)
// ---------------------------------------------------------------------------
// Tile variants of the connected-configuration engine: GL lanes per row x MPL
// hidden units per lane (width GL * MPL); the one used for a width M is the
// narrowest that holds it.
constexpr int kNumVariants = 7;
__host__ __device__ __forceinline__ int variant_width(int v)
{
    return v == 0 ? 16 : v == 1 ? 32 : v == 2 ? 72 : v == 3 ? 128 : v == 4 ? 256 : v == 5 ? 416 : 512;
}
__host__ __device__ __forceinline__ int default_variant(int M)
{
    int v = 0;
    while (v < kNumVariants - 1 && variant_width(v) < M) ++v;
    return v;
}
// Smallest row stride of the connected-configuration tables: M padded to the
// width of its variant, with neutral entries (T = 0, e^{+-4W} = 1) past M so
// that the inner loops need no bound.  A model may use a larger stride.
__host__ __device__ __forceinline__ int conn_mpad(int M) { return variant_width(default_variant(M)); }

// p = 1 Lanczos step from the normalised moments m1, m2, m3 (Sec. 3.3, Eqs.
// 15-17): the lowest eigenpair of H in span{psi0, psi1}.  out = {E, v, alpha}
// with v^2 = m2 - m1^2, d = (m3 - 3 m1 m2 + 2 m1^3) / (2 v^3),
// alpha = d - sqrt(d^2 + 1), E = m1 + v alpha; an exact eigenstate
// (v^2 <= 1e-14 m1^2) gives E = m1, alpha = 0.
__device__ __forceinline__ void lanczos_p1(double m1, double m2, double m3, double *out)
{
    const double v2 = m2 - m1 * m1;
    if (v2 <= 1e-14 * m1 * m1 || v2 <= 0.0) {
        out[0] = m1; out[1] = v2 > 0.0 ? sqrt(v2) : 0.0; out[2] = 0.0;
    } else {
        const double vv = sqrt(v2);
        const double d = (m3 - 3.0 * m1 * m2 + 2.0 * m1 * m1 * m1) / (2.0 * v2 * vv);
        const double al = d - sqrt(d * d + 1.0);
        out[0] = m1 + vv * al; out[1] = vv; out[2] = al;
    }
}

template <typename T> struct DevModel {
    int L, N, K, M, G, nsign, use_bias, nbonds, nwords, chiP;
    int Mp;                 // row stride of Tb and S4 (>= conn_mpad(M))
    T J1, J2;
    const uint8_t *perm;    // [G][N]   image of site i under g
    const T *chi;           // [G]      +-1
    const cx<T> *Wt;        // [K][N][M] transposed weights
    const cx<T> *bvec;      // [K][M]
    const cx<T> *avec;      // [K][N]
    const cx<T> *logc;      // [K]
    const cx2<T> *X;        // [K][N][M]  (exp(-2W_mk), exp(+2W_mk))
    const cx2<T> *XA;       // [K][N]     (exp(-2a_k),  exp(+2a_k))
    // connected-configuration tables (bond b' = (a, b) of the bond list,
    // D0_m = -2 (W_ma - W_mb) the change of theta_m when s_a = +1, s_b = -1
    // are exchanged):
    const cx<T> *Tb;        // [K][2][4N][Mp] exp(+2 D0_m) - 1, exp(-2 D0_m) - 1
    const cx<T> *Cb;        // [K][4N]        -2 (a_a - a_b) + 2 sum_m (W_ma - W_mb)
    const cx<T> *S4;        // [K][2][N][Mp]  exp(-4 W_mk), exp(+4 W_mk)
    const cx<T> *CS;        // [K][N]         sum_m W_mk
    const uint16_t *bperm;  // [G][4N]        image bond of b under g | (orientation flip << 15)
    const sc<T> *ES;        // [K][2][N]      exp(+-Cs_k), Cs_k = 2 sum_m W_mk - 2 a_k (site prefactors)
    const int16_t *bond_i;  // [4N]
    const int16_t *bond_j;  // [4N]
    const uint8_t *bond_t;  // [4N] 1 = J1, 2 = J2
    int *status;            // device status word
};

template <typename T> __device__ __forceinline__ T bondJ(const DevModel<T> &md, int b)
{
    return md.bond_t[b] == 1 ? md.J1 : md.J2;
}

__device__ __forceinline__ int spin_of(const uint64_t *w, int i) { return ((w[i >> 6] >> (i & 63)) & 1ull) ? 1 : -1; }

}  // namespace nnqs
