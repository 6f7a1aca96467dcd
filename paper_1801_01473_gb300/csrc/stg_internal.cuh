// stg_internal.cuh -- device-side building blocks of the staggered hot path:
// complex arithmetic, internal field and link layouts, lattice geometry.
//
// Layouts (all structure-of-arrays over the Vh sites of one parity, so a warp
// reading 32 consecutive half indices issues fully coalesced 8- or 16-byte loads):
//   F64 field   3 x Vh double2 (one array per colour)                       48 B/site
//   F32 field   Vh float4 (colours 0,1) then Vh float2 (colour 2)           24 B/site
//   links       [mu][parity][chunks over Vh] per (precision, compression):
//     F64/18    9 x Vh double2      U00 U01 U02 U10 U11 U12 U20 U21 U22      144 B
//     F64/12    6 x Vh double2      rows 0 and 1                             96 B
//     F32/18    4 x Vh float4 + Vh float2 (U00U01 U02U10 U11U12 U20U21, U22)  72 B
//     F32/12    3 x Vh float4       (U00U01 U02U10 U11U12)                   48 B
//     16/12     Vh x 8 halves + Vh x 4 halves (U00..U10, U11 U12)            24 B
// Row 3 of a 12-real link is rebuilt as (r1 x r2)^* (link compression, Sec. 4.1).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace stg {

constexpr int kMaxShifts = 32;

// ------------------------------------------------------------------ complex

template <typename R>
struct cx {
    R re, im;
};

template <typename R>
__device__ __forceinline__ cx<R> cmk(R a, R b) { return cx<R>{a, b}; }

// acc += a * b
template <typename R>
__device__ __forceinline__ void cmac(cx<R> &acc, const cx<R> &a, const cx<R> &b)
{
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(-a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(a.im, b.re, acc.im);
}

// acc += conj(a) * b
template <typename R>
__device__ __forceinline__ void cmac_conj(cx<R> &acc, const cx<R> &a, const cx<R> &b)
{
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(-a.im, b.re, acc.im);
}

template <typename R>
__device__ __forceinline__ cx<R> cmul(const cx<R> &a, const cx<R> &b)
{
    return cx<R>{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}

template <typename R>
__device__ __forceinline__ cx<R> cconj(const cx<R> &a) { return cx<R>{a.re, -a.im}; }

// conj(a b - c d) as one chain of a product and three multiply-adds per real part
template <typename R>
__device__ __forceinline__ cx<R> conj_cross(const cx<R> &a, const cx<R> &b, const cx<R> &c, const cx<R> &d)
{
    const R re = fma(a.re, b.re, fma(-a.im, b.im, fma(-c.re, d.re, c.im * d.im)));
    const R im = fma(-a.re, b.im, fma(-a.im, b.re, fma(c.re, d.im, c.im * d.re)));
    return cx<R>{re, im};
}

// third row of an SU(3) matrix from the first two: r3 = (r1 x r2)^*
template <typename R>
__device__ __forceinline__ void reconstruct_row3(cx<R> U[3][3])
{
    U[2][0] = conj_cross(U[0][1], U[1][2], U[0][2], U[1][1]);
    U[2][1] = conj_cross(U[0][2], U[1][0], U[0][0], U[1][2]);
    U[2][2] = conj_cross(U[0][0], U[1][1], U[0][1], U[1][0]);
}

// ------------------------------------------------------------------ FP64 <-> FP32 on the integer pipes
// GB300 executes FP64 <-> FP32 conversions on its narrow FP64 unit (~2 per clock per SM), which
// makes plain conversion loops FP64-bound at a fraction of HBM bandwidth.  For normal numbers both
// directions are bit manipulations of the IEEE 754 binary64 / binary32 formats (sign, biased
// exponent 1023 / 127, 52 / 23 fraction bits); these do them on the integer pipes, rounding to
// nearest even, and leave zeros, subnormals, infinities and NaNs (and results in those ranges) to
// the hardware conversion.  Results are bit-identical to __double2float_rn and (double)f.
__device__ __forceinline__ float f64_to_f32_rn(double d)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const unsigned top = (unsigned)(b >> 32);
    const int e = (int)((top >> 20) & 0x7ffu) - 896;  // binary32 biased exponent
    if (e <= 0 || e >= 255) return __double2float_rn(d);
    const unsigned long long m = b & 0xfffffffffffffull;
    unsigned r = ((unsigned)e << 23) | (unsigned)(m >> 29);
    const unsigned rem = (unsigned)(m & 0x1fffffffu);  // the 29 dropped fraction bits
    r += (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) ? 1u : 0u;  // carries into the exponent
    return __uint_as_float(r | (top & 0x80000000u));
}

__device__ __forceinline__ double f32_to_f64(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) return (double)f;
    const unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                                 ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)b);
}

// ------------------------------------------------------------------ double-single numbers
// A value hi + lo held in two floats with |lo| <= ulp(hi)/2: a 48-bit significand (relative
// rounding ~2^-47) computed on the FP32 pipes, which GB300 runs ~64x faster than FP64.
// Sums use Knuth's TwoSum and Dekker's Fast2Sum, products the FMA form of Dekker's
// TwoProduct (Dekker 1971, "A floating-point technique for extending the available
// precision"; Knuth, TAOCP vol. 2, 4.2.2).  The _rn intrinsics keep the compiler from
// contracting or reassociating the error-free transformations.
struct dsf {
    float hi, lo;
    dsf() = default;
    __device__ __forceinline__ constexpr dsf(float h, float l) : hi(h), lo(l) {}
    __device__ __forceinline__ dsf(int i) : hi((float)i), lo(0.f) {}
    __device__ __forceinline__ explicit dsf(float f) : hi(f), lo(0.f) {}
    // hi = RN(d), lo = RN(d - hi): d - hi is the exact integer remainder of the 53-bit significand
    // after rounding it to 24 bits, scaled by the last place of d (integer pipes; the hardware
    // conversions for exponents outside the range where both parts are normal floats)
    __device__ __forceinline__ explicit dsf(double d)
    {
        const unsigned long long b = (unsigned long long)__double_as_longlong(d);
        const unsigned top = (unsigned)(b >> 32);
        const int e = (int)((top >> 20) & 0x7ffu) - 896;
        if (e < 53 || e >= 254) {
            hi = __double2float_rn(d);
            lo = __double2float_rn(d - (double)hi);
            return;
        }
        const long long sig = (long long)((b & 0xfffffffffffffull) | 0x10000000000000ull);  // 53 bits
        const unsigned rem = (unsigned)(sig & 0x1fffffff);
        long long m24 = sig >> 29;
        m24 += (rem > 0x10000000u || (rem == 0x10000000u && (m24 & 1))) ? 1 : 0;
        const unsigned sign = top & 0x80000000u;
        hi = __uint_as_float(((unsigned)(e << 23) + (unsigned)(m24 - (1ll << 23))) | sign);
        const int low = (int)(sig - (m24 << 29));  // |low| <= 2^28
        const float scale = __uint_as_float((unsigned)(e - 52) << 23);  // 2^(exponent of d's last place)
        lo = __fmul_rn(__int2float_rn(sign ? -low : low), scale);
    }
    __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
    __device__ __forceinline__ explicit operator float() const { return __fadd_rn(hi, lo); }
};

__device__ __forceinline__ dsf ds_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return dsf(s, e);
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ dsf ds_fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return dsf(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ dsf operator-(const dsf &a) { return dsf(-a.hi, -a.lo); }

__device__ __forceinline__ dsf operator+(const dsf &a, const dsf &b)
{
    const dsf s = ds_two_sum(a.hi, b.hi);
    return ds_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ dsf operator-(const dsf &a, const dsf &b) { return a + (-b); }

__device__ __forceinline__ dsf operator*(const dsf &a, const dsf &b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return ds_fast_two_sum(p, e);
}

// a * b + c  (the float/double overloads of fma stay visible inside this namespace)
using ::fma;
__device__ __forceinline__ dsf fma(const dsf &a, const dsf &b, const dsf &c)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const dsf s = ds_two_sum(p, c.hi);
    return ds_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(e, c.lo)));
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over a warp of a double-single value (xor butterfly: every lane ends with the same sum).
__device__ __forceinline__ dsf warp_sum_ds(dsf v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = v + dsf(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
    return v;
}

// Accumulator of products of two values of type R for the FP64 partial sums (<p,q>, |r|^2):
// FP64 for double; for float and double-single a double-single sum of the exact products
// (rounding ~2^-44 per operation) reduced over the warp on the FP32 pipes, with one conversion
// to FP64 per warp.  GB300 issues FP64 (and FP32<->FP64 conversion) ~64x slower than FP32, so
// converting every site's terms to FP64 made the FP32 vector kernels ALU-bound.
template <typename R>
struct ProdSum {
    double s = 0.0;
    __device__ __forceinline__ void add(R a, R b) { s = fma((double)a, (double)b, s); }
    __device__ __forceinline__ double warp_total() const { return warp_sum(s); }
};
template <>
struct ProdSum<float> {
    dsf s = dsf(0.f, 0.f);
    __device__ __forceinline__ void add(float a, float b)
    {
        const float p = __fmul_rn(a, b);
        const float e = __fmaf_rn(a, b, -p);  // a b = p + e exactly
        const dsf t = ds_two_sum(p, s.hi);
        s = ds_fast_two_sum(t.hi, __fadd_rn(t.lo, __fadd_rn(e, s.lo)));
    }
    __device__ __forceinline__ double warp_total() const { return (double)warp_sum_ds(s); }
};
template <>
struct ProdSum<dsf> {
    dsf s = dsf(0.f, 0.f);
    __device__ __forceinline__ void add(const dsf &a, const dsf &b) { s = fma(a, b, s); }
    __device__ __forceinline__ double warp_total() const { return (double)warp_sum_ds(s); }
};

// ------------------------------------------------------------------ geometry

// Quotient n / d for 0 <= n < 2^31 by one multiply-high, one add and one shift, with (m, s)
// precomputed on the host for the invariant divisor d (Granlund and Montgomery, "Division by
// invariant integers using multiplication", PLDI 1994, Sec. 4): s = ceil(log2 d),
// m = floor(2^32 (2^s - d) / d) + 1 and n / d = (umulhi(m, n) + n) >> s; the sum stays below
// 2^32 because umulhi(m, n) < n < 2^31.  A runtime integer division costs ~20 instructions.
struct FastDiv {
    unsigned m;
    int s;
};

inline FastDiv make_fast_div(unsigned d)
{
    int s = 0;
    while ((1ull << s) < d) ++s;
    const unsigned long long m = ((1ull << 32) * ((1ull << s) - d)) / d + 1;
    return FastDiv{(unsigned)m, s};
}

__device__ __forceinline__ int fast_div(int n, const FastDiv &f)
{
    return (int)((__umulhi(f.m, (unsigned)n) + (unsigned)n) >> f.s);
}

struct Geom {
    int L[4];       // Lx Ly Lz Lt (of the stored lattice)
    int Vh;         // sites per parity (the stride of every field and link array)
    int antiperiodic;
    FastDiv div[3];  // by Lx / 2, Ly and Lz (geom_init)
    // Output half-index range of the D kernels, [h_begin, h_end): the whole parity on a full
    // lattice; the interior time slices on a slab, whose stored lattice carries halo slices.
    int h_begin, h_end;
    // global time of stored slice 0 and the global time extent (0 and Lt on a full lattice): the
    // antiperiodic sign sits on the t-links at global time Lt_glob - 1
    int t_off, Lt_glob;
};

// Fills the derived members of a Geom whose extents, Vh and antiperiodic flag are set (a full
// lattice: every site is an output, stored time = global time).
inline void geom_init(Geom &g)
{
    g.div[0] = make_fast_div((unsigned)(g.L[0] >> 1));
    g.div[1] = make_fast_div((unsigned)g.L[1]);
    g.div[2] = make_fast_div((unsigned)g.L[2]);
    g.h_begin = 0;
    g.h_end = g.Vh;
    g.t_off = 0;
    g.Lt_glob = g.L[3];
}

// Coordinates and lexicographic index of the site with half index h on parity par.
struct Site {
    int x, y, z, t;
    int i;  // lexicographic index
};

__device__ __forceinline__ Site site_of(const Geom &g, int par, int h)
{
    Site s;
    const int lxh = g.L[0] >> 1;
    const int r = fast_div(h, g.div[0]);
    const int xh = h - r * lxh;
    const int r2 = fast_div(r, g.div[1]);
    s.y = r - r2 * g.L[1];
    s.t = fast_div(r2, g.div[2]);
    s.z = r2 - s.t * g.L[2];
    int odd = (par + s.y + s.z + s.t) & 1;
    s.x = 2 * xh + odd;
    s.i = 2 * h + odd;
    return s;
}

// Half indices of the forward/backward neighbours along mu (periodic wrap), and
// the link phases u_mu(x) and u_mu(x-mu) of the forward and backward hops.
struct Hop {
    int hf, hb;
    float sf, sb;
};

__device__ __forceinline__ Hop hop_of(const Geom &g, const Site &s, int mu)
{
    Hop o;
    int c, L, stride;
    if (mu == 0) { c = s.x; L = g.L[0]; stride = 1; }
    else if (mu == 1) { c = s.y; L = g.L[1]; stride = g.L[0]; }
    else if (mu == 2) { c = s.z; L = g.L[2]; stride = g.L[0] * g.L[1]; }
    else { c = s.t; L = g.L[3]; stride = g.L[0] * g.L[1] * g.L[2]; }
    int f = (c == L - 1) ? s.i - (L - 1) * stride : s.i + stride;
    int b = (c == 0) ? s.i + (L - 1) * stride : s.i - stride;
    o.hf = f >> 1;
    o.hb = b >> 1;
    // staggered phase eta_mu(x) = (-1)^(x_0 + ... + x_{mu-1}); it does not depend on x_mu,
    // so the backward link (x - mu, mu) carries the same eta.
    int e = (mu == 0) ? 0 : (mu == 1) ? s.x : (mu == 2) ? (s.x + s.y) : (s.x + s.y + s.z);
    float eta = (e & 1) ? -1.f : 1.f;
    o.sf = eta;
    o.sb = eta;
    if (mu == 3 && g.antiperiodic) {
        const int tg = s.t + g.t_off;          // global time of the site
        if (tg == g.Lt_glob - 1) o.sf = -o.sf;  // forward link sits on x_t = Lt-1
        if (tg == 0) o.sb = -o.sb;              // backward link (x - t) sits on x_t = Lt-1
    }
    return o;
}

// ------------------------------------------------------------------ fields

template <typename R>
struct Field;

template <>
struct Field<double> {
    static constexpr int kBytesPerSite = 48;
    __device__ __forceinline__ static void load(const void *base, int Vh, int h, cx<double> v[3])
    {
        const double2 *p = static_cast<const double2 *>(base);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double2 d = __ldg(p + (size_t)c * Vh + h);
            v[c] = cx<double>{d.x, d.y};
        }
    }
    __device__ __forceinline__ static void store(void *base, int Vh, int h, const cx<double> v[3])
    {
        double2 *p = static_cast<double2 *>(base);
#pragma unroll
        for (int c = 0; c < 3; ++c) p[(size_t)c * Vh + h] = make_double2(v[c].re, v[c].im);
    }
    // plain (non-texture-path) load for buffers written earlier in the same kernel sequence
    __device__ __forceinline__ static void load_rw(const void *base, int Vh, int h, cx<double> v[3])
    {
        const double2 *p = static_cast<const double2 *>(base);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double2 d = p[(size_t)c * Vh + h];
            v[c] = cx<double>{d.x, d.y};
        }
    }
};

template <>
struct Field<float> {
    static constexpr int kBytesPerSite = 24;
    __device__ __forceinline__ static void load(const void *base, int Vh, int h, cx<float> v[3])
    {
        const float4 *a = static_cast<const float4 *>(base);
        const float2 *b = reinterpret_cast<const float2 *>(a + Vh);
        float4 u = __ldg(a + h);
        float2 w = __ldg(b + h);
        v[0] = cx<float>{u.x, u.y};
        v[1] = cx<float>{u.z, u.w};
        v[2] = cx<float>{w.x, w.y};
    }
    __device__ __forceinline__ static void store(void *base, int Vh, int h, const cx<float> v[3])
    {
        float4 *a = static_cast<float4 *>(base);
        float2 *b = reinterpret_cast<float2 *>(a + Vh);
        a[h] = make_float4(v[0].re, v[0].im, v[1].re, v[1].im);
        b[h] = make_float2(v[2].re, v[2].im);
    }
    __device__ __forceinline__ static void load_rw(const void *base, int Vh, int h, cx<float> v[3])
    {
        const float4 *a = static_cast<const float4 *>(base);
        const float2 *b = reinterpret_cast<const float2 *>(a + Vh);
        float4 u = a[h];
        float2 w = b[h];
        v[0] = cx<float>{u.x, u.y};
        v[1] = cx<float>{u.z, u.w};
        v[2] = cx<float>{w.x, w.y};
    }
};

// double-single field: 3 arrays of Vh float4 (re.hi, re.lo, im.hi, im.lo), 48 B/site
template <>
struct Field<dsf> {
    static constexpr int kBytesPerSite = 48;
    __device__ __forceinline__ static void load(const void *base, int Vh, int h, cx<dsf> v[3])
    {
        const float4 *p = static_cast<const float4 *>(base);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float4 d = __ldg(p + (size_t)c * Vh + h);
            v[c] = cx<dsf>{dsf(d.x, d.y), dsf(d.z, d.w)};
        }
    }
    __device__ __forceinline__ static void store(void *base, int Vh, int h, const cx<dsf> v[3])
    {
        float4 *p = static_cast<float4 *>(base);
#pragma unroll
        for (int c = 0; c < 3; ++c) p[(size_t)c * Vh + h] = make_float4(v[c].re.hi, v[c].re.lo, v[c].im.hi, v[c].im.lo);
    }
    __device__ __forceinline__ static void load_rw(const void *base, int Vh, int h, cx<dsf> v[3])
    {
        const float4 *p = static_cast<const float4 *>(base);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float4 d = p[(size_t)c * Vh + h];
            v[c] = cx<dsf>{dsf(d.x, d.y), dsf(d.z, d.w)};
        }
    }
};

// ------------------------------------------------------------------ links
// Each link type: real type R used for arithmetic, bytes per link, loader
// into a full 3x3 complex matrix, and a packer from a canonical 3x3 complex128.

struct LinkF64R18 {
    using R = double;
    static constexpr int kBytes = 144;
    __device__ __forceinline__ static void load(const void *blk, int Vh, int h, cx<double> U[3][3])
    {
        const double2 *p = static_cast<const double2 *>(blk);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            double2 d = __ldg(p + (size_t)k * Vh + h);
            U[k / 3][k % 3] = cx<double>{d.x, d.y};
        }
    }
    __device__ __forceinline__ static void pack(void *blk, int Vh, int h, const double2 *m)
    {
        double2 *p = static_cast<double2 *>(blk);
        for (int k = 0; k < 9; ++k) p[(size_t)k * Vh + h] = m[k];
    }
};

struct LinkF64R12 {
    using R = double;
    static constexpr int kBytes = 96;
    __device__ __forceinline__ static void load(const void *blk, int Vh, int h, cx<double> U[3][3])
    {
        const double2 *p = static_cast<const double2 *>(blk);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            double2 d = __ldg(p + (size_t)k * Vh + h);
            U[k / 3][k % 3] = cx<double>{d.x, d.y};
        }
        reconstruct_row3(U);
    }
    __device__ __forceinline__ static void pack(void *blk, int Vh, int h, const double2 *m)
    {
        double2 *p = static_cast<double2 *>(blk);
        for (int k = 0; k < 6; ++k) p[(size_t)k * Vh + h] = m[k];
    }
};

struct LinkF32R18 {
    using R = float;
    static constexpr int kBytes = 72;
    __device__ __forceinline__ static void load(const void *blk, int Vh, int h, cx<float> U[3][3])
    {
        const float4 *p = static_cast<const float4 *>(blk);
        const float2 *q = reinterpret_cast<const float2 *>(p + 4 * (size_t)Vh);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float4 d = __ldg(p + (size_t)k * Vh + h);
            U[(2 * k) / 3][(2 * k) % 3] = cx<float>{d.x, d.y};
            U[(2 * k + 1) / 3][(2 * k + 1) % 3] = cx<float>{d.z, d.w};
        }
        float2 e = __ldg(q + h);
        U[2][2] = cx<float>{e.x, e.y};
    }
    __device__ __forceinline__ static void pack(void *blk, int Vh, int h, const double2 *m)
    {
        float4 *p = static_cast<float4 *>(blk);
        float2 *q = reinterpret_cast<float2 *>(p + 4 * (size_t)Vh);
        for (int k = 0; k < 4; ++k)
            p[(size_t)k * Vh + h] = make_float4(f64_to_f32_rn(m[2 * k].x), f64_to_f32_rn(m[2 * k].y),
                                                f64_to_f32_rn(m[2 * k + 1].x), f64_to_f32_rn(m[2 * k + 1].y));
        q[h] = make_float2(f64_to_f32_rn(m[8].x), f64_to_f32_rn(m[8].y));
    }
};

struct LinkF32R12 {
    using R = float;
    static constexpr int kBytes = 48;
    __device__ __forceinline__ static void load(const void *blk, int Vh, int h, cx<float> U[3][3])
    {
        const float4 *p = static_cast<const float4 *>(blk);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float4 d = __ldg(p + (size_t)k * Vh + h);
            U[(2 * k) / 3][(2 * k) % 3] = cx<float>{d.x, d.y};
            U[(2 * k + 1) / 3][(2 * k + 1) % 3] = cx<float>{d.z, d.w};
        }
        reconstruct_row3(U);
    }
    __device__ __forceinline__ static void pack(void *blk, int Vh, int h, const double2 *m)
    {
        float4 *p = static_cast<float4 *>(blk);
        for (int k = 0; k < 3; ++k)
            p[(size_t)k * Vh + h] = make_float4(f64_to_f32_rn(m[2 * k].x), f64_to_f32_rn(m[2 * k].y),
                                                f64_to_f32_rn(m[2 * k + 1].x), f64_to_f32_rn(m[2 * k + 1].y));
    }
};

// 16-bit storage (bf16 or fp16) of the two first rows; arithmetic in FP32.
template <typename H>
struct Half;
template <>
struct Half<__nv_bfloat16> {
    __device__ __forceinline__ static float to_f(uint16_t b) { return __bfloat162float(__ushort_as_bfloat16(b)); }
    __device__ __forceinline__ static uint16_t from_d(double v) { return __bfloat16_as_ushort(__double2bfloat16(v)); }
};
template <>
struct Half<__half> {
    __device__ __forceinline__ static float to_f(uint16_t b) { return __half2float(__ushort_as_half(b)); }
    __device__ __forceinline__ static uint16_t from_d(double v) { return __half_as_ushort(__double2half(v)); }
};

template <typename H>
struct Link16R12 {
    using R = float;
    static constexpr int kBytes = 24;
    __device__ __forceinline__ static void load(const void *blk, int Vh, int h, cx<float> U[3][3])
    {
        const uint4 *p = static_cast<const uint4 *>(blk);
        const uint2 *q = reinterpret_cast<const uint2 *>(p + Vh);
        uint4 a = __ldg(p + h);
        uint2 b = __ldg(q + h);
        uint32_t w[6] = {a.x, a.y, a.z, a.w, b.x, b.y};
#pragma unroll
        for (int k = 0; k < 6; ++k)
            U[k / 3][k % 3] = cx<float>{Half<H>::to_f((uint16_t)(w[k] & 0xffffu)), Half<H>::to_f((uint16_t)(w[k] >> 16))};
        reconstruct_row3(U);
    }
    __device__ __forceinline__ static void pack(void *blk, int Vh, int h, const double2 *m)
    {
        uint32_t w[6];
        for (int k = 0; k < 6; ++k)
            w[k] = (uint32_t)Half<H>::from_d(m[k].x) | ((uint32_t)Half<H>::from_d(m[k].y) << 16);
        uint4 *p = static_cast<uint4 *>(blk);
        uint2 *q = reinterpret_cast<uint2 *>(p + Vh);
        p[h] = make_uint4(w[0], w[1], w[2], w[3]);
        q[h] = make_uint2(w[4], w[5]);
    }
};

// double-single links: one float4 (re.hi, re.lo, im.hi, im.lo) per complex entry
template <int NCHUNK>
struct LinkDS {
    using R = dsf;
    static constexpr int kBytes = 16 * NCHUNK;
    __device__ __forceinline__ static void load(const void *blk, int Vh, int h, cx<dsf> U[3][3])
    {
        const float4 *p = static_cast<const float4 *>(blk);
#pragma unroll
        for (int k = 0; k < NCHUNK; ++k) {
            float4 d = __ldg(p + (size_t)k * Vh + h);
            U[k / 3][k % 3] = cx<dsf>{dsf(d.x, d.y), dsf(d.z, d.w)};
        }
        if (NCHUNK == 6) reconstruct_row3(U);
    }
    __device__ __forceinline__ static void pack(void *blk, int Vh, int h, const double2 *m)
    {
        float4 *p = static_cast<float4 *>(blk);
        for (int k = 0; k < NCHUNK; ++k) {
            const dsf re(m[k].x), im(m[k].y);
            p[(size_t)k * Vh + h] = make_float4(re.hi, re.lo, im.hi, im.lo);
        }
    }
};
using LinkDSR18 = LinkDS<9>;
using LinkDSR12 = LinkDS<6>;

// Base of the (mu, parity) block of an internal link array.
// Phase factor exp(i theta) from its stored form: an angle (float: cos + i sin on line, the
// paper's trade of 4 bytes for ~15 FP32 flops) or the precomputed pair (cos, sin) (double2: FP64
// trigonometry costs more than the 16 bytes on GB300, whose FP64 rate is 1/64 of FP32).
template <typename R>
__device__ __forceinline__ cx<R> phase_of(float t)
{
    float sn, cs;
    sincosf(t, &sn, &cs);
    return cx<R>{R(cs), R(sn)};
}
template <typename R>
__device__ __forceinline__ cx<R> phase_of(double2 p)
{
    return cx<R>{R(p.x), R(p.y)};
}

// A link with a U(1) phase u = exp(i theta) (Sec. 4.1: each flavour's U(1) field -- imaginary
// chemical potential, background fields).  Inside each (mu, parity) block the base link's chunks
// are followed by one chunk of Vh phase entries of type T (float angle for FP32/16-bit links,
// double2 (cos, sin) for FP64 and double-single links).  load() returns the SU(3) link; the
// operator multiplies its products U v by phase() (and by the conjugate on the backward hop),
// 3 complex products per link instead of 9.  The staggered and boundary signs stay separate.
template <typename Base, typename T>
struct LinkU1 {
    using R = typename Base::R;
    using BaseLink = Base;
    using Theta = T;
    static constexpr int kBytes = Base::kBytes + (int)sizeof(T);
    __device__ __forceinline__ static const T *theta(const void *blk, int Vh)
    {
        return reinterpret_cast<const T *>(static_cast<const char *>(blk) + (size_t)Base::kBytes * Vh);
    }
    __device__ __forceinline__ static cx<R> phase(const void *blk, int Vh, int h)
    {
        return phase_of<R>(__ldg(theta(blk, Vh) + h));
    }
    __device__ __forceinline__ static void load(const void *blk, int Vh, int h, cx<R> U[3][3])
    {
        Base::load(blk, Vh, h, U);
    }
    __device__ __forceinline__ static void pack(void *blk, int Vh, int h, const double2 *m) { Base::pack(blk, Vh, h, m); }
};

// Base link type and phase of a (possibly phased) link type.
template <typename L>
struct LinkTraits {
    using Base = L;
    static constexpr bool kU1 = false;
    __device__ __forceinline__ static cx<typename L::R> phase(const void *, int, int)
    {
        return cx<typename L::R>{typename L::R(1), typename L::R(0)};
    }
};
template <typename B, typename T>
struct LinkTraits<LinkU1<B, T>> {
    using Base = B;
    static constexpr bool kU1 = true;
    __device__ __forceinline__ static cx<typename B::R> phase(const void *blk, int Vh, int h)
    {
        return LinkU1<B, T>::phase(blk, Vh, h);
    }
};

template <typename LinkT>
__device__ __forceinline__ const void *link_block(const void *links, int Vh, int mu, int par)
{
    return static_cast<const char *>(links) + (size_t)(mu * 2 + par) * Vh * LinkT::kBytes;
}

// ------------------------------------------------------------------ programmatic dependent launch
// Kernels launched with launch_pdl may start while the previous kernel of the stream is still
// draining: each block first lets the next kernel launch, then waits until every earlier grid of
// the stream has completed and its writes are visible, before touching global memory.  Without
// the launch attribute both instructions are no-ops.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ------------------------------------------------------------------ reductions


// Deterministic block sum (fixed tree); result valid in thread 0.  `sh` holds >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double *sh)
{
    v = warp_sum(v);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (wid == 0) {
        int nw = (blockDim.x + 31) >> 5;
        s = lane < nw ? sh[lane] : 0.0;
        s = warp_sum(s);
    }
    return s;
}

}  // namespace stg
