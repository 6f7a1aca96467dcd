// su3.cuh -- 3x3 complex matrices in registers (T = double or float), for the kernels that work on
// whole links in the canonical layout [4][V][3][3] (complex128, or complex64 for the FP32 variants
// of the MD kernels): loads/stores, products with optional daggers, the traceless anti-Hermitian
// projection, lexicographic neighbours, and exp(iQ) of a traceless Hermitian Q as
// f0 + f1 Q + f2 Q^2 (with the derivatives of the f_j for chain rules).
#pragma once

#include "stg_internal.cuh"

namespace stg {
namespace su3 {

template <typename T>
struct M3T {
    cx<T> m[3][3];
};
using M3 = M3T<double>;

// storage type of one complex number of precision T
template <typename T>
struct C2;
template <>
struct C2<double> {
    using type = double2;
};
template <>
struct C2<float> {
    using type = float2;
};

struct LinkGeo {
    int L[4];
    long long stride[4];
    long long V;
};

inline LinkGeo link_geo(const Geom &geo)
{
    LinkGeo g;
    long long s = 1;
    for (int mu = 0; mu < 4; ++mu) {
        g.L[mu] = geo.L[mu];
        g.stride[mu] = s;
        s *= g.L[mu];
    }
    g.V = s;
    return g;
}

// lexicographic index of x + step * mu (periodic; |step| <= L_mu)
__device__ __forceinline__ long long nb(const LinkGeo &g, long long i, int mu, int step)
{
    const int xm = (int)((i / g.stride[mu]) % g.L[mu]);
    long long j = i + step * g.stride[mu];
    if (xm + step >= g.L[mu]) j -= g.L[mu] * g.stride[mu];
    if (xm + step < 0) j += g.L[mu] * g.stride[mu];
    return j;
}

template <typename T>
__device__ __forceinline__ void ld(const typename C2<T>::type *__restrict__ base, const LinkGeo &g, int mu, long long i,
                                   M3T<T> &a)
{
    const typename C2<T>::type *p = base + ((long long)mu * g.V + i) * 9;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const typename C2<T>::type v = p[k];
        a.m[k / 3][k % 3] = cx<T>{v.x, v.y};
    }
}

template <typename T>
__device__ __forceinline__ void st(typename C2<T>::type *__restrict__ base, const LinkGeo &g, int mu, long long i,
                                   const M3T<T> &a)
{
    typename C2<T>::type *p = base + ((long long)mu * g.V + i) * 9;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        p[k].x = a.m[k / 3][k % 3].re;
        p[k].y = a.m[k / 3][k % 3].im;
    }
}

// element (r, c) of a or of a^dag
template <bool D, typename T>
__device__ __forceinline__ cx<T> el(const M3T<T> &a, int r, int c)
{
    return D ? cconj(a.m[c][r]) : a.m[r][c];
}

// acc (+)= op(a) op(b)
template <bool DA, bool DB, typename T>
__device__ __forceinline__ void mul_acc(M3T<T> &acc, const M3T<T> &a, const M3T<T> &b)
{
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int k = 0; k < 3; ++k) cmac(acc.m[r][c], el<DA>(a, r, k), el<DB>(b, k, c));
}

template <typename T = double>
__device__ __forceinline__ M3T<T> zero3()
{
    M3T<T> z;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) z.m[r][c] = cx<T>{T(0), T(0)};
    return z;
}

template <bool DA, bool DB, typename T>
__device__ __forceinline__ M3T<T> mul(const M3T<T> &a, const M3T<T> &b)
{
    M3T<T> z = zero3<T>();
    mul_acc<DA, DB>(z, a, b);
    return z;
}

// TA(X) = (X - X^dag)/2 - tr(X - X^dag)/6
template <typename T>
__device__ __forceinline__ M3T<T> ta(const M3T<T> &x)
{
    M3T<T> y;
    const T im_tr = (x.m[0][0].im + x.m[1][1].im + x.m[2][2].im) / T(3);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            y.m[r][c] = cx<T>{T(0.5) * (x.m[r][c].re - x.m[c][r].re), T(0.5) * (x.m[r][c].im + x.m[c][r].im)};
            if (r == c) y.m[r][c].im -= im_tr;
        }
    return y;
}

// f_j of exp(iQ) = f0 + f1 Q + f2 Q^2 and (DERIV) df_j/dc0, df_j/dc1.
template <typename T>
struct ExpCoefT {
    cx<T> f[3], d0[3], d1[3];
};
using ExpCoef = ExpCoefT<double>;

template <bool DERIV, typename T>
__device__ ExpCoefT<T> exp_coef(T c0, T c1)
{
    ExpCoefT<T> e;
#pragma unroll
    for (int j = 0; j < 3; ++j) e.f[j] = e.d0[j] = e.d1[j] = cx<T>{T(0), T(0)};
    e.f[0].re = T(1);  // n = 0
    T a = T(1), b = T(0), c = T(0);                                     // Q^n = a + b Q + c Q^2
    T a0 = T(0), b0 = T(0), cc0 = T(0), a1 = T(0), b1 = T(0), cc1 = T(0);  // d/dc0, d/dc1
    T r = sqrt(fmax(T(2) * c1, T(0)));                                  // >= spectral radius of Q
    if (r < T(1)) r = T(1);
    // remaining terms of the coefficients (and of their c-derivatives, polynomial in n times
    // r^n/n!) below the precision's resolution
    const T stop = sizeof(T) == 4 ? T(1e-9) : T(1e-18);
    T w = T(1), bound = T(1);                                            // 1/n!, r^n/n!
#pragma unroll 1
    for (int n = 1; n < 128; ++n) {
        if (DERIV) {
            const T na0 = c + c0 * cc0, nb0 = a0 + c1 * cc0, nc0 = b0;
            const T na1 = c0 * cc1, nb1 = a1 + c + c1 * cc1, nc1 = b1;
            a0 = na0; b0 = nb0; cc0 = nc0; a1 = na1; b1 = nb1; cc1 = nc1;
        }
        const T na = c0 * c, nb = a + c1 * c, nc = b;
        a = na; b = nb; c = nc;
        w /= T(n);
        bound *= r / T(n);
        // i^n / n!
        const T s = (n & 2) ? -w : w;
        if (n & 1) {
            e.f[0].im += s * a; e.f[1].im += s * b; e.f[2].im += s * c;
            if (DERIV) {
                e.d0[0].im += s * a0; e.d0[1].im += s * b0; e.d0[2].im += s * cc0;
                e.d1[0].im += s * a1; e.d1[1].im += s * b1; e.d1[2].im += s * cc1;
            }
        } else {
            e.f[0].re += s * a; e.f[1].re += s * b; e.f[2].re += s * c;
            if (DERIV) {
                e.d0[0].re += s * a0; e.d0[1].re += s * b0; e.d0[2].re += s * cc0;
                e.d1[0].re += s * a1; e.d1[1].re += s * b1; e.d1[2].re += s * cc1;
            }
        }
        const T m = T(n + 1);
        if (n >= 6 && bound * m * m * m < stop) break;
    }
    return e;
}

// c0 = det Q, c1 = tr Q^2 / 2 of a Hermitian Q (both real)
template <typename T>
__device__ __forceinline__ void char_coefs(const M3T<T> &q, const M3T<T> &q2, T &c0, T &c1)
{
    c1 = T(0.5) * (q2.m[0][0].re + q2.m[1][1].re + q2.m[2][2].re);
    // det = q00 (q11 q22 - q12 q21) - q01 (q10 q22 - q12 q20) + q02 (q10 q21 - q11 q20)
    cx<T> t = cmul(q.m[1][1], q.m[2][2]), u = cmul(q.m[1][2], q.m[2][1]);
    const cx<T> d = cmul(q.m[0][0], cx<T>{t.re - u.re, t.im - u.im});
    t = cmul(q.m[1][0], q.m[2][2]); u = cmul(q.m[1][2], q.m[2][0]);
    const cx<T> e1 = cmul(q.m[0][1], cx<T>{t.re - u.re, t.im - u.im});
    t = cmul(q.m[1][0], q.m[2][1]); u = cmul(q.m[1][1], q.m[2][0]);
    const cx<T> e2 = cmul(q.m[0][2], cx<T>{t.re - u.re, t.im - u.im});
    c0 = d.re - e1.re + e2.re;
}

// E = f0 + f1 Q + f2 Q^2
template <typename T>
__device__ __forceinline__ M3T<T> poly3(const cx<T> f[3], const M3T<T> &q, const M3T<T> &q2)
{
    M3T<T> e;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            cx<T> v = cmul(f[1], q.m[r][c]);
            cmac(v, f[2], q2.m[r][c]);
            if (r == c) { v.re += f[0].re; v.im += f[0].im; }
            e.m[r][c] = v;
        }
    return e;
}

}  // namespace su3
}  // namespace stg
