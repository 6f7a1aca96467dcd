// su3.cuh -- FP64 3x3 complex matrices in registers, for the kernels that work on whole links
// in the canonical complex128 layout [4][V][3][3] (stout smearing, gauge action and force, MD
// link updates): loads/stores, products with optional daggers, the traceless anti-Hermitian
// projection, lexicographic neighbours, and exp(iQ) of a traceless Hermitian Q as
// f0 + f1 Q + f2 Q^2 (with the derivatives of the f_j for chain rules).
#pragma once

#include "stg_internal.cuh"

namespace stg {
namespace su3 {

struct M3 {
    cx<double> m[3][3];
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

__device__ __forceinline__ void ld(const double2 *__restrict__ base, const LinkGeo &g, int mu, long long i, M3 &a)
{
    const double2 *p = base + ((long long)mu * g.V + i) * 9;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const double2 v = p[k];
        a.m[k / 3][k % 3] = cx<double>{v.x, v.y};
    }
}

__device__ __forceinline__ void st(double2 *__restrict__ base, const LinkGeo &g, int mu, long long i, const M3 &a)
{
    double2 *p = base + ((long long)mu * g.V + i) * 9;
#pragma unroll
    for (int k = 0; k < 9; ++k) p[k] = make_double2(a.m[k / 3][k % 3].re, a.m[k / 3][k % 3].im);
}

// element (r, c) of a or of a^dag
template <bool D>
__device__ __forceinline__ cx<double> el(const M3 &a, int r, int c)
{
    return D ? cconj(a.m[c][r]) : a.m[r][c];
}

// acc (+)= op(a) op(b)
template <bool DA, bool DB>
__device__ __forceinline__ void mul_acc(M3 &acc, const M3 &a, const M3 &b)
{
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int k = 0; k < 3; ++k) cmac(acc.m[r][c], el<DA>(a, r, k), el<DB>(b, k, c));
}

template <bool DA, bool DB>
__device__ __forceinline__ M3 mul(const M3 &a, const M3 &b)
{
    M3 z;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) z.m[r][c] = cx<double>{0.0, 0.0};
    mul_acc<DA, DB>(z, a, b);
    return z;
}

__device__ __forceinline__ M3 zero3()
{
    M3 z;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) z.m[r][c] = cx<double>{0.0, 0.0};
    return z;
}

// TA(X) = (X - X^dag)/2 - tr(X - X^dag)/6
__device__ __forceinline__ M3 ta(const M3 &x)
{
    M3 y;
    const double im_tr = (x.m[0][0].im + x.m[1][1].im + x.m[2][2].im) / 3.0;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            y.m[r][c] = cx<double>{0.5 * (x.m[r][c].re - x.m[c][r].re), 0.5 * (x.m[r][c].im + x.m[c][r].im)};
            if (r == c) y.m[r][c].im -= im_tr;
        }
    return y;
}

// f_j of exp(iQ) = f0 + f1 Q + f2 Q^2 and (DERIV) df_j/dc0, df_j/dc1.
struct ExpCoef {
    cx<double> f[3], d0[3], d1[3];
};

template <bool DERIV>
__device__ ExpCoef exp_coef(double c0, double c1)
{
    ExpCoef e;
#pragma unroll
    for (int j = 0; j < 3; ++j) e.f[j] = e.d0[j] = e.d1[j] = cx<double>{0.0, 0.0};
    e.f[0].re = 1.0;  // n = 0
    double a = 1.0, b = 0.0, c = 0.0;                        // Q^n = a + b Q + c Q^2
    double a0 = 0.0, b0 = 0.0, cc0 = 0.0, a1 = 0.0, b1 = 0.0, cc1 = 0.0;  // d/dc0, d/dc1
    const double r = fmax(sqrt(fmax(2.0 * c1, 0.0)), 1.0);  // >= spectral radius of Q, >= 1
    double w = 1.0, bound = 1.0;                             // 1/n!, r^n/n!
#pragma unroll 1
    for (int n = 1; n < 128; ++n) {
        if (DERIV) {
            const double na0 = c + c0 * cc0, nb0 = a0 + c1 * cc0, nc0 = b0;
            const double na1 = c0 * cc1, nb1 = a1 + c + c1 * cc1, nc1 = b1;
            a0 = na0; b0 = nb0; cc0 = nc0; a1 = na1; b1 = nb1; cc1 = nc1;
        }
        const double na = c0 * c, nb = a + c1 * c, nc = b;
        a = na; b = nb; c = nc;
        w /= n;
        bound *= r / n;
        // i^n / n!
        const double s = (n & 2) ? -w : w;
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
        // remaining terms of the coefficients (and of their c-derivatives, polynomial in n
        // times r^n/n!) are below FP64 resolution
        const double m = (double)(n + 1);
        if (n >= 6 && bound * m * m * m < 1e-18) break;
    }
    return e;
}

// c0 = det Q, c1 = tr Q^2 / 2 of a Hermitian Q (both real)
__device__ __forceinline__ void char_coefs(const M3 &q, const M3 &q2, double &c0, double &c1)
{
    c1 = 0.5 * (q2.m[0][0].re + q2.m[1][1].re + q2.m[2][2].re);
    // det = q00 (q11 q22 - q12 q21) - q01 (q10 q22 - q12 q20) + q02 (q10 q21 - q11 q20)
    cx<double> t = cmul(q.m[1][1], q.m[2][2]), u = cmul(q.m[1][2], q.m[2][1]);
    const cx<double> d = cmul(q.m[0][0], cx<double>{t.re - u.re, t.im - u.im});
    t = cmul(q.m[1][0], q.m[2][2]); u = cmul(q.m[1][2], q.m[2][0]);
    const cx<double> e1 = cmul(q.m[0][1], cx<double>{t.re - u.re, t.im - u.im});
    t = cmul(q.m[1][0], q.m[2][1]); u = cmul(q.m[1][1], q.m[2][0]);
    const cx<double> e2 = cmul(q.m[0][2], cx<double>{t.re - u.re, t.im - u.im});
    c0 = d.re - e1.re + e2.re;
}

// E = f0 + f1 Q + f2 Q^2
__device__ __forceinline__ M3 poly3(const cx<double> f[3], const M3 &q, const M3 &q2)
{
    M3 e;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            cx<double> v = cmul(f[1], q.m[r][c]);
            cmac(v, f[2], q2.m[r][c]);
            if (r == c) { v.re += f[0].re; v.im += f[0].im; }
            e.m[r][c] = v;
        }
    return e;
}


}  // namespace su3
}  // namespace stg
