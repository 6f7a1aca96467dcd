// stout.cu -- stout smearing of the gauge links and the force chain rule through it (Sec. 2:
// the Dirac operator uses the k-times stout-smeared links U^(k); Sec. 3: the MD evolves U^(0),
// so the fermion force is pulled back through the k smearing steps).
//
// One step, per link (x, mu):  C = rho * (sum of the six staples around the link),
// i Q = TA(C U^dag), U' = exp(iQ) U.  exp(iQ) = f0 + f1 Q + f2 Q^2: Q^n reduces to
// a_n + b_n Q + c_n Q^2 by the Cayley-Hamilton identity Q^3 = c1 Q + c0 (c0 = det Q,
// c1 = tr Q^2 / 2, Q traceless Hermitian), so the f_j are the Taylor series of exp with
// scalar coefficient recursions -- no transcendental functions, and entire in (c0, c1), so the
// chain rule needs no special case at degenerate eigenvalues.  The recursion also carries
// d/dc0 and d/dc1 of the coefficients for the backward pass.
//
// Gradients follow torch's convention (G = dS/dRe U + i dS/dIm U, dS = Re tr(G^dag dU)).  The
// backward step is two kernels: k_stout_back_link (per link: the exp/TA/Omega part, writes the
// link's own gradient terms and Y = rho G_Omega U, the gradient of the unweighted staple sum)
// and k_stout_back_staples (per link: adds the product-rule terms of every staple of the other
// links' C that contains this link, gathered from Y -- each output is written by one thread).
//
// Layout: canonical complex128 [4][V][3][3] (site index x + Lx (y + Ly (z + Lz t))); one thread
// per link.  All arithmetic FP64 (GB300's FP64 rate bounds these kernels, not HBM).
#include <cmath>
#include <cstring>
#include <string>

#include "stg_common.h"
#include "su3.cuh"

namespace stg {
namespace {
using namespace su3;

// Weighted staple sum C_mu(x) = rho * sum_{nu != mu} (upper + lower staple).
template <typename T>
__device__ M3T<T> staple_sum(const typename C2<T>::type *__restrict__ U, const LinkGeo &g, int mu, long long i,
                             T rho)
{
    M3T<T> c = zero3<T>();
#pragma unroll 1
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        M3T<T> a, b, t;
        // U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag
        ld(U, g, nu, i, a);
        ld(U, g, mu, nb(g, i, nu, 1), b);
        t = mul<false, false>(a, b);
        ld(U, g, nu, nb(g, i, mu, 1), a);
        mul_acc<false, true>(c, t, a);
        // U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu)
        const long long xm = nb(g, i, nu, -1);
        ld(U, g, nu, xm, a);
        ld(U, g, mu, xm, b);
        t = mul<true, false>(a, b);
        ld(U, g, nu, nb(g, xm, mu, 1), a);
        mul_acc<false, false>(c, t, a);
    }
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) c.m[r][k] = cx<T>{rho * c.m[r][k].re, rho * c.m[r][k].im};
    return c;
}

// Q = -i TA(C U^dag) and its square; returns nothing else
template <typename T>
__device__ __forceinline__ void make_q(const M3T<T> &C, const M3T<T> &u, M3T<T> &q, M3T<T> &q2)
{
    const M3T<T> a = ta(mul<false, true>(C, u));  // = i Q
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) q.m[r][c] = cx<T>{a.m[r][c].im, -a.m[r][c].re};
    q2 = mul<false, false>(q, q);
}

template <typename T>
struct StoutArgs {
    using C = typename C2<T>::type;
    LinkGeo g;
    T rho;
    const C *U;  // links of this step
    const C *G;  // gradient of the step's output (backward)
    C *out;      // smeared links (forward) / gradient of U (backward)
    C *Y;        // rho G_Omega U (backward)
};

constexpr int kStoutBlock = 128;

template <typename T>
__global__ void __launch_bounds__(kStoutBlock) k_stout_fwd(const __grid_constant__ StoutArgs<T> a)
{
    const int mu = blockIdx.y;
    const long long i = (long long)blockIdx.x * kStoutBlock + threadIdx.x;
    if (i >= a.g.V) return;
    M3T<T> q, q2, u;
    {
        const M3T<T> C = staple_sum(a.U, a.g, mu, i, a.rho);
        ld(a.U, a.g, mu, i, u);
        make_q(C, u, q, q2);
    }
    T c0, c1;
    char_coefs(q, q2, c0, c1);
    const ExpCoefT<T> e = exp_coef<false>(c0, c1);
    const M3T<T> E = poly3(e.f, q, q2);
    st(a.out, a.g, mu, i, mul<false, false>(E, u));
}

template <typename T>
__global__ void __launch_bounds__(kStoutBlock) k_stout_back_link(const __grid_constant__ StoutArgs<T> a)
{
    const int mu = blockIdx.y;
    const long long i = (long long)blockIdx.x * kStoutBlock + threadIdx.x;
    if (i >= a.g.V) return;
    M3T<T> u, q, q2, gp;
    const M3T<T> C = staple_sum(a.U, a.g, mu, i, a.rho);
    ld(a.U, a.g, mu, i, u);
    make_q(C, u, q, q2);
    T c0, c1;
    char_coefs(q, q2, c0, c1);
    const ExpCoefT<T> e = exp_coef<true>(c0, c1);
    ld(a.G, a.g, mu, i, gp);
    // the link's own terms: E^dag G' (later + G_Omega^dag C)
    M3T<T> gu = mul<true, false>(poly3(e.f, q, q2), gp);
    const M3T<T> M = mul<false, true>(gp, u);  // gradient of E
    // Tr_j = tr(M^dag Q^j);  K = sum_j Re(T_j df_j/dc)
    cx<T> Tr[3] = {cx<T>{T(0), T(0)}, cx<T>{T(0), T(0)}, cx<T>{T(0), T(0)}};
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        Tr[0] = cx<T>{Tr[0].re + M.m[r][r].re, Tr[0].im - M.m[r][r].im};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            cmac_conj(Tr[1], M.m[k][r], q.m[k][r]);
            cmac_conj(Tr[2], M.m[k][r], q2.m[k][r]);
        }
    }
    T K0 = T(0), K1 = T(0);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        K0 += Tr[j].re * e.d0[j].re - Tr[j].im * e.d0[j].im;
        K1 += Tr[j].re * e.d1[j].re - Tr[j].im * e.d1[j].im;
    }
    // G_Q = K1 Q + K0 Q^2 + conj(f1) M + conj(f2) (M Q + Q M)
    M3T<T> gq = mul<false, false>(M, q);
    mul_acc<false, false>(gq, q, M);
    const cx<T> f1c = cconj(e.f[1]), f2c = cconj(e.f[2]);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            cx<T> v = cmul(f2c, gq.m[r][c]);
            cmac(v, f1c, M.m[r][c]);
            v.re += K1 * q.m[r][c].re + K0 * q2.m[r][c].re;
            v.im += K1 * q.m[r][c].im + K0 * q2.m[r][c].im;
            gq.m[r][c] = cx<T>{-v.im, v.re};  // i G_Q
        }
    const M3T<T> go = ta(gq);  // G_Omega
    mul_acc<true, false>(gu, go, C);
    st(a.out, a.g, mu, i, gu);
    M3T<T> y = mul<false, false>(go, u);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) y.m[r][c] = cx<T>{a.rho * y.m[r][c].re, a.rho * y.m[r][c].im};
    st(a.Y, a.g, mu, i, y);
}

// Adds to the gradient of link (y, nu) the staple terms: for every mu != nu, the link sits in
//   C_mu(y)       as the first factor of the upper staple      -> Y_mu(y) U_nu(y+mu) U_mu(y+nu)^dag
//   C_mu(y+nu)    as the first factor of the lower staple      -> U_mu(y) U_nu(y+mu) Y_mu(y+nu)^dag
//   C_nu(y+mu)    as the middle factor of the lower staple     -> U_mu(y) Y_nu(y+mu) U_mu(y+nu)^dag
//   C_mu(y-mu)    as the last factor of the upper staple       -> Y_mu(y-mu)^dag U_nu(y-mu) U_mu(y-mu+nu)
//   C_mu(y-mu+nu) as the last factor of the lower staple       -> U_mu(y-mu)^dag U_nu(y-mu) Y_mu(y-mu+nu)
//   C_nu(y-mu)    as the middle factor of the upper staple     -> U_mu(y-mu)^dag Y_nu(y-mu) U_mu(y-mu+nu)
// with Y the gradient of the unweighted staple sums.
template <typename T>
__global__ void __launch_bounds__(kStoutBlock) k_stout_back_staples(const __grid_constant__ StoutArgs<T> a)
{
    const int nu = blockIdx.y;
    const long long i = (long long)blockIdx.x * kStoutBlock + threadIdx.x;
    if (i >= a.g.V) return;
    M3T<T> acc;
    ld(a.out, a.g, nu, i, acc);
#pragma unroll 1
    for (int mu = 0; mu < 4; ++mu) {
        if (mu == nu) continue;
        const long long yp = nb(a.g, i, mu, 1), yn = nb(a.g, i, nu, 1);
        const long long ym = nb(a.g, i, mu, -1), ymn = nb(a.g, ym, nu, 1);
        M3T<T> p, q, t;
        // forward side: U_nu(y+mu) shared by the first two terms
        ld(a.U, a.g, nu, yp, p);   // U_nu(y+mu)
        ld(a.U, a.g, mu, yn, q);   // U_mu(y+nu)
        t = mul<false, true>(p, q);
        ld(a.Y, a.g, mu, i, q);    // Y_mu(y)
        mul_acc<false, false>(acc, q, t);
        ld(a.U, a.g, mu, i, q);    // U_mu(y)
        t = mul<false, false>(q, p);
        ld(a.Y, a.g, mu, yn, p);   // Y_mu(y+nu)
        mul_acc<false, true>(acc, t, p);
        ld(a.Y, a.g, nu, yp, p);   // Y_nu(y+mu)
        t = mul<false, false>(q, p);
        ld(a.U, a.g, mu, yn, q);   // U_mu(y+nu)
        mul_acc<false, true>(acc, t, q);
        // backward side: U_mu(y-mu)^dag leads the last two terms
        ld(a.U, a.g, nu, ym, p);   // U_nu(y-mu)
        ld(a.U, a.g, mu, ymn, q);  // U_mu(y-mu+nu)
        t = mul<false, false>(p, q);
        ld(a.Y, a.g, mu, ym, q);   // Y_mu(y-mu)
        mul_acc<true, false>(acc, q, t);
        ld(a.Y, a.g, mu, ymn, q);  // Y_mu(y-mu+nu)
        t = mul<false, false>(p, q);
        ld(a.Y, a.g, nu, ym, p);   // Y_nu(y-mu)
        ld(a.U, a.g, mu, ymn, q);  // U_mu(y-mu+nu)
        mul_acc<false, false>(t, p, q);
        ld(a.U, a.g, mu, ym, p);   // U_mu(y-mu)
        mul_acc<true, false>(acc, p, t);
    }
    st(a.out, a.g, nu, i, acc);
}

// F = TA(U G^dag) in place over G
template <typename T>
__global__ void __launch_bounds__(kStoutBlock) k_lie_force(const __grid_constant__ StoutArgs<T> a)
{
    const int mu = blockIdx.y;
    const long long i = (long long)blockIdx.x * kStoutBlock + threadIdx.x;
    if (i >= a.g.V) return;
    M3T<T> u, gr;
    ld(a.U, a.g, mu, i, u);
    ld(a.out, a.g, mu, i, gr);
    st(a.out, a.g, mu, i, ta(mul<false, true>(u, gr)));
}

stg_status check_common(const stg_lattice *lat, int nstep, double rho, const char *fn)
{
    const std::string f(fn);
    if (!lat) return set_error(STG_ERR_ARG, f + ": null lattice");
    if (nstep < 1 || nstep > 16) return set_error(STG_ERR_ARG, f + ": nstep must be in 1..16");
    if (!(fabs(rho) <= 0.5)) return set_error(STG_ERR_ARG, f + ": |rho| must be <= 0.5");
    return STG_OK;
}

bool misaligned(const void *p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 15) != 0; }

template <typename T>
cudaError_t smear_t(const LinkGeo &g, int nstep, double rho, const void *links, void *levels, cudaStream_t st)
{
    using C = typename C2<T>::type;
    StoutArgs<T> a;
    memset(&a, 0, sizeof(a));
    a.g = g;
    a.rho = (T)rho;
    const size_t level = (size_t)4 * g.V * 9;  // complex numbers per level
    const dim3 grid((unsigned)((g.V + kStoutBlock - 1) / kStoutBlock), 4);
    for (int k = 0; k < nstep; ++k) {
        a.U = k == 0 ? static_cast<const C *>(links) : static_cast<const C *>(levels) + (size_t)(k - 1) * level;
        a.out = static_cast<C *>(levels) + (size_t)k * level;
        k_stout_fwd<T><<<grid, kStoutBlock, 0, st>>>(a);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename T>
cudaError_t force_t(const LinkGeo &g, int nstep, double rho, const void *links, const void *levels, const void *grad,
                    void *out_v, int kind, cudaStream_t st)
{
    using C = typename C2<T>::type;
    StoutArgs<T> a;
    memset(&a, 0, sizeof(a));
    a.g = g;
    a.rho = (T)rho;
    const size_t level = (size_t)4 * g.V * 9;
    C *ws = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&ws, 2 * level * sizeof(C), st);
    if (e != cudaSuccess) return e;
    C *Y = ws, *tmp = ws + level, *out = static_cast<C *>(out_v);
    const dim3 grid((unsigned)((g.V + kStoutBlock - 1) / kStoutBlock), 4);
    const C *g_in = static_cast<const C *>(grad);
    for (int k = nstep - 1; k >= 0 && e == cudaSuccess; --k) {
        // the last step (k = 0) lands in out; earlier ones alternate so that it does
        C *dst = (k % 2 == 0) ? out : tmp;
        a.U = k == 0 ? static_cast<const C *>(links) : static_cast<const C *>(levels) + (size_t)(k - 1) * level;
        a.G = g_in;
        a.out = dst;
        a.Y = Y;
        k_stout_back_link<T><<<grid, kStoutBlock, 0, st>>>(a);
        k_stout_back_staples<T><<<grid, kStoutBlock, 0, st>>>(a);
        e = cudaGetLastError();
        g_in = dst;
    }
    if (e == cudaSuccess && kind == 0) {
        a.U = static_cast<const C *>(links);
        a.out = out;
        k_lie_force<T><<<grid, kStoutBlock, 0, st>>>(a);
        e = cudaGetLastError();
    }
    const cudaError_t f = cudaFreeAsync(ws, st);
    return e != cudaSuccess ? e : f;
}

}  // namespace
}  // namespace stg

using namespace stg;

extern "C" stg_status stg_stout_smear(const stg_lattice *lat, stg_prec prec, int32_t nstep, double rho,
                                      const void *links_dev, void *levels_dev, void *stream)
{
    if (lat && stg::geom_is_slab(lat->g))
        return stg::set_error(STG_ERR_SHAPE, "stg_stout_smear: not available on a slab lattice (stg_dslash* only)");
    stg_status s = check_common(lat, nstep, rho, "stg_stout_smear");
    if (s != STG_OK) return s;
    if (prec != STG_F64 && prec != STG_F32) return set_error(STG_ERR_ARG, "stg_stout_smear: prec must be F64 or F32");
    if (misaligned(links_dev) || misaligned(levels_dev))
        return set_error(STG_ERR_ARG, "stg_stout_smear: buffers must be non-null and 16-byte aligned");
    const LinkGeo g = link_geo(lat->g);
    cudaStream_t st = (cudaStream_t)stream;
    STG_CUDA_TRY(prec == STG_F64 ? smear_t<double>(g, nstep, rho, links_dev, levels_dev, st)
                                 : smear_t<float>(g, nstep, rho, links_dev, levels_dev, st));
    return STG_OK;
}

extern "C" stg_status stg_stout_force(const stg_lattice *lat, stg_prec prec, int32_t nstep, double rho,
                                      const void *links_dev, const void *levels_dev, const void *grad_dev,
                                      void *out_dev, int32_t kind, void *stream)
{
    if (lat && stg::geom_is_slab(lat->g))
        return stg::set_error(STG_ERR_SHAPE, "stg_stout_force: not available on a slab lattice (stg_dslash* only)");
    stg_status s = check_common(lat, nstep, rho, "stg_stout_force");
    if (s != STG_OK) return s;
    if (prec != STG_F64 && prec != STG_F32) return set_error(STG_ERR_ARG, "stg_stout_force: prec must be F64 or F32");
    if (misaligned(links_dev) || misaligned(grad_dev) || misaligned(out_dev) || (nstep > 1 && misaligned(levels_dev)))
        return set_error(STG_ERR_ARG, "stg_stout_force: buffers must be non-null and 16-byte aligned");
    if (kind != 0 && kind != 1) return set_error(STG_ERR_ARG, "stg_stout_force: kind must be 0 or 1");
    if (out_dev == grad_dev || out_dev == links_dev)
        return set_error(STG_ERR_ARG, "stg_stout_force: out must not alias the inputs");
    const LinkGeo g = link_geo(lat->g);
    cudaStream_t st = (cudaStream_t)stream;
    STG_CUDA_TRY(prec == STG_F64 ? force_t<double>(g, nstep, rho, links_dev, levels_dev, grad_dev, out_dev, kind, st)
                                 : force_t<float>(g, nstep, rho, links_dev, levels_dev, grad_dev, out_dev, kind, st));
    return STG_OK;
}
