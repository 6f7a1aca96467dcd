// gauge.cu -- the tree-level Symanzik gauge action S_g and its force (Sec. 2: S_g is built from
// the traces of 1x1 plaquettes and 1x2 rectangles of the unsmeared links; Sec. 3: the gauge term
// of the MD force needs the products of links along those loops, the "staples").
//
//   S_g = -(beta/3) sum_x sum_{mu != nu} [ c0 Re tr P_{mu nu}(x) + c1 Re tr R_{mu nu}(x) ]
//   c0 = 5/6, c1 = -1/12 (tree-level coefficients; ordered pairs: each plaquette twice, each
//   2x1 rectangle once), links periodic in all four directions.
//
// Force: for the link U_mu(x) every loop through it reads Re tr(U_mu(x) B) with B the rest of the
// loop, so G = dS/dRe U + i dS/dIm U = -(beta/3) sum c B^dag; B^dag is the "staple".  Per link:
// 2 plaquette staples (weight 2 c0) and 6 rectangle staples (weight c1) per direction nu != mu.
// Output kind 1: G; kind 0: F = TA(U G^dag) (dS/deps = tr(X F) along U -> exp(eps X) U).
//
// One thread per link (force) or per site (action), canonical complex128 [4][V][3][3], FP64
// (the staples are 84 complex 3x3 products per link: GB300's FP64 rate bounds this, not HBM).
#include <cmath>
#include <cstring>

#include "stg_common.h"
#include "su3.cuh"

namespace stg {
namespace {
using namespace su3;

constexpr double kC0 = 5.0 / 6.0, kC1 = -1.0 / 12.0;
constexpr int kGaugeBlock = 128;

template <typename T>
struct GaugeArgs {
    using C = typename C2<T>::type;
    LinkGeo g;
    double beta;
    const C *U;
    C *out;
    int kind;
    double *partial;  // action: [2][nblocks] (plaquette sums, rectangle sums)
    double *out3;     // action: S_g, plaquette sum, rectangle sum
    int nblocks;
};

template <typename T>
__device__ __forceinline__ M3T<T> lk(const typename C2<T>::type *__restrict__ U, const LinkGeo &g, int d,
                                     long long site)
{
    M3T<T> m;
    ld(U, g, d, site, m);
    return m;
}

// acc += w * op(a) op(b)
template <bool DA, bool DB, typename T>
__device__ __forceinline__ void mul_acc_w(M3T<T> &acc, T w, const M3T<T> &a, const M3T<T> &b)
{
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            cx<T> z = cx<T>{T(0), T(0)};
#pragma unroll
            for (int k = 0; k < 3; ++k) cmac(z, el<DA>(a, r, k), el<DB>(b, k, c));
            acc.m[r][c].re = fma(w, z.re, acc.m[r][c].re);
            acc.m[r][c].im = fma(w, z.im, acc.m[r][c].im);
        }
}

// Re tr(a b)
__device__ __forceinline__ double retr_mul(const M3 &a, const M3 &b)
{
    double s = 0.0;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) s += a.m[r][k].re * b.m[k][r].re - a.m[r][k].im * b.m[k][r].im;
    return s;
}

// One block per SM as the bound keeps ptxas from a low register target and heavy spills (FP32 with
// three blocks per SM spilled and ran 18.5 ms instead of 15.2 ms at 48^4)
template <typename T>
__global__ void __launch_bounds__(kGaugeBlock, 1) k_gauge_force(const __grid_constant__ GaugeArgs<T> a)
{
    const int mu = blockIdx.y;
    const long long x = (long long)blockIdx.x * kGaugeBlock + threadIdx.x;
    if (x >= a.g.V) return;
    const LinkGeo g = a.g;
    const typename C2<T>::type *__restrict__ Ub = a.U;
    // G = -(beta/3) (2 c0 sum of plaquette staples + c1 sum of rectangle staples)
    const T wp = T(-a.beta / 3.0 * 2.0 * kC0), wr = T(-a.beta / 3.0 * kC1);
    M3T<T> G = zero3<T>();
    const long long xpm = nb(g, x, mu, 1), xmm = nb(g, x, mu, -1), xp2m = nb(g, xpm, mu, 1);
#pragma unroll 1
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        const long long xpn = nb(g, x, nu, 1), xmn = nb(g, x, nu, -1);
        const long long xpm_pn = nb(g, xpm, nu, 1), xpm_mn = nb(g, xpm, nu, -1);
        M3T<T> t;
        // plaquette staples: U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag and U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu)
        t = mul<false, false>(lk<T>(Ub, g, nu, x), lk<T>(Ub, g, mu, xpn));
        mul_acc_w<false, true>(G, wp, t, lk<T>(Ub, g, nu, xpm));
        t = mul<true, false>(lk<T>(Ub, g, nu, xmn), lk<T>(Ub, g, mu, xmn));
        mul_acc_w<false, false>(G, wp, t, lk<T>(Ub, g, nu, xpm_mn));
        // r1: U_nu(x) U_mu(x+nu) U_mu(x+mu+nu) U_nu(x+2mu)^dag U_mu(x+mu)^dag
        t = mul<false, false>(lk<T>(Ub, g, nu, x), lk<T>(Ub, g, mu, xpn));
        t = mul<false, false>(t, lk<T>(Ub, g, mu, xpm_pn));
        t = mul<false, true>(t, lk<T>(Ub, g, nu, xp2m));
        mul_acc_w<false, true>(G, wr, t, lk<T>(Ub, g, mu, xpm));
        // r2: U_mu(x-mu)^dag U_nu(x-mu) U_mu(x-mu+nu) U_mu(x+nu) U_nu(x+mu)^dag
        const long long xmm_pn = nb(g, xmm, nu, 1), xmm_mn = nb(g, xmm, nu, -1);
        t = mul<true, false>(lk<T>(Ub, g, mu, xmm), lk<T>(Ub, g, nu, xmm));
        t = mul<false, false>(t, lk<T>(Ub, g, mu, xmm_pn));
        t = mul<false, false>(t, lk<T>(Ub, g, mu, xpn));
        mul_acc_w<false, true>(G, wr, t, lk<T>(Ub, g, nu, xpm));
        // r3: U_nu(x-nu)^dag U_mu(x-nu) U_mu(x+mu-nu) U_nu(x+2mu-nu) U_mu(x+mu)^dag
        t = mul<true, false>(lk<T>(Ub, g, nu, xmn), lk<T>(Ub, g, mu, xmn));
        t = mul<false, false>(t, lk<T>(Ub, g, mu, xpm_mn));
        t = mul<false, false>(t, lk<T>(Ub, g, nu, nb(g, xp2m, nu, -1)));
        mul_acc_w<false, true>(G, wr, t, lk<T>(Ub, g, mu, xpm));
        // r4: U_mu(x-mu)^dag U_nu(x-mu-nu)^dag U_mu(x-mu-nu) U_mu(x-nu) U_nu(x+mu-nu)
        t = mul<true, true>(lk<T>(Ub, g, mu, xmm), lk<T>(Ub, g, nu, xmm_mn));
        t = mul<false, false>(t, lk<T>(Ub, g, mu, xmm_mn));
        t = mul<false, false>(t, lk<T>(Ub, g, mu, xmn));
        mul_acc_w<false, false>(G, wr, t, lk<T>(Ub, g, nu, xpm_mn));
        // r5: U_nu(x) U_nu(x+nu) U_mu(x+2nu) U_nu(x+mu+nu)^dag U_nu(x+mu)^dag
        t = mul<false, false>(lk<T>(Ub, g, nu, x), lk<T>(Ub, g, nu, xpn));
        t = mul<false, false>(t, lk<T>(Ub, g, mu, nb(g, xpn, nu, 1)));
        t = mul<false, true>(t, lk<T>(Ub, g, nu, xpm_pn));
        mul_acc_w<false, true>(G, wr, t, lk<T>(Ub, g, nu, xpm));
        // r6: U_nu(x-nu)^dag U_nu(x-2nu)^dag U_mu(x-2nu) U_nu(x+mu-2nu) U_nu(x+mu-nu)
        const long long xm2n = nb(g, xmn, nu, -1);
        t = mul<true, true>(lk<T>(Ub, g, nu, xmn), lk<T>(Ub, g, nu, xm2n));
        t = mul<false, false>(t, lk<T>(Ub, g, mu, xm2n));
        t = mul<false, false>(t, lk<T>(Ub, g, nu, nb(g, xpm_mn, nu, -1)));
        mul_acc_w<false, false>(G, wr, t, lk<T>(Ub, g, nu, xpm_mn));
    }
    if (a.kind == 0) G = ta(mul<false, true>(lk<T>(Ub, g, mu, x), G));
    st(a.out, g, mu, x, G);
}

__global__ void __launch_bounds__(kGaugeBlock, 1) k_gauge_action(const __grid_constant__ GaugeArgs<double> a)
{
    __shared__ double sh[33];
    const long long x = (long long)blockIdx.x * kGaugeBlock + threadIdx.x;
    const LinkGeo g = a.g;
    const double2 *__restrict__ Ub = a.U;
    double ps = 0.0, rs = 0.0;
    if (x < g.V) {
#pragma unroll 1
        for (int mu = 0; mu < 4; ++mu) {
            const long long xpm = nb(g, x, mu, 1);
#pragma unroll 1
            for (int nu = mu + 1; nu < 4; ++nu) {
                const long long xpn = nb(g, x, nu, 1);
                // P = U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
                M3 t = mul<false, false>(lk<double>(Ub, g, mu, x), lk<double>(Ub, g, nu, xpm));
                M3 w = mul<true, true>(lk<double>(Ub, g, mu, xpn), lk<double>(Ub, g, nu, x));
                ps += retr_mul(t, w);
                // R_{mu nu} = U_mu(x) U_mu(x+mu) U_nu(x+2mu) U_mu(x+mu+nu)^dag U_mu(x+nu)^dag U_nu(x)^dag
                t = mul<false, false>(lk<double>(Ub, g, mu, x), lk<double>(Ub, g, mu, xpm));
                t = mul<false, false>(t, lk<double>(Ub, g, nu, nb(g, xpm, mu, 1)));
                w = mul<true, true>(lk<double>(Ub, g, mu, nb(g, xpm, nu, 1)), lk<double>(Ub, g, mu, xpn));
                w = mul<false, true>(w, lk<double>(Ub, g, nu, x));
                rs += retr_mul(t, w);
                // R_{nu mu} = U_nu(x) U_nu(x+nu) U_mu(x+2nu) U_nu(x+nu+mu)^dag U_nu(x+mu)^dag U_mu(x)^dag
                t = mul<false, false>(lk<double>(Ub, g, nu, x), lk<double>(Ub, g, nu, xpn));
                t = mul<false, false>(t, lk<double>(Ub, g, mu, nb(g, xpn, nu, 1)));
                w = mul<true, true>(lk<double>(Ub, g, nu, nb(g, xpn, mu, 1)), lk<double>(Ub, g, nu, xpm));
                w = mul<false, true>(w, lk<double>(Ub, g, mu, x));
                rs += retr_mul(t, w);
            }
        }
    }
    ps = block_sum(ps, sh);
    __syncthreads();
    rs = block_sum(rs, sh);
    if (threadIdx.x == 0) {
        a.partial[blockIdx.x] = ps;
        a.partial[a.nblocks + blockIdx.x] = rs;
    }
}

// fixed-order sum of the block partials by one block; writes S_g, plaquette sum, rectangle sum
__global__ void __launch_bounds__(256) k_gauge_action_finish(const __grid_constant__ GaugeArgs<double> a)
{
    __shared__ double sh[33];
    double ps = 0.0, rs = 0.0;
    for (int k = threadIdx.x; k < a.nblocks; k += blockDim.x) {
        ps += a.partial[k];
        rs += a.partial[a.nblocks + k];
    }
    ps = block_sum(ps, sh);
    __syncthreads();
    rs = block_sum(rs, sh);
    if (threadIdx.x == 0) {
        // sum over ordered pairs: each plaquette twice (ps counts it once), each rectangle once
        a.out3[0] = -a.beta / 3.0 * (2.0 * kC0 * ps + kC1 * rs);
        a.out3[1] = ps;
        a.out3[2] = rs;
    }
}

bool misaligned(const void *p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 15) != 0; }

}  // namespace
}  // namespace stg

using namespace stg;

template <typename T>
static cudaError_t gauge_force_t(const stg_lattice *lat, double beta, const void *links, void *out, int kind,
                                 cudaStream_t st)
{
    GaugeArgs<T> a;
    memset(&a, 0, sizeof(a));
    a.g = link_geo(lat->g);
    a.beta = beta;
    a.U = static_cast<const typename C2<T>::type *>(links);
    a.out = static_cast<typename C2<T>::type *>(out);
    a.kind = kind;
    const dim3 grid((unsigned)((a.g.V + kGaugeBlock - 1) / kGaugeBlock), 4);
    k_gauge_force<T><<<grid, kGaugeBlock, 0, st>>>(a);
    return cudaGetLastError();
}

extern "C" stg_status stg_gauge_force(const stg_lattice *lat, stg_prec prec, double beta, const void *links_dev,
                                      void *out_dev, int32_t kind, void *stream)
{
    if (lat && stg::geom_is_slab(lat->g))
        return stg::set_error(STG_ERR_SHAPE, "stg_gauge_force: not available on a slab lattice (stg_dslash* only)");
    if (!lat) return set_error(STG_ERR_ARG, "stg_gauge_force: null lattice");
    if (prec != STG_F64 && prec != STG_F32) return set_error(STG_ERR_ARG, "stg_gauge_force: prec must be F64 or F32");
    if (misaligned(links_dev) || misaligned(out_dev))
        return set_error(STG_ERR_ARG, "stg_gauge_force: buffers must be non-null and 16-byte aligned");
    if (out_dev == links_dev) return set_error(STG_ERR_ARG, "stg_gauge_force: out must not alias the links");
    if (kind != 0 && kind != 1) return set_error(STG_ERR_ARG, "stg_gauge_force: kind must be 0 or 1");
    if (!std::isfinite(beta)) return set_error(STG_ERR_ARG, "stg_gauge_force: beta must be finite");
    cudaStream_t st = (cudaStream_t)stream;
    STG_CUDA_TRY(prec == STG_F64 ? gauge_force_t<double>(lat, beta, links_dev, out_dev, kind, st)
                                 : gauge_force_t<float>(lat, beta, links_dev, out_dev, kind, st));
    return STG_OK;
}

extern "C" stg_status stg_gauge_action(const stg_lattice *lat, double beta, const void *links_c128_dev, double *out3_dev,
                                       void *stream)
{
    if (lat && stg::geom_is_slab(lat->g))
        return stg::set_error(STG_ERR_SHAPE, "stg_gauge_action: not available on a slab lattice (stg_dslash* only)");
    if (!lat) return set_error(STG_ERR_ARG, "stg_gauge_action: null lattice");
    if (misaligned(links_c128_dev)) return set_error(STG_ERR_ARG, "stg_gauge_action: links must be non-null and 16-byte aligned");
    if (!out3_dev || (reinterpret_cast<uintptr_t>(out3_dev) & 7))
        return set_error(STG_ERR_ARG, "stg_gauge_action: out3 must be non-null and 8-byte aligned");
    if (!std::isfinite(beta)) return set_error(STG_ERR_ARG, "stg_gauge_action: beta must be finite");
    cudaStream_t st = (cudaStream_t)stream;
    GaugeArgs<double> a;
    memset(&a, 0, sizeof(a));
    a.g = link_geo(lat->g);
    a.beta = beta;
    a.U = static_cast<const double2 *>(links_c128_dev);
    a.out3 = out3_dev;
    a.nblocks = (int)((a.g.V + kGaugeBlock - 1) / kGaugeBlock);
    STG_CUDA_TRY(cudaMallocAsync((void **)&a.partial, 2 * sizeof(double) * a.nblocks, st));
    k_gauge_action<<<a.nblocks, kGaugeBlock, 0, st>>>(a);
    k_gauge_action_finish<<<1, 256, 0, st>>>(a);
    const cudaError_t e = cudaGetLastError();
    cudaFreeAsync(a.partial, st);
    STG_CUDA_TRY(e);
    return STG_OK;
}
