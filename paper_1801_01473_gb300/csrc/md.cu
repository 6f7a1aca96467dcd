// md.cu -- the per-link steps of the molecular dynamics evolution (Sec. 2: RHMC samples
// exp(-H^2/2 - S) with momenta H conjugate to the links; Sec. 3: each MD iteration computes the
// forces, evolves the momenta, then evolves the links -- "embarrassingly parallel" once the
// force is known).
//
// With U' = i H U and the Lie-algebra force F = TA(U G^dag) (dS/deps = tr(X F) along
// U -> exp(eps X) U), the Hamiltonian (1/2) sum tr H^2 + S is conserved by H' = -i F:
//   momenta:  H <- H - eps i F                     (stg_md_update_momenta)
//   links:    U <- exp(i eps H) U                  (stg_md_update_links)
//   heatbath: H = sum_a xi_a lambda_a / sqrt(2)    (stg_md_momenta; xi standard normal, passed in,
//             lambda_a the Gell-Mann matrices, so (1/2) tr H^2 = (1/2) sum xi_a^2)
//   kinetic:  (1/2) sum_links tr H^2              (stg_md_kinetic, fixed-order FP64 sum)
// exp(i eps H) uses the Cayley-Hamilton series of su3.cuh (FP64).  Canonical complex128 layout
// [4][V][3][3], one thread per link.
#include <cmath>
#include <algorithm>
#include <cstring>

#include "stg_common.h"
#include "su3.cuh"

namespace stg {
namespace {
using namespace su3;

constexpr int kMdBlock = 128;

struct MdArgs {
    long long nlink;  // 4 V
    double eps;
    const double *xi;
    const void *F;
    double2 *H;
    double2 *U;
    double *partial;
    double *out;
    int nblocks;
};

__device__ __forceinline__ void ldl(const double2 *__restrict__ p, long long l, M3 &a)
{
    p += l * 9;
#pragma unroll
    for (int k = 0; k < 9; ++k) a.m[k / 3][k % 3] = cx<double>{p[k].x, p[k].y};
}

__device__ __forceinline__ void stl(double2 *__restrict__ p, long long l, const M3 &a)
{
    p += l * 9;
#pragma unroll
    for (int k = 0; k < 9; ++k) p[k] = make_double2(a.m[k / 3][k % 3].re, a.m[k / 3][k % 3].im);
}

__global__ void __launch_bounds__(kMdBlock) k_md_momenta(const __grid_constant__ MdArgs a)
{
    const long long l = (long long)blockIdx.x * kMdBlock + threadIdx.x;
    if (l >= a.nlink) return;
    const double *x = a.xi + l * 8;
    const double s = 0.70710678118654752440;  // 1/sqrt(2)
    const double r3 = 0.57735026918962576451;  // 1/sqrt(3)
    M3 h;
    // sum_a xi_a lambda_a: the Gell-Mann matrices written out entry by entry
    h.m[0][0] = cx<double>{s * (x[2] + r3 * x[7]), 0.0};
    h.m[1][1] = cx<double>{s * (-x[2] + r3 * x[7]), 0.0};
    h.m[2][2] = cx<double>{s * (-2.0 * r3 * x[7]), 0.0};
    h.m[0][1] = cx<double>{s * x[0], -s * x[1]};
    h.m[1][0] = cx<double>{s * x[0], s * x[1]};
    h.m[0][2] = cx<double>{s * x[3], -s * x[4]};
    h.m[2][0] = cx<double>{s * x[3], s * x[4]};
    h.m[1][2] = cx<double>{s * x[5], -s * x[6]};
    h.m[2][1] = cx<double>{s * x[5], s * x[6]};
    stl(a.H, l, h);
}

__global__ void __launch_bounds__(kMdBlock) k_md_update_links(const __grid_constant__ MdArgs a)
{
    const long long l = (long long)blockIdx.x * kMdBlock + threadIdx.x;
    if (l >= a.nlink) return;
    M3 q, u;
    ldl(a.H, l, q);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) q.m[r][c] = cx<double>{a.eps * q.m[r][c].re, a.eps * q.m[r][c].im};
    // exp(iQ) of the Hermitian part (H is Hermitian and traceless up to rounding)
    const M3 q2 = mul<false, false>(q, q);
    double c0, c1;
    char_coefs(q, q2, c0, c1);
    const ExpCoef e = exp_coef<false>(c0, c1);
    ldl(a.U, l, u);
    stl(a.U, l, mul<false, false>(poly3(e.f, q, q2), u));
}

// elementwise over the 9 nlink complex entries (coalesced); FP32 forces widened on the integer pipes
__device__ __forceinline__ double widen(double v) { return v; }
__device__ __forceinline__ double widen(float v) { return f32_to_f64(v); }

template <typename C>
__global__ void __launch_bounds__(kMdBlock) k_md_update_momenta(const __grid_constant__ MdArgs a)
{
    const long long n = a.nlink * 9;
    const C *f = static_cast<const C *>(a.F);
    for (long long k = (long long)blockIdx.x * kMdBlock + threadIdx.x; k < n; k += (long long)gridDim.x * kMdBlock) {
        const C fv = f[k];
        double2 hv = a.H[k];
        // H - eps i F:  i (fr + i fi) = -fi + i fr
        hv.x = fma(a.eps, widen(fv.y), hv.x);
        hv.y = fma(-a.eps, widen(fv.x), hv.y);
        a.H[k] = hv;
    }
}

// complex128 <-> complex64 arrays (count complex numbers)
template <typename S, typename D>
__global__ void k_convert(long long n, const S *__restrict__ src, D *__restrict__ dst)
{
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const S v = src[k];
        D w;
        if constexpr (sizeof(v.x) == 8 && sizeof(w.x) == 4) {
            w.x = f64_to_f32_rn(v.x);
            w.y = f64_to_f32_rn(v.y);
        } else if constexpr (sizeof(v.x) == 4 && sizeof(w.x) == 8) {
            w.x = f32_to_f64(v.x);
            w.y = f32_to_f64(v.y);
        } else {
            w.x = v.x;
            w.y = v.y;
        }
        dst[k] = w;
    }
}

__global__ void __launch_bounds__(kMdBlock) k_md_kinetic(const __grid_constant__ MdArgs a)
{
    __shared__ double sh[33];
    const long long l = (long long)blockIdx.x * kMdBlock + threadIdx.x;
    double t = 0.0;
    if (l < a.nlink) {
        M3 h;
        ldl(a.H, l, h);
        // tr H^2 = sum_rc H_rc H_cr
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) t += h.m[r][c].re * h.m[c][r].re - h.m[r][c].im * h.m[c][r].im;
    }
    t = block_sum(t, sh);
    if (threadIdx.x == 0) a.partial[blockIdx.x] = t;
}

__global__ void __launch_bounds__(256) k_md_kinetic_finish(const __grid_constant__ MdArgs a)
{
    __shared__ double sh[33];
    double t = 0.0;
    for (int k = threadIdx.x; k < a.nblocks; k += blockDim.x) t += a.partial[k];
    t = block_sum(t, sh);
    if (threadIdx.x == 0) *a.out = 0.5 * t;
}

bool bad(const void *p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 15) != 0; }

MdArgs md_args(const stg_lattice *lat)
{
    MdArgs a;
    memset(&a, 0, sizeof(a));
    a.nlink = 4 * lat->V;
    return a;
}

unsigned md_grid(const MdArgs &a) { return (unsigned)((a.nlink + kMdBlock - 1) / kMdBlock); }

}  // namespace
}  // namespace stg

using namespace stg;

extern "C" stg_status stg_md_momenta(const stg_lattice *lat, const double *xi_dev, void *mom_c128_dev, void *stream)
{
    if (lat && stg::geom_is_slab(lat->g))
        return stg::set_error(STG_ERR_SHAPE, "stg_md_momenta: not available on a slab lattice (stg_dslash* only)");
    if (!lat || !xi_dev || (reinterpret_cast<uintptr_t>(xi_dev) & 7) || bad(mom_c128_dev))
        return set_error(STG_ERR_ARG, "stg_md_momenta: null or misaligned pointer");
    MdArgs a = md_args(lat);
    a.xi = xi_dev;
    a.H = static_cast<double2 *>(mom_c128_dev);
    k_md_momenta<<<md_grid(a), kMdBlock, 0, (cudaStream_t)stream>>>(a);
    STG_CUDA_TRY(cudaGetLastError());
    return STG_OK;
}

extern "C" stg_status stg_md_update_links(const stg_lattice *lat, double eps, const void *mom_c128_dev,
                                          void *links_c128_dev, void *stream)
{
    if (lat && stg::geom_is_slab(lat->g))
        return stg::set_error(STG_ERR_SHAPE, "stg_md_update_links: not available on a slab lattice (stg_dslash* only)");
    if (!lat || bad(mom_c128_dev) || bad(links_c128_dev))
        return set_error(STG_ERR_ARG, "stg_md_update_links: null or misaligned pointer");
    if (mom_c128_dev == links_c128_dev) return set_error(STG_ERR_ARG, "stg_md_update_links: momenta alias the links");
    if (!std::isfinite(eps) || fabs(eps) > 1.0)
        return set_error(STG_ERR_ARG, "stg_md_update_links: eps must be finite with |eps| <= 1");
    MdArgs a = md_args(lat);
    a.eps = eps;
    a.H = const_cast<double2 *>(static_cast<const double2 *>(mom_c128_dev));
    a.U = static_cast<double2 *>(links_c128_dev);
    k_md_update_links<<<md_grid(a), kMdBlock, 0, (cudaStream_t)stream>>>(a);
    STG_CUDA_TRY(cudaGetLastError());
    return STG_OK;
}

extern "C" stg_status stg_md_update_momenta(const stg_lattice *lat, stg_prec force_prec, double eps,
                                            const void *force_dev, void *mom_c128_dev, void *stream)
{
    if (lat && stg::geom_is_slab(lat->g))
        return stg::set_error(STG_ERR_SHAPE, "stg_md_update_momenta: not available on a slab lattice (stg_dslash* only)");
    if (!lat || bad(force_dev) || bad(mom_c128_dev))
        return set_error(STG_ERR_ARG, "stg_md_update_momenta: null or misaligned pointer");
    if (force_prec != STG_F64 && force_prec != STG_F32)
        return set_error(STG_ERR_ARG, "stg_md_update_momenta: force precision must be F64 or F32");
    if (!std::isfinite(eps)) return set_error(STG_ERR_ARG, "stg_md_update_momenta: eps must be finite");
    MdArgs a = md_args(lat);
    a.eps = eps;
    a.F = force_dev;
    a.H = static_cast<double2 *>(mom_c128_dev);
    if (force_prec == STG_F64)
        k_md_update_momenta<double2><<<md_grid(a), kMdBlock, 0, (cudaStream_t)stream>>>(a);
    else
        k_md_update_momenta<float2><<<md_grid(a), kMdBlock, 0, (cudaStream_t)stream>>>(a);
    STG_CUDA_TRY(cudaGetLastError());
    return STG_OK;
}

extern "C" stg_status stg_complex_convert(int64_t count, stg_prec src_prec, const void *src_dev, stg_prec dst_prec,
                                          void *dst_dev, void *stream)
{
    if (count < 0 || bad(src_dev) || bad(dst_dev) || src_dev == dst_dev)
        return set_error(STG_ERR_ARG, "stg_complex_convert: bad count or null, misaligned or aliasing pointer");
    const bool ok = (src_prec == STG_F64 || src_prec == STG_F32) && (dst_prec == STG_F64 || dst_prec == STG_F32);
    if (!ok) return set_error(STG_ERR_ARG, "stg_complex_convert: precisions must be F64 or F32");
    if (count == 0) return STG_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned nb = (unsigned)std::min<long long>((count + 255) / 256, 152LL * 16);
    if (src_prec == STG_F64 && dst_prec == STG_F32)
        k_convert<<<nb, 256, 0, st>>>(count, static_cast<const double2 *>(src_dev), static_cast<float2 *>(dst_dev));
    else if (src_prec == STG_F32 && dst_prec == STG_F64)
        k_convert<<<nb, 256, 0, st>>>(count, static_cast<const float2 *>(src_dev), static_cast<double2 *>(dst_dev));
    else if (src_prec == STG_F64)
        k_convert<<<nb, 256, 0, st>>>(count, static_cast<const double2 *>(src_dev), static_cast<double2 *>(dst_dev));
    else
        k_convert<<<nb, 256, 0, st>>>(count, static_cast<const float2 *>(src_dev), static_cast<float2 *>(dst_dev));
    STG_CUDA_TRY(cudaGetLastError());
    return STG_OK;
}

extern "C" stg_status stg_md_kinetic(const stg_lattice *lat, const void *mom_c128_dev, double *out_dev, void *stream)
{
    if (lat && stg::geom_is_slab(lat->g))
        return stg::set_error(STG_ERR_SHAPE, "stg_md_kinetic: not available on a slab lattice (stg_dslash* only)");
    if (!lat || bad(mom_c128_dev) || !out_dev || (reinterpret_cast<uintptr_t>(out_dev) & 7))
        return set_error(STG_ERR_ARG, "stg_md_kinetic: null or misaligned pointer");
    cudaStream_t st = (cudaStream_t)stream;
    MdArgs a = md_args(lat);
    a.H = const_cast<double2 *>(static_cast<const double2 *>(mom_c128_dev));
    a.out = out_dev;
    a.nblocks = (int)md_grid(a);
    STG_CUDA_TRY(cudaMallocAsync((void **)&a.partial, sizeof(double) * a.nblocks, st));
    k_md_kinetic<<<a.nblocks, kMdBlock, 0, st>>>(a);
    k_md_kinetic_finish<<<1, 256, 0, st>>>(a);
    const cudaError_t e = cudaGetLastError();
    cudaFreeAsync(a.partial, st);
    STG_CUDA_TRY(e);
    return STG_OK;
}
