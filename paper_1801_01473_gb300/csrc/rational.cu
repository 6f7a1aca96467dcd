// rational.cu -- a rational function of the shifted normal operator applied to a field (Sec. 2:
// the RHMC applies the rational approximation of a fractional power of the Dirac operator as a
// sum over poles, each term one system of Eq. shift_eo, all solved by one multi-shift CG):
//     out = alpha0 b + sum_i r_i (m^2 + sigma_i - D_eo D_oe)^-1 b
// The pseudofermion heatbath (power +1/8 for a rooted staggered flavour) and the evaluation of
// the fermion action (power -1/4) are both of this form; the action itself,
//     S = alpha0 |b|^2 + sum_i r_i Re(b^dag x_i),
// is a fixed-order FP64 reduction over the solutions (stg_pseudofermion_action).
#include <cstdint>
#include <cstring>
#include <vector>

#include "stg_common.h"

namespace stg {
namespace {

struct Combine {
    int Vh, n;
    double alpha0;
    double r[kMaxShifts];
    const double2 *b;
    const double2 *x[kMaxShifts];
    double2 *out;
};

// out = alpha0 b + sum_i r_i x_i per complex component, terms added in pole order (FP64)
__global__ void k_rational_combine(const __grid_constant__ Combine c)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 3LL * c.Vh) return;
    const double2 bv = c.b[k];
    double re = c.alpha0 * bv.x, im = c.alpha0 * bv.y;
    for (int i = 0; i < c.n; ++i) {
        const double2 xv = c.x[i][k];
        re = fma(c.r[i], xv.x, re);
        im = fma(c.r[i], xv.y, im);
    }
    c.out[k] = make_double2(re, im);
}

// Pseudofermion action from the solutions: one FP64 partial per block of
//     alpha0 |b_k|^2 + sum_i r_i Re(conj(b_k) x_i[k])
// over complex elements k (pole order within an element, a grid-stride loop of a fixed grid, then
// the block's fixed tree), and one block adding the partials in a fixed order.
constexpr int kActBlock = 256;
constexpr int kActGrid = 1024;

struct ActionArgs {
    long long n;  // complex elements: 3 Vh
    int nshift;
    double alpha0;
    double r[kMaxShifts];
    const double2 *b;
    const double2 *x[kMaxShifts];
    double *part;
};

__global__ void __launch_bounds__(kActBlock) k_pf_action_partial(const __grid_constant__ ActionArgs a)
{
    __shared__ double sh[32];
    double acc = 0.0;
    for (long long k = (long long)blockIdx.x * kActBlock + threadIdx.x; k < a.n; k += (long long)kActGrid * kActBlock) {
        const double2 bv = a.b[k];
        double t = a.alpha0 * fma(bv.x, bv.x, bv.y * bv.y);
        for (int i = 0; i < a.nshift; ++i) {
            const double2 xv = a.x[i][k];
            t = fma(a.r[i], fma(bv.x, xv.x, bv.y * xv.y), t);
        }
        acc += t;
    }
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) a.part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kActBlock) k_pf_action_final(const double *part, double *out)
{
    __shared__ double sh[32];
    double acc = 0.0;
    for (int k = threadIdx.x; k < kActGrid; k += kActBlock) acc += part[k];
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) *out = s;
}

}  // namespace
}  // namespace stg

using namespace stg;

extern "C" stg_status stg_pseudofermion_action(const stg_lattice *lat, int32_t nshift, double alpha0,
                                               const double *residues, const void *b_c128_dev,
                                               const void *const *x_c128_dev, double *s_dev, void *stream)
{
    if (lat && stg::geom_is_slab(lat->g))
        return stg::set_error(STG_ERR_SHAPE, "stg_pseudofermion_action: not available on a slab lattice (stg_dslash* only)");
    if (!lat || !b_c128_dev || !s_dev || (nshift > 0 && (!residues || !x_c128_dev)))
        return set_error(STG_ERR_ARG, "stg_pseudofermion_action: null pointer");
    if (nshift < 0 || nshift > kMaxShifts)
        return set_error(STG_ERR_ARG, "stg_pseudofermion_action: nshift must be in 0..32");
    if ((reinterpret_cast<uintptr_t>(b_c128_dev) & 15) || (reinterpret_cast<uintptr_t>(s_dev) & 7))
        return set_error(STG_ERR_ARG, "stg_pseudofermion_action: misaligned field or result");
    ActionArgs a;
    memset(&a, 0, sizeof(a));
    a.n = 3LL * lat->g.Vh;
    a.nshift = nshift;
    a.alpha0 = alpha0;
    a.b = static_cast<const double2 *>(b_c128_dev);
    for (int i = 0; i < nshift; ++i) {
        if (!x_c128_dev[i]) return set_error(STG_ERR_ARG, "stg_pseudofermion_action: null solution");
        if (reinterpret_cast<uintptr_t>(x_c128_dev[i]) & 15)
            return set_error(STG_ERR_ARG, "stg_pseudofermion_action: misaligned solution");
        a.r[i] = residues[i];
        a.x[i] = static_cast<const double2 *>(x_c128_dev[i]);
    }
    cudaStream_t st = (cudaStream_t)stream;
    STG_CUDA_TRY(cudaMallocAsync((void **)&a.part, sizeof(double) * kActGrid, st));
    k_pf_action_partial<<<kActGrid, kActBlock, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        k_pf_action_final<<<1, kActBlock, 0, st>>>(a.part, s_dev);
        e = cudaGetLastError();
    }
    const cudaError_t f = cudaFreeAsync(a.part, st);
    if (e != cudaSuccess) return cuda_error(e, "stg_pseudofermion_action");
    if (f != cudaSuccess) return cuda_error(f, "stg_pseudofermion_action: cudaFreeAsync");
    return STG_OK;
}

extern "C" stg_status stg_rational_apply(const stg_gauge *g_f64, const stg_gauge *g_inner, const stg_mscg_params *params,
                                         double alpha0, const double *residues, const void *b_c128_dev,
                                         void *out_c128_dev, stg_mscg_stats *stats, void *stream)
{
    if (g_f64 && stg::geom_is_slab(g_f64->g))
        return stg::set_error(STG_ERR_SHAPE, "stg_rational_apply: not available on a slab lattice (stg_dslash* only)");
    if (!g_f64 || !params || !residues || !b_c128_dev || !out_c128_dev)
        return set_error(STG_ERR_ARG, "stg_rational_apply: null pointer");
    if (params->nshift < 1 || params->nshift > kMaxShifts)
        return set_error(STG_ERR_ARG, "stg_rational_apply: nshift must be in 1..32");
    if ((reinterpret_cast<uintptr_t>(b_c128_dev) & 15) || (reinterpret_cast<uintptr_t>(out_c128_dev) & 15))
        return set_error(STG_ERR_ARG, "stg_rational_apply: fields must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    const int n = params->nshift, Vh = g_f64->g.Vh;
    const size_t fb = (size_t)Vh * 3 * sizeof(double2);
    char *ws = nullptr;
    STG_CUDA_TRY(cudaMallocAsync((void **)&ws, (size_t)n * fb, st));
    struct Free {
        void *p;
        cudaStream_t s;
        ~Free() { cudaFreeAsync(p, s); }
    } fr{ws, st};
    std::vector<void *> xs(n);
    for (int i = 0; i < n; ++i) xs[i] = ws + (size_t)i * fb;
    stg_status s = stg_mscg_solve(g_f64, g_inner, params, b_c128_dev, xs.data(), stats, stream);
    if (s != STG_OK) return s;
    Combine c;
    memset(&c, 0, sizeof(c));
    c.Vh = Vh;
    c.n = n;
    c.alpha0 = alpha0;
    for (int i = 0; i < n; ++i) {
        c.r[i] = residues[i];
        c.x[i] = static_cast<const double2 *>(xs[i]);
    }
    c.b = static_cast<const double2 *>(b_c128_dev);
    c.out = static_cast<double2 *>(out_c128_dev);
    const long long m = 3LL * Vh;
    k_rational_combine<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(c);
    STG_CUDA_TRY(cudaGetLastError());
    return STG_OK;
}
