// rational.cu -- a rational function of the shifted normal operator applied to a field (Sec. 2:
// the RHMC applies the rational approximation of a fractional power of the Dirac operator as a
// sum over poles, each term one system of Eq. shift_eo, all solved by one multi-shift CG):
//     out = alpha0 b + sum_i r_i (m^2 + sigma_i - D_eo D_oe)^-1 b
// The pseudofermion heatbath (power +1/8 for a rooted staggered flavour) and the evaluation of
// the fermion action (power -1/4) are both of this form.
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

}  // namespace
}  // namespace stg

using namespace stg;

extern "C" stg_status stg_rational_apply(const stg_gauge *g_f64, const stg_gauge *g_inner, const stg_mscg_params *params,
                                         double alpha0, const double *residues, const void *b_c128_dev,
                                         void *out_c128_dev, stg_mscg_stats *stats, void *stream)
{
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
