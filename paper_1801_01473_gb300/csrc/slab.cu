// slab.cu -- the pieces of a multi-shift CG on a lattice split along t into slabs, one per process
// (Sec. 3.1: one-dimensional tiling; Sec. 4.2 and Alg. 1: D on the local sites once the 1-site
// halos of its input are current).  The caller exchanges the halo slices and sums the per-process
// reductions; the library provides D with its fused axpy and dot, the vector updates restricted to
// the local slices, and the FP64 scalar recurrences of the shifted CG as host functions.
#include <cmath>
#include <cstdint>
#include <cstring>

#include "stg_common.h"

namespace stg {
namespace {

constexpr int kSlabBlock = 256;

// fixed-order sum of n partials into *out (one block)
__global__ void __launch_bounds__(kSlabBlock) k_slab_sum(const double *__restrict__ part, int n, double *__restrict__ out)
{
    __shared__ double sh[32];
    double s = 0.0;
    for (int k = threadIdx.x; k < n; k += kSlabBlock) s += part[k];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) *out = s;
}

// y += alpha x on [h0, h1), block partial of |y|^2 (fixed tree) when part != nullptr
template <typename R>
__global__ void __launch_bounds__(kSlabBlock) k_slab_axpy_norm(int Vh, int h0, int h1, double alpha, const void *x, void *y,
                                                               double *part)
{
    __shared__ double sh[32];
    const int h = h0 + blockIdx.x * kSlabBlock + threadIdx.x;
    double n2 = 0.0;
    if (h < h1) {
        cx<R> a[3], b[3];
        Field<R>::load_rw(x, Vh, h, a);
        Field<R>::load_rw(y, Vh, h, b);
        const R al = (R)alpha;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            b[c] = cx<R>{fma(al, a[c].re, b[c].re), fma(al, a[c].im, b[c].im)};
            n2 = fma((double)b[c].re, (double)b[c].re, n2);
            n2 = fma((double)b[c].im, (double)b[c].im, n2);
        }
        Field<R>::store(y, Vh, h, b);
    }
    if (part != nullptr) {
        const double s = block_sum(n2, sh);
        if (threadIdx.x == 0) part[blockIdx.x] = s;
    }
}

struct ShiftUpd {
    int Vh, h0, h1, n;
    double cx[kMaxShifts], cr[kMaxShifts], cp[kMaxShifts];
    int ux[kMaxShifts], up[kMaxShifts];
    void *x[kMaxShifts];
    void *p[kMaxShifts];
    const void *r;
};

// x_i += cx_i p_i ; p_i = cr_i r + cp_i p_i on [h0, h1)
template <typename R>
__global__ void __launch_bounds__(kSlabBlock) k_slab_shift_update(const __grid_constant__ ShiftUpd u)
{
    const int h = u.h0 + blockIdx.x * kSlabBlock + threadIdx.x;
    if (h >= u.h1) return;
    cx<R> r[3];
    Field<R>::load_rw(u.r, u.Vh, h, r);
    for (int i = 0; i < u.n; ++i) {
        if (!u.ux[i] && !u.up[i]) continue;
        cx<R> p[3];
        Field<R>::load_rw(u.p[i], u.Vh, h, p);
        if (u.ux[i]) {
            cx<R> x[3];
            Field<R>::load_rw(u.x[i], u.Vh, h, x);
            const R a = (R)u.cx[i];
#pragma unroll
            for (int c = 0; c < 3; ++c) x[c] = cx<R>{fma(a, p[c].re, x[c].re), fma(a, p[c].im, x[c].im)};
            Field<R>::store(u.x[i], u.Vh, h, x);
        }
        if (u.up[i]) {
            const R zr = (R)u.cr[i], bb = (R)u.cp[i];
#pragma unroll
            for (int c = 0; c < 3; ++c) p[c] = cx<R>{fma(zr, r[c].re, bb * p[c].re), fma(zr, r[c].im, bb * p[c].im)};
            Field<R>::store(u.p[i], u.Vh, h, p);
        }
    }
}

bool aligned(const void *p, unsigned a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

}  // namespace
}  // namespace stg

using namespace stg;

extern "C" stg_status stg_slab_dslash_part(const stg_gauge *g, int32_t out_parity, int32_t part, void *out_dev,
                                           const void *in_dev, void *stream)
{
    if (!g || !out_dev || !in_dev) return set_error(STG_ERR_ARG, "stg_slab_dslash_part: null pointer");
    if (out_parity != 0 && out_parity != 1) return set_error(STG_ERR_ARG, "stg_slab_dslash_part: out_parity must be 0 or 1");
    if (part < 0 || part > 2) return set_error(STG_ERR_ARG, "stg_slab_dslash_part: part must be 0, 1 or 2");
    if (!geom_is_slab(g->g)) return set_error(STG_ERR_SHAPE, "stg_slab_dslash_part: needs a slab lattice");
    if (!aligned(out_dev, 16) || !aligned(in_dev, 16))
        return set_error(STG_ERR_ARG, "stg_slab_dslash_part: pointers must be 16-byte aligned");
    if (out_dev == in_dev) return set_error(STG_ERR_ARG, "stg_slab_dslash_part: out and in must differ");
    const int hs = g->g.L[0] * g->g.L[1] * g->g.L[2] / 2;  // sites of one parity per time slice
    const int lt = g->g.L[3] - 4;                          // local slices
    DArgs a;
    memset(&a, 0, sizeof(a));
    a.out_par = out_parity;
    auto add = [&](int s0, int s1) {  // stored slices [s0, s1)
        if (s1 <= s0) return;
        DGroup &G = a.grp[a.ngroups++];
        G.g = g->g;
        G.g.h_begin = s0 * hs;
        G.g.h_end = s1 * hs;
        G.links = g->links;
        G.nrhs = 1;
        G.in[0] = in_dev;
        G.out[0] = out_dev;
    };
    if (part == 0) add(2, lt + 2);
    if (part == 1) {
        add(2, 3);
        add(lt + 1, lt + 2);
    }
    if (part == 2) add(3, lt + 1);
    if (a.ngroups == 0) return STG_OK;
    STG_CUDA_TRY(launch_dslash(g->kind, a, 0, (cudaStream_t)stream));
    return STG_OK;
}

extern "C" stg_status stg_slab_dslash_xpay(const stg_gauge *g, int32_t out_parity, double coef, void *out_dev,
                                           const void *in_dev, const void *p_dev, double *pq_dev, void *stream)
{
    if (!g || !out_dev || !in_dev || !p_dev) return set_error(STG_ERR_ARG, "stg_slab_dslash_xpay: null pointer");
    if (out_parity != 0 && out_parity != 1) return set_error(STG_ERR_ARG, "stg_slab_dslash_xpay: out_parity must be 0 or 1");
    if (!aligned(out_dev, 16) || !aligned(in_dev, 16) || !aligned(p_dev, 16))
        return set_error(STG_ERR_ARG, "stg_slab_dslash_xpay: pointers must be 16-byte aligned");
    if (out_dev == in_dev || out_dev == p_dev) return set_error(STG_ERR_ARG, "stg_slab_dslash_xpay: out must differ from in and p");
    cudaStream_t st = (cudaStream_t)stream;
    DArgs a;
    memset(&a, 0, sizeof(a));
    a.ngroups = 1;
    a.out_par = out_parity;
    DGroup &G = a.grp[0];
    G.g = g->g;
    G.links = g->links;
    G.nrhs = 1;
    G.in[0] = in_dev;
    G.out[0] = out_dev;
    G.epi_p[0] = p_dev;
    G.coef[0] = coef;
    G.partial[0] = pq_dev ? g->scratch : nullptr;
    STG_CUDA_TRY(launch_dslash(g->kind, a, 1, st));
    if (pq_dev) {
        k_slab_sum<<<1, kSlabBlock, 0, st>>>(g->scratch, dslash_partials(g->g.h_end - g->g.h_begin), pq_dev);
        STG_CUDA_TRY(cudaGetLastError());
    }
    return STG_OK;
}

extern "C" stg_status stg_slab_axpy_norm(const stg_lattice *lat, stg_prec vec_prec, double alpha, const void *x_dev,
                                         void *y_dev, double *norm2_dev, void *stream)
{
    if (!lat || !x_dev || !y_dev) return set_error(STG_ERR_ARG, "stg_slab_axpy_norm: null pointer");
    if (vec_prec != STG_F64 && vec_prec != STG_F32) return set_error(STG_ERR_ARG, "stg_slab_axpy_norm: vec_prec must be F64 or F32");
    if (!aligned(x_dev, 16) || !aligned(y_dev, 16)) return set_error(STG_ERR_ARG, "stg_slab_axpy_norm: fields must be 16-byte aligned");
    const Geom &g = lat->g;
    const int nout = g.h_end - g.h_begin;
    const int nblk = (nout + kSlabBlock - 1) / kSlabBlock;
    cudaStream_t st = (cudaStream_t)stream;
    double *part = nullptr;
    if (norm2_dev) STG_CUDA_TRY(cudaMallocAsync((void **)&part, sizeof(double) * nblk, st));
    if (vec_prec == STG_F64)
        k_slab_axpy_norm<double><<<nblk, kSlabBlock, 0, st>>>(g.Vh, g.h_begin, g.h_end, alpha, x_dev, y_dev, part);
    else
        k_slab_axpy_norm<float><<<nblk, kSlabBlock, 0, st>>>(g.Vh, g.h_begin, g.h_end, alpha, x_dev, y_dev, part);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && norm2_dev) {
        k_slab_sum<<<1, kSlabBlock, 0, st>>>(part, nblk, norm2_dev);
        e = cudaGetLastError();
    }
    if (part) {
        const cudaError_t f = cudaFreeAsync(part, st);
        if (e == cudaSuccess) e = f;
    }
    if (e != cudaSuccess) return cuda_error(e, "stg_slab_axpy_norm");
    return STG_OK;
}

extern "C" stg_status stg_slab_shift_update(const stg_lattice *lat, stg_prec vec_prec, int32_t n, const double *cx,
                                            const double *cr, const double *cp, const int32_t *upd_x,
                                            const int32_t *upd_p, void *const *x_dev, void *const *p_dev,
                                            const void *r_dev, void *stream)
{
    if (!lat || !cx || !cr || !cp || !upd_x || !upd_p || !x_dev || !p_dev || !r_dev)
        return set_error(STG_ERR_ARG, "stg_slab_shift_update: null pointer");
    if (n < 1 || n > kMaxShifts) return set_error(STG_ERR_ARG, "stg_slab_shift_update: n must be in 1..32");
    if (vec_prec != STG_F64 && vec_prec != STG_F32)
        return set_error(STG_ERR_ARG, "stg_slab_shift_update: vec_prec must be F64 or F32");
    ShiftUpd u;
    memset(&u, 0, sizeof(u));
    const Geom &g = lat->g;
    u.Vh = g.Vh;
    u.h0 = g.h_begin;
    u.h1 = g.h_end;
    u.n = n;
    u.r = r_dev;
    for (int i = 0; i < n; ++i) {
        if (!x_dev[i] || !p_dev[i]) return set_error(STG_ERR_ARG, "stg_slab_shift_update: null field");
        u.cx[i] = cx[i];
        u.cr[i] = cr[i];
        u.cp[i] = cp[i];
        u.ux[i] = upd_x[i] != 0;
        u.up[i] = upd_p[i] != 0;
        u.x[i] = x_dev[i];
        u.p[i] = p_dev[i];
    }
    const int nblk = (g.h_end - g.h_begin + kSlabBlock - 1) / kSlabBlock;
    cudaStream_t st = (cudaStream_t)stream;
    if (vec_prec == STG_F64)
        k_slab_shift_update<double><<<nblk, kSlabBlock, 0, st>>>(u);
    else
        k_slab_shift_update<float><<<nblk, kSlabBlock, 0, st>>>(u);
    STG_CUDA_TRY(cudaGetLastError());
    return STG_OK;
}

// ------------------------------------------------------------------ host scalar recurrences

extern "C" stg_status stg_mscg_state_init(stg_mscg_state *st, int32_t nshift, const double *shifts, double tol,
                                          double bnorm2, int32_t max_iter)
{
    if (!st || !shifts) return set_error(STG_ERR_ARG, "stg_mscg_state_init: null pointer");
    if (nshift < 1 || nshift > 32) return set_error(STG_ERR_ARG, "stg_mscg_state_init: nshift must be in 1..32");
    if (max_iter < 1) return set_error(STG_ERR_ARG, "stg_mscg_state_init: max_iter must be positive");
    memset(st, 0, sizeof(*st));
    int i0 = 0;
    for (int i = 0; i < nshift; ++i) {
        if (!(shifts[i] >= 0.0)) return set_error(STG_ERR_ARG, "stg_mscg_state_init: shifts must be >= 0");
        if (shifts[i] < shifts[i0]) i0 = i;
    }
    st->nshift = nshift;
    st->i0 = i0;
    st->max_iter = max_iter;
    for (int i = 0; i < nshift; ++i) {
        st->s[i] = shifts[i] - shifts[i0];
        st->zeta[i] = st->zeta_old[i] = st->zeta_new[i] = 1.0;
        st->active[i] = bnorm2 > 0.0;
    }
    st->alpha_old = 1.0;
    st->beta_old = 0.0;
    st->rr = bnorm2;
    st->tol2 = tol * tol * bnorm2;
    st->nactive = bnorm2 > 0.0 ? nshift : 0;
    st->running = bnorm2 > 0.0;
    st->phase = 0;
    return STG_OK;
}

extern "C" stg_status stg_mscg_state_alpha(stg_mscg_state *st, double pq)
{
    if (!st) return set_error(STG_ERR_ARG, "stg_mscg_state_alpha: null pointer");
    if (st->phase != 0 || !st->running) return set_error(STG_ERR_ARG, "stg_mscg_state_alpha: called out of order");
    const double alpha = st->rr / pq;
    for (int i = 0; i < st->nshift; ++i) {
        if (!st->active[i]) {
            st->cx[i] = 0.0;
            continue;
        }
        const double z = st->zeta[i], zo = st->zeta_old[i];
        const double zn = z * zo * st->alpha_old /
                          (alpha * st->beta_old * (zo - z) + zo * st->alpha_old * (1.0 + st->s[i] * alpha));
        st->zeta_new[i] = zn;
        st->cx[i] = alpha * zn / z;
    }
    st->alpha = alpha;
    st->phase = 1;
    return STG_OK;
}

extern "C" stg_status stg_mscg_state_beta(stg_mscg_state *st, double rr_new)
{
    if (!st) return set_error(STG_ERR_ARG, "stg_mscg_state_beta: null pointer");
    if (st->phase != 1) return set_error(STG_ERR_ARG, "stg_mscg_state_beta: called out of order");
    const double beta = rr_new / st->rr;
    int nact = 0;
    for (int i = 0; i < st->nshift; ++i) {
        if (st->active[i]) {
            const double z = st->zeta[i], zn = st->zeta_new[i];
            const double ratio = zn / z;
            st->cr[i] = zn;
            st->cp[i] = beta * ratio * ratio;
            st->upd_x[i] = 1;
            if (zn * zn * rr_new <= st->tol2) {
                st->active[i] = 0;
                st->shift_iters[i] = st->iters + 1;
                st->upd_p[i] = 0;
            } else {
                st->upd_p[i] = 1;
                ++nact;
            }
            st->zeta_old[i] = z;
            st->zeta[i] = zn;
        } else {
            st->upd_x[i] = 0;
            st->upd_p[i] = 0;
        }
    }
    const bool cont = nact > 0 && st->iters + 1 < st->max_iter;
    // the base direction p = r + beta p continues while any shift does (its zeta stays 1)
    if (cont) {
        st->upd_p[st->i0] = 1;
        st->cr[st->i0] = 1.0;
        st->cp[st->i0] = beta;
    } else {
        for (int i = 0; i < st->nshift; ++i) st->upd_p[i] = 0;
    }
    st->alpha_old = st->alpha;
    st->beta_old = beta;
    st->rr = rr_new;
    st->iters += 1;
    st->nactive = nact;
    st->running = cont ? 1 : 0;
    if (!cont)
        for (int i = 0; i < st->nshift; ++i)
            if (st->active[i]) st->shift_iters[i] = st->iters;
    st->phase = 0;
    return STG_OK;
}
