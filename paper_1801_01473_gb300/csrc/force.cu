// force.cu -- fermion force of the pseudofermion action S = sum_i r_i Re(b^dag x_i),
// x_i = (m^2 + sigma_i - D_eo D_oe)^-1 b: the adjoint of D_eo / D_oe over the multi-shift
// solutions (the fermionic MD force of Sec. 4).
//
// dS = -sum_i r_i x_i^dag dA_i x_i with dA_i = -(dD_eo D_oe + D_eo dD_oe) and D_eo = -D_oe^dag,
// so with y_i = D_oe x_i the change of one link U_mu(z) enters as dS = Re tr(dU W):
//     z even:  W = + sum_i r_i u_mu(z) y_i(z+mu) x_i(z)^dag
//     z odd :  W = - sum_i r_i u_mu(z) x_i(z+mu) y_i(z)^dag
// Output kind 0: F = TA(U W) (traceless anti-Hermitian; dS/deps = tr(X F) along U -> exp(eps X) U);
// kind 1: W^dag (dS/dRe U + i dS/dIm U).  With a U(1) phase field u carries exp(i theta) as well
// (D uses u U and its adjoint), and U is the SU(3) link without the phase.
//
// Work split: y_i = D_oe x_i for all shifts by the D kernel on the double-single copy of the links
// (48-bit significand, ~3x the FP64 operator's speed on GB300); then one thread per site z and
// direction mu gathers its rank-nshift sum of outer products (no atomics: every link is owned by
// exactly one thread) -- in double-single on the FP32 pipes (k_force_ds, the default: GB300 issues
// FP64 at 1/64 of FP32, and the FP64 gather was FP64-pipe bound at ~94 %), or in FP64 (k_force,
// with STG_FORCE_FP64=1).  F = TA(U W) and W^dag are formed in FP64 from the double-single W.
#include <cstdlib>
#include <cstring>
#include <vector>

#include "stg_common.h"

namespace stg {

struct ForceArgs {
    Geom g;
    const void *links;
    const void *x[kMaxShifts];  // even FP64 internal fields
    const void *y[kMaxShifts];  // odd FP64 internal fields, r_i D_oe x_i
    int nshift;
    int kind;
    double2 *out;  // canonical [4][V][3][3]
};

constexpr int kForceBlock = 128;

template <typename LinkT>
__global__ void __launch_bounds__(kForceBlock) k_force(const __grid_constant__ ForceArgs a)
{
    const int par = blockIdx.y;
    const int h = blockIdx.x * kForceBlock + threadIdx.x;
    const int Vh = a.g.Vh;
    if (h >= Vh) return;
    const Site s = site_of(a.g, par, h);
    const long long V = 2LL * Vh;
    for (int mu = 0; mu < 4; ++mu) {
        const Hop hp = hop_of(a.g, s, mu);
        const double u = (double)hp.sf;  // u_mu(z) of the link (z, mu)
        cx<double> W[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) W[r][c] = cx<double>{0.0, 0.0};
        // y holds r_i y_i, so W = sign * sum_i f_i g_i^dag with sign = +u (z even), -u (z odd)
        for (int i = 0; i < a.nshift; ++i) {
            cx<double> f[3], g[3];
            if (par == 0) {
                Field<double>::load(a.y[i], Vh, hp.hf, f);
                Field<double>::load(a.x[i], Vh, h, g);
            } else {
                Field<double>::load(a.x[i], Vh, hp.hf, f);
                Field<double>::load(a.y[i], Vh, h, g);
            }
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) cmac_conj(W[r][c], g[c], f[r]);  // W_rc += f_r conj(g_c)
        }
        // u = sign * exp(i theta) (theta = 0 without a phase field)
        const double sign = par == 0 ? u : -u;
        const void *blk = link_block<LinkT>(a.links, Vh, mu, par);
        cx<double> ph = LinkTraits<LinkT>::phase(blk, Vh, h);
        ph = cx<double>{sign * ph.re, sign * ph.im};
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) W[r][c] = cmul(ph, W[r][c]);
        double2 *o = a.out + ((long long)mu * V + s.i) * 9;
        if (a.kind == 1) {
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) o[r * 3 + c] = make_double2(W[c][r].re, -W[c][r].im);
            continue;
        }
        cx<double> U[3][3];
        LinkTraits<LinkT>::Base::load(blk, Vh, h, U);  // the SU(3) link, without its phase
        cx<double> Z[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                cx<double> z = cx<double>{0.0, 0.0};
#pragma unroll
                for (int k = 0; k < 3; ++k) cmac(z, U[r][k], W[k][c]);
                Z[r][c] = z;
            }
        // TA(Z) = (Z - Z^dag)/2 - tr(Z - Z^dag)/6: the trace of Z - Z^dag is 2i Im tr Z
        const double im_tr = (Z[0][0].im + Z[1][1].im + Z[2][2].im) / 3.0;
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                double re = 0.5 * (Z[r][c].re - Z[c][r].re);
                double im = 0.5 * (Z[r][c].im + Z[c][r].im);
                if (r == c) im -= im_tr;
                o[r * 3 + c] = make_double2(re, im);
            }
    }
}

struct ForceArgsDS {
    Geom g;
    const void *links;          // double-single companion links (possibly with U(1) phases)
    const void *x[kMaxShifts];  // even double-single fields
    const void *y[kMaxShifts];  // odd double-single fields D_oe x_i
    float2 res[kMaxShifts];     // residues as double-single (hi, lo), split on the host
    int nshift;
    int kind;
    double2 *out;  // canonical [4][V][3][3]
};

template <typename LinkT>
__global__ void __launch_bounds__(kForceBlock) k_force_ds(const __grid_constant__ ForceArgsDS a)
{
    const int par = blockIdx.y;
    const int h = blockIdx.x * kForceBlock + threadIdx.x;
    const int Vh = a.g.Vh;
    if (h >= Vh) return;
    const Site s = site_of(a.g, par, h);
    const long long V = 2LL * Vh;
    for (int mu = 0; mu < 4; ++mu) {
        const Hop hp = hop_of(a.g, s, mu);
        cx<dsf> W[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) W[r][c] = cx<dsf>{dsf(0.f, 0.f), dsf(0.f, 0.f)};
        // W = sum_i r_i f_i g_i^dag  (f = y(z+mu), g = x(z) for even z; f = x(z+mu), g = y(z) for odd z)
        for (int i = 0; i < a.nshift; ++i) {
            cx<dsf> f[3], g[3];
            if (par == 0) {
                Field<dsf>::load(a.y[i], Vh, hp.hf, f);
                Field<dsf>::load(a.x[i], Vh, h, g);
            } else {
                Field<dsf>::load(a.x[i], Vh, hp.hf, f);
                Field<dsf>::load(a.y[i], Vh, h, g);
            }
            const dsf ri = dsf(a.res[i].x, a.res[i].y);
#pragma unroll
            for (int c = 0; c < 3; ++c) f[c] = cx<dsf>{ri * f[c].re, ri * f[c].im};
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) cmac_conj(W[r][c], g[c], f[r]);  // W_rc += f_r conj(g_c)
        }
        // u = sign * exp(i theta) (theta = 0 without a phase field); sign = +u_mu(z) even, -u_mu(z) odd
        const void *blk = link_block<LinkT>(a.links, Vh, mu, par);
        cx<dsf> ph = LinkTraits<LinkT>::phase(blk, Vh, h);
        if ((par == 0 ? hp.sf : -hp.sf) < 0.f) ph = cx<dsf>{-ph.re, -ph.im};
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) W[r][c] = cmul(ph, W[r][c]);
        double2 *o = a.out + ((long long)mu * V + s.i) * 9;
        if (a.kind == 1) {
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) o[r * 3 + c] = make_double2((double)W[c][r].re, -(double)W[c][r].im);
            continue;
        }
        // Z = U W with the SU(3) link in double-single, then TA(Z) in FP64
        cx<dsf> U[3][3];
        LinkTraits<LinkT>::Base::load(blk, Vh, h, U);
        cx<double> Z[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                cx<dsf> z = cx<dsf>{dsf(0.f, 0.f), dsf(0.f, 0.f)};
#pragma unroll
                for (int k = 0; k < 3; ++k) cmac(z, U[r][k], W[k][c]);
                Z[r][c] = cx<double>{(double)z.re, (double)z.im};
            }
        const double im_tr = (Z[0][0].im + Z[1][1].im + Z[2][2].im) / 3.0;
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                double re = 0.5 * (Z[r][c].re - Z[c][r].re);
                double im = 0.5 * (Z[r][c].im + Z[c][r].im);
                if (r == c) im -= im_tr;
                o[r * 3 + c] = make_double2(re, im);
            }
    }
}

struct ForceArgsF32 {
    Geom g;
    const void *links;          // FP32 12-real companion links (possibly with U(1) phases)
    const void *x[kMaxShifts];  // even FP32 fields
    const void *y[kMaxShifts];  // odd FP32 fields D_oe x_i
    float res[kMaxShifts];
    int nshift;
    int kind;
    float2 *out;  // canonical complex64 [4][V][3][3]
};

// The gather of k_force_ds in FP32 arithmetic on FP32 fields (single-precision MD forces)
template <typename LinkT>
__global__ void __launch_bounds__(kForceBlock) k_force_f32(const __grid_constant__ ForceArgsF32 a)
{
    const int par = blockIdx.y;
    const int h = blockIdx.x * kForceBlock + threadIdx.x;
    const int Vh = a.g.Vh;
    if (h >= Vh) return;
    const Site s = site_of(a.g, par, h);
    const long long V = 2LL * Vh;
    for (int mu = 0; mu < 4; ++mu) {
        const Hop hp = hop_of(a.g, s, mu);
        cx<float> W[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) W[r][c] = cx<float>{0.f, 0.f};
        for (int i = 0; i < a.nshift; ++i) {
            cx<float> f[3], g[3];
            if (par == 0) {
                Field<float>::load(a.y[i], Vh, hp.hf, f);
                Field<float>::load(a.x[i], Vh, h, g);
            } else {
                Field<float>::load(a.x[i], Vh, hp.hf, f);
                Field<float>::load(a.y[i], Vh, h, g);
            }
            const float ri = a.res[i];
#pragma unroll
            for (int c = 0; c < 3; ++c) f[c] = cx<float>{ri * f[c].re, ri * f[c].im};
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) cmac_conj(W[r][c], g[c], f[r]);  // W_rc += f_r conj(g_c)
        }
        const void *blk = link_block<LinkT>(a.links, Vh, mu, par);
        cx<float> ph = LinkTraits<LinkT>::phase(blk, Vh, h);
        if ((par == 0 ? hp.sf : -hp.sf) < 0.f) ph = cx<float>{-ph.re, -ph.im};
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) W[r][c] = cmul(ph, W[r][c]);
        float2 *o = a.out + ((long long)mu * V + s.i) * 9;
        if (a.kind == 1) {
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) o[r * 3 + c] = make_float2(W[c][r].re, -W[c][r].im);
            continue;
        }
        cx<float> U[3][3];
        LinkTraits<LinkT>::Base::load(blk, Vh, h, U);
        cx<float> Z[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                cx<float> z = cx<float>{0.f, 0.f};
#pragma unroll
                for (int k = 0; k < 3; ++k) cmac(z, U[r][k], W[k][c]);
                Z[r][c] = z;
            }
        const float im_tr = (Z[0][0].im + Z[1][1].im + Z[2][2].im) / 3.f;
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float re = 0.5f * (Z[r][c].re - Z[c][r].re);
                float im = 0.5f * (Z[r][c].im + Z[c][r].im);
                if (r == c) im -= im_tr;
                o[r * 3 + c] = make_float2(re, im);
            }
    }
}

template <typename R>
__device__ __forceinline__ R from_f64(double d) { return (R)d; }
template <>
__device__ __forceinline__ float from_f64<float>(double d) { return f64_to_f32_rn(d); }

template <typename R>
__global__ void k_pack_many(int Vh, const double2 *const *__restrict__ canon, void *const *__restrict__ out)
{
    int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= Vh) return;
    const double2 *src = canon[blockIdx.y];
    cx<R> v[3];
    for (int c = 0; c < 3; ++c) {
        double2 d = src[(size_t)h * 3 + c];
        v[c] = cx<R>{from_f64<R>(d.x), from_f64<R>(d.y)};
    }
    Field<R>::store(out[blockIdx.y], Vh, h, v);
}

struct Residues {
    double r[kMaxShifts];
};

// field i = blockIdx.y at y0 + i * stride: double-single -> FP64 scaled by the residue r_i, in place
__global__ void k_ds_to_f64_scaled(int Vh, const void *y0, size_t stride, const Residues res)
{
    int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= Vh) return;
    void *f = const_cast<char *>(static_cast<const char *>(y0)) + blockIdx.y * stride;
    const double r = res.r[blockIdx.y];
    cx<dsf> v[3];
    cx<double> w[3];
    Field<dsf>::load_rw(f, Vh, h, v);
    for (int c = 0; c < 3; ++c) w[c] = cx<double>{r * (double)v[c].re, r * (double)v[c].im};
    Field<double>::store(f, Vh, h, w);
}

}  // namespace stg

using namespace stg;

// single precision: y_i = D_oe x_i with the FP32 12-real companion, the gather in FP32, complex64 out
static stg_status force_f32(const stg_gauge *g, int32_t nshift, const double *residues, const void *const *x_c128_dev,
                            void *out_c64_dev, int32_t kind, cudaStream_t st)
{
    const int Vh = g->g.Vh;
    const size_t fb = (size_t)Vh * 24;
    const stg_gauge *g32 = nullptr;
    {
        stg_status s = f32_companion(g, st, &g32);
        if (s != STG_OK) return s;
    }
    char *ws = nullptr;
    const size_t ptr_bytes = 2 * kMaxShifts * sizeof(void *);
    STG_CUDA_TRY(cudaMallocAsync((void **)&ws, 2 * nshift * fb + ptr_bytes, st));
    struct Free {
        void *p;
        cudaStream_t s;
        ~Free() { cudaFreeAsync(p, s); }
    } fr{ws, st};
    std::vector<const void *> ptrs(2 * kMaxShifts, nullptr);
    ForceArgsF32 b;
    memset(&b, 0, sizeof(b));
    b.g = g->g;
    b.links = g32->links;
    b.nshift = nshift;
    b.kind = kind;
    b.out = static_cast<float2 *>(out_c64_dev);
    for (int i = 0; i < nshift; ++i) {
        b.x[i] = ws + (size_t)i * fb;
        b.y[i] = ws + (size_t)(nshift + i) * fb;
        b.res[i] = (float)residues[i];
        ptrs[i] = x_c128_dev[i];
        ptrs[kMaxShifts + i] = b.x[i];
    }
    void **d_ptrs = reinterpret_cast<void **>(ws + 2 * nshift * fb);
    STG_CUDA_TRY(cudaMemcpyAsync(d_ptrs, ptrs.data(), ptr_bytes, cudaMemcpyHostToDevice, st));
    k_pack_many<float><<<dim3((Vh + 255) / 256, nshift), 256, 0, st>>>(
        Vh, reinterpret_cast<const double2 *const *>(d_ptrs), d_ptrs + kMaxShifts);
    STG_CUDA_TRY(cudaGetLastError());
    for (int base = 0; base < nshift;) {
        DArgs d;
        memset(&d, 0, sizeof(d));
        d.out_par = 1;
        int ng = 0;
        while (ng < kMaxGroups && base < nshift) {
            DGroup &G = d.grp[ng++];
            G.g = g32->g;
            G.links = g32->links;
            G.nrhs = (nshift - base) < kMaxRhs ? (nshift - base) : kMaxRhs;
            for (int j = 0; j < G.nrhs; ++j) {
                G.in[j] = b.x[base + j];
                G.out[j] = const_cast<void *>(b.y[base + j]);
            }
            base += G.nrhs;
        }
        d.ngroups = ng;
        STG_CUDA_TRY(launch_dslash(g32->kind, d, 0, st));
    }
    const dim3 grid((Vh + kForceBlock - 1) / kForceBlock, 2);
    if (kind_has_u1(g32->kind))
        k_force_f32<LinkU1<LinkF32R12, float>><<<grid, kForceBlock, 0, st>>>(b);
    else
        k_force_f32<LinkF32R12><<<grid, kForceBlock, 0, st>>>(b);
    STG_CUDA_TRY(cudaGetLastError());
    return STG_OK;
}

extern "C" stg_status stg_fermion_force_prec(const stg_gauge *g, stg_prec prec, int32_t nshift, const double *residues,
                                             const void *const *x_c128_dev, void *out_dev, int32_t kind, void *stream)
{
    if (g && stg::geom_is_slab(g->g))
        return stg::set_error(STG_ERR_SHAPE, "stg_fermion_force_prec: not available on a slab lattice (stg_dslash* only)");
    if (prec == STG_F64) return stg_fermion_force(g, nshift, residues, x_c128_dev, out_dev, kind, stream);
    if (prec != STG_F32) return set_error(STG_ERR_ARG, "stg_fermion_force_prec: prec must be F64 or F32");
    if (!g || !residues || !x_c128_dev || !out_dev) return set_error(STG_ERR_ARG, "stg_fermion_force_prec: null pointer");
    if (!kind_is_f64(g->kind)) return set_error(STG_ERR_ARG, "stg_fermion_force_prec: needs an F64 gauge");
    if (nshift < 1 || nshift > kMaxShifts) return set_error(STG_ERR_ARG, "stg_fermion_force_prec: nshift must be in 1..32");
    if (kind != 0 && kind != 1) return set_error(STG_ERR_ARG, "stg_fermion_force_prec: kind must be 0 or 1");
    for (int i = 0; i < nshift; ++i)
        if (!x_c128_dev[i] || (reinterpret_cast<uintptr_t>(x_c128_dev[i]) & 15))
            return set_error(STG_ERR_ARG, "stg_fermion_force_prec: x must be non-null and 16-byte aligned");
    if (reinterpret_cast<uintptr_t>(out_dev) & 15)
        return set_error(STG_ERR_ARG, "stg_fermion_force_prec: out must be 16-byte aligned");
    return force_f32(g, nshift, residues, x_c128_dev, out_dev, kind, (cudaStream_t)stream);
}

extern "C" stg_status stg_fermion_force(const stg_gauge *g, int32_t nshift, const double *residues,
                                        const void *const *x_c128_dev, void *out_c128_dev, int32_t kind, void *stream)
{
    if (g && stg::geom_is_slab(g->g))
        return stg::set_error(STG_ERR_SHAPE, "stg_fermion_force: not available on a slab lattice (stg_dslash* only)");
    if (!g || !residues || !x_c128_dev || !out_c128_dev) return set_error(STG_ERR_ARG, "stg_fermion_force: null pointer");
    if (!kind_is_f64(g->kind)) return set_error(STG_ERR_ARG, "stg_fermion_force: needs an F64 gauge");
    if (nshift < 1 || nshift > kMaxShifts) return set_error(STG_ERR_ARG, "stg_fermion_force: nshift must be in 1..32");
    if (kind != 0 && kind != 1) return set_error(STG_ERR_ARG, "stg_fermion_force: kind must be 0 or 1");
    for (int i = 0; i < nshift; ++i)
        if (!x_c128_dev[i] || (reinterpret_cast<uintptr_t>(x_c128_dev[i]) & 15))
            return set_error(STG_ERR_ARG, "stg_fermion_force: x must be non-null and 16-byte aligned");
    if (reinterpret_cast<uintptr_t>(out_c128_dev) & 15)
        return set_error(STG_ERR_ARG, "stg_fermion_force: out must be 16-byte aligned");

    cudaStream_t st = (cudaStream_t)stream;
    const int Vh = g->g.Vh;
    const size_t fb = (size_t)Vh * 48;
    // y_i = D_oe x_i runs on the double-single companion of the links (FP64-class, ~3x faster
    // than the FP64 operator on GB300); the per-link accumulation of W stays in FP64
    const stg_gauge *gds = nullptr;
    {
        stg_status s = ds_companion(g, st, &gds);
        if (s != STG_OK) return s;
    }
    char *ws = nullptr;
    const size_t ptr_bytes = 3 * kMaxShifts * sizeof(void *);
    STG_CUDA_TRY(cudaMallocAsync((void **)&ws, 3 * nshift * fb + ptr_bytes, st));
    struct Free {
        void *p;
        cudaStream_t s;
        ~Free() { cudaFreeAsync(p, s); }
    } fr{ws, st};

    std::vector<const void *> ptrs(3 * kMaxShifts, nullptr);
    ForceArgs a;
    memset(&a, 0, sizeof(a));
    a.g = g->g;
    a.links = g->links;
    a.nshift = nshift;
    a.kind = kind;
    a.out = static_cast<double2 *>(out_c128_dev);
    for (int i = 0; i < nshift; ++i) {
        a.x[i] = ws + (size_t)i * fb;
        a.y[i] = ws + (size_t)(nshift + i) * fb;
        ptrs[i] = x_c128_dev[i];
        ptrs[kMaxShifts + i] = a.x[i];
        ptrs[2 * kMaxShifts + i] = ws + (size_t)(2 * nshift + i) * fb;  // x_i in double-single
    }
    const char *fp64_env = getenv("STG_FORCE_FP64");
    const bool fp64_gather = fp64_env && fp64_env[0] == '1';
    void **d_ptrs = reinterpret_cast<void **>(ws + 3 * nshift * fb);
    STG_CUDA_TRY(cudaMemcpyAsync(d_ptrs, ptrs.data(), ptr_bytes, cudaMemcpyHostToDevice, st));
    if (fp64_gather)  // FP64 copies of x_i only for the FP64 gather
        k_pack_many<double><<<dim3((Vh + 255) / 256, nshift), 256, 0, st>>>(
            Vh, reinterpret_cast<const double2 *const *>(d_ptrs), d_ptrs + kMaxShifts);
    k_pack_many<dsf><<<dim3((Vh + 255) / 256, nshift), 256, 0, st>>>(
        Vh, reinterpret_cast<const double2 *const *>(d_ptrs), d_ptrs + 2 * kMaxShifts);
    STG_CUDA_TRY(cudaGetLastError());

    // y_i = D_oe x_i, link loads shared across up to kMaxRhs shifts per group
    for (int base = 0; base < nshift;) {
        DArgs d;
        memset(&d, 0, sizeof(d));
        d.out_par = 1;
        int ng = 0;
        while (ng < kMaxGroups && base < nshift) {
            DGroup &G = d.grp[ng++];
            G.g = gds->g;
            G.links = gds->links;
            G.nrhs = (nshift - base) < kMaxRhs ? (nshift - base) : kMaxRhs;
            for (int j = 0; j < G.nrhs; ++j) {
                G.in[j] = ptrs[2 * kMaxShifts + base + j];
                G.out[j] = const_cast<void *>(a.y[base + j]);
            }
            base += G.nrhs;
        }
        d.ngroups = ng;
        STG_CUDA_TRY(launch_dslash(gds->kind, d, 0, st));
    }
    if (!fp64_gather) {
        ForceArgsDS b;
        memset(&b, 0, sizeof(b));
        b.g = g->g;
        b.links = gds->links;
        b.nshift = nshift;
        b.kind = kind;
        b.out = static_cast<double2 *>(out_c128_dev);
        for (int i = 0; i < nshift; ++i) {
            b.x[i] = ptrs[2 * kMaxShifts + i];
            b.y[i] = a.y[i];
            const float hi = (float)residues[i];
            b.res[i] = make_float2(hi, (float)(residues[i] - (double)hi));
        }
        const dim3 grid_ds((Vh + kForceBlock - 1) / kForceBlock, 2);
        switch (gds->kind) {
        case kDSR18: k_force_ds<LinkDSR18><<<grid_ds, kForceBlock, 0, st>>>(b); break;
        case kDSR12: k_force_ds<LinkDSR12><<<grid_ds, kForceBlock, 0, st>>>(b); break;
        case kDSR18 | kU1: k_force_ds<LinkU1<LinkDSR18, double2>><<<grid_ds, kForceBlock, 0, st>>>(b); break;
        default: k_force_ds<LinkU1<LinkDSR12, double2>><<<grid_ds, kForceBlock, 0, st>>>(b); break;
        }
        STG_CUDA_TRY(cudaGetLastError());
        return STG_OK;
    }
    // FP64 gather: r_i y_i, double-single -> FP64 in place (same 48-byte site layout)
    Residues rs;
    for (int i = 0; i < kMaxShifts; ++i) rs.r[i] = i < nshift ? residues[i] : 0.0;
    k_ds_to_f64_scaled<<<dim3((Vh + 255) / 256, nshift), 256, 0, st>>>(Vh, a.y[0], fb, rs);
    STG_CUDA_TRY(cudaGetLastError());
    dim3 grid((Vh + kForceBlock - 1) / kForceBlock, 2);
    switch (g->kind) {
    case kF64R18: k_force<LinkF64R18><<<grid, kForceBlock, 0, st>>>(a); break;
    case kF64R12: k_force<LinkF64R12><<<grid, kForceBlock, 0, st>>>(a); break;
    case kF64R18 | kU1: k_force<LinkU1<LinkF64R18, double2>><<<grid, kForceBlock, 0, st>>>(a); break;
    default: k_force<LinkU1<LinkF64R12, double2>><<<grid, kForceBlock, 0, st>>>(a); break;
    }
    STG_CUDA_TRY(cudaGetLastError());
    return STG_OK;
}
