// dslash.cuh -- the staggered hopping term D_eo / D_oe (Sec. 2) as one CUDA kernel,
// templated on the link storage (precision, 18/12-real compression), the number of
// right-hand sides that share each link load, and the epilogue.
//
// One thread per output site.  For each direction the thread loads the forward link
// U_mu(x) (same parity as x) and the backward link U_mu(x - mu) (other parity) once and
// applies them to every right-hand side:
//     acc_j += u_mu(x) U_mu(x) in_j(x + mu) - u_mu(x - mu) U_mu(x - mu)^dag in_j(x - mu)
// The link phases are sign flips computed from the coordinates (no phase storage).
// Epilogues (fused into the D_eo pass of the normal operator, Eq. shift_eo):
//     MODE 0   out_j = acc_j / 2
//     MODE 1   out_j = c_j p_j - acc_j / 2             partial_j[block] = Re<p_j, out_j>
//     MODE 2   out_j = b_j - (c_j p_j - acc_j / 2)     partial_j[block] = |out_j|^2
// Partials are FP64, one per block and right-hand side (deterministic fixed-order tree).
#pragma once

#include "stg_internal.cuh"

namespace stg {

constexpr int kMaxRhs = 8;
constexpr int kMaxGroups = 4;
constexpr int kDslashBlock = 128;

// A set of right-hand sides on one lattice and gauge.  blockIdx.y selects the group.
struct DGroup {
    Geom g;
    const void *links;
    int nrhs;
    const void *in[kMaxRhs];
    void *out[kMaxRhs];
    const void *epi_p[kMaxRhs];
    const void *epi_b[kMaxRhs];
    double coef[kMaxRhs];
    double *partial[kMaxRhs];
    const int *skip[kMaxRhs];  // device flag; nonzero -> leave this rhs untouched
};

struct DArgs {
    DGroup grp[kMaxGroups];
    int ngroups;
    int out_par;  // parity of the output sites: 0 -> D_eo, 1 -> D_oe
};

template <typename LinkT, int NRHS, int MODE>
__global__ void __launch_bounds__(kDslashBlock) k_dslash(const __grid_constant__ DArgs a)
{
    using R = typename LinkT::R;
    const DGroup &G = a.grp[blockIdx.y];
    const int Vh = G.g.Vh;
    if ((int)(blockIdx.x * kDslashBlock) >= Vh) return;  // block-uniform

    bool act[NRHS];
    bool any = false;
#pragma unroll
    for (int j = 0; j < NRHS; ++j) {
        act[j] = j < G.nrhs && !(G.skip[j] != nullptr && *G.skip[j] != 0);
        any |= act[j];
    }
    if (!any) return;  // block-uniform

    const int h = blockIdx.x * kDslashBlock + threadIdx.x;
    const bool live = h < Vh;
    const int op = a.out_par;

    cx<R> acc[NRHS][3];
#pragma unroll
    for (int j = 0; j < NRHS; ++j)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[j][c] = cx<R>{R(0), R(0)};

    if (live) {
        const Site s = site_of(G.g, op, h);
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            const Hop hp = hop_of(G.g, s, mu);
            cx<R> U[3][3];
            // forward hop: u_mu(x) U_mu(x) in(x + mu)
            LinkT::load(link_block<LinkT>(G.links, Vh, mu, op), Vh, h, U);
#pragma unroll
            for (int j = 0; j < NRHS; ++j) {
                if (!act[j]) continue;
                cx<R> v[3];
                Field<R>::load(G.in[j], Vh, hp.hf, v);
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    cx<R> w = cx<R>{R(0), R(0)};
#pragma unroll
                    for (int c = 0; c < 3; ++c) cmac(w, U[r][c], v[c]);
                    acc[j][r].re = fma(R(hp.sf), w.re, acc[j][r].re);
                    acc[j][r].im = fma(R(hp.sf), w.im, acc[j][r].im);
                }
            }
            // backward hop: - u_mu(x - mu) U_mu(x - mu)^dag in(x - mu)
            LinkT::load(link_block<LinkT>(G.links, Vh, mu, 1 - op), Vh, hp.hb, U);
#pragma unroll
            for (int j = 0; j < NRHS; ++j) {
                if (!act[j]) continue;
                cx<R> v[3];
                Field<R>::load(G.in[j], Vh, hp.hb, v);
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    cx<R> w = cx<R>{R(0), R(0)};
#pragma unroll
                    for (int c = 0; c < 3; ++c) cmac_conj(w, U[c][r], v[c]);
                    acc[j][r].re = fma(R(-hp.sb), w.re, acc[j][r].re);
                    acc[j][r].im = fma(R(-hp.sb), w.im, acc[j][r].im);
                }
            }
        }
    }

    __shared__ double sh[32];
#pragma unroll
    for (int j = 0; j < NRHS; ++j) {
        if (!act[j]) continue;  // uniform over the block
        double part = 0.0;
        if (live) {
            cx<R> o[3];
            if (MODE == 0) {
#pragma unroll
                for (int c = 0; c < 3; ++c) o[c] = cx<R>{R(0.5) * acc[j][c].re, R(0.5) * acc[j][c].im};
            } else {
                cx<R> p[3];
                Field<R>::load(G.epi_p[j], Vh, h, p);
                const R cj = (R)G.coef[j];
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    o[c] = cx<R>{fma(cj, p[c].re, R(-0.5) * acc[j][c].re), fma(cj, p[c].im, R(-0.5) * acc[j][c].im)};
                if (MODE == 1) {
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        part += (double)p[c].re * (double)o[c].re + (double)p[c].im * (double)o[c].im;
                } else {
                    cx<R> b[3];
                    Field<R>::load(G.epi_b[j], Vh, h, b);
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        o[c] = cx<R>{b[c].re - o[c].re, b[c].im - o[c].im};
                        part += (double)o[c].re * (double)o[c].re + (double)o[c].im * (double)o[c].im;
                    }
                }
            }
            Field<R>::store(G.out[j], Vh, h, o);
        }
        if (MODE != 0 && G.partial[j] != nullptr) {
            double t = block_sum(part, sh);
            if (threadIdx.x == 0) G.partial[j][blockIdx.x] = t;
        }
    }
}

// Host-side launcher: picks the NRHS instantiation (>= the largest group's nrhs).
template <typename LinkT>
cudaError_t launch_dslash_t(const DArgs &a, int mode, cudaStream_t st)
{
    int maxv = 0, maxr = 0;
    for (int k = 0; k < a.ngroups; ++k) {
        if (a.grp[k].g.Vh > maxv) maxv = a.grp[k].g.Vh;
        if (a.grp[k].nrhs > maxr) maxr = a.grp[k].nrhs;
    }
    if (a.ngroups <= 0 || maxv <= 0 || maxr <= 0) return cudaSuccess;
    dim3 grid((maxv + kDslashBlock - 1) / kDslashBlock, a.ngroups);
    dim3 block(kDslashBlock);
#define STG_DSL_CASE(N)                                                                         \
    if (maxr <= N) {                                                                            \
        if (mode == 0) k_dslash<LinkT, N, 0><<<grid, block, 0, st>>>(a);                         \
        else if (mode == 1) k_dslash<LinkT, N, 1><<<grid, block, 0, st>>>(a);                    \
        else k_dslash<LinkT, N, 2><<<grid, block, 0, st>>>(a);                                   \
        return cudaGetLastError();                                                              \
    }
    STG_DSL_CASE(1)
    STG_DSL_CASE(2)
    STG_DSL_CASE(4)
    STG_DSL_CASE(8)
#undef STG_DSL_CASE
    return cudaErrorInvalidValue;
}

}  // namespace stg
