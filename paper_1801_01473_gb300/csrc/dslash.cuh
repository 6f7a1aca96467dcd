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
// Partials are FP64, one per 64 output sites and right-hand side (fixed-order trees), so the
// reduced values do not depend on the block size the autotuner picks.
#pragma once

#include <type_traits>

#include "stg_internal.cuh"

namespace stg {

constexpr int kMaxRhs = 8;
constexpr int kMaxGroups = 16;  // groups per launch (blockIdx.y): a DArgs of 16 groups is ~8.5 KB of kernel parameters
constexpr int kDslashBlock = 128;   // default block; the autotuner may pick 64, 128 or 256
constexpr int kPartialSites = 64;   // one FP64 partial per 64 output sites, whatever the block size

// Number of FP64 partial sums an epilogue launch writes for a lattice of Vh sites per parity.
__host__ __device__ inline int dslash_partials(int Vh) { return (Vh + kPartialSites - 1) / kPartialSites; }

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

// hi + lo += a * b for double-single a, b (see the kLazyDS path of k_dslash)
__device__ __forceinline__ void lazy_mac(float &hi, float &lo, const dsf &a, const dsf &b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const float t = __fadd_rn(hi, p);
    const float bb = __fsub_rn(t, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bb)), __fsub_rn(p, bb));
    hi = t;
    lo = __fadd_rn(lo, __fadd_rn(err, e));
}

template <typename R>
__device__ __forceinline__ void neg3(cx<R> v[3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) v[c] = cx<R>{-v[c].re, -v[c].im};
}

// Epilogue of the D kernels: scale (MODE 0) or fuse the shifted normal operator and its FP64
// partial sums (MODE 1, 2), store, and write one partial per 64 output sites.  `sh` holds >= 32
// doubles of shared memory; `act` is uniform over the block.
template <typename R, int NRHS, int MODE, int BS>
__device__ __forceinline__ void dslash_epilogue(const DGroup &G, const bool act[NRHS], bool live, int h,
                                                const cx<R> acc[NRHS][3], double *sh,
                                                const cx<R> (*pre_p)[3] = nullptr)
{
    const int Vh = G.g.Vh;
#pragma unroll
    for (int j = 0; j < NRHS; ++j) {
        if (!act[j]) continue;  // uniform over the block
        ProdSum<R> part;
        if (live) {
            cx<R> o[3];
            if (MODE == 0) {
#pragma unroll
                for (int c = 0; c < 3; ++c) o[c] = cx<R>{R(0.5) * acc[j][c].re, R(0.5) * acc[j][c].im};
            } else {
                cx<R> p[3];
                if (pre_p != nullptr) {  // loaded by the caller ahead of time
#pragma unroll
                    for (int c = 0; c < 3; ++c) p[c] = pre_p[j][c];
                } else {
                    Field<R>::load(G.epi_p[j], Vh, h, p);
                }
                const R cj = (R)G.coef[j];
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    o[c] = cx<R>{fma(cj, p[c].re, R(-0.5) * acc[j][c].re), fma(cj, p[c].im, R(-0.5) * acc[j][c].im)};
                if (MODE == 1) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        part.add(p[c].re, o[c].re);
                        part.add(p[c].im, o[c].im);
                    }
                } else {
                    cx<R> b[3];
                    Field<R>::load(G.epi_b[j], Vh, h, b);
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        o[c] = cx<R>{b[c].re - o[c].re, b[c].im - o[c].im};
                        part.add(o[c].re, o[c].re);
                        part.add(o[c].im, o[c].im);
                    }
                }
            }
            Field<R>::store(G.out[j], Vh, h, o);
        }
        if (MODE != 0 && G.partial[j] != nullptr) {
            // two warps per 64-site chunk: warp sums, then pairs of warps
            const double pv = part.warp_total();
            __syncthreads();
            if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = pv;
            __syncthreads();
            constexpr int kChunks = BS / kPartialSites;
            const int c = blockIdx.x * kChunks + threadIdx.x;
            if (threadIdx.x < kChunks && c < dslash_partials(G.g.h_end - G.g.h_begin))
                G.partial[j][c] = sh[2 * threadIdx.x] + sh[2 * threadIdx.x + 1];
        }
    }
}

// Hop loop of the multi-rhs FP32 12-real operator with its loads one hop ahead: while hop k is
// applied, the link of hop k + 1 and every rhs's neighbour vector of hop k + 1 are already in
// flight in registers.  With several rhs per thread the plain loop is latency-bound (each hop's
// multiply-adds wait for that hop's loads: 4 rhs at 32^4 reach 0.61 of HBM bandwidth with 28
// warps per SM); one hop of lookahead costs registers (127, 16 warps per SM) but keeps loads in
// flight through the arithmetic (0.71).  With an epilogue (MODE 1, 2) the last hop loads p_j at the
// output site instead.  Same operations in the same order as the plain loop, so results are
// bitwise equal.
template <int NRHS, int MODE>
__device__ __forceinline__ void dslash_hops_ahead_f32r12(const DGroup &G, int op, int h, const Site &s,
                                                         const bool act[NRHS], cx<float> acc[NRHS][3],
                                                         cx<float> pre_p[NRHS][3])
{
    const int Vh = G.g.Vh;
    Hop hq[4];
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) hq[mu] = hop_of(G.g, s, mu);
    // hop k = 2 mu (forward: link (mu, op) at h, input at hf) or 2 mu + 1 (backward: link (mu, 1 - op)
    // and input at hb); a link is 3 float4 (rows 1 and 2), an FP32 vector a float4 and a float2
    auto load = [&](int k, float4 l[3], float4 va[NRHS], float2 vb[NRHS]) {
        const int mu = k >> 1;
        const bool fw = (k & 1) == 0;
        const int li = fw ? h : hq[mu].hb, vi = fw ? hq[mu].hf : hq[mu].hb;
        const float4 *q = static_cast<const float4 *>(link_block<LinkF32R12>(G.links, Vh, mu, fw ? op : 1 - op));
#pragma unroll
        for (int c = 0; c < 3; ++c) l[c] = __ldg(q + (size_t)c * Vh + li);
#pragma unroll
        for (int j = 0; j < NRHS; ++j) {
            if (!act[j]) continue;
            va[j] = __ldg(static_cast<const float4 *>(G.in[j]) + vi);
            vb[j] = __ldg(reinterpret_cast<const float2 *>(static_cast<const float4 *>(G.in[j]) + Vh) + vi);
        }
    };
    float4 lc[3], ln[3], vac[NRHS], van[NRHS];
    float2 vbc[NRHS], vbn[NRHS];
    load(0, lc, vac, vbc);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (k < 7) {
            load(k + 1, ln, van, vbn);
        } else if (MODE != 0) {
            // the last hop overlaps the epilogue's loads of p_j at the output site
#pragma unroll
            for (int j = 0; j < NRHS; ++j) {
                if (!act[j]) continue;
                van[j] = __ldg(static_cast<const float4 *>(G.epi_p[j]) + h);
                vbn[j] = __ldg(reinterpret_cast<const float2 *>(static_cast<const float4 *>(G.epi_p[j]) + Vh) + h);
            }
        }
        cx<float> U[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            U[(2 * c) / 3][(2 * c) % 3] = cx<float>{lc[c].x, lc[c].y};
            U[(2 * c + 1) / 3][(2 * c + 1) % 3] = cx<float>{lc[c].z, lc[c].w};
        }
        reconstruct_row3(U);
        const int mu = k >> 1;
        const float sg = (k & 1) == 0 ? hq[mu].sf : -hq[mu].sb;
#pragma unroll
        for (int j = 0; j < NRHS; ++j) {
            if (!act[j]) continue;
            const cx<float> v[3] = {cx<float>{vac[j].x, vac[j].y}, cx<float>{vac[j].z, vac[j].w},
                                    cx<float>{vbc[j].x, vbc[j].y}};
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                cx<float> w = cx<float>{0.f, 0.f};
                if ((k & 1) == 0) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) cmac(w, U[r][c], v[c]);
                } else {
#pragma unroll
                    for (int c = 0; c < 3; ++c) cmac_conj(w, U[c][r], v[c]);
                }
                acc[j][r].re = fmaf(sg, w.re, acc[j][r].re);
                acc[j][r].im = fmaf(sg, w.im, acc[j][r].im);
            }
        }
        if (k < 7) {
#pragma unroll
            for (int c = 0; c < 3; ++c) lc[c] = ln[c];
#pragma unroll
            for (int j = 0; j < NRHS; ++j) {
                vac[j] = van[j];
                vbc[j] = vbn[j];
            }
        }
    }
    if (MODE != 0) {
#pragma unroll
        for (int j = 0; j < NRHS; ++j) {
            pre_p[j][0] = cx<float>{van[j].x, van[j].y};
            pre_p[j][1] = cx<float>{van[j].z, van[j].w};
            pre_p[j][2] = cx<float>{vbn[j].x, vbn[j].y};
        }
    }
}

// AHEAD selects the hop loop with one hop of load lookahead (FP32 12-real links only).
template <typename LinkT, int NRHS, int MODE, int BS, bool AHEAD = false>
__global__ void __launch_bounds__(BS) k_dslash(const __grid_constant__ DArgs a)
{
    using R = typename LinkT::R;
    pdl_enter();
    const DGroup &G = a.grp[blockIdx.y];
    const int Vh = G.g.Vh;
    const int nout = G.g.h_end - G.g.h_begin;
    if ((int)(blockIdx.x * BS) >= nout) return;  // block-uniform

    bool act[NRHS];
    bool any = false;
#pragma unroll
    for (int j = 0; j < NRHS; ++j) {
        act[j] = j < G.nrhs && !(G.skip[j] != nullptr && *G.skip[j] != 0);
        any |= act[j];
    }
    if (!any) return;  // block-uniform

    const int h = G.g.h_begin + blockIdx.x * BS + threadIdx.x;
    const bool live = h < G.g.h_end;
    const int op = a.out_par;

    cx<R> acc[NRHS][3];
#pragma unroll
    for (int j = 0; j < NRHS; ++j)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[j][c] = cx<R>{R(0), R(0)};

    // Double-single links without phases: every real output is a signed sum of 48 products of
    // double-single numbers; each product is formed to ~2^-48 (FMA TwoProduct of the high parts plus
    // the two cross terms) and added with TwoSum to a running FP32 head, all rounding errors
    // collecting in an FP32 tail that is folded in once at the end (Ogita-Rump-Oishi style
    // compensated dot product): ~12 FP32 operations per product instead of ~28 for double-single
    // multiply-adds renormalised at every step.
    constexpr bool kLazyDS = std::is_same<R, dsf>::value && !LinkTraits<LinkT>::kU1;
    if constexpr (kLazyDS) {
        if (live) {
            float ahi[NRHS][3][2], alo[NRHS][3][2];
#pragma unroll
            for (int j = 0; j < NRHS; ++j)
#pragma unroll
                for (int r = 0; r < 3; ++r) ahi[j][r][0] = ahi[j][r][1] = alo[j][r][0] = alo[j][r][1] = 0.f;
            const Site s = site_of(G.g, op, h);
#pragma unroll
            for (int mu = 0; mu < 4; ++mu) {
                const Hop hp = hop_of(G.g, s, mu);
                cx<R> U[3][3];
                LinkT::load(link_block<LinkT>(G.links, Vh, mu, op), Vh, h, U);
#pragma unroll
                for (int j = 0; j < NRHS; ++j) {
                    if (!act[j]) continue;
                    cx<R> v[3];
                    Field<R>::load(G.in[j], Vh, hp.hf, v);
                    if (hp.sf < 0.f) neg3(v);
#pragma unroll
                    for (int r = 0; r < 3; ++r)
#pragma unroll
                        for (int c = 0; c < 3; ++c) {  // U[r][c] v[c]
                            lazy_mac(ahi[j][r][0], alo[j][r][0], U[r][c].re, v[c].re);
                            lazy_mac(ahi[j][r][0], alo[j][r][0], -U[r][c].im, v[c].im);
                            lazy_mac(ahi[j][r][1], alo[j][r][1], U[r][c].re, v[c].im);
                            lazy_mac(ahi[j][r][1], alo[j][r][1], U[r][c].im, v[c].re);
                        }
                }
                LinkT::load(link_block<LinkT>(G.links, Vh, mu, 1 - op), Vh, hp.hb, U);
#pragma unroll
                for (int j = 0; j < NRHS; ++j) {
                    if (!act[j]) continue;
                    cx<R> v[3];
                    Field<R>::load(G.in[j], Vh, hp.hb, v);
                    if (hp.sb > 0.f) neg3(v);  // the backward hop enters with -u_mu(x - mu)
#pragma unroll
                    for (int r = 0; r < 3; ++r)
#pragma unroll
                        for (int c = 0; c < 3; ++c) {  // conj(U[c][r]) v[c]
                            lazy_mac(ahi[j][r][0], alo[j][r][0], U[c][r].re, v[c].re);
                            lazy_mac(ahi[j][r][0], alo[j][r][0], U[c][r].im, v[c].im);
                            lazy_mac(ahi[j][r][1], alo[j][r][1], U[c][r].re, v[c].im);
                            lazy_mac(ahi[j][r][1], alo[j][r][1], -U[c][r].im, v[c].re);
                        }
                }
            }
#pragma unroll
            for (int j = 0; j < NRHS; ++j)
#pragma unroll
                for (int r = 0; r < 3; ++r)
                    acc[j][r] = cx<R>{ds_two_sum(ahi[j][r][0], alo[j][r][0]), ds_two_sum(ahi[j][r][1], alo[j][r][1])};
        }
    } else if (AHEAD) {
        if constexpr (std::is_same<LinkT, LinkF32R12>::value) {
            cx<float> pre_p[NRHS][3];
            if (live) dslash_hops_ahead_f32r12<NRHS, MODE>(G, op, h, site_of(G.g, op, h), act, acc, pre_p);
            __shared__ double sh[32];
            dslash_epilogue<R, NRHS, MODE, BS>(G, act, live, h, acc, sh, MODE != 0 ? pre_p : nullptr);
            return;
        }
    } else if (live) {
        const Site s = site_of(G.g, op, h);
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            const Hop hp = hop_of(G.g, s, mu);
            cx<R> U[3][3];
            // forward hop: u_mu(x) U_mu(x) in(x + mu)
            const void *blk_f = link_block<LinkT>(G.links, Vh, mu, op);
            LinkT::load(blk_f, Vh, h, U);
            cx<R> ph_f;
            if constexpr (LinkTraits<LinkT>::kU1) ph_f = LinkTraits<LinkT>::phase(blk_f, Vh, h);
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
                    if constexpr (LinkTraits<LinkT>::kU1) w = cmul(ph_f, w);
                    acc[j][r].re = fma(R(hp.sf), w.re, acc[j][r].re);
                    acc[j][r].im = fma(R(hp.sf), w.im, acc[j][r].im);
                }
            }
            // backward hop: - u_mu(x - mu) U_mu(x - mu)^dag in(x - mu)
            const void *blk_b = link_block<LinkT>(G.links, Vh, mu, 1 - op);
            LinkT::load(blk_b, Vh, hp.hb, U);
            cx<R> ph_b;
            if constexpr (LinkTraits<LinkT>::kU1) ph_b = cconj(LinkTraits<LinkT>::phase(blk_b, Vh, hp.hb));
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
                    if constexpr (LinkTraits<LinkT>::kU1) w = cmul(ph_b, w);
                    acc[j][r].re = fma(R(-hp.sb), w.re, acc[j][r].re);
                    acc[j][r].im = fma(R(-hp.sb), w.im, acc[j][r].im);
                }
            }
        }
    }

    __shared__ double sh[32];
    dslash_epilogue<R, NRHS, MODE, BS>(G, act, live, h, acc, sh);
}

// Shared-link variant for groups of several right-hand sides on FP32 / 16-bit links (R = float).
// A block covers 64 output sites and every right-hand side of its group.  First all its threads
// load the 8 links of the 64 sites (decoded, with the hop signs folded in: +u U forward, -u U
// backward) into shared memory, together with the neighbours' half indices; after one barrier,
// warps 2j and 2j+1 apply the operator to rhs j on the two 32-site halves from those links.  Every
// link is read from memory once per block whatever the rhs count, and each thread holds the
// registers of a one-rhs operator.  Sign folding is exact, so outputs and partial sums are bitwise
// those of k_dslash.
constexpr int kShSites = 64;
constexpr size_t kShBytes = (size_t)8 * 18 * kShSites * sizeof(float) + (size_t)8 * kShSites * sizeof(int);

template <typename LinkT, int MODE>
__global__ void __launch_bounds__(512) k_dslash_sh(const __grid_constant__ DArgs a)
{
    using R = typename LinkT::R;
    static_assert(sizeof(R) == sizeof(float), "shared-link operator is for FP32 arithmetic");
    extern __shared__ float sh_links[];  // [8 hops][18 reals][64 sites], then int [8 hops][64 sites]
    int *sh_nb = reinterpret_cast<int *>(sh_links + 8 * 18 * kShSites);
    __shared__ double sh_part[16];
    pdl_enter();
    const DGroup &G = a.grp[blockIdx.y];
    const int Vh = G.g.Vh;
    const int nout = G.g.h_end - G.g.h_begin;
    if ((int)(blockIdx.x * kShSites) >= nout) return;  // block-uniform
    const int h0 = G.g.h_begin + blockIdx.x * kShSites;
    const int hend = G.g.h_end;
    const int op = a.out_par;
    // stage the links: hop k = 2 mu (forward) or 2 mu + 1 (backward) of site s
    for (int t = threadIdx.x; t < 8 * kShSites; t += blockDim.x) {
        const int k = t / kShSites, sl = t - k * kShSites, h = h0 + sl;
        if (h >= hend) continue;
        const int mu = k >> 1;
        const Hop hp = hop_of(G.g, site_of(G.g, op, h), mu);
        cx<R> U[3][3];
        R sign;
        if ((k & 1) == 0) {
            LinkT::load(link_block<LinkT>(G.links, Vh, mu, op), Vh, h, U);
            sign = R(hp.sf);
            sh_nb[k * kShSites + sl] = hp.hf;
        } else {
            LinkT::load(link_block<LinkT>(G.links, Vh, mu, 1 - op), Vh, hp.hb, U);
            sign = R(-hp.sb);
            sh_nb[k * kShSites + sl] = hp.hb;
        }
        float *dst = sh_links + (size_t)k * 18 * kShSites + sl;
#pragma unroll
        for (int e = 0; e < 9; ++e) {
            dst[(2 * e) * kShSites] = sign * U[e / 3][e % 3].re;
            dst[(2 * e + 1) * kShSites] = sign * U[e / 3][e % 3].im;
        }
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, j = warp >> 1;
    const int sl = ((warp & 1) << 5) + (threadIdx.x & 31);
    const int h = h0 + sl;
    const bool act = j < G.nrhs && !(G.skip[j] != nullptr && *G.skip[j] != 0);  // warp-uniform
    const bool live = act && h < hend;
    ProdSum<R> part;
    if (live) {
        cx<R> acc[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[c] = cx<R>{R(0), R(0)};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float *src = sh_links + (size_t)k * 18 * kShSites + sl;
            cx<R> U[3][3], v[3];
#pragma unroll
            for (int e = 0; e < 9; ++e) U[e / 3][e % 3] = cx<R>{src[(2 * e) * kShSites], src[(2 * e + 1) * kShSites]};
            Field<R>::load(G.in[j], Vh, sh_nb[k * kShSites + sl], v);
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                cx<R> w = cx<R>{R(0), R(0)};
                if ((k & 1) == 0) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) cmac(w, U[r][c], v[c]);
                } else {
#pragma unroll
                    for (int c = 0; c < 3; ++c) cmac_conj(w, U[c][r], v[c]);
                }
                acc[r].re = acc[r].re + w.re;
                acc[r].im = acc[r].im + w.im;
            }
        }
        cx<R> o[3];
        if (MODE == 0) {
#pragma unroll
            for (int c = 0; c < 3; ++c) o[c] = cx<R>{R(0.5) * acc[c].re, R(0.5) * acc[c].im};
        } else {
            cx<R> pv[3];
            Field<R>::load(G.epi_p[j], Vh, h, pv);
            const R cj = (R)G.coef[j];
#pragma unroll
            for (int c = 0; c < 3; ++c)
                o[c] = cx<R>{fma(cj, pv[c].re, R(-0.5) * acc[c].re), fma(cj, pv[c].im, R(-0.5) * acc[c].im)};
            if (MODE == 1) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    part.add(pv[c].re, o[c].re);
                    part.add(pv[c].im, o[c].im);
                }
            } else {
                cx<R> b[3];
                Field<R>::load(G.epi_b[j], Vh, h, b);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    o[c] = cx<R>{b[c].re - o[c].re, b[c].im - o[c].im};
                    part.add(o[c].re, o[c].re);
                    part.add(o[c].im, o[c].im);
                }
            }
        }
        Field<R>::store(G.out[j], Vh, h, o);
    }
    if (MODE != 0) {
        const double pv = part.warp_total();
        if ((threadIdx.x & 31) == 0) sh_part[warp] = pv;
        __syncthreads();
        const int jj = threadIdx.x;  // one thread per rhs writes its 64-site partial
        if (jj < G.nrhs && 2 * jj + 1 < (int)(blockDim.x >> 5) && G.partial[jj] != nullptr &&
            !(G.skip[jj] != nullptr && *G.skip[jj] != 0))
            G.partial[jj][blockIdx.x] = sh_part[2 * jj] + sh_part[2 * jj + 1];
    }
}

// Launches `kernel` with the programmatic-stream-serialization attribute (the kernel must start
// with pdl_enter()); STG_PDL=0 in the environment launches without it.
bool pdl_enabled();

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args &&>(args)...);
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl_smem(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                            Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args &&>(args)...);
}

// Host-side launcher: picks the NRHS instantiation (>= the largest group's nrhs) and the
// block size `bs` (64, 128 or 256; anything else falls back to 128).
template <typename LinkT, int NRHS, int BS>
cudaError_t launch_dslash_nb(const DArgs &a, int mode, int maxv, cudaStream_t st)
{
    dim3 grid((maxv + BS - 1) / BS, a.ngroups);
    if (mode == 0) return launch_pdl(k_dslash<LinkT, NRHS, 0, BS>, grid, dim3(BS), st, a);
    if (mode == 1) return launch_pdl(k_dslash<LinkT, NRHS, 1, BS>, grid, dim3(BS), st, a);
    return launch_pdl(k_dslash<LinkT, NRHS, 2, BS>, grid, dim3(BS), st, a);
}

template <typename LinkT, int NRHS>
cudaError_t launch_dslash_n(const DArgs &a, int mode, int maxv, int bs, cudaStream_t st)
{
    if (bs == 64) return launch_dslash_nb<LinkT, NRHS, 64>(a, mode, maxv, st);
    if (bs == 256) return launch_dslash_nb<LinkT, NRHS, 256>(a, mode, maxv, st);
    return launch_dslash_nb<LinkT, NRHS, 128>(a, mode, maxv, st);
}

inline void dslash_extent(const DArgs &a, int &maxv, int &maxr)
{
    maxv = 0;
    maxr = 0;
    for (int k = 0; k < a.ngroups; ++k) {
        const int nout = a.grp[k].g.h_end - a.grp[k].g.h_begin;  // output sites of the group
        if (nout > maxv) maxv = nout;
        if (a.grp[k].nrhs > maxr) maxr = a.grp[k].nrhs;
    }
}

// NRHS template the launcher uses for a largest group of `maxr` right-hand sides.
inline int dslash_nrhs_template(int maxr) { return maxr <= 1 ? 1 : maxr <= 2 ? 2 : maxr <= 4 ? 4 : 8; }

// Launch shape code: a block size (64, 128, 256) for the rhs-in-registers kernel, kSharedLinks
// for k_dslash_sh (64 x nrhs threads per block; FP32 arithmetic only), or kLoadsAhead for the
// rhs-in-registers kernel with one hop of load lookahead (64-thread blocks; FP32 12-real links and
// 3 or 4 rhs, where it measured faster: 8 rhs spill).
constexpr int kSharedLinks = 1 << 16;
constexpr int kLoadsAhead = 1 << 17;
template <typename LinkT>
cudaError_t launch_dslash_t(const DArgs &a, int mode, int bs, cudaStream_t st)
{
    int maxv, maxr;
    dslash_extent(a, maxv, maxr);
    if (a.ngroups <= 0 || maxv <= 0 || maxr <= 0) return cudaSuccess;
    if (bs == kSharedLinks) {
        if constexpr (sizeof(typename LinkT::R) == sizeof(float) && !LinkTraits<LinkT>::kU1) {
            if (maxr > kMaxRhs) return cudaErrorInvalidValue;
            const dim3 grid((maxv + kShSites - 1) / kShSites, a.ngroups), block(64 * maxr);
            if (mode == 0) return launch_pdl_smem(k_dslash_sh<LinkT, 0>, grid, block, kShBytes, st, a);
            if (mode == 1) return launch_pdl_smem(k_dslash_sh<LinkT, 1>, grid, block, kShBytes, st, a);
            return launch_pdl_smem(k_dslash_sh<LinkT, 2>, grid, block, kShBytes, st, a);
        } else {
            return cudaErrorInvalidValue;
        }
    }
    if (bs == kLoadsAhead) {
        if constexpr (std::is_same<LinkT, LinkF32R12>::value) {
            if (dslash_nrhs_template(maxr) != 4) return cudaErrorInvalidValue;
            const dim3 grid((maxv + 63) / 64, a.ngroups);
            if (mode == 0) return launch_pdl(k_dslash<LinkT, 4, 0, 64, true>, grid, dim3(64), st, a);
            if (mode == 1) return launch_pdl(k_dslash<LinkT, 4, 1, 64, true>, grid, dim3(64), st, a);
            return launch_pdl(k_dslash<LinkT, 4, 2, 64, true>, grid, dim3(64), st, a);
        } else {
            return cudaErrorInvalidValue;
        }
    }
    switch (dslash_nrhs_template(maxr)) {
    case 1: return launch_dslash_n<LinkT, 1>(a, mode, maxv, bs, st);
    case 2: return launch_dslash_n<LinkT, 2>(a, mode, maxv, bs, st);
    case 4: return launch_dslash_n<LinkT, 4>(a, mode, maxv, bs, st);
    default: return maxr <= kMaxRhs ? launch_dslash_n<LinkT, 8>(a, mode, maxv, bs, st) : cudaErrorInvalidValue;
    }
}

}  // namespace stg
