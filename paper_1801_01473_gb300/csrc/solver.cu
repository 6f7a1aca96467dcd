// solver.cu -- multi-shift CG for (m^2 - D_eo D_oe + sigma_i) x_i = b (Sec. 2, Eq. shift_eo),
// batched over lattices, right-hand sides and shifts, with an optional low-precision inner
// solve and FP64 reliable updates.
//
// A "system" is one right-hand side b with its shifts.  The solve runs in two phases.
//
// Phase 1 (multi-shift CG, inner precision R = double or float).  One Krylov space for all
// shifts of a system: base shift sigma_0 = min sigma_i, relative shifts s_i = sigma_i - sigma_0.
// Per iteration, for every system of the batch at once:
//   D_oe p -> t ;  q = (m^2 + sigma_0) p - D_eo t  with the partial sums of Re<p,q>   (k_dslash)
//   alpha = <r,r>/Re<p,q>;  zeta_i' and alpha_i = alpha zeta_i'/zeta_i  (FP64)          (k_alpha)
//   r -= alpha q  with the partial sums of |r|^2                                        (k_update_r)
//   beta = |r|^2_new/|r|^2_old;  beta_i = beta (zeta_i'/zeta_i)^2;  per-shift stop test
//   zeta_i' |r| <= tol |b|;  history rotation  (FP64)                                    (k_beta)
//   x_i += alpha_i p_i ;  p_i = zeta_i' r + beta_i p_i   (one pass over all live shifts)  (k_update_shifts)
// The base direction p is the p_i of the base shift (zeta = 1, alpha_0 = alpha, beta_0 = beta).
// Reductions are FP64 per block, summed in a fixed order: results do not depend on timing.
// Iterations are captured into a CUDA graph in chunks; converged systems skip all work, so the
// host only looks at convergence flags between chunks.
//
// Phase 2 (per-shift refinement, FP64 reliable updates).  Every (system, shift) pair gets its
// FP64 true residual r = b - A_i x_i.  Pairs above tol run CG on A_i in the inner precision
// (the phase-1 kernels with one shift), accumulating a correction y; whenever the iterated
// residual has fallen by reliable_delta, or reached tol, the host folds x += y in FP64 and
// recomputes r = b - A_i x in FP64 (a reliable update), continuing from the new r with the
// same search direction.  A pair stops when its FP64 true residual is <= tol |b|.
// For a pure-FP64 solve (no inner gauge) phase 1 runs to tol and phase 2 only checks.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "stg_common.h"

namespace stg {

constexpr int kVecBlock = 256;

// Vector-kernel partial sums are per warp: one FP64 value per 32 consecutive sites, in site
// order, written by lane 0 without block barriers (fixed-order, so still deterministic).
__device__ __forceinline__ void warp_partial(double v, int h, int Vh, double *part)
{
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0 && h < Vh) part[h >> 5] = v;
}
template <typename R>
__device__ __forceinline__ void warp_partial(const ProdSum<R> &a, int h, int Vh, double *part)
{
    const double v = a.warp_total();
    if ((threadIdx.x & 31) == 0 && h < Vh) part[h >> 5] = v;
}

struct SysScal {
    double rr, alpha, alpha_old, beta_old, bnorm2, tol2, tol2_true, rr_last, delta2, coef, rr_best;
    double zeta[kMaxShifts], zeta_old[kMaxShifts], zeta_new[kMaxShifts], s[kMaxShifts];
    double cx[kMaxShifts], cr[kMaxShifts], cp[kMaxShifts];
    int upd_x[kMaxShifts], upd_p[kMaxShifts], active[kMaxShifts], shift_iters[kMaxShifts];
    int nshift, i0, running, iters, max_iter, nactive, phase2, stalls;
    int win_start, hist_overflow;  // deferred update: iteration at the window start, entry overflow
};

struct HistEntry {
    double ax, pr, pp;  // iteration of a window: x_i += ax p_i ; p_i = pr r + pp p_i
};

constexpr int kHistMax = 256;     // deferred update: residuals per window (a multiple of the chunk)
constexpr int kFlushShifts = 8;   // shifts per thread block of the window flush

// Coefficients of one window flush of one system (filled by k_flush_coef)
struct FlushCoef {
    float a[kHistMax][kMaxShifts];  // x_i += sum_t a[t][i] r^(t) + e[i] P0_i
    float d[kHistMax][kMaxShifts];  // p_i  = sum_t d[t][i] r^(t) + f[i] P0_i
    float e[kMaxShifts], f[kMaxShifts];
    int xupd[kMaxShifts], pmat[kMaxShifts];
    int n, first_slot;
};

struct SysVecs {
    void *r, *q, *t;                         // inner precision: r, q even; t odd
    void *x[kMaxShifts], *p[kMaxShifts];     // inner precision
    void *xhi, *rhi, *t64, *b64;             // phase 2: FP64 solution, residual, odd temp, source
    void *yhi;                               // anchored refinement: the correction y in precision H
    const double2 *bcanon;                   // canonical source (phase 1)
    double *part_d, *part_v, *part_v2;       // partial sums (64-site dslash chunks / 32-site warps)
    int Vh, nblk_d, nblk_v, npart_v;  // nblk_v: kVecBlock-site blocks; npart_v: partials (one per 32 sites)
    // deferred update (phase 1 of mixed solves): r is a ring of nslot residual fields (slot k % nslot
    // holds r^k), pstart the base direction at the window start, hist/coef the window's scalars
    int nslot;
    size_t slot_bytes;
    void *pstart;
    HistEntry *hist;  // [kHistMax][kMaxShifts]
    FlushCoef *coef;
};

template <typename R>
__device__ __forceinline__ void *ring_slot(const SysVecs &V, int k)
{
    return static_cast<char *>(V.r) + (size_t)(k % V.nslot) * V.slot_bytes;
}

// ------------------------------------------------------------------ vector kernels

// |v|^2 of one site added to a partial-sum accumulator of the iteration precision
template <typename R>
__device__ __forceinline__ void norm2_site(ProdSum<R> &acc, const cx<R> v[3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        acc.add(v[c].re, v[c].re);
        acc.add(v[c].im, v[c].im);
    }
}

// phase-1 start: r = p_i = b (rounded to R), x_i = 0, b64 = b (in H); partials |r|^2 (R) and |b|^2 (FP64)
template <typename R, typename H>
__global__ void __launch_bounds__(kVecBlock) k_p1_init(const SysVecs *__restrict__ sv, int nshift)
{
    const SysVecs &V = sv[blockIdx.y];
    if ((int)(blockIdx.x * kVecBlock) >= V.Vh) return;
    int h = blockIdx.x * kVecBlock + threadIdx.x;
    ProdSum<R> pr;
    double pb = 0.0;
    if (h < V.Vh) {
        cx<R> v[3];
        cx<H> z[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double2 d = V.bcanon[(size_t)h * 3 + c];
            pb += d.x * d.x + d.y * d.y;
            v[c] = cx<R>{(R)d.x, (R)d.y};
            z[c] = cx<H>{H(0), H(0)};
        }
        norm2_site(pr, v);
        Field<R>::store(V.r, V.Vh, h, v);
        for (int i = 0; i < nshift; ++i) {
            Field<R>::store(V.p[i], V.Vh, h, v);
            Field<H>::store(V.x[i], V.Vh, h, z);
        }
        if (V.pstart) Field<R>::store(V.pstart, V.Vh, h, v);
        if (V.b64) {
            cx<H> w[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                double2 d = V.bcanon[(size_t)h * 3 + c];
                w[c] = cx<H>{H(d.x), H(d.y)};
            }
            Field<H>::store(V.b64, V.Vh, h, w);
        }
    }
    warp_partial(pr, h, V.Vh, V.part_v);
    warp_partial(pb, h, V.Vh, V.part_v2);
}

// Work list of the per-iteration vector kernels: the kVecBlock-site blocks of every system laid
// end to end (system s owns items [start[s], start[s+1])).  The kernels run persistently, each
// thread block striding over the items; items of systems that are not running are skipped at the
// cost of one flag read, so a batch of many systems does not launch hundreds of thousands of
// mostly idle blocks per iteration.
struct WorkList {
    const int *start;  // [nsys + 1]
    int nsys, total;
};

// first system whose items include `b`, scanning forward from `s` (items are visited in order)
__device__ __forceinline__ int advance_sys(const WorkList &w, int s, int b)
{
    while (s + 1 < w.nsys && w.start[s + 1] <= b) ++s;
    return s;
}

// r -= alpha q, partial |r|^2
template <typename R>
__global__ void __launch_bounds__(kVecBlock) k_update_r(const SysScal *__restrict__ sc, const SysVecs *__restrict__ sv,
                                                         const WorkList w)
{
    pdl_enter();
    int s = 0;
    for (int b = blockIdx.x; b < w.total; b += gridDim.x) {
        s = advance_sys(w, s, b);
        const SysScal &S = sc[s];
        if (!S.running) continue;  // uniform over the block
        const SysVecs &V = sv[s];
        const int lb = b - w.start[s];
        const int h = lb * kVecBlock + threadIdx.x;
        ProdSum<R> pr;
        if (h < V.Vh) {
            const R a = (R)S.alpha;
            // in a ring, r^(k+1) goes to the next slot and r^k stays for the window flush
            void *rin = V.nslot ? ring_slot<R>(V, S.iters) : V.r;
            void *rout = V.nslot ? ring_slot<R>(V, S.iters + 1) : V.r;
            cx<R> r[3], q[3];
            Field<R>::load_rw(rin, V.Vh, h, r);
            Field<R>::load_rw(V.q, V.Vh, h, q);
#pragma unroll
            for (int c = 0; c < 3; ++c) r[c] = cx<R>{fma(-a, q[c].re, r[c].re), fma(-a, q[c].im, r[c].im)};
            Field<R>::store(rout, V.Vh, h, r);
            norm2_site(pr, r);
        }
        warp_partial(pr, h, V.Vh, V.part_v);
    }
}

// x_i += cx_i p_i ; p_i = cr_i r + cp_i p_i  for the shifts flagged by k_beta.
// p_i and r are in the iteration precision R, the solutions x_i in X (FP64 or double-single, so
// that x_i keeps digits the FP32 search directions cannot).
template <typename R, typename X>
__global__ void __launch_bounds__(kVecBlock) k_update_shifts(const SysScal *__restrict__ sc,
                                                              const SysVecs *__restrict__ sv, const WorkList w)
{
    pdl_enter();
    __shared__ X s_cx[kMaxShifts];
    __shared__ R s_cr[kMaxShifts], s_cp[kMaxShifts];
    __shared__ int s_ux[kMaxShifts], s_up[kMaxShifts];
    int s = 0, loaded = -1;
    for (int b = blockIdx.x; b < w.total; b += gridDim.x) {
        s = advance_sys(w, s, b);
        const SysScal &S = sc[s];
        if (!S.running) continue;  // uniform over the block
        const SysVecs &V = sv[s];
        const int ns = S.nshift;
        if (loaded != s) {
            __syncthreads();  // previous item's readers are done with the coefficients
            if (threadIdx.x < ns) {
                s_cx[threadIdx.x] = X(S.cx[threadIdx.x]);
                s_cr[threadIdx.x] = (R)S.cr[threadIdx.x];
                s_cp[threadIdx.x] = (R)S.cp[threadIdx.x];
                s_ux[threadIdx.x] = S.upd_x[threadIdx.x];
                s_up[threadIdx.x] = S.upd_p[threadIdx.x];
            }
            __syncthreads();
            loaded = s;
        }
        const int h = (b - w.start[s]) * kVecBlock + threadIdx.x;
        if (h >= V.Vh) continue;
        cx<R> r[3];
        Field<R>::load_rw(V.r, V.Vh, h, r);
        for (int i = 0; i < ns; ++i) {
            const int ux = s_ux[i], up = s_up[i];
            if (!ux && !up) continue;
            cx<R> p[3];
            Field<R>::load_rw(V.p[i], V.Vh, h, p);
            if (ux) {
                cx<X> x[3];
                Field<X>::load_rw(V.x[i], V.Vh, h, x);
                const X a = s_cx[i];
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    x[c] = cx<X>{fma(a, X(p[c].re), x[c].re), fma(a, X(p[c].im), x[c].im)};
                Field<X>::store(V.x[i], V.Vh, h, x);
            }
            if (up) {
                const R zr = s_cr[i], bb = s_cp[i];
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    p[c] = cx<R>{fma(zr, r[c].re, bb * p[c].re), fma(zr, r[c].im, bb * p[c].im)};
                Field<R>::store(V.p[i], V.Vh, h, p);
            }
        }
    }
}

// Deferred multi-shift update (phase 1 of mixed solves).  Instead of moving x_i and p_i of every
// live shift each iteration, the residuals r^k of a window of n iterations stay in a ring and the
// window's scalars in a history; per iteration only the base direction p (the input of D) is
// updated.  Unrolling x_i += ax_t p_i ; p_i = pr_t r^(t) + pp_t p_i over the window t = 1..n gives
//   x_i <- x_i + sum_t a_t r^(t) + e P0_i ,   p_i <- sum_t d_t r^(t) + f P0_i
// with P0_i the p_i at the window start and, backwards from S_n = 0, P_n = 1,
//   a_t = pr_t S_t ,  d_t = pr_t P_t ,  S_{t-1} = ax_t + pp_t S_t ,  P_{t-1} = pp_t P_t ,  e = S_0 ,  f = P_0 :
// the same solutions in exact arithmetic, for 3 fields of traffic per iteration instead of 8 per
// live shift.  The window is flushed when it is full (p_i materialised for the next window) and at
// the end of the phase (x_i only).

// p = pr r^k + pp p for the base direction (r^k the newest ring slot)
template <typename R>
__global__ void __launch_bounds__(kVecBlock) k_update_pbase(const SysScal *__restrict__ sc,
                                                             const SysVecs *__restrict__ sv, const WorkList w)
{
    pdl_enter();
    int s = 0;
    for (int b = blockIdx.x; b < w.total; b += gridDim.x) {
        s = advance_sys(w, s, b);
        const SysScal &S = sc[s];
        if (!S.running || !S.upd_p[S.i0]) continue;  // uniform over the block
        const SysVecs &V = sv[s];
        const int h = (b - w.start[s]) * kVecBlock + threadIdx.x;
        if (h >= V.Vh) continue;
        const R zr = (R)S.cr[S.i0], bb = (R)S.cp[S.i0];
        cx<R> r[3], p[3];
        Field<R>::load_rw(ring_slot<R>(V, S.iters), V.Vh, h, r);
        Field<R>::load_rw(V.p[S.i0], V.Vh, h, p);
#pragma unroll
        for (int c = 0; c < 3; ++c) p[c] = cx<R>{fma(zr, r[c].re, bb * p[c].re), fma(zr, r[c].im, bb * p[c].im)};
        Field<R>::store(V.p[S.i0], V.Vh, h, p);
    }
}

// coefficients of a window flush, one warp per system, one lane per shift (backward recursion in FP64)
__global__ void k_flush_coef(SysScal *sc, const SysVecs *sv, int final_flush)
{
    SysScal &S = sc[blockIdx.x];
    const SysVecs &V = sv[blockIdx.x];
    FlushCoef &C = *V.coef;
    const int n = min(S.iters - S.win_start, kHistMax);
    const int i = threadIdx.x;
    if (i < S.nshift) {
        double sx = 0.0, pp = 1.0;
        int any = 0;
        for (int t = n - 1; t >= 0; --t) {
            const HistEntry h = V.hist[t * kMaxShifts + i];
            C.a[t][i] = (float)(h.pr * sx);
            C.d[t][i] = (float)(h.pr * pp);
            sx = h.ax + h.pp * sx;
            pp = h.pp * pp;
            any |= h.ax != 0.0;
        }
        C.e[i] = (float)sx;
        C.f[i] = (float)pp;
        C.xupd[i] = any;
        C.pmat[i] = !final_flush && n > 0 && i != S.i0 && S.active[i];
    }
    __syncwarp();
    if (threadIdx.x == 0) {
        C.n = n;
        C.first_slot = (S.win_start + 1) % V.nslot;
        S.win_start = S.iters;
    }
}

template <typename H>
__device__ __forceinline__ void fold_acc(H &acc, float v);
template <>
__device__ __forceinline__ void fold_acc<dsf>(dsf &acc, float v)
{
    const dsf t = ds_two_sum(acc.hi, v);
    acc = ds_fast_two_sum(t.hi, __fadd_rn(t.lo, acc.lo));
}
template <>
__device__ __forceinline__ void fold_acc<double>(double &acc, float v)
{
    acc += (double)v;
}

// One window flush over the complex elements of the FP32 fields (element e of a field is its
// float2 number e: colours 0, 1 of site e/2 for e < 2Vh, colour 2 of site e - 2Vh above), each thread
// block covering kFlushShifts shifts.  Sums of 8 terms are formed in FP32 and folded into an
// accumulator of the solution precision H.
template <typename H, bool MATP, bool PREFETCH>
__device__ __forceinline__ void flush_body(const SysScal *__restrict__ sc, const SysVecs *__restrict__ sv, int nchunk)
{
    __shared__ __align__(16) float s_a[kHistMax][kFlushShifts];
    __shared__ __align__(16) float s_d[MATP ? kHistMax : 1][kFlushShifts];
    __shared__ int s_any;
    const SysScal &S = sc[blockIdx.y];
    const SysVecs &V = sv[blockIdx.y];
    const FlushCoef &C = *V.coef;
    const int chunk = blockIdx.x % nchunk, eb = blockIdx.x / nchunk;
    const int i0c = chunk * kFlushShifts, nsc = min(kFlushShifts, S.nshift - i0c);
    const int nel = 3 * V.Vh;
    if (nsc <= 0 || eb * kVecBlock >= nel) return;  // uniform over the block
    const int n = C.n;
    if (threadIdx.x == 0) {
        int any = 0;
        for (int j = 0; j < nsc; ++j) any |= C.xupd[i0c + j] | (MATP ? C.pmat[i0c + j] | (i0c + j == S.i0) : 0);
        s_any = any;
    }
    for (int k = threadIdx.x; k < n * kFlushShifts; k += kVecBlock) {
        const int t = k / kFlushShifts, j = k % kFlushShifts;
        s_a[t][j] = j < nsc ? C.a[t][i0c + j] : 0.f;
        if constexpr (MATP) s_d[t][j] = j < nsc ? C.d[t][i0c + j] : 0.f;
    }
    __syncthreads();
    if (!s_any) return;
    const int e = eb * kVecBlock + threadIdx.x;
    if (e >= nel) return;

    float2 bx[kFlushShifts], bp[kFlushShifts];
    H ax[kFlushShifts], ay[kFlushShifts];
#pragma unroll
    for (int j = 0; j < kFlushShifts; ++j) {
        bx[j] = make_float2(0.f, 0.f);
        bp[j] = make_float2(0.f, 0.f);
        ax[j] = H(0);
        ay[j] = H(0);
    }
    int slot = C.first_slot;
    const int nslot = V.nslot;
    int pslot = PREFETCH ? (slot + 8) % nslot : 0;  // slot of the residual 8 iterations on
    const char *ring = static_cast<const char *>(V.r);
    for (int t0 = 0; t0 < n; t0 += 8) {
        const int m = min(8, n - t0);
        float2 rv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (u < m) {
                rv[u] = reinterpret_cast<const float2 *>(ring + (size_t)slot * V.slot_bytes)[e];
                if constexpr (PREFETCH) {
                    // the residual 8 slots on is requested into L2 now, so that the next group's
                    // loads find it there while this group's multiply-adds run (the same in-bounds
                    // slot and element that the next group loads)
                    if (t0 + 8 + u < n)
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const float2 *>(
                                         ring + (size_t)pslot * V.slot_bytes) + e));
                    pslot = pslot + 1 == nslot ? 0 : pslot + 1;
                }
                slot = slot + 1 == nslot ? 0 : slot + 1;
            } else {
                rv[u] = make_float2(0.f, 0.f);
            }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int t = t0 + u < n ? t0 + u : n - 1;  // rv[u] is zero past the end
            const float4 a0 = *reinterpret_cast<const float4 *>(&s_a[t][0]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&s_a[t][4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
            for (int j = 0; j < kFlushShifts; ++j) {
                bx[j].x = fmaf(av[j], rv[u].x, bx[j].x);
                bx[j].y = fmaf(av[j], rv[u].y, bx[j].y);
            }
            if constexpr (MATP) {
                const float4 d0 = *reinterpret_cast<const float4 *>(&s_d[t][0]);
                const float4 d1 = *reinterpret_cast<const float4 *>(&s_d[t][4]);
                const float dv[8] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
#pragma unroll
                for (int j = 0; j < kFlushShifts; ++j) {
                    bp[j].x = fmaf(dv[j], rv[u].x, bp[j].x);
                    bp[j].y = fmaf(dv[j], rv[u].y, bp[j].y);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < kFlushShifts; ++j) {
            fold_acc<H>(ax[j], bx[j].x);
            fold_acc<H>(ay[j], bx[j].y);
            bx[j] = make_float2(0.f, 0.f);
        }
    }
    // element e -> (site, colour) of the solution fields
    const int h = e < 2 * V.Vh ? e >> 1 : e - 2 * V.Vh;
    const int c = e < 2 * V.Vh ? e & 1 : 2;
#pragma unroll
    for (int j = 0; j < kFlushShifts; ++j) {
        const int i = i0c + j;
        if (j >= nsc) break;
        const bool base = i == S.i0;
        float2 *p0 = reinterpret_cast<float2 *>(base ? V.pstart : V.p[i]);
        const float2 pv = p0[e];
        if (C.xupd[i] || C.e[i] != 0.f) {
            fold_acc<H>(ax[j], C.e[i] * pv.x);
            fold_acc<H>(ay[j], C.e[i] * pv.y);
            if constexpr (std::is_same<H, dsf>::value) {
                float4 *xp = static_cast<float4 *>(V.x[i]) + (size_t)c * V.Vh + h;
                const float4 xv = *xp;
                const dsf re = dsf(xv.x, xv.y) + ax[j], im = dsf(xv.z, xv.w) + ay[j];
                *xp = make_float4(re.hi, re.lo, im.hi, im.lo);
            } else {
                double2 *xp = static_cast<double2 *>(V.x[i]) + (size_t)c * V.Vh + h;
                const double2 xv = *xp;
                *xp = make_double2(xv.x + ax[j], xv.y + ay[j]);
            }
        }
        if constexpr (MATP) {
            if (base) {
                p0[e] = reinterpret_cast<const float2 *>(V.p[i])[e];  // the explicit base direction
            } else if (C.pmat[i]) {
                p0[e] = make_float2(fmaf(C.f[i], pv.x, bp[j].x), fmaf(C.f[i], pv.y, bp[j].y));
            }
        }
    }
}

template <typename H, bool MATP>
__global__ void __launch_bounds__(kVecBlock) k_flush(const SysScal *__restrict__ sc, const SysVecs *__restrict__ sv,
                                                      int nchunk)
{
    flush_body<H, MATP, false>(sc, sv, nchunk);
}

// The final flush of the mixed solves (solutions only, double-single): each thread keeps one group
// of 8 residual loads in flight and requests the next group into L2 meanwhile, at three blocks of
// 80 registers per SM.
__global__ void __launch_bounds__(kVecBlock, 3) k_flush_final_ds(const SysScal *__restrict__ sc,
                                                                 const SysVecs *__restrict__ sv, int nchunk)
{
    flush_body<dsf, false, true>(sc, sv, nchunk);
}

// ------------------------------------------------------------------ scalar kernels (one warp per system)

__device__ __forceinline__ double warp_sum_strided(const double *a, int n)
{
    double s = 0.0;
    for (int k = threadIdx.x; k < n; k += 32) s += a[k];
    return warp_sum(s);
}

// Fixed-order sum of n partials by a whole block of NT threads (each thread a strided slice with
// eight independent accumulators, then a fixed tree), returned to every thread.  Many loads in
// flight: a one-warp sum of the 16384 partials of a 32^4 lattice is latency-bound at tens of
// microseconds.  NT = 256 by default (STG_SCALAR_BLOCK=1024 selects 1024-thread blocks, which
// wait longer for a free SM behind the previous kernel).
template <int kScalBlock>
__device__ __forceinline__ double block_sum_strided(const double *a, int n, double *sh)
{
    double s[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    int k = threadIdx.x;
    for (; k + 7 * kScalBlock < n; k += 8 * kScalBlock) {
#pragma unroll
        for (int u = 0; u < 8; ++u) s[u] += a[k + u * kScalBlock];
    }
#pragma unroll
    for (int u = 0; u < 7; ++u)
        if (k + u * kScalBlock < n) s[u] += a[k + u * kScalBlock];
    double t = block_sum(((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7])), sh);
    if (threadIdx.x == 0) sh[32] = t;
    __syncthreads();
    t = sh[32];
    __syncthreads();
    return t;
}

__device__ __forceinline__ int warp_sum_int(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// phase-1 scalar start
__global__ void k_p1_init_scal(SysScal *sc, const SysVecs *sv, int *done, double tol)
{
    SysScal &S = sc[blockIdx.x];
    const SysVecs &V = sv[blockIdx.x];
    const double rr = warp_sum_strided(V.part_v, V.npart_v);
    const double bb = warp_sum_strided(V.part_v2, V.npart_v);
    for (int i = threadIdx.x; i < S.nshift; i += 32) {
        S.zeta[i] = S.zeta_old[i] = S.zeta_new[i] = 1.0;
        S.active[i] = bb > 0.0;
        S.upd_x[i] = S.upd_p[i] = 0;
        S.shift_iters[i] = 0;
        S.cx[i] = S.cr[i] = S.cp[i] = 0.0;
    }
    if (threadIdx.x == 0) {
        S.rr = rr;
        S.bnorm2 = bb;
        S.tol2 = tol * tol * bb;
        S.alpha = 0.0;
        S.alpha_old = 1.0;
        S.beta_old = 0.0;
        S.iters = 0;
        S.running = 0;
        S.nactive = bb > 0.0 ? S.nshift : 0;
        done[blockIdx.x] = bb > 0.0 ? 0 : 1;
    }
}

template <int kScalBlock>
__global__ void __launch_bounds__(kScalBlock) k_alpha(SysScal *sc, const SysVecs *sv, const int *done)
{
    pdl_enter();
    SysScal &S = sc[blockIdx.x];
    if (done[blockIdx.x]) {
        if (threadIdx.x == 0) S.running = 0;
        return;
    }
    const SysVecs &V = sv[blockIdx.x];
    __shared__ double sh[33];
    const double pq = block_sum_strided<kScalBlock>(V.part_d, V.nblk_d, sh);
    if (threadIdx.x >= 32) return;  // the per-shift recurrences run in warp 0
    const double alpha = S.rr / pq;
    for (int i = threadIdx.x; i < S.nshift; i += 32) {
        if (!S.active[i]) continue;
        const double z = S.zeta[i], zo = S.zeta_old[i];
        const double zn = z * zo * S.alpha_old /
                          (alpha * S.beta_old * (zo - z) + zo * S.alpha_old * (1.0 + S.s[i] * alpha));
        S.zeta_new[i] = zn;
        S.cx[i] = alpha * zn / z;
    }
    if (threadIdx.x == 0) {
        S.alpha = alpha;
        S.running = 1;
    }
}

template <int kScalBlock>
__global__ void __launch_bounds__(kScalBlock) k_beta(SysScal *sc, const SysVecs *sv, int *done, int *need_rel,
                                                      double *log, int log_rows)
{
    pdl_enter();
    SysScal &S = sc[blockIdx.x];
    if (!S.running) return;
    const SysVecs &V = sv[blockIdx.x];
    __shared__ double sh[33];
    const double rr_new = block_sum_strided<kScalBlock>(V.part_v, V.npart_v, sh);
    if (threadIdx.x >= 32) return;  // the per-shift recurrences run in warp 0
    const double beta = rr_new / S.rr;
    const int ns = S.nshift;
    int nact = 0;
    for (int i = threadIdx.x; i < ns; i += 32) {
        if (S.active[i]) {
            const double z = S.zeta[i], zn = S.zeta_new[i];
            const double ratio = zn / z;
            S.cr[i] = zn;
            S.cp[i] = beta * ratio * ratio;
            S.upd_x[i] = 1;
            const bool conv = zn * zn * rr_new <= S.tol2;
            if (conv) {
                S.active[i] = 0;
                S.shift_iters[i] = S.iters + 1;
                S.upd_p[i] = 0;
            } else {
                S.upd_p[i] = 1;
                ++nact;
            }
            S.zeta_old[i] = z;
            S.zeta[i] = zn;
        } else {
            S.upd_x[i] = 0;
            S.upd_p[i] = 0;
        }
    }
    nact = warp_sum_int(nact);
    const bool cont = nact > 0 && S.iters + 1 < S.max_iter;
    const int slot = S.iters - S.win_start;  // deferred update: this iteration's history entry
    for (int i = threadIdx.x; i < ns; i += 32) {
        if (!cont) {
            S.upd_p[i] = 0;
        } else if (i == S.i0) {  // the base direction continues while any shift does
            S.upd_p[i] = 1;
            S.cr[i] = 1.0;
            S.cp[i] = beta;
        }
        if (V.hist != nullptr && slot < kHistMax) {
            HistEntry h;
            h.ax = S.upd_x[i] ? S.cx[i] : 0.0;
            h.pr = S.upd_p[i] ? S.cr[i] : 0.0;
            h.pp = S.upd_p[i] ? S.cp[i] : 1.0;
            V.hist[slot * kMaxShifts + i] = h;
        }
        if (log != nullptr && blockIdx.x == 0 && S.iters < log_rows)
            log[(size_t)S.iters * (2 + ns) + 2 + i] = S.upd_x[i] ? S.zeta[i] : 0.0;
    }
    __syncwarp();
    if (threadIdx.x == 0) {
        if (log != nullptr && blockIdx.x == 0 && S.iters < log_rows) {
            log[(size_t)S.iters * (2 + ns)] = S.alpha;
            log[(size_t)S.iters * (2 + ns) + 1] = beta;
        }
        S.alpha_old = S.alpha;
        S.beta_old = beta;
        S.rr = rr_new;
        S.iters += 1;
        S.nactive = nact;
        if (V.hist != nullptr && slot >= V.nslot - 1) S.hist_overflow = 1;
        if (!cont) done[blockIdx.x] = 1;
        if (S.phase2 && (!cont || rr_new < S.delta2 * S.rr_last)) need_rel[blockIdx.x] = 1;
    }
}

// ------------------------------------------------------------------ phase-2 kernels

// x_hi (H) += y (inner), y = 0   for pairs in the current reliable update
template <typename R, typename H>
__global__ void __launch_bounds__(kVecBlock) k_rel_fold(const SysVecs *__restrict__ sv, const int *__restrict__ noupd)
{
    if (noupd[blockIdx.y]) return;
    const SysVecs &V = sv[blockIdx.y];
    int h = blockIdx.x * kVecBlock + threadIdx.x;
    if (h >= V.Vh) return;
    cx<R> y[3], z[3];
    cx<H> x[3];
    Field<R>::load_rw(V.x[0], V.Vh, h, y);
    Field<H>::load_rw(V.xhi, V.Vh, h, x);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        x[c] = cx<H>{x[c].re + H(y[c].re), x[c].im + H(y[c].im)};
        z[c] = cx<R>{R(0), R(0)};
    }
    Field<H>::store(V.xhi, V.Vh, h, x);
    Field<R>::store(V.x[0], V.Vh, h, z);
}

// x_hi (H) += y, y_hi = y (H), y = 0: the anchored refinement then updates r_hi -= A y_hi
template <typename R, typename H>
__global__ void __launch_bounds__(kVecBlock) k_rel_fold_keep(const SysVecs *__restrict__ sv, const int *__restrict__ noupd)
{
    if (noupd[blockIdx.y]) return;
    const SysVecs &V = sv[blockIdx.y];
    int h = blockIdx.x * kVecBlock + threadIdx.x;
    if (h >= V.Vh) return;
    cx<R> y[3], z[3];
    cx<H> x[3], yh[3];
    Field<R>::load_rw(V.x[0], V.Vh, h, y);
    Field<H>::load_rw(V.xhi, V.Vh, h, x);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        yh[c] = cx<H>{H(y[c].re), H(y[c].im)};
        x[c] = cx<H>{x[c].re + yh[c].re, x[c].im + yh[c].im};
        z[c] = cx<R>{R(0), R(0)};
    }
    Field<H>::store(V.xhi, V.Vh, h, x);
    Field<H>::store(V.yhi, V.Vh, h, yh);
    Field<R>::store(V.x[0], V.Vh, h, z);
}

// after the FP64 residual r_hi = b - A x_hi (partials of |r_hi|^2 in part_d): decide per pair
__global__ void k_rel_finish(SysScal *sc, const SysVecs *sv, const int *noupd, int *done, int *need_rel,
                             int *finished, double *true_rr, int *rel_count)
{
    const int s = blockIdx.x;
    if (noupd[s]) return;
    SysScal &S = sc[s];
    const SysVecs &V = sv[s];
    const double rr = warp_sum_strided(V.part_d, V.nblk_d);
    if (threadIdx.x == 0) {
        true_rr[s] = rr;
        rel_count[s] += 1;
        need_rel[s] = 0;
        // stagnation guard: give up after 8 consecutive updates without halving the best residual
        if (rel_count[s] == 1 || rr < 0.25 * S.rr_best) {
            S.rr_best = rr;
            S.stalls = 0;
        } else {
            S.stalls += 1;
        }
        if (rr <= S.tol2_true || S.iters >= S.max_iter || S.stalls >= 8) {
            finished[s] = 1;
            done[s] = 1;
        } else {
            done[s] = 0;
            S.active[0] = 1;
            S.nactive = 1;
        }
    }
}

// r = inner(r_hi) (and, at the start of phase 2, p = r, y = 0); partial |r|^2
template <typename R, typename H>
__global__ void __launch_bounds__(kVecBlock) k_rel_copy(const SysVecs *__restrict__ sv, const int *__restrict__ noupd,
                                                         const int *__restrict__ finished, int start)
{
    const int s = blockIdx.y;
    const SysVecs &V = sv[s];
    if (noupd[s] || finished[s] || (int)(blockIdx.x * kVecBlock) >= V.Vh) return;
    int h = blockIdx.x * kVecBlock + threadIdx.x;
    ProdSum<R> pr;
    if (h < V.Vh) {
        cx<H> rh[3];
        cx<R> r[3];
        Field<H>::load_rw(V.rhi, V.Vh, h, rh);
#pragma unroll
        for (int c = 0; c < 3; ++c) r[c] = cx<R>{(R)rh[c].re, (R)rh[c].im};
        Field<R>::store(V.r, V.Vh, h, r);
        if (start) {
            cx<R> z[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) z[c] = cx<R>{R(0), R(0)};
            Field<R>::store(V.p[0], V.Vh, h, r);
            Field<R>::store(V.x[0], V.Vh, h, z);
        }
        norm2_site(pr, r);
    }
    warp_partial(pr, h, V.Vh, V.part_v);
}

__global__ void k_rel_scal(SysScal *sc, const SysVecs *sv, const int *noupd, const int *finished, int start)
{
    const int s = blockIdx.x;
    if (noupd[s] || finished[s]) return;
    SysScal &S = sc[s];
    const double rr = warp_sum_strided(sv[s].part_v, sv[s].npart_v);
    if (threadIdx.x == 0) {
        S.rr = rr;
        S.rr_last = rr;
        if (start) {
            S.zeta[0] = S.zeta_old[0] = S.zeta_new[0] = 1.0;
            S.s[0] = 0.0;
            S.active[0] = 1;
            S.nactive = 1;
            S.alpha_old = 1.0;
            S.beta_old = 0.0;
            S.iters = 0;
            S.running = 0;
        }
    }
}

// FP64 verification: true_rr = |r|^2 from the partials of the FP64 residual epilogue (pairs with
// noupd set were not verified and keep their double-single value)
__global__ void k_verify(const SysVecs *sv, double *true_rr, const int *noupd)
{
    if (noupd[blockIdx.x]) return;
    const double rr = warp_sum_strided(sv[blockIdx.x].part_d, sv[blockIdx.x].nblk_d);
    if (threadIdx.x == 0) true_rr[blockIdx.x] = rr;
}

// one (source, destination) field pair of a batched conversion
struct ConvPair {
    const void *src;
    void *dst;
    int Vh;
};

// field conversion src (type S) -> dst (type D), one (src, dst) pair per blockIdx.y; src may
// equal dst when both layouts have the same size (each thread rewrites its own 16-byte slots)
template <typename S, typename D>
__global__ void __launch_bounds__(kVecBlock) k_convert_pairs(const ConvPair *__restrict__ pr)
{
    const ConvPair &P = pr[blockIdx.y];
    int h = blockIdx.x * kVecBlock + threadIdx.x;
    if (h >= P.Vh) return;
    cx<S> v[3];
    cx<D> w[3];
    Field<S>::load_rw(P.src, P.Vh, h, v);
#pragma unroll
    for (int c = 0; c < 3; ++c) w[c] = cx<D>{D(v[c].re), D(v[c].im)};
    Field<D>::store(P.dst, P.Vh, h, w);
}

template <typename H>
__global__ void __launch_bounds__(kVecBlock) k_unpack_pairs(const ConvPair *__restrict__ pr)
{
    const ConvPair &P = pr[blockIdx.y];
    int h = blockIdx.x * kVecBlock + threadIdx.x;
    if (h >= P.Vh) return;
    cx<H> v[3];
    Field<H>::load_rw(P.src, P.Vh, h, v);
    double2 *o = static_cast<double2 *>(P.dst);
#pragma unroll
    for (int c = 0; c < 3; ++c) o[(size_t)h * 3 + c] = make_double2((double)v[c].re, (double)v[c].im);
}

// ------------------------------------------------------------------ host engine

namespace {

// Solve workspace: fields under 16 MiB are 256-byte-aligned pieces cut from 64 MiB chunks of the
// stream-ordered pool, larger ones pool blocks of their own (a batch asks for thousands of fields,
// and one pool call per field cost ~1 us of host time each, 3.7 ms for the 256-pair batch).
// Everything is released when the solve ends.
struct DevBuf {
    std::vector<void *> ptrs;
    cudaStream_t st = nullptr;
    cudaError_t err = cudaSuccess;
    char *cur = nullptr;
    size_t left = 0;
    static constexpr size_t kChunk = (size_t)64 << 20, kAlign = 256;
    void *alloc(size_t bytes)
    {
        if (err != cudaSuccess) return nullptr;
        bytes = (std::max<size_t>(bytes, 16) + kAlign - 1) & ~(kAlign - 1);
        if (bytes >= kChunk / 4) {  // large fields (residual rings) get pool blocks of their own
            void *p = nullptr;
            err = cudaMallocAsync(&p, bytes, st);
            if (err != cudaSuccess) return nullptr;
            ptrs.push_back(p);
            return p;
        }
        if (bytes > left) {
            const size_t want = std::max(bytes, kChunk);
            void *p = nullptr;
            err = cudaMallocAsync(&p, want, st);
            if (err != cudaSuccess) return nullptr;
            ptrs.push_back(p);
            cur = static_cast<char *>(p);
            left = want;
        }
        void *r = cur;
        cur += bytes;
        left -= bytes;
        return r;
    }
    ~DevBuf()
    {
        for (void *p : ptrs) cudaFreeAsync(p, st);
    }
};

struct InstInfo {
    const stg_gauge *gi;   // gauge of the multi-shift iterations
    const stg_gauge *gr;   // gauge of the refinement iterations
    const stg_gauge *g64;  // FP64 gauge
    const stg_gauge *gh;   // gauge of the true residuals (g64 or its double-single companion)
    int nrhs;
    int sys0;              // first phase-1 system of this instance
};

// D_oe / D_eo argument lists for a set of systems on their instances' gauges
struct DPlan {
    std::vector<DArgs> oe, eo;  // launched with modes 0 and (1 or 2)
};

// Appends a group to the launch list; out_par = 1 for D_oe lists, 0 for D_eo lists.
static void add_group(std::vector<DArgs> &lst, const DGroup &G, int out_par)
{
    if (lst.empty() || lst.back().ngroups == kMaxGroups) {
        DArgs a;
        memset(&a, 0, sizeof(a));
        a.out_par = out_par;
        lst.push_back(a);
    }
    DArgs &a = lst.back();
    a.grp[a.ngroups++] = G;
}

}  // namespace

// R: precision of the iterations (float: mixed solve, double: pure FP64 solve).
// H: precision of the solutions, sources and true residuals (double, or dsf for the mixed solve's
//    reliable updates, whose results are then verified in FP64; *retry_f64 is set when that
//    verification fails so the caller can repeat the solve with H = double).
template <typename R, typename H>
static stg_status solve_impl(int ninst, const stg_instance *inst, const stg_mscg_params *prm, cudaStream_t user_st,
                             bool *retry_f64)
{
    const bool mixed = !std::is_same<R, double>::value;
    constexpr bool kDS = std::is_same<H, dsf>::value;
    *retry_f64 = false;
    const int ns = prm->nshift;
    const double mass2 = prm->mass * prm->mass;
    double sigma0 = prm->shifts[0];
    int i0 = 0;
    for (int i = 1; i < ns; ++i)
        if (prm->shifts[i] < sigma0) { sigma0 = prm->shifts[i]; i0 = i; }

    std::vector<InstInfo> ii(ninst);
    int nsys = 0;
    for (int k = 0; k < ninst; ++k) {
        ii[k].g64 = inst[k].g_f64;
        ii[k].gi = mixed ? inst[k].g_inner : inst[k].g_f64;
        ii[k].gr = ii[k].gi;
        ii[k].nrhs = inst[k].nrhs;
        ii[k].sys0 = nsys;
        nsys += inst[k].nrhs;
    }
    const int npair = nsys * ns;
    const int kind_i = ii[0].gi->kind, kind_64 = ii[0].g64->kind;
    // 16-bit links are too coarse for the refinement to converge on ill-conditioned shifts
    // (their rounding error times the condition number exceeds one): refine on FP32 links.
    const bool refine_f32 = base_kind(kind_i) == kBF16R12 || base_kind(kind_i) == kF16R12;
    if (refine_f32)
        for (int k = 0; k < ninst; ++k) {
            stg_status s = f32_companion(ii[k].g64, user_st, &ii[k].gr);
            if (s != STG_OK) return s;
        }
    const int kind_r = ii[0].gr->kind;
    // operator of the true residuals: the F64 gauge, or its double-single companion
    for (int k = 0; k < ninst; ++k) {
        ii[k].gh = ii[k].g64;
        if (kDS) {
            stg_status s = ds_companion(ii[k].g64, user_st, &ii[k].gh);
            if (s != STG_OK) return s;
        }
    }
    const int kind_h = ii[0].gh->kind;
    // defaults measured on the 32^4, 16-pole workload (m = 0.01, tol 1e-10): the true residual of
    // the FP32 multi-shift solutions stalls near 3e-7 whatever the iterated residual, so the phase
    // stops at an iterated 1e-8 (175 iterations; 1e-9: 207, refinement 59 -> 70 iterations), and
    // reliable updates every three decades take 20 double-single residuals instead of 29 (0.0855 ->
    // 0.0818 s per solve; 1e-7 and 3e-8 were slower: the refinement grows faster than the phase
    // shrinks)
    const double inner_tol = mixed ? (prm->inner_tol > 0 ? prm->inner_tol
                                                          : (base_kind(kind_i) == kBF16R12 || base_kind(kind_i) == kF16R12 ? 1e-4 : 1e-8))
                                   : prm->tol;
    const double delta = prm->reliable_delta > 0 ? prm->reliable_delta : 1e-3;
    // A double-single residual certifies a shift on its own when tol exceeds tenfold a worst-case
    // bound e of its rounding error relative to |b| (64 operations of relative error 2^-44 on terms
    // of size (m^2 + sigma + 16) |x|, |x| <= |b| / (m^2 + sigma)).  When some shift's tol is below
    // that (tight solves), the refinement is anchored instead: one FP64 residual b - A x of each
    // multi-shift solution at its start, then each reliable update subtracts A y of the correction
    // y in double-single (an error of the order 2^-44 (m^2 + sigma + 16) |y|, |y| far below |x|),
    // with no FP64 operator afterwards.
    bool anchored = false;
    if (kDS)
        for (int i = 0; i < ns; ++i) {
            const double e = 64.0 * std::ldexp(1.0, -44) * (1.0 + 16.0 / (mass2 + prm->shifts[i]));
            if (prm->tol < 10.0 * e) anchored = true;
        }
    const int vb = Field<R>::kBytesPerSite;

    // The workspace comes from the device's default stream-ordered memory pool.  Keep up to
    // 64 GiB of freed pool memory mapped between solves (the default threshold of 0 returns it at
    // every synchronisation and the next solve pays for mapping it again).
    {
        int dev = 0;
        cudaMemPool_t pool;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = 64ull << 30;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        cudaGetLastError();
    }
    const bool verbose = getenv("STG_VERBOSE") && getenv("STG_VERBOSE")[0] == '1';
    auto t_start = std::chrono::steady_clock::now();
    auto stamp = [&](const char *what) {
        if (!verbose) return;
        double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
        fprintf(stderr, "[stg mscg] %8.3f ms  %s\n", ms, what);
    };

    // work stream ordered after the caller's stream
    cudaStream_t ws;
    STG_CUDA_TRY(cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking));
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamSynchronize(s); cudaStreamDestroy(s); }
    } sguard{ws};
    cudaEvent_t ev;
    STG_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    struct EventGuard {
        cudaEvent_t e;
        ~EventGuard() { cudaEventDestroy(e); }
    } eguard{ev};
    STG_CUDA_TRY(cudaEventRecord(ev, user_st));
    STG_CUDA_TRY(cudaStreamWaitEvent(ws, ev, 0));

    DevBuf mem;
    mem.st = ws;

    // ---------------- buffers
    std::vector<SysVecs> v1(nsys), v2(npair);
    std::vector<SysScal> s1(nsys), s2(npair);
    memset(v1.data(), 0, sizeof(SysVecs) * nsys);
    memset(v2.data(), 0, sizeof(SysVecs) * npair);
    memset(s1.data(), 0, sizeof(SysScal) * nsys);
    memset(s2.data(), 0, sizeof(SysScal) * npair);
    // Deferred multi-shift update (FP32 phase 1): window length W (a multiple of the chunk), ring of
    // W + 1 residuals per system; prm->history: 0 automatic (up to kHistMax within 16 GiB of rings),
    // 1 per-iteration updates, >= 8 that many residuals per window
    int hist_w = 0;
    if (std::is_same<R, float>::value && prm->history != 1) {
        size_t ring_field = 0;
        for (int k = 0; k < ninst; ++k)
            ring_field += (size_t)ii[k].nrhs * ii[k].g64->g.Vh * Field<R>::kBytesPerSite;
        if (prm->history >= 2) {
            hist_w = std::min(kHistMax, std::max(8, prm->history));
        } else {
            // slots that fit the budget, less the one holding the current residual (at least the
            // minimum window when even that does not fit)
            const size_t budget = (size_t)16 << 30;  // 16 GiB of the GPU's ~280 GB
            const size_t fit = budget / std::max<size_t>(ring_field, 1);
            hist_w = fit > 1 ? (int)std::min<size_t>(kHistMax, fit - 1) : 8;
        }
        hist_w = std::max(8, hist_w - hist_w % 8);
    }
    int nblkv_max = 0;
    for (int k = 0; k < ninst; ++k) {
        const int Vh = ii[k].g64->g.Vh;
        const int nbd = dslash_partials(Vh), nbv = (Vh + kVecBlock - 1) / kVecBlock, npv = (Vh + 31) / 32;
        nblkv_max = std::max(nblkv_max, nbv);
        const size_t fb = (size_t)Vh * vb, f64b = (size_t)Vh * 48;
        for (int r = 0; r < ii[k].nrhs; ++r) {
            const int s = ii[k].sys0 + r;
            SysVecs &V = v1[s];
            V.Vh = Vh;
            V.nblk_d = nbd;
            V.nblk_v = nbv;
            V.npart_v = npv;
            if (hist_w > 0) {
                V.nslot = hist_w + 1;
                V.slot_bytes = fb;
                V.r = mem.alloc(fb * V.nslot);
                V.pstart = mem.alloc(fb);
                V.hist = static_cast<HistEntry *>(mem.alloc(sizeof(HistEntry) * kHistMax * kMaxShifts));
                V.coef = static_cast<FlushCoef *>(mem.alloc(sizeof(FlushCoef)));
            } else {
                V.r = mem.alloc(fb);
            }
            V.q = mem.alloc(fb);
            V.t = mem.alloc(fb);
            for (int i = 0; i < ns; ++i) {
                V.p[i] = mem.alloc(fb);
                V.x[i] = nullptr;  // accumulated straight into the pair's x_hi (precision H)
            }
            V.b64 = mem.alloc(f64b);
            V.bcanon = static_cast<const double2 *>(inst[k].b[r]);
            V.part_d = static_cast<double *>(mem.alloc(sizeof(double) * nbd));
            V.part_v = static_cast<double *>(mem.alloc(sizeof(double) * npv));
            V.part_v2 = static_cast<double *>(mem.alloc(sizeof(double) * npv));
            SysScal &S = s1[s];
            S.nshift = ns;
            S.i0 = i0;
            S.max_iter = prm->max_iter;
            for (int i = 0; i < ns; ++i) S.s[i] = prm->shifts[i] - sigma0;
            S.coef = mass2 + sigma0;
            for (int i = 0; i < ns; ++i) {
                const int pidx = s * ns + i;
                SysVecs &W = v2[pidx];
                W.Vh = Vh;
                W.nblk_d = nbd;
                W.nblk_v = nbv;
                W.npart_v = npv;
                W.xhi = mem.alloc(f64b);
                V.x[i] = W.xhi;
                W.rhi = mem.alloc(f64b);
                W.yhi = anchored ? mem.alloc(f64b) : nullptr;
                W.t64 = mem.alloc(f64b);
                W.b64 = V.b64;
                W.part_d = static_cast<double *>(mem.alloc(sizeof(double) * nbd));
                W.part_v = static_cast<double *>(mem.alloc(sizeof(double) * npv));
                SysScal &P = s2[pidx];
                P.nshift = 1;
                P.i0 = 0;
                P.max_iter = prm->max_iter;
                P.phase2 = 1;
                P.delta2 = delta * delta;
                P.coef = mass2 + prm->shifts[i];
            }
        }
    }
    if (mem.err != cudaSuccess) return cuda_error(mem.err, "stg_mscg_solve: workspace allocation");

    SysVecs *d_v1 = static_cast<SysVecs *>(mem.alloc(sizeof(SysVecs) * nsys));
    SysScal *d_s1 = static_cast<SysScal *>(mem.alloc(sizeof(SysScal) * nsys));
    SysVecs *d_v2 = static_cast<SysVecs *>(mem.alloc(sizeof(SysVecs) * npair));
    SysScal *d_s2 = static_cast<SysScal *>(mem.alloc(sizeof(SysScal) * npair));
    // int flags: done1[nsys], need1[nsys], done2[npair], need2[npair], noupd[npair], finished[npair], relcnt[npair]
    int *d_flags = static_cast<int *>(mem.alloc(sizeof(int) * (2 * nsys + 5 * npair)));
    double *d_true_rr = static_cast<double *>(mem.alloc(sizeof(double) * npair));
    double *d_log = prm->log_rows > 0 ? static_cast<double *>(mem.alloc(sizeof(double) * prm->log_rows * (2 + ns)))
                                      : nullptr;
    ConvPair *d_pairs = static_cast<ConvPair *>(mem.alloc(sizeof(ConvPair) * (2 * npair + nsys)));
    if (mem.err != cudaSuccess) return cuda_error(mem.err, "stg_mscg_solve: workspace allocation");
    int *done1 = d_flags, *need1 = d_flags + nsys, *done2 = d_flags + 2 * nsys, *need2 = done2 + npair,
        *noupd = need2 + npair, *finished = noupd + npair, *relcnt = finished + npair;

    // phase-2 inner vectors (allocated after the FP64 ones so phase 1 stays compact)
    for (int s = 0; s < nsys; ++s)
        for (int i = 0; i < ns; ++i) {
            SysVecs &W = v2[s * ns + i];
            const size_t fb = (size_t)W.Vh * vb;
            W.r = mem.alloc(fb);
            W.q = mem.alloc(fb);
            W.t = mem.alloc(fb);
            W.p[0] = mem.alloc(fb);
            W.x[0] = mem.alloc(fb);
        }
    if (mem.err != cudaSuccess) return cuda_error(mem.err, "stg_mscg_solve: workspace allocation");

    STG_CUDA_TRY(cudaMemcpyAsync(d_v1, v1.data(), sizeof(SysVecs) * nsys, cudaMemcpyHostToDevice, ws));
    STG_CUDA_TRY(cudaMemcpyAsync(d_s1, s1.data(), sizeof(SysScal) * nsys, cudaMemcpyHostToDevice, ws));
    STG_CUDA_TRY(cudaMemcpyAsync(d_v2, v2.data(), sizeof(SysVecs) * npair, cudaMemcpyHostToDevice, ws));
    STG_CUDA_TRY(cudaMemcpyAsync(d_s2, s2.data(), sizeof(SysScal) * npair, cudaMemcpyHostToDevice, ws));
    STG_CUDA_TRY(cudaMemsetAsync(d_flags, 0, sizeof(int) * (2 * nsys + 5 * npair), ws));

    // ---------------- dslash plans
    // phase 1: rhs of one instance share link loads (groups of up to kMaxRhs)
    DPlan p1;
    for (int k = 0; k < ninst; ++k) {
        for (int r0 = 0; r0 < ii[k].nrhs; r0 += kMaxRhs) {
            DGroup Goe, Geo;
            memset(&Goe, 0, sizeof(Goe));
            Goe.g = ii[k].gi->g;
            Goe.links = ii[k].gi->links;
            Goe.nrhs = std::min(kMaxRhs, ii[k].nrhs - r0);
            Geo = Goe;
            for (int j = 0; j < Goe.nrhs; ++j) {
                const int s = ii[k].sys0 + r0 + j;
                Goe.in[j] = v1[s].p[i0];
                Goe.out[j] = v1[s].t;
                Goe.skip[j] = done1 + s;
                Geo.in[j] = v1[s].t;
                Geo.out[j] = v1[s].q;
                Geo.epi_p[j] = v1[s].p[i0];
                Geo.coef[j] = mass2 + sigma0;
                Geo.partial[j] = v1[s].part_d;
                Geo.skip[j] = done1 + s;
            }
            add_group(p1.oe, Goe, 1);
            add_group(p1.eo, Geo, 0);
        }
    }
    // phase 2: the (rhs, shift) pairs of one instance share link loads, in groups of `rg`
    // right-hand sides per thread (STG_REFINE_GROUP, 1..8, default 4: faster than 8 at 32^4)
    int rg = 4;
    if (const char *e = getenv("STG_REFINE_GROUP")) rg = std::max(1, std::min(kMaxRhs, atoi(e)));
    DPlan p2, p64, p64f;  // p64: residuals with gh; p64f: the same with the F64 gauge (verification)
    DPlan pinc;           // anchored refinement: r_hi = r_hi - A y_hi with gh
    for (int k = 0; k < ninst; ++k) {
        const int first = ii[k].sys0 * ns, cnt = ii[k].nrhs * ns;
        for (int q0 = 0; q0 < cnt; q0 += rg) {
            DGroup Goe, Geo, Hoe, Heo;
            memset(&Goe, 0, sizeof(Goe));
            Goe.g = ii[k].gr->g;
            Goe.links = ii[k].gr->links;
            Goe.nrhs = std::min(rg, cnt - q0);
            Geo = Goe;
            Hoe = Goe;
            Hoe.links = ii[k].gh->links;
            Heo = Hoe;
            for (int j = 0; j < Goe.nrhs; ++j) {
                const int pidx = first + q0 + j;
                const SysVecs &W = v2[pidx];
                Goe.in[j] = W.p[0];
                Goe.out[j] = W.t;
                Goe.skip[j] = done2 + pidx;
                Geo.in[j] = W.t;
                Geo.out[j] = W.q;
                Geo.epi_p[j] = W.p[0];
                Geo.coef[j] = s2[pidx].coef;
                Geo.partial[j] = W.part_d;
                Geo.skip[j] = done2 + pidx;
                // FP64 true residual r_hi = b - A x_hi
                Hoe.in[j] = W.xhi;
                Hoe.out[j] = W.t64;
                Hoe.skip[j] = noupd + pidx;
                Heo.in[j] = W.t64;
                Heo.out[j] = W.rhi;
                Heo.epi_p[j] = W.xhi;
                Heo.epi_b[j] = W.b64;
                Heo.coef[j] = s2[pidx].coef;
                Heo.partial[j] = W.part_d;
                Heo.skip[j] = noupd + pidx;
            }
            add_group(p2.oe, Goe, 1);
            add_group(p2.eo, Geo, 0);
            add_group(p64.oe, Hoe, 1);
            add_group(p64.eo, Heo, 0);
            if (anchored) {
                DGroup Ioe = Hoe, Ieo = Heo;
                for (int j = 0; j < Goe.nrhs; ++j) {
                    const SysVecs &W = v2[first + q0 + j];
                    Ioe.in[j] = W.yhi;
                    Ieo.epi_p[j] = W.yhi;
                    Ieo.epi_b[j] = W.rhi;  // out = r_hi - A y_hi, in place
                }
                add_group(pinc.oe, Ioe, 1);
                add_group(pinc.eo, Ieo, 0);
            }
            Hoe.links = Heo.links = ii[k].g64->links;
            add_group(p64f.oe, Hoe, 1);
            add_group(p64f.eo, Heo, 0);
        }
    }

    const dim3 vgrid1(nblkv_max, nsys), vgrid2(nblkv_max, npair);

    // work lists of the persistent per-iteration vector kernels (phase 1: systems, phase 2: pairs)
    WorkList wl1, wl2;
    {
        std::vector<int> st1(nsys + 1, 0), st2(npair + 1, 0);
        for (int s = 0; s < nsys; ++s) st1[s + 1] = st1[s] + v1[s].nblk_v;
        for (int q = 0; q < npair; ++q) st2[q + 1] = st2[q] + v2[q].nblk_v;
        int *d_st = static_cast<int *>(mem.alloc(sizeof(int) * (nsys + npair + 2)));
        if (mem.err != cudaSuccess) return cuda_error(mem.err, "stg_mscg_solve: workspace allocation");
        STG_CUDA_TRY(cudaMemcpyAsync(d_st, st1.data(), sizeof(int) * (nsys + 1), cudaMemcpyHostToDevice, ws));
        STG_CUDA_TRY(cudaMemcpyAsync(d_st + nsys + 1, st2.data(), sizeof(int) * (npair + 1), cudaMemcpyHostToDevice, ws));
        wl1 = WorkList{d_st, nsys, st1[nsys]};
        wl2 = WorkList{d_st + nsys + 1, npair, st2[npair]};
    }
    int nsm = 152;
    {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    }
    // persistent grids: exactly the blocks that fit at once (one wave), per kernel
    auto wave = [&](const void *kernel, int total) -> dim3 {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kVecBlock, 0) != cudaSuccess || per_sm < 1)
            per_sm = 1;
        return dim3(std::max(1, std::min(total, per_sm * nsm)));
    };
    const dim3 g_r1 = wave((const void *)k_update_r<R>, wl1.total), g_r2 = wave((const void *)k_update_r<R>, wl2.total);
    const dim3 g_s1 = wave((const void *)k_update_shifts<R, H>, wl1.total);
    const dim3 g_pb = wave((const void *)k_update_pbase<R>, wl1.total);
    const dim3 g_s2 = wave((const void *)k_update_shifts<R, R>, wl2.total);
    cudaGetLastError();

    const bool scal_wide = getenv("STG_SCALAR_BLOCK") && atoi(getenv("STG_SCALAR_BLOCK")) == 1024;
    auto iterate = [&](int kind, const DPlan &pl, SysScal *dS, SysVecs *dV, int *dn, int *nr, int n, dim3 /*vg*/,
                       double *log, int log_rows) -> cudaError_t {
        cudaError_t e;
        const bool ph1 = &pl == &p1;
        const WorkList &wl = ph1 ? wl1 : wl2;
        for (const DArgs &a : pl.oe)
            if ((e = launch_dslash(kind, a, 0, ws)) != cudaSuccess) return e;
        for (const DArgs &a : pl.eo)
            if ((e = launch_dslash(kind, a, 1, ws)) != cudaSuccess) return e;
        e = scal_wide ? launch_pdl(k_alpha<1024>, dim3(n), dim3(1024), ws, dS, (const SysVecs *)dV, (const int *)dn)
                      : launch_pdl(k_alpha<256>, dim3(n), dim3(256), ws, dS, (const SysVecs *)dV, (const int *)dn);
        if (e != cudaSuccess) return e;
        if ((e = launch_pdl(k_update_r<R>, ph1 ? g_r1 : g_r2, dim3(kVecBlock), ws, (const SysScal *)dS,
                            (const SysVecs *)dV, wl)) !=
            cudaSuccess)
            return e;
        e = scal_wide ? launch_pdl(k_beta<1024>, dim3(n), dim3(1024), ws, dS, (const SysVecs *)dV, dn, nr, log, log_rows)
                      : launch_pdl(k_beta<256>, dim3(n), dim3(256), ws, dS, (const SysVecs *)dV, dn, nr, log, log_rows);
        if (e != cudaSuccess) return e;
        if (ph1 && hist_w > 0)  // deferred multi-shift update: the base direction only
            e = launch_pdl(k_update_pbase<R>, g_pb, dim3(kVecBlock), ws, (const SysScal *)dS, (const SysVecs *)dV, wl);
        else if (ph1)  // multi-shift phase: solutions in H
            e = launch_pdl(k_update_shifts<R, H>, g_s1, dim3(kVecBlock), ws, (const SysScal *)dS, (const SysVecs *)dV, wl);
        else      // refinement: the correction y in R
            e = launch_pdl(k_update_shifts<R, R>, g_s2, dim3(kVecBlock), ws, (const SysScal *)dS, (const SysVecs *)dV, wl);
        return e;
    };

    // window flush of the deferred update (every system of phase 1)
    int nblke_max = 0;
    for (int q = 0; q < nsys; ++q) nblke_max = std::max(nblke_max, (3 * v1[q].Vh + kVecBlock - 1) / kVecBlock);
    const int nchunk = (ns + kFlushShifts - 1) / kFlushShifts;
    auto flush = [&](bool final_flush) -> cudaError_t {
        if (hist_w == 0) return cudaSuccess;
        k_flush_coef<<<nsys, 32, 0, ws>>>(d_s1, d_v1, final_flush ? 1 : 0);
        const dim3 g((unsigned)(nchunk * nblke_max), nsys);
        if (final_flush && std::is_same<H, dsf>::value)
            k_flush_final_ds<<<g, kVecBlock, 0, ws>>>(d_s1, d_v1, nchunk);
        else if (final_flush)
            k_flush<H, false><<<g, kVecBlock, 0, ws>>>(d_s1, d_v1, nchunk);
        else
            k_flush<H, true><<<g, kVecBlock, 0, ws>>>(d_s1, d_v1, nchunk);
        return cudaGetLastError();
    };

    // Chunks of `kChunk` iterations are captured once per phase into a CUDA graph and replayed;
    // converged systems make every kernel of the chunk a no-op, so overshooting is cheap.
    struct GraphCache {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        int state = 0;  // 0 not built, 1 graph, 2 direct launches
        ~GraphCache()
        {
            if (exec) cudaGraphExecDestroy(exec);
            if (graph) cudaGraphDestroy(graph);
        }
    };
    constexpr int kChunk = 8;
    // Runs chunks until every system's done flag is set (or, with stop_on_need, until some
    // system asks for a reliable update).
    auto run_until_done = [&](GraphCache &gc, int kind, const DPlan &pl, SysScal *dS, SysVecs *dV, int *dn, int *nr, int n,
                              dim3 vg, double *log, int log_rows, bool stop_on_need, std::vector<int> &h_done,
                              std::vector<int> &h_need, int flush_every = 0) -> stg_status {
        if (gc.state == 0) {
            // the D launches of one iteration, outside capture, settle the autotuned block sizes;
            // their outputs (t, q, partials) are recomputed by the first captured iteration
            for (const DArgs &a : pl.oe) STG_CUDA_TRY(launch_dslash(kind, a, 0, ws));
            for (const DArgs &a : pl.eo) STG_CUDA_TRY(launch_dslash(kind, a, 1, ws));
            gc.state = 2;
            if (cudaStreamBeginCapture(ws, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                cudaError_t e = cudaSuccess;
                for (int k = 0; k < kChunk && e == cudaSuccess; ++k)
                    e = iterate(kind, pl, dS, dV, dn, nr, n, vg, log, log_rows);
                cudaError_t e2 = cudaStreamEndCapture(ws, &gc.graph);
                if (e == cudaSuccess && e2 == cudaSuccess && cudaGraphInstantiate(&gc.exec, gc.graph, 0) == cudaSuccess)
                    gc.state = 1;
                else
                    cudaGetLastError();
            } else {
                cudaGetLastError();
            }
        }
        const long long cap = (long long)prm->max_iter / kChunk + 4;
        for (long long c = 0; c <= cap; ++c) {
            cudaError_t e = gc.state == 1 ? cudaGraphLaunch(gc.exec, ws) : cudaSuccess;
            for (int k = 0; gc.state != 1 && k < kChunk && e == cudaSuccess; ++k)
                e = iterate(kind, pl, dS, dV, dn, nr, n, vg, log, log_rows);
            if (e == cudaSuccess && flush_every > 0 && (c + 1) % flush_every == 0) e = flush(false);
            if (e == cudaSuccess) e = cudaMemcpyAsync(h_done.data(), dn, sizeof(int) * n, cudaMemcpyDeviceToHost, ws);
            if (e == cudaSuccess && stop_on_need)
                e = cudaMemcpyAsync(h_need.data(), nr, sizeof(int) * n, cudaMemcpyDeviceToHost, ws);
            if (e == cudaSuccess) e = cudaStreamSynchronize(ws);
            if (e != cudaSuccess) return cuda_error(e, "stg_mscg_solve: iteration");
            bool all = true, any_need = false;
            for (int s = 0; s < n; ++s) {
                all &= h_done[s] != 0;
                if (stop_on_need) any_need |= h_need[s] != 0;
            }
            if (all || any_need) break;
        }
        return STG_OK;
    };
    GraphCache gc1, gc2;

    if (verbose) {
        cudaStreamSynchronize(ws);
        stamp("workspace ready");
    }
    // ---------------- phase 1
    k_p1_init<R, H><<<vgrid1, kVecBlock, 0, ws>>>(d_v1, ns);
    k_p1_init_scal<<<nsys, 32, 0, ws>>>(d_s1, d_v1, done1, inner_tol);
    STG_CUDA_TRY(cudaGetLastError());
    std::vector<int> h_done1(nsys), h_need1(nsys);
    stg_status st = run_until_done(gc1, kind_i, p1, d_s1, d_v1, done1, need1, nsys, vgrid1, d_log, prm->log_rows, false,
                                   h_done1, h_need1, hist_w / kChunk);
    if (st != STG_OK) return st;
    STG_CUDA_TRY(flush(true));
    stamp("phase 1 (multi-shift CG) done");

    // ---------------- phase 2: true residuals (precision H), refinement with reliable updates
    // per-pair |b|^2 and tolerances from phase 1
    {
        std::vector<SysScal> tmp(nsys);
        STG_CUDA_TRY(cudaMemcpyAsync(tmp.data(), d_s1, sizeof(SysScal) * nsys, cudaMemcpyDeviceToHost, ws));
        STG_CUDA_TRY(cudaStreamSynchronize(ws));
        for (int s = 0; s < nsys; ++s)
            if (tmp[s].hist_overflow) return set_error(STG_ERR_CUDA, "stg_mscg_solve: internal error: residual history overflow");
        for (int s = 0; s < nsys; ++s) {
            s1[s] = tmp[s];
            for (int i = 0; i < ns; ++i) {
                SysScal &P = s2[s * ns + i];
                P.bnorm2 = tmp[s].bnorm2;
                P.tol2_true = prm->tol * prm->tol * tmp[s].bnorm2;
                P.tol2 = 0.25 * P.tol2_true;
            }
        }
        STG_CUDA_TRY(cudaMemcpyAsync(d_s2, s2.data(), sizeof(SysScal) * npair, cudaMemcpyHostToDevice, ws));
    }
    std::vector<int> h_done2(npair, 1), h_need2(npair, 1), h_fin(npair, 0), h_noupd(npair, 0);
    // x_hi of every pair and b of every system between precision H and FP64, in place
    auto convert_xb = [&](bool to_f64, bool with_r) -> stg_status {
        std::vector<ConvPair> cp;
        for (int q = 0; q < npair; ++q) {
            cp.push_back(ConvPair{v2[q].xhi, v2[q].xhi, v2[q].Vh});
            if (with_r) cp.push_back(ConvPair{v2[q].rhi, v2[q].rhi, v2[q].Vh});
        }
        for (int s = 0; s < nsys; ++s) cp.push_back(ConvPair{v1[s].b64, v1[s].b64, v1[s].Vh});
        STG_CUDA_TRY(cudaMemcpyAsync(d_pairs, cp.data(), sizeof(ConvPair) * cp.size(), cudaMemcpyHostToDevice, ws));
        if (to_f64)
            k_convert_pairs<H, double><<<dim3(nblkv_max, (unsigned)cp.size()), kVecBlock, 0, ws>>>(d_pairs);
        else
            k_convert_pairs<double, H><<<dim3(nblkv_max, (unsigned)cp.size()), kVecBlock, 0, ws>>>(d_pairs);
        STG_CUDA_TRY(cudaGetLastError());
        return STG_OK;
    };
    auto reliable_update = [&](bool start) -> stg_status {
        STG_CUDA_TRY(cudaMemcpyAsync(noupd, h_noupd.data(), sizeof(int) * npair, cudaMemcpyHostToDevice, ws));
        if (anchored && start) {
            // the FP64 anchor: r_hi = b - A x_hi with the F64 gauge, then everything back to H
            stg_status cs = convert_xb(true, false);
            if (cs != STG_OK) return cs;
            for (const DArgs &a : p64f.oe) STG_CUDA_TRY(launch_dslash(kind_64, a, 0, ws));
            for (const DArgs &a : p64f.eo) STG_CUDA_TRY(launch_dslash(kind_64, a, 2, ws));
            cs = convert_xb(false, true);
            if (cs != STG_OK) return cs;
        } else if (anchored) {
            k_rel_fold_keep<R, H><<<vgrid2, kVecBlock, 0, ws>>>(d_v2, noupd);
            for (const DArgs &a : pinc.oe) STG_CUDA_TRY(launch_dslash(kind_h, a, 0, ws));
            for (const DArgs &a : pinc.eo) STG_CUDA_TRY(launch_dslash(kind_h, a, 2, ws));
        } else {
            if (!start) k_rel_fold<R, H><<<vgrid2, kVecBlock, 0, ws>>>(d_v2, noupd);
            for (const DArgs &a : p64.oe) STG_CUDA_TRY(launch_dslash(kind_h, a, 0, ws));
            for (const DArgs &a : p64.eo) STG_CUDA_TRY(launch_dslash(kind_h, a, 2, ws));
        }
        k_rel_finish<<<npair, 32, 0, ws>>>(d_s2, d_v2, noupd, done2, need2, finished, d_true_rr, relcnt);
        k_rel_copy<R, H><<<vgrid2, kVecBlock, 0, ws>>>(d_v2, noupd, finished, start ? 1 : 0);
        k_rel_scal<<<npair, 32, 0, ws>>>(d_s2, d_v2, noupd, finished, start ? 1 : 0);
        STG_CUDA_TRY(cudaGetLastError());
        STG_CUDA_TRY(cudaMemcpyAsync(h_fin.data(), finished, sizeof(int) * npair, cudaMemcpyDeviceToHost, ws));
        STG_CUDA_TRY(cudaStreamSynchronize(ws));
        return STG_OK;
    };
    // every pair starts with a true-residual check
    st = reliable_update(true);
    if (st != STG_OK) return st;
    stamp("FP64 residuals of the multi-shift solutions done");
    std::vector<double> trr0(npair);
    STG_CUDA_TRY(cudaMemcpy(trr0.data(), d_true_rr, sizeof(double) * npair, cudaMemcpyDeviceToHost));
    int rounds = 0;
    const long long rel_cap = 4LL * prm->max_iter + 64;
    for (long long round = 0; round < rel_cap; ++round) {
        bool all = true;
        for (int q = 0; q < npair; ++q) all &= h_fin[q] != 0;
        if (all) break;
        st = run_until_done(gc2, kind_r, p2, d_s2, d_v2, done2, need2, npair, vgrid2, nullptr, 0, true, h_done2, h_need2);
        if (st != STG_OK) return st;
        bool any = false;
        for (int q = 0; q < npair; ++q) {
            h_noupd[q] = (h_need2[q] && !h_fin[q]) ? 0 : 1;
            any |= h_noupd[q] == 0;
        }
        if (!any) {
            // nothing flagged yet: every live pair is still iterating
            bool live = false;
            for (int q = 0; q < npair; ++q) live |= !h_fin[q] && !h_done2[q];
            if (!live) break;
            continue;
        }
        st = reliable_update(false);
        if (st != STG_OK) return st;
        ++rounds;
    }
    if (verbose) {
        char buf[96];
        snprintf(buf, sizeof buf, "phase 2 (refinement) done: %d reliable-update rounds", rounds);
        stamp(buf);
    }

    // ---------------- FP64 verification of double-single results
    if (kDS && anchored) {
        // the residuals are FP64-anchored: no further operator (the output unpack widens x_hi)
        stamp("anchored refinement: no FP64 verification needed");
    } else if (kDS) {
        // x_hi (per pair) and b (per system) to FP64 in place: same 48-byte site layout
        st = convert_xb(true, false);
        if (st != STG_OK) return st;
        // A pair's double-single residual certifies it on its own when tol exceeds tenfold a
        // worst-case bound e of that residual's rounding error relative to |b| (64 operations of
        // relative error 2^-44 on terms of size (m^2 + sigma + 16) |x|, |x| <= |b| / (m^2 + sigma))
        // and the residual is below (tol - e) |b|.  Only the other pairs get the FP64 residual
        // (loose tolerances, e.g. MD force solves, skip the FP64 operator entirely).
        std::vector<double> trr_ds(npair);
        STG_CUDA_TRY(cudaMemcpyAsync(trr_ds.data(), d_true_rr, sizeof(double) * npair, cudaMemcpyDeviceToHost, ws));
        STG_CUDA_TRY(cudaStreamSynchronize(ws));
        bool any_verify = false;
        for (int q = 0; q < npair; ++q) {
            const double sm = mass2 + prm->shifts[q % ns];
            const double e = 64.0 * std::ldexp(1.0, -44) * (1.0 + 16.0 / sm);
            const double margin = 1.0 - e / prm->tol;
            const bool cert = prm->tol >= 10.0 * e && h_fin[q] && trr_ds[q] <= s2[q].tol2_true * margin * margin;
            h_noupd[q] = cert ? 1 : 0;
            any_verify |= !cert;
        }
        STG_CUDA_TRY(cudaMemcpyAsync(noupd, h_noupd.data(), sizeof(int) * npair, cudaMemcpyHostToDevice, ws));
        if (any_verify) {
            for (const DArgs &a : p64f.oe) STG_CUDA_TRY(launch_dslash(kind_64, a, 0, ws));
            for (const DArgs &a : p64f.eo) STG_CUDA_TRY(launch_dslash(kind_64, a, 2, ws));
            k_verify<<<npair, 32, 0, ws>>>(d_v2, d_true_rr, noupd);
            STG_CUDA_TRY(cudaGetLastError());
        }
        std::vector<double> trr_f64(npair);
        STG_CUDA_TRY(cudaMemcpyAsync(trr_f64.data(), d_true_rr, sizeof(double) * npair, cudaMemcpyDeviceToHost, ws));
        STG_CUDA_TRY(cudaStreamSynchronize(ws));
        for (int q = 0; q < npair; ++q)
            if (!h_noupd[q] && trr_f64[q] > s2[q].tol2_true && h_fin[q]) {
                std::vector<SysScal> one(1);
                STG_CUDA_TRY(cudaMemcpy(one.data(), d_s2 + q, sizeof(SysScal), cudaMemcpyDeviceToHost));
                if (one[0].iters < prm->max_iter) *retry_f64 = true;  // converged in DS, not in FP64
            }
        if (*retry_f64) {
            stamp("FP64 verification failed: repeating with FP64 reliable updates");
            return STG_OK;
        }
        stamp("FP64 verification done");
    }

    // ---------------- outputs and statistics
    {
        std::vector<ConvPair> cp(npair);
        for (int k = 0; k < ninst; ++k)
            for (int r = 0; r < ii[k].nrhs; ++r)
                for (int i = 0; i < ns; ++i) {
                    const int s = ii[k].sys0 + r, pidx = s * ns + i;
                    cp[pidx] = ConvPair{v2[pidx].xhi, inst[k].x[r * ns + i], v2[pidx].Vh};
                }
        STG_CUDA_TRY(cudaMemcpyAsync(d_pairs, cp.data(), sizeof(ConvPair) * npair, cudaMemcpyHostToDevice, ws));
        if (kDS && anchored)
            k_unpack_pairs<H><<<vgrid2, kVecBlock, 0, ws>>>(d_pairs);  // x_hi still double-single
        else
            k_unpack_pairs<double><<<vgrid2, kVecBlock, 0, ws>>>(d_pairs);  // x_hi is FP64 here
        STG_CUDA_TRY(cudaGetLastError());
    }
    std::vector<SysScal> f1(nsys), f2(npair);
    std::vector<double> trr(npair);
    std::vector<int> rc(npair);
    std::vector<double> hlog(prm->log_rows > 0 ? (size_t)prm->log_rows * (2 + ns) : 0);
    STG_CUDA_TRY(cudaMemcpyAsync(f1.data(), d_s1, sizeof(SysScal) * nsys, cudaMemcpyDeviceToHost, ws));
    STG_CUDA_TRY(cudaMemcpyAsync(f2.data(), d_s2, sizeof(SysScal) * npair, cudaMemcpyDeviceToHost, ws));
    STG_CUDA_TRY(cudaMemcpyAsync(trr.data(), d_true_rr, sizeof(double) * npair, cudaMemcpyDeviceToHost, ws));
    STG_CUDA_TRY(cudaMemcpyAsync(rc.data(), relcnt, sizeof(int) * npair, cudaMemcpyDeviceToHost, ws));
    if (d_log)
        STG_CUDA_TRY(cudaMemcpyAsync(hlog.data(), d_log, sizeof(double) * hlog.size(), cudaMemcpyDeviceToHost, ws));
    STG_CUDA_TRY(cudaStreamSynchronize(ws));
    if (d_log) {
        const int rows = std::min(prm->log_rows, f1[0].iters);
        memcpy(prm->scalar_log, hlog.data(), sizeof(double) * rows * (2 + ns));
    }

    bool conv = true;
    for (int k = 0; k < ninst; ++k)
        for (int r = 0; r < ii[k].nrhs; ++r) {
            const int s = ii[k].sys0 + r;
            stg_mscg_stats *S = inst[k].stats ? &inst[k].stats[r] : nullptr;
            int rel = 0, ref = 0;
            for (int i = 0; i < ns; ++i) {
                const int pidx = s * ns + i;
                const double bb = f1[s].bnorm2;
                const double res = bb > 0 ? std::sqrt(trr[pidx] / bb) : 0.0;
                conv &= res <= prm->tol;
                rel += std::max(0, rc[pidx] - 1);
                ref = std::max(ref, f2[pidx].iters);
                if (S && S->true_resid) S->true_resid[i] = res;
                if (S && S->inner_resid) S->inner_resid[i] = bb > 0 ? std::sqrt(trr0[pidx] / bb) : 0.0;
                if (S && S->shift_iters) S->shift_iters[i] = f1[s].shift_iters[i] ? f1[s].shift_iters[i] : f1[s].iters;
                if (S && S->refine_shift_iters) S->refine_shift_iters[i] = f2[pidx].iters;
                if (S && S->shift_reliable_updates) S->shift_reliable_updates[i] = std::max(0, rc[pidx] - 1);
            }
            if (S) {
                S->iters = f1[s].iters;
                S->reliable_updates = rel;
                S->refine_iters = ref;
                S->fp64_fallback = mixed && !kDS ? 1 : 0;
            }
        }
    STG_CUDA_TRY(cudaEventRecord(ev, ws));
    STG_CUDA_TRY(cudaStreamWaitEvent(user_st, ev, 0));
    stamp("outputs written");
    if (!conv) return set_error(STG_ERR_NOCONV, "stg_mscg_solve: a shift is above tol after max_iter");
    return STG_OK;
}

static stg_status validate(int ninst, const stg_instance *inst, const stg_mscg_params *prm, bool &mixed)
{
    if (!inst || !prm) return set_error(STG_ERR_ARG, "stg_mscg_solve: null pointer");
    if (ninst < 1 || ninst > 16) return set_error(STG_ERR_ARG, "stg_mscg_solve: ninst must be in 1..16");
    for (int k = 0; k < ninst; ++k)
        if (inst[k].g_f64 && geom_is_slab(inst[k].g_f64->g))
            return set_error(STG_ERR_SHAPE, "stg_mscg_solve: not available on a slab lattice (see slab.py)");
    if (prm->nshift < 1 || prm->nshift > kMaxShifts || !prm->shifts)
        return set_error(STG_ERR_ARG, "stg_mscg_solve: nshift must be in 1..32 with a shifts array");
    for (int i = 0; i < prm->nshift; ++i)
        if (!(prm->shifts[i] >= 0.0) || !std::isfinite(prm->shifts[i]))
            return set_error(STG_ERR_ARG, "stg_mscg_solve: shifts must be finite and >= 0");
    if (!std::isfinite(prm->mass) || !(prm->tol > 0.0) || prm->max_iter < 1)
        return set_error(STG_ERR_ARG, "stg_mscg_solve: need finite mass, tol > 0, max_iter > 0");
    if (prm->history < 0) return set_error(STG_ERR_ARG, "stg_mscg_solve: history must be >= 0");
    if (prm->log_rows < 0 || (prm->log_rows > 0 && !prm->scalar_log))
        return set_error(STG_ERR_ARG, "stg_mscg_solve: scalar_log required when log_rows > 0");
    mixed = inst[0].g_inner != nullptr;
    int kind_i = -1, kind_64 = -1;
    for (int k = 0; k < ninst; ++k) {
        const stg_instance &I = inst[k];
        if (!I.g_f64 || !I.b || !I.x) return set_error(STG_ERR_ARG, "stg_mscg_solve: null gauge/b/x");
        if (!kind_is_f64(I.g_f64->kind)) return set_error(STG_ERR_ARG, "stg_mscg_solve: g_f64 must be an F64 gauge");
        if ((I.g_inner != nullptr) != mixed)
            return set_error(STG_ERR_ARG, "stg_mscg_solve: all instances must be mixed, or none");
        if (I.nrhs < 1 || I.nrhs > 16) return set_error(STG_ERR_ARG, "stg_mscg_solve: nrhs must be in 1..16");
        if (kind_64 >= 0 && I.g_f64->kind != kind_64)
            return set_error(STG_ERR_ARG, "stg_mscg_solve: all FP64 gauges must share one storage kind");
        kind_64 = I.g_f64->kind;
        if (mixed) {
            if (kind_is_f64(I.g_inner->kind))
                return set_error(STG_ERR_ARG, "stg_mscg_solve: g_inner must be an F32, BF16 or F16 gauge");
            for (int d = 0; d < 4; ++d)
                if (I.g_inner->g.L[d] != I.g_f64->g.L[d] || I.g_inner->g.antiperiodic != I.g_f64->g.antiperiodic)
                    return set_error(STG_ERR_SHAPE, "stg_mscg_solve: g_inner and g_f64 lattices differ");
            if (kind_i >= 0 && I.g_inner->kind != kind_i)
                return set_error(STG_ERR_ARG, "stg_mscg_solve: all inner gauges must share one storage kind");
            kind_i = I.g_inner->kind;
        }
        for (int r = 0; r < I.nrhs; ++r) {
            if (!I.b[r] || (reinterpret_cast<uintptr_t>(I.b[r]) & 15))
                return set_error(STG_ERR_ARG, "stg_mscg_solve: b must be non-null and 16-byte aligned");
            for (int i = 0; i < prm->nshift; ++i) {
                const void *x = I.x[r * prm->nshift + i];
                if (!x || (reinterpret_cast<uintptr_t>(x) & 15))
                    return set_error(STG_ERR_ARG, "stg_mscg_solve: x must be non-null and 16-byte aligned");
                if (x == I.b[r]) return set_error(STG_ERR_ARG, "stg_mscg_solve: x may not alias b");
            }
        }
    }
    return STG_OK;
}

}  // namespace stg

using namespace stg;

extern "C" {

stg_status stg_mscg_solve_batched(int32_t ninst, const stg_instance *inst, const stg_mscg_params *params, void *stream)
{
    bool mixed = false;
    stg_status s = validate(ninst, inst, params, mixed);
    if (s != STG_OK) return s;
    bool retry = false;
    if (!mixed) return solve_impl<double, double>(ninst, inst, params, (cudaStream_t)stream, &retry);
    // mixed: reliable updates in double-single, every result verified in FP64; if a shift passes
    // in double-single but not in FP64 (a very ill-conditioned shift), redo with FP64 updates
    s = solve_impl<float, dsf>(ninst, inst, params, (cudaStream_t)stream, &retry);
    if (s != STG_OK || !retry) return s;
    return solve_impl<float, double>(ninst, inst, params, (cudaStream_t)stream, &retry);
}

stg_status stg_mscg_solve(const stg_gauge *g_f64, const stg_gauge *g_inner, const stg_mscg_params *params,
                          const void *b_c128_dev, void *const *x_c128_dev, stg_mscg_stats *stats, void *stream)
{
    if (!g_f64 || !params || !b_c128_dev || !x_c128_dev) return set_error(STG_ERR_ARG, "stg_mscg_solve: null pointer");
    const void *b[1] = {b_c128_dev};
    stg_instance in;
    in.g_f64 = g_f64;
    in.g_inner = g_inner;
    in.nrhs = 1;
    in.b = b;
    in.x = x_c128_dev;
    in.stats = stats;
    return stg_mscg_solve_batched(1, &in, params, stream);
}

}  // extern "C"
