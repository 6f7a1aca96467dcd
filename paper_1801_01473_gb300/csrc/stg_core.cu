// stg_core.cu -- C ABI: lattice and gauge handles, field packing, D_eo / D_oe and the
// shifted normal operator (Sec. 2, Eq. shift_eo; link compression and phases, Sec. 4.1).
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <type_traits>
#include <new>
#include <string>
#include <tuple>

#include "stg_common.h"

namespace stg {

static thread_local std::string g_last_error;

stg_status set_error(stg_status s, const std::string &msg)
{
    g_last_error = msg;
    return s;
}

stg_status cuda_error(cudaError_t e, const char *where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return set_error(e == cudaErrorMemoryAllocation ? STG_ERR_OOM : STG_ERR_CUDA, m);
}

int link_bytes(int kind)
{
    if (kind_has_u1(kind)) {
        const int b = link_bytes(base_kind(kind));
        return b ? b + theta_bytes(kind) : 0;
    }
    switch (kind) {
    case kF64R18: return LinkF64R18::kBytes;
    case kF64R12: return LinkF64R12::kBytes;
    case kF32R18: return LinkF32R18::kBytes;
    case kF32R12: return LinkF32R12::kBytes;
    case kBF16R12: return Link16R12<__nv_bfloat16>::kBytes;
    case kF16R12: return Link16R12<__half>::kBytes;
    case kDSR18: return LinkDSR18::kBytes;
    case kDSR12: return LinkDSR12::kBytes;
    }
    return 0;
}

cudaError_t launch_dslash_bs(int kind, const DArgs &a, int mode, int bs, cudaStream_t st)
{
    if (kind_has_u1(kind)) return launch_dslash_u1(kind, a, mode, bs, st);
    switch (kind) {
    case kF64R18: return launch_dslash_f64r18(a, mode, bs, st);
    case kF64R12: return launch_dslash_f64r12(a, mode, bs, st);
    case kF32R18: return launch_dslash_f32r18(a, mode, bs, st);
    case kF32R12: return launch_dslash_f32r12(a, mode, bs, st);
    case kBF16R12: return launch_dslash_bf16r12(a, mode, bs, st);
    case kF16R12: return launch_dslash_f16r12(a, mode, bs, st);
    case kDSR18: return launch_dslash_dsr18(a, mode, bs, st);
    case kDSR12: return launch_dslash_dsr12(a, mode, bs, st);
    }
    return cudaErrorInvalidValue;
}

bool pdl_enabled()
{
    static const bool on = [] {
        const char *e = getenv("STG_PDL");
        return !(e && e[0] == '0');
    }();
    return on;
}

// Launch-shape autotuner of the D kernel.  Keyed by (device, storage kind, epilogue, rhs
// template, largest Vh of the launch): the first launch of a key outside stream capture runs
// the kernel with 64-, 128- and 256-thread blocks and, for several right-hand sides on FP32 /
// 16-bit links, the shared-link operator and (FP32 12-real, 3-4 rhs) the one-hop-lookahead loop
// (each launch recomputes the same outputs, so the
// repetition is harmless; launches that update an input in place are never tuned), times them
// with CUDA events on the launch stream and keeps the fastest.  Launches during capture use the tuned size when known, else 128.  STG_AUTOTUNE=0
// disables tuning.
namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int>, int> g_tuned;
}  // namespace

static cudaError_t launch_dslash_tuned(int kind, const DArgs &a, int mode, cudaStream_t st);

// Double-single D is bound by the FP32 pipes, not by link traffic: several right-hand sides per
// thread only cost registers and occupancy (measured: 4 rhs per thread run at half the per-rhs
// speed of 1).  Its multi-rhs launches are therefore split into one-rhs groups, and so are those
// of links with a U(1) phase field (instantiated for one rhs only).
cudaError_t launch_dslash(int kind, const DArgs &a, int mode, cudaStream_t st)
{
    int maxv, maxr;
    dslash_extent(a, maxv, maxr);
    if ((!kind_is_ds(kind) && !kind_has_u1(kind)) || maxr <= 1) return launch_dslash_tuned(kind, a, mode, st);
    DArgs b;
    memset(&b, 0, sizeof(b));
    b.out_par = a.out_par;
    for (int k = 0; k < a.ngroups; ++k) {
        const DGroup &G = a.grp[k];
        for (int j = 0; j < G.nrhs; ++j) {
            DGroup &H = b.grp[b.ngroups++];
            H = G;
            H.nrhs = 1;
            H.in[0] = G.in[j];
            H.out[0] = G.out[j];
            H.epi_p[0] = G.epi_p[j];
            H.epi_b[0] = G.epi_b[j];
            H.coef[0] = G.coef[j];
            H.partial[0] = G.partial[j];
            H.skip[0] = G.skip[j];
            if (b.ngroups == kMaxGroups) {
                cudaError_t e = launch_dslash_tuned(kind, b, mode, st);
                if (e != cudaSuccess) return e;
                b.ngroups = 0;
            }
        }
    }
    return b.ngroups ? launch_dslash_tuned(kind, b, mode, st) : cudaSuccess;
}

static cudaError_t launch_dslash_tuned(int kind, const DArgs &a, int mode, cudaStream_t st)
{
    int maxv, maxr;
    dslash_extent(a, maxv, maxr);
    if (a.ngroups <= 0 || maxv <= 0 || maxr <= 0) return cudaSuccess;
    const int nt = dslash_nrhs_template(maxr);
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_tuple(dev, kind, mode, nt, maxv);
    // the lookahead kernel exists for FP32 12-real links with 3 or 4 right-hand sides
    const bool ahead_ok = kind == kF32R12 && nt == 4;
    // STG_DSLASH_SHAPE=64|128|256|shared|ahead fixes the launch shape (tests use it to run each variant)
    if (const char *fix = getenv("STG_DSLASH_SHAPE")) {
        const bool sh = strcmp(fix, "shared") == 0;
        if (sh && maxr >= 2 && !kind_has_u1(kind) && !kind_is_f64(kind) && !kind_is_ds(kind))
            return launch_dslash_bs(kind, a, mode, kSharedLinks, st);
        if (strcmp(fix, "ahead") == 0 && ahead_ok) return launch_dslash_bs(kind, a, mode, kLoadsAhead, st);
        const int bs = atoi(fix);
        if (bs == 64 || bs == 128 || bs == 256) return launch_dslash_bs(kind, a, mode, bs, st);
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) return launch_dslash_bs(kind, a, mode, it->second, st);
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        return launch_dslash_bs(kind, a, mode, kDslashBlock, st);
    // a launch that updates one of its own inputs in place (out aliasing epi_b, epi_p or in) must
    // run exactly once: it is not tuned (the default shape now, the tuned one once another launch
    // of the same key has been tuned)
    for (int k = 0; k < a.ngroups; ++k)
        for (int j = 0; j < a.grp[k].nrhs; ++j) {
            const DGroup &G = a.grp[k];
            if (G.out[j] == G.in[j] || G.out[j] == G.epi_b[j] || G.out[j] == G.epi_p[j])
                return launch_dslash_bs(kind, a, mode, kDslashBlock, st);
        }
    const char *env = getenv("STG_AUTOTUNE");
    int best = kDslashBlock;
    if (!(env && env[0] == '0')) {
        cudaEvent_t e0, e1;
        if (cudaEventCreate(&e0) != cudaSuccess) return cudaGetLastError();
        if (cudaEventCreate(&e1) != cudaSuccess) {
            cudaEventDestroy(e0);
            return cudaGetLastError();
        }
        float best_t = 1e30f;
        // the shared-link operator only for several right-hand sides on FP32 / 16-bit links
        const bool shared_ok = maxr >= 2 && !kind_has_u1(kind) && !kind_is_f64(kind) && !kind_is_ds(kind);
        const int cands[5] = {64, 128, 256, kSharedLinks, kLoadsAhead};
        // two passes over the candidates, each candidate keeping its faster pass: one pass of three
        // launches picked 256-thread blocks for the solver's 4-rhs D_eo in one process and 64 in
        // another (10 % apart per launch)
        float t_min[5] = {1e30f, 1e30f, 1e30f, 1e30f, 1e30f};
        for (int pass = 0; pass < 2; ++pass)
            for (int ci = 0; ci < 5; ++ci) {
                const int bs = cands[ci];
                if (bs == kSharedLinks && !shared_ok) continue;
                if (bs == kLoadsAhead && !ahead_ok) continue;
                cudaError_t e = launch_dslash_bs(kind, a, mode, bs, st);  // warm-up
                if (e == cudaSuccess) e = cudaEventRecord(e0, st);
                for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = launch_dslash_bs(kind, a, mode, bs, st);
                if (e == cudaSuccess) e = cudaEventRecord(e1, st);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) {
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    return e;
                }
                t_min[ci] = std::min(t_min[ci], ms);
            }
        for (int ci = 0; ci < 5; ++ci)
            if (t_min[ci] < best_t) {
                best_t = t_min[ci];
                best = cands[ci];
            }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[key] = best;
    }
    return launch_dslash_bs(kind, a, mode, best, st);
}

// ------------------------------------------------------------------ packing kernels

// One thread per link (mu, i): canonical [mu][i][3][3] complex128 -> block (mu, parity(i)) at i>>1.
template <typename LinkT>
__global__ void k_pack_links(Geom g, const double2 *__restrict__ canon, void *__restrict__ links)
{
    long long V = 2LL * g.Vh;
    long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= 4 * V) return;
    int mu = (int)(tid / V);
    int i = (int)(tid - (long long)mu * V);
    int x = i % g.L[0], r = i / g.L[0];
    int y = r % g.L[1], r2 = r / g.L[1];
    int z = r2 % g.L[2], t = r2 / g.L[2];
    int par = (x + y + z + t) & 1;
    double2 m[9];
    for (int k = 0; k < 9; ++k) m[k] = canon[tid * 9 + k];
    void *blk = static_cast<char *>(links) + (size_t)(mu * 2 + par) * g.Vh * LinkT::kBytes;
    LinkT::pack(blk, g.Vh, i >> 1, m);
}

template <typename LinkT>
static cudaError_t pack_links_t(const Geom &g, const void *canon, void *links, cudaStream_t st)
{
    long long n = 4LL * 2 * g.Vh;
    int bs = 256;
    k_pack_links<LinkT><<<(unsigned)((n + bs - 1) / bs), bs, 0, st>>>(g, static_cast<const double2 *>(canon), links);
    return cudaGetLastError();
}

// a phase in its stored form: the angle, or (cos, sin)
__device__ __forceinline__ void store_phase(float *p, double theta) { *p = (float)theta; }
__device__ __forceinline__ void store_phase(double2 *p, double theta)
{
    double sn, cs;
    sincos(theta, &sn, &cs);
    *p = make_double2(cs, sn);
}
__device__ __forceinline__ double angle_of(float t) { return (double)t; }
__device__ __forceinline__ double angle_of(double2 p) { return atan2(p.y, p.x); }

// canonical angles theta [4][V] (FP64) -> the phase chunk of every (mu, parity) block of a LinkU1 layout
template <typename LinkT>
__global__ void k_pack_theta(Geom g, const double *__restrict__ theta, void *__restrict__ links)
{
    using T = typename LinkT::Theta;
    long long V = 2LL * g.Vh;
    long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= 4 * V) return;
    int mu = (int)(tid / V);
    int i = (int)(tid - (long long)mu * V);
    int x = i % g.L[0], r = i / g.L[0];
    int y = r % g.L[1], r2 = r / g.L[1];
    int z = r2 % g.L[2], t = r2 / g.L[2];
    int par = (x + y + z + t) & 1;
    char *blk = static_cast<char *>(links) + (size_t)(mu * 2 + par) * g.Vh * LinkT::kBytes;
    T *th = reinterpret_cast<T *>(blk + (size_t)LinkT::BaseLink::kBytes * g.Vh);
    store_phase(th + (i >> 1), theta[tid]);
}

template <typename LinkT>
static cudaError_t pack_u1_t(const Geom &g, const void *canon, const double *theta, void *links, cudaStream_t st)
{
    cudaError_t e = pack_links_t<LinkT>(g, canon, links, st);
    if (e != cudaSuccess) return e;
    long long n = 8LL * g.Vh;
    k_pack_theta<LinkT><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, theta, links);
    return cudaGetLastError();
}

cudaError_t launch_pack_links_u1(int kind, const Geom &g, const void *canon, const double *theta, void *links,
                                 cudaStream_t st)
{
    switch (base_kind(kind)) {
    case kF64R18: return pack_u1_t<LinkU1<LinkF64R18, double2>>(g, canon, theta, links, st);
    case kF64R12: return pack_u1_t<LinkU1<LinkF64R12, double2>>(g, canon, theta, links, st);
    case kF32R18: return pack_u1_t<LinkU1<LinkF32R18, float>>(g, canon, theta, links, st);
    case kF32R12: return pack_u1_t<LinkU1<LinkF32R12, float>>(g, canon, theta, links, st);
    case kBF16R12: return pack_u1_t<LinkU1<Link16R12<__nv_bfloat16>, float>>(g, canon, theta, links, st);
    case kF16R12: return pack_u1_t<LinkU1<Link16R12<__half>, float>>(g, canon, theta, links, st);
    case kDSR18: return pack_u1_t<LinkU1<LinkDSR18, double2>>(g, canon, theta, links, st);
    case kDSR12: return pack_u1_t<LinkU1<LinkDSR12, double2>>(g, canon, theta, links, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_pack_links(int kind, const Geom &g, const void *canon, void *links, cudaStream_t st)
{
    switch (kind) {
    case kF64R18: return pack_links_t<LinkF64R18>(g, canon, links, st);
    case kF64R12: return pack_links_t<LinkF64R12>(g, canon, links, st);
    case kF32R18: return pack_links_t<LinkF32R18>(g, canon, links, st);
    case kF32R12: return pack_links_t<LinkF32R12>(g, canon, links, st);
    case kBF16R12: return pack_links_t<Link16R12<__nv_bfloat16>>(g, canon, links, st);
    case kF16R12: return pack_links_t<Link16R12<__half>>(g, canon, links, st);
    case kDSR18: return pack_links_t<LinkDSR18>(g, canon, links, st);
    case kDSR12: return pack_links_t<LinkDSR12>(g, canon, links, st);
    }
    return cudaErrorInvalidValue;
}

// Phase chunk copy between two LinkU1 layouts (no-op for links without phases).
template <typename SrcT, typename DstT>
__device__ __forceinline__ void copy_theta(const char *sblk, char *dblk, int Vh, int h)
{
    if constexpr (LinkTraits<SrcT>::kU1) {
        using SB = typename LinkTraits<SrcT>::Base;
        using DB = typename LinkTraits<DstT>::Base;
        const typename SrcT::Theta v = reinterpret_cast<const typename SrcT::Theta *>(sblk + (size_t)SB::kBytes * Vh)[h];
        typename DstT::Theta *d = reinterpret_cast<typename DstT::Theta *>(dblk + (size_t)DB::kBytes * Vh) + h;
        if constexpr (std::is_same<typename SrcT::Theta, typename DstT::Theta>::value)
            *d = v;
        else
            store_phase(d, angle_of(v));
    }
}

// internal F64 links -> internal F32 12-real links (one thread per link); phases copied as floats
template <typename SrcT, typename DstT>
__global__ void k_links_to_f32r12(Geom g, const void *__restrict__ src, void *__restrict__ dst)
{
    const int Vh = g.Vh;
    long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= 8LL * Vh) return;
    const int blk = (int)(tid / Vh), h = (int)(tid - (long long)blk * Vh);
    const char *sblk = static_cast<const char *>(src) + (size_t)blk * Vh * SrcT::kBytes;
    char *dblk = static_cast<char *>(dst) + (size_t)blk * Vh * DstT::kBytes;
    cx<double> U[3][3];
    LinkTraits<SrcT>::Base::load(sblk, Vh, h, U);  // without the phase
    double2 m[9];
    for (int k = 0; k < 9; ++k) m[k] = make_double2(U[k / 3][k % 3].re, U[k / 3][k % 3].im);
    LinkF32R12::pack(dblk, Vh, h, m);
    copy_theta<SrcT, DstT>(sblk, dblk, Vh, h);
}

// internal F64 links -> internal double-single links of the same compression (and phases)
template <typename SrcT, typename DstT>
__global__ void k_links_to_ds(Geom g, const void *__restrict__ src, void *__restrict__ dst)
{
    using DB = typename LinkTraits<DstT>::Base;
    const int Vh = g.Vh;
    long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= 8LL * Vh) return;
    const int blk = (int)(tid / Vh), h = (int)(tid - (long long)blk * Vh);
    const char *sblk = static_cast<const char *>(src) + (size_t)blk * Vh * SrcT::kBytes;
    char *dblk = static_cast<char *>(dst) + (size_t)blk * Vh * DstT::kBytes;
    const double2 *p = reinterpret_cast<const double2 *>(sblk);
    double2 m[9];
    for (int k = 0; k < DB::kBytes / 16; ++k) m[k] = p[(size_t)k * Vh + h];
    DB::pack(dblk, Vh, h, m);
    copy_theta<SrcT, DstT>(sblk, dblk, Vh, h);
}

// (re)fill the companions of an F64 gauge from its links
static cudaError_t fill_ds_companion(const stg_gauge *g64, stg_gauge *g, cudaStream_t st)
{
    const long long n = 8LL * g->g.Vh;
    const unsigned nb = (unsigned)((n + 255) / 256);
    switch (g64->kind) {
    case kF64R18: k_links_to_ds<LinkF64R18, LinkDSR18><<<nb, 256, 0, st>>>(g->g, g64->links, g->links); break;
    case kF64R12: k_links_to_ds<LinkF64R12, LinkDSR12><<<nb, 256, 0, st>>>(g->g, g64->links, g->links); break;
    case kF64R18 | kU1:
        k_links_to_ds<LinkU1<LinkF64R18, double2>, LinkU1<LinkDSR18, double2>><<<nb, 256, 0, st>>>(g->g, g64->links, g->links);
        break;
    default:
        k_links_to_ds<LinkU1<LinkF64R12, double2>, LinkU1<LinkDSR12, double2>><<<nb, 256, 0, st>>>(g->g, g64->links, g->links);
        break;
    }
    return cudaGetLastError();
}

static cudaError_t fill_f32_companion(const stg_gauge *g64, stg_gauge *g, cudaStream_t st)
{
    const long long n = 8LL * g->g.Vh;
    const unsigned nb = (unsigned)((n + 255) / 256);
    using F32U = LinkU1<LinkF32R12, float>;
    switch (g64->kind) {
    case kF64R18: k_links_to_f32r12<LinkF64R18, LinkF32R12><<<nb, 256, 0, st>>>(g->g, g64->links, g->links); break;
    case kF64R12: k_links_to_f32r12<LinkF64R12, LinkF32R12><<<nb, 256, 0, st>>>(g->g, g64->links, g->links); break;
    case kF64R18 | kU1:
        k_links_to_f32r12<LinkU1<LinkF64R18, double2>, F32U><<<nb, 256, 0, st>>>(g->g, g64->links, g->links);
        break;
    default:
        k_links_to_f32r12<LinkU1<LinkF64R12, double2>, F32U><<<nb, 256, 0, st>>>(g->g, g64->links, g->links);
        break;
    }
    return cudaGetLastError();
}

static std::mutex g_companion_mu;

stg_status ds_companion(const stg_gauge *g64, cudaStream_t st, const stg_gauge **out)
{
    std::lock_guard<std::mutex> lk(g_companion_mu);
    if (!g64->ds_copy) {
        stg_gauge *g = new (std::nothrow) stg_gauge;
        if (!g) return set_error(STG_ERR_OOM, "ds_companion: host allocation");
        *g = *g64;
        g->kind = (base_kind(g64->kind) == kF64R18 ? kDSR18 : kDSR12) | (g64->kind & kU1);
        g->bytes = (size_t)4 * g64->lat->V * link_bytes(g->kind);
        g->scratch = nullptr;
        g->links = nullptr;
        g->f32_copy = nullptr;
        g->ds_copy = nullptr;
        cudaError_t e = cudaMalloc(&g->links, g->bytes);
        if (e == cudaSuccess) e = cudaMalloc(&g->scratch, g->scratch_count * sizeof(double));
        if (e == cudaSuccess) e = fill_ds_companion(g64, g, st);
        if (e != cudaSuccess) {
            cudaFree(g->links);
            cudaFree(g->scratch);
            delete g;
            return cuda_error(e, "ds_companion");
        }
        g64->ds_copy = g;
    }
    *out = g64->ds_copy;
    return STG_OK;
}

stg_status f32_companion(const stg_gauge *g64, cudaStream_t st, const stg_gauge **out)
{
    std::lock_guard<std::mutex> lk(g_companion_mu);
    if (!g64->f32_copy) {
        stg_gauge *g = new (std::nothrow) stg_gauge;
        if (!g) return set_error(STG_ERR_OOM, "f32_companion: host allocation");
        *g = *g64;
        g->prec = STG_F32;
        g->recon = STG_RECON12;
        g->kind = kF32R12 | (g64->kind & kU1);
        g->bytes = (size_t)4 * g64->lat->V * link_bytes(g->kind);
        g->scratch = nullptr;
        g->links = nullptr;
        g->f32_copy = nullptr;
        g->ds_copy = nullptr;
        cudaError_t e = cudaMalloc(&g->links, g->bytes);
        if (e == cudaSuccess) e = cudaMalloc(&g->scratch, g->scratch_count * sizeof(double));
        if (e == cudaSuccess) e = fill_f32_companion(g64, g, st);
        if (e != cudaSuccess) {
            cudaFree(g->links);
            cudaFree(g->scratch);
            delete g;
            return cuda_error(e, "f32_companion");
        }
        g64->f32_copy = g;
    }
    *out = g64->f32_copy;
    return STG_OK;
}

// canonical [Vh][3] complex128 <-> internal field
template <typename R, typename C = double2>
__global__ void k_pack_field(int Vh, const C *__restrict__ canon, void *__restrict__ out)
{
    int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= Vh) return;
    cx<R> v[3];
    for (int c = 0; c < 3; ++c) {
        const C d = canon[(size_t)h * 3 + c];
        v[c] = cx<R>{(R)d.x, (R)d.y};
    }
    Field<R>::store(out, Vh, h, v);
}

template <typename R, typename C = double2>
__global__ void k_unpack_field(int Vh, const void *__restrict__ in, C *__restrict__ canon)
{
    int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= Vh) return;
    cx<R> v[3];
    Field<R>::load_rw(in, Vh, h, v);
    for (int c = 0; c < 3; ++c) {
        C d;
        d.x = (decltype(d.x))(double)v[c].re;
        d.y = (decltype(d.y))(double)v[c].im;
        canon[(size_t)h * 3 + c] = d;
    }
}

// Pack / unpack between a canonical complex64 field and the internal layout of vec_prec (the
// single-precision host fields of stg_dslash_host).
cudaError_t launch_field_pack_c64(stg_prec vec_prec, int Vh, const void *canon, void *internal, cudaStream_t st)
{
    const int bs = 256;
    const float2 *c = static_cast<const float2 *>(canon);
    if (vec_prec == STG_F64) k_pack_field<double, float2><<<(Vh + bs - 1) / bs, bs, 0, st>>>(Vh, c, internal);
    else if (vec_prec == STG_F32) k_pack_field<float, float2><<<(Vh + bs - 1) / bs, bs, 0, st>>>(Vh, c, internal);
    else k_pack_field<dsf, float2><<<(Vh + bs - 1) / bs, bs, 0, st>>>(Vh, c, internal);
    return cudaGetLastError();
}

cudaError_t launch_field_unpack_c64(stg_prec vec_prec, int Vh, const void *internal, void *canon, cudaStream_t st)
{
    const int bs = 256;
    float2 *c = static_cast<float2 *>(canon);
    if (vec_prec == STG_F64) k_unpack_field<double, float2><<<(Vh + bs - 1) / bs, bs, 0, st>>>(Vh, internal, c);
    else if (vec_prec == STG_F32) k_unpack_field<float, float2><<<(Vh + bs - 1) / bs, bs, 0, st>>>(Vh, internal, c);
    else k_unpack_field<dsf, float2><<<(Vh + bs - 1) / bs, bs, 0, st>>>(Vh, internal, c);
    return cudaGetLastError();
}

// fixed-order sum of n partials into *out (one block)
__global__ void k_sum_partials(const double *__restrict__ part, int n, double *__restrict__ out)
{
    __shared__ double sh[32];
    double s = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) s += part[k];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) *out = s;
}

}  // namespace stg

using namespace stg;

// ------------------------------------------------------------------ C ABI

static bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

extern "C" {

const char *stg_status_string(stg_status s)
{
    switch (s) {
    case STG_OK: return "STG_OK";
    case STG_ERR_ARG: return "STG_ERR_ARG: invalid argument";
    case STG_ERR_SHAPE: return "STG_ERR_SHAPE: invalid lattice shape";
    case STG_ERR_CUDA: return "STG_ERR_CUDA: CUDA runtime error";
    case STG_ERR_NOCONV: return "STG_ERR_NOCONV: solver did not converge";
    case STG_ERR_TIMEOUT: return "STG_ERR_TIMEOUT: bounded device wait gave up";
    case STG_ERR_OOM: return "STG_ERR_OOM: device allocation failed";
    }
    return "STG_ERR_UNKNOWN";
}

const char *stg_last_error(void) { return g_last_error.c_str(); }

const char *stg_version(void) { return "stg 0.2 (sm_103a)"; }

stg_status stg_lattice_create(const int32_t dims[4], int32_t t_antiperiodic, stg_lattice **out)
{
    if (!dims || !out) return set_error(STG_ERR_ARG, "stg_lattice_create: null pointer");
    *out = nullptr;
    long long V = 1;
    for (int k = 0; k < 4; ++k) {
        if (dims[k] < 2 || (dims[k] & 1))
            return set_error(STG_ERR_SHAPE, "stg_lattice_create: every extent must be even and >= 2");
        V *= dims[k];
    }
    if (V > (1LL << 31)) return set_error(STG_ERR_SHAPE, "stg_lattice_create: volume above 2^31 sites");
    stg_lattice *l = new (std::nothrow) stg_lattice;
    if (!l) return set_error(STG_ERR_OOM, "stg_lattice_create: host allocation");
    for (int k = 0; k < 4; ++k) l->g.L[k] = dims[k];
    l->g.Vh = (int)(V / 2);
    l->g.antiperiodic = t_antiperiodic ? 1 : 0;
    geom_init(l->g);
    l->V = V;
    *out = l;
    return STG_OK;
}

stg_status stg_lattice_create_slab(const int32_t dims_local[4], int32_t t0, int32_t Lt_global, int32_t t_antiperiodic,
                                   stg_lattice **out)
{
    if (!dims_local || !out) return set_error(STG_ERR_ARG, "stg_lattice_create_slab: null pointer");
    *out = nullptr;
    for (int k = 0; k < 4; ++k)
        if (dims_local[k] < 2 || (dims_local[k] & 1))
            return set_error(STG_ERR_SHAPE, "stg_lattice_create_slab: every local extent must be even and >= 2");
    if ((t0 & 1) || t0 < 0 || Lt_global < 2 || (Lt_global & 1) || t0 + dims_local[3] > Lt_global)
        return set_error(STG_ERR_SHAPE, "stg_lattice_create_slab: need t0 even, Lt_global even and "
                                        "0 <= t0, t0 + Lt_loc <= Lt_global");
    // stored lattice: the local slices plus two halo-side slices below and above (the inner one of
    // each pair holds the neighbour's border; the outer one keeps the stored parity equal to the
    // global one, since stored slice 0 then sits at the even global time t0 - 2)
    const int32_t ext[4] = {dims_local[0], dims_local[1], dims_local[2], dims_local[3] + 4};
    stg_status st = stg_lattice_create(ext, t_antiperiodic, out);
    if (st != STG_OK) return st;
    Geom &g = (*out)->g;
    const int half_slice = dims_local[0] * dims_local[1] * dims_local[2] / 2;
    g.h_begin = 2 * half_slice;
    g.h_end = (dims_local[3] + 2) * half_slice;
    g.t_off = t0 - 2;
    g.Lt_glob = Lt_global;
    return STG_OK;
}

stg_status stg_slab_layout(const stg_lattice *lat, stg_prec vec_prec, int32_t *nchunk, int64_t offset[3],
                           int32_t elem_bytes[3], int64_t *slice_sites)
{
    if (!lat || !nchunk || !offset || !elem_bytes || !slice_sites)
        return set_error(STG_ERR_ARG, "stg_slab_layout: null pointer");
    const long long Vh = lat->g.Vh;
    *slice_sites = (long long)lat->g.L[0] * lat->g.L[1] * lat->g.L[2] / 2;
    if (vec_prec == STG_F64 || vec_prec == STG_DS) {  // three arrays of one 16-byte word per site
        *nchunk = 3;
        for (int k = 0; k < 3; ++k) {
            offset[k] = 16LL * Vh * k;
            elem_bytes[k] = 16;
        }
        return STG_OK;
    }
    if (vec_prec == STG_F32) {  // colours 0, 1 as one float4 per site, then colour 2 as a float2
        *nchunk = 2;
        offset[0] = 0;
        elem_bytes[0] = 16;
        offset[1] = 16LL * Vh;
        elem_bytes[1] = 8;
        offset[2] = 0;
        elem_bytes[2] = 0;
        return STG_OK;
    }
    return set_error(STG_ERR_ARG, "stg_slab_layout: vec_prec must be F64, DS or F32");
}

void stg_lattice_destroy(stg_lattice *lat) { delete lat; }

int64_t stg_lattice_sites(const stg_lattice *lat, int32_t parity)
{
    if (!lat) return -1;
    if (parity == 0 || parity == 1) return lat->g.Vh;
    if (parity == -1) return lat->V;
    return -1;
}

static stg_status gauge_create(const stg_lattice *lat, const void *links_c128_dev, const double *theta_dev,
                               stg_prec prec, stg_recon recon, void *stream, stg_gauge **out)
{
    if (!lat || !links_c128_dev || !out) return set_error(STG_ERR_ARG, "stg_gauge_create: null pointer");
    *out = nullptr;
    if (!aligned16(links_c128_dev)) return set_error(STG_ERR_ARG, "stg_gauge_create: links not 16-byte aligned");
    int kind = -1;
    if (recon != STG_RECON18 && recon != STG_RECON12) return set_error(STG_ERR_ARG, "stg_gauge_create: bad recon");
    switch (prec) {
    case STG_F64: kind = recon == STG_RECON18 ? kF64R18 : kF64R12; break;
    case STG_F32: kind = recon == STG_RECON18 ? kF32R18 : kF32R12; break;
    case STG_BF16: kind = recon == STG_RECON12 ? kBF16R12 : -1; break;
    case STG_F16: kind = recon == STG_RECON12 ? kF16R12 : -1; break;
    case STG_DS: kind = recon == STG_RECON18 ? kDSR18 : kDSR12; break;
    default: break;
    }
    if (kind < 0) return set_error(STG_ERR_ARG, "stg_gauge_create: unsupported precision/compression pair");
    if (theta_dev) kind |= kU1;

    stg_gauge *g = new (std::nothrow) stg_gauge;
    if (!g) return set_error(STG_ERR_OOM, "stg_gauge_create: host allocation");
    g->lat = lat;
    g->g = lat->g;
    g->prec = prec;
    g->recon = recon;
    g->kind = kind;
    g->bytes = (size_t)4 * lat->V * link_bytes(kind);
    g->links = nullptr;
    g->scratch = nullptr;
    g->f32_copy = nullptr;
    g->ds_copy = nullptr;
    g->scratch_count = (size_t)dslash_partials(lat->g.Vh);
    cudaError_t e = cudaMalloc(&g->links, g->bytes);
    if (e == cudaSuccess) e = cudaMalloc(&g->scratch, g->scratch_count * sizeof(double));
    if (e == cudaSuccess)
        e = theta_dev ? launch_pack_links_u1(kind, lat->g, links_c128_dev, theta_dev, g->links, (cudaStream_t)stream)
                      : launch_pack_links(kind, lat->g, links_c128_dev, g->links, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        stg_status s = cuda_error(e, "stg_gauge_create");
        cudaFree(g->links);
        cudaFree(g->scratch);
        delete g;
        return s;
    }
    *out = g;
    return STG_OK;
}

stg_status stg_gauge_create(const stg_lattice *lat, const void *links_c128_dev, stg_prec prec, stg_recon recon,
                            void *stream, stg_gauge **out)
{
    return gauge_create(lat, links_c128_dev, nullptr, prec, recon, stream, out);
}

stg_status stg_gauge_update(stg_gauge *g, const void *links_c128_dev, const double *theta_dev, void *stream)
{
    if (!g || !links_c128_dev) return set_error(STG_ERR_ARG, "stg_gauge_update: null pointer");
    if (!aligned16(links_c128_dev)) return set_error(STG_ERR_ARG, "stg_gauge_update: links not 16-byte aligned");
    const bool u1 = kind_has_u1(g->kind);
    if (u1 != (theta_dev != nullptr))
        return set_error(STG_ERR_ARG, "stg_gauge_update: theta must be given exactly when the gauge carries phases");
    if (theta_dev && (reinterpret_cast<uintptr_t>(theta_dev) & 7))
        return set_error(STG_ERR_ARG, "stg_gauge_update: theta not 8-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    STG_CUDA_TRY(u1 ? launch_pack_links_u1(g->kind, g->g, links_c128_dev, theta_dev, g->links, st)
                    : launch_pack_links(g->kind, g->g, links_c128_dev, g->links, st));
    std::lock_guard<std::mutex> lk(g_companion_mu);
    if (g->ds_copy) STG_CUDA_TRY(fill_ds_companion(g, g->ds_copy, st));
    if (g->f32_copy) STG_CUDA_TRY(fill_f32_companion(g, g->f32_copy, st));
    return STG_OK;
}

stg_status stg_gauge_create_u1(const stg_lattice *lat, const void *links_c128_dev, const double *theta_dev, stg_prec prec,
                               stg_recon recon, void *stream, stg_gauge **out)
{
    if (!theta_dev || (reinterpret_cast<uintptr_t>(theta_dev) & 7))
        return set_error(STG_ERR_ARG, "stg_gauge_create_u1: theta must be non-null and 8-byte aligned");
    return gauge_create(lat, links_c128_dev, theta_dev, prec, recon, stream, out);
}

void stg_gauge_destroy(stg_gauge *g)
{
    if (!g) return;
    if (g->f32_copy) stg_gauge_destroy(g->f32_copy);
    if (g->ds_copy) stg_gauge_destroy(g->ds_copy);
    cudaFree(g->links);
    cudaFree(g->scratch);
    delete g;
}

size_t stg_gauge_bytes(const stg_gauge *g) { return g ? g->bytes : 0; }

size_t stg_field_bytes(const stg_lattice *lat, stg_prec vec_prec)
{
    if (!lat) return 0;
    if (vec_prec == STG_F64) return (size_t)lat->g.Vh * Field<double>::kBytesPerSite;
    if (vec_prec == STG_DS) return (size_t)lat->g.Vh * Field<dsf>::kBytesPerSite;
    if (vec_prec == STG_F32) return (size_t)lat->g.Vh * Field<float>::kBytesPerSite;
    return 0;
}

stg_status stg_field_pack(const stg_lattice *lat, stg_prec vec_prec, const void *canon_c128_dev, void *internal_dev,
                          void *stream)
{
    if (!lat || !canon_c128_dev || !internal_dev) return set_error(STG_ERR_ARG, "stg_field_pack: null pointer");
    if (!aligned16(canon_c128_dev) || !aligned16(internal_dev))
        return set_error(STG_ERR_ARG, "stg_field_pack: pointers must be 16-byte aligned");
    int Vh = lat->g.Vh, bs = 256;
    if (vec_prec == STG_F64)
        k_pack_field<double><<<(Vh + bs - 1) / bs, bs, 0, (cudaStream_t)stream>>>(Vh, (const double2 *)canon_c128_dev,
                                                                                  internal_dev);
    else if (vec_prec == STG_F32)
        k_pack_field<float><<<(Vh + bs - 1) / bs, bs, 0, (cudaStream_t)stream>>>(Vh, (const double2 *)canon_c128_dev,
                                                                                 internal_dev);
    else if (vec_prec == STG_DS)
        k_pack_field<dsf><<<(Vh + bs - 1) / bs, bs, 0, (cudaStream_t)stream>>>(Vh, (const double2 *)canon_c128_dev,
                                                                               internal_dev);
    else
        return set_error(STG_ERR_ARG, "stg_field_pack: vector precision must be F64, DS or F32");
    STG_CUDA_TRY(cudaGetLastError());
    return STG_OK;
}

stg_status stg_field_unpack(const stg_lattice *lat, stg_prec vec_prec, const void *internal_dev, void *canon_c128_dev,
                            void *stream)
{
    if (!lat || !canon_c128_dev || !internal_dev) return set_error(STG_ERR_ARG, "stg_field_unpack: null pointer");
    if (!aligned16(canon_c128_dev) || !aligned16(internal_dev))
        return set_error(STG_ERR_ARG, "stg_field_unpack: pointers must be 16-byte aligned");
    int Vh = lat->g.Vh, bs = 256;
    if (vec_prec == STG_F64)
        k_unpack_field<double><<<(Vh + bs - 1) / bs, bs, 0, (cudaStream_t)stream>>>(Vh, internal_dev,
                                                                                    (double2 *)canon_c128_dev);
    else if (vec_prec == STG_F32)
        k_unpack_field<float><<<(Vh + bs - 1) / bs, bs, 0, (cudaStream_t)stream>>>(Vh, internal_dev,
                                                                                   (double2 *)canon_c128_dev);
    else if (vec_prec == STG_DS)
        k_unpack_field<dsf><<<(Vh + bs - 1) / bs, bs, 0, (cudaStream_t)stream>>>(Vh, internal_dev,
                                                                                 (double2 *)canon_c128_dev);
    else
        return set_error(STG_ERR_ARG, "stg_field_unpack: vector precision must be F64, DS or F32");
    STG_CUDA_TRY(cudaGetLastError());
    return STG_OK;
}

stg_status stg_dslash_multi(const stg_gauge *g, int32_t out_parity, int32_t nrhs, void *out_dev, const void *in_dev,
                            size_t stride_bytes, void *stream)
{
    if (!g || !out_dev || !in_dev) return set_error(STG_ERR_ARG, "stg_dslash: null pointer");
    if (out_parity != 0 && out_parity != 1) return set_error(STG_ERR_ARG, "stg_dslash: out_parity must be 0 or 1");
    if (nrhs < 1 || nrhs > 64) return set_error(STG_ERR_ARG, "stg_dslash: nrhs must be in 1..64");
    size_t fb = (size_t)g->g.Vh * kind_vec_bytes(g->kind);
    if (nrhs > 1 && (stride_bytes < fb || (stride_bytes & 15)))
        return set_error(STG_ERR_ARG, "stg_dslash: stride must be >= the field size and a multiple of 16 bytes");
    if (!aligned16(out_dev) || !aligned16(in_dev)) return set_error(STG_ERR_ARG, "stg_dslash: pointers must be 16-byte aligned");
    const char *ib = static_cast<const char *>(in_dev);
    char *ob = static_cast<char *>(out_dev);
    if (ib < ob + (nrhs - 1) * stride_bytes + fb && ob < ib + (nrhs - 1) * stride_bytes + fb)
        return set_error(STG_ERR_ARG, "stg_dslash: input and output overlap");
    for (int base = 0; base < nrhs;) {
        DArgs a;
        memset(&a, 0, sizeof(a));
        a.out_par = out_parity;
        int ng = 0;
        while (ng < kMaxGroups && base < nrhs) {
            DGroup &G = a.grp[ng++];
            G.g = g->g;
            G.links = g->links;
            G.nrhs = (nrhs - base) < kMaxRhs ? (nrhs - base) : kMaxRhs;
            for (int j = 0; j < G.nrhs; ++j) {
                G.in[j] = ib + (size_t)(base + j) * stride_bytes;
                G.out[j] = ob + (size_t)(base + j) * stride_bytes;
            }
            base += G.nrhs;
        }
        a.ngroups = ng;
        STG_CUDA_TRY(launch_dslash(g->kind, a, 0, (cudaStream_t)stream));
    }
    return STG_OK;
}

stg_status stg_dslash_eo(const stg_gauge *g, void *out_even_dev, const void *in_odd_dev, void *stream)
{
    return stg_dslash_multi(g, 0, 1, out_even_dev, in_odd_dev, 0, stream);
}

stg_status stg_dslash_oe(const stg_gauge *g, void *out_odd_dev, const void *in_even_dev, void *stream)
{
    return stg_dslash_multi(g, 1, 1, out_odd_dev, in_even_dev, 0, stream);
}

stg_status stg_dslash(const stg_gauge *g, int32_t out_parity, void *out_dev, const void *in_dev, void *stream)
{
    if (out_parity != 0 && out_parity != 1) return set_error(STG_ERR_ARG, "stg_dslash: out_parity must be 0 or 1");
    return stg_dslash_multi(g, out_parity, 1, out_dev, in_dev, 0, stream);
}

stg_status stg_normal_op(const stg_gauge *g, double mass, double shift, void *out_even_dev, const void *in_even_dev,
                         void *tmp_odd_dev, double *pq_dev, void *stream)
{
    if (g && stg::geom_is_slab(g->g))
        return stg::set_error(STG_ERR_SHAPE, "stg_normal_op: not available on a slab lattice (stg_dslash* only)");
    if (!g || !out_even_dev || !in_even_dev || !tmp_odd_dev) return set_error(STG_ERR_ARG, "stg_normal_op: null pointer");
    if (!aligned16(out_even_dev) || !aligned16(in_even_dev) || !aligned16(tmp_odd_dev))
        return set_error(STG_ERR_ARG, "stg_normal_op: pointers must be 16-byte aligned");
    if (out_even_dev == in_even_dev || tmp_odd_dev == in_even_dev || tmp_odd_dev == out_even_dev)
        return set_error(STG_ERR_ARG, "stg_normal_op: in, out and tmp must be distinct");
    cudaStream_t st = (cudaStream_t)stream;
    DArgs a;
    memset(&a, 0, sizeof(a));
    a.ngroups = 1;
    DGroup &G = a.grp[0];
    G.g = g->g;
    G.links = g->links;
    G.nrhs = 1;
    // D_oe: even -> odd
    a.out_par = 1;
    G.in[0] = in_even_dev;
    G.out[0] = tmp_odd_dev;
    STG_CUDA_TRY(launch_dslash(g->kind, a, 0, st));
    // D_eo with the fused epilogue out = (m^2 + shift) in - D_eo tmp, partial Re<in, out>
    a.out_par = 0;
    G.in[0] = tmp_odd_dev;
    G.out[0] = out_even_dev;
    G.epi_p[0] = in_even_dev;
    G.coef[0] = mass * mass + shift;
    G.partial[0] = pq_dev ? g->scratch : nullptr;
    STG_CUDA_TRY(launch_dslash(g->kind, a, 1, st));
    if (pq_dev) {
        k_sum_partials<<<1, 256, 0, st>>>(g->scratch, dslash_partials(g->g.Vh), pq_dev);
        STG_CUDA_TRY(cudaGetLastError());
    }
    return STG_OK;
}

}  // extern "C"
