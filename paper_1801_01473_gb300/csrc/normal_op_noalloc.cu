// normal_op_noalloc.cu -- stg_normal_op_noalloc: the shifted normal operator with its FP64
// <in, out> reduction, for callers that cannot allocate device memory at call time.
//
// stg_normal_op needs an odd-parity temporary from the caller and reduces <in, out> through a
// buffer the gauge handle allocated.  Some callers can do neither: a host framework that owns
// every byte of device memory through its own pool (and forbids driver allocations once the
// run has started), or an integrator loop that must not call cudaMalloc / cudaFree because
// those calls can synchronize the whole device or fail when memory is already partitioned.
// This variant keeps its scratch -- the odd temporary and the partial sums -- in one
// file-scope __device__ array of fixed size, so a call allocates nothing.
#include <cstring>
#include <mutex>

#include "stg_common.h"

namespace stg {

// Fixed scratch for every call on a device: holds the odd temporary (48 B per site for F64 and
// double-single gauges, 24 B for the F32/BF16/F16 ones) and one double per 64 sites.  32 MiB
// covers a 32^4 lattice at FP64 (25.2 MB + 64 KB).  Every GPU that loads the library holds it
// until the process exits.
constexpr size_t kStaticScratchBytes = 32u << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// fixed-order sum of n partials into *out (one block of 256 threads)
__global__ void k_noalloc_sum(const double *__restrict__ part, int n, double *__restrict__ out)
{
    __shared__ double sh[32];
    double s = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) s += part[k];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) *out = s;
}

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
void *g_addr[kMaxDevices];  // device address of g_static_scratch, per device (set-up once)
}  // namespace

// Device address of the scratch array on the current device.  In host code the name
// g_static_scratch is only a host-side stand-in, so the address must come from
// cudaGetSymbolAddress, with the device current, once per device.
static stg_status static_scratch(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "stg_normal_op_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return set_error(STG_ERR_ARG, "stg_normal_op_noalloc: device index too large");
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_error(e, "stg_normal_op_noalloc: cudaGetSymbolAddress");
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return STG_OK;
}

}  // namespace stg

using namespace stg;

extern "C" stg_status stg_normal_op_noalloc(const stg_gauge *g, double mass, double shift, void *out_even_dev,
                                            const void *in_even_dev, double *pq_dev, void *stream)
{
    if (g && stg::geom_is_slab(g->g))
        return stg::set_error(STG_ERR_SHAPE, "stg_normal_op_noalloc: not available on a slab lattice (stg_dslash* only)");
    if (!g || !out_even_dev || !in_even_dev) return set_error(STG_ERR_ARG, "stg_normal_op_noalloc: null pointer");
    if ((reinterpret_cast<uintptr_t>(out_even_dev) & 15) || (reinterpret_cast<uintptr_t>(in_even_dev) & 15))
        return set_error(STG_ERR_ARG, "stg_normal_op_noalloc: pointers must be 16-byte aligned");
    const int Vh = g->g.Vh;
    {
        // any overlap of the two fields: the fused D_eo epilogue reads in while it writes out
        const uintptr_t i0 = reinterpret_cast<uintptr_t>(in_even_dev), o0 = reinterpret_cast<uintptr_t>(out_even_dev);
        const uintptr_t n = (uintptr_t)Vh * (uintptr_t)kind_vec_bytes(g->kind);
        if (i0 < o0 + n && o0 < i0 + n) return set_error(STG_ERR_ARG, "stg_normal_op_noalloc: in and out overlap");
    }
    const size_t tmp_bytes = ((size_t)Vh * kind_vec_bytes(g->kind) + 255) & ~(size_t)255;
    const size_t part_bytes = sizeof(double) * (size_t)dslash_partials(Vh);
    if (tmp_bytes + part_bytes > kStaticScratchBytes)
        return set_error(STG_ERR_ARG, "stg_normal_op_noalloc: lattice too large for the 32 MiB static scratch "
                                      "(at most 697232 sites per parity for F64/DS gauges, 1390848 for the others)");
    void *base = nullptr;
    stg_status s = static_scratch(&base);
    if (s != STG_OK) return s;
    void *tmp_odd = base;
    double *part = reinterpret_cast<double *>(static_cast<char *>(base) + tmp_bytes);

    cudaStream_t st = (cudaStream_t)stream;
    DArgs a;
    memset(&a, 0, sizeof(a));
    a.ngroups = 1;
    DGroup &G = a.grp[0];
    G.g = g->g;
    G.links = g->links;
    G.nrhs = 1;
    a.out_par = 1;  // D_oe: even -> odd, into the static temporary
    G.in[0] = in_even_dev;
    G.out[0] = tmp_odd;
    STG_CUDA_TRY(launch_dslash_bs(g->kind, a, 0, kDslashBlock, st));
    a.out_par = 0;  // D_eo with the fused epilogue out = (m^2 + shift) in - D_eo tmp
    G.in[0] = tmp_odd;
    G.out[0] = out_even_dev;
    G.epi_p[0] = in_even_dev;
    G.coef[0] = mass * mass + shift;
    G.partial[0] = pq_dev ? part : nullptr;
    STG_CUDA_TRY(launch_dslash_bs(g->kind, a, 1, kDslashBlock, st));
    if (pq_dev) {
        k_noalloc_sum<<<1, 256, 0, st>>>(part, dslash_partials(Vh), pq_dev);
        STG_CUDA_TRY(cudaGetLastError());
    }
    return STG_OK;
}
