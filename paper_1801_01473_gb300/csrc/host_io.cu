// host_io.cu -- D_eo / D_oe applied to many fields that live in host memory (the sources of
// Sec. 2's multiple pseudofermions, streamed through the operator): a three-stage pipeline in which
// the host->device copy of field k+1, the pack / D / unpack of field k and the device->host copy of
// field k-1 run concurrently on three streams, with two device staging slots per stage.  With
// pinned host buffers the transfers overlap the compute; the call returns when every output is in
// host memory.
#include <cstring>
#include <vector>

#include "stg_common.h"

namespace stg {
namespace {

constexpr int kSlots = 2;

struct Pipe {
    cudaStream_t s_in = nullptr, s_cmp = nullptr, s_out = nullptr;
    cudaEvent_t in_ready[kSlots] = {}, in_free[kSlots] = {}, out_ready[kSlots] = {}, out_free[kSlots] = {};
    cudaEvent_t start = nullptr, end = nullptr;
    void *mem = nullptr;
    cudaStream_t user = nullptr;
    cudaError_t create()
    {
        cudaError_t e = cudaSuccess;
        auto ev = [&](cudaEvent_t *p) {
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(p, cudaEventDisableTiming);
        };
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s_in, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s_cmp, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s_out, cudaStreamNonBlocking);
        for (int k = 0; k < kSlots; ++k) {
            ev(&in_ready[k]);
            ev(&in_free[k]);
            ev(&out_ready[k]);
            ev(&out_free[k]);
        }
        ev(&start);
        ev(&end);
        return e;
    }
    ~Pipe()
    {
        // every copy and kernel of the pipeline has finished before the staging memory goes
        if (s_in) cudaStreamSynchronize(s_in);
        if (s_cmp) cudaStreamSynchronize(s_cmp);
        if (s_out) cudaStreamSynchronize(s_out);
        if (mem) cudaFree(mem);
        for (int k = 0; k < kSlots; ++k) {
            if (in_ready[k]) cudaEventDestroy(in_ready[k]);
            if (in_free[k]) cudaEventDestroy(in_free[k]);
            if (out_ready[k]) cudaEventDestroy(out_ready[k]);
            if (out_free[k]) cudaEventDestroy(out_free[k]);
        }
        if (start) cudaEventDestroy(start);
        if (end) cudaEventDestroy(end);
        if (s_in) cudaStreamDestroy(s_in);
        if (s_cmp) cudaStreamDestroy(s_cmp);
        if (s_out) cudaStreamDestroy(s_out);
    }
};

}  // namespace
}  // namespace stg

using namespace stg;

extern "C" stg_status stg_dslash_host(const stg_gauge *g, int32_t out_parity, stg_prec host_prec, int32_t nfield,
                                      const void *const *in_host, void *const *out_host, void *stream)
{
    if (g && stg::geom_is_slab(g->g))
        return stg::set_error(STG_ERR_SHAPE, "stg_dslash_host: not available on a slab lattice (stg_dslash* only)");
    if (host_prec != STG_F64 && host_prec != STG_F32)
        return set_error(STG_ERR_ARG, "stg_dslash_host: host fields must be F64 (complex128) or F32 (complex64)");
    if (!g || (nfield > 0 && (!in_host || !out_host)))
        return set_error(STG_ERR_ARG, "stg_dslash_host: null pointer");
    if (out_parity != 0 && out_parity != 1) return set_error(STG_ERR_ARG, "stg_dslash_host: out_parity must be 0 or 1");
    if (nfield < 0) return set_error(STG_ERR_ARG, "stg_dslash_host: nfield must be >= 0");
    for (int k = 0; k < nfield; ++k)
        if (!in_host[k] || !out_host[k] || in_host[k] == out_host[k])
            return set_error(STG_ERR_ARG, "stg_dslash_host: null or aliasing host field");
    if (nfield == 0) return STG_OK;

    const int Vh = g->g.Vh;
    const bool c64 = host_prec == STG_F32;
    const size_t canon = (size_t)Vh * 3 * (c64 ? sizeof(float2) : sizeof(double2));  // one canonical field
    const size_t inter = ((size_t)Vh * kind_vec_bytes(g->kind) + 255) & ~(size_t)255;  // one internal field
    const stg_prec vp = kind_is_f64(g->kind) ? STG_F64 : kind_is_ds(g->kind) ? STG_DS : STG_F32;

    Pipe P;
    P.user = (cudaStream_t)stream;
    STG_CUDA_TRY(P.create());
    // staging: per slot a canonical input, an internal input, an internal output, a canonical output
    // (canonical slots rounded to 256 bytes so that every staging buffer stays aligned)
    const size_t canon_al = (canon + 255) & ~(size_t)255;
    STG_CUDA_TRY(cudaMalloc(&P.mem, kSlots * (2 * canon_al + 2 * inter)));
    char *base = static_cast<char *>(P.mem);
    char *c_in[kSlots], *i_in[kSlots], *i_out[kSlots], *c_out[kSlots];
    for (int k = 0; k < kSlots; ++k) {
        char *b = base + (size_t)k * (2 * canon_al + 2 * inter);
        c_in[k] = b;
        c_out[k] = b + canon_al;
        i_in[k] = b + 2 * canon_al;
        i_out[k] = b + 2 * canon_al + inter;
    }
    // order after the work already queued on the caller's stream
    STG_CUDA_TRY(cudaEventRecord(P.start, P.user));
    STG_CUDA_TRY(cudaStreamWaitEvent(P.s_in, P.start, 0));
    STG_CUDA_TRY(cudaStreamWaitEvent(P.s_cmp, P.start, 0));

    DArgs a;
    memset(&a, 0, sizeof(a));
    a.ngroups = 1;
    a.out_par = out_parity;
    a.grp[0].g = g->g;
    a.grp[0].links = g->links;
    a.grp[0].nrhs = 1;
    for (int k = 0; k < nfield; ++k) {
        const int s = k % kSlots;
        // stage 1: host -> device, once the slot's previous input has been packed
        if (k >= kSlots) STG_CUDA_TRY(cudaStreamWaitEvent(P.s_in, P.in_free[s], 0));
        STG_CUDA_TRY(cudaMemcpyAsync(c_in[s], in_host[k], canon, cudaMemcpyHostToDevice, P.s_in));
        STG_CUDA_TRY(cudaEventRecord(P.in_ready[s], P.s_in));
        // stage 2: pack, D, unpack, once the slot's previous output has left the device
        STG_CUDA_TRY(cudaStreamWaitEvent(P.s_cmp, P.in_ready[s], 0));
        if (c64) {
            STG_CUDA_TRY(launch_field_pack_c64(vp, Vh, c_in[s], i_in[s], P.s_cmp));
        } else {
            const stg_status st = stg_field_pack(g->lat, vp, c_in[s], i_in[s], P.s_cmp);
            if (st != STG_OK) return st;
        }
        STG_CUDA_TRY(cudaEventRecord(P.in_free[s], P.s_cmp));
        if (k >= kSlots) STG_CUDA_TRY(cudaStreamWaitEvent(P.s_cmp, P.out_free[s], 0));
        a.grp[0].in[0] = i_in[s];
        a.grp[0].out[0] = i_out[s];
        STG_CUDA_TRY(launch_dslash(g->kind, a, 0, P.s_cmp));
        if (c64) {
            STG_CUDA_TRY(launch_field_unpack_c64(vp, Vh, i_out[s], c_out[s], P.s_cmp));
        } else {
            const stg_status st = stg_field_unpack(g->lat, vp, i_out[s], c_out[s], P.s_cmp);
            if (st != STG_OK) return st;
        }
        STG_CUDA_TRY(cudaEventRecord(P.out_ready[s], P.s_cmp));
        // stage 3: device -> host
        STG_CUDA_TRY(cudaStreamWaitEvent(P.s_out, P.out_ready[s], 0));
        STG_CUDA_TRY(cudaMemcpyAsync(out_host[k], c_out[s], canon, cudaMemcpyDeviceToHost, P.s_out));
        STG_CUDA_TRY(cudaEventRecord(P.out_free[s], P.s_out));
    }
    STG_CUDA_TRY(cudaEventRecord(P.end, P.s_out));
    STG_CUDA_TRY(cudaStreamWaitEvent(P.user, P.end, 0));
    STG_CUDA_TRY(cudaStreamSynchronize(P.s_out));
    return STG_OK;  // the pipeline's streams, events and staging are released by ~Pipe
}
