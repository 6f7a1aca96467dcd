// stg_common.h -- host-side definitions shared by the translation units of libstg:
// the opaque handles, the link-storage kinds, error reporting and the launchers
// implemented in the per-precision dslash units.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "../../include/stg.h"
#include "dslash.cuh"

namespace stg {

// Link storage kinds (precision x compression); index of the dslash instantiation.
enum LinkKind { kF64R18 = 0, kF64R12 = 1, kF32R18 = 2, kF32R12 = 3, kBF16R12 = 4, kF16R12 = 5, kDSR18 = 6, kDSR12 = 7 };
// flag on a kind: the links carry a U(1) phase field theta (LinkU1 layout)
constexpr int kU1 = 8;
inline int base_kind(int kind) { return kind & 7; }
inline bool kind_has_u1(int kind) { return (kind & kU1) != 0; }

// A slab lattice (stg_lattice_create_slab): halo time slices around the interior outputs.
inline bool geom_is_slab(const Geom &g) { return g.h_begin != 0 || g.h_end != g.Vh || g.t_off != 0; }

int link_bytes(int kind);
inline bool kind_is_f64(int kind) { return base_kind(kind) == kF64R18 || base_kind(kind) == kF64R12; }
inline bool kind_is_ds(int kind) { return base_kind(kind) == kDSR18 || base_kind(kind) == kDSR12; }
// bytes of one stored phase: (cos, sin) as double2 for FP64 and double-single links, a float
// angle otherwise
inline int theta_bytes(int kind) { return kind_is_f64(kind) || kind_is_ds(kind) ? 16 : 4; }
// bytes per site of the fields a gauge of this kind works on
inline int kind_vec_bytes(int kind) { return kind_is_f64(kind) || kind_is_ds(kind) ? 48 : 24; }

// Launchers, one per storage kind, implemented in dslash_f64.cu / dslash_f32.cu / dslash_h16.cu;
// `bs` is the thread-block size (64, 128 or 256).
cudaError_t launch_dslash_f64r18(const DArgs &a, int mode, int bs, cudaStream_t st);
// links with a U(1) phase field, one right-hand side per group (dslash_u1.cu)
cudaError_t launch_dslash_u1(int kind, const DArgs &a, int mode, int bs, cudaStream_t st);
cudaError_t launch_dslash_f64r12(const DArgs &a, int mode, int bs, cudaStream_t st);
cudaError_t launch_dslash_f32r18(const DArgs &a, int mode, int bs, cudaStream_t st);
cudaError_t launch_dslash_f32r12(const DArgs &a, int mode, int bs, cudaStream_t st);
cudaError_t launch_dslash_bf16r12(const DArgs &a, int mode, int bs, cudaStream_t st);
cudaError_t launch_dslash_f16r12(const DArgs &a, int mode, int bs, cudaStream_t st);
cudaError_t launch_dslash_dsr18(const DArgs &a, int mode, int bs, cudaStream_t st);
cudaError_t launch_dslash_dsr12(const DArgs &a, int mode, int bs, cudaStream_t st);
// Launches the D kernel for storage `kind` with the autotuned block size (stg_core.cu).
cudaError_t launch_dslash(int kind, const DArgs &a, int mode, cudaStream_t st);
cudaError_t launch_dslash_bs(int kind, const DArgs &a, int mode, int bs, cudaStream_t st);

// Pack canonical complex128 links [4][V][3][3] into the internal layout of `kind`.
cudaError_t launch_pack_links(int kind, const Geom &g, const void *canon, void *links, cudaStream_t st);
// canonical complex64 field <-> internal layout of vec_prec (stg_core.cu)
cudaError_t launch_field_pack_c64(stg_prec vec_prec, int Vh, const void *canon, void *internal, cudaStream_t st);
cudaError_t launch_field_unpack_c64(stg_prec vec_prec, int Vh, const void *internal, void *canon, cudaStream_t st);

// F32 12-real copy of an F64 gauge (created on first use, owned by the F64 gauge): the operator
// of the refinement iterations when the multi-shift phase runs on 16-bit links.
stg_status f32_companion(const stg_gauge *g64, cudaStream_t st, const stg_gauge **out);
// Double-single copy of an F64 gauge, same compression (created on first use, owned by the F64
// gauge): the operator of the mixed solver's FP64-accurate residuals, run on the FP32 pipes.
stg_status ds_companion(const stg_gauge *g64, cudaStream_t st, const stg_gauge **out);

// Error reporting (thread-local message read by stg_last_error).
stg_status set_error(stg_status s, const std::string &msg);
stg_status cuda_error(cudaError_t e, const char *where);

}  // namespace stg

struct stg_lattice {
    stg::Geom g;
    long long V;
};

struct stg_gauge {
    const stg_lattice *lat;
    stg::Geom g;
    stg_prec prec;
    stg_recon recon;
    int kind;
    void *links;
    size_t bytes;
    double *scratch;       // per-block partial sums of stg_normal_op's reduction
    size_t scratch_count;  // doubles in scratch
    mutable stg_gauge *f32_copy;  // lazily created F32 12-real companion (F64 gauges only)
    mutable stg_gauge *ds_copy;   // lazily created double-single companion (F64 gauges only)
};

#define STG_CUDA_TRY(call)                                       \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return stg::cuda_error(e_, #call); \
    } while (0)
