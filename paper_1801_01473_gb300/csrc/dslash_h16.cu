// D_eo / D_oe instantiations for 16-bit (bf16 or fp16) 12-real links; FP32 arithmetic on FP32 fields.
#include "stg_common.h"

namespace stg {
cudaError_t launch_dslash_bf16r12(const DArgs &a, int mode, int bs, cudaStream_t st) { return launch_dslash_t<Link16R12<__nv_bfloat16>>(a, mode, bs, st); }
cudaError_t launch_dslash_f16r12(const DArgs &a, int mode, int bs, cudaStream_t st) { return launch_dslash_t<Link16R12<__half>>(a, mode, bs, st); }
}  // namespace stg
