// D_eo / D_oe instantiations for FP64 links (18-real and 12-real) on FP64 fields.
#include "stg_common.h"

namespace stg {
cudaError_t launch_dslash_f64r18(const DArgs &a, int mode, int bs, cudaStream_t st) { return launch_dslash_t<LinkF64R18>(a, mode, bs, st); }
cudaError_t launch_dslash_f64r12(const DArgs &a, int mode, int bs, cudaStream_t st) { return launch_dslash_t<LinkF64R12>(a, mode, bs, st); }
}  // namespace stg
