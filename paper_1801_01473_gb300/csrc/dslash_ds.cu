// D_eo / D_oe instantiations for double-single (FP32-pair) links on double-single fields:
// FP64-class results computed on the FP32 pipes (the FP64-accurate residuals of the mixed solver).
#include "stg_common.h"

namespace stg {
cudaError_t launch_dslash_dsr18(const DArgs &a, int mode, int bs, cudaStream_t st) { return launch_dslash_t<LinkDSR18>(a, mode, bs, st); }
cudaError_t launch_dslash_dsr12(const DArgs &a, int mode, int bs, cudaStream_t st) { return launch_dslash_t<LinkDSR12>(a, mode, bs, st); }
}  // namespace stg
