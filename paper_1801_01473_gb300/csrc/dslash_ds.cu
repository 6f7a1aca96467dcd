// D_eo / D_oe instantiations for double-single (FP32-pair) links on double-single fields:
// FP64-class results computed on the FP32 pipes (the FP64-accurate residuals of the mixed solver).
// The operator is FP32-ALU bound, so the launcher always splits multi-rhs launches into one-rhs
// groups: only the one-rhs kernels are instantiated.
#include "stg_common.h"

namespace stg {
namespace {
template <typename LinkT>
cudaError_t launch_one_rhs(const DArgs &a, int mode, int bs, cudaStream_t st)
{
    int maxv, maxr;
    dslash_extent(a, maxv, maxr);
    if (a.ngroups <= 0 || maxv <= 0 || maxr <= 0) return cudaSuccess;
    if (maxr != 1) return cudaErrorInvalidValue;
    return launch_dslash_n<LinkT, 1>(a, mode, maxv, bs, st);
}
}  // namespace

cudaError_t launch_dslash_dsr18(const DArgs &a, int mode, int bs, cudaStream_t st) { return launch_one_rhs<LinkDSR18>(a, mode, bs, st); }
cudaError_t launch_dslash_dsr12(const DArgs &a, int mode, int bs, cudaStream_t st) { return launch_one_rhs<LinkDSR12>(a, mode, bs, st); }
}  // namespace stg
