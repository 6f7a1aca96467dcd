// D_eo / D_oe instantiations for links carrying a U(1) phase field (LinkU1: exp(i theta) U, the
// per-flavour phases of Sec. 4.1).  Groups hold one right-hand side each (the launcher splits
// multi-rhs launches), which keeps the instantiation count small.
#include "stg_common.h"

namespace stg {
namespace {
template <typename LinkT>
cudaError_t launch_u1_t(const DArgs &a, int mode, int bs, cudaStream_t st)
{
    int maxv, maxr;
    dslash_extent(a, maxv, maxr);
    if (a.ngroups <= 0 || maxv <= 0 || maxr <= 0) return cudaSuccess;
    if (maxr != 1) return cudaErrorInvalidValue;
    return launch_dslash_n<LinkT, 1>(a, mode, maxv, bs, st);
}
}  // namespace

cudaError_t launch_dslash_u1(int kind, const DArgs &a, int mode, int bs, cudaStream_t st)
{
    switch (base_kind(kind)) {
    case kF64R18: return launch_u1_t<LinkU1<LinkF64R18, double2>>(a, mode, bs, st);
    case kF64R12: return launch_u1_t<LinkU1<LinkF64R12, double2>>(a, mode, bs, st);
    case kF32R18: return launch_u1_t<LinkU1<LinkF32R18, float>>(a, mode, bs, st);
    case kF32R12: return launch_u1_t<LinkU1<LinkF32R12, float>>(a, mode, bs, st);
    case kBF16R12: return launch_u1_t<LinkU1<Link16R12<__nv_bfloat16>, float>>(a, mode, bs, st);
    case kF16R12: return launch_u1_t<LinkU1<Link16R12<__half>, float>>(a, mode, bs, st);
    case kDSR18: return launch_u1_t<LinkU1<LinkDSR18, double2>>(a, mode, bs, st);
    case kDSR12: return launch_u1_t<LinkU1<LinkDSR12, double2>>(a, mode, bs, st);
    }
    return cudaErrorInvalidValue;
}
}  // namespace stg
