// The FP32 marching kernels with the force term on the tensor cores
// (mma.sync; 3xTF32 or split-BF16 products, FP32 accumulation): the
// instantiations of the 2D pair kernel and the 1D line kernel for the
// velocity slabs that tile into 16 x 8 x 8 blocks.
#include "hlb_line.cuh"
#include "hlb_pair.cuh"

namespace hlb {

#define HLB_TC_LIST(X) X(16, 8) X(32, 16)

bool force_tc_available(int QX2, int VY) {
#define HLB_AV(A, B) if (QX2 == A && VY == B) return true;
    HLB_TC_LIST(HLB_AV)
#undef HLB_AV
    return false;
}

namespace {
template <int FM>
cudaError_t prepare_tc_form(bool pair, int adv, int QX2, int VY) {
#define HLB_PR(A, B)                                                                                    \
    if (QX2 == A && VY == B) {                                                                          \
        if (pair) return adv == HLB_WENO5_ ? prepare_pair_t<HLB_WENO5_, A, B, FM>()                     \
                                           : prepare_pair_t<HLB_UPWIND2_, A, B, FM>();                  \
        return adv == HLB_WENO5_ ? prepare_line_t<HLB_WENO5_, A, B, FM>() : prepare_line_t<HLB_UPWIND2_, A, B, FM>(); \
    }
    HLB_TC_LIST(HLB_PR)
#undef HLB_PR
    return cudaErrorInvalidValue;
}

template <int FM>
void launch_tc_form(bool pair, int adv, int QX2, int VY, const GroupDev& g, const Work* works, int nworks,
                    const void* fs, const void* fn, void* fo, int stage, cudaStream_t st) {
#define HLB_LA(A, B)                                                                                                \
    if (QX2 == A && VY == B) {                                                                                      \
        if (pair) {                                                                                                 \
            if (adv == HLB_WENO5_) launch_pair_t<HLB_WENO5_, A, B, FM>(g, works, nworks, fs, fn, fo, stage, st);   \
            else launch_pair_t<HLB_UPWIND2_, A, B, FM>(g, works, nworks, fs, fn, fo, stage, st);                   \
        } else {                                                                                                    \
            if (adv == HLB_WENO5_) launch_line_t<HLB_WENO5_, A, B, FM>(g, works, nworks, fs, fn, fo, stage, st);   \
            else launch_line_t<HLB_UPWIND2_, A, B, FM>(g, works, nworks, fs, fn, fo, stage, st);                   \
        }                                                                                                           \
        return;                                                                                                     \
    }
    HLB_TC_LIST(HLB_LA)
#undef HLB_LA
}
}  // namespace

cudaError_t prepare_pair_tc(int adv, int QX2, int VY, int form) {
    return form == kForceBF16x6 ? prepare_tc_form<kForceBF16x6>(true, adv, QX2, VY)
                                : prepare_tc_form<kForceTF32x3>(true, adv, QX2, VY);
}
cudaError_t prepare_line_tc(int adv, int QX2, int VY, int form) {
    return form == kForceBF16x6 ? prepare_tc_form<kForceBF16x6>(false, adv, QX2, VY)
                                : prepare_tc_form<kForceTF32x3>(false, adv, QX2, VY);
}
void launch_pair_tc(int adv, int QX2, int VY, int form, const GroupDev& g, const Work* works, int nworks,
                    const void* fs, const void* fn, void* fo, int stage, cudaStream_t st) {
    if (form == kForceBF16x6) launch_tc_form<kForceBF16x6>(true, adv, QX2, VY, g, works, nworks, fs, fn, fo, stage, st);
    else launch_tc_form<kForceTF32x3>(true, adv, QX2, VY, g, works, nworks, fs, fn, fo, stage, st);
}
void launch_line_tc(int adv, int QX2, int VY, int form, const GroupDev& g, const Work* works, int nworks,
                    const void* fs, const void* fn, void* fo, int stage, cudaStream_t st) {
    if (form == kForceBF16x6) launch_tc_form<kForceBF16x6>(false, adv, QX2, VY, g, works, nworks, fs, fn, fo, stage, st);
    else launch_tc_form<kForceTF32x3>(false, adv, QX2, VY, g, works, nworks, fs, fn, fo, stage, st);
}

}  // namespace hlb
