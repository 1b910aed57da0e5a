// The 2D FP32 stage kernel with the FMA force term: instantiations and
// dispatch (the tensor-core forms are instantiated in hlb_tc.cu).
#include "hlb_pair.cuh"

namespace hlb {

#define HLB_PAIR_LIST(X) X(8, 4) X(16, 8) X(32, 16)

bool pair_available(int QX2, int VY) {
#define HLB_AV(A, B) if (QX2 == A && VY == B) return true;
    HLB_PAIR_LIST(HLB_AV)
#undef HLB_AV
    return false;
}

cudaError_t prepare_pair(int adv, int QX2, int VY, int form) {
    if (form >= kForceField) {          // FMA force term with a field (FF) and / or stochastic rounding (SR)
        const int ff = form != kForceFMASR, sr = form != kForceField;
#define HLB_PRF(A, B)                                                                                   \
        if (QX2 == A && VY == B) {                                                                      \
            if (adv == HLB_WENO5_)                                                                      \
                return ff ? (sr ? prepare_pair_t<HLB_WENO5_, A, B, kForceFMA, 1, 1>()                   \
                                : prepare_pair_t<HLB_WENO5_, A, B, kForceFMA, 1, 0>())                  \
                          : prepare_pair_t<HLB_WENO5_, A, B, kForceFMA, 0, 1>();                        \
            return ff ? (sr ? prepare_pair_t<HLB_UPWIND2_, A, B, kForceFMA, 1, 1>()                     \
                            : prepare_pair_t<HLB_UPWIND2_, A, B, kForceFMA, 1, 0>())                    \
                      : prepare_pair_t<HLB_UPWIND2_, A, B, kForceFMA, 0, 1>();                          \
        }
        HLB_PAIR_LIST(HLB_PRF)
#undef HLB_PRF
        return cudaErrorInvalidValue;
    }
    if (form != kForceFMA) return prepare_pair_tc(adv, QX2, VY, form);
#define HLB_PR(A, B)                                                                          \
    if (QX2 == A && VY == B)                                                                  \
        return adv == HLB_WENO5_ ? prepare_pair_t<HLB_WENO5_, A, B, kForceFMA>()              \
                                 : prepare_pair_t<HLB_UPWIND2_, A, B, kForceFMA>();
    HLB_PAIR_LIST(HLB_PR)
#undef HLB_PR
    return cudaErrorInvalidValue;
}

void launch_pair(int adv, int QX2, int VY, int form, const GroupDev& g, const Work* works, int nworks,
                 const void* fs, const void* fn, void* fo, int stage, cudaStream_t st) {
    if (form >= kForceField) {
        const int ff = form != kForceFMASR, sr = form != kForceField;
#define HLB_LAF(A, B)                                                                                       \
        if (QX2 == A && VY == B) {                                                                          \
            if (adv == HLB_WENO5_) {                                                                        \
                if (!sr) launch_pair_t<HLB_WENO5_, A, B, kForceFMA, 1, 0>(g, works, nworks, fs, fn, fo, stage, st); \
                else if (ff) launch_pair_t<HLB_WENO5_, A, B, kForceFMA, 1, 1>(g, works, nworks, fs, fn, fo, stage, st); \
                else launch_pair_t<HLB_WENO5_, A, B, kForceFMA, 0, 1>(g, works, nworks, fs, fn, fo, stage, st); \
            } else {                                                                                         \
                if (!sr) launch_pair_t<HLB_UPWIND2_, A, B, kForceFMA, 1, 0>(g, works, nworks, fs, fn, fo, stage, st); \
                else if (ff) launch_pair_t<HLB_UPWIND2_, A, B, kForceFMA, 1, 1>(g, works, nworks, fs, fn, fo, stage, st); \
                else launch_pair_t<HLB_UPWIND2_, A, B, kForceFMA, 0, 1>(g, works, nworks, fs, fn, fo, stage, st); \
            }                                                                                               \
            return;                                                                                         \
        }
        HLB_PAIR_LIST(HLB_LAF)
#undef HLB_LAF
        return;
    }
    if (form != kForceFMA) {
        launch_pair_tc(adv, QX2, VY, form, g, works, nworks, fs, fn, fo, stage, st);
        return;
    }
#define HLB_LA(A, B)                                                                                          \
    if (QX2 == A && VY == B) {                                                                                \
        if (adv == HLB_WENO5_) launch_pair_t<HLB_WENO5_, A, B, kForceFMA>(g, works, nworks, fs, fn, fo, stage, st); \
        else launch_pair_t<HLB_UPWIND2_, A, B, kForceFMA>(g, works, nworks, fs, fn, fo, stage, st);              \
        return;                                                                                               \
    }
    HLB_PAIR_LIST(HLB_LA)
#undef HLB_LA
}

}  // namespace hlb
