// snap_yi_g2.cu -- unit kernel of coupling group 2 of the FP32 Y step
// (snap_yi.cuh); the group's couplings are those whose coupled momentum c is
// in yi_mask(2).
#include "snap_yi.cuh"

namespace mala {

int yi_upload_g2(const float* cg, int n, const int* info, const float* fnorm) {
    return yi_upload<yi_mask(2)>(cg, n, info, fnorm);
}
int yi_launch_g2(const YiLaunch& a) { return yi_launch<yi_mask(2)>(a); }

}  // namespace mala
