// snap_zb_alt.cu -- the FP32 compute_zi + compute_bi kernel with another
// warp count per CTA (kZbWarpsAlt; more registers a thread, fewer warps to
// hide latency), one of the shapes the tuner times.  Compiled apart from
// snap_zb.cu so the two instantiations build in parallel; it holds its own
// copy of the constant tables, uploaded beside the default one's.
#include "snap_zb.cuh"

namespace mala {

int upload_zb_alt_cg(const float2* cg2, int bytes) {
    MALA_CUDA_TRY(cudaMemcpyToSymbol(c_cg2, cg2, (size_t)bytes));
    return MALA_OK;
}

int upload_zb_alt_jp1(const float* jp1, int bytes, int offset) {
    MALA_CUDA_TRY(cudaMemcpyToSymbol(c_zb_jp1, jp1, (size_t)bytes, (size_t)offset));
    return MALA_OK;
}

void launch_zb_alt(Ctx* c, int twojmax, const float* u_half, const BatchSnap* bs, int nsnap, int64_t tile0,
                   int64_t ntiles, const int* nbr_cnt, double wself, float* B, cudaStream_t st) {
    zb_units_launch<kZbWarpsAlt>(c, twojmax, u_half, bs, nsnap, tile0, ntiles, nbr_cnt, wself, B, st);
}

}  // namespace mala
