// snap_zb_f64.cu -- FP64 instantiation of compute_zi + compute_bi (the plain
// FP64 path).  The Clebsch-Gordan factors come from a global-memory FP64 table;
// the warp assignment of the triples is the same as in the FP32 kernel.
#include "snap_zb.cuh"

namespace mala {

int upload_zb_lists_f64(const int* lists, int bytes) {
    MALA_CUDA_TRY(cudaMemcpyToSymbol(c_zb_list, lists, (size_t)bytes));
    return MALA_OK;
}

template <>
void launch_zb<double>(Ctx* c, int twojmax, const double* u_half, const BatchSnap* bs, int nsnap, int64_t tile0,
                       int64_t ntiles, const int*, double, double* B, cudaStream_t st, int) {
    if (ntiles <= 0) return;
    cudaFuncSetAttribute(k_zb<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    zb_launch_impl<double>(nullptr, twojmax, u_half, bs, nsnap, tile0, ntiles, c->tables.cg_d, B, st);
}

}  // namespace mala
