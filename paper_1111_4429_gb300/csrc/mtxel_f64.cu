// FP64 instantiation of the matrix-element kernels (plain path).
#include "mtxel_kernels.cuh"

namespace bgw {
cudaError_t mtxel_exec_f64(const MtxelExec& x) { return mtxel_exec_t<double>(x); }
cudaError_t mtxel_init_f64() { return upload_twiddles(); }
}  // namespace bgw
