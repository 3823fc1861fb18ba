// FP32 instantiation of the matrix-element kernels (mixed-precision path:
// complex64 grids and M, FP64 input coefficients rounded once on load).
#include "mtxel_kernels.cuh"

namespace bgw {
cudaError_t mtxel_exec_f32(const MtxelExec& x) { return mtxel_exec_t<float>(x); }
cudaError_t mtxel_init_f32() { return upload_twiddles(); }
}  // namespace bgw
