// Mixed-precision polarizability on the tensor cores (placeholder until the
// tcgen05 kernel lands).
#include "runtime.h"

namespace bgw {
int chi_mixed_run(Ctx* c, int prec, long long K, int ng, const void* M, const double* w, int nrow,
                  double scale, int accumulate, void* chi, cudaStream_t st) {
  (void)prec; (void)K; (void)ng; (void)M; (void)w; (void)nrow; (void)scale; (void)accumulate; (void)chi; (void)st;
  return fail(c, BGW_EUNSUPPORTED, "mixed-precision chi is not built yet");
}
}  // namespace bgw
