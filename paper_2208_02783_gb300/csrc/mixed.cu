// Mixed-precision slot engine (placeholder until the FP32 iteration lands).
#include "mixed.cuh"

namespace transec {

int run_mixed(transec_ctx* ctx, int, int, const double*, const int*, const long long*, double*,
              double*, int*, int*) {
  ctx->err = "mixed precision is not built yet";
  return TRANSEC_EINVAL;
}

}  // namespace transec
