// Fourier neural operator (filled in below).
#include "nn_kernels.cuh"

namespace nop {
int fno_forward_raw(nop_ctx* ctx, int, const float*, int, int, float*, bool) {
    ctx->set_error("FNO not available");
    return NOP_EINVAL;
}
int fno_backward(nop_ctx* ctx, int, int, int, const float*) {
    ctx->set_error("FNO not available");
    return NOP_EINVAL;
}
int fno_recast(nop_ctx* ctx, double, int, double*, int*, int*, bool, const double*) {
    ctx->set_error("FNO not available");
    return NOP_EINVAL;
}
}  // namespace nop
