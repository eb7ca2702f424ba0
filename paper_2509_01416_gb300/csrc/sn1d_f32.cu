// FP32 instantiation of the batched 1D slab solver (see sn1d_impl.cuh).
#include "sn1d_impl.cuh"

namespace nop {
template int sn1d_run<float>(nop_ctx*, const nop_solve_opts*, bool, const double*, const double*,
                          double*, bool, double*, nop_stats*);
}  // namespace nop
