// FP32 instantiation of the batched 1D slab solver (see sn1d_impl.cuh).
#include "sn1d_impl.cuh"

namespace nop {
template int sn1d_run<float>(nop_ctx*, const nop_solve_opts*, bool, const double*, const double*,
                          double*, bool, double*, nop_stats*);
}  // namespace nop

namespace nop {
// Raises sn1d_kernel<float>'s dynamic shared-memory limit to
// SN1D_STAGE_BYTES on the current device (once per device before
// sn1d_launch_f32; the allocation-free entry point's set-up).
int sn1d_f32_raise_smem_limit() {
    return cudaFuncSetAttribute(sn1d_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)SN1D_STAGE_BYTES) == cudaSuccess
               ? NOP_OK
               : NOP_ECUDA;
}

// Launch sequence of one single-group slab solve whose every buffer the
// caller supplies (used by the allocation-free entry point): preparation,
// the persistent solve kernel on one block, conversion of the flux.  The
// caller has raised sn1d_kernel<float>'s dynamic shared-memory limit to
// SN1D_STAGE_BYTES on this device beforehand.
int sn1d_launch_f32(const Sn1dArgs& a, long long C, const double* sigt, const double* sigs,
                    const double* src, Cell4<float>* X, float* ext, double* phi_out,
                    cudaStream_t stream) {
    const int pb = (int)std::max<long long>(1, std::min<long long>((C + 255) / 256, 1024));
    sn1d_prepare<float><<<pb, 256, 0, stream>>>(C, 1, sigt, sigs, src, nullptr, nullptr, 0, X,
                                                nullptr, ext, nullptr, nullptr, nullptr, nullptr);
    sn1d_kernel<float><<<1, SN1D_THREADS, SN1D_STAGE_BYTES, stream>>>(a);
    sn1d_finish<float><<<pb, 256, 0, stream>>>(C, X, phi_out);
    return cudaGetLastError() == cudaSuccess ? NOP_OK : NOP_ECUDA;
}
}  // namespace nop
