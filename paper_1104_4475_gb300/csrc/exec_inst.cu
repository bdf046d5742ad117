// One instantiation of the persistent executor, exec_kernel<TQR_G, TQR_PREC>:
// the build compiles this file once per (G, PREC) pair with -DTQR_G=...
// -DTQR_PREC=..., so the nine kernels compile in parallel.
#include "executor.cuh"

#if !defined(TQR_G) || !defined(TQR_PREC)
#error "compile with -DTQR_G=<4|8|16> -DTQR_PREC=<0|1|2>"
#endif

namespace tqr {

template <int G, int PREC>
cudaError_t launch_exec(const ExecParams& P, int smem, int grid, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(exec_kernel<G, PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    exec_kernel<G, PREC><<<grid, kThreads, smem, s>>>(P);
    return cudaGetLastError();
}

template cudaError_t launch_exec<TQR_G, TQR_PREC>(const ExecParams&, int, int, cudaStream_t);

}  // namespace tqr
