// fse_kernel_fixw.cu -- the persistent concealment kernel for image classes of
// FFT size 64 with reduced-precision residual storage (16-bit fixed-point W
// after the first updates), 128 and 256 threads per CTA.
#include "fse_kernels.cuh"

namespace fse {

template <int NT>
static cudaError_t prepare_nt(size_t smem, int *ctas_per_sm) {
    cudaError_t e =
        cudaFuncSetAttribute(fse_batch_kernel<NT, kSetFixW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, fse_batch_kernel<NT, kSetFixW>, NT, smem);
}

cudaError_t batch_kernel_prepare_fixw(int nt, size_t smem, int *ctas_per_sm) {
    return nt == 256 ? prepare_nt<256>(smem, ctas_per_sm) : prepare_nt<128>(smem, ctas_per_sm);
}

cudaError_t batch_kernel_launch_fixw(int nt, int grid, size_t smem, cudaStream_t s, const DevParams &P) {
    if (nt == 256) fse_batch_kernel<256, kSetFixW><<<grid, 256, smem, s>>>(P);
    else fse_batch_kernel<128, kSetFixW><<<grid, 128, smem, s>>>(P);
    return cudaGetLastError();
}
}  // namespace fse
