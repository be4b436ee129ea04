// fse_kernel_f64.cu -- the persistent concealment kernel for image classes of
// FFT size 64 only (the paper's 48 x 48 areas in a 64 x 64 FFT), 128 and 256
// threads per CTA.
#include "fse_kernels.cuh"

namespace fse {

template <int NT>
static cudaError_t prepare_nt(size_t smem, int *ctas_per_sm) {
    cudaError_t e =
        cudaFuncSetAttribute(fse_batch_kernel<NT, kSetF64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, fse_batch_kernel<NT, kSetF64>, NT, smem);
}

cudaError_t batch_kernel_prepare_f64(int nt, size_t smem, int *ctas_per_sm) {
    return nt == 256 ? prepare_nt<256>(smem, ctas_per_sm) : prepare_nt<128>(smem, ctas_per_sm);
}

cudaError_t batch_kernel_launch_f64(int nt, int grid, size_t smem, cudaStream_t s, const DevParams &P) {
    if (nt == 256) fse_batch_kernel<256, kSetF64><<<grid, 256, smem, s>>>(P);
    else fse_batch_kernel<128, kSetF64><<<grid, 128, smem, s>>>(P);
    return cudaGetLastError();
}
}  // namespace fse
