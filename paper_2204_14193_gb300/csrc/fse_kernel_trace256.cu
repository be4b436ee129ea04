// fse_kernel_trace256.cu -- the persistent concealment kernel for video volumes
// and ordered concealment as well, 256 threads per CTA.
#include "fse_kernels.cuh"

namespace fse {

cudaError_t batch_kernel_prepare_trace256(size_t smem, int *ctas_per_sm) {
    cudaError_t e =
        cudaFuncSetAttribute(fse_batch_kernel<256, kSetTrace>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, fse_batch_kernel<256, kSetTrace>, 256, smem);
}

cudaError_t batch_kernel_launch_trace256(int grid, size_t smem, cudaStream_t s, const DevParams &P) {
    fse_batch_kernel<256, kSetTrace><<<grid, 256, smem, s>>>(P);
    return cudaGetLastError();
}

}  // namespace fse
