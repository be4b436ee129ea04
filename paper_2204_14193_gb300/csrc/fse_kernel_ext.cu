// fse_kernel_ext.cu -- the persistent concealment kernel for video volumes and
// ordered concealment as well, 128 threads per CTA (the 256-thread
// instantiation is in fse_kernel_ext256.cu: the two compile in parallel).
#include "fse_kernels.cuh"

namespace fse {

template <int NT>
static cudaError_t prepare_nt(size_t smem, int *ctas_per_sm) {
    cudaError_t e =
        cudaFuncSetAttribute(fse_batch_kernel<NT, kSetExt>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, fse_batch_kernel<NT, kSetExt>, NT, smem);
}

cudaError_t batch_kernel_prepare_ext(int nt, size_t smem, int *ctas_per_sm) {
    return nt == 256 ? batch_kernel_prepare_ext256(smem, ctas_per_sm) : prepare_nt<128>(smem, ctas_per_sm);
}

cudaError_t batch_kernel_launch_ext(int nt, int grid, size_t smem, cudaStream_t s, const DevParams &P) {
    if (nt == 256) return batch_kernel_launch_ext256(grid, smem, s, P);
    fse_batch_kernel<128, kSetExt><<<grid, 128, smem, s>>>(P);
    return cudaGetLastError();
}
}  // namespace fse
