// fse_kernel_image.cu -- the persistent concealment kernel for image classes of
// every FFT size, 128 and 256 threads per CTA; the dispatch over the kernel
// sets.
#include "fse_kernels.cuh"

namespace fse {

template <int NT>
static cudaError_t prepare_nt(size_t smem, int *ctas_per_sm) {
    cudaError_t e =
        cudaFuncSetAttribute(fse_batch_kernel<NT, kSetImage>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, fse_batch_kernel<NT, kSetImage>, NT, smem);
}

cudaError_t batch_kernel_prepare_image(int nt, size_t smem, int *ctas_per_sm) {
    return nt == 256 ? prepare_nt<256>(smem, ctas_per_sm) : prepare_nt<128>(smem, ctas_per_sm);
}

cudaError_t batch_kernel_launch_image(int nt, int grid, size_t smem, cudaStream_t s, const DevParams &P) {
    if (nt == 256) fse_batch_kernel<256, kSetImage><<<grid, 256, smem, s>>>(P);
    else fse_batch_kernel<128, kSetImage><<<grid, 128, smem, s>>>(P);
    return cudaGetLastError();
}

int kernel_set_for(bool ext, bool all_f64, bool trace, bool fixw) {
    return fixw ? kSetFixW : trace ? kSetTrace : ext ? kSetExt : all_f64 ? kSetF64 : kSetImage;
}

cudaError_t batch_kernel_prepare(int ks, int nt, size_t smem, int *ctas_per_sm) {
    if (ks == kSetExt) return batch_kernel_prepare_ext(nt, smem, ctas_per_sm);
    if (ks == kSetTrace) return batch_kernel_prepare_trace(nt, smem, ctas_per_sm);
    if (ks == kSetF64) return batch_kernel_prepare_f64(nt, smem, ctas_per_sm);
    if (ks == kSetFixW) return batch_kernel_prepare_fixw(nt, smem, ctas_per_sm);
    return batch_kernel_prepare_image(nt, smem, ctas_per_sm);
}

cudaError_t batch_kernel_launch(int ks, int nt, int grid, size_t smem, cudaStream_t s, const DevParams &P) {
    if (ks == kSetExt) return batch_kernel_launch_ext(nt, grid, smem, s, P);
    if (ks == kSetTrace) return batch_kernel_launch_trace(nt, grid, smem, s, P);
    if (ks == kSetF64) return batch_kernel_launch_f64(nt, grid, smem, s, P);
    if (ks == kSetFixW) return batch_kernel_launch_fixw(nt, grid, smem, s, P);
    return batch_kernel_launch_image(nt, grid, smem, s, P);
}
}  // namespace fse
