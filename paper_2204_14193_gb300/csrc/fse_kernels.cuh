// fse_kernels.cuh -- host-side entry points of the persistent concealment
// kernel.  Each kernel set (fse_device.cuh: kSetImage, kSetExt, kSetF64) is
// instantiated in a translation unit of its own (fse_kernel_*.cu), so the
// instantiations compile in parallel and a host file never instantiates them.
#pragma once

#include <cuda_runtime.h>

#include "fse_device.cuh"

namespace fse {

// Smallest kernel set that conceals every class of a batch: reduced-precision
// residual storage runs kSetFixW (FFT-64 image classes only, traced or not);
// other traced batches run kSetTrace; video volumes or ordered concealment
// need kSetExt; image classes of FFT size 64 alone run kSetF64; any other mix
// of image classes kSetImage.
int kernel_set_for(bool ext, bool all_f64, bool trace = false, bool fixw = false);

// Sets the dynamic shared-memory limit of the instantiation (ks, nt) to smem
// bytes and returns in *ctas_per_sm how many of its CTAs fit on an SM.
cudaError_t batch_kernel_prepare(int ks, int nt, size_t smem, int *ctas_per_sm);

// One persistent launch of the instantiation (ks, nt) on stream s.
cudaError_t batch_kernel_launch(int ks, int nt, int grid, size_t smem, cudaStream_t s, const DevParams &P);

// the per-set definitions (fse_kernel_image.cu, fse_kernel_ext.cu and
// fse_kernel_ext256.cu, fse_kernel_trace.cu and fse_kernel_trace256.cu,
// fse_kernel_f64.cu, fse_kernel_fixw.cu)
cudaError_t batch_kernel_prepare_image(int nt, size_t smem, int *ctas_per_sm);
cudaError_t batch_kernel_launch_image(int nt, int grid, size_t smem, cudaStream_t s, const DevParams &P);
cudaError_t batch_kernel_prepare_ext(int nt, size_t smem, int *ctas_per_sm);
cudaError_t batch_kernel_launch_ext(int nt, int grid, size_t smem, cudaStream_t s, const DevParams &P);
cudaError_t batch_kernel_prepare_ext256(size_t smem, int *ctas_per_sm);
cudaError_t batch_kernel_launch_ext256(int grid, size_t smem, cudaStream_t s, const DevParams &P);
cudaError_t batch_kernel_prepare_trace(int nt, size_t smem, int *ctas_per_sm);
cudaError_t batch_kernel_launch_trace(int nt, int grid, size_t smem, cudaStream_t s, const DevParams &P);
cudaError_t batch_kernel_prepare_trace256(size_t smem, int *ctas_per_sm);
cudaError_t batch_kernel_launch_trace256(int grid, size_t smem, cudaStream_t s, const DevParams &P);
cudaError_t batch_kernel_prepare_f64(int nt, size_t smem, int *ctas_per_sm);
cudaError_t batch_kernel_launch_f64(int nt, int grid, size_t smem, cudaStream_t s, const DevParams &P);
cudaError_t batch_kernel_prepare_fixw(int nt, size_t smem, int *ctas_per_sm);
cudaError_t batch_kernel_launch_fixw(int nt, int grid, size_t smem, cudaStream_t s, const DevParams &P);

}  // namespace fse
