// fse_peaks.cu -- measured shared-memory bandwidth of the device, the
// denominator of the concealment kernel's roofline.
//
// The concealment iterations read one 8-byte W operand per bin from shared
// memory (16-byte LDS per register pair).  The peak they are measured against
// is what a plain stream of conflict-free 16-byte shared-memory loads reaches
// on every SM of the device, timed with CUDA events: one CTA of 1024 threads
// per SM, 32 KB of shared memory, eight independent loads in flight per
// thread, the loaded words folded into a value that is written out so that no
// load can be dropped.
#include <cuda_runtime.h>

#include <cstdio>

#include "fse.h"
#include "fse_alloc.cuh"

void fse_internal_set_global_error(const char *msg);   // fse_api.cu: text of fse_last_error(NULL)

namespace {

constexpr int kThreads = 1024;
constexpr int kWords = 32 * 1024 / 16;   // uint4 words of the shared buffer (32 KB)
constexpr int kUnroll = 8;

__global__ void __launch_bounds__(kThreads, 1) smem_stream_kernel(int rounds, unsigned *out) {
    __shared__ uint4 buf[kWords];
    for (int i = threadIdx.x; i < kWords; i += kThreads)
        buf[i] = make_uint4(i, i * 3u + 1u, i * 5u + 2u, i * 7u + 3u);
    __syncthreads();
    unsigned acc[kUnroll] = {};
    // consecutive lanes read consecutive 16-byte words (conflict-free); the
    // kUnroll loads of a round read kUnroll different words, and every round
    // moves on by one warp's width
    constexpr int kStride = kWords / kUnroll;
    int base = threadIdx.x;
    for (int r = 0; r < rounds; ++r) {
#pragma unroll
        for (int k = 0; k < kUnroll; ++k) {
            const uint4 v = buf[(base + k * kStride) & (kWords - 1)];
            acc[k] ^= v.x ^ v.y ^ v.z ^ v.w;
        }
        base = (base + 32) & (kWords - 1);
    }
    unsigned a = 0;
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) a ^= acc[k];
    if (a == 0x9e3779b9u) out[blockIdx.x] = a;   // practically never; keeps the loads
}

}  // namespace

extern "C" fse_status fse_measure_smem_bandwidth(int device, double *gbytes_per_s) {
    if (!gbytes_per_s) {
        fse_internal_set_global_error("fse_measure_smem_bandwidth: result pointer is NULL");
        return FSE_ERR_INVALID_ARG;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) {
        fse_internal_set_global_error("fse_measure_smem_bandwidth: cannot select the device");
        return FSE_ERR_INVALID_ARG;
    }
    fse_status st = FSE_OK;
    int sms = 0;
    unsigned *d_out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t s = nullptr;
    float ms = 0.f;
    const int rounds = 4096;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        fse::dev_malloc(&d_out, sizeof(unsigned) * sms) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        st = FSE_ERR_CUDA;
    } else {
        smem_stream_kernel<<<sms, kThreads, 0, s>>>(rounds, d_out);   // warm-up
        float best = 1e30f;
        for (int rep = 0; rep < 5 && st == FSE_OK; ++rep) {
            cudaEventRecord(e0, s);
            smem_stream_kernel<<<sms, kThreads, 0, s>>>(rounds, d_out);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                st = FSE_ERR_CUDA;
            else if (ms < best)
                best = ms;
        }
        if (st == FSE_OK) {
            const double bytes = (double)sms * kThreads * rounds * kUnroll * 16.0;
            *gbytes_per_s = bytes / (best * 1e-3) / 1e9;
        }
    }
    if (st != FSE_OK) fse_internal_set_global_error("fse_measure_smem_bandwidth: a CUDA call failed");
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (d_out) fse::dev_free(d_out);
    if (prev >= 0) cudaSetDevice(prev);
    return st;
}
