// fse_tables.cuh -- constant tables of the concealment kernel, computed on
// the device once per handle (or per call of the allocation-free entry).
// The kernels have internal linkage: every translation unit that launches
// them includes its own copy.
#pragma once

#include <cuda_runtime.h>

namespace fse {

// Eq. (3) weight table of one class, evaluated in FP64 and rounded once; for
// a volume of T frames the distance includes the frame offset from the
// centre frame (T = 1: the area's table).
static __global__ void weight_table_kernel(float *wtab, int M, int T, double rho) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= T * M * M) return;
    const int tau = i / (M * M), m = (i / M) % M, n = i % M;
    const double cm = 0.5 * (M - 1), ct = 0.5 * (T - 1);
    const double dist = sqrt((tau - ct) * (tau - ct) + (m - cm) * (m - cm) + (n - cm) * (n - cm));
    wtab[i] = (float)pow(rho, dist);
}

// (cos, sin)(2 pi t / 64), FP64 then rounded once.
static __global__ void twiddle_kernel(float2 *tw) {
    const int t = threadIdx.x;
    if (t >= 64) return;
    double s, c;
    sincospi((double)t / 32.0, &s, &c);
    tw[t] = make_float2((float)c, (float)s);
}

}  // namespace fse
