// fse_cnn.cuh -- sm_103a kernels of the learned-initialisation network.
//
// Network (per extrapolation area of H x W samples): four 3x3 convolutions,
// "same" zero padding, dilations 1, 2, 4, 8, channels 2 -> 32 -> 32 -> 32 -> 1,
// ReLU after the first three.  Input channel 0 is the support sample / 255
// (0 off the support), channel 1 the support indicator; the output is the
// estimate of the whole area / 255.
//
// Precision: weights and stored activations in bfloat16, every product
// accumulated in FP32 (forward on the tensor cores); gradients in FP32.
//
// Layouts: activations NHWC ([pixel][channel], pixel = (n * H + y) * W + x);
// forward weights as the B operand of the implicit GEMM, Wb[n][k] with
// k = tap * Cin + ci (tap = ky * 3 + kx), rows padded to NP (32 or 8) and k to
// a multiple of 16; backward weights Wt[tap][co][ci] FP32.  The flat FP32
// parameter vector holds, per layer, W[co][ci][ky][kx] then b[co].
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstdint>

namespace fse_net {

constexpr int kLayers = 4;
constexpr int kParams = 19393;
__host__ __device__ constexpr int cin_of(int l) { return l == 0 ? 2 : 32; }
__host__ __device__ constexpr int cout_of(int l) { return l == 3 ? 1 : 32; }
__host__ __device__ constexpr int dil_of(int l) { return 1 << l; }
__host__ __device__ constexpr int np_of(int l) { return l == 3 ? 8 : 32; }             // padded N
__host__ __device__ constexpr int kp_of(int l) { return (9 * cin_of(l) + 15) / 16 * 16; }  // padded K
__host__ __device__ constexpr int woff_of(int l) {                                      // W offset in params
    return l == 0 ? 0 : woff_of(l - 1) + cout_of(l - 1) * cin_of(l - 1) * 9 + cout_of(l - 1);
}
__host__ __device__ constexpr int wb_off(int l) { return l == 0 ? 0 : wb_off(l - 1) + np_of(l - 1) * kp_of(l - 1); }
__host__ __device__ constexpr int wt_off(int l) { return l == 0 ? 0 : wt_off(l - 1) + 9 * cout_of(l - 1) * cin_of(l - 1); }
constexpr int kWbTotal = wb_off(kLayers);
constexpr int kWtTotal = wt_off(kLayers);
static_assert(woff_of(kLayers) == kParams, "parameter count");

// ---------------------------------------------------------------- weights
// Flat FP32 parameters -> forward B operands (bf16) and backward weights.
static __global__ void pack_weights_kernel(const float *__restrict__ params, __nv_bfloat16 *__restrict__ wb,
                                    float *__restrict__ wt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    // forward operands
    if (i < kWbTotal) {
        int l = 0;
        while (l + 1 < kLayers && i >= wb_off(l + 1)) ++l;
        const int r = i - wb_off(l), kp = kp_of(l), cin = cin_of(l);
        const int n = r / kp, k = r % kp;
        float v = 0.f;
        if (n < cout_of(l) && k < 9 * cin) {
            const int tap = k / cin, ci = k % cin;
            v = params[woff_of(l) + (n * cin + ci) * 9 + tap];
        }
        wb[i] = __float2bfloat16_rn(v);
    }
    // backward weights (the same bf16-rounded values, held as FP32)
    if (i < kWtTotal) {
        int l = 0;
        while (l + 1 < kLayers && i >= wt_off(l + 1)) ++l;
        const int r = i - wt_off(l), cin = cin_of(l), cout = cout_of(l);
        const int tap = r / (cout * cin), co = (r / cin) % cout, ci = r % cin;
        wt[i] = __bfloat162float(__float2bfloat16_rn(params[woff_of(l) + (co * cin + ci) * 9 + tap]));
    }
}

// FP32 NCHW input [N][2][H][W] -> bf16 NHWC [N*H*W][2]
static __global__ void input_kernel(const float *__restrict__ x, __nv_bfloat162 *__restrict__ xin, int N, int HW) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (long long)N * HW) return;
    const long long n = p / HW, r = p % HW;
    xin[p] = __floats2bfloat162_rn(x[(n * 2) * HW + r], x[(n * 2 + 1) * HW + r]);
}

// ---------------------------------------------------------------- forward
static __device__ __forceinline__ void mma_bf16(float *c, const uint32_t *a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Implicit-GEMM 3x3 dilated convolution, M = pixels, N = output channels,
// K = 9 * Cin.  128 threads; each warp computes 32 pixels x NP channels with
// mma.m16n8k16 (A: 16 pixels x 16 k from the NHWC input, zero outside the
// image; B: 16 k x 8 channels from shared memory).  Epilogue: bias, then
// ReLU + bf16 NHWC store (hidden layers) or FP32 store of channel 0 (output).
template <int L>
__global__ void __launch_bounds__(128) conv_fwd_kernel(const __nv_bfloat16 *__restrict__ in,
                                                       const __nv_bfloat16 *__restrict__ wb_all,
                                                       const float *__restrict__ params, void *__restrict__ out,
                                                       int N, int H, int W) {
    constexpr int CIN = cin_of(L), COUT = cout_of(L), NP = np_of(L), KP = kp_of(L), D = dil_of(L);
    constexpr int NT = NP / 8, KS = KP / 16;
    __shared__ __align__(16) __nv_bfloat16 wsm[NP * KP];
    __shared__ float bsm[NP];
    for (int i = threadIdx.x; i < NP * KP / 2; i += 128)
        reinterpret_cast<uint32_t *>(wsm)[i] = reinterpret_cast<const uint32_t *>(wb_all + wb_off(L))[i];
    for (int i = threadIdx.x; i < NP; i += 128) bsm[i] = i < COUT ? params[woff_of(L) + COUT * CIN * 9 + i] : 0.f;
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, tig = lane & 3;
    const long long P = (long long)N * H * W;
    const long long base = (long long)blockIdx.x * 128 + warp * 32;
    // the four pixels of this thread: rows g, g+8 of m-tiles 0 and 1
    int py[4], px[4];
    long long pimg[4];
    bool pv[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const long long p = base + (r >> 1) * 16 + (r & 1) * 8 + g;
        pv[r] = p < P;
        const long long pc = pv[r] ? p : 0;
        pimg[r] = pc / (H * W) * (long long)(H * W);
        const int rem = (int)(pc % (H * W));
        py[r] = rem / W;
        px[r] = rem % W;
    }
    float acc[2][NT][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.f;

    const uint32_t *in32 = reinterpret_cast<const uint32_t *>(in);
#pragma unroll 2
    for (int ks = 0; ks < KS; ++ks) {
        uint32_t a[2][4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int mt = r >> 1, hi = r & 1;   // hi: row g+8
#pragma unroll
            for (int half = 0; half < 2; ++half) {   // k offset 0 or 8
                int tap, cofs;
                if constexpr (CIN == 2) {
                    tap = ks * 8 + half * 4 + tig;
                    cofs = 0;
                } else {
                    tap = ks >> 1;
                    cofs = (ks & 1) * 16 + half * 8 + tig * 2;
                }
                uint32_t v = 0u;
                if (tap < 9 && pv[r]) {
                    const int yy = py[r] + (tap / 3 - 1) * D, xx = px[r] + (tap % 3 - 1) * D;
                    if (yy >= 0 && yy < H && xx >= 0 && xx < W)
                        v = __ldg(in32 + ((pimg[r] + (long long)yy * W + xx) * CIN + cofs) / 2);
                }
                a[mt][hi + 2 * half] = v;
            }
        }
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            const uint32_t *bp = reinterpret_cast<const uint32_t *>(wsm + (nt * 8 + g) * KP + ks * 16 + tig * 2);
            const uint32_t b0 = bp[0], b1 = bp[4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) mma_bf16(acc[mt][nt], a[mt], b0, b1);
        }
    }
    // epilogue
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int hi = 0; hi < 2; ++hi) {
            const int r = mt * 2 + hi;
            if (!pv[r]) continue;
            const long long p = base + mt * 16 + hi * 8 + g;
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                const int co = nt * 8 + tig * 2;
                const float v0 = acc[mt][nt][hi * 2] + bsm[co];
                const float v1 = acc[mt][nt][hi * 2 + 1] + bsm[co + 1];
                if constexpr (L < kLayers - 1) {
                    reinterpret_cast<__nv_bfloat162 *>(out)[(p * COUT + co) / 2] =
                        __floats2bfloat162_rn(fmaxf(v0, 0.f), fmaxf(v1, 0.f));
                } else {
                    if (co == 0) reinterpret_cast<float *>(out)[p] = v0;
                }
            }
        }
}

// --------------------------------------------------------------- backward
// dL/dout = 2 lam (out - t) / count; per-CTA partial loss sums (256 threads).
static __global__ void out_grad_kernel(const float *__restrict__ y, const float *__restrict__ t,
                                const float *__restrict__ lam, float *__restrict__ gy, double *__restrict__ lpart,
                                long long P, float scale) {
    __shared__ double red[256];
    const long long p = (long long)blockIdx.x * 256 + threadIdx.x;
    double l = 0.0;
    if (p < P) {
        const float e = y[p] - t[p];
        const float lw = lam ? lam[p] : 1.f;
        gy[p] = scale * lw * e;
        l = (double)lw * e * e;
    }
    red[threadIdx.x] = l;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) lpart[blockIdx.x] = red[0];
}

// Data gradient of layer L: dx[p][ci] = sum_tap sum_co Wt[tap][co][ci] *
// dy[p - off(tap)][co], then gated by the ReLU of the layer's input
// (act_in[p][ci] > 0).  One thread per input pixel.
template <int L>
__global__ void __launch_bounds__(128) conv_bwd_data_kernel(const float *__restrict__ dy,
                                                            const float *__restrict__ wt_all,
                                                            const __nv_bfloat16 *__restrict__ act_in,
                                                            float *__restrict__ dx, int N, int H, int W) {
    constexpr int CIN = cin_of(L), COUT = cout_of(L), D = dil_of(L);
    __shared__ float wsm[9 * COUT * CIN];
    for (int i = threadIdx.x; i < 9 * COUT * CIN; i += 128) wsm[i] = wt_all[wt_off(L) + i];
    __syncthreads();
    const long long P = (long long)N * H * W;
    const long long p = (long long)blockIdx.x * 128 + threadIdx.x;
    if (p >= P) return;
    const long long img = p / (H * W) * (long long)(H * W);
    const int rem = (int)(p % (H * W)), y = rem / W, x = rem % W;
    float acc[CIN];
#pragma unroll
    for (int ci = 0; ci < CIN; ++ci) acc[ci] = 0.f;
    for (int tap = 0; tap < 9; ++tap) {
        const int yy = y - (tap / 3 - 1) * D, xx = x - (tap % 3 - 1) * D;
        if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
        const float *g = dy + (img + (long long)yy * W + xx) * COUT;
        for (int co = 0; co < COUT; ++co) {
            const float gv = g[co];
            const float *w = wsm + (tap * COUT + co) * CIN;
#pragma unroll
            for (int ci = 0; ci < CIN; ++ci) acc[ci] = fmaf(w[ci], gv, acc[ci]);
        }
    }
    const __nv_bfloat16 *a = act_in + p * CIN;
#pragma unroll
    for (int ci = 0; ci < CIN; ++ci) dx[p * CIN + ci] = __bfloat162float(a[ci]) > 0.f ? acc[ci] : 0.f;
}

// Weight and bias gradients of layer L, partial sums per CTA (fixed order):
// part[cta][e] for e < COUT*9*CIN: sum_p dy[p][co] x[p + off(tap)][ci] with
// e = (co * 9 + tap) * CIN + ci; then COUT bias sums.  256 threads; each CTA
// covers `span` consecutive pixels.
template <int L>
__global__ void __launch_bounds__(256) conv_bwd_weight_kernel(const float *__restrict__ dy,
                                                              const __nv_bfloat16 *__restrict__ x,
                                                              float *__restrict__ part, int N, int H, int W,
                                                              long long span) {
    constexpr int CIN = cin_of(L), COUT = cout_of(L), D = dil_of(L);
    constexpr int NE = COUT * 9 * CIN + COUT;
    constexpr int PER = (NE + 255) / 256;
    const long long P = (long long)N * H * W;
    const long long p0 = (long long)blockIdx.x * span, p1 = min(P, p0 + span);
    float acc[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) acc[j] = 0.f;
    for (long long p = p0; p < p1; ++p) {
        const long long img = p / (H * W) * (long long)(H * W);
        const int rem = (int)(p % (H * W)), y = rem / W, xq = rem % W;
        const float *g = dy + p * COUT;
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const int e = threadIdx.x + 256 * j;
            if (e >= NE) continue;
            if (e >= COUT * 9 * CIN) {          // bias
                acc[j] += g[e - COUT * 9 * CIN];
                continue;
            }
            const int ci = e % CIN, tap = (e / CIN) % 9, co = e / (9 * CIN);
            const int yy = y + (tap / 3 - 1) * D, xx = xq + (tap % 3 - 1) * D;
            if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
            acc[j] = fmaf(g[co], __bfloat162float(x[(img + (long long)yy * W + xx) * CIN + ci]), acc[j]);
        }
    }
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int e = threadIdx.x + 256 * j;
        if (e < NE) part[(long long)blockIdx.x * NE + e] = acc[j];
    }
}

// Sum the partials of layer L in a fixed order (FP64) and scatter them into
// the flat parameter-gradient vector.
template <int L>
__global__ void reduce_grad_kernel(const float *__restrict__ part, int nparts, float *__restrict__ grad) {
    constexpr int CIN = cin_of(L), COUT = cout_of(L);
    constexpr int NE = COUT * 9 * CIN + COUT;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NE) return;
    double s = 0.0;
    for (int k = 0; k < nparts; ++k) s += part[(long long)k * NE + e];
    int dst;
    if (e < COUT * 9 * CIN) {
        const int ci = e % CIN, tap = (e / CIN) % 9, co = e / (9 * CIN);
        dst = woff_of(L) + (co * CIN + ci) * 9 + tap;
    } else {
        dst = woff_of(L) + COUT * CIN * 9 + (e - COUT * 9 * CIN);
    }
    grad[dst] = (float)s;
}

static __global__ void sum_loss_kernel(const double *__restrict__ lpart, int n, double *__restrict__ out, double inv) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += lpart[i];
    *out = s * inv;
}

// Adam with bias correction on the FP32 master parameters.
static __global__ void adam_kernel(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                            const float *__restrict__ g, int n, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace fse_net
