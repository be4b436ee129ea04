// fse_device.cuh -- sm_103a device code of the cFSE hot path.
//
// One persistent kernel conceals every lost block of a batch.  A CTA has 128
// threads and pulls work items from an atomic counter; an item is one F=64
// block, four F=32 blocks or sixteen F=16 blocks, so every thread always owns
// 32 frequency bins of one block.  Per block (Algorithm 1):
//   gather + Eq. (3) weights  -> z = w s + j alpha w on the F x F grid (smem)
//   one complex FFT2 of z      -> R_w = FFT{w s}, W = FFT{w} (real-input split)
//   I iterations               -> argmax |R_w|^2, c = gamma R_w[u,v] / W[0,0],
//                                 R_w[k,l] -= c W[k-u, l-v] (circular)
//   Re{g} on B                 -> g = sum c phi_(u,v), accumulated per selection
//
// Layout of one block's spectrum (F x F bins, k = row, l = column):
//   thread t of the block (t < F*F/32) owns column c = t % (F/2) and its
//   partner column c + F/2, on the 16 rows k_i = t / (F/2) + i * (F/16).  The
//   32 residual values live in registers as packed f32x2 pairs
//   (R[k_i][c], R[k_i][c+F/2]).
//   W lives in shared memory in a "dual chunk" layout: chunk (r, q), q < F,
//   is 16 bytes {Re W[r][q], Re W[r][q+F/2], Im W[r][q], Im W[r][q+F/2]}
//   (column indices mod F).  The shifted operand W[k_i-u][c-v],
//   W[k_i-u][c+F/2-v] of one register pair is therefore ONE 16-byte load of
//   chunk ((k_i-u) mod F, (c-v) mod F); lanes with consecutive c read
//   consecutive chunks, so a warp's LDS.128 is free of bank conflicts.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace fse {

constexpr int kThreads = 128;   // threads per CTA, every class
constexpr int kMaxPix = 8;      // B samples per thread (b*b <= 8 * F*F/32)
constexpr int kMaxClasses = 4;

struct DevClass {
    int F, b, d, M, off, iters, bpi;  // bpi: blocks per work item (4096 / F^2)
    float gamma;
    const float *wtab;                // M*M Eq. (3) weights
};

struct BlockRec {                     // one lost block, in queue order
    int image, x, y, orig;            // orig: index in the caller's order
    long long patch_off;              // offset of its b*b patch
    long long pad;
};

struct DevParams {
    const void *images;
    int dtype;                        // 0 = u8, 1 = f32
    int H, W;
    long long pitch;                  // bytes per image row
    const uint8_t *mask;
    float *out;                       // FP32 image or nullptr
    float *patches;                   // compact patches or nullptr
    const BlockRec *blocks;
    int n_seg;                        // queue segments (one per class present)
    int seg_cls[kMaxClasses];
    int seg_item_end[kMaxClasses];    // cumulative item count
    int seg_block_start[kMaxClasses];
    int seg_block_count[kMaxClasses];
    int total_items;
    DevClass cls[kMaxClasses];
    int *counter;                     // work-queue head (zeroed before launch)
    int *tr_sel;                      // trace (nullptr = off)
    float *tr_energy;
    float2 *tr_coef;
    int tr_stride;
    const float2 *tw;                 // 64 entries (cos, sin)(2 pi t / 64)
};

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ uint64_t pk(float lo, float hi) {
    return ((uint64_t)__float_as_uint(hi) << 32) | (uint64_t)__float_as_uint(lo);
}
__device__ __forceinline__ float lo_of(uint64_t v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float hi_of(uint64_t v) { return __uint_as_float((uint32_t)(v >> 32)); }
// d = a * b + c on two FP32 lanes, round to nearest even
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
// |R|^2 of a register pair: exactly the same instruction sequence wherever it
// is evaluated, so a recomputed energy is bit-identical to the loop's.
__device__ __forceinline__ uint64_t energy2(uint64_t re, uint64_t im) {
    return fma2(im, im, mul2(re, re));
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// a * e^{-j theta} with tw = (cos theta, sin theta)
__device__ __forceinline__ float2 cmul_conj_tw(float2 a, float2 tw) {
    return make_float2(a.x * tw.x + a.y * tw.y, a.y * tw.x - a.x * tw.y);
}

// forward DFT of length 4 (e^{-j}) in registers
__device__ __forceinline__ void dft4(float2 &x0, float2 &x1, float2 &x2, float2 &x3) {
    const float2 a0 = cadd(x0, x2), a1 = csub(x0, x2), a2 = cadd(x1, x3), a3 = csub(x1, x3);
    x0 = cadd(a0, a2);
    x2 = csub(a0, a2);
    x1 = make_float2(a1.x + a3.y, a1.y - a3.x);   // a1 - j a3
    x3 = make_float2(a1.x - a3.y, a1.y + a3.x);   // a1 + j a3
}
// forward DFT of length 8 (e^{-j}) in registers, natural order in and out
__device__ __forceinline__ void dft8(float2 *x) {
    float2 e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
    float2 o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
    dft4(e0, e1, e2, e3);
    dft4(o0, o1, o2, o3);
    const float c = 0.70710678118654752440f;
    const float2 t1 = make_float2(c * (o1.x + o1.y), c * (o1.y - o1.x));   // o1 e^{-j pi/4}
    const float2 t2 = make_float2(o2.y, -o2.x);                            // o2 e^{-j pi/2}
    const float2 t3 = make_float2(c * (o3.y - o3.x), -c * (o3.x + o3.y));  // o3 e^{-j 3pi/4}
    x[0] = cadd(e0, o0); x[4] = csub(e0, o0);
    x[1] = cadd(e1, t1); x[5] = csub(e1, t1);
    x[2] = cadd(e2, t2); x[6] = csub(e2, t2);
    x[3] = cadd(e3, t3); x[7] = csub(e3, t3);
}
template <int R>
__device__ __forceinline__ void dftR(float2 *x) {
    if constexpr (R == 8) dft8(x);
    else dft4(x[0], x[1], x[2], x[3]);
}

// --------------------------------------------------------- group utilities
// A "group" is the set of threads working on one block: the whole CTA for
// F = 64 (4 warps), one warp for F = 32, eight lanes for F = 16.
template <int F>
struct Geo {
    static constexpr int TB = F * F / 32;            // threads per block
    static constexpr int LPR = F / 2;                // lanes per spectrum row
    static constexpr int RSTEP = F / 16;             // row step between a thread's rows
    static constexpr int REGION = 16 * F * F;        // smem bytes per block
    static constexpr int FP = F + 1;                 // padded row of the FFT buffer
    static constexpr int R1 = (F == 16) ? 4 : 8;     // four-step FFT radices
    static constexpr int R2 = F / R1;
    static constexpr int BPI = kThreads / TB;        // blocks per item
};

template <int F>
__device__ __forceinline__ void gsync(unsigned amask) {
    if constexpr (F == 64) __syncthreads();
    else __syncwarp(amask);
}

template <int F>
__device__ __forceinline__ float group_sum(float v, unsigned amask, float *s_buf) {
    constexpr int TB = Geo<F>::TB;
    constexpr int W = TB < 32 ? TB : 32;
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(amask, v, o);
    if constexpr (TB > 32) {
        const int warp = threadIdx.x >> 5;
        if ((threadIdx.x & 31) == 0) s_buf[warp] = v;
        __syncthreads();
        float t = 0.f;
#pragma unroll
        for (int i = 0; i < TB / 32; ++i) t += s_buf[i];
        __syncthreads();
        return t;
    }
    return v;
}

// ------------------------------------------------------------- FFT2 (smem)
// One 1-D pass of length F = R1 * R2 over all F lines of the padded F x F
// buffer Z (four-step algorithm: n = R2 n1 + n2, k = k1 + R1 k2).
//   step 1: for each (line, n2): DFT_R1 over n1, twiddle e^{-j 2pi n2 k1 / F},
//           stored back in place at R2 k1 + n2;
//   step 2: for each (line, k1): DFT_R2 over n2 of the values at R2 k1 + n2,
//           stored at k1 + R1 k2 (all loads before all stores).
// ROWS selects rows (element stride 1) or columns (element stride FP).
template <int F, bool ROWS>
__device__ __forceinline__ void fft_pass(float2 *Z, const float2 *s_tw, int lt, unsigned amask) {
    using G = Geo<F>;
    constexpr int TB = G::TB, R1 = G::R1, R2 = G::R2, FP = G::FP;
    constexpr int LS = ROWS ? FP : 1;     // line stride
    constexpr int ES = ROWS ? 1 : FP;     // element stride
    // step 1
#pragma unroll
    for (int t = lt; t < F * R2; t += TB) {
        const int line = t % F, n2 = t / F;
        float2 x[R1];
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) x[n1] = Z[line * LS + (R2 * n1 + n2) * ES];
        dftR<R1>(x);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) {
            const float2 tw = s_tw[((n2 * k1) * (64 / F)) & 63];
            Z[line * LS + (R2 * k1 + n2) * ES] = cmul_conj_tw(x[k1], tw);
        }
    }
    gsync<F>(amask);
    // step 2
    constexpr int NT = F * R1 / TB;       // tasks per thread
    float2 y[NT][R2];
#pragma unroll
    for (int j = 0; j < NT; ++j) {
        const int t = lt + j * TB;
        const int line = t % F, k1 = t / F;
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) y[j][n2] = Z[line * LS + (R2 * k1 + n2) * ES];
        dftR<R2>(y[j]);
    }
    gsync<F>(amask);
#pragma unroll
    for (int j = 0; j < NT; ++j) {
        const int t = lt + j * TB;
        const int line = t % F, k1 = t / F;
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) Z[line * LS + (k1 + R1 * k2) * ES] = y[j][k2];
    }
    gsync<F>(amask);
}

// ------------------------------------------------------- argmax reduction
// Result of one selection: bin index, R_w at that bin, max energy bits.
struct Pick {
    uint32_t idx;
    float rr, ri;
    uint32_t ebits;
};

// Find, in one thread, the first (smallest linear index) of its bins whose
// energy bits equal M, searching only quartet J (pairs 4J .. 4J+3).
template <int J>
__device__ __forceinline__ bool search_quartet(const uint64_t *Rre, const uint64_t *Rim, uint32_t M,
                                               int &hit, float &rr, float &ri) {
#pragma unroll
    for (int i = 4 * J; i < 4 * J + 4; ++i) {
        const uint64_t e = energy2(Rre[i], Rim[i]);
        if (__float_as_uint(lo_of(e)) == M) { hit = 2 * i; rr = lo_of(Rre[i]); ri = lo_of(Rim[i]); return true; }
        if (__float_as_uint(hi_of(e)) == M) { hit = 2 * i + 1; rr = hi_of(Rre[i]); ri = hi_of(Rim[i]); return true; }
    }
    return false;
}

// Search all bins of this thread for energy M (the thread's max equals M).
// Returns the local slot (2 i + h) or -1, with the residual at that bin.
__device__ __forceinline__ int thread_search(const uint64_t *Rre, const uint64_t *Rim, const float *q,
                                             uint32_t M, float &rr, float &ri) {
    int hit = -1;
    bool done = false;
    if (__float_as_uint(q[0]) == M) done = search_quartet<0>(Rre, Rim, M, hit, rr, ri);
    if (!done && __float_as_uint(q[1]) == M) done = search_quartet<1>(Rre, Rim, M, hit, rr, ri);
    if (!done && __float_as_uint(q[2]) == M) done = search_quartet<2>(Rre, Rim, M, hit, rr, ri);
    if (!done && __float_as_uint(q[3]) == M) done = search_quartet<3>(Rre, Rim, M, hit, rr, ri);
    return hit;
}

struct RedShared {
    uint32_t red[4];
    uint4 win[4];
    float sum[4];
};

// Group-wide argmax of |R_w|^2 with ties to the smallest linear index.
// tmax: this thread's max energy; q: its quartet maxima.
template <int F>
__device__ __forceinline__ Pick group_argmax(const uint64_t *Rre, const uint64_t *Rim, float tmax,
                                             const float *q, int lt, unsigned amask, RedShared *rs) {
    using G = Geo<F>;
    const uint32_t mt = __float_as_uint(tmax);
    const int c0 = lt % G::LPR, r0 = lt / G::LPR;
    auto lin = [&](int slot) -> uint32_t {      // slot -> linear bin index
        const int i = slot >> 1, h = slot & 1;
        return (uint32_t)((r0 + i * G::RSTEP) * F + c0 + h * (F / 2));
    };
    Pick p;
    if constexpr (F == 64) {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const uint32_t mw = __reduce_max_sync(0xffffffffu, mt);
        if (lane == 0) rs->red[warp] = mw;
        __syncthreads();
        const uint4 r4 = *reinterpret_cast<const uint4 *>(rs->red);
        const uint32_t M = max(max(r4.x, r4.y), max(r4.z, r4.w));
        if (mw == M) {
            uint32_t cand = 0xffffffffu;
            float rr = 0.f, ri = 0.f;
            if (mt == M) {
                const int hit = thread_search(Rre, Rim, q, M, rr, ri);
                if (hit >= 0) cand = lin(hit);
            }
            const uint32_t iw = __reduce_min_sync(0xffffffffu, cand);
            if (cand == iw && cand != 0xffffffffu)
                rs->win[warp] = make_uint4(iw, __float_as_uint(rr), __float_as_uint(ri), 0u);
        }
        __syncthreads();
        p.idx = 0xffffffffu; p.rr = 0.f; p.ri = 0.f; p.ebits = M;
        const uint32_t rw[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            if (rw[w] == M) {
                const uint4 e = rs->win[w];
                if (e.x < p.idx) { p.idx = e.x; p.rr = __uint_as_float(e.y); p.ri = __uint_as_float(e.z); }
            }
        }
    } else {
        constexpr int W = G::TB;                  // 32 (F=32) or 8 (F=16) lanes
        uint32_t M = mt;
#pragma unroll
        for (int o = W / 2; o > 0; o >>= 1) M = max(M, __shfl_xor_sync(amask, M, o));
        uint32_t cand = 0xffffffffu;
        float rr = 0.f, ri = 0.f;
        if (mt == M) {
            const int hit = thread_search(Rre, Rim, q, M, rr, ri);
            if (hit >= 0) cand = lin(hit);
        }
        uint32_t iw = cand;
#pragma unroll
        for (int o = W / 2; o > 0; o >>= 1) iw = min(iw, __shfl_xor_sync(amask, iw, o));
        const int lane = threadIdx.x & 31;
        const unsigned gm = (W == 32) ? 0xffffffffu : (0xffu << (lane & ~7));
        const unsigned who = __ballot_sync(amask, cand == iw) & gm;
        const int src = who ? __ffs(who) - 1 : (lane & ~(W - 1));
        p.idx = (iw == 0xffffffffu) ? 0xffffffffu : iw;
        p.rr = __shfl_sync(amask, rr, src);
        p.ri = __shfl_sync(amask, ri, src);
        p.ebits = M;
    }
    if (p.idx == 0xffffffffu) { p.idx = 0; p.rr = 0.f; p.ri = 0.f; }
    return p;
}

// ------------------------------------------------------- per-block worker
template <int F>
__device__ __forceinline__ void process(const DevParams &P, const DevClass &C, int first, int count,
                                        unsigned char *smem, const float2 *s_tw, RedShared *rsh) {
    using G = Geo<F>;
    constexpr int TB = G::TB, LPR = G::LPR, RSTEP = G::RSTEP, FP = G::FP;
    const int gidx = threadIdx.x / TB;
    const int lt = threadIdx.x % TB;
    const bool active = gidx < count;
    const unsigned amask = __ballot_sync(0xffffffffu, active);
    if (!active) return;

    const BlockRec blk = P.blocks[first + gidx];
    unsigned char *region = smem + gidx * G::REGION;
    float2 *Z = reinterpret_cast<float2 *>(region);

    const int b = C.b, d = C.d, M = C.M, off = C.off;
    // ---- S0/S1: gather the area, Eq. (3) weights, z = (w s, w) ----
    float sws2 = 0.f, sw = 0.f;
    for (int pix = lt; pix < F * F; pix += TB) {
        const int m = pix / F, n = pix % F;
        const int am = m - off, an = n - off;
        float ws = 0.f, w = 0.f;
        if (am >= 0 && am < M && an >= 0 && an < M) {
            const int yy = blk.y - d + am, xx = blk.x - d + an;
            const bool inB = am >= d && am < d + b && an >= d && an < d + b;
            if (!inB && yy >= 0 && yy < P.H && xx >= 0 && xx < P.W) {
                const size_t mi = ((size_t)blk.image * P.H + yy) * P.W + xx;
                if (P.mask[mi] == 0) {
                    const char *row = static_cast<const char *>(P.images) +
                                      ((long long)blk.image * P.H + yy) * P.pitch;
                    const float s = P.dtype == 0 ? (float)reinterpret_cast<const uint8_t *>(row)[xx]
                                                 : reinterpret_cast<const float *>(row)[xx];
                    w = __ldg(&C.wtab[am * M + an]);
                    ws = w * s;
                    sws2 = fmaf(ws, s, sws2);
                    sw += w;
                }
            }
        }
        Z[m * FP + n] = make_float2(ws, w);
    }
    // alpha = power of two near the weighted RMS of s: balances the two real
    // signals packed into one complex FFT (exact scaling)
    const float tsw = group_sum<F>(sw, amask, rsh->sum);
    const float tsws2 = group_sum<F>(sws2, amask, rsh->sum);
    float alpha = 1.f;
    if (tsw > 0.f && tsws2 > 0.f) {
        int e;
        frexpf(sqrtf(tsws2 / tsw), &e);
        alpha = ldexpf(1.f, e);
    }
    for (int pix = lt; pix < F * F; pix += TB) {
        const int m = pix / F, n = pix % F;
        Z[m * FP + n].y *= alpha;
    }
    gsync<F>(amask);
    // ---- S2/S3: FFT2 of z ----
    fft_pass<F, true>(Z, s_tw, lt, amask);
    fft_pass<F, false>(Z, s_tw, lt, amask);

    // ---- split into R_w = FFT{w s} and W = FFT{w} ----
    // W chunk rows k >= F/2 + 1 lie beyond the padded FFT buffer, so they are
    // written at once; the others are held until every thread has read Z.
    const int c0 = lt % LPR, r0 = lt / LPR;
    const float ainv = 1.f / alpha;
    float4 *Wd = reinterpret_cast<float4 *>(region);
    constexpr int SAFE = F / 2 + 1;
    uint64_t Rre[16], Rim[16];
    float4 Wc[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int k = r0 + i * RSTEP, km = (F - k) & (F - 1);
        float2 R2[2], W2[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int l = c0 + h * (F / 2), lm = (F - l) & (F - 1);
            const float2 z = Z[k * FP + l], zm = Z[km * FP + lm];
            R2[h] = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
            W2[h] = make_float2(0.5f * ainv * (z.y + zm.y), 0.5f * ainv * (zm.x - z.x));
        }
        Rre[i] = pk(R2[0].x, R2[1].x);
        Rim[i] = pk(R2[0].y, R2[1].y);
        Wc[i] = make_float4(W2[0].x, W2[1].x, W2[0].y, W2[1].y);
        if ((i + 1) * RSTEP > SAFE && k >= SAFE) {   // (first test is compile-time)
            Wd[k * F + c0] = Wc[i];
            Wd[k * F + c0 + F / 2] = make_float4(Wc[i].y, Wc[i].x, Wc[i].w, Wc[i].z);
        }
    }
    const float W00 = Z[0].y * ainv;
    gsync<F>(amask);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int k = r0 + i * RSTEP;
        if (i * RSTEP < SAFE && k < SAFE) {
            Wd[k * F + c0] = Wc[i];
            Wd[k * F + c0 + F / 2] = make_float4(Wc[i].y, Wc[i].x, Wc[i].w, Wc[i].z);
        }
    }
    gsync<F>(amask);

    // ---- B samples owned by this thread ----
    const int npix = (b * b + TB - 1) / TB;
    int pm_[kMaxPix], pn_[kMaxPix];
    float acc[kMaxPix];
#pragma unroll
    for (int t = 0; t < kMaxPix; ++t) {
        const int j = lt + t * TB;
        pm_[t] = off + d + j / b;
        pn_[t] = off + d + j % b;
        acc[t] = 0.f;
    }
    const float W0bar = W00 > 0.f ? 1.f / W00 : 0.f;
    const float cg = C.gamma * W0bar;

    // ---- S5: first selection (energies of R_w^(0)) ----
    float q[4];
    float tmax;
    {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint64_t e0 = energy2(Rre[4 * j], Rim[4 * j]), e1 = energy2(Rre[4 * j + 1], Rim[4 * j + 1]);
            const uint64_t e2 = energy2(Rre[4 * j + 2], Rim[4 * j + 2]), e3 = energy2(Rre[4 * j + 3], Rim[4 * j + 3]);
            const float a = max3f(lo_of(e0), hi_of(e0), lo_of(e1));
            const float bq = max3f(hi_of(e1), lo_of(e2), hi_of(e2));
            q[j] = max3f(a, bq, fmaxf(lo_of(e3), hi_of(e3)));
        }
        tmax = fmaxf(max3f(q[0], q[1], q[2]), q[3]);
    }
    const int iters = C.iters;
    Pick pick;
    if (iters > 0) pick = group_argmax<F>(Rre, Rim, tmax, q, lt, amask, rsh);

    for (int nu = 1; nu <= iters; ++nu) {
        // ---- S6/S7: coefficient and model ----
        const float cr = pick.rr * cg, ci = pick.ri * cg;
        const int u = (int)(pick.idx / F), v = (int)(pick.idx % F);
        if (P.tr_sel != nullptr && lt == 0) {
            const size_t o = (size_t)blk.orig * P.tr_stride + (nu - 1);
            P.tr_sel[o] = (int)pick.idx;
            P.tr_energy[o] = __uint_as_float(pick.ebits);
            P.tr_coef[o] = make_float2(cr, ci);
        }
#pragma unroll
        for (int t = 0; t < kMaxPix; ++t) {
            if (t < npix) {
                const int ph = (u * pm_[t] + v * pn_[t]) & (F - 1);
                const float2 tw = s_tw[ph * (64 / F)];
                acc[t] = fmaf(cr, tw.x, fmaf(-ci, tw.y, acc[t]));
            }
        }
        if (nu == iters) break;
        // ---- S8: R_w[k,l] -= c W[k-u, l-v] fused with |R_w|^2 and max ----
        const uint64_t ncr = pk(-cr, -cr), pci = pk(ci, ci), nci = pk(-ci, -ci);
        const int qcol = (c0 - v) & (F - 1);
        const int rbase = r0 - u;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float ev[8];
#pragma unroll
            for (int ii = 0; ii < 4; ++ii) {
                const int i = 4 * j + ii;
                const int r = (rbase + i * RSTEP) & (F - 1);
                const float4 w = Wd[r * F + qcol];
                const uint64_t wre = pk(w.x, w.y), wim = pk(w.z, w.w);
                uint64_t a = fma2(ncr, wre, Rre[i]);
                Rre[i] = fma2(pci, wim, a);
                uint64_t bb = fma2(ncr, wim, Rim[i]);
                Rim[i] = fma2(nci, wre, bb);
                const uint64_t e = energy2(Rre[i], Rim[i]);
                ev[2 * ii] = lo_of(e);
                ev[2 * ii + 1] = hi_of(e);
            }
            const float a = max3f(ev[0], ev[1], ev[2]);
            const float bq = max3f(ev[3], ev[4], ev[5]);
            q[j] = max3f(a, bq, fmaxf(ev[6], ev[7]));
        }
        tmax = fmaxf(max3f(q[0], q[1], q[2]), q[3]);
        // ---- S5: next selection ----
        pick = group_argmax<F>(Rre, Rim, tmax, q, lt, amask, rsh);
    }

    // ---- S10: write Re{g} on B ----
#pragma unroll
    for (int t = 0; t < kMaxPix; ++t) {
        const int j = lt + t * TB;
        if (t < npix && j < b * b) {
            const int pm = j / b, pn = j % b;
            if (P.out != nullptr)
                P.out[((size_t)blk.image * P.H + blk.y + pm) * P.W + blk.x + pn] = acc[t];
            if (P.patches != nullptr) P.patches[blk.patch_off + j] = acc[t];
        }
    }
}

// ------------------------------------------------------ persistent kernel
__global__ void __launch_bounds__(kThreads, 3) fse_batch_kernel(const __grid_constant__ DevParams P) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ float2 s_tw[64];
    __shared__ int s_item;
    __shared__ RedShared rsh;
    for (int i = threadIdx.x; i < 64; i += kThreads) s_tw[i] = P.tw[i];
    __syncthreads();
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(P.counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= P.total_items) break;
        int sg = 0;
        while (sg + 1 < P.n_seg && item >= P.seg_item_end[sg]) ++sg;
        const int item0 = sg ? P.seg_item_end[sg - 1] : 0;
        const DevClass &C = P.cls[P.seg_cls[sg]];
        const int first = P.seg_block_start[sg] + (item - item0) * C.bpi;
        const int count = min(C.bpi, P.seg_block_start[sg] + P.seg_block_count[sg] - first);
        switch (C.F) {
            case 64: process<64>(P, C, first, count, smem, s_tw, &rsh); break;
            case 32: process<32>(P, C, first, count, smem, s_tw, &rsh); break;
            default: process<16>(P, C, first, count, smem, s_tw, &rsh); break;
        }
        __syncthreads();
    }
}

// Eq. (3) weight table of one class, evaluated in FP64 and rounded once.
__global__ void weight_table_kernel(float *wtab, int M, double rho) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M * M) return;
    const int m = i / M, n = i % M;
    const double cm = 0.5 * (M - 1);
    const double dist = sqrt((m - cm) * (m - cm) + (n - cm) * (n - cm));
    wtab[i] = (float)pow(rho, dist);
}

// (cos, sin)(2 pi t / 64), FP64 then rounded once.
__global__ void twiddle_kernel(float2 *tw) {
    const int t = threadIdx.x;
    if (t >= 64) return;
    double s, c;
    sincospi((double)t / 32.0, &s, &c);
    tw[t] = make_float2((float)c, (float)s);
}

}  // namespace fse
