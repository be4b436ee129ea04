// fse_device.cuh -- sm_103a device code of the cFSE hot path.
//
// One persistent kernel conceals every lost block of a batch.  A CTA has 128
// or 256 threads and pulls work items from an atomic counter; an item is one
// F=64 block, four F=32 blocks or sixteen F=16 blocks, so every thread always
// owns 32 (or 16) frequency bins of one block.  Per block (Algorithm 1):
//   gather + Eq. (3) weights  -> z = w s + j alpha w on the F x F grid (smem)
//   one complex FFT2 of z      -> R_w = FFT{w s}, W = FFT{w} (real-input split)
//   I iterations               -> argmax |R_w|^2, c = gamma R_w[u,v] / W[0,0],
//                                 R_w[k,l] -= c W[k-u, l-v] (circular)
//   Re{g} on B                 -> g = sum c phi_(u,v), accumulated per selection
// Video volumes (class frames = 3) run the same steps on a 4 x F x F grid
// (the block's frame and its neighbours; a temporal pass completes the
// transform, shifts are circular in all three dimensions).  Ordered
// concealment lets a block wait for the earlier blocks in its area and reuse
// their concealed samples.
//
// Layout of one block's spectrum (F x F bins, k = row, l = column):
//   thread t of the block owns column c = t % (F/2) and its partner column
//   c + F/2, on PAIRS rows k_i = t / (F/2) + i * (F/PAIRS).  The residual
//   values live in registers as packed f32x2 pairs (R[k_i][c], R[k_i][c+F/2]).
//   W lives in shared memory in a "dual chunk" layout: chunk (r, q), q < F,
//   is 16 bytes {Re W[r][q], Re W[r][q+F/2], Im W[r][q], Im W[r][q+F/2]}
//   (column indices mod F).  The shifted operand W[k_i-u][c-v],
//   W[k_i-u][c+F/2-v] of one register pair is therefore ONE 16-byte load of
//   chunk ((k_i-u) mod F, (c-v) mod F); lanes with consecutive c read
//   consecutive chunks, so a warp's LDS.128 is free of bank conflicts.
#pragma once

#include <cuda.h>   // CUtensorMap (the type only; no driver-API calls here)
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

namespace fse {

constexpr int kMaxClasses = 4;

struct DevClass {
    int F, b, d, M, off, iters, bpi;  // bpi: blocks per work item (4096 / (FT F^2))
    float gamma;
    const float *wtab;                // T*M*M weights (Eq. (3), extended by the frame offset)
    int FT = 1;                       // temporal transform size (1: images; 4: video volumes)
    int T = 1;                        // frames of the volume (odd), centred on the block's frame
    int tc = 0;                       // the block's frame in the volume, (T - 1) / 2
    int toff = 0;                     // first grid plane of the volume, (FT - T) / 2
};

struct BlockRec {                     // one lost block, in queue order
    int image, x, y, orig;            // orig: index in the caller's order
    long long patch_off;              // offset of its b*b patch
    long long pad;
};

struct DevParams {
    const void *images;
    int dtype;                        // 0 = u8, 1 = f32
    int n_images;                     // frames of a video (support of volume classes)
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
    float *tr_second;                 // trace: largest |R_w|^2 besides the pick (nullptr = off)
    int tr_stride;
    const float2 *tw;                 // 64 entries (cos, sin)(2 pi t / 64)
    const float *est;                 // warm start: per-block estimate (sample units) or nullptr
    long long est_stride;             // floats between two blocks' estimates (block order: orig)
    // ordered concealment: blocks (caller order = queue order) reuse the
    // concealed samples of the earlier blocks listed for them
    int ordered;
    float beta;                       // weight factor of reused samples
    const int *nb_start, *nb_list;    // CSR: earlier blocks whose B meets the block's area
    int *done;                        // per block: concealed output visible (zeroed per launch)
    int *err;                         // device status word: kErr* bits (nullptr: not reported)
    unsigned long long wait_ns;       // limit of every bounded device wait
    int clamp_u8;                     // outputs clamped to [0, 255] and rounded half to even
    // reduced-precision residual storage (kSetFixW): the updates of
    // iterations fix_from, fix_from + 1, ... (0-based) read W as 16-bit
    // fixed-point codes of W / W[0,0] (scale 32767) instead of FP32
    int fix_from;
    // F = 64 windows of 8-bit images fetched as tiles by the tensor-memory
    // accelerator: 2-D maps over [n_images * H rows, W columns] of the images
    // and the mask, box tma_bw columns x tma_bh rows (tma = 0: plain loads)
    int tma;
    int tma_bw, tma_bh;
    CUtensorMap tm_img, tm_mask;
};

// bits of the device status word (read and cleared by fse_sync)
constexpr int kErrTimeout = 1;    // a bounded wait ran out
constexpr int kErrUnmarked = 2;   // a block's loss area B is not marked lost in the mask
constexpr int kErrBounds = 4;     // (bounds-checked builds) an index left its buffer; the access was skipped
// after an expired wait the kernel still waits this long, at most, for its
// own asynchronous copies in flight
constexpr unsigned long long kDrainNs = 1000000000ull;

__device__ __forceinline__ void report(const DevParams &P, int bit) {
    if (P.err != nullptr) atomicOr(P.err, bit);
}

#ifdef FSE_BOUNDS_CHECK
// Bounds-checked builds (-DFSE_BOUNDS_CHECK, libfse_checked.so): index i of a
// buffer of n elements.  Outside [0, n) it is recorded in the status word
// (kErrBounds, reported by fse_sync) and 0 is used instead, so the access
// stays inside the buffer and the kernel runs on.  Other builds compile the
// unchecked expressions.
__device__ __forceinline__ long long bchk(const DevParams &P, long long i, long long n) {
    if (i < 0 || i >= n) {
        report(P, kErrBounds);
        return 0;
    }
    return i;
}
#define FSE_IX(i, n) bchk(P, (i), (n))
#define FSE_LD(base, ptr, n) (base)[bchk(P, (ptr) - (base), (n))]
#else
#define FSE_IX(i, n) (i)
#define FSE_LD(base, ptr, n) (*(ptr))
#endif

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ int ld_acquire_gpu(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(int *p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

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
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// ---- 16-bit fixed-point spectrum (reduced-precision residual storage) ----
// A value x of W is held as the code q = rint(x * 32767 / W[0,0]) in
// [-32767, 32767] (|W| <= W[0,0] for a non-negative weight), stored biased as
// the 16-bit integer q + 32768.  Decoding needs no conversion instruction:
// the 16 bits placed under the exponent of 2^23 form the float 2^23 + q +
// 32768, and subtracting 2^23 + 32768 (exact: both lie in [2^23, 2^24))
// leaves q.  The update then multiplies q by c W[0,0] / 32767.
constexpr uint32_t kFixMagic = 0x4B000000u;        // bits of 2^23
constexpr float kFixBias = 8421376.f;              // 2^23 + 32768

__device__ __forceinline__ uint32_t fix_code16(float x, float qs) {
    const float q = fminf(fmaxf(rintf(x * qs), -32767.f), 32767.f);
    return (uint32_t)((int)q + 32768);
}

// codes of (a, b) as one word: a in the low half, b in the high half
__device__ __forceinline__ uint32_t fix_pack(float a, float b, float qs) {
    return fix_code16(a, qs) | (fix_code16(b, qs) << 16);
}

// the codes of one word as an f32x2 pair (low half, high half)
__device__ __forceinline__ uint64_t fix_unpack(uint32_t w, uint64_t nbias2) {
    const uint32_t lo = __byte_perm(w, kFixMagic, 0x7610), hi = __byte_perm(w, kFixMagic, 0x7632);
    return add2((uint64_t)lo | ((uint64_t)hi << 32), nbias2);
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
// A "group" is the set of threads working on one block.  A CTA of NT threads
// gives every thread PAIRS = 2048 / NT register pairs (2 * PAIRS bins), so a
// block of F x F bins needs TB = F*F / (2 * PAIRS) threads and a work item
// holds NT / TB = 4096 / F^2 blocks whatever NT is.
//   NT = 128 (16 pairs): F=64 -> 4 warps, F=32 -> 1 warp, F=16 -> 8 lanes
//   NT = 256 ( 8 pairs): F=64 -> 8 warps, F=32 -> 2 warps, F=16 -> 16 lanes
// The window tiles of an F = 64 block (TMA gather, below) are staged at this
// offset of its region: after the padded FFT buffer, which the gather writes
// while it reads them; the W chunks overwrite both later.
constexpr int kTmaStage = 40960;
constexpr int kTmaStageMax = 16384;   // two tiles of at most 128 x 64 bytes

template <int F, int PAIRS, int FT = 1>
struct Geo {
    static constexpr int TB = FT * F * F / (2 * PAIRS);   // threads per block
    static constexpr int LPR = F / 2;                // lanes per spectrum row
    static constexpr int RSTEP = TB / LPR;           // row groups of the block's threads
    // F = 64 (F = 32): a thread's rows are runs of RL = 8 (4) consecutive
    // rows, and W carries a copy of rows 0..RL-2 after row F-1, so a shifted
    // run never wraps (its RL loads address one base with immediate
    // offsets).  Volumes of F = 32
    // (VRUNS): in every temporal plane a thread's rows are a run of KPR
    // consecutive rows, and each plane of W carries a copy of its rows 0..2
    // after its row F-1 (PROWS rows per plane), so each plane's KPR loads
    // address one base with immediate offsets.  Other sizes: rows r0, r0 +
    // RSTEP, ... and one select (images) or one register offset (volumes)
    // per load.
    static constexpr bool RUNS = (F == 64 || F == 32) && FT == 1;
    static constexpr int RL = F == 64 ? 8 : 4;       // rows per run (images)
    static constexpr int RLS = F == 64 ? 3 : 2;      // log2(RL)
    static constexpr bool VRUNS = F == 32 && FT == 4;
    static constexpr int KPR = F / RSTEP > 0 ? F / RSTEP : 1;   // a thread's rows per plane (volumes)
    static constexpr int KPS = KPR >= 4 ? 2 : KPR == 2 ? 1 : 0;   // log2(KPR) for the volume runs
    static constexpr int WROWS = RUNS ? F + RL - 1 : F;   // W chunk rows in shared memory (images)
    static constexpr int PROWS = VRUNS ? F + 3 : F;  // W chunk rows per plane (volumes)
    static constexpr int REGION = RUNS ? 16 * F * WROWS : 16 * F * PROWS * FT;   // smem bytes per block
    __device__ __forceinline__ static int row(int r0, int i) {   // spectrum row of pair i
        // (shifts: i may be a run-time slot index, whose sign the compiler
        // cannot see)
        if constexpr (RUNS) return (((i >> RLS) * RSTEP + r0) << RLS) + (i & (RL - 1));
        else if constexpr (VRUNS) return (i >> KPS) * F + (r0 << KPS) + (i & (KPR - 1));
        else return r0 + i * RSTEP;
    }
    // W chunk row in shared memory of spectrum row k (plane k / F)
    __device__ __forceinline__ static int wrow(int k) {
        if constexpr (VRUNS) return (k / F) * PROWS + k % F;
        else return k;
    }
    static constexpr int FP = F + 1;                 // padded row of the FFT buffer
    static constexpr int R1 = (F == 16) ? 4 : 8;     // four-step FFT radices
    static constexpr int R2 = F / R1;
    static constexpr int WPG = TB >= 32 ? TB / 32 : 1;   // warps per group
    static constexpr int LANES = TB < 32 ? TB : 32;      // lanes per group and warp
    static constexpr int NQ = PAIRS / 4;                 // quartets of pairs
    static_assert(RSTEP * PAIRS == FT * F, "thread rows must tile the spectrum");
    static_assert(FT == 1 || F % RSTEP == 0, "a thread's rows repeat in every temporal plane");
    static_assert(!RUNS || PAIRS % RL == 0, "a thread's rows are whole runs");
    static_assert(!RUNS || RL == (1 << RLS), "runs of a power-of-two length");
    static_assert(!VRUNS || (KPR == (1 << KPS) && KPR * RSTEP == F && KPR * FT == PAIRS && KPR - 1 <= PROWS - F),
                  "volume runs tile every plane and the copied rows cover a shifted run");
    static_assert(REGION >= 8 * FT * F * FP, "the FFT buffer fits the region");
    static_assert(F != 64 || (kTmaStage >= 8 * F * FP && kTmaStage + kTmaStageMax <= REGION),
                  "the TMA staging area lies between the FFT buffer and the end of the region");
};

// dynamic shared memory of one CTA working on blocks of FFT size F (one
// F = 64 block, or 4096 / F^2 smaller blocks) or on volumes (FT = 4: one F =
// 32 volume with its copied rows, or four F = 16 volumes)
__host__ __device__ constexpr int cta_region_bytes(int F, int FT = 1) {
    // F = 32: four blocks (or one volume) of 35 W chunk rows per plane
    return F == 64 ? 16 * 64 * (64 + 7) : F == 32 ? 16 * 32 * (32 + 3) * 4 : 65536;
}

constexpr int kMaxWarps = 8;

// kernel sets of fse_batch_kernel (see there)
constexpr int kSetImage = 0, kSetExt = 1, kSetF64 = 2, kSetTrace = 3, kSetFixW = 4;
constexpr int kNumSets = 5;

struct RedShared {
    uint4 win[2][kMaxWarps];   // per-warp argmax candidates, double-buffered by iteration parity
    float sum[kMaxWarps];
    uint32_t sec[2][kMaxWarps];   // per-warp second-largest energies (traced launches)
    unsigned long long mbar;   // completion barrier of the window tiles (TMA gather)
};

// ------------------------------------------------ TMA gather of a window

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// 2-D tiled TMA load of the box at (x, y) (x: innermost, in elements) into
// shared memory, completing on bar
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
// Wait for phase `parity` of bar, bounded by limit_ns of %globaltimer; false
// if the wait ran out.  The first poll does not block (test_wait), so a
// limit of 0 expires as soon as the phase is found incomplete; later polls
// use try_wait, which may suspend the thread for a while.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity, unsigned long long limit_ns) {
    const uint32_t a = smem_u32(bar);
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    if (limit_ns == 0) return false;
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
        if (globaltimer_ns() - t0 > limit_ns) return false;
    }
}

struct Grp {
    int g;            // group index inside the CTA
    int lt;           // thread index inside the group
    unsigned amask;   // lanes of this warp that belong to active groups
};

__device__ __forceinline__ void named_barrier(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

template <int F, int PAIRS, int NT, int FT = 1>
__device__ __forceinline__ void gsync(const Grp &gr) {
    using G = Geo<F, PAIRS, FT>;
    if constexpr (G::TB == NT) __syncthreads();
    else if constexpr (G::TB > 32) named_barrier(1 + gr.g, G::TB);
    else __syncwarp(gr.amask);
}

// Maximum of a non-negative float over the group.  A maximum does not depend
// on the order in which it is taken, so the result is the same for every
// thread-to-bin mapping the autotuner may choose.
// The switch to reduced-precision residual storage: every 16-byte FP32 chunk
// e of the block's W (Geo::REGION) becomes the 8-byte chunk e of 16-bit codes
// {Re W, Re W'}, {Im W, Im W'} (same dual-chunk order), in place.  Rounds of
// RND chunks: a round reads its FP32 chunks into registers, waits for the
// group, then writes its code chunks.  The codes of round r land in bytes
// [8 lo, 8 hi) of FP32 chunks lo .. hi - 1, below 16 hi, so they overwrite only
// chunks that this or an earlier round has read, and the next round's reads
// (from byte 16 hi on) are untouched: one group barrier per round.
template <int F, int PAIRS, int NT>
__device__ __forceinline__ void compact_w(unsigned char *region, float qs, const Grp &gr) {
    using G = Geo<F, PAIRS>;
    constexpr int TB = G::TB, NCH = G::WROWS * F, CPT = 2, RND = TB * CPT;
    const float4 *src = reinterpret_cast<const float4 *>(region);
    uint2 *dst = reinterpret_cast<uint2 *>(region);
    for (int base = 0; base < NCH; base += RND) {
        uint2 cv[CPT];
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
            const int e = base + j * TB + gr.lt;
            if (e < NCH) {
                const float4 f = src[e];
                cv[j] = make_uint2(fix_pack(f.x, f.y, qs), fix_pack(f.z, f.w, qs));
            }
        }
        gsync<F, PAIRS, NT>(gr);
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
            const int e = base + j * TB + gr.lt;
            if (e < NCH) dst[e] = cv[j];
        }
    }
    gsync<F, PAIRS, NT>(gr);
}

template <int F, int PAIRS, int NT, int FT = 1>
__device__ __forceinline__ float group_max(float v, const Grp &gr, RedShared *rs) {
    using G = Geo<F, PAIRS, FT>;
#pragma unroll
    for (int o = G::LANES / 2; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(gr.amask, v, o));
    if constexpr (G::TB > 32) {
        const int warp = threadIdx.x >> 5;
        if ((threadIdx.x & 31) == 0) rs->sum[warp] = v;
        gsync<F, PAIRS, NT, FT>(gr);
        float t = 0.f;
#pragma unroll
        for (int i = 0; i < G::WPG; ++i) t = fmaxf(t, rs->sum[gr.g * G::WPG + i]);
        gsync<F, PAIRS, NT, FT>(gr);
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
template <int F, int PAIRS, int NT, bool ROWS, int FT = 1>
__device__ __forceinline__ void fft_pass(float2 *Z, const float2 *s_tw, const Grp &gr) {
    using G = Geo<F, PAIRS, FT>;
    constexpr int TB = G::TB, R1 = G::R1, R2 = G::R2, FP = G::FP;
    constexpr int LS = ROWS ? FP : 1;     // line stride within a plane
    constexpr int ES = ROWS ? 1 : FP;     // element stride
    constexpr int NL = FT * F;            // lines over all FT planes of F x FP
    constexpr int N1 = NL * R2 / TB;      // step-1 tasks per thread
    constexpr int N2 = NL * R1 / TB;      // step-2 tasks per thread
    static_assert(N1 * TB == NL * R2 && N2 * TB == NL * R1, "FFT tasks must tile the group");
    // line L of plane L / F: offset (L / F) F FP + (L % F) LS (images: L LS)
    auto lbase = [](int L) {
        if constexpr (FT == 1) return L * LS;
        else return (L / F) * F * FP + (L % F) * LS;
    };
#pragma unroll
    for (int j = 0; j < N1; ++j) {
        const int t = gr.lt + j * TB;
        const int line = lbase(t % NL), n2 = t / NL;
        float2 x[R1];
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) x[n1] = Z[line + (R2 * n1 + n2) * ES];
        dftR<R1>(x);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) {
            const float2 tw = s_tw[((n2 * k1) * (64 / F)) & 63];
            Z[line + (R2 * k1 + n2) * ES] = cmul_conj_tw(x[k1], tw);
        }
    }
    gsync<F, PAIRS, NT, FT>(gr);
    float2 y[N2][R2];
#pragma unroll
    for (int j = 0; j < N2; ++j) {
        const int t = gr.lt + j * TB;
        const int line = lbase(t % NL), k1 = t / NL;
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) y[j][n2] = Z[line + (R2 * k1 + n2) * ES];
        dftR<R2>(y[j]);
    }
    gsync<F, PAIRS, NT, FT>(gr);
#pragma unroll
    for (int j = 0; j < N2; ++j) {
        const int t = gr.lt + j * TB;
        const int line = lbase(t % NL), k1 = t / NL;
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) Z[line + (k1 + R1 * k2) * ES] = y[j][k2];
    }
    gsync<F, PAIRS, NT, FT>(gr);
}

// The temporal pass of a volume's transform (FT = 4): for every spatial bin,
// the length-4 DFT across the four planes (exact: the twiddles are +-1, +-j).
template <int F, int PAIRS, int NT, int FT>
__device__ __forceinline__ void time_pass(float2 *Z, const Grp &gr) {
    using G = Geo<F, PAIRS, FT>;
    constexpr int TB = G::TB, FP = G::FP, PS = F * FP;   // plane stride
    static_assert(FT == 4, "temporal transform of length 4");
    static_assert(F * F % TB == 0, "tasks tile the group");
#pragma unroll
    for (int j = 0; j < F * F / TB; ++j) {
        const int q = gr.lt + j * TB;
        float2 *z = Z + (q / F) * FP + (q % F);
        float2 x0 = z[0], x1 = z[PS], x2 = z[2 * PS], x3 = z[3 * PS];
        dft4(x0, x1, x2, x3);
        z[0] = x0; z[PS] = x1; z[2 * PS] = x2; z[3 * PS] = x3;
    }
    gsync<F, PAIRS, NT, FT>(gr);
}

// ------------------------------------------------------- argmax reduction
// Result of one selection: bin index, R_w at that bin, max energy bits.
struct Pick {
    uint32_t idx;
    float rr, ri;
    uint32_t ebits;
    uint32_t sbits;   // largest energy of the other bins (traced launches only)
};

// The largest energy of this thread's bins other than slot `skip` (the
// energies are recomputed with the loop's own instruction sequence).
template <int PAIRS>
__device__ __forceinline__ uint32_t thread_second(const uint64_t *Rre, const uint64_t *Rim, int skip) {
    float m = 0.f;
#pragma unroll
    for (int i = 0; i < PAIRS; ++i) {
        const uint64_t e = energy2(Rre[i], Rim[i]);
        m = max3f(m, 2 * i == skip ? 0.f : lo_of(e), 2 * i + 1 == skip ? 0.f : hi_of(e));
    }
    return __float_as_uint(m);
}

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

// Search the bins of this thread for energy M (the thread's max equals M).
// jb is the first quartet whose maximum equals the thread's maximum (carried
// out of the update), so the first hit inside it has the smallest linear
// index of the thread.  Returns the local slot (2 i + h) or -1, with the
// residual there.
template <int NQ>
__device__ __forceinline__ int thread_search(const uint64_t *Rre, const uint64_t *Rim, int jb, uint32_t M,
                                             float &rr, float &ri) {
    int hit = -1;
    if (jb == 0) search_quartet<0>(Rre, Rim, M, hit, rr, ri);
    else if (jb == 1) search_quartet<1>(Rre, Rim, M, hit, rr, ri);
    if constexpr (NQ > 2) {
        if (jb == 2) search_quartet<2>(Rre, Rim, M, hit, rr, ri);
        else if (jb == 3) search_quartet<3>(Rre, Rim, M, hit, rr, ri);
    }
    return hit;
}

// Running maximum over the quartets of a thread with the index of the first
// quartet that holds it (the strict comparison keeps the first).
__device__ __forceinline__ void quartet_max(int j, float qj, float &tmax, int &jb) {
    if (j == 0) {
        tmax = qj;
        jb = 0;
    } else {
        jb = qj > tmax ? j : jb;
        tmax = fmaxf(tmax, qj);
    }
}

// Group-wide argmax of |R_w|^2 with ties to the smallest linear index.
// tmax: this thread's max energy; jb: the first quartet holding it; parity:
// iteration parity (double-buffers the cross-warp exchange).
//
// Every warp-wide step (shuffle, redux, shared-memory exchange) waits in the
// SM's memory-instruction queue behind the residual update's 16-byte loads,
// so the reduction is built from as few DEPENDENT such steps as possible:
// one redux.sync for the max, the owner's register search, one redux.sync for
// the smallest index, and (multi-warp groups) one shared-memory exchange.
// GAP (compiled in: the traced kernel set) and gap (at run time): also the
// largest energy of the other bins, for the trace's top-two gap.
template <int F, int PAIRS, int NT, int FT = 1, bool GAP = false>
__device__ __forceinline__ Pick group_argmax(const uint64_t *Rre, const uint64_t *Rim, float tmax, int jb,
                                             const Grp &gr, RedShared *rs, int parity, bool gap = false) {
    using G = Geo<F, PAIRS, FT>;
    const uint32_t mt = __float_as_uint(tmax);
    const int c0 = gr.lt % G::LPR, r0 = gr.lt / G::LPR;
    auto lin = [&](int slot) -> uint32_t {      // slot -> linear bin index
        const int i = slot >> 1, h = slot & 1;
        return (uint32_t)(G::row(r0, i) * F + c0 + h * (F / 2));
    };
    const int lane = threadIdx.x & 31;
    Pick p;
    if constexpr (G::TB > 32) {
        // whole warps: each warp finds its own candidate (max energy, smallest
        // index, residual there), one exchange, every thread picks the best
        const int warp = threadIdx.x >> 5;
        const int w0 = gr.g * G::WPG;
        const uint32_t mw = __reduce_max_sync(0xffffffffu, mt);
        uint32_t cand = 0xffffffffu;
        float rr = 0.f, ri = 0.f;
        int hit = -1;
        if (mt == mw) {
            hit = thread_search<G::NQ>(Rre, Rim, jb, mw, rr, ri);
            if (hit >= 0) cand = lin(hit);
        }
        const uint32_t iw = __reduce_min_sync(0xffffffffu, cand);
        uint4 *win = rs->win[parity];
        const bool writer = (cand == iw && cand != 0xffffffffu) || (iw == 0xffffffffu && lane == 0);
        if (writer) win[warp] = make_uint4(mw, iw, __float_as_uint(rr), __float_as_uint(ri));
        if constexpr (GAP) {
            if (gap) {   // the warp's second: the candidate's owner without the candidate, the others' maxima
                const uint32_t sl = (cand == iw && cand != 0xffffffffu) ? thread_second<PAIRS>(Rre, Rim, hit) : mt;
                const uint32_t sw = __reduce_max_sync(0xffffffffu, sl);
                if (writer) rs->sec[parity][warp] = sw;
            }
        }
        gsync<F, PAIRS, NT, FT>(gr);
        // the warps' candidates combined as a tree (log2 WPG dependent steps;
        // the order (larger energy, then smaller index) is total, so any
        // combination order gives the same pick)
        uint4 e[G::WPG];
#pragma unroll
        for (int i = 0; i < G::WPG; ++i) e[i] = win[w0 + i];
        auto better = [](const uint4 &a, const uint4 &b) {
            return (b.x > a.x || (b.x == a.x && b.y < a.y)) ? b : a;
        };
#pragma unroll
        for (int s = 1; s < G::WPG; s <<= 1)
#pragma unroll
            for (int i = 0; i + s < G::WPG; i += 2 * s) e[i] = better(e[i], e[i + s]);
        p.ebits = e[0].x; p.idx = e[0].y; p.rr = __uint_as_float(e[0].z); p.ri = __uint_as_float(e[0].w);
        p.sbits = 0u;
        if constexpr (GAP) {
            if (gap) {   // the winning warp contributes its second, the others their maxima
#pragma unroll
                for (int i = 0; i < G::WPG; ++i) {
                    const uint4 c = win[w0 + i];
                    p.sbits = max(p.sbits, c.y == p.idx ? rs->sec[parity][w0 + i] : c.x);
                }
            }
        }
    } else {
        constexpr int W = G::LANES;               // lanes of one group (8, 16 or 32)
        constexpr int NG = 32 / W;                // groups per warp
        const int mygrp = lane / W;
        // one redux per group; they do not depend on each other
        uint32_t M = 0u;
#pragma unroll
        for (int k = 0; k < NG; ++k) {
            const uint32_t r = __reduce_max_sync(gr.amask, mygrp == k ? mt : 0u);
            if (mygrp == k) M = r;
        }
        uint32_t cand = 0xffffffffu;
        float rr = 0.f, ri = 0.f;
        int hit = -1;
        if (mt == M) {
            hit = thread_search<G::NQ>(Rre, Rim, jb, M, rr, ri);
            if (hit >= 0) cand = lin(hit);
        }
        uint32_t iw = 0xffffffffu;
#pragma unroll
        for (int k = 0; k < NG; ++k) {
            const uint32_t r = __reduce_min_sync(gr.amask, mygrp == k ? cand : 0xffffffffu);
            if (mygrp == k) iw = r;
        }
        const unsigned gm = (W == 32) ? 0xffffffffu : (((1u << W) - 1u) << (lane & ~(W - 1)));
        const unsigned who = __ballot_sync(gr.amask, cand == iw) & gm;
        const int src = who ? __ffs(who) - 1 : (lane & ~(W - 1));
        p.idx = iw;
        p.rr = __shfl_sync(gr.amask, rr, src);
        p.ri = __shfl_sync(gr.amask, ri, src);
        p.ebits = M;
        p.sbits = 0u;
        if constexpr (GAP) {
            if (gap) {   // the owner of the pick without it, the group's other lanes their maxima
                const uint32_t sl = (cand == iw && cand != 0xffffffffu) ? thread_second<PAIRS>(Rre, Rim, hit) : mt;
#pragma unroll
                for (int k = 0; k < NG; ++k) {
                    const uint32_t r = __reduce_max_sync(gr.amask, mygrp == k ? sl : 0u);
                    if (mygrp == k) p.sbits = r;
                }
            }
        }
    }
    if (p.idx == 0xffffffffu) { p.idx = 0; p.rr = 0.f; p.ri = 0.f; }
    return p;
}

// ------------------------------------------------------- per-block worker
// NP: B samples per thread (compile time; the caller picks the smallest
// variant that covers b*b).  EXT: built with ordered concealment.  GAP: the
// traced kernel set (selection trace with the top-two gap; other sets write
// no trace).  TMA: the FFT-64 sets (windows of 8-bit images by TMA).  FIXW:
// reduced-precision residual storage from iteration P.fix_from on (its set
// also writes the selection trace, without the gap).
template <int F, int PAIRS, int NT, int NP, bool EXT = false, bool GAP = false, bool TMA = false,
          bool FIXW = false>
__device__ __forceinline__ void process(const DevParams &P, const DevClass &C, int first, int count,
                                        unsigned char *smem, const float2 *s_tw, RedShared *rsh, uint32_t &tph) {
    using G = Geo<F, PAIRS>;
    static_assert(!FIXW || (G::RUNS && F == 64), "the fixed-point spectrum uses the F = 64 chunk rows");
    constexpr bool TRW = GAP || FIXW;   // trace writes compiled in
    constexpr int TB = G::TB, LPR = G::LPR, RSTEP = G::RSTEP, FP = G::FP, NQ = G::NQ;
    Grp gr;
    gr.g = threadIdx.x / TB;
    gr.lt = threadIdx.x % TB;
    const bool active = gr.g < count;
    gr.amask = __ballot_sync(0xffffffffu, active);
    if (!active) return;
    const int lt = gr.lt;

    const BlockRec blk = P.blocks[first + gr.g];
#ifdef FSE_BOUNDS_CHECK
    // the block lies inside its image (the host validates this too); the
    // whole group skips a block that does not
    if (blk.image < 0 || blk.image >= P.n_images || blk.x < 0 || blk.y < 0 || blk.x + C.b > P.W ||
        blk.y + C.b > P.H) {
        report(P, kErrBounds);
        return;
    }
#endif
    unsigned char *region = smem + gr.g * G::REGION;
    float2 *Z = reinterpret_cast<float2 *>(region);

    const int b = C.b, d = C.d, M = C.M, off = C.off;
    // ordered concealment (EXT builds only): the blocks this one reuses must
    // have written their output (bounded wait)
    int nb0 = 0, nb1 = 0;
    if constexpr (EXT) {
        if (P.ordered) {
            nb0 = P.nb_start[blk.orig];
            nb1 = P.nb_start[blk.orig + 1];
            if (lt == 0) {
                const uint64_t t0 = globaltimer_ns();
                for (int q = nb0; q < nb1; ++q)
                    while (ld_acquire_gpu(&P.done[P.nb_list[q]]) == 0) {
                        if (globaltimer_ns() - t0 > P.wait_ns) {
                            report(P, kErrTimeout);
                            break;
                        }
                        __nanosleep(128);
                    }
            }
            gsync<F, PAIRS, NT>(gr);
        }
    }
    // ---- S0/S1: gather the area, Eq. (3) weights, z = (w s, w) ----
    // All loads of the thread's grid positions are issued first (clamped to
    // the image, so always in bounds), then the weights are applied: one
    // memory round trip instead of one per position.
    constexpr int NPOS = F * F / TB;
    float sv[NPOS];
    uint8_t mk[NPOS];
    if (TMA && F == 64 && P.tma) {
        // 8-bit F = 64 windows: the image and mask tiles of the M x M area
        // arrive in shared memory by two TMA copies.  The tile's first column
        // is the area's first column rounded down to a 16-byte boundary (xs
        // columns before it); rows and columns outside the images read 0 and
        // are excluded below like in the plain gather.
        unsigned char *stage = region + kTmaStage;
        const int bw = P.tma_bw, bh = P.tma_bh, moff = (bw * bh + 127) & ~127;
        const int gx = blk.x - d, x0 = gx & ~15, xs = gx - x0;
        if (lt == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(&rsh->mbar, 2u * (uint32_t)(bw * bh));
            tma_load_2d(stage, &P.tm_img, x0, blk.image * P.H + blk.y - d, &rsh->mbar);
            tma_load_2d(stage + moff, &P.tm_mask, x0, blk.image * P.H + blk.y - d, &rsh->mbar);
        }
        if (!mbar_wait(&rsh->mbar, tph, P.wait_ns)) {
            // expired: report it, then let the copies in flight land (bounded)
            // before the region is reused
            report(P, kErrTimeout);
            mbar_wait(&rsh->mbar, tph, kDrainNs);
        }
        tph ^= 1u;
#pragma unroll
        for (int t = 0; t < NPOS; ++t) {
            const int pix = lt + t * TB;
            const int am = pix / F - off, an = pix % F - off;
            const bool in = am >= 0 && am < M && an >= 0 && an < M;
            const int o = in ? am * bw + xs + an : 0;
            mk[t] = in ? stage[moff + o] : 1;
            sv[t] = in ? (float)stage[o] : 0.f;
        }
    } else {
#pragma unroll
        for (int t = 0; t < NPOS; ++t) {
            const int pix = lt + t * TB;
            const int yy = min(max(blk.y - d + pix / F - off, 0), P.H - 1);
            const int xx = min(max(blk.x - d + pix % F - off, 0), P.W - 1);
            mk[t] = P.mask[((size_t)blk.image * P.H + yy) * P.W + xx];
            const char *row = static_cast<const char *>(P.images) + ((long long)blk.image * P.H + yy) * P.pitch;
            sv[t] = P.dtype == 0 ? (float)reinterpret_cast<const uint8_t *>(row)[xx]
                                 : reinterpret_cast<const float *>(row)[xx];
        }
    }
    float smax = 0.f;
    bool unmarked = false;   // a sample of the block's own B not marked lost
#pragma unroll
    for (int t = 0; t < NPOS; ++t) {
        const int pix = lt + t * TB;
        const int m = pix / F, n = pix % F;
        const int am = m - off, an = n - off;
        const int yy = blk.y - d + am, xx = blk.x - d + an;
        unmarked |= am >= d && am < d + b && an >= d && an < d + b && mk[t] == 0;
        bool inA = am >= 0 && am < M && an >= 0 && an < M &&
                   !(am >= d && am < d + b && an >= d && an < d + b) &&
                   yy >= 0 && yy < P.H && xx >= 0 && xx < P.W && mk[t] == 0;
        float wscale = 1.f;
        if constexpr (EXT) {
            // ordered: a lost sample of an earlier block is reused at its concealed value
            if (P.ordered && !inA && am >= 0 && am < M && an >= 0 && an < M &&
                !(am >= d && am < d + b && an >= d && an < d + b) && yy >= 0 && yy < P.H && xx >= 0 && xx < P.W) {
                bool reuse = false;
                for (int q = nb0; q < nb1 && !reuse; ++q) {
                    const BlockRec nbk = P.blocks[P.nb_list[q]];
                    reuse = yy >= nbk.y && yy < nbk.y + b && xx >= nbk.x && xx < nbk.x + b;
                }
                if (reuse) {
                    inA = true;
                    wscale = P.beta;
                    sv[t] = __ldcg(&P.out[((size_t)blk.image * P.H + yy) * P.W + xx]);
                }
            }
        }
        float w = inA ? __ldg(&C.wtab[am * M + an]) : 0.f;
        if constexpr (EXT) w *= wscale;
        // warm start: the support holds the residual of the estimate
        const float sr = (inA && P.est != nullptr) ? sv[t] - P.est[blk.orig * P.est_stride + am * M + an] : sv[t];
        const float ws = w * sr;
        if (inA) smax = fmaxf(smax, fabsf(sr));
        Z[m * FP + n] = make_float2(ws, w);
    }
    if (unmarked) report(P, kErrUnmarked);
    // alpha = the power of two in (max|s| / 2, max|s|] over the support:
    // balances the two real signals packed into one complex FFT (an exact
    // scaling; a maximum, so it is independent of the thread mapping)
    const float tmaxs = group_max<F, PAIRS, NT>(smax, gr, rsh);
    float alpha = 1.f;
    if (tmaxs > 0.f) {
        int e;
        frexpf(tmaxs, &e);
        alpha = ldexpf(1.f, e - 1);
    }
    for (int pix = lt; pix < F * F; pix += TB) {
        const int m = pix / F, n = pix % F;
        Z[m * FP + n].y *= alpha;
    }
    gsync<F, PAIRS, NT>(gr);
    // ---- S2/S3: FFT2 of z ----
    fft_pass<F, PAIRS, NT, true>(Z, s_tw, gr);
    fft_pass<F, PAIRS, NT, false>(Z, s_tw, gr);

    // ---- split into R_w = FFT{w s} and W = FFT{w} ----
    // W chunk rows k >= F/2 + 1 lie beyond the padded FFT buffer, so they are
    // written at once; the others are held until every thread has read Z.
    const int c0 = lt % LPR, r0 = lt / LPR;
    const float ainv = 1.f / alpha;
    float4 *Wd = reinterpret_cast<float4 *>(region);
    constexpr int SAFE = F / 2 + 1;
    uint64_t Rre[PAIRS], Rim[PAIRS];
    float4 Wc[PAIRS];
#pragma unroll
    for (int i = 0; i < PAIRS; ++i) {
        const int k = G::row(r0, i), km = (F - k) & (F - 1);
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
        if (k >= SAFE) {
            Wd[FSE_IX(k * F + c0, G::REGION / 16)] = Wc[i];
            Wd[FSE_IX(k * F + c0 + F / 2, G::REGION / 16)] = make_float4(Wc[i].y, Wc[i].x, Wc[i].w, Wc[i].z);
        }
    }
    const float W00 = Z[0].y * ainv;
    gsync<F, PAIRS, NT>(gr);
#pragma unroll
    for (int i = 0; i < PAIRS; ++i) {
        const int k = G::row(r0, i);
        if (k < SAFE) {
            Wd[FSE_IX(k * F + c0, G::REGION / 16)] = Wc[i];
            Wd[FSE_IX(k * F + c0 + F / 2, G::REGION / 16)] = make_float4(Wc[i].y, Wc[i].x, Wc[i].w, Wc[i].z);
        }
        if (G::RUNS && k < G::WROWS - F) {   // the copy of the first rows after row F-1
            Wd[FSE_IX((k + F) * F + c0, G::REGION / 16)] = Wc[i];
            Wd[FSE_IX((k + F) * F + c0 + F / 2, G::REGION / 16)] = make_float4(Wc[i].y, Wc[i].x, Wc[i].w, Wc[i].z);
        }
    }
    gsync<F, PAIRS, NT>(gr);

    // ---- B samples owned by this thread (NP of them; samples j >= b*b are
    //      computed but never stored) ----
    int pm_[NP], pn_[NP];
    float acc[NP];
#pragma unroll
    for (int t = 0; t < NP; ++t) {
        const int j = lt + t * TB;
        pm_[t] = off + d + j / b;
        pn_[t] = off + d + j % b;
        acc[t] = 0.f;
    }
    const float W0bar = W00 > 0.f ? 1.f / W00 : 0.f;
    const float cg = C.gamma * W0bar;

    // ---- S5: first selection (energies of R_w^(0)) ----
    float tmax = 0.f;
    int jb = 0;
#pragma unroll
    for (int j = 0; j < NQ; ++j) {
        const uint64_t e0 = energy2(Rre[4 * j], Rim[4 * j]), e1 = energy2(Rre[4 * j + 1], Rim[4 * j + 1]);
        const uint64_t e2 = energy2(Rre[4 * j + 2], Rim[4 * j + 2]), e3 = energy2(Rre[4 * j + 3], Rim[4 * j + 3]);
        const float a = max3f(lo_of(e0), hi_of(e0), lo_of(e1));
        const float bq = max3f(hi_of(e1), lo_of(e2), hi_of(e2));
        quartet_max(j, max3f(a, bq, fmaxf(lo_of(e3), hi_of(e3))), tmax, jb);
    }
    const int iters = C.iters;
    Pick pick;
    const bool gap = GAP && P.tr_second != nullptr;
    if (iters > 0) pick = group_argmax<F, PAIRS, NT, 1, GAP>(Rre, Rim, tmax, jb, gr, rsh, 0, gap);

    // Two copies of the iteration loop: the kernel sets without reduced-
    // precision storage keep the single loop below (the two-phase form, even
    // with its second phase compiled out, changed their register allocation
    // and spills); kSetFixW runs the two-phase form after it.
    if constexpr (!FIXW) {
        const ulonglong2 *Wq = reinterpret_cast<const ulonglong2 *>(region);
        for (int nu = 1; nu <= iters; ++nu) {
            // ---- S6/S7: coefficient and model ----
            const float cr = pick.rr * cg, ci = pick.ri * cg;
            const int u = (int)(pick.idx / F), v = (int)(pick.idx % F);
            if (GAP && P.tr_sel != nullptr && lt == 0) {   // traced launches (their own kernel set)
                const size_t o = (size_t)blk.orig * P.tr_stride + (nu - 1);
                P.tr_sel[o] = (int)pick.idx;
                P.tr_energy[o] = __uint_as_float(pick.ebits);
                P.tr_coef[o] = make_float2(cr, ci);
                if (P.tr_second != nullptr) P.tr_second[o] = __uint_as_float(pick.sbits);
            }
            // model update of this selection, evaluated on B: g += c phi_(u,v)
            // (independent of the residual update and of the next reduction)
            auto model = [&]() {
    #pragma unroll
                for (int t = 0; t < NP; ++t) {
                    const int ph = (u * pm_[t] + v * pn_[t]) & (F - 1);
                    const float2 tw = s_tw[ph * (64 / F)];
                    acc[t] = fmaf(cr, tw.x, fmaf(-ci, tw.y, acc[t]));
                }
            };
            if (nu == iters) {
                model();
                break;
            }
            // ---- S8: R_w[k,l] -= c W[k-u, l-v] fused with |R_w|^2 and max ----
            const uint64_t ncr = pk(-cr, -cr), pci = pk(ci, ci), nci = pk(-ci, -ci);
            // Non-runs: the row of pair i is (r0 - u + i*RSTEP) mod F; it wraps once,
            // at pair iw.  Pairs before the wrap address from A, the others from
            // A - F*F, so each load needs one select and an immediate offset.
            // Runs: run j starts at row (row(r0, RL j) - u) mod F and its RL rows are
            // contiguous in W (rows F.. repeat rows 0..RL-2): one base per run.
            const int qcol = (c0 - v) & (F - 1);
            const int rb = (r0 - u) & (F - 1);
            const int iw = (F - rb + RSTEP - 1) / RSTEP;
            const ulonglong2 *A = Wq + rb * F + qcol;
            const ulonglong2 *A2 = A - F * F;
            const ulonglong2 *Ar[G::RUNS ? PAIRS / G::RL : 1];
    #pragma unroll
            for (int r = 0; r < (G::RUNS ? PAIRS / G::RL : 1); ++r)
                Ar[r] = Wq + ((G::row(r0, G::RL * r) - u) & (F - 1)) * F + qcol;
            tmax = 0.f;
    #pragma unroll
            for (int j = 0; j < NQ; ++j) {
                float ev[8];
    #pragma unroll
                for (int ii = 0; ii < 4; ++ii) {
                    const int i = 4 * j + ii;
                    // one 16-byte load: (Re W, Re W') and (Im W, Im W') as two f32x2 operands
                    const ulonglong2 w =
                        G::RUNS ? FSE_LD(Wq, Ar[G::RUNS ? i / G::RL : 0] + (i % G::RL) * F, G::REGION / 16)
                                : FSE_LD(Wq, (i < iw ? A : A2) + i * RSTEP * F, G::REGION / 16);
                    const uint64_t wre = w.x, wim = w.y;
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
                quartet_max(j, max3f(a, bq, fmaxf(ev[6], ev[7])), tmax, jb);
            }
            model();
            // ---- S5: next selection ----
            pick = group_argmax<F, PAIRS, NT, 1, GAP>(Rre, Rim, tmax, jb, gr, rsh, nu & 1, gap);
        }
    } else {
        // One iteration: coefficient and model of pick nu, then (unless it is the
        // last) the residual update and the next pick.  FX: the update reads the
        // 16-bit codes of W (after the switch) instead of FP32 W.  Returns true
        // after the last iteration.
        const float dq = W00 * (1.f / 32767.f);   // value of one code step (FX)
        auto step = [&](int nu, auto fx) -> bool {
            constexpr bool FX = decltype(fx)::value;
            // ---- S6/S7: coefficient and model ----
            const float cr = pick.rr * cg, ci = pick.ri * cg;
            const int u = (int)(pick.idx / F), v = (int)(pick.idx % F);
            if (TRW && P.tr_sel != nullptr && lt == 0) {   // traced launches (their own kernel sets)
                const size_t o = (size_t)blk.orig * P.tr_stride + (nu - 1);
                P.tr_sel[o] = (int)pick.idx;
                P.tr_energy[o] = __uint_as_float(pick.ebits);
                P.tr_coef[o] = make_float2(cr, ci);
                if (GAP && P.tr_second != nullptr) P.tr_second[o] = __uint_as_float(pick.sbits);
            }
            // model update of this selection, evaluated on B: g += c phi_(u,v)
            // (independent of the residual update and of the next reduction)
            auto model = [&]() {
    #pragma unroll
                for (int t = 0; t < NP; ++t) {
                    const int ph = (u * pm_[t] + v * pn_[t]) & (F - 1);
                    const float2 tw = s_tw[ph * (64 / F)];
                    acc[t] = fmaf(cr, tw.x, fmaf(-ci, tw.y, acc[t]));
                }
            };
            if (nu == iters) {
                model();
                return true;
            }
            // ---- S8: R_w[k,l] -= c W[k-u, l-v] fused with |R_w|^2 and max ----
            // (FX: c scaled to code units, W read as codes)
            const float sr = FX ? cr * dq : cr, si = FX ? ci * dq : ci;
            const uint64_t ncr = pk(-sr, -sr), pci = pk(si, si), nci = pk(-si, -si);
            const uint64_t nbias2 = pk(-kFixBias, -kFixBias);
            // Non-runs: the row of pair i is (r0 - u + i*RSTEP) mod F; it wraps once,
            // at pair iw.  Pairs before the wrap address from A, the others from
            // A - F*F, so each load needs one select and an immediate offset.
            // Runs: run j starts at row (row(r0, RL j) - u) mod F and its RL rows are
            // contiguous in W (rows F.. repeat rows 0..RL-2): one base per run.
            using Chunk = typename std::conditional<FX, uint2, ulonglong2>::type;
            const Chunk *Wq = reinterpret_cast<const Chunk *>(region);
            const int qcol = (c0 - v) & (F - 1);
            const int rb = (r0 - u) & (F - 1);
            const int iw = (F - rb + RSTEP - 1) / RSTEP;
            const Chunk *A = Wq + rb * F + qcol;
            const Chunk *A2 = A - F * F;
            const Chunk *Ar[G::RUNS ? PAIRS / G::RL : 1];
    #pragma unroll
            for (int r = 0; r < (G::RUNS ? PAIRS / G::RL : 1); ++r)
                Ar[r] = Wq + ((G::row(r0, G::RL * r) - u) & (F - 1)) * F + qcol;
            tmax = 0.f;
    #pragma unroll
            for (int j = 0; j < NQ; ++j) {
                float ev[8];
    #pragma unroll
                for (int ii = 0; ii < 4; ++ii) {
                    const int i = 4 * j + ii;
                    // one load: (Re W, Re W') and (Im W, Im W') as two f32x2
                    // operands (16 bytes of FP32, or 8 bytes of codes)
                    const Chunk w =
                        G::RUNS ? FSE_LD(Wq, Ar[G::RUNS ? i / G::RL : 0] + (i % G::RL) * F, G::WROWS * F)
                                : FSE_LD(Wq, (i < iw ? A : A2) + i * RSTEP * F, G::WROWS * F);
                    uint64_t wre, wim;
                    if constexpr (FX) {
                        wre = fix_unpack(w.x, nbias2);
                        wim = fix_unpack(w.y, nbias2);
                    } else {
                        wre = w.x;
                        wim = w.y;
                    }
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
                quartet_max(j, max3f(a, bq, fmaxf(ev[6], ev[7])), tmax, jb);
            }
            model();
            // ---- S5: next selection ----
            pick = group_argmax<F, PAIRS, NT, 1, GAP>(Rre, Rim, tmax, jb, gr, rsh, nu & 1, gap);
            return false;
        };
        // updates before the switch: all of them unless FIXW
        int kfix = iters;
        if constexpr (FIXW) kfix = min(iters, max(P.fix_from, 0));
        for (int nu = 1; nu <= kfix; ++nu)
            if (step(nu, std::false_type{})) break;
        if constexpr (FIXW) {
            if (kfix < iters) {
                // W's FP32 chunks -> codes; the codes are decided in FP32 with the
                // scale 32767 / W[0,0]
                compact_w<F, PAIRS, NT>(region, 32767.f * W0bar, gr);
                for (int nu = kfix + 1; nu <= iters; ++nu)
                    if (step(nu, std::true_type{})) break;
            }
        }
    }

    // ---- S10: write Re{g} on B ----
#pragma unroll
    for (int t = 0; t < NP; ++t) {
        const int j = lt + t * TB;
        if (j < b * b) {
            const int pm = j / b, pn = j % b;
            float val = acc[t] + (P.est != nullptr ? P.est[blk.orig * P.est_stride + (d + pm) * M + d + pn] : 0.f);
            if (P.clamp_u8) val = rintf(fminf(fmaxf(val, 0.f), 255.f));
            if (P.out != nullptr)
                P.out[FSE_IX(((size_t)blk.image * P.H + blk.y + pm) * P.W + blk.x + pn,
                             (long long)P.n_images * P.H * P.W)] = val;
            if (P.patches != nullptr) P.patches[blk.patch_off + j] = val;
        }
    }
    if constexpr (EXT) {
        if (P.ordered) {   // publish: every thread's output stores, then the flag
            __threadfence();
            gsync<F, PAIRS, NT>(gr);
            if (lt == 0) st_release_gpu(&P.done[blk.orig], 1);
        }
    }
}

// Video volumes: the same steps for a volume of C.T frames centred on the
// block's frame, transform grid FT x F x F with bins indexed (t F + k) F + l
// -- Algorithm 1 with 3-D basis functions and 3-D circular shifts.  (Kept
// apart from process() so that the image path's code is not touched by the
// temporal dimension.)
template <int F, int PAIRS, int NT, int NP, int FT, bool GAP = false>
__device__ __forceinline__ void process_vol(const DevParams &P, const DevClass &C, int first, int count,
                                            unsigned char *smem, const float2 *s_tw, RedShared *rsh) {
    static_assert(FT > 1, "image areas run process()");
    constexpr bool EXT = false;   // ordered concealment is for image classes
    using G = Geo<F, PAIRS, FT>;
    constexpr int TB = G::TB, LPR = G::LPR, RSTEP = G::RSTEP, FP = G::FP, NQ = G::NQ;
    Grp gr;
    gr.g = threadIdx.x / TB;
    gr.lt = threadIdx.x % TB;
    const bool active = gr.g < count;
    gr.amask = __ballot_sync(0xffffffffu, active);
    if (!active) return;
    const int lt = gr.lt;

    const BlockRec blk = P.blocks[first + gr.g];
#ifdef FSE_BOUNDS_CHECK
    // the block lies inside its image (the host validates this too); the
    // whole group skips a block that does not
    if (blk.image < 0 || blk.image >= P.n_images || blk.x < 0 || blk.y < 0 || blk.x + C.b > P.W ||
        blk.y + C.b > P.H) {
        report(P, kErrBounds);
        return;
    }
#endif
    unsigned char *region = smem + gr.g * G::REGION;
    float2 *Z = reinterpret_cast<float2 *>(region);

    const int b = C.b, d = C.d, M = C.M, off = C.off;
    const bool ordered = EXT && FT == 1 && P.ordered;   // EXT: compiled with ordered concealment
    int nb0 = 0, nb1 = 0;
    if (ordered) {
        // the blocks this one reuses must have written their output (bounded)
        nb0 = P.nb_start[blk.orig];
        nb1 = P.nb_start[blk.orig + 1];
        if (lt == 0) {
            const uint64_t t0 = globaltimer_ns();
            for (int q = nb0; q < nb1; ++q)
                while (ld_acquire_gpu(&P.done[P.nb_list[q]]) == 0) {
                    if (globaltimer_ns() - t0 > P.wait_ns) {
                        report(P, kErrTimeout);
                        break;
                    }
                    __nanosleep(128);
                }
        }
        gsync<F, PAIRS, NT, FT>(gr);
    }
    // ---- S0/S1: gather the area, Eq. (3) weights, z = (w s, w) ----
    // All loads of the thread's grid positions are issued first (clamped to
    // the image, so always in bounds), then the weights are applied: one
    // memory round trip instead of one per position.
    constexpr int NPOS = FT * F * F / TB;
    float sv[NPOS];
    uint8_t mk[NPOS];
    // volume plane t holds frame blk.image + t - toff - tc (clamped for the
    // load; frames outside the video are not support)
#pragma unroll
    for (int t = 0; t < NPOS; ++t) {
        const int pix = lt + t * TB;
        const int pl = pix / (F * F), pp = pix % (F * F);
        const int fr = FT == 1 ? blk.image : min(max(blk.image + pl - C.toff - C.tc, 0), P.n_images - 1);
        const int yy = min(max(blk.y - d + pp / F - off, 0), P.H - 1);
        const int xx = min(max(blk.x - d + pp % F - off, 0), P.W - 1);
        mk[t] = P.mask[((size_t)fr * P.H + yy) * P.W + xx];
        const char *row = static_cast<const char *>(P.images) + ((long long)fr * P.H + yy) * P.pitch;
        sv[t] = P.dtype == 0 ? (float)reinterpret_cast<const uint8_t *>(row)[xx]
                             : reinterpret_cast<const float *>(row)[xx];
    }
    float smax = 0.f;
    bool unmarked = false;   // a sample of the block's own B not marked lost
#pragma unroll
    for (int t = 0; t < NPOS; ++t) {
        const int pix = lt + t * TB;
        const int pl = pix / (F * F), pp = pix % (F * F);
        const int m = pp / F, n = pp % F;
        const int am = m - off, an = n - off;
        const int yy = blk.y - d + am, xx = blk.x - d + an;
        const int tau = pl - C.toff;                       // frame of the volume (FT = 1: 0)
        const int fr = blk.image + tau - C.tc;
        const bool own = tau == C.tc && am >= d && am < d + b && an >= d && an < d + b;
        unmarked |= own && mk[t] == 0;
        const bool inV = am >= 0 && am < M && an >= 0 && an < M && !own && yy >= 0 && yy < P.H && xx >= 0 &&
                         xx < P.W && (FT == 1 || (tau >= 0 && tau < C.T && fr >= 0 && fr < P.n_images));
        // ordered: a lost sample of an earlier block is reused at its concealed value
        bool reuse = false;
        if (ordered && inV && mk[t] != 0) {
            for (int q = nb0; q < nb1 && !reuse; ++q) {
                const BlockRec nbk = P.blocks[P.nb_list[q]];
                reuse = yy >= nbk.y && yy < nbk.y + b && xx >= nbk.x && xx < nbk.x + b;
            }
        }
        const bool inA = inV && (mk[t] == 0 || reuse);
        const float w = inA ? __ldg(&C.wtab[(FT == 1 ? 0 : tau * M * M) + am * M + an]) * (reuse ? P.beta : 1.f)
                            : 0.f;
        if (reuse) sv[t] = __ldcg(&P.out[((size_t)blk.image * P.H + yy) * P.W + xx]);
        // warm start: the support holds the residual of the estimate
        const float sr = (inA && P.est != nullptr) ? sv[t] - P.est[blk.orig * P.est_stride + am * M + an] : sv[t];
        const float ws = w * sr;
        if (inA) smax = fmaxf(smax, fabsf(sr));
        Z[(pl * F + m) * FP + n] = make_float2(ws, w);
    }
    // alpha = the power of two in (max|s| / 2, max|s|] over the support:
    // balances the two real signals packed into one complex FFT (an exact
    // scaling; a maximum, so it is independent of the thread mapping)
    if (unmarked) report(P, kErrUnmarked);
    const float tmaxs = group_max<F, PAIRS, NT, FT>(smax, gr, rsh);
    float alpha = 1.f;
    if (tmaxs > 0.f) {
        int e;
        frexpf(tmaxs, &e);
        alpha = ldexpf(1.f, e - 1);
    }
    for (int pix = lt; pix < FT * F * F; pix += TB) {
        const int r = pix / F, n = pix % F;                 // r: plane * F + row
        Z[r * FP + n].y *= alpha;
    }
    gsync<F, PAIRS, NT, FT>(gr);
    // ---- S2/S3: FFT2 of z (and the temporal pass of a volume) ----
    fft_pass<F, PAIRS, NT, true, FT>(Z, s_tw, gr);
    fft_pass<F, PAIRS, NT, false, FT>(Z, s_tw, gr);
    if constexpr (FT > 1) time_pass<F, PAIRS, NT, FT>(Z, gr);

    // ---- split into R_w = FFT{w s} and W = FFT{w} ----
    // W chunk rows k >= SAFE lie beyond the padded FFT buffer, so they are
    // written at once; the others are held until every thread has read Z.
    // (Rows are plane * F + row for a volume; the mirror bin of (t, k, l) is
    // (-t, -k, -l).)
    const int c0 = lt % LPR, r0 = lt / LPR;
    const float ainv = 1.f / alpha;
    float4 *Wd = reinterpret_cast<float4 *>(region);
    constexpr int SAFE = (FT * FP + 1) / 2;                // ceil(FT F FP 8 / (F 16))
    uint64_t Rre[PAIRS], Rim[PAIRS];
    float4 Wc[PAIRS];
#pragma unroll
    for (int i = 0; i < PAIRS; ++i) {
        const int k = G::row(r0, i);
        const int km = (((FT - k / F) & (FT - 1)) * F) + ((F - k % F) & (F - 1));   // mirror row
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
        const int kw = G::wrow(k);
        if (kw >= SAFE) {
            Wd[FSE_IX(kw * F + c0, G::REGION / 16)] = Wc[i];
            Wd[FSE_IX(kw * F + c0 + F / 2, G::REGION / 16)] = make_float4(Wc[i].y, Wc[i].x, Wc[i].w, Wc[i].z);
        }
    }
    const float W00 = Z[0].y * ainv;
    gsync<F, PAIRS, NT, FT>(gr);
#pragma unroll
    for (int i = 0; i < PAIRS; ++i) {
        const int k = G::row(r0, i), kw = G::wrow(k);
        if (kw < SAFE) {
            Wd[FSE_IX(kw * F + c0, G::REGION / 16)] = Wc[i];
            Wd[FSE_IX(kw * F + c0 + F / 2, G::REGION / 16)] = make_float4(Wc[i].y, Wc[i].x, Wc[i].w, Wc[i].z);
        }
        if (G::VRUNS && k % F < G::PROWS - F) {   // each plane's copy of its first rows after row F-1
            Wd[FSE_IX((kw + F) * F + c0, G::REGION / 16)] = Wc[i];
            Wd[FSE_IX((kw + F) * F + c0 + F / 2, G::REGION / 16)] = make_float4(Wc[i].y, Wc[i].x, Wc[i].w, Wc[i].z);
        }
    }
    gsync<F, PAIRS, NT, FT>(gr);

    // ---- B samples owned by this thread (NP of them; samples j >= b*b are
    //      computed but never stored) ----
    int pm_[NP], pn_[NP];
    float acc[NP];
#pragma unroll
    for (int t = 0; t < NP; ++t) {
        const int j = lt + t * TB;
        pm_[t] = off + d + j / b;
        pn_[t] = off + d + j % b;
        acc[t] = 0.f;
    }
    const float W0bar = W00 > 0.f ? 1.f / W00 : 0.f;
    const float cg = C.gamma * W0bar;

    // ---- S5: first selection (energies of R_w^(0)) ----
    float tmax = 0.f;
    int jb = 0;
#pragma unroll
    for (int j = 0; j < NQ; ++j) {
        const uint64_t e0 = energy2(Rre[4 * j], Rim[4 * j]), e1 = energy2(Rre[4 * j + 1], Rim[4 * j + 1]);
        const uint64_t e2 = energy2(Rre[4 * j + 2], Rim[4 * j + 2]), e3 = energy2(Rre[4 * j + 3], Rim[4 * j + 3]);
        const float a = max3f(lo_of(e0), hi_of(e0), lo_of(e1));
        const float bq = max3f(hi_of(e1), lo_of(e2), hi_of(e2));
        quartet_max(j, max3f(a, bq, fmaxf(lo_of(e3), hi_of(e3))), tmax, jb);
    }
    const int iters = C.iters;
    Pick pick;
    const bool gap = GAP && P.tr_second != nullptr;
    if (iters > 0) pick = group_argmax<F, PAIRS, NT, FT, GAP>(Rre, Rim, tmax, jb, gr, rsh, 0, gap);

    const ulonglong2 *Wq = reinterpret_cast<const ulonglong2 *>(region);
    for (int nu = 1; nu <= iters; ++nu) {
        // ---- S6/S7: coefficient and model ----
        const float cr = pick.rr * cg, ci = pick.ri * cg;
        const int u = (int)((pick.idx / F) % F), v = (int)(pick.idx % F);
        const int wt = FT == 1 ? 0 : (int)(pick.idx / (F * F));   // temporal frequency
        // the temporal part of the phase on B's plane, in 64ths of a turn
        const int tphase = FT == 1 ? 0 : (wt * (C.toff + C.tc) * (64 / FT)) & 63;
        if (GAP && P.tr_sel != nullptr && lt == 0) {   // traced launches (their own kernel set)
            const size_t o = (size_t)blk.orig * P.tr_stride + (nu - 1);
            P.tr_sel[o] = (int)pick.idx;
            P.tr_energy[o] = __uint_as_float(pick.ebits);
            P.tr_coef[o] = make_float2(cr, ci);
            if (P.tr_second != nullptr) P.tr_second[o] = __uint_as_float(pick.sbits);
        }
        // model update of this selection, evaluated on B: g += c phi_(u,v)
        // (independent of the residual update and of the next reduction)
        auto model = [&]() {
#pragma unroll
            for (int t = 0; t < NP; ++t) {
                const int ph = ((u * pm_[t] + v * pn_[t]) * (64 / F) + tphase) & 63;
                const float2 tw = s_tw[ph];
                acc[t] = fmaf(cr, tw.x, fmaf(-ci, tw.y, acc[t]));
            }
        };
        if (nu == iters) {
            model();
            break;
        }
        // ---- S8: R_w[k,l] -= c W[k-u, l-v] fused with |R_w|^2 and max ----
        const uint64_t ncr = pk(-cr, -cr), pci = pk(ci, ci), nci = pk(-ci, -ci);
        // Non-runs: the row of pair i is (r0 - u + i*RSTEP) mod F; it wraps once,
        // at pair iw.  Pairs before the wrap address from A, the others from
        // A - F*F, so each load needs one select and an immediate offset.
        // Runs: run j starts at row (row(r0, RL j) - u) mod F and its RL rows are
        // contiguous in W (rows F.. repeat rows 0..RL-2): one base per run.
        const int qcol = (c0 - v) & (F - 1);
        const int rb = (r0 - u) & (F - 1);
        const int iw = (F - rb + RSTEP - 1) / RSTEP;
        const ulonglong2 *A = Wq + rb * F + qcol;
        const ulonglong2 *A2 = A - F * F;
        const ulonglong2 *Ar[G::RUNS ? PAIRS / G::RL : 1];
#pragma unroll
        for (int r = 0; r < (G::RUNS ? PAIRS / G::RL : 1); ++r)
            Ar[r] = Wq + ((G::row(r0, G::RL * r) - u) & (F - 1)) * F + qcol;
        // Volumes: pair i lies in plane i / KP at row r0 + (i % KP) RSTEP; its
        // shifted chunk is plane (i / KP - wt) mod FT, row (r0 + (i % KP) RSTEP
        // - u) mod F: KP row offsets and FT plane offsets per iteration.
        // Volume runs (VRUNS): pair i lies in plane i / KP at row KP r0 +
        // i % KP; the shifted rows of one plane are consecutive from (KP r0 -
        // u) mod F (the plane's copied rows absorb the wrap): one base per
        // plane, immediate offsets.
        constexpr int KP = FT == 1 ? 1 : F / RSTEP;
        int kofs[KP], tofs[FT];
        const ulonglong2 *Pb[FT];
        if constexpr (G::VRUNS) {
            const int rbase = ((KP * r0 - u) & (F - 1)) * F + qcol;
#pragma unroll
            for (int p2 = 0; p2 < FT; ++p2) Pb[p2] = Wq + ((p2 - wt) & (FT - 1)) * G::PROWS * F + rbase;
        } else {
#pragma unroll
            for (int j2 = 0; j2 < KP; ++j2) kofs[j2] = ((r0 + j2 * RSTEP - u) & (F - 1)) * F + qcol;
#pragma unroll
            for (int p2 = 0; p2 < FT; ++p2) tofs[p2] = ((p2 - wt) & (FT - 1)) * F * F;
        }
        tmax = 0.f;
#pragma unroll
        for (int j = 0; j < NQ; ++j) {
            float ev[8];
#pragma unroll
            for (int ii = 0; ii < 4; ++ii) {
                const int i = 4 * j + ii;
                // one 16-byte load: (Re W, Re W') and (Im W, Im W') as two f32x2 operands
                const ulonglong2 w =
                    G::VRUNS ? FSE_LD(Wq, Pb[G::VRUNS ? i / KP : 0] + (i % KP) * F, G::REGION / 16)
                    : FT > 1 ? FSE_LD(Wq, Wq + tofs[i / KP] + kofs[i % KP], G::REGION / 16)
                    : G::RUNS ? FSE_LD(Wq, Ar[G::RUNS ? i / G::RL : 0] + (i % G::RL) * F, G::REGION / 16)
                              : FSE_LD(Wq, (i < iw ? A : A2) + i * RSTEP * F, G::REGION / 16);
                const uint64_t wre = w.x, wim = w.y;
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
            quartet_max(j, max3f(a, bq, fmaxf(ev[6], ev[7])), tmax, jb);
        }
        model();
        // ---- S5: next selection ----
        pick = group_argmax<F, PAIRS, NT, FT, GAP>(Rre, Rim, tmax, jb, gr, rsh, nu & 1, gap);
    }

    // ---- S10: write Re{g} on B ----
#pragma unroll
    for (int t = 0; t < NP; ++t) {
        const int j = lt + t * TB;
        if (j < b * b) {
            const int pm = j / b, pn = j % b;
            float val = acc[t] + (P.est != nullptr ? P.est[blk.orig * P.est_stride + (d + pm) * M + d + pn] : 0.f);
            if (P.clamp_u8) val = rintf(fminf(fmaxf(val, 0.f), 255.f));
            if (P.out != nullptr)
                P.out[FSE_IX(((size_t)blk.image * P.H + blk.y + pm) * P.W + blk.x + pn,
                             (long long)P.n_images * P.H * P.W)] = val;
            if (P.patches != nullptr) P.patches[blk.patch_off + j] = val;
        }
    }
    if (ordered) {   // publish: every thread's output stores, then the flag
        __threadfence();
        gsync<F, PAIRS, NT, FT>(gr);
        if (lt == 0) st_release_gpu(&P.done[blk.orig], 1);
    }
}

template <int F, int PAIRS, int NT, int FT = 1, bool EXT = false, bool GAP = false, bool TMA = false,
          bool FIXW = false>
__device__ __forceinline__ void process_class(const DevParams &P, const DevClass &C, int first, int count,
                                              unsigned char *smem, const float2 *s_tw, RedShared *rsh,
                                              uint32_t &tph) {
    constexpr int TB = Geo<F, PAIRS, FT>::TB;
    if constexpr (FT == 1) {
        constexpr int NPS = PAIRS >= 16 ? 2 : 1;      // covers b <= F/4
        constexpr int NPL = PAIRS / 2;                // covers b <= F/2
        if (C.b * C.b <= TB * NPS)
            process<F, PAIRS, NT, NPS, EXT, GAP, TMA, FIXW>(P, C, first, count, smem, s_tw, rsh, tph);
        else process<F, PAIRS, NT, NPL, EXT, GAP, TMA, FIXW>(P, C, first, count, smem, s_tw, rsh, tph);
    } else {
        // a volume's block group is FT times larger: b <= F/2 needs
        // F^2/4 / TB = PAIRS / (2 FT) samples per thread (at least 1)
        constexpr int NPV = PAIRS / (2 * FT) > 0 ? PAIRS / (2 * FT) : 1;
        process_vol<F, PAIRS, NT, NPV, FT, GAP>(P, C, first, count, smem, s_tw, rsh);
    }
}

// ------------------------------------------------------ persistent kernel
// NT threads per CTA (128 or 256), up to 71 KB of dynamic shared memory, at
// most three CTAs per SM.  KS selects what the instantiation carries:
//   kSetImage  image classes of every FFT size (16, 32, 64)
//   kSetExt    also video volumes and ordered concealment
//   kSetF64    image classes of FFT size 64 only
//   kSetTrace  everything kSetExt runs, plus the trace's top-two gap (the
//              largest energy besides each pick): traced batches only
//   kSetFixW   image classes of FFT size 64 with reduced-precision residual
//              storage (16-bit fixed-point W from iteration P.fix_from on;
//              writes the selection trace when one is requested)
// A batch runs the smallest set that covers its classes, so the code and
// register allocation of the common cases are not burdened by the others.
template <int NT, int KS>
__global__ void __launch_bounds__(NT, 3) fse_batch_kernel(const __grid_constant__ DevParams P) {
    constexpr int PAIRS = 2048 / NT;
    constexpr bool EXT = KS == kSetExt || KS == kSetTrace;
    constexpr bool GAP = KS == kSetTrace;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ float2 s_tw[64];
    __shared__ int s_item;
    __shared__ RedShared rsh;
    for (int i = threadIdx.x; i < 64; i += NT) s_tw[i] = P.tw[i];
    if ((KS == kSetF64 || KS == kSetFixW) && threadIdx.x == 0 && P.tma) mbar_init(&rsh.mbar, 1);
    uint32_t tph = 0;   // phase of rsh.mbar the next window waits for
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
        if (EXT && C.FT == 4) {
            if constexpr (EXT) {
                if (C.F == 32) process_class<32, PAIRS, NT, 4, true, GAP>(P, C, first, count, smem, s_tw, &rsh, tph);
                else process_class<16, PAIRS, NT, 4, true, GAP>(P, C, first, count, smem, s_tw, &rsh, tph);
            }
        } else if constexpr (KS == kSetF64) {
            process_class<64, PAIRS, NT, 1, false, false, true>(P, C, first, count, smem, s_tw, &rsh, tph);
        } else if constexpr (KS == kSetFixW) {
            process_class<64, PAIRS, NT, 1, false, false, true, true>(P, C, first, count, smem, s_tw, &rsh, tph);
        } else {
            switch (C.F) {
                case 64: process_class<64, PAIRS, NT, 1, EXT, GAP>(P, C, first, count, smem, s_tw, &rsh, tph); break;
                case 32: process_class<32, PAIRS, NT, 1, EXT, GAP>(P, C, first, count, smem, s_tw, &rsh, tph); break;
                default: process_class<16, PAIRS, NT, 1, EXT, GAP>(P, C, first, count, smem, s_tw, &rsh, tph); break;
            }
        }
        __syncthreads();
    }
}

}  // namespace fse
