// Learned cell-skip proposal: an opt-in approximate mode on top of the exact
// path (the paper has no counterpart; the exact path stays the fallback and
// the reference the proposal's recall is measured against).
//
// k_skipnet    one CTA per 26 x 12 block of the 1/8-scale logit map of an
//              image.  It box-averages 8x8 blocks of level 0 (scaled to
//              [-0.5, 0.5]) and runs three 3x3 convolutions with zero padding
//              (1 -> 16 -> 16 -> 1 channels, ReLU after the first two) on the
//              5th-generation tensor cores: tcgen05.mma kind::f16 with BF16
//              operands in shared memory and FP32 accumulators in tensor
//              memory.  Inputs and activations are rounded to BF16 between
//              layers; weights are BF16 as stored in the model.
// k_skipcells  one thread per s0 culling cell: the cell is skipped when the
//              largest logit over its block of the 1/8 map is below the
//              threshold.  The detection kernel then ignores every cell of
//              any level whose centre projects into a skipped s0 cell.
//
// Convolution as GEMM.  All grids (input X, first activation a1, second
// activation a2, logits) share one row pitch P = 32 positions, so a 3x3 tap
// (dy, dx) of a convolution is the previous grid shifted by s = dy * P + dx
// rows: layer l computes D[m][co] = sum over taps t and input channels ci of
// In[m + s_t][ci] * W[co][ci][t].  Rows m whose column is too close to the
// right edge wrap into the next grid row; they are computed and discarded
// (each GEMM row depends only on its own A row).  Operands are K-major
// without swizzle: a grid is stored as two 8-channel chunks, row m of chunk c
// at c * chunk_bytes + 16 m, so an 8-row core matrix starting at ANY row is
// 128 contiguous bytes and the A operand of tap t starts 16 s_t bytes later
// (descriptor: leading-dimension offset = chunk_bytes between the two K
// chunks, stride offset = 128 bytes between 8-row groups).  Layer 1 has one
// input channel and uses an explicit im2col (K = 9 taps padded to 16).
#include <cuda_bf16.h>

#include "jslam_internal.h"

namespace jslam {

constexpr int kSkipTW = kSkipTileW;   // logits per CTA: 26 columns
constexpr int kSkipTH = kSkipTileH;   //                 12 rows
constexpr int kSkipP = kSkipTW + 6;   // common grid pitch (32)
constexpr int kSkipThreads = 256;
constexpr int kMmaM = 128, kMmaN = 16;

constexpr int round128(int v) { return (v + 127) / 128 * 128; }
constexpr int kR3 = kSkipTH * kSkipP;                     // logit rows computed: 384
constexpr int kR2 = round128(kR3 + 2 * kSkipP + 2);       // a2 rows: 512
constexpr int kR1 = round128(kR2 + 2 * kSkipP + 2);       // a1 rows: 640
constexpr int kXRows = (kR1 + 2 * kSkipP + 2 + kSkipP - 1) / kSkipP;  // input grid rows: 23
constexpr int kT1 = kR1 / kMmaM, kT2 = kR2 / kMmaM, kT3 = kR3 / kMmaM;  // M tiles: 5, 4, 3
constexpr uint32_t kTmemCols = 128;                       // >= 16 * max(kT1, kT2, kT3)
static_assert(kSkipP == 32, "grid pitch");
static_assert(16 * kT1 <= (int)kTmemCols && 16 * kT2 <= (int)kTmemCols && 16 * kT3 <= (int)kTmemCols, "TMEM");
static_assert(kR3 % kMmaM == 0, "logit rows fill whole M tiles");

// Shared-memory layout (byte offsets; every operand 128-byte aligned).
constexpr int kChunk1 = kR1 * 16;                 // bytes per 8-channel chunk of A1 / a1
constexpr int kChunk2 = kR2 * 16;                 // of a2
constexpr int kOffU = 0;                          // A1 (im2col of X), later a2
constexpr int kOffA1 = kOffU + 2 * kChunk1;       // a1
constexpr int kOffX = kOffA1 + 2 * kChunk1;       // X, FP32, kXRows x P
constexpr int kOffB1 = kOffX + kXRows * kSkipP * 4;
constexpr int kOffB2 = kOffB1 + 512;              // 9 taps x 512 bytes
constexpr int kOffB3 = kOffB2 + 9 * 512;
constexpr int kOffBias = kOffB3 + 9 * 512;        // b1[16], b2[16], b3
constexpr int kOffBar = kOffBias + 144;           // mbarrier (8 bytes) + TMEM base (4 bytes)
constexpr int kSkipSmem = kOffBar + 16;
static_assert(kChunk2 <= kChunk1, "a2 fits where A1 was");
static_assert(kOffX % 128 == 0 && kOffB1 % 128 == 0 && kOffB2 % 128 == 0 && kOffB3 % 128 == 0, "alignment");
// The largest A row any layer reads stays inside its grid.
static_assert((kT2 - 1) * kMmaM + 127 + 2 * kSkipP + 2 < kR1, "layer 2 reads inside a1");
static_assert((kT3 - 1) * kMmaM + 127 + 2 * kSkipP + 2 < kR2, "layer 3 reads inside a2");
static_assert(kR1 - 1 + 2 * kSkipP + 2 < kXRows * kSkipP, "im2col reads inside X");

// Instruction descriptor of tcgen05.mma kind::f16: D FP32 (bits 4-5 = 1),
// A and B BF16 (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kMmaN >> 3) << 17) |
                            ((uint32_t)(kMmaM >> 4) << 24);

// Shared-memory matrix descriptor, no swizzle: start address, leading-
// dimension byte offset (between the two K chunks of an MMA), stride byte
// offset (between 8-row groups), all in 16-byte units; bits 46-48 = 0b001.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ uint32_t saddr_of(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, bool accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(kIdesc), "r"((uint32_t)accumulate) : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// Wait for the mbarrier phase `parity`, giving up after about a second.
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity)
{
    const long long start = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
        if (clock64() - start > (1ll << 31)) return false;
    }
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float tmem_ld1(uint32_t taddr)
{
    uint32_t r;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    return __uint_as_float(r);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// Bias + ReLU + BF16 of 16 accumulator channels of GEMM row r, stored as the
// two 8-channel chunks of row r of an activation grid (zero where the row's
// position lies outside the 1/8 map or in the discarded right-edge columns).
__device__ __forceinline__ void store_act(uint8_t *grid, int chunk_bytes, int r, const float (&acc)[16],
                                          const float *bias, bool keep)
{
    uint32_t w[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float a = keep ? fmaxf(acc[2 * i] + bias[2 * i], 0.0f) : 0.0f;
        const float c = keep ? fmaxf(acc[2 * i + 1] + bias[2 * i + 1], 0.0f) : 0.0f;
        w[i] = pack_bf16(a, c);
    }
    *reinterpret_cast<uint4 *>(grid + 16 * r) = make_uint4(w[0], w[1], w[2], w[3]);
    *reinterpret_cast<uint4 *>(grid + chunk_bytes + 16 * r) = make_uint4(w[4], w[5], w[6], w[7]);
}

// Order this thread's shared-memory writes before the tensor cores' reads
// and the TMEM reads before later MMAs, across a CTA barrier.
__device__ __forceinline__ void sync_for_mma()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__global__ void __launch_bounds__(kSkipThreads) k_skipnet(Batch b, const SkipModelDev m)
{
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ int s_ok;
    const int img = blockIdx.y;
    const ImageDesc &I = b.images[img];
    const int W8 = I.skip_w8, H8 = I.skip_h8;
    const int tiles_x = (W8 + kSkipTW - 1) / kSkipTW;
    const int tile = blockIdx.x;
    if (tile >= tiles_x * ((H8 + kSkipTH - 1) / kSkipTH)) return;  // before any TMEM is held
    const int tx0 = (tile % tiles_x) * kSkipTW, ty0 = (tile / tiles_x) * kSkipTH;
    const LevelDesc &L0 = b.levels[I.level_base];
    const uint8_t *raw = L0.raw;
    const int pitch = L0.pitch, W0 = I.W0, H0 = I.H0;

    uint8_t *U = smem + kOffU;
    uint8_t *A1g = smem + kOffA1;
    float *X = reinterpret_cast<float *>(smem + kOffX);
    uint16_t *B1 = reinterpret_cast<uint16_t *>(smem + kOffB1);
    uint16_t *B2 = reinterpret_cast<uint16_t *>(smem + kOffB2);
    uint16_t *B3 = reinterpret_cast<uint16_t *>(smem + kOffB3);
    float *bias = reinterpret_cast<float *>(smem + kOffBias);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + kOffBar);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + kOffBar + 8);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr_of(tmem_slot)),
                     "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 32) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr_of(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }

    // B operands, K-major: element (n, k) of a 16 x 16 tap matrix at byte
    // (k / 8) * 256 + n * 16 + (k % 8) * 2.  B1: k = tap (9 of 16);
    // B2[t]: k = input channel; B3[t]: only n = 0 is a real output.
    for (int i = threadIdx.x; i < 256; i += kSkipThreads) {
        const int n = i >> 4, k = i & 15;
        const int o = (k >> 3) * 128 + n * 8 + (k & 7);
        B1[o] = k < 9 ? m.w1[n * 9 + k] : (uint16_t)0;
    }
    static_assert(kSkipThreads == 256, "one tap matrix element per thread and tap");
#pragma unroll
    for (int t9 = 0; t9 < 9; ++t9) {  // unrolled: the 18 weight loads of a thread in flight together
        const int i = t9 * 256 + threadIdx.x;
        const int t = i >> 8, n = (i >> 4) & 15, k = i & 15;
        const int o = t * 256 + (k >> 3) * 128 + n * 8 + (k & 7);
        B2[o] = m.w2[(n * kSkipC + k) * 9 + t];
        B3[o] = n == 0 ? m.w3[k * 9 + t] : (uint16_t)0;
    }
    if (threadIdx.x < kSkipC) {
        bias[threadIdx.x] = m.b1[threadIdx.x];
        bias[16 + threadIdx.x] = m.b2[threadIdx.x];
    }
    if (threadIdx.x == 0) bias[32] = m.b3;

    // X: box means of 8x8 level-0 blocks on the input grid (row iy, column ix
    // is 1/8-map position (ty0 - 3 + iy, tx0 - 3 + ix)); zero outside the map
#pragma unroll
    for (int j = 0; j < (kXRows * kSkipP + kSkipThreads - 1) / kSkipThreads; ++j) {
        const int i = j * kSkipThreads + threadIdx.x;
        if (i >= kXRows * kSkipP) break;
        const int iy = i / kSkipP, ix = i - iy * kSkipP;
        const int gy = ty0 - 3 + iy, gx = tx0 - 3 + ix;
        float v = 0.0f;
        if (gy >= 0 && gy < H8 && gx >= 0 && gx < W8) {
            const int y0 = 8 * gy, x0 = 8 * gx;
            const int y1 = min(y0 + 8, H0), x1 = min(x0 + 8, W0);
            uint32_t sum = 0;
            if (x1 - x0 == 8) {
                // the block's rows requested together (the loop is unrolled
                // with a guard), then summed: one memory latency per block
                const uint8_t *col = raw + (size_t)y0 * pitch + x0;
                uint2 w[8];
#pragma unroll
                for (int dy = 0; dy < 8; ++dy)
                    w[dy] = y0 + dy < y1 ? __ldg(reinterpret_cast<const uint2 *>(col + (size_t)dy * pitch))
                                         : make_uint2(0u, 0u);
#pragma unroll
                for (int dy = 0; dy < 8; ++dy) sum = __vsadu4(w[dy].x, 0u) + __vsadu4(w[dy].y, 0u) + sum;
            } else {
                for (int y = y0; y < y1; ++y) {
                    const uint8_t *row = raw + (size_t)y * pitch;
                    for (int x = x0; x < x1; ++x) sum += row[x];
                }
            }
            v = (float)sum / (float)((y1 - y0) * (x1 - x0)) / 255.0f - 0.5f;
        }
        X[i] = v;
    }
    __syncthreads();

    // A1: im2col of X, row r = the 9 taps of X around grid row r (K padded to 16)
    for (int r = threadIdx.x; r < kR1; r += kSkipThreads) {
        float t[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) t[k] = X[r + (k / 3) * kSkipP + (k % 3)];
        *reinterpret_cast<uint4 *>(U + 16 * r) =
            make_uint4(pack_bf16(t[0], t[1]), pack_bf16(t[2], t[3]), pack_bf16(t[4], t[5]), pack_bf16(t[6], t[7]));
        *reinterpret_cast<uint4 *>(U + kChunk1 + 16 * r) = make_uint4(pack_bf16(t[8], 0.0f), 0u, 0u, 0u);
    }
    sync_for_mma();
    const uint32_t tmem = *tmem_slot;
    const uint32_t bar_a = saddr_of(bar);
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;  // this warp's TMEM lane quarter
    uint32_t phase = 0;
    bool ok;

    // Completion of one layer's MMAs (issued by thread 0) through the
    // mbarrier.  On a timeout the error is flagged and, after a second
    // bounded wait for MMAs still in flight, the CTA frees TMEM and stops.
    auto finish_layer = [&]() -> bool {
        if (threadIdx.x == 0) {
            mma_commit(bar_a);
            const bool done = bar_wait(bar_a, phase);
            if (!done) {
                atomicOr(b.err, kErrTimeout);
                bar_wait(bar_a, phase);
            }
            s_ok = done ? 1 : 0;
        }
        __syncthreads();
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        return s_ok != 0;
    };

    // ---- layer 1: A1 (im2col) x B1 -> TMEM columns 16 j
    if (threadIdx.x == 0) {
        const uint64_t bd = smem_desc(saddr_of(B1), 256, 128);
        for (int j = 0; j < kT1; ++j)
            mma_bf16(tmem + 16 * j, smem_desc(saddr_of(U + j * kMmaM * 16), kChunk1, 128), bd, false);
    }
    ok = finish_layer();
    if (ok) {
        // a1 at grid row r is 1/8-map position (ty0 - 2 + y, tx0 - 2 + x);
        // columns x >= P - 2 are wrapped rows
        for (int j = warp >> 2; j < kT1; j += 2) {
            float acc[16];
            tmem_ld16(tmem + lane_base + 16 * j, acc);
            const int r = j * kMmaM + 32 * (warp & 3) + lane;
            const int y = r / kSkipP, x = r - y * kSkipP;
            const int gy = ty0 - 2 + y, gx = tx0 - 2 + x;
            const bool keep = x < kSkipP - 2 && gy >= 0 && gy < H8 && gx >= 0 && gx < W8;
            store_act(A1g, kChunk1, r, acc, bias, keep);
        }
        sync_for_mma();

        // ---- layer 2: 9 shifted views of a1 x B2[t] -> TMEM columns 16 j
        if (threadIdx.x == 0) {
            for (int j = 0; j < kT2; ++j)
                for (int t = 0; t < 9; ++t) {
                    const int s = (t / 3) * kSkipP + (t % 3);
                    mma_bf16(tmem + 16 * j, smem_desc(saddr_of(A1g + (j * kMmaM + s) * 16), kChunk1, 128),
                             smem_desc(saddr_of(B2 + t * 256), 256, 128), t > 0);
                }
        }
        ok = finish_layer();
    }
    if (ok) {
        // a2 (where A1 was) at (ty0 - 1 + y, tx0 - 1 + x); columns x >= P - 4 wrapped
        for (int j = warp >> 2; j < kT2; j += 2) {
            float acc[16];
            tmem_ld16(tmem + lane_base + 16 * j, acc);
            const int r = j * kMmaM + 32 * (warp & 3) + lane;
            const int y = r / kSkipP, x = r - y * kSkipP;
            const int gy = ty0 - 1 + y, gx = tx0 - 1 + x;
            const bool keep = x < kSkipP - 4 && gy >= 0 && gy < H8 && gx >= 0 && gx < W8;
            store_act(U, kChunk2, r, acc, bias + 16, keep);
        }
        sync_for_mma();

        // ---- layer 3: 9 shifted views of a2 x B3[t] -> TMEM column 16 j holds the logit
        if (threadIdx.x == 0) {
            for (int j = 0; j < kT3; ++j)
                for (int t = 0; t < 9; ++t) {
                    const int s = (t / 3) * kSkipP + (t % 3);
                    mma_bf16(tmem + 16 * j, smem_desc(saddr_of(U + (j * kMmaM + s) * 16), kChunk2, 128),
                             smem_desc(saddr_of(B3 + t * 256), 256, 128), t > 0);
                }
        }
        ok = finish_layer();
    }
    if (ok) {
        for (int j = warp >> 2; j < kT3; j += 2) {
            const float acc = tmem_ld1(tmem + lane_base + 16 * j);
            const int r = j * kMmaM + 32 * (warp & 3) + lane;
            const int y = r / kSkipP, x = r - y * kSkipP;
            const int gy = ty0 + y, gx = tx0 + x;
            if (x < kSkipTW && gy < H8 && gx < W8) I.skip_logits[(size_t)gy * W8 + gx] = acc + bias[32];
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

__global__ void k_skipcells(Batch b, float thresh)
{
    const int img = blockIdx.y;
    const ImageDesc &I = b.images[img];
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= I.skip_cells_x * I.skip_cells_y) return;
    const int cy = cell / I.skip_cells_x, cx = cell - cy * I.skip_cells_x;
    const int c0 = I.skip_c0;
    // 1/8-map block of the s0 cell [cx c0, (cx + 1) c0) x [cy c0, (cy + 1) c0)
    const int x0 = (cx * c0) / 8, x1 = min(((cx + 1) * c0 + 7) / 8, I.skip_w8);
    const int y0 = (cy * c0) / 8, y1 = min(((cy + 1) * c0 + 7) / 8, I.skip_h8);
    float best = -INFINITY;
    for (int y = y0; y < y1; ++y)
        for (int x = x0; x < x1; ++x) best = fmaxf(best, I.skip_logits[(size_t)y * I.skip_w8 + x]);
    I.skip[cell] = best < thresh ? 1 : 0;
    if (best < thresh) atomicOr(b.skip_any + img, 1);  // zeroed before the launch
}

int skipnet_smem_bytes() { return kSkipSmem; }

cudaError_t launch_skipnet(const Batch &b, const SkipModelDev &m, float thresh, cudaStream_t stream)
{
    if (b.n_images == 0 || b.skip_max_tiles == 0) return cudaSuccess;
    dim3 grid(b.skip_max_tiles, b.n_images);
    k_skipnet<<<grid, kSkipThreads, kSkipSmem, stream>>>(b, m);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(b.skip_any, 0, sizeof(int32_t) * (size_t)b.n_images, stream)) != cudaSuccess) return e;
    dim3 g2((b.skip_max_cells + 255) / 256, b.n_images);
    k_skipcells<<<g2, 256, 0, stream>>>(b, thresh);
    return cudaGetLastError();
}

cudaError_t configure_skipnet()
{
    return cudaFuncSetAttribute(k_skipnet, cudaFuncAttributeMaxDynamicSharedMemorySize, kSkipSmem);
}

}  // namespace jslam
