// Learned cell-skip proposal: an opt-in approximate mode on top of the exact
// path (the paper has no counterpart; its exact path stays the fallback and
// the judge of the proposal).
//
// k_skipnet    one CTA per 14x14 block of the 1/8-scale logit map of an
//              image: box-averages 8x8 blocks of level 0 (normalised to
//              [-0.5, 0.5]), then three 3x3 convolutions with zero padding
//              (1 -> 16 -> 16 -> 1 channels, ReLU between), BF16 weights
//              widened to FP32, FP32 accumulation, all in shared memory.
// k_skipcells  one thread per s0 culling cell: the cell is skipped when the
//              largest logit over its block of the 1/8 map is below the
//              threshold.  The detection kernel then ignores every cell of
//              any level whose centre projects into a skipped s0 cell.
#include "jslam_internal.h"

namespace jslam {

// 14 x 14 logits per CTA: the second layer's 16 x 16 positions (one-deep
// halo) then fill the 256 threads exactly once; that layer holds 90 % of the
// arithmetic.
constexpr int kSkipT = kSkipTile;
constexpr int kSkipIn = kSkipT + 6;          // box-mean input with a 3-deep halo
constexpr int kSkipA1 = kSkipT + 4;          // first activation with a 2-deep halo
constexpr int kSkipA2 = kSkipT + 2;          // second activation with a 1-deep halo
constexpr int kSkipThreads = 256;

struct SkipSmem {
    float in[kSkipIn][kSkipIn];
    float a1[kSkipC][kSkipA1][kSkipA1];
    float a2[kSkipC][kSkipA2][kSkipA2];
    float w1[kSkipC][9];
    float w2t[kSkipC][9][kSkipC];  // [in channel][tap][out channel]: 16 outputs per broadcast load
    float w3[kSkipC][9];
    float b1[kSkipC], b2[kSkipC], b3;
};

__device__ __forceinline__ float bf16_to_f32(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }

__global__ void __launch_bounds__(kSkipThreads) k_skipnet(Batch b, const SkipModelDev m)
{
    extern __shared__ __align__(16) uint8_t smem_raw[];
    SkipSmem &s = *reinterpret_cast<SkipSmem *>(smem_raw);
    const int img = blockIdx.y;
    const ImageDesc &I = b.images[img];
    const int W8 = I.skip_w8, H8 = I.skip_h8;
    const int tiles_x = (W8 + kSkipT - 1) / kSkipT;
    const int tile = blockIdx.x;
    if (tile >= tiles_x * ((H8 + kSkipT - 1) / kSkipT)) return;
    const int tx0 = (tile % tiles_x) * kSkipT, ty0 = (tile / tiles_x) * kSkipT;
    const LevelDesc &L0 = b.levels[I.level_base];
    const uint8_t *raw = L0.raw;
    const int pitch = L0.pitch, W0 = I.W0, H0 = I.H0;

    // weights (BF16 -> FP32) and biases
    for (int i = threadIdx.x; i < kSkipC * 9; i += kSkipThreads) {
        s.w1[i / 9][i % 9] = bf16_to_f32(m.w1[i]);
        s.w3[i / 9][i % 9] = bf16_to_f32(m.w3[i]);
    }
    for (int i = threadIdx.x; i < kSkipC * kSkipC * 9; i += kSkipThreads) {
        const int co = i / (kSkipC * 9), ci = (i / 9) % kSkipC, k = i % 9;  // source layout [co][ci][k]
        s.w2t[ci][k][co] = bf16_to_f32(m.w2[i]);
    }
    if (threadIdx.x < kSkipC) { s.b1[threadIdx.x] = m.b1[threadIdx.x]; s.b2[threadIdx.x] = m.b2[threadIdx.x]; }
    if (threadIdx.x == 0) s.b3 = m.b3;

    // box means of 8x8 level-0 blocks; zero outside the 1/8 map (padding).
    // Rows of the aligned level-0 copy are read 8 bytes at a time.
    for (int i = threadIdx.x; i < kSkipIn * kSkipIn; i += kSkipThreads) {
        const int iy = i / kSkipIn, ix = i - iy * kSkipIn;
        const int gy = ty0 - 3 + iy, gx = tx0 - 3 + ix;
        float v = 0.0f;
        if (gy >= 0 && gy < H8 && gx >= 0 && gx < W8) {
            const int y0 = 8 * gy, x0 = 8 * gx;
            const int y1 = min(y0 + 8, H0), x1 = min(x0 + 8, W0);
            uint32_t sum = 0;
            if (x1 - x0 == 8) {
                for (int y = y0; y < y1; ++y) {
                    const uint2 w = __ldg(reinterpret_cast<const uint2 *>(raw + (size_t)y * pitch + x0));
                    sum = __vsadu4(w.x, 0u) + __vsadu4(w.y, 0u) + sum;
                }
            } else {
                for (int y = y0; y < y1; ++y) {
                    const uint8_t *row = raw + (size_t)y * pitch;
                    for (int x = x0; x < x1; ++x) sum += row[x];
                }
            }
            v = (float)sum / (float)((y1 - y0) * (x1 - x0)) / 255.0f - 0.5f;
        }
        s.in[iy][ix] = v;
    }
    __syncthreads();

    // layer 1: 1 -> 16, ReLU; one position per thread, all 16 channels
    for (int p = threadIdx.x; p < kSkipA1 * kSkipA1; p += kSkipThreads) {
        const int y = p / kSkipA1, x = p - y * kSkipA1;
        const int gy = ty0 - 2 + y, gx = tx0 - 2 + x;
        const bool inside = gy >= 0 && gy < H8 && gx >= 0 && gx < W8;
        float in9[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) in9[k] = s.in[y + k / 3][x + k % 3];
#pragma unroll
        for (int c = 0; c < kSkipC; ++c) {
            float acc = s.b1[c];
#pragma unroll
            for (int k = 0; k < 9; ++k) acc = fmaf(s.w1[c][k], in9[k], acc);
            s.a1[c][y][x] = inside ? fmaxf(acc, 0.0f) : 0.0f;
        }
    }
    __syncthreads();

    // layer 2: 16 -> 16, ReLU; one position per thread, every input loaded once
    for (int p = threadIdx.x; p < kSkipA2 * kSkipA2; p += kSkipThreads) {
        const int y = p / kSkipA2, x = p - y * kSkipA2;
        const int gy = ty0 - 1 + y, gx = tx0 - 1 + x;
        float acc[kSkipC];
#pragma unroll
        for (int c = 0; c < kSkipC; ++c) acc[c] = s.b2[c];
        for (int ci = 0; ci < kSkipC; ++ci) {
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const float a = s.a1[ci][y + k / 3][x + k % 3];
#pragma unroll
                for (int c = 0; c < kSkipC; ++c) acc[c] = fmaf(s.w2t[ci][k][c], a, acc[c]);
            }
        }
        const bool inside = gy >= 0 && gy < H8 && gx >= 0 && gx < W8;
#pragma unroll
        for (int c = 0; c < kSkipC; ++c) s.a2[c][y][x] = inside ? fmaxf(acc[c], 0.0f) : 0.0f;
    }
    __syncthreads();

    // layer 3: 16 -> 1, the logit
    for (int p = threadIdx.x; p < kSkipT * kSkipT; p += kSkipThreads) {
        const int y = p / kSkipT, x = p - y * kSkipT;
        const int gy = ty0 + y, gx = tx0 + x;
        if (gy >= H8 || gx >= W8) continue;
        float acc = s.b3;
        for (int ci = 0; ci < kSkipC; ++ci) {
#pragma unroll
            for (int k = 0; k < 9; ++k) acc = fmaf(s.w3[ci][k], s.a2[ci][y + k / 3][x + k % 3], acc);
        }
        I.skip_logits[(size_t)gy * W8 + gx] = acc;
    }
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
}

int skipnet_smem_bytes() { return (int)sizeof(SkipSmem); }

cudaError_t launch_skipnet(const Batch &b, const SkipModelDev &m, float thresh, cudaStream_t stream)
{
    if (b.n_images == 0 || b.skip_max_tiles == 0) return cudaSuccess;
    dim3 grid(b.skip_max_tiles, b.n_images);
    k_skipnet<<<grid, kSkipThreads, sizeof(SkipSmem), stream>>>(b, m);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 g2((b.skip_max_cells + 255) / 256, b.n_images);
    k_skipcells<<<g2, 256, 0, stream>>>(b, thresh);
    return cudaGetLastError();
}

cudaError_t configure_skipnet()
{
    return cudaFuncSetAttribute(k_skipnet, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SkipSmem));
}

}  // namespace jslam
