// Feature Culling the way the paper's kernels do it (Sec. II-C-1), kept as
// an ablation baseline beside the fused detection kernel, which culls
// inside detection with shared-memory atomics and never writes a CRF-matrix.
//
// k_crf      one thread per pixel of every level of every image: Eq. 1-3 at
//            the primary threshold (corner table of Sec. III in global
//            memory) and the SAD response; writes the CRF-matrix (response
//            of corners, 0 elsewhere and in the border) as uint16.
// k_fc_mlpt  per level: Multi-Location-Per-Thread culling under
//            Thread-Efficient Warp Allocation.  A block is 128 threads wide
//            (as many whole cells as fit side by side, one thread per cell
//            column) and N_t = ceil(c / N_max) threads tall.  Vertical pass:
//            thread (x, y) takes N_max consecutive rows of its column and the
//            first thread of the column reduces the N_t partial maxima;
//            horizontal pass: the first N_t threads of a cell each take the
//            cell's columns at a stride of N_t and the cell's first thread
//            reduces them.  The maximum is taken over the key
//            response << 16 | (0xFFFF - index in cell) (0 for no corner), so
//            ties resolve as in the fused kernel and the oracle.
#include "jslam_internal.h"
#include "ring_response.cuh"

namespace jslam {

constexpr int kTewaX = 128;
constexpr int kTewaMaxNt = 8;   // 128 x 8 = 1024 threads per block at most

__global__ void __launch_bounds__(256) k_crf(Batch b, uint16_t *crf, const uint64_t *off)
{
    const int li = blockIdx.y;
    const LevelDesc &L = b.levels[li];
    const ImageDesc &I = b.images[L.image];
    const int W = L.W, H = L.H;
    const int pix = blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= W * H) return;
    const int y = pix / W, x = pix - y * W;
    const int border = b.prm.border, eps = I.eps_hi;
    uint16_t out = 0;
    if (x >= border && x < W - border && y >= border && y < H - border) {
        constexpr int DX[16] = { 0, 1, 2, 3, 3, 3, 2, 1, 0, -1, -2, -3, -3, -3, -2, -1 };
        constexpr int DY[16] = { 3, 3, 2, 1, 0, -1, -2, -3, -3, -3, -2, -1, 0, 1, 2, 3 };
        const uint8_t *p = L.raw + (size_t)y * L.pitch + x;
        const int ic = p[0];
        uint32_t mb = 0, md = 0;
        int r = 0;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int d = (int)p[DY[q] * L.pitch + DX[q]] - ic;
            mb |= (uint32_t)(d > eps) << q;
            md |= (uint32_t)(d < -eps) << q;
            r += abs(d);
        }
        const uint32_t cb = (__ldg(b.corner_lut + (mb >> 5)) >> (mb & 31)) & 1u;
        const uint32_t cd = (__ldg(b.corner_lut + (md >> 5)) >> (md & 31)) & 1u;
        if (cb | cd) out = (uint16_t)(b.prm.resp_arc ? ring_arc(p, L.pitch, eps, b.prm.p_min, b.prm.p_max) : r);
    }
    crf[off[li] + pix] = out;
}

// grid: (blocks across a cell row, cell rows, images); block (128, N_t)
__global__ void k_fc_mlpt(Batch b, const uint16_t *crf, const uint64_t *off, uint32_t *keys, int level, int n_max)
{
    __shared__ uint32_t part[kTewaMaxNt][kTewaX];   // N_t rows of partial column maxima
    __shared__ uint32_t colmax[kTewaX];
    const int img = blockIdx.z;
    const ImageDesc &I = b.images[img];
    if (level >= I.levels) return;
    const int li = I.level_base + level;
    const LevelDesc &L = b.levels[li];
    const int c = L.c, W = L.W, H = L.H;
    const int cpb = kTewaX / c;                       // cells per block (TEWA)
    const int nt = (c + n_max - 1) / n_max;           // threads per column
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int lc = tx / c, col = tx - lc * c;        // cell within the block, column within the cell
    const int cx = blockIdx.x * cpb + lc, cy = blockIdx.y;
    const bool active = tx < cpb * c && cx < L.cells_x && cy < L.cells_y && ty < nt;
    const uint16_t *m = crf + off[li];
    // vertical: rows [ty n_max, (ty + 1) n_max) of the column
    uint32_t best = 0;
    if (active) {
        const int x = cx * c + col;
        const int r1 = min((ty + 1) * n_max, c);
        for (int r = ty * n_max; r < r1; ++r) {
            const int y = cy * c + r;
            if (x < W && y < H) {
                const uint32_t v = m[(size_t)y * W + x];
                const uint32_t key = v ? (v << 16) | (0xFFFFu - (uint32_t)(r * c + col)) : 0u;
                best = max(best, key);
            }
        }
    }
    part[ty][tx] = best;
    __syncthreads();
    if (ty == 0) {
        uint32_t v = 0;
        for (int t = 0; t < nt && t < (int)blockDim.y; ++t) v = max(v, part[t][tx]);
        colmax[tx] = v;
    }
    __syncthreads();
    // horizontal: the first nt threads of the cell take its columns at a stride of nt
    if (ty == 0) {
        uint32_t v = 0;
        if (active && col < nt)
            for (int j = col; j < c; j += nt) v = max(v, colmax[lc * c + j]);
        part[0][tx] = v;
    }
    __syncthreads();
    if (ty == 0 && active && col == 0) {
        uint32_t v = 0;
        for (int t = 0; t < nt && t < c; ++t) v = max(v, part[0][lc * c + t]);
        keys[L.slot_base + cy * L.cells_x + cx] = v;
    }
}

cudaError_t launch_fc_ablation(const Batch &b, uint16_t *crf, const uint64_t *off, uint32_t *keys,
                               const int *level_blocks, int max_pixels, int max_levels, const int *level_cells_y,
                               const int *level_c, int n_max, cudaStream_t stream, cudaEvent_t mid)
{
    if (b.n_levels == 0) return cudaSuccess;
    dim3 g1((max_pixels + 255) / 256, b.n_levels);
    k_crf<<<g1, 256, 0, stream>>>(b, crf, off);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (mid && (e = cudaEventRecord(mid, stream)) != cudaSuccess) return e;
    for (int l = 0; l < max_levels; ++l) {
        const int c = level_c[l];
        const int nt = (c + n_max - 1) / n_max;
        dim3 block(kTewaX, nt);
        dim3 grid(level_blocks[l], level_cells_y[l], b.n_images);
        k_fc_mlpt<<<grid, block, 0, stream>>>(b, crf, off, keys, l, n_max);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace jslam
