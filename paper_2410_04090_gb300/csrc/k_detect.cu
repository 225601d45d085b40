// Detection stage: image pyramid with Gaussian filtering, then FAST with
// Bounded Rectification, per-cell culling and the scatter half of PFA.
//
// k_pyramid   one CTA per 128x32 output tile of any (image, level): resamples
//             the level from level 0 (bilinear, Q8 taps from host tables),
//             writes it (level 0: an aligned copy of the input), and writes its
//             7-tap Gaussian (Sec. III, streamlined multiscale detection and
//             extraction: Gaussian filtering before ORB).
// k_fast_cull persistent CTAs over blocks of culling cells of any (image,
//             level): stage the raw tile plus its halo in shared memory (TMA),
//             evaluate the 16-pixel ring of every pixel (Sec. II-A, Eq. 1 labels, Eq. 3
//             bounded run length; Sec. III bit masks and SAD response), keeps
//             the top-k corners of each cell (Sec. II-C-1, Feature Culling)
//             and adds each survivor to the s0 score map (Sec. II-C-2, PFA
//             steps 1-2: K_l and K_r accumulate in one packed word).
// k_fast_bits the same results for run bounds [9, 13] (the default): the tile
//             is transposed into bit-planes and each thread tests 32 pixels
//             of a row at once with bitwise arithmetic (carry-chain compares,
//             run windows), scoring its corners in place; tiles come with
//             host-made records staged by bulk copies.
#include <algorithm>

#include <cuda.h>

#include "jslam_internal.h"
#include "ring_response.cuh"

namespace jslam {

__constant__ int32_t c_blur_w[7];
// The same weights as bytes for the 2-way dot products of the horizontal
// pass: {0, w0, w1, w2}, {w3, w4, w5, w6}, {w0, w1, w2, w3}, {w4, w5, w6, 0}
// (byte 0 first; every weight is below 256).
__constant__ uint32_t c_blur_pk[4];

cudaError_t set_blur_weights(const int32_t w[7])
{
    cudaError_t e = cudaMemcpyToSymbol(c_blur_w, w, sizeof(int32_t) * 7);
    if (e != cudaSuccess) return e;
    const auto B = [](int b0, int b1, int b2, int b3) {
        return (uint32_t)b0 | ((uint32_t)b1 << 8) | ((uint32_t)b2 << 16) | ((uint32_t)b3 << 24);
    };
    const uint32_t pk[4] = { B(0, w[0], w[1], w[2]), B(w[3], w[4], w[5], w[6]), B(w[0], w[1], w[2], w[3]),
                             B(w[4], w[5], w[6], 0) };
    return cudaMemcpyToSymbol(c_blur_pk, pk, sizeof(pk));
}

// ---------------------------------------------------------------- pyramid
//
// Per 128x32 output tile: the raw level over the tile plus a halo (3 rows, 4
// columns) is built in shared memory -- level 0 is copied from the input,
// deeper levels are resampled from level 0 separably and exactly: every
// needed source row is interpolated horizontally once ((256-a) p0 + a p1,
// exact in 16 bits), then pairs of those rows vertically with rounding.
// The raw interior is written to the level buffer (level 0 included: an
// aligned copy of the input).  The 7-tap Gaussian runs vertically first on
// bytes in 16-bit lanes (two pixels per multiply; the symmetric taps need 3
// adds and 4 multiplies), then horizontally on the 16-bit column sums.

constexpr int kPyrCols = kPyrTW + 8;         // raw tile columns: x in [x0 - 4, x0 + 132)
constexpr int kPyrRows = kPyrTH + 6;         // raw tile rows: y in [y0 - 3, y0 + 35)
constexpr int kPyrSrcRows = 2 * kPyrRows;    // level-0 rows interpolated per tile, at most

__device__ __forceinline__ uint32_t blur7_sym(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t a4,
                                              uint32_t a5, uint32_t a6)
{
    return c_blur_w[0] * (a0 + a6) + c_blur_w[1] * (a1 + a5) + c_blur_w[2] * (a2 + a4) + c_blur_w[3] * a3;
}

__global__ void __launch_bounds__(kPyrThreads) k_pyramid(Batch b)
{
    __shared__ __align__(16) uint8_t raw[kPyrRows][kPyrCols];
    __shared__ __align__(16) uint16_t V[kPyrTH][kPyrCols];
    __shared__ __align__(16) uint16_t Hs[kPyrSrcRows][kPyrCols];
    __shared__ uint32_t tx[kPyrCols];
    __shared__ int src_row[kPyrSrcRows];
    __shared__ uint8_t ia[kPyrRows], ib[kPyrRows];
    __shared__ uint16_t wb[kPyrRows];
    __shared__ int s_ya[kPyrRows];
    __shared__ int nsrc;

    const int tile = b.pyr_pass < 0 ? (int)blockIdx.x : __ldg(b.pyr_order + b.pyr_pass_first[b.pyr_pass] + blockIdx.x);
    const int li = __ldg(b.pyr_tile_level + tile);
    const LevelDesc &L = b.levels[li];
    const ImageDesc &I = b.images[L.image];
    const int t = tile - b.pyr_tile_base[li];
    const int tiles_x = (L.W + kPyrTW - 1) / kPyrTW;
    const int x0 = (t % tiles_x) * kPyrTW, y0 = (t / tiles_x) * kPyrTH;
    // level 0 reads the input; deeper levels resample the input, or in the
    // cascaded pyramid the level above (complete: an earlier launch)
    const uint8_t *L0 = L.src ? L.src : b.in.ptr[L.image];
    const int W0 = L.src ? L.src_W : I.W0, H0 = L.src ? L.src_H : I.H0;
    const int pitch0 = L.src ? L.src_pitch : b.in.pitch[L.image];
    const int W = L.W, H = L.H;
    constexpr int WPR = kPyrCols / 4;

    if (L.level == 0) {
        for (int i = threadIdx.x; i < kPyrRows * WPR; i += kPyrThreads) {
            const int r = i / WPR, w = i - r * WPR;
            const uint8_t *row = L0 + (size_t)min(max(y0 - 3 + r, 0), H - 1) * pitch0;
            const int gx = x0 - 4 + 4 * w;
            uint32_t v;
            if (gx >= 0 && gx + 3 < W) {
                // the two aligned words holding bytes gx .. gx + 3 (each holds
                // at least one byte of the row, so neither leaves the buffer)
                const uintptr_t a = reinterpret_cast<uintptr_t>(row + gx);
                const uint32_t *p = reinterpret_cast<const uint32_t *>(a & ~static_cast<uintptr_t>(3));
                const uint32_t sh = (uint32_t)(a & 3u) * 8u;
                v = sh ? __funnelshift_r(__ldg(p), __ldg(p + 1), sh) : __ldg(p);
            } else {
                v = 0;
#pragma unroll
                for (int q = 0; q < 4; ++q) v |= (uint32_t)__ldg(row + min(max(gx + q, 0), W - 1)) << (8 * q);
            }
            *reinterpret_cast<uint32_t *>(&raw[r][4 * w]) = v;
        }
    } else {
        for (int c = threadIdx.x; c < kPyrCols; c += kPyrThreads)
            tx[c] = __ldg(L.tapx + min(max(x0 - 4 + c, 0), W - 1));
        if (threadIdx.x < kPyrRows) {
            const uint32_t ty = __ldg(L.tapy + min(max(y0 - 3 + (int)threadIdx.x, 0), H - 1));
            s_ya[threadIdx.x] = ty & 0xFFFF;
            wb[threadIdx.x] = (uint16_t)(ty >> 16);
        }
        __syncthreads();
        // level-0 rows needed by the tile's raw rows: a contiguous range when
        // it is short enough, else two rows per raw row
        const int first = s_ya[0], last = min(s_ya[kPyrRows - 1] + 1, H0 - 1);
        const bool contiguous = last - first + 1 <= kPyrSrcRows;
        if (threadIdx.x < kPyrRows) {
            const int r = threadIdx.x, ya = s_ya[r], yb = min(ya + 1, H0 - 1);
            ia[r] = (uint8_t)(contiguous ? ya - first : 2 * r);
            ib[r] = (uint8_t)(contiguous ? yb - first : 2 * r + 1);
        }
        const int nrows = contiguous ? last - first + 1 : kPyrSrcRows;
        for (int j = threadIdx.x; j < nrows; j += kPyrThreads)
            src_row[j] = contiguous ? first + j : ((j & 1) ? min(s_ya[j >> 1] + 1, H0 - 1) : s_ya[j >> 1]);
        if (threadIdx.x == 0) nsrc = nrows;
        __syncthreads();
        const int ns = nsrc;
        // horizontal interpolation: a thread owns 4 adjacent columns, keeps
        // their taps in registers and walks the source rows
        constexpr int kQuads = kPyrCols / 4, kRowSlots = kPyrThreads / kQuads;
        const int q = threadIdx.x % kQuads, slot = threadIdx.x / kQuads;
        if (slot < kRowSlots) {
            int xa[4], xb[4];
            uint32_t wa[4], wbx[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t tp = tx[4 * q + k];
                xa[k] = tp & 0xFFFF;
                xb[k] = min(xa[k] + 1, W0 - 1);
                wbx[k] = tp >> 16;
                wa[k] = 256u - wbx[k];
            }
            for (int j = slot; j < ns; j += kRowSlots) {
                // 32-bit offsets from the image's base (images are below 4 GB)
                const uint32_t ro = (uint32_t)src_row[j] * (uint32_t)pitch0;
                uint32_t h[4];
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    h[k] = wa[k] * __ldg(L0 + (ro + (uint32_t)xa[k])) + wbx[k] * __ldg(L0 + (ro + (uint32_t)xb[k]));
                *reinterpret_cast<uint2 *>(&Hs[j][4 * q]) = make_uint2(h[0] | (h[1] << 16), h[2] | (h[3] << 16));
            }
        }
        __syncthreads();
        // vertical interpolation, 4 columns per thread (16-bit taps read as words)
        for (int i = threadIdx.x; i < kPyrRows * (kPyrCols / 4); i += kPyrThreads) {
            const int r = i / (kPyrCols / 4), q = i - r * (kPyrCols / 4);
            const uint32_t w = wb[r], w0 = 256u - w;
            const uint2 ha = *reinterpret_cast<const uint2 *>(&Hs[ia[r]][4 * q]);
            const uint2 hb = *reinterpret_cast<const uint2 *>(&Hs[ib[r]][4 * q]);
            // rounded sums below 2^24: the result is byte 2 of each, packed by byte permutes
            const uint32_t v0 = w0 * (ha.x & 0xFFFFu) + w * (hb.x & 0xFFFFu) + 32768u;
            const uint32_t v1 = w0 * (ha.x >> 16) + w * (hb.x >> 16) + 32768u;
            const uint32_t v2 = w0 * (ha.y & 0xFFFFu) + w * (hb.y & 0xFFFFu) + 32768u;
            const uint32_t v3 = w0 * (ha.y >> 16) + w * (hb.y >> 16) + 32768u;
            *reinterpret_cast<uint32_t *>(&raw[r][4 * q]) =
                __byte_perm(__byte_perm(v0, v1, 0x0062), __byte_perm(v2, v3, 0x0062), 0x5410);
        }
    }
    __syncthreads();

    // raw interior -> level buffer (whole words; the row pitch covers the tile)
    for (int i = threadIdx.x; i < kPyrTH * (kPyrTW / 4); i += kPyrThreads) {
        const int r = i / (kPyrTW / 4), w = i - r * (kPyrTW / 4);
        const int gy = y0 + r, gx = x0 + 4 * w;
        if (gy < H && gx < W)
            *reinterpret_cast<uint32_t *>(L.raw_w + (size_t)gy * L.pitch + gx) =
                *reinterpret_cast<const uint32_t *>(&raw[r + 3][4 * w + 4]);
    }
    // vertical 7-tap sums, two pixels per 32-bit lane pair: a thread owns one
    // word column and slides a 7-row window down a run of rows
    {
        constexpr int kSegs = kPyrThreads / WPR, kRun = (kPyrTH + kSegs - 1) / kSegs;
        const int w = threadIdx.x % WPR, seg = threadIdx.x / WPR;
        if (seg < kSegs) {
            const int r0 = seg * kRun;
            uint32_t e[7], o[7];
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                const uint32_t x = *reinterpret_cast<const uint32_t *>(&raw[min(r0 + j, kPyrRows - 1)][4 * w]);
                e[j] = x & 0x00FF00FFu;
                o[j] = (x >> 8) & 0x00FF00FFu;
            }
#pragma unroll
            for (int k = 0; k < kRun; ++k) {
                const int r = r0 + k;
                if (r < kPyrTH) {
                    const uint32_t x = *reinterpret_cast<const uint32_t *>(&raw[r + 6][4 * w]);
                    e[6] = x & 0x00FF00FFu;
                    o[6] = (x >> 8) & 0x00FF00FFu;
                    const uint32_t se = blur7_sym(e[0], e[1], e[2], e[3], e[4], e[5], e[6]);
                    const uint32_t so = blur7_sym(o[0], o[1], o[2], o[3], o[4], o[5], o[6]);
                    *reinterpret_cast<uint2 *>(&V[r][4 * w]) =
                        make_uint2(__byte_perm(se, so, 0x5410), __byte_perm(se, so, 0x7632));
                }
#pragma unroll
                for (int j = 0; j < 6; ++j) { e[j] = e[j + 1]; o[j] = o[j + 1]; }
            }
        }
    }
    __syncthreads();
    // horizontal 7-tap on the column sums: a thread owns a row and a run of
    // 4 quads (16 output pixels).  The 16-bit sums sit two to a word (word i:
    // columns 2i, 2i + 1 of the run), so each output is four 2-way byte dot
    // products over aligned words, with the weights packed for its parity
    // (the same integer sum as the 7 products; one rounding at the end).
    {
        constexpr int kQuadRun = 4, kRunsPerRow = (kPyrTW / 4) / kQuadRun;
        static_assert(kPyrTH * kRunsPerRow == kPyrThreads, "one run per thread");
        const int r = threadIdx.x / kRunsPerRow, q0 = (threadIdx.x % kRunsPerRow) * kQuadRun;
        const int gy = y0 + r;
        const uint32_t *src = reinterpret_cast<const uint32_t *>(&V[r][4 * q0]);
        const uint32_t A = c_blur_pk[0], Bw = c_blur_pk[1], Cw = c_blur_pk[2], Dw = c_blur_pk[3];
        uint32_t u[2 * kQuadRun + 4];
#pragma unroll
        for (int j = 0; j < 2 * kQuadRun + 4; ++j) u[j] = src[j];
#pragma unroll
        for (int k = 0; k < kQuadRun; ++k) {
            // output m of the quad reads columns 4 k + m + 1 .. 4 k + m + 7
            const uint32_t *w = u + 2 * k;
            // words i .. i + 3 against the weight words P (first two) and Q (last
            // two); the rounding term starts each sum, the sums stay below 2^24,
            // so each result is byte 2 of its sum, packed by byte permutes
            const auto dot7 = [&](int i, uint32_t P, uint32_t Q) {
                const uint32_t lo = __dp2a_hi(w[i + 1], P, __dp2a_lo(w[i], P, 32768u));
                return __dp2a_hi(w[i + 3], Q, __dp2a_lo(w[i + 2], Q, lo));
            };
            const uint32_t s0 = dot7(0, A, Bw), s1 = dot7(1, Cw, Dw), s2 = dot7(1, A, Bw), s3 = dot7(2, Cw, Dw);
            const uint32_t out = __byte_perm(__byte_perm(s0, s1, 0x0062), __byte_perm(s2, s3, 0x0062), 0x5410);
            const int gx = x0 + 4 * (q0 + k);
            if (gy < H && gx < W) *reinterpret_cast<uint32_t *>(L.blur + (size_t)gy * L.blur_pitch + gx) = out;
        }
    }
}

const void *pyramid_kernel() { return reinterpret_cast<const void *>(k_pyramid); }

cudaError_t launch_pyramid(const Batch &b, cudaStream_t stream)
{
    if (b.pyr_tiles == 0) return cudaSuccess;
    if (b.pyr_pass < 0) {
        k_pyramid<<<b.pyr_tiles, kPyrThreads, 0, stream>>>(b);
        return cudaGetLastError();
    }
    // cascaded: level number n after n - 1, each launch over every image
    for (int n = 0; n < kMaxLevels; ++n) {
        const int tiles = b.pyr_pass_first[n + 1] - b.pyr_pass_first[n];
        if (tiles == 0) continue;
        Batch bn = b;
        bn.pyr_pass = n;
        k_pyramid<<<tiles, kPyrThreads, 0, stream>>>(bn);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------- FAST + FC
//
// One persistent CTA loops over detection tiles (a block of whole culling
// cells of any image and level).  The raw tile plus its halo is fetched by
// TMA (one 2-D tensor map per level) into one of two shared-memory buffers
// while the CTA works on the other, with an mbarrier per buffer.  Per tile:
//   1. primary threshold: every thread classifies 4 horizontally adjacent
//      pixels at once (one 32-bit word of centres).  (a) Cardinal pre-test:
//      the ring positions 0, 4, 8, 12 are compared with the 4 per-pixel
//      thresholds by byte-wise carries (no carry crosses a byte); groups
//      with a pixel that may hold an arc of P_min >= 8 are compacted.  (b)
//      Full test of those groups: all 16 positions, the flags gathered into
//      per-pixel 16-bit bright / dark masks, and the corner test of Eq. 3 as
//      a look-up in the 64 Ki-entry bit table of Sec. III (built on the host
//      for P_min, P_max).  Corners go to a compacted list and mark their cell;
//   2. fallback threshold, only for pixels of cells left without a corner
//      (cells with no pixel inside the border never ask for it);
//   3. for each listed corner the SAD response is computed and the cell's
//      top-k is kept by atomicMax on the key response << 16 | (0xFFFF -
//      index in cell) (strongest first, then smaller y, then smaller x);
//   4. slots are written and every survivor is added to the s0 score map
//      (PFA steps 1-2: K_l << 16 | K_r in one word).

// Ring offsets (dx, dy) of the radius-3 Bresenham circle, index 0 below the
// centre (image y down), in ring order.
__constant__ int8_t c_ring_dx[16] = { 0, 1, 2, 3, 3, 3, 2, 1, 0, -1, -2, -3, -3, -3, -2, -1 };
__constant__ int8_t c_ring_dy[16] = { 3, 3, 2, 1, 0, -1, -2, -3, -3, -3, -2, -1, 0, 1, 2, 3 };

constexpr uint32_t kH = 0x80808080u, kL7 = 0x7F7F7F7Fu;

// Majority of three words, bitwise: at each byte's MSB, with c the carry into
// that bit from the low 7 bits, it is the carry out of the byte sum a + b.
__device__ __forceinline__ uint32_t maj3(uint32_t a, uint32_t b, uint32_t c) { return (a & b) | (c & (a | b)); }

struct FastLayout {
    int buf0, buf1, clist, ckey, cand, has_hi, sel, bar, total;
};

__host__ __device__ inline int fast_align(int v, int a) { return (v + a - 1) / a * a; }

// A group is 4 pixels of a row; a tile of max_px pixels whose rows hold at
// most kFastMaxTile pixels has at most max_px / 4 + kFastMaxTile groups.
// `cand` lists the groups that pass the cardinal pre-test.
__host__ __device__ inline FastLayout fast_layout(int max_box, int max_px, int max_cells, int k)
{
    FastLayout l;
    int o = kLutWords * 4;
    l.buf0 = o;  o += fast_align(max_box, 128);
    l.buf1 = o;  o += fast_align(max_box, 128);
    l.clist = o; o += fast_align(max_px * 2, 16);
    l.ckey = o;  o += k > 1 ? fast_align(max_px * 4, 16) : 0;
    l.cand = o;  o += fast_align((max_px / 4 + kFastMaxTile) * 2, 16);
    l.has_hi = o; o += fast_align(max_cells, 16);
    l.sel = o;   o += fast_align(max_cells * k * 4, 16);
    l.bar = o;   o += 16;
    l.total = o;
    return l;
}

// Dynamic shared memory of the bit-sliced kernel: the two tile boxes, the
// box's bit-planes (max_planes bytes: box rows of (chunks + 1) x 8 words and
// a 16-byte pad, see bs_row_units), the corner list and keys only for k > 1
// (k = 1 takes each cell's best corner as it is found), cell states,
// selections and the work list of a pass (16-bit item indices; a tile has at
// most kFastMaxTile rows of 4 items).  The fixed-size parts (corner windows,
// tile records, staged projections, mbarriers) are static arrays of the
// kernel.
constexpr int kBitsWin = 128;
constexpr int kBitsMaxItems = kFastMaxTile * (kFastMaxTile / 32);
struct BitsLayout {
    int buf0, buf1, planes, clist, ckey, has_hi, sel, wlist, total;
};
__host__ __device__ inline BitsLayout bits_layout(int max_box, int max_px, int max_cells, int k, int max_planes)
{
    BitsLayout l;
    int o = 0;
    l.buf0 = o;   o += fast_align(max_box, 128);
    l.buf1 = o;   o += fast_align(max_box, 128);
    l.planes = o; o += fast_align(max_planes, 16);
    l.clist = o;  o += k > 1 ? fast_align(max_px * 2, 16) : 0;
    l.ckey = o;   o += k > 1 ? fast_align(max_px * 4, 16) : 0;
    l.has_hi = o; o += fast_align(max_cells, 16);
    l.sel = o;    o += fast_align(max_cells * k * 4, 16);
    l.wlist = o;  o += kBitsMaxItems * 2;
    l.total = o;
    return l;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Position of a detection tile: its cells, pixels and the TMA box origin.
struct TileGeom {
    int li, ccx0, ccy0, ncx, ncy, x0, y0, tw, th, xs, ys, delta;
};

__device__ __forceinline__ TileGeom tile_geom(const Batch &b, int t)
{
    TileGeom G;
    G.li = __ldg(b.fast_tile_level + t);
    const LevelDesc &L = b.levels[G.li];
    const int tt = t - __ldg(b.fast_tile_base + G.li);
    const int ctas_x = (L.cells_x + L.bx - 1) / L.bx;
    const int ty = tt / ctas_x;
    G.ccx0 = (tt - ty * ctas_x) * L.bx;
    G.ccy0 = ty * L.by;
    G.ncx = min(L.bx, L.cells_x - G.ccx0);
    G.ncy = min(L.by, L.cells_y - G.ccy0);
    G.x0 = G.ccx0 * L.c;
    G.y0 = G.ccy0 * L.c;
    G.tw = min(G.ncx * L.c, L.W - G.x0);
    G.th = min(G.ncy * L.c, L.H - G.y0);
    // box columns start on a 16-byte boundary at or before x0 - 4; the
    // tile's first column (x0 - 4) sits delta bytes into each box row
    G.xs = L.tmap ? ((G.x0 - 4) & ~15) : G.x0 - 4;
    G.ys = G.y0 - 3;
    G.delta = G.x0 - 4 - G.xs;
    return G;
}

// Issue the TMA of tile t into buf; completion arrives on the mbarrier.
__device__ __forceinline__ void issue_tile(const Batch &b, int t, uint8_t *buf, uint64_t *bar)
{
    const TileGeom G = tile_geom(b, t);
    const LevelDesc &L = b.levels[G.li];
    if (!L.tmap) return;
    const uint32_t bytes = (uint32_t)(L.box_w * L.box_h);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(buf)), "l"(reinterpret_cast<uint64_t>(L.tmap)), "r"(G.xs), "r"(G.ys), "r"(smem_u32(bar))
        : "memory");
}

// Wait for the mbarrier phase `parity`, giving up after about a second.
__device__ __forceinline__ bool wait_tile(uint64_t *bar, uint32_t parity)
{
    const long long start = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done) : "r"(smem_u32(bar)), "r"(parity) : "memory");
        if (done) return true;
        if (clock64() - start > (1ll << 31)) return false;
    }
}

// Failure-detection self-test: a tile wait on an mbarrier that nothing
// arrives on runs out after its limit, sets kErrTimeout and returns, as the
// detection kernels do when a tile load does not complete.
__global__ void k_wait_selftest(uint32_t *err)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (!wait_tile(&bar, 0u) && threadIdx.x == 0) atomicOr(err, kErrTimeout);
}

cudaError_t launch_wait_selftest(uint32_t *err, cudaStream_t stream)
{
    k_wait_selftest<<<1, 32, 0, stream>>>(err);
    return cudaGetLastError();
}

// Corner bits (bit j: pixel 4g + j) of a group of 4 pixels; `base` points at
// the word left of the group's centre word in the first of its 7 tile rows.
__device__ __forceinline__ uint32_t group_corners(const uint32_t *base, int wpr, uint32_t e0, uint32_t e1,
                                                  const uint32_t *lut, int p_min)
{
    constexpr int RDX[16] = { 0, 1, 2, 3, 3, 3, 2, 1, 0, -1, -2, -3, -3, -3, -2, -1 };
    constexpr int RDY[16] = { 3, 3, 2, 1, 0, -1, -2, -3, -3, -3, -2, -1, 0, 1, 2, 3 };
    uint32_t w[7][3];
#pragma unroll
    for (int r = 0; r < 7; ++r) {
        w[r][0] = base[r * wpr + 0];
        w[r][1] = base[r * wpr + 1];
        w[r][2] = base[r * wpr + 2];
    }
    const uint32_t C = w[3][1];
    // per byte: Tb = C + eps and Td = C - eps (wrapped); nb / nd flag the
    // bytes where no ring pixel can be brighter than C + eps (C + eps >= 255)
    // or darker than C - eps (C <= eps)
    const uint32_t sb0 = (C & kL7) + (e0 & kL7);
    const uint32_t Tb = sb0 ^ ((C ^ e0) & kH);
    const uint32_t sb1 = (C & kL7) + (e1 & kL7);
    const uint32_t nb = maj3(C, e1, sb1) & kH;
    const uint32_t sd0 = (C | kH) - (e0 & kL7);
    const uint32_t Td = sd0 ^ (~(C ^ e0) & kH);
    const uint32_t sd1 = (C | kH) - (e1 & kL7);
    const uint32_t nd = ~((C & ~e1) | (~(C ^ e1) & sd1)) & kH;
    const uint32_t N = ~Tb, N7 = N & kL7, K = (Td & kL7) + kL7;
    uint32_t b_lo = 0, b_hi = 0, d_lo = 0, d_hi = 0;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int r = RDY[q] + 3, dx = RDX[q];
        uint32_t P;
        if (dx == 0) P = w[r][1];
        else if (dx > 0) P = __funnelshift_r(w[r][1], w[r][2], 8 * dx);
        else P = __funnelshift_r(w[r][0], w[r][1], 8 * (4 + dx));
        const uint32_t Pl = P & kL7;
        const uint32_t gb = maj3(P, N, Pl + N7);    // MSB: carry of P + ~(C + eps), i.e. P > C + eps
        const uint32_t gd = maj3(Td, ~P, K - Pl);   // MSB: carry of (C - eps) + ~P, i.e. P < C - eps
        const int sh = q < 8 ? 7 - q : 15 - q;
        const uint32_t m = kH >> sh;
        if (q < 8) { b_lo |= (gb >> sh) & m; d_lo |= (gd >> sh) & m; }
        else { b_hi |= (gb >> sh) & m; d_hi |= (gd >> sh) & m; }
    }
    const uint32_t nbx = (nb >> 7) * 0xFFu, ndx = (nd >> 7) * 0xFFu;
    b_lo &= ~nbx; b_hi &= ~nbx; d_lo &= ~ndx; d_hi &= ~ndx;
    uint32_t bits = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t sel = (uint32_t)j | ((uint32_t)(4 + j) << 4);
        const uint32_t mb = __byte_perm(b_lo, b_hi, sel) & 0xFFFFu;
        const uint32_t md = __byte_perm(d_lo, d_hi, sel) & 0xFFFFu;
        // a mask with fewer than P_min set bits has no run of P_min: skip the
        // look-up (lanes that skip issue no shared-memory request).  Brighter
        // and darker flags are disjoint, so for P_min >= 9 at most one of the
        // two masks can reach P_min and one look-up suffices.
        const int pb = __popc(mb), pd = __popc(md);
        uint32_t ok = 0;
        if (p_min >= 9) {
            const uint32_t m = pb >= p_min ? mb : md;
            if (max(pb, pd) >= p_min) ok = lut[m >> 5] >> (m & 31);
        } else {
            if (pb >= p_min) ok = lut[mb >> 5] >> (mb & 31);
            if (pd >= p_min) ok |= lut[md >> 5] >> (md & 31);
        }
        bits |= (ok & 1u) << j;
    }
    return bits;
}

// floor(v / c) for 0 <= v < 128 and 1 <= c <= 128 with cinv = ceil(2^16 / c):
// exact because v * c < 2^16.
// Cardinal pre-test of a group (bit j: pixel 4g + j may be a corner).  An
// arc of 8 or more contiguous ring pixels holds two neighbouring cardinal
// points (ring positions 0, 4, 8, 12), so a pixel whose cardinal flags
// satisfy neither (F0 | F8) & (F4 | F12) for brighter nor for darker is no
// corner at any P_min >= 8 (8 contiguous positions hold two neighbouring
// cardinal points; 7 may hold only one).  The flags use the same byte compares as the
// full test (without its never-masks, which only clear flags), so every
// corner passes.  `base` as for group_corners.
__device__ __forceinline__ uint32_t group_pretest(const uint32_t *base, int wpr, uint32_t e0)
{
    const uint32_t C = base[3 * wpr + 1];
    const uint32_t P0 = base[6 * wpr + 1];                          // ( 0, +3)
    const uint32_t P4 = __funnelshift_r(C, base[3 * wpr + 2], 24);  // (+3,  0)
    const uint32_t P8 = base[1];                                    // ( 0, -3)
    const uint32_t P12 = __funnelshift_r(base[3 * wpr], C, 8);      // (-3,  0)
    const uint32_t sb0 = (C & kL7) + (e0 & kL7);
    const uint32_t Tb = sb0 ^ ((C ^ e0) & kH);
    const uint32_t sd0 = (C | kH) - (e0 & kL7);
    const uint32_t Td = sd0 ^ (~(C ^ e0) & kH);
    const uint32_t N = ~Tb, N7 = N & kL7, K = (Td & kL7) + kL7;
    uint32_t gb[4], gd[4];
    const uint32_t P[4] = { P0, P4, P8, P12 };
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t Pl = P[i] & kL7;
        gb[i] = maj3(P[i], N, Pl + N7);
        gd[i] = maj3(Td, ~P[i], K - Pl);
    }
    const uint32_t x = (((gb[0] | gb[2]) & (gb[1] | gb[3])) | ((gd[0] | gd[2]) & (gd[1] | gd[3]))) & kH;
    // byte MSBs (bits 7, 15, 23, 31) to bits 0..3: after >> 7 they sit at
    // 0, 8, 16, 24; the multiply moves them to 21..24 without carries
    return (((x >> 7) * 0x00204081u) >> 21) & 0xFu;
}

// ---- bit-sliced ring test (P_min = 9, P_max = 13): 32 pixels per word, bit
// j of word i = bit i of pixel j's byte.  a > b for 8-bit numbers: the carry
// out of a + ~b, one majority per bit; c + e: a ripple adder against the
// constant's bit masks, returning the carry out.

// Bit-planes of a 32-byte chunk (bytes j of words a, z in memory order):
// output word i, bit j = bit i of byte j.  Each 8-byte block is an 8 x 8 bit
// matrix (row = byte, column = bit) transposed by three delta swaps (2 x 2,
// 4 x 4 and 8 x 8 sub-blocks); byte i of the transposed block b is then byte
// b of output word i.
__device__ __forceinline__ void bs_transpose(uint4 a, uint4 z, uint4 *dst)
{
    uint32_t w[8] = { a.x, a.y, a.z, a.w, z.x, z.y, z.z, z.w };
#pragma unroll
    for (int blk = 0; blk < 4; ++blk) {
        uint32_t lo = w[2 * blk], hi = w[2 * blk + 1], t;
        t = (lo ^ (lo >> 7)) & 0x00AA00AAu;  lo ^= t ^ (t << 7);
        t = (hi ^ (hi >> 7)) & 0x00AA00AAu;  hi ^= t ^ (t << 7);
        t = (lo ^ (lo >> 14)) & 0x0000CCCCu; lo ^= t ^ (t << 14);
        t = (hi ^ (hi >> 14)) & 0x0000CCCCu; hi ^= t ^ (t << 14);
        t = (lo ^ (hi << 4)) & 0xF0F0F0F0u;  lo ^= t; hi ^= t >> 4;
        w[2 * blk] = lo; w[2 * blk + 1] = hi;
    }
    uint32_t o[8];
#pragma unroll
    for (int half = 0; half < 2; ++half)
#pragma unroll
        for (int i = 0; i < 4; i += 2) {
            const uint32_t sel = (uint32_t)i | ((uint32_t)(4 + i) << 4) | ((uint32_t)(i + 1) << 8) |
                                 ((uint32_t)(5 + i) << 12);
            const uint32_t A = __byte_perm(w[half], w[2 + half], sel);
            const uint32_t B = __byte_perm(w[4 + half], w[6 + half], sel);
            o[4 * half + i] = __byte_perm(A, B, 0x5410u);
            o[4 * half + i + 1] = __byte_perm(A, B, 0x7632u);
        }
    dst[0] = make_uint4(o[0], o[1], o[2], o[3]);
    dst[1] = make_uint4(o[4], o[5], o[6], o[7]);
}

__device__ __forceinline__ uint32_t bs_greater(const uint32_t (&a)[8], const uint32_t (&b)[8])
{
    uint32_t c = a[0] & ~b[0];
#pragma unroll
    for (int i = 1; i < 8; ++i) c = maj3(a[i], ~b[i], c);
    return c;
}

__device__ __forceinline__ uint32_t bs_add_const(const uint32_t (&c)[8], uint32_t e, uint32_t (&t)[8])
{
    uint32_t k = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const uint32_t E = 0u - ((e >> i) & 1u);
        t[i] = c[i] ^ E ^ k;
        k = maj3(c[i], E, k);
    }
    return k;
}

// Longest circular run of the 16 flag words in [9, 13], with three-input
// ANDs: A3 = windows of 3, A9 = three A3 end to end, a run of 14 = an A9
// followed by two overlapping A3 (positions q + 9 .. q + 13).
__device__ __forceinline__ uint32_t bs_run_9_13(const uint32_t (&F)[16])
{
    uint32_t A3[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) A3[q] = F[q] & F[(q + 1) & 15] & F[(q + 2) & 15];
    uint32_t r9 = 0, r14 = 0;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const uint32_t a9 = A3[q] & A3[(q + 3) & 15] & A3[(q + 6) & 15];
        r9 |= a9;
        r14 |= a9 & A3[(q + 9) & 15] & A3[(q + 11) & 15];
    }
    return r9 & ~r14;
}

// Bounded-rectification response of the pixel at p (rows rowb bytes apart):
// the sum of |ring pixel - centre| over the 16 ring positions, the ring
// bytes packed four to a word (rows +-3: dx = -1, 0, 1; rows +-2: dx = +-2;
// rows +-1 and 0: dx = +-3) and summed by byte-SIMD absolute differences.
__device__ __forceinline__ int ring_sad(const uint8_t *p, int rowb)
{
    const uint8_t *u3 = p + 3 * rowb, *d3 = p - 3 * rowb, *u2 = p + 2 * rowb, *d2 = p - 2 * rowb;
    const uint8_t *u1 = p + rowb, *d1 = p - rowb;
    const uint32_t w0 = (uint32_t)u3[-1] | ((uint32_t)u3[0] << 8) | ((uint32_t)u3[1] << 16) | ((uint32_t)d3[-1] << 24);
    const uint32_t w1 = (uint32_t)d3[0] | ((uint32_t)d3[1] << 8) | ((uint32_t)u2[-2] << 16) | ((uint32_t)u2[2] << 24);
    const uint32_t w2 = (uint32_t)d2[-2] | ((uint32_t)d2[2] << 8) | ((uint32_t)u1[-3] << 16) | ((uint32_t)u1[3] << 24);
    const uint32_t w3 = (uint32_t)d1[-3] | ((uint32_t)d1[3] << 8) | ((uint32_t)p[-3] << 16) | ((uint32_t)p[3] << 24);
    const uint32_t cc = (uint32_t)p[0] * 0x01010101u;
    return (int)(__vsadu4(w0, cc) + __vsadu4(w1, cc) + __vsadu4(w2, cc) + __vsadu4(w3, cc));
}

// Corner bits of the 32 pixels of tile row py, chunk m (pixels 32 m + j).
// `planes`: box rows of `ru` 16-byte units, chunk m at unit 2 m; tile pixel 0
// sits at box column sb, so pixel 32 m + j + dx is bit sb + dx + j of chunks
// (m, m + 1).
__device__ __forceinline__ uint32_t bs_corners(const uint32_t *planes, int ru, int py, int m, int sb, int eps)
{
    constexpr int RDX[16] = { 0, 1, 2, 3, 3, 3, 2, 1, 0, -1, -2, -3, -3, -3, -2, -1 };
    constexpr int RDY[16] = { 3, 3, 2, 1, 0, -1, -2, -3, -3, -3, -2, -1, 0, 1, 2, 3 };
    uint32_t C[8], Tb[8], Td[8];
    {
        const uint4 *r = reinterpret_cast<const uint4 *>(planes) + (py + 3) * ru + 2 * m;
        const uint4 l0 = r[0], l1 = r[1], h0 = r[2], h1 = r[3];
        const uint32_t lo[8] = { l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w };
        const uint32_t hi[8] = { h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w };
#pragma unroll
        for (int i = 0; i < 8; ++i) C[i] = __funnelshift_r(lo[i], hi[i], sb);
    }
    // a centre with C + eps >= 256 is never brighter (threshold 255, which
    // no P exceeds); one with C < eps never darker (threshold 0)
    const uint32_t nb = bs_add_const(C, (uint32_t)eps, Tb);
    if (eps > 0) {
        const uint32_t nd = ~bs_add_const(C, (uint32_t)(256 - eps), Td);
#pragma unroll
        for (int i = 0; i < 8; ++i) Td[i] &= ~nd;
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) Td[i] = C[i];
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) Tb[i] |= nb;
    uint32_t Fb[16], Fd[16];
#pragma unroll
    for (int dy = 3; dy >= -3; --dy) {
        const uint4 *r = reinterpret_cast<const uint4 *>(planes) + (py + 3 + dy) * ru + 2 * m;
        const uint4 l0 = r[0], l1 = r[1], h0 = r[2], h1 = r[3];
        const uint32_t lo[8] = { l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w };
        const uint32_t hi[8] = { h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w };
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            if (RDY[q] != dy) continue;
            uint32_t P[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) P[i] = __funnelshift_r(lo[i], hi[i], sb + RDX[q]);
            Fb[q] = bs_greater(P, Tb);
            Fd[q] = bs_greater(Td, P);
        }
    }
    return bs_run_9_13(Fb) | bs_run_9_13(Fd);
}

// Bits j of the 32 pixels of tile row chunk px0..px0+31 whose cell state
// (row of states `st`, cells of c pixels) satisfies keep(state).
template <typename Keep>
__device__ __forceinline__ uint32_t cell_bits(const uint8_t *st, int px0, int tw, int c, uint32_t cinv, Keep keep)
{
    const int x_last = min(px0 + 31, tw - 1);
    const int c0 = (int)(((uint32_t)px0 * cinv) >> 16), c1 = (int)(((uint32_t)x_last * cinv) >> 16);
    uint32_t bits = 0;
    for (int cx = c0; cx <= c1; ++cx) {
        if (!keep(st[cx])) continue;
        const int a = max(cx * c - px0, 0), z = min((cx + 1) * c - px0, 32);
        bits |= (z >= 32 ? 0xFFFFFFFFu : ((1u << z) - 1u)) & (0xFFFFFFFFu << a);
    }
    return bits;
}

__device__ __forceinline__ int div_small(int v, uint32_t cinv) { return (int)(((uint32_t)v * cinv) >> 16); }

// Bits j of the 32 pixels px0 + j of a tile row that lie inside the level's
// evaluated columns [plo, phi) (tile coordinates).
__device__ __forceinline__ uint32_t border_bits(int px0, int plo, int phi)
{
    const int lo = min(max(plo - px0, 0), 32), hi = min(max(phi - px0, 0), 32);
    return (hi >= 32 ? 0xFFFFFFFFu : ((1u << hi) - 1u)) & (lo >= 32 ? 0u : (0xFFFFFFFFu << lo));
}

// Work list of a pass of k_fast_bits: appends to wlist (count in *n) every
// item (row r0 + itm / nch, chunk itm % nch) holding an evaluated pixel whose
// cell state satisfies keep(state), so that the pass runs full warps over
// those items only.  Warp-uniform loop; one atomic per warp and round.
template <typename Keep>
__device__ __forceinline__ void list_items(uint16_t *wlist, int *n, int items, int nch, uint32_t nchinv, int r0,
                                           int plo, int phi, const uint8_t *has_hi, int ncx, int tw, int c,
                                           uint32_t cinv, int lane, int warp, Keep keep)
{
    for (int base = warp * 32; base < items; base += kFastThreads) {
        const int itm = base + lane;
        bool need = false;
        if (itm < items) {
            const int rr = div_small(itm, nchinv), px0 = 32 * (itm - rr * nch);
            const uint32_t v = border_bits(px0, plo, phi);
            need = v && (v & cell_bits(has_hi + div_small(r0 + rr, cinv) * ncx, px0, tw, c, cinv, keep));
        }
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, need);
        int at = 0;
        if (lane == 0 && bal) at = atomicAdd(n, __popc(bal));
        at = __shfl_sync(0xFFFFFFFFu, at, 0);
        if (need) wlist[at + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)itm;
    }
}

// Byte-lane ring test with the cardinal pre-test and the corner table (any
// P_min, P_max).
__global__ void __launch_bounds__(kFastThreads) k_fast_cull(Batch b)
{
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ int n_corner, need_lo, n_skipped, n_cand[2];
    const int k = b.prm.k, border = b.prm.border, p_min = b.prm.p_min;
    const FastLayout lay = fast_layout(b.fast_max_box, b.fast_max_px, b.fast_max_cells, k);
    uint32_t *lut = reinterpret_cast<uint32_t *>(smem);
    uint8_t *const buf0 = smem + lay.buf0, *const buf1 = smem + lay.buf1;
    uint16_t *clist = reinterpret_cast<uint16_t *>(smem + lay.clist);
    uint32_t *ckey = reinterpret_cast<uint32_t *>(smem + lay.ckey);
    uint16_t *cand = reinterpret_cast<uint16_t *>(smem + lay.cand);
    uint8_t *has_hi = smem + lay.has_hi;
    uint32_t *sel = reinterpret_cast<uint32_t *>(smem + lay.sel);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + lay.bar);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    // TMA destinations must be 128-byte aligned; refuse to run otherwise
    if ((smem_u32(buf0) | smem_u32(buf1)) & 127u) {
        if (threadIdx.x == 0) atomicOr(b.err, kErrDecode);
        return;
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = threadIdx.x; i < kLutWords; i += kFastThreads) lut[i] = __ldg(b.corner_lut + i);
    __syncthreads();
    if (threadIdx.x == 0 && blockIdx.x < b.fast_tiles) issue_tile(b, blockIdx.x, buf0, &bars[0]);
    uint32_t phase0 = 0u, phase1 = 0u;

    int it = 0;
    for (int t = blockIdx.x; t < b.fast_tiles; t += gridDim.x, ++it) {
        const int cur = it & 1;
        const TileGeom G = tile_geom(b, t);
        const LevelDesc &L = b.levels[G.li];
        const ImageDesc &I = b.images[L.image];
        // prefetch the next tile into the other buffer (its readers finished
        // at the barrier that ended the previous iteration)
        if (threadIdx.x == 0 && t + (int)gridDim.x < b.fast_tiles)
            issue_tile(b, t + gridDim.x, cur ? buf0 : buf1, &bars[cur ^ 1]);
        const int c = L.c, cells_x = L.cells_x, W = L.W, Hh = L.H;
        const uint32_t cinv = (uint32_t)L.cinv;
        const int ncx = G.ncx, x0 = G.x0, y0 = G.y0, tw = G.tw, th = G.th;
        const int rowb = L.box_w, wpr = rowb >> 2;
        const int cells = ncx * G.ncy;
        uint8_t *tb = cur ? buf1 : buf0;

        if (L.tmap) {
            if (!wait_tile(&bars[cur], cur ? phase1 : phase0)) {
                if (threadIdx.x == 0) {
                    atomicOr(b.err, kErrTimeout);
                    // wait once more, with the same limit, for this tile's box
                    // and the next one's, so that no copy lands in the shared
                    // memory of a CTA that has ended
                    wait_tile(&bars[cur], cur ? phase1 : phase0);
                    const int tn = t + (int)gridDim.x;
                    if (tn < b.fast_tiles && b.levels[tile_geom(b, tn).li].tmap)
                        wait_tile(&bars[cur ^ 1], cur ? phase0 : phase1);
                }
                return;
            }
            if (cur) phase1 ^= 1u; else phase0 ^= 1u;
        } else {
            // levels whose tiles cannot start on a word boundary: plain loads,
            // the same layout (box rows of box_w bytes, delta = 0)
            uint32_t *tw32 = reinterpret_cast<uint32_t *>(tb);
            for (int i = threadIdx.x; i < L.box_h * wpr; i += kFastThreads) {
                const int r = i / wpr, wi = i - r * wpr;
                const uint8_t *row = L.raw + (size_t)min(max(G.ys + r, 0), Hh - 1) * L.pitch;
                const int gx = G.xs + 4 * wi;
                uint32_t v = 0;
#pragma unroll
                for (int q = 0; q < 4; ++q) v |= (uint32_t)__ldg(row + min(max(gx + q, 0), W - 1)) << (8 * q);
                tw32[i] = v;
            }
        }
        // cell state: 0 no corner yet, 1 primary-threshold corner, 2 skipped by
        // the learned proposal (its centre projects into a skipped s0 cell),
        // 3 no pixel inside the evaluation border (never holds a corner, so it
        // neither calls for the fallback pass nor joins it)
        int my_skipped = 0;
        for (int i = threadIdx.x; i < cells; i += kFastThreads) {
            const int lcy = i / ncx, lcx = i - lcy * ncx;
            const int cx0 = (G.ccx0 + lcx) * c, cy0 = (G.ccy0 + lcy) * c;
            const bool evaluated = cx0 + c > border && cx0 < W - border && cy0 + c > border && cy0 < Hh - border;
            uint8_t st = evaluated ? 0 : 3;
            if (I.skip && evaluated) {
                const int px = min(cx0 + c / 2, W - 1), py = min(cy0 + c / 2, Hh - 1);
                const int X = __ldg(L.projx + px), Y = __ldg(L.projy + py);
                st = I.skip[(Y / I.skip_c0) * I.skip_cells_x + X / I.skip_c0] ? 2 : 0;
            }
            if (I.skip && st != 0) { st = 2; ++my_skipped; }  // skip mode: never-cells count as skipped
            has_hi[i] = st;
        }
        for (int i = threadIdx.x; i < cells * k; i += kFastThreads) sel[i] = 0;
        if (threadIdx.x == 0) { n_corner = 0; need_lo = 0; n_skipped = 0; n_cand[0] = n_cand[1] = 0; }
        __syncthreads();
        if (I.skip) {  // uniform: the skipped-cell count only matters in skip mode
            if (my_skipped) atomicAdd(&n_skipped, my_skipped);
            __syncthreads();
        }
        const bool all_skipped = n_skipped == cells;
        const bool some_skipped = n_skipped > 0;  // tiles without skipped cells run as in exact mode

        // pixels evaluated: tile-local x in [plo, phi), rows whose y is inside the border
        const int plo = max(border - x0, 0), phi = min(W - border - x0, tw);
        // groups that hold evaluated pixels: rows [r0, r1) and group columns
        // [g0, g1) of the tile (only the first and last column can be partial)
        const int r0 = max(border - y0, 0), r1 = min(Hh - border - y0, th);
        const int g0 = plo >> 2, g1 = (phi + 3) >> 2;
        const int gw = max(g1 - g0, 0), nitems = max(r1 - r0, 0) * gw;
        // word of tile column 0 (pixel x0 - 4) within a box row
        const uint32_t *words = reinterpret_cast<const uint32_t *>(tb) + (G.delta >> 2);
        // 1./2. per threshold pass: (a) cardinal pre-test of every group, the
        // survivors compacted with their pixel masks (entry: row << 9 | group
        // << 4 | mask); (b) full ring test of the survivors, corners pushed to
        // the compacted corner list.
        for (int pass = 0; pass < 2 && !all_skipped; ++pass) {
            const int eps = pass == 0 ? I.eps_hi : I.eps_lo;
            if (pass == 1) {
                if (eps <= 0) break;
                __syncthreads();  // has_hi complete, pass-0 readers of cand done
                for (int i = threadIdx.x; i < cells; i += kFastThreads)
                    if (!has_hi[i]) need_lo = 1;
                __syncthreads();
                if (!need_lo) break;
            }
            const uint32_t e0 = (uint32_t)eps * 0x01010101u, e1 = (uint32_t)(eps + 1) * 0x01010101u;
            const int gstep_y = gw > 0 ? kFastThreads / gw : 0, gstep_x = kFastThreads - gstep_y * gw;
            int py = gw > 0 ? r0 + (int)threadIdx.x / gw : 0;
            int g = gw > 0 ? g0 + (int)threadIdx.x % gw : 0;
            for (int base = warp * 32; base < nitems; base += kFastThreads) {
                const int gi = base + lane;
                uint32_t pre = 0;
                if (gi < nitems) {
                    const int px0 = 4 * g;
                    {
                        // pixels px0 + j with plo <= px0 + j < phi
                        const int lo = min(max(plo - px0, 0), 4), hi = min(max(phi - px0, 0), 4);
                        uint32_t valid = (0xFu >> (4 - hi)) & (0xFu << lo) & 0xFu;
                        const int crow = div_small(py, cinv) * ncx;
                        if (pass == 1) {
                            // fallback pass: only cells without a corner (and not skipped)
                            uint32_t keep = 0;
#pragma unroll
                            for (int j = 0; j < 4; ++j)
                                keep |= (uint32_t)(has_hi[crow + div_small(min(px0 + j, tw - 1), cinv)] == 0) << j;
                            valid &= keep;
                        }
                        // the pre-test holds for arcs of 8 or more (P_min >= 8)
                        if (valid) pre = p_min >= 8 ? group_pretest(words + py * wpr + g, wpr, e0) & valid : valid;
                        if (pre && pass == 0 && some_skipped) {
                            // skip mode: drop pixels of skipped cells (after the cheap pre-test,
                            // which already rejects the flat regions skipped cells tend to be)
                            uint32_t keep = 0;
#pragma unroll
                            for (int j = 0; j < 4; ++j)
                                keep |= (uint32_t)(has_hi[crow + div_small(min(px0 + j, tw - 1), cinv)] != 2) << j;
                            pre &= keep;
                        }
                    }
                }
                const uint32_t m = __ballot_sync(0xFFFFFFFFu, pre != 0);
                int start = 0;
                if (lane == 0 && m) start = atomicAdd(&n_cand[pass], __popc(m));
                start = __shfl_sync(0xFFFFFFFFu, start, 0);
                if (pre) cand[start + __popc(m & ((1u << lane) - 1u))] = (uint16_t)((py << 9) | (g << 4) | pre);
                g += gstep_x; py += gstep_y;
                if (g >= g1) { g -= gw; ++py; }
            }
            __syncthreads();
            const int ncand = n_cand[pass];
            for (int base = warp * 32; base < ncand; base += kFastThreads) {
                const int gi = base + lane;
                uint32_t bits = 0;
                int cpy = 0, cg = 0;
                if (gi < ncand) {
                    const uint32_t e = cand[gi];
                    cpy = (int)(e >> 9);
                    cg = (int)(e >> 4) & 31;
                    bits = group_corners(words + cpy * wpr + cg, wpr, e0, e1, lut, p_min) & e & 0xFu;
                }
                // warp-aggregated append of this iteration's corners
                const int cnt = __popc(bits);
                int incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                    if (lane >= o) incl += y;
                }
                const int total = __shfl_sync(0xFFFFFFFFu, incl, 31);
                int start = 0;
                if (lane == 31 && total) start = atomicAdd(&n_corner, total);
                start = __shfl_sync(0xFFFFFFFFu, start, 31) + incl - cnt;
                if (bits) {
                    const int crow = div_small(cpy, cinv) * ncx;
                    do {
                        const int j = __ffs(bits) - 1;
                        bits &= bits - 1;
                        const int px = 4 * cg + j;
                        clist[start++] = (uint16_t)((cpy << 7) | px);
                        if (pass == 0) has_hi[crow + div_small(px, cinv)] = 1;
                    } while (bits);
                }
            }
        }
        __syncthreads();

        // 3. response of every listed corner and the per-cell top-k.
        const int nc = n_corner;
        const uint8_t *tbytes = tb + G.delta;  // pixel (x, y) at (y - y0 + 3) * rowb + (x - x0 + 4)
        for (int i = threadIdx.x; i < nc; i += kFastThreads) {
            const int e = clist[i];
            const int py = e >> 7, px = e & 127;
            const uint8_t *p = tbytes + (py + 3) * rowb + (px + 4);
            const int cy = div_small(py, cinv), cx = div_small(px, cinv);
            int r = 0;
            if (b.prm.resp_arc) {
                // the threshold the corner was found at: fallback corners lie
                // in cells without a primary-threshold corner
                r = ring_arc(p, rowb, has_hi[cy * ncx + cx] == 1 ? I.eps_hi : I.eps_lo, b.prm.p_min, b.prm.p_max);
            } else {
                const int ic = p[0];
#pragma unroll
                for (int q = 0; q < 16; ++q) r += abs((int)p[c_ring_dy[q] * rowb + c_ring_dx[q]] - ic);
            }
            const uint32_t inidx = (uint32_t)((py - cy * c) * c + (px - cx * c));
            const uint32_t key = ((uint32_t)r << 16) | (0xFFFFu - inidx);
            const int cell = cy * ncx + cx;
            if (k == 1) atomicMax(&sel[cell], key);
            else ckey[i] = key;
        }
        if (k > 1) {
            __syncthreads();
            for (int j = 0; j < k; ++j) {
                for (int i = threadIdx.x; i < nc; i += kFastThreads) {
                    const int e = clist[i];
                    const int cell = div_small(e >> 7, cinv) * ncx + div_small(e & 127, cinv);
                    const uint32_t key = ckey[i];
                    if (j == 0 || key < sel[cell * k + j - 1]) atomicMax(&sel[cell * k + j], key);
                }
                __syncthreads();
            }
        }
        __syncthreads();

        // 4. slots and the s0 score map.
        for (int e = threadIdx.x; e < cells * k; e += kFastThreads) {
            const int cell = e / k, j = e - cell * k;
            const int lcy = cell / ncx;
            const int gcx = G.ccx0 + cell - lcy * ncx, gcy = G.ccy0 + lcy;
            const uint32_t key = sel[e];
            b.slots[L.slot_base + (gcy * cells_x + gcx) * k + j] = key;
            if (key) {
                const int inidx = 0xFFFF - (int)(key & 0xFFFFu);
                const int x = gcx * c + inidx % c, y = gcy * c + inidx / c;
                if (x >= W || y >= Hh) { atomicOr(b.err, kErrDecode); continue; }
                const int X = __ldg(L.projx + x), Y = __ldg(L.projy + y);
                atomicAdd(I.map + (size_t)Y * I.W0 + X, (1u << 16) + (key >> 16));
            }
        }
        __syncthreads();  // every reader of this buffer is done before it is refilled
    }
}

// Bulk copy of tile record t into shared memory, completing on `bar`.
__device__ __forceinline__ void fetch_rec(const Batch &b, int t, TileRec *dst, uint64_t *bar)
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"((uint32_t)sizeof(TileRec)) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(b.tile_rec + t)),
                 "r"((uint32_t)sizeof(TileRec)), "r"(smem_u32(bar)) : "memory");
}

// The tile box (TMA, levels with a tensor map) and the tile's projection
// ranges (bulk copies) of record R, all completing on `bar`.
__device__ __forceinline__ void issue_rec_tile(const TileRec &R, uint8_t *buf, uint8_t *prj, uint64_t *bar)
{
    const uint32_t box = R.tmap ? (uint32_t)(R.box_w * R.box_h) : 0u;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(box + (uint32_t)(R.prj_bytes_x + R.prj_bytes_y)) : "memory");
    if (R.tmap)
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
            ::"r"(smem_u32(buf)), "l"(reinterpret_cast<uint64_t>(R.tmap)), "r"(R.xs), "r"(R.ys), "r"(smem_u32(bar))
            : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(prj)), "l"(reinterpret_cast<uint64_t>(R.prj_src_x)), "r"((uint32_t)R.prj_bytes_x),
                 "r"(smem_u32(bar)) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(prj + kPrjBytes)), "l"(reinterpret_cast<uint64_t>(R.prj_src_y)),
                 "r"((uint32_t)R.prj_bytes_y), "r"(smem_u32(bar)) : "memory");
}

// Thread 0 of k_fast_bits after the wait for tile t's box ran out: wait once
// more, with the same limit, for every copy it still has in flight (this
// box; then either the next tile's box and the record after it, or the next
// record if its wait ran out too), so that no copy lands in the shared
// memory of a CTA that has ended.  rph bit s is the parity of the next
// completion of record barrier 2 + s, phases bit p that of box barrier p.
__device__ __forceinline__ void drain_bits(const Batch &b, uint64_t *bars, int t, int grid, int cur, int s3,
                                        uint32_t phases, uint32_t rph, int aborted)
{
    wait_tile(&bars[cur], (phases >> cur) & 1u);
    if (t + grid >= b.fast_tiles) return;
    const int sn = s3 == 2 ? 0 : s3 + 1, sa = s3 == 0 ? 2 : s3 - 1;
    if (aborted) {
        wait_tile(&bars[2 + sn], (rph >> sn) & 1u);
        return;
    }
    wait_tile(&bars[cur ^ 1], (phases >> (cur ^ 1)) & 1u);
    if (t + 2 * grid < b.fast_tiles) wait_tile(&bars[2 + sa], (rph >> sa) & 1u);
}

// Bit-sliced ring test (P_min = 9, P_max = 13), the same results as
// k_fast_cull.  Tiles come with host-made records: thread 0 fetches the
// record of the tile after next and, once the next tile's record is in,
// issues that tile's box and projection ranges, so every tile starts from
// shared memory.  Per tile: tile wait, cell states, bit-planes, one barrier;
// each threshold pass classifies 32 pixels of a row per thread, and every
// warp scores its own corners right away through a window of entries in
// shared memory (k = 1: atomic maximum of the cell's key; k > 1: corner list
// for the top-k rounds); a barrier ends each pass and one the tile.  The
// counters of a tile live in one of two sets by tile parity, so the set of
// the next tile is cleared while the current one is in use.
// Compile-time variants: kArc, the corner response (the arc's, an opt-in
// reading, or the whole ring's SAD); kSkip, the learned cell-skip mode;
// kTop1, one keypoint per cell (k = 1, the default) or the top-k rounds.
template <bool kArc, bool kSkip, bool kTop1>
__global__ void __launch_bounds__(kFastThreads, 3) k_fast_bits(Batch b)
{
    extern __shared__ __align__(128) uint8_t smem[];
    // per set: corners listed (k > 1), skipped cells, cells open at the
    // start (state 0), open cells that got a primary-threshold corner
    __shared__ int cnt[2][4];
    __shared__ int s_nlist[2];  // work-list lengths of pass 0 (cells skipped) and pass 1
    __shared__ int s_abort;
    __shared__ uint32_t s_rph;  // thread 0: parity of the next completion of each record barrier (bit s)
    __shared__ __align__(16) uint16_t s_wbuf[kFastThreads / 32][kBitsWin];
    __shared__ __align__(16) TileRec recs[3];
    __shared__ __align__(16) uint8_t s_prj[2][2 * kPrjBytes];  // per box: x range, y range
    __shared__ __align__(8) uint64_t bars[5];                   // [0..1] boxes, [2..4] records
    const int k = kTop1 ? 1 : b.prm.k, border = b.prm.border;
    const BitsLayout lay = bits_layout(b.fast_max_box, b.fast_max_px, b.fast_max_cells, k, b.fast_max_planes);
    uint8_t *const buf0 = smem + lay.buf0, *const buf1 = smem + lay.buf1;
    uint32_t *planes = reinterpret_cast<uint32_t *>(smem + lay.planes);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint16_t *wbuf = s_wbuf[warp];
    uint16_t *clist = reinterpret_cast<uint16_t *>(smem + lay.clist);
    uint32_t *ckey = reinterpret_cast<uint32_t *>(smem + lay.ckey);
    uint8_t *has_hi = smem + lay.has_hi;
    uint32_t *sel = reinterpret_cast<uint32_t *>(smem + lay.sel);
    uint16_t *wlist = reinterpret_cast<uint16_t *>(smem + lay.wlist);

    if ((smem_u32(buf0) | smem_u32(buf1)) & 127u) {
        if (threadIdx.x == 0) atomicOr(b.err, kErrDecode);
        return;
    }
    const int grid = (int)gridDim.x;
    if (threadIdx.x == 0) {
        for (int i = 0; i < 5; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[i])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
        const int t0 = blockIdx.x;
        if (t0 < b.fast_tiles) {
            fetch_rec(b, t0, &recs[0], &bars[2]);
            if (t0 + grid < b.fast_tiles) fetch_rec(b, t0 + grid, &recs[1], &bars[3]);
            if (wait_tile(&bars[2], 0u)) issue_rec_tile(recs[0], buf0, s_prj[0], &bars[0]);
            else {
                // give up, after waiting once more (same limit) for both
                // record copies, so that none lands after the CTA has ended
                atomicOr(b.err, kErrTimeout);
                s_abort = 1;
                wait_tile(&bars[2], 0u);
                if (t0 + grid < b.fast_tiles) wait_tile(&bars[3], 0u);
            }
        }
        s_rph = 1u;
    }
    if (threadIdx.x < 8) cnt[threadIdx.x >> 2][threadIdx.x & 3] = 0;
    __syncthreads();
    if (s_abort) return;
    uint32_t phases = 0u;  // bit p: parity of the next completion of box barrier p

    int it = 0;
    for (int t = blockIdx.x; t < b.fast_tiles; t += grid, ++it) {
        const int cur = it & 1, s3 = it % 3;
        int *const C = cnt[cur];
        const TileRec &R = recs[s3];
        const uint16_t *prj = reinterpret_cast<const uint16_t *>(s_prj[cur]);
        if (threadIdx.x == 0) {
            // the next tile's record was fetched one tile ago; the slot of the
            // tile after it, the other box and its projections were last read
            // before the barrier that ended the previous tile
            // (after a record wait runs out nothing more is issued; the CTA
            // stops at the abort check after the tile's bit-plane barrier)
            if (t + grid < b.fast_tiles) {
                const int sn = s3 == 2 ? 0 : s3 + 1;
                if (wait_tile(&bars[2 + sn], (s_rph >> sn) & 1u)) {
                    issue_rec_tile(recs[sn], cur ? buf0 : buf1, s_prj[cur ^ 1], &bars[cur ^ 1]);
                    s_rph ^= 1u << sn;
                    if (t + 2 * grid < b.fast_tiles) {
                        const int sa = s3 == 0 ? 2 : s3 - 1;
                        fetch_rec(b, t + 2 * grid, &recs[sa], &bars[2 + sa]);
                    }
                } else { atomicOr(b.err, kErrTimeout); s_abort = 1; }
            }
            cnt[cur ^ 1][0] = cnt[cur ^ 1][1] = cnt[cur ^ 1][2] = cnt[cur ^ 1][3] = 0;
            // the lists of the previous tile were last read before its closing
            // barrier; this tile's are built after a barrier that follows this
            s_nlist[0] = s_nlist[1] = 0;
        }
        uint8_t *const tb = cur ? buf1 : buf0;
        // the box and the projections (every tile waits: the projections
        // come on the same barrier whether or not the box does)
        if (!wait_tile(&bars[cur], (phases >> cur) & 1u)) {
            if (threadIdx.x == 0) {
                atomicOr(b.err, kErrTimeout);
                drain_bits(b, bars, t, grid, cur, s3, phases, s_rph, s_abort);
            }
            return;
        }
        phases ^= 1u << cur;
        bool all_skipped;
        {
        // record fields are read where needed (shared memory): values read
        // before a barrier are not carried across it
        const int c = R.c, W = R.W, Hh = R.H, x0 = R.x0, y0 = R.y0, rowb = R.box_w;
        const int ncx = R.ncx, cells = ncx * R.ncy;
        // learned skip: the image's proposal skipped at least one cell (an
        // image with none takes the exact path: no per-cell flags, no extra
        // barrier)
        const bool tskip = kSkip && R.skip != nullptr && __ldg(b.skip_any + R.image) != 0;
        if (!R.tmap) {
            // levels whose tiles cannot start on a word boundary: plain loads
            // (box rows of box_w bytes, delta = 0)
            const int wpr = rowb >> 2;
            uint32_t *tw32 = reinterpret_cast<uint32_t *>(tb);
            for (int i = threadIdx.x; i < R.box_h * wpr; i += kFastThreads) {
                const int r = i / wpr, wi = i - r * wpr;
                const uint8_t *row = R.raw + (size_t)min(max(R.ys + r, 0), Hh - 1) * R.pitch;
                const int gx = R.xs + 4 * wi;
                uint32_t v = 0;
#pragma unroll
                for (int q = 0; q < 4; ++q) v |= (uint32_t)__ldg(row + min(max(gx + q, 0), W - 1)) << (8 * q);
                tw32[i] = v;
            }
        }
        // cell states (as in k_fast_cull) and cleared selections
        int my_skipped = 0, my_open = 0;
        for (int i = threadIdx.x; i < cells; i += kFastThreads) {
            const int lcy = i / ncx, lcx = i - lcy * ncx;
            const int cx0 = (R.ccx0 + lcx) * c, cy0 = (R.ccy0 + lcy) * c;
            const bool evaluated = cx0 + c > border && cx0 < W - border && cy0 + c > border && cy0 < Hh - border;
            uint8_t st = evaluated ? 0 : 3;
            if (tskip && evaluated) {
                const int px = min(cx0 + c / 2, W - 1), py = min(cy0 + c / 2, Hh - 1);
                const int X = prj[R.prj_off_x + px - x0], Y = prj[kPrjBytes / 2 + R.prj_off_y + py - y0];
                st = R.skip[(Y / R.skip_c0) * R.skip_cells_x + X / R.skip_c0] ? 2 : 0;
            }
            if (tskip && st != 0) { st = 2; ++my_skipped; }
            my_open += st == 0;
            has_hi[i] = st;
        }
        for (int i = threadIdx.x; i < cells * k; i += kFastThreads) sel[i] = 0;
        if (my_skipped) atomicAdd(&C[1], my_skipped);
        if (my_open) atomicAdd(&C[2], my_open);
        // a box loaded with plain loads, the cell states and, in skip mode,
        // the skipped count are complete before the planes
        if (!R.tmap || tskip) __syncthreads();
        all_skipped = tskip && C[1] == cells;

        // bit-planes of the box rows [r0, r1 + 6) that the evaluated rows
        // [r0, r1) read, chunks 0..nch (an item of chunk m reads m and m + 1),
        // one 32-byte chunk per thread; chunks at or past the box's end
        // (a row's last may hold only 16 bytes) are zero
        const int r0 = max(border - y0, 0), r1 = min(Hh - border - y0, R.th);
        const int nch = (R.tw + 31) >> 5;
        const int nbc = (rowb + 31) >> 5, ru = bs_row_units(nch);
        if (!all_skipped) {
            const int nrows = max(r1 - r0, 0) > 0 ? r1 - r0 + 6 : 0;
            for (int ci = threadIdx.x; ci < nrows * (nch + 1); ci += kFastThreads) {
                const int rr = ci / (nch + 1), kc = ci - rr * (nch + 1), r = r0 + rr;
                uint4 a = make_uint4(0u, 0u, 0u, 0u), z = a;
                if (kc < nbc) {
                    const uint4 *src = reinterpret_cast<const uint4 *>(tb + r * rowb + 32 * kc);
                    a = src[0];
                    if (32 * kc + 16 < rowb) z = src[1];
                }
                bs_transpose(a, z, reinterpret_cast<uint4 *>(planes) + r * ru + 2 * kc);
            }
            // cells skipped by the proposal: pass 0 runs over the items that
            // hold a pixel of a cell that is not (states are complete: skip
            // mode has a barrier after them)
            if (tskip && C[1] > 0) {
                const int plo = max(border - x0, 0), phi = min(W - border - x0, R.tw);
                list_items(wlist, &s_nlist[0], max(r1 - r0, 0) * nch, nch, (65536u + nch - 1) / nch, r0, plo, phi,
                           has_hi, ncx, R.tw, c, (uint32_t)R.cinv, lane, warp,
                           [](uint8_t st) { return st != 2; });
            }
        }
        }
        __syncthreads();
        if (s_abort) {  // thread 0 could not start the next tile
            if (threadIdx.x == 0) {
                const int sn = s3 == 2 ? 0 : s3 + 1;
                wait_tile(&bars[2 + sn], (s_rph >> sn) & 1u);  // the record copy that did not complete
            }
            return;
        }
        const bool some_skipped = kSkip && C[1] > 0;  // constant false outside skip mode

        {
        const int c = R.c, W = R.W, Hh = R.H, x0 = R.x0, y0 = R.y0, tw = R.tw, rowb = R.box_w, ncx = R.ncx;
        const uint32_t cinv = (uint32_t)R.cinv;
        const int plo = max(border - x0, 0), phi = min(W - border - x0, tw);
        const int r0 = max(border - y0, 0), r1 = min(Hh - border - y0, R.th);
        const int nch = (tw + 31) >> 5, sb = R.delta + 4, ru = bs_row_units(nch);
        const uint32_t nchinv = (65536u + nch - 1) / nch;  // item / nch by a multiply (item < 2^9)
        const int items = max(r1 - r0, 0) * nch;
        const uint8_t *tbytes = tb + R.delta;  // pixel (x, y) at (y - y0 + 3) * rowb + (x - x0 + 4)
        for (int pass = 0; pass < 2 && !all_skipped; ++pass) {
            const int eps = pass == 0 ? R.eps_hi : R.eps_lo;
            // fallback pass only while an open cell got no corner
            if (pass == 1 && (eps <= 0 || C[3] >= C[2])) break;
            // pass 0 covers every item, or the listed ones when cells are
            // skipped; pass 1 lists the items holding a pixel of a cell still
            // without a corner (cell states are final after pass 0's barrier)
            const bool listed = pass == 1 || some_skipped;
            if (pass == 1) {
                list_items(wlist, &s_nlist[1], items, nch, nchinv, r0, plo, phi, has_hi, ncx, tw, c, cinv, lane, warp,
                           [](uint8_t st) { return st == 0; });
                __syncthreads();
            }
            const int n_work = listed ? s_nlist[pass] : items;
            for (int base = warp * 32; base < n_work; base += kFastThreads) {
                const int w = base + lane;
                uint32_t bits = 0;
                int py = 0, px0 = 0;
                if (w < n_work) {
                    const int itm = listed ? (int)wlist[w] : w;
                    const int rr = div_small(itm, nchinv), m = itm - rr * nch;
                    py = r0 + rr;
                    px0 = 32 * m;
                    uint32_t valid = border_bits(px0, plo, phi);
                    const uint8_t *strow = has_hi + div_small(py, cinv) * ncx;
                    if (pass == 1 && valid)  // only cells without a corner (and not skipped)
                        valid &= cell_bits(strow, px0, tw, c, cinv, [](uint8_t st) { return st == 0; });
                    else if (some_skipped && valid)  // not in a skipped cell
                        valid &= cell_bits(strow, px0, tw, c, cinv, [](uint8_t st) { return st != 2; });
                    if (valid) bits = bs_corners(planes, ru, py, m, sb, eps) & valid;
                }
                // the warp's corners in order, scored through windows of kBitsWin entries
                const int nb = __popc(bits);
                int incl = nb;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                    if (lane >= o) incl += y;
                }
                const int total = __shfl_sync(0xFFFFFFFFu, incl, 31);
                if (pass == 0 && bits) {
                    // mark the open cells that got a corner, each counted once
                    const int crow = div_small(py, cinv) * ncx;
                    const int ca = div_small(px0 + __ffs(bits) - 1, cinv), cz = div_small(px0 + 31 - __clz(bits), cinv);
                    for (int cx = ca; cx <= cz; ++cx) {
                        const int a = max(cx * c - px0, 0), z = min((cx + 1) * c - px0, 32);
                        const uint32_t span = (z >= 32 ? 0xFFFFFFFFu : ((1u << z) - 1u)) & (0xFFFFFFFFu << a);
                        const int cell = crow + cx;
                        if ((bits & span) && has_hi[cell] == 0) {
                            const uint32_t sh = 8u * (uint32_t)(cell & 3);
                            const uint32_t old = atomicOr(reinterpret_cast<uint32_t *>(has_hi) + (cell >> 2), 1u << sh);
                            if (((old >> sh) & 0xFFu) == 0u) atomicAdd(&C[3], 1);
                        }
                    }
                }
                const int ebase = (py << 7) | px0;  // entry of pixel px0 + j: ebase + j
                for (int w0 = 0; w0 < total; w0 += kBitsWin) {
                    uint32_t bb = bits;
                    for (int id = incl - nb; bb && id < w0 + kBitsWin; ++id) {
                        const int j = __ffs(bb) - 1;
                        bb &= bb - 1;
                        if (id >= w0) wbuf[id - w0] = (uint16_t)(ebase + j);
                    }
                    __syncwarp();
                    const int n = min(total - w0, kBitsWin);
                    int lbase = 0;
                    if (k > 1) {
                        if (lane == 0) lbase = atomicAdd(&C[0], n);
                        lbase = __shfl_sync(0xFFFFFFFFu, lbase, 0);
                    }
                    for (int i = lane; i < n; i += 32) {
                        const int e = wbuf[i];
                        const int cy_ = e >> 7, cx_ = e & 127;
                        const uint8_t *pp = tbytes + (cy_ + 3) * rowb + (cx_ + 4);
                        const int r = kArc ? ring_arc(pp, rowb, eps, b.prm.p_min, b.prm.p_max)
                                                     : ring_sad(pp, rowb);
                        const int ccy = div_small(cy_, cinv), ccx = div_small(cx_, cinv);
                        const uint32_t inidx = (uint32_t)((cy_ - ccy * c) * c + (cx_ - ccx * c));
                        const uint32_t key = ((uint32_t)r << 16) | (0xFFFFu - inidx);
                        if (k == 1) atomicMax(&sel[ccy * ncx + ccx], key);
                        else { clist[lbase + i] = (uint16_t)e; ckey[lbase + i] = key; }
                    }
                    __syncwarp();
                }
            }
            __syncthreads();  // selections, marks and counts of this pass complete
        }
        }
        if (k > 1) {
            const uint32_t cinv = (uint32_t)R.cinv;
            const int ncx = R.ncx, nc = C[0];
            for (int j = 0; j < k; ++j) {
                for (int i = threadIdx.x; i < nc; i += kFastThreads) {
                    const int e = clist[i];
                    const int cell = div_small(e >> 7, cinv) * ncx + div_small(e & 127, cinv);
                    const uint32_t key = ckey[i];
                    if (j == 0 || key < sel[cell * k + j - 1]) atomicMax(&sel[cell * k + j], key);
                }
                __syncthreads();
            }
        }

        // slots and the s0 score map (as in k_fast_cull), projections from
        // the staged ranges
        const int c = R.c, ncx = R.ncx, cells = ncx * R.ncy;
        for (int e = threadIdx.x; e < cells * k; e += kFastThreads) {
            const int cell = e / k, j = e - cell * k;
            const int lcy = cell / ncx;
            const int gcx = R.ccx0 + cell - lcy * ncx, gcy = R.ccy0 + lcy;
            const uint32_t key = sel[e];
            b.slots[R.slot_base + (gcy * R.cells_x + gcx) * k + j] = key;
            if (key) {
                const int inidx = 0xFFFF - (int)(key & 0xFFFFu);
                const int x = gcx * c + inidx % c, y = gcy * c + inidx / c;
                if (x >= R.W || y >= R.H) { atomicOr(b.err, kErrDecode); continue; }
                const int X = prj[R.prj_off_x + x - R.x0], Y = prj[kPrjBytes / 2 + R.prj_off_y + y - R.y0];
                atomicAdd(R.map + (size_t)Y * R.W0 + X, (1u << 16) + (key >> 16));
            }
        }
        __syncthreads();  // every reader of this box, its projections, the planes and this set is done
    }
}

int fast_smem_bytes(int max_box, int max_px, int max_cells, int k, int max_planes)
{
    return max_planes > 0 ? bits_layout(max_box, max_px, max_cells, k, max_planes).total
                          : fast_layout(max_box, max_px, max_cells, k).total;
}

// The bit-sliced detection kernel for a batch's response kind, skip mode and
// keypoints per cell (index kArc * 4 + kSkip * 2 + kTop1).
static const void *const kFastBitsVariants[8] = {
    reinterpret_cast<const void *>(k_fast_bits<false, false, false>),
    reinterpret_cast<const void *>(k_fast_bits<false, false, true>),
    reinterpret_cast<const void *>(k_fast_bits<false, true, false>),
    reinterpret_cast<const void *>(k_fast_bits<false, true, true>),
    reinterpret_cast<const void *>(k_fast_bits<true, false, false>),
    reinterpret_cast<const void *>(k_fast_bits<true, false, true>),
    reinterpret_cast<const void *>(k_fast_bits<true, true, false>),
    reinterpret_cast<const void *>(k_fast_bits<true, true, true>),
};

// The detection kernel of a batch: the bit-sliced test for the default run
// bounds (in the variant of its response, skip mode and k), else the
// per-pixel test.
static const void *detect_kernel_of(const Batch &b)
{
    if (!b.fast_bits) return reinterpret_cast<const void *>(k_fast_cull);
    return kFastBitsVariants[(b.prm.resp_arc ? 4 : 0) + (b.skip_any ? 2 : 0) + (b.prm.k == 1 ? 1 : 0)];
}

cudaError_t launch_fast_cull(const Batch &b, cudaStream_t stream)
{
    if (b.fast_tiles == 0) return cudaSuccess;
    static int cached_smem = -1, cached_blocks = 0, n_sm = 0;
    static const void *cached_fn = nullptr;
    cudaError_t e;
    if (n_sm == 0) {
        int dev = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    }
    const void *fn = detect_kernel_of(b);
    if (cached_smem != b.fast_smem || cached_fn != fn) {
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cached_blocks, fn, kFastThreads, b.fast_smem)) !=
            cudaSuccess)
            return e;
        cached_smem = b.fast_smem;
        cached_fn = fn;
    }
    int per_sm = std::max(1, cached_blocks);
    if (b.fast_ctas_per_sm > 0) per_sm = std::min(per_sm, b.fast_ctas_per_sm);
    const int grid = std::min(b.fast_tiles, per_sm * n_sm);
    void *args[] = { const_cast<Batch *>(&b) };
    return cudaLaunchKernel(fn, dim3(grid), dim3(kFastThreads), args, (size_t)b.fast_smem, stream);
}

// Detection CTAs of this batch's launch that fit on one SM at once.
cudaError_t detect_ctas_that_fit(const Batch &b, int *per_sm)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, detect_kernel_of(b), kFastThreads, b.fast_smem);
}

cudaError_t configure_kernels()
{
    cudaError_t e = cudaSuccess;
    for (int v = 0; v < 8 && e == cudaSuccess; ++v)
        e = cudaFuncSetAttribute(kFastBitsVariants[v], cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_fast_cull, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

}  // namespace jslam
