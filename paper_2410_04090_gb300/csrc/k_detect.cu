// Detection stage: image pyramid with Gaussian filtering, then FAST with
// Bounded Rectification, per-cell culling and the scatter half of PFA.
//
// k_pyramid   one CTA per 128x32 output tile of any (image, level): resamples
//             the level from level 0 (bilinear, Q8 taps from host tables),
//             writes it, and writes its 7-tap Gaussian (Sec. III, streamlined
//             multiscale detection and extraction: "Gaussian filtering ...
//             essential for robustness").
// k_fast_cull one CTA per block of culling cells of any (image, level): stages
//             the raw tile plus a 3-pixel halo in shared memory, evaluates the
//             16-pixel ring of every pixel (Sec. II-A, Eq. 1 labels, Eq. 3
//             bounded run length; Sec. III bit masks and SAD response), keeps
//             the top-k corners of each cell (Sec. II-C-1, Feature Culling)
//             and adds each survivor to the s0 score map (Sec. II-C-2, PFA
//             steps 1-2: K_l and K_r accumulate in one packed word).
#include "jslam_internal.h"

namespace jslam {

__constant__ int32_t c_blur_w[7];

cudaError_t set_blur_weights(const int32_t w[7])
{
    return cudaMemcpyToSymbol(c_blur_w, w, sizeof(int32_t) * 7);
}

// Largest i in [0, n) with base[i] <= v (base non-decreasing, base[0] = 0).
__device__ __forceinline__ int find_bucket(const int32_t *base, int n, int v)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(base + mid) <= v) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------- pyramid

__global__ void __launch_bounds__(kPyrThreads) k_pyramid(Batch b)
{
    constexpr int RW = kPyrTW + 6, RH = kPyrTH + 6;
    __shared__ uint8_t rs[RH][kPyrTW + 8];
    __shared__ uint16_t hs[RH][kPyrTW];

    const int li = find_bucket(b.pyr_tile_base, b.n_levels, blockIdx.x);
    const LevelDesc L = b.levels[li];
    const ImageDesc &I = b.images[L.image];
    const int t = blockIdx.x - b.pyr_tile_base[li];
    const int tiles_x = (L.W + kPyrTW - 1) / kPyrTW;
    const int x0 = (t % tiles_x) * kPyrTW, y0 = (t / tiles_x) * kPyrTH;
    const uint8_t *L0 = b.in.ptr[L.image];
    const int W0 = I.W0, H0 = I.H0, pitch0 = b.in.pitch[L.image];

    // Raw level values over the tile plus a 3-pixel halo; coordinates outside
    // the level are clamped (replicated border of the blur).
    for (int i = threadIdx.x; i < RW * RH; i += kPyrThreads) {
        const int ry = i / RW, rx = i - ry * RW;
        const int gy = min(max(y0 - 3 + ry, 0), L.H - 1);
        const int gx = min(max(x0 - 3 + rx, 0), L.W - 1);
        uint32_t v;
        if (L.level == 0) {
            v = __ldg(L0 + (size_t)gy * pitch0 + gx);
        } else {
            const uint32_t tx = __ldg(L.tapx + gx), ty = __ldg(L.tapy + gy);
            const int xa = tx & 0xFFFF, a = tx >> 16, xb = min(xa + 1, W0 - 1);
            const int ya = ty & 0xFFFF, wb = ty >> 16, yb = min(ya + 1, H0 - 1);
            const uint8_t *ra = L0 + (size_t)ya * pitch0, *rb = L0 + (size_t)yb * pitch0;
            const uint32_t top = (256u - a) * __ldg(ra + xa) + (uint32_t)a * __ldg(ra + xb);
            const uint32_t bot = (256u - a) * __ldg(rb + xa) + (uint32_t)a * __ldg(rb + xb);
            v = ((256u - wb) * top + (uint32_t)wb * bot + 32768u) >> 16;
        }
        rs[ry][rx] = (uint8_t)v;
    }
    __syncthreads();

    if (L.level > 0) {
        for (int i = threadIdx.x; i < kPyrTW * kPyrTH; i += kPyrThreads) {
            const int ry = i / kPyrTW, rx = i % kPyrTW;
            const int gy = y0 + ry, gx = x0 + rx;
            if (gy < L.H && gx < L.W) L.raw_w[(size_t)gy * L.pitch + gx] = rs[ry + 3][rx + 3];
        }
    }
    // Horizontal pass over every halo row.
    for (int i = threadIdx.x; i < kPyrTW * RH; i += kPyrThreads) {
        const int ry = i / kPyrTW, rx = i % kPyrTW;
        uint32_t acc = 0;
#pragma unroll
        for (int k = 0; k < 7; ++k) acc += (uint32_t)c_blur_w[k] * rs[ry][rx + k];
        hs[ry][rx] = (uint16_t)acc;
    }
    __syncthreads();
    // Vertical pass and rounding.
    for (int i = threadIdx.x; i < kPyrTW * kPyrTH; i += kPyrThreads) {
        const int ry = i / kPyrTW, rx = i % kPyrTW;
        const int gy = y0 + ry, gx = x0 + rx;
        if (gy < L.H && gx < L.W) {
            uint32_t acc = 0;
#pragma unroll
            for (int k = 0; k < 7; ++k) acc += (uint32_t)c_blur_w[k] * hs[ry + k][rx];
            L.blur[(size_t)gy * L.blur_pitch + gx] = (uint8_t)((acc + 32768u) >> 16);
        }
    }
}

cudaError_t launch_pyramid(const Batch &b, cudaStream_t stream)
{
    if (b.pyr_tiles == 0) return cudaSuccess;
    k_pyramid<<<b.pyr_tiles, kPyrThreads, 0, stream>>>(b);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- FAST + FC

// Ring offsets (dx, dy) of the radius-3 Bresenham circle, index 0 below the
// centre (image y down), in ring order.
__constant__ int8_t c_ring_dx[16] = { 0, 1, 2, 3, 3, 3, 2, 1, 0, -1, -2, -3, -3, -3, -2, -1 };
__constant__ int8_t c_ring_dy[16] = { 3, 3, 2, 1, 0, -1, -2, -3, -3, -3, -2, -1, 0, 1, 2, 3 };

// Positions i where bits i .. i+n-1 of d are all set, non-empty iff d holds a
// run of n ones (n <= 16).  R_{a+b} = R_a & (R_b >> a).
struct RunTest {
    int n;
    __device__ __forceinline__ bool operator()(uint32_t d) const
    {
        const uint32_t r1 = d, r2 = r1 & (r1 >> 1), r4 = r2 & (r2 >> 2), r8 = r4 & (r4 >> 4);
        const uint32_t r16 = r8 & (r8 >> 8);
        uint32_t acc = 0xFFFFFFFFu;
        int off = 0;
        if (n & 16) { acc &= r16 >> off; off += 16; }
        if (n & 8) { acc &= r8 >> off; off += 8; }
        if (n & 4) { acc &= r4 >> off; off += 4; }
        if (n & 2) { acc &= r2 >> off; off += 2; }
        if (n & 1) { acc &= r1 >> off; }
        return acc != 0;
    }
};

// Eq. 3 on one 16-bit ring mask: P_min <= longest circular run <= P_max.
// The ring is doubled into 32 bits so that circular runs become linear.
__device__ __forceinline__ bool bounded_run(uint32_t m, RunTest lo, RunTest hi, bool upper)
{
    const uint32_t d = m | (m << 16);
    return lo(d) && !(upper && hi(d));
}

struct FastSmem {
    int rwp, rh, tw, th, cells;
    __host__ __device__ static int align16(int v) { return (v + 15) & ~15; }
    __host__ __device__ int raw_bytes() const { return align16(rwp * rh); }
    __host__ __device__ int code_bytes() const { return align16(tw * th * 2); }
    __host__ __device__ int hi_bytes() const { return align16(cells); }
    __host__ __device__ int total(int k) const { return raw_bytes() + code_bytes() + hi_bytes() + cells * k * 4; }
};

__global__ void __launch_bounds__(kFastThreads) k_fast_cull(Batch b)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const int li = find_bucket(b.fast_tile_base, b.n_levels, blockIdx.x);
    const LevelDesc L = b.levels[li];
    const ImageDesc &I = b.images[L.image];
    const int k = b.prm.k, border = b.prm.border;
    const int t = blockIdx.x - b.fast_tile_base[li];
    const int ctas_x = (L.cells_x + L.bx - 1) / L.bx;
    const int ccx0 = (t % ctas_x) * L.bx, ccy0 = (t / ctas_x) * L.by;
    const int c = L.c;
    const int ncx = min(L.bx, L.cells_x - ccx0), ncy = min(L.by, L.cells_y - ccy0);
    const int x0 = ccx0 * c, y0 = ccy0 * c;
    const int tw = min(ncx * c, L.W - x0), th = min(ncy * c, L.H - y0);
    const int rw = tw + 6, rh = th + 6;

    FastSmem lay;
    lay.rwp = (rw + 3) & ~3; lay.rh = rh; lay.tw = tw; lay.th = th; lay.cells = ncx * ncy;
    uint8_t *rs = smem;
    uint16_t *code = reinterpret_cast<uint16_t *>(smem + lay.raw_bytes());
    uint8_t *has_hi = smem + lay.raw_bytes() + lay.code_bytes();
    uint32_t *sel = reinterpret_cast<uint32_t *>(smem + lay.raw_bytes() + lay.code_bytes() + lay.hi_bytes());
    const int rwp = lay.rwp;

    const uint8_t *raw = L.level == 0 ? b.in.ptr[L.image] : L.raw;
    const int pitch = L.level == 0 ? b.in.pitch[L.image] : L.pitch;
    for (int i = threadIdx.x; i < rw * rh; i += kFastThreads) {
        const int ry = i / rw, rx = i - ry * rw;
        const int gy = min(max(y0 - 3 + ry, 0), L.H - 1);
        const int gx = min(max(x0 - 3 + rx, 0), L.W - 1);
        rs[ry * rwp + rx] = __ldg(raw + (size_t)gy * pitch + gx);
    }
    for (int i = threadIdx.x; i < lay.cells; i += kFastThreads) has_hi[i] = 0;
    for (int i = threadIdx.x; i < lay.cells * k; i += kFastThreads) sel[i] = 0;
    __syncthreads();

    int ring[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) ring[q] = c_ring_dy[q] * rwp + c_ring_dx[q];
    const int eps = I.eps_hi, eps2 = I.eps_lo;
    const bool use_lo = eps2 > 0;
    const RunTest run_lo{b.prm.p_min}, run_hi{b.prm.p_max + 1};
    const bool upper = b.prm.p_max < 16;

    // CRF-matrix of the tile, packed: response | hi << 12 | lo << 13 (0 off-corner).
    for (int i = threadIdx.x; i < tw * th; i += kFastThreads) {
        const int py = i / tw, px = i - py * tw;
        const int gx = x0 + px, gy = y0 + py;
        uint32_t cd = 0;
        if (gx >= border && gx < L.W - border && gy >= border && gy < L.H - border) {
            const uint8_t *p = rs + (py + 3) * rwp + (px + 3);
            const int ic = p[0];
            uint32_t bb = 0, bd = 0, bb2 = 0, bd2 = 0;
            int r = 0;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int d = (int)p[ring[q]] - ic;
                bb |= (uint32_t)(d > eps) << q;
                bd |= (uint32_t)(d < -eps) << q;
                bb2 |= (uint32_t)(d > eps2) << q;
                bd2 |= (uint32_t)(d < -eps2) << q;
                r += abs(d);
            }
            const bool hi = bounded_run(bb, run_lo, run_hi, upper) || bounded_run(bd, run_lo, run_hi, upper);
            const bool lo = use_lo && (bounded_run(bb2, run_lo, run_hi, upper) || bounded_run(bd2, run_lo, run_hi, upper));
            if (hi || lo) cd = (uint32_t)r | ((uint32_t)hi << 12) | ((uint32_t)lo << 13);
            if (hi) has_hi[(py / c) * ncx + px / c] = 1;
        }
        code[i] = (uint16_t)cd;
    }
    __syncthreads();

    // Top-k per cell by key = response << 16 | (0xFFFF - index in cell): the
    // largest key is the strongest corner, ties resolved towards the smaller
    // y, then the smaller x.  Cells with a primary-threshold corner choose
    // among those only; the others fall back to the lower threshold.
    for (int j = 0; j < k; ++j) {
        for (int i = threadIdx.x; i < tw * th; i += kFastThreads) {
            const uint32_t cd = code[i];
            if (!cd) continue;
            const int py = i / tw, px = i - py * tw;
            const int cell = (py / c) * ncx + px / c;
            const bool ok = has_hi[cell] ? (cd & 0x1000u) : (cd & 0x2000u);
            if (!ok) continue;
            const uint32_t inidx = (uint32_t)((py % c) * c + (px % c));
            const uint32_t key = ((cd & 0xFFFu) << 16) | (0xFFFFu - inidx);
            if (j == 0 || key < sel[cell * k + j - 1]) atomicMax(&sel[cell * k + j], key);
        }
        __syncthreads();
    }

    // Store the cell slots and scatter survivors into the s0 score map.
    for (int e = threadIdx.x; e < lay.cells * k; e += kFastThreads) {
        const int cell = e / k, j = e - cell * k;
        const int gcx = ccx0 + cell % ncx, gcy = ccy0 + cell / ncx;
        const uint32_t key = sel[e];
        b.slots[L.slot_base + (gcy * L.cells_x + gcx) * k + j] = key;
        if (key) {
            const int inidx = 0xFFFF - (int)(key & 0xFFFFu);
            const int x = gcx * c + inidx % c, y = gcy * c + inidx / c;
            if (x >= L.W || y >= L.H) { atomicOr(b.err, kErrDecode); continue; }
            const int X = __ldg(L.projx + x), Y = __ldg(L.projy + y);
            atomicAdd(I.map + (size_t)Y * I.W0 + X, (1u << 16) + (key >> 16));
        }
    }
}

int fast_smem_bytes(int tw, int th, int cells, int k)
{
    FastSmem lay;
    lay.rwp = (tw + 6 + 3) & ~3; lay.rh = th + 6; lay.tw = tw; lay.th = th; lay.cells = cells;
    return lay.total(k);
}

cudaError_t launch_fast_cull(const Batch &b, cudaStream_t stream)
{
    if (b.fast_tiles == 0) return cudaSuccess;
    k_fast_cull<<<b.fast_tiles, kFastThreads, b.fast_smem, stream>>>(b);
    return cudaGetLastError();
}

cudaError_t configure_kernels()
{
    return cudaFuncSetAttribute(k_fast_cull, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

}  // namespace jslam
