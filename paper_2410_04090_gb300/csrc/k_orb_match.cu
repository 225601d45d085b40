// ORB extraction for all scales at once and stereo row matching (Sec. III:
// streamlined multiscale detection and extraction; middle-end stereo
// matching by descriptor-distance minimisation).
//
// k_orient_desc  one warp per keypoint of any image and level.  The lanes
//                read the radius-15 disk of the raw level as aligned words
//                (9 per row) and accumulate the intensity moments m10, m01
//                with byte dot products over the bytes inside the disk; they
//                stage the 27 x 27 blurred patch the BRIEF pattern reaches in
//                shared memory the same way (8 words per row); lanes 0..29 each test
//                one sector boundary (float with an error margin, IEEE double
//                with explicit rounding inside it, so the sector equals the
//                one the host-side definition gives); the 256 BRIEF
//                comparisons read the patch 32 at a time and are packed into
//                words by a ballot.
// k_match        one warp per left keypoint: for each right level within one
//                of the keypoint's level, takes the s0 row band of the
//                canonical (level, y, x) list (Y is non-decreasing in y) from
//                the row index (two independent loads per level), scans the
//                band with the lanes, and keeps the smallest (Hamming
//                distance, disparity, index) by a warp min-reduction.
#include "jslam_internal.h"

namespace jslam {

constexpr int kPatW = 2 * kPatR + 1;      // 27
constexpr int kDiskWords = 9;             // aligned words covering the 31 disk columns of a row
// largest |dx| with dx^2 + dy^2 <= kDiskR^2, by |dy|
__constant__ int8_t c_disk_umax[kDiskR + 1] = { 15, 14, 14, 14, 14, 14, 13, 13, 12, 12, 11, 10, 9, 7, 5, 0 };

__global__ void __launch_bounds__(256) k_orient_desc(Batch b)
{
    __shared__ __align__(16) uint8_t s_patch[8][kPatW * kPatPitch];
    const int img = blockIdx.y;
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
    const ImageDesc &I = b.images[img];
    if (i >= *I.count) return;
    const KpOut &o = I.out;
    const int lvl = o.level[i], x = o.x[i], y = o.y[i];
    const LevelDesc &L = b.levels[I.level_base + lvl];
    const uint8_t *raw = L.raw;
    const int pitch = L.pitch;
    const int bpitch = L.blur_pitch;
    uint8_t *patch = s_patch[threadIdx.x >> 5];

    // The keypoint is at least `border` (>= 16) from every edge, so the
    // 31 x 31 square of the moment disk and the 27 x 27 patch of the BRIEF
    // pattern are inside the level.  Both are read as aligned 32-bit words
    // (rows start on 128-byte boundaries; a row's last word may reach 3
    // bytes past the level's width, into the pitch or the buffer's slack),
    // every load independent of the others.
    // Patch: 27 rows x 8 words from word column (x - 13) / 4 of the blurred
    // level, staged with a pitch of 32 bytes.
    const int pw0 = (x - kPatR) >> 2;
    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(L.blur + (size_t)(y - kPatR) * bpitch) + pw0;
        uint32_t *dst = reinterpret_cast<uint32_t *>(patch);
#pragma unroll
        for (int k = 0; k < (kPatW * 8 + 31) / 32; ++k) {
            const int it = k * 32 + lane;
            if (it < kPatW * 8) {
                const int r = it >> 3, w = it & 7;
                dst[it] = __ldg(src + (size_t)r * (bpitch >> 2) + w);
            }
        }
    }
    // Disk moments: 31 rows x 9 words from word column (x - 15) / 4 of the
    // raw level.  Lane l < 27 keeps word column l mod 9 and takes rows
    // l / 9, l / 9 + 3, ...; per word, the bytes inside the disk
    // (|dx| <= umax(|dy|)) are kept and two byte dot products give the row
    // sum and the sum of (dx + 18) I (weights 3..36, unsigned, fixed per
    // lane); m10 = that - 18 sum I.
    int m10 = 0, m01 = 0;
    if (lane < 3 * kDiskWords) {
        const int dw0 = (x - kDiskR) >> 2;
        const int w = lane % kDiskWords, r0 = lane / kDiskWords;
        const int cx0 = 4 * (dw0 + w) - x;  // dx of the word's byte 0
        const uint32_t wdx = (uint32_t)(cx0 + 18) * 0x01010101u + 0x03020100u;
        const uint32_t *src = reinterpret_cast<const uint32_t *>(raw + (size_t)(y - kDiskR + r0) * pitch) + dw0 + w;
        const size_t step = (size_t)3 * (pitch >> 2);
        int s = 0, sw = 0;
#pragma unroll
        for (int k = 0; k < (2 * kDiskR + 1 + 2) / 3; ++k) {
            const int r = r0 + 3 * k;
            if (r <= 2 * kDiskR) {
                const uint32_t v = __ldg(src + k * step);
                const int dy = r - kDiskR;
                const int um = c_disk_umax[abs(dy)];
                const int lo = max(-um - cx0, 0), hi = min(um - cx0, 3);
                const uint32_t mask = hi < lo ? 0u : (0xFFFFFFFFu >> (24 - 8 * (hi - lo))) << (8 * lo);
                const uint32_t vm = v & mask;
                const int rs = (int)__dp4a(vm, 0x01010101u, 0u);
                s += rs;
                m01 += dy * rs;
                sw += (int)__dp4a(vm, wdx, 0u);
            }
        }
        m10 = sw - 18 * s;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        m10 += __shfl_xor_sync(0xFFFFFFFFu, m10, off);
        m01 += __shfl_xor_sync(0xFFFFFFFFu, m01, off);
    }

    // Sector b is the one whose lower boundary has the moment vector on its
    // left (m01 cos - m10 sin >= 0 in IEEE double) and whose upper boundary
    // does not.  The test runs in float first: |m| < 2^24 is exact, and the
    // float result is within (|m01| + |m10|) 2^-22 of the exact value with
    // the double table entries, so outside 2^-20 times that its sign is the
    // double test's; lanes inside the margin (rare) take the double test.
    bool left_of = false;
    if (lane < kBins) {
        const float fa = (float)m01, fb = (float)m10;
        const float t = __fsub_rn(__fmul_rn(fa, __ldg(b.bin_cosf + lane)), __fmul_rn(fb, __ldg(b.bin_sinf + lane)));
        const float margin = (fabsf(fa) + fabsf(fb)) * 0x1p-20f;
        if (fabsf(t) > margin) {
            left_of = t > 0.0f;
        } else {
            const double t1 = __dmul_rn((double)m01, b.bin_cos[lane]);
            const double t2 = __dmul_rn((double)m10, b.bin_sin[lane]);
            left_of = __dsub_rn(t1, t2) >= 0.0;
        }
    }
    const uint32_t S = __ballot_sync(0xFFFFFFFFu, left_of) & ((1u << kBins) - 1u);
    const uint32_t next = (S >> 1) | ((S & 1u) << (kBins - 1));
    const uint32_t T = S & ~next & ((1u << kBins) - 1u);
    const bool zero = (m10 == 0 && m01 == 0);
    const int bin = (zero || T == 0) ? 0 : __ffs(T) - 1;

    __syncwarp();  // the patch is complete
    const uint32_t *pat = b.pattern_off + (size_t)bin * kPairs;
    const uint8_t *centre = patch + kPatR * kPatPitch + (x - kPatR - 4 * pw0) + kPatR;
    uint32_t myword = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        const uint32_t o = __ldg(pat + w * 32 + lane);  // offsets of p and q in the staged patch
        const int a = centre[(int16_t)(o & 0xFFFFu)];
        const int c = centre[(int16_t)(o >> 16)];
        const uint32_t word = __ballot_sync(0xFFFFFFFFu, a < c);
        if (lane == w) myword = word;
    }
    if (lane < 8) o.desc[(size_t)i * 8 + lane] = myword;
    if (lane == 0) {
        o.angle[i] = zero ? 0.0f : atan2f((float)m01, (float)m10);
        o.angle_bin[i] = (uint8_t)bin;
    }
}

cudaError_t launch_orient_desc(const Batch &b, cudaStream_t stream)
{
    if (b.n_images == 0 || b.max_capacity == 0) return cudaSuccess;
    dim3 grid((b.max_capacity + 7) / 8, b.n_images);
    k_orient_desc<<<grid, 256, 0, stream>>>(b);
    return cudaGetLastError();
}

// Eight CTAs per SM (32 registers): the kernel waits on gathers from L2, and
// the fuller SM hides more of them than the spill of the eight descriptor
// words costs (0.148 -> 0.123 ms per KITTI-shaped launch).
__global__ void __launch_bounds__(256, 8) k_match(Batch b)
{
    const int pair = blockIdx.y;
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
    const PairDesc &P = b.pairs[pair];
    const ImageDesc &Il = b.images[P.left];
    const ImageDesc &Ir = b.images[P.right];
    if (i >= *Il.count) return;
    const KpOut &ol = Il.out, &orr = Ir.out;
    const int n = ol.level[i];
    const int X = ol.X[i], Y = ol.Y[i];
    const int band = b.levels[Il.level_base + n].band;
    uint32_t dl[8];
#pragma unroll
    for (int w = 0; w < 8; ++w) dl[w] = ol.desc[(size_t)i * 8 + w];

    unsigned long long best = ~0ull;
    const int m_lo = max(0, n - 1), m_hi = min(Ir.levels - 1, n + 1);
    // the band [Y - band, Y + band] of each level: lower bounds of Y - band
    // and Y + band + 1 from the row index (rows clamped to [0, H0]; a level
    // without keypoints has an empty band and an unwritten table)
    const int va = min(max(Y - band, 0), Ir.H0), vz = min(max(Y + band + 1, 0), Ir.H0);
    int ra[3], rz[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int m = m_lo + q;
        ra[q] = rz[q] = 0;
        if (m <= m_hi) {
            const int s = __ldg(Ir.level_start + m), e = __ldg(Ir.level_start + m + 1);
            const int32_t *rf = Ir.row_first + (size_t)m * (Ir.H0 + 1);
            ra[q] = e > s ? __ldg(rf + va) : s;
            rz[q] = e > s ? __ldg(rf + vz) : s;
        }
    }
    // the three bands as one run of candidates over the lanes (a band of a
    // level outside the frame, or of an empty level, is empty), so a few
    // dozen candidates take one pass of loads, not one per level
    const int c0 = rz[0] - ra[0], c01 = c0 + (rz[1] - ra[1]), T = c01 + (rz[2] - ra[2]);
    for (int t = lane; t < T; t += 32) {
        const int j = t < c0 ? ra[0] + t : (t < c01 ? ra[1] + (t - c0) : ra[2] + (t - c01));
        const int disp = X - (int)orr.X[j];
        if (disp < 0 || disp > b.prm.max_disp) continue;
        const uint4 *dr = reinterpret_cast<const uint4 *>(orr.desc + (size_t)j * 8);
        const uint4 r0 = dr[0], r1 = dr[1];
        const int d = __popc(dl[0] ^ r0.x) + __popc(dl[1] ^ r0.y) + __popc(dl[2] ^ r0.z) +
                      __popc(dl[3] ^ r0.w) + __popc(dl[4] ^ r1.x) + __popc(dl[5] ^ r1.y) +
                      __popc(dl[6] ^ r1.z) + __popc(dl[7] ^ r1.w);
        const unsigned long long key = ((unsigned long long)d << 48) |
                                       ((unsigned long long)disp << 32) | (unsigned)j;
        best = key < best ? key : best;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xFFFFFFFFu, best, off);
        best = other < best ? other : best;
    }
    if (lane == 0) {
        if (best == ~0ull) {
            P.match_idx[i] = -1; P.disparity[i] = 0; P.dist[i] = 0xFFFF;
        } else {
            const int d = (int)(best >> 48);
            if (d <= b.prm.max_dist) {
                P.match_idx[i] = (int)(best & 0xFFFFFFFFu);
                P.disparity[i] = (int16_t)((best >> 32) & 0xFFFFu);
                P.dist[i] = (uint16_t)d;
            } else {
                P.match_idx[i] = -1; P.disparity[i] = 0; P.dist[i] = (uint16_t)d;
            }
        }
    }
}

// Feature tracking by projection (middle-end): one warp per query.  For each
// level of the band the row index narrows the frame's canonical list to a
// conservative Y range; lanes take the exact float window test and the
// Hamming distance, and a warp reduction keeps the smallest (distance,
// index) and the second-smallest distance.
__global__ void __launch_bounds__(256) k_track(Batch b, TrackArgs a)
{
    const int lane = threadIdx.x & 31;
    const int q = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (q >= a.n) return;
    const ImageDesc &I = b.images[a.image];
    const int lv = a.level[q];
    unsigned long long best = ~0ull;   // distance << 32 | index
    uint32_t second = 0xFFFFFFFFu;
    // the band lv - 1 .. lv + 1 clipped to the frame's levels: a query one
    // level past the deepest meets that level (its window scaled by
    // zeta^lv), a deeper one meets none
    if (lv <= kMaxLevels) {
        const float u = a.u[q], v = a.v[q];
        const float r = __fmul_rn(a.radius, a.zeta_f[lv]);
        uint32_t dq[8];
#pragma unroll
        for (int w = 0; w < 8; ++w) dq[w] = __ldg(a.desc + (size_t)q * 8 + w);
        const KpOut &o = I.out;
        const int m_lo = max(0, lv - 1), m_hi = min(I.levels - 1, lv + 1);
        const int ylo = (int)floorf(v - r) - 1, yhi = (int)ceilf(v + r) + 1;  // covers every Y that can pass
        // rows of the row index, clamped to [0, H0] (64-bit: yhi may be INT_MAX)
        const int va = (int)min(max((long long)ylo, 0ll), (long long)I.H0);
        const int vz = (int)min(max((long long)yhi + 1, 0ll), (long long)I.H0);
        for (int m = m_lo; m <= m_hi; ++m) {
            const int s = I.level_start[m], e = I.level_start[m + 1];
            const int32_t *rf = I.row_first + (size_t)m * (I.H0 + 1);
            const int z0 = e > s ? __ldg(rf + va) : s;
            const int z1 = e > s ? max(__ldg(rf + vz), z0) : s;
            for (int j = z0 + lane; j < z1; j += 32) {
                const float dx = __fsub_rn((float)o.X[j], u), dy = __fsub_rn((float)o.Y[j], v);
                if (fabsf(dx) > r || fabsf(dy) > r) continue;
                const uint4 *dr = reinterpret_cast<const uint4 *>(o.desc + (size_t)j * 8);
                const uint4 r0 = dr[0], r1 = dr[1];
                const uint32_t d = __popc(dq[0] ^ r0.x) + __popc(dq[1] ^ r0.y) + __popc(dq[2] ^ r0.z) +
                                   __popc(dq[3] ^ r0.w) + __popc(dq[4] ^ r1.x) + __popc(dq[5] ^ r1.y) +
                                   __popc(dq[6] ^ r1.z) + __popc(dq[7] ^ r1.w);
                const unsigned long long key = ((unsigned long long)d << 32) | (unsigned)j;
                if (key < best) {
                    second = min(second, (uint32_t)(best >> 32));
                    best = key;
                } else {
                    second = min(second, d);
                }
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long ob = __shfl_xor_sync(0xFFFFFFFFu, best, off);
            const uint32_t os = __shfl_xor_sync(0xFFFFFFFFu, second, off);
            const unsigned long long lo = ob < best ? ob : best, hi = ob < best ? best : ob;
            second = min(min(second, os), (uint32_t)(hi >> 32));
            best = lo;
        }
    }
    if (lane == 0) {
        if (best == ~0ull) {
            a.out_idx[q] = -1;
            a.out_dist[q] = 0xFFFF;
        } else {
            const uint32_t d = (uint32_t)(best >> 32);
            const bool ok = (int)d <= a.max_dist && (second == 0xFFFFFFFFu || 10u * d <= 9u * second);
            a.out_idx[q] = ok ? (int)(best & 0xFFFFFFFFu) : -1;
            a.out_dist[q] = (uint16_t)d;
        }
    }
}

cudaError_t launch_track(const Batch &b, const TrackArgs &a, cudaStream_t stream)
{
    if (a.n == 0) return cudaSuccess;
    k_track<<<(a.n + 7) / 8, 256, 0, stream>>>(b, a);
    return cudaGetLastError();
}

cudaError_t launch_match(const Batch &b, cudaStream_t stream)
{
    if (b.n_pairs == 0 || b.max_capacity == 0) return cudaSuccess;
    dim3 grid((b.max_capacity + 7) / 8, b.n_pairs);
    k_match<<<grid, 256, 0, stream>>>(b);
    return cudaGetLastError();
}

}  // namespace jslam
