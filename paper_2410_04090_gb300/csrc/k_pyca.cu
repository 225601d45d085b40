// Pyramidal Feature Aggregation, steps 3 and the aggregation (Sec. II-C-2).
//
// k_pfa_nms       one CTA per segment = (image, level, cell row), or one warp
//                 per segment (four per CTA) when every segment of the batch
//                 has at most 96 slots.  Each
//                 culled corner reads its own packed (K_l, K_r) and those of
//                 the q x q window around its s0 projection from the score map
//                 filled by the detection kernel, and is suppressed when a
//                 neighbour dominates it (sparse NMS: only occupied pixels are
//                 looked at).  Survivors are ranked by (y, x) inside the
//                 segment; segments of one level are already in y order.
// k_pfa_finalize  one CTA per image: prefix-sums the segment counts into
//                 canonical positions (level, y, x), clears the score map
//                 entries it used, applies the keypoint cap by a radix select
//                 on (K_l, K_r, response) with canonical order breaking ties,
//                 and writes the compacted keypoint list.
#include "jslam_internal.h"

namespace jslam {

struct SlotPos {
    int x, y, r;
};

__device__ __forceinline__ SlotPos decode_slot(uint32_t key, int rel, int cells_x, int c, int k)
{
    const int cell = rel / k;
    const int cy = cell / cells_x, cx = cell - cy * cells_x;
    const int inidx = 0xFFFF - (int)(key & 0xFFFFu);
    SlotPos p;
    p.x = cx * c + inidx % c;
    p.y = cy * c + inidx / c;
    p.r = (int)(key >> 16);
    return p;
}

__global__ void __launch_bounds__(kNmsThreads) k_pfa_nms(Batch b)
{
    __shared__ uint32_t sk[kMaxSegment];
    __shared__ int alive_total;
    const int seg = blockIdx.x;
    const LevelDesc L = b.levels[b.seg_level[seg]];
    const ImageDesc &I = b.images[L.image];
    const int k = b.prm.k, rad = b.prm.nms_rad, rule = b.prm.rule;
    const int cy = seg - L.seg_base;
    const int m = L.cells_x * k;
    if (m > kMaxSegment) {
        if (threadIdx.x == 0) { atomicOr(b.err, kErrSegment); b.seg_count[seg] = 0; }
        return;
    }
    const int base = L.slot_base + cy * m;
    if (threadIdx.x == 0) alive_total = 0;
    __syncthreads();
    int my_alive = 0;
    for (int i = threadIdx.x; i < m; i += kNmsThreads) {
        const uint32_t key = b.slots[base + i];
        uint32_t v = 0xFFFFFFFFu;
        if (key) {
            const SlotPos p = decode_slot(key, cy * m + i, L.cells_x, L.c, k);
            const int X = __ldg(L.projx + p.x), Y = __ldg(L.projy + p.y);
            const uint32_t own = I.map[(size_t)Y * I.W0 + X];
            const uint32_t kl = own >> 16, kr = own & 0xFFFFu;
            bool dom = false;
            for (int dy = -rad; dy <= rad; ++dy) {
                const int qy = Y + dy;
                if (qy < 0 || qy >= I.H0) continue;
                for (int dx = -rad; dx <= rad; ++dx) {
                    const int qx = X + dx;
                    if ((dx | dy) == 0 || qx < 0 || qx >= I.W0) continue;
                    const uint32_t w = I.map[(size_t)qy * I.W0 + qx];
                    if (!w) continue;
                    const uint32_t ql = w >> 16, qr = w & 0xFFFFu;
                    dom |= rule == 0 ? (ql > kl && qr > kr) : (ql > kl || (ql == kl && qr > kr));
                }
            }
            b.slot_k[base + i] = own;
            if (!dom) { v = ((uint32_t)p.y << 16) | (uint32_t)p.x; ++my_alive; }
        }
        sk[i] = v;
    }
    if (my_alive) atomicAdd(&alive_total, my_alive);
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += kNmsThreads) {
        const uint32_t v = sk[i];
        int rank = -1;
        if (v != 0xFFFFFFFFu) {
            rank = 0;
            for (int j = 0; j < m; ++j) rank += sk[j] < v;
        }
        b.slot_rank[base + i] = rank;
    }
    if (threadIdx.x == 0) b.seg_count[seg] = alive_total;
}

// The same per segment with one warp, for batches whose segments (cell rows:
// cells_x x k slots) all have at most 32 S slots: lane l takes slots l,
// l + 32, ..., and every step of their chains of dependent loads (slot ->
// projection -> own score -> neighbours) is issued for all S slots before
// the next, so the chains overlap; a CTA of four warps takes four segments.
template <int S>
__global__ void __launch_bounds__(kNmsThreads) k_pfa_nms_warp(Batch b)
{
    __shared__ uint32_t sk[kNmsThreads / 32][32 * S];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int seg = blockIdx.x * (kNmsThreads / 32) + warp;
    if (seg >= b.n_segments) return;  // whole warps only
    const LevelDesc &L = b.levels[b.seg_level[seg]];
    const ImageDesc &I = b.images[L.image];
    const int k = b.prm.k, rad = b.prm.nms_rad, rule = b.prm.rule;
    const int cy = seg - L.seg_base;
    const int m = L.cells_x * k;
    if (m > 32 * S) {  // the host launches this kernel only when no segment is wider
        if (lane == 0) { atomicOr(b.err, kErrSegment); b.seg_count[seg] = 0; }
        return;
    }
    const int base = L.slot_base + cy * m;
    const int W0 = I.W0, H0 = I.H0;
    uint32_t key[S], own[S];
    int X[S], Y[S], px[S], py[S];
    bool dom[S];
#pragma unroll
    for (int q = 0; q < S; ++q) key[q] = lane + 32 * q < m ? b.slots[base + lane + 32 * q] : 0u;
#pragma unroll
    for (int q = 0; q < S; ++q) {
        X[q] = Y[q] = px[q] = py[q] = 0;
        if (key[q]) {
            const SlotPos p = decode_slot(key[q], cy * m + lane + 32 * q, L.cells_x, L.c, k);
            px[q] = p.x; py[q] = p.y;
            X[q] = __ldg(L.projx + p.x);
            Y[q] = __ldg(L.projy + p.y);
        }
    }
#pragma unroll
    for (int q = 0; q < S; ++q) {
        own[q] = key[q] ? I.map[(size_t)Y[q] * W0 + X[q]] : 0u;
        dom[q] = false;
    }
    for (int dy = -rad; dy <= rad; ++dy)
        for (int dx = -rad; dx <= rad; ++dx) {
            if ((dx | dy) == 0) continue;
            uint32_t w[S];
#pragma unroll
            for (int q = 0; q < S; ++q) {
                const int qx = X[q] + dx, qy = Y[q] + dy;
                w[q] = key[q] && qx >= 0 && qx < W0 && qy >= 0 && qy < H0 ? I.map[(size_t)qy * W0 + qx] : 0u;
            }
#pragma unroll
            for (int q = 0; q < S; ++q)
                if (w[q]) {
                    const uint32_t ql = w[q] >> 16, qr = w[q] & 0xFFFFu, kl = own[q] >> 16, kr = own[q] & 0xFFFFu;
                    dom[q] |= rule == 0 ? (ql > kl && qr > kr) : (ql > kl || (ql == kl && qr > kr));
                }
        }
    uint32_t v[S];
    int alive = 0;
#pragma unroll
    for (int q = 0; q < S; ++q) {
        v[q] = 0xFFFFFFFFu;
        if (key[q]) {
            b.slot_k[base + lane + 32 * q] = own[q];
            if (!dom[q]) { v[q] = ((uint32_t)py[q] << 16) | (uint32_t)px[q]; ++alive; }
        }
        sk[warp][lane + 32 * q] = v[q];
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < S; ++q)
        if (lane + 32 * q < m) {
            int rank = -1;
            if (v[q] != 0xFFFFFFFFu) {
                rank = 0;
                for (int j = 0; j < m; ++j) rank += sk[warp][j] < v[q];
            }
            b.slot_rank[base + lane + 32 * q] = rank;
        }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) alive += __shfl_xor_sync(0xFFFFFFFFu, alive, off);
    if (lane == 0) b.seg_count[seg] = alive;
}

cudaError_t launch_pfa_nms(const Batch &b, cudaStream_t stream)
{
    if (b.n_segments == 0) return cudaSuccess;
    constexpr int per = kNmsThreads / 32;
    if (b.nms_kernel == 1) {
        k_pfa_nms<<<b.n_segments, kNmsThreads, 0, stream>>>(b);
    } else if (b.max_segment <= 32) {
        k_pfa_nms_warp<1><<<(b.n_segments + per - 1) / per, kNmsThreads, 0, stream>>>(b);
    } else if (b.max_segment <= 64) {
        k_pfa_nms_warp<2><<<(b.n_segments + per - 1) / per, kNmsThreads, 0, stream>>>(b);
    } else if (b.max_segment <= 96) {
        k_pfa_nms_warp<3><<<(b.n_segments + per - 1) / per, kNmsThreads, 0, stream>>>(b);
    } else {
        k_pfa_nms<<<b.n_segments, kNmsThreads, 0, stream>>>(b);
    }
    return cudaGetLastError();
}

// Exclusive block-wide prefix sum of v; *total receives the block sum.
template <int NT>
__device__ __forceinline__ int block_excl_scan(int v, int *ws, int *total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = lane < NT / 32 ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < NT / 32) ws[lane] = s;
    }
    __syncthreads();
    const int pre = w > 0 ? ws[w - 1] : 0;
    *total = ws[NT / 32 - 1];
    __syncthreads();
    return pre + x - v;
}

// Cap priorities of the first kFinPrioCache canonical survivors, kept in
// shared memory for the four radix passes and the compaction (32 KB; two
// CTAs still fit an SM).  Images with more survivors read the rest through
// their slots.
constexpr int kFinPrioCache = 8192;

// Row index of an image's canonical list, for the stereo matching (all
// threads of the finalisation's CTA, after its barrier: the keypoints'
// levels and Y and the level starts in lstart, kMaxLevels + 1 entries whose
// last is the count, are complete).  Entry v of level l's table is the
// first index of the level whose Y is >= v, else the level's end: keypoint
// j owns the entries (Y[j - 1], Y[j]] when it is not the level's first;
// the entries up to the first keypoint's Y (the level's start) and after
// the last one's (its end) are spread over the CTA.  Every level with
// keypoints gets all H0 + 1 entries.  Not inlined: its registers stay out
// of the finalisation's allocation.
__device__ __noinline__ void fill_row_index(const ImageDesc &I, const int *lstart)
{
    const int rows = I.H0 + 1, keep = lstart[kMaxLevels];
    const KpOut &o = I.out;
    for (int j = threadIdx.x; j < keep; j += kFinThreads) {
        const int l = o.level[j];
        if (j == lstart[l]) continue;
        const int Yj = o.Y[j];
        int32_t *rf = I.row_first + (size_t)l * rows;
        for (int v = (int)o.Y[j - 1] + 1; v <= Yj; ++v) rf[v] = j;
    }
    for (int t = threadIdx.x; t < I.levels * rows; t += kFinThreads) {
        const int l = t / rows, v = t - l * rows;
        const int s = lstart[l], e = lstart[l + 1];
        if (s == e) continue;
        if (v <= (int)o.Y[s]) I.row_first[t] = s;
        else if (v > (int)o.Y[e - 1]) I.row_first[t] = e;
    }
}

__global__ void __launch_bounds__(kFinThreads, 2) k_pfa_finalize(Batch b)
{
    __shared__ uint32_t s_prio[kFinPrioCache];
    __shared__ int ws[32];
    __shared__ int hist[256];
    __shared__ int sh_digit, sh_need;
    __shared__ int lstart[kMaxLevels + 1];
    __shared__ LevelDesc levs[kMaxLevels];
    const int img = blockIdx.x;
    const ImageDesc &I = b.images[img];
    const int k = b.prm.k;
    const int nl = I.levels;
    if (threadIdx.x < nl) levs[threadIdx.x] = b.levels[I.level_base + threadIdx.x];
    __syncthreads();

    // Canonical offsets of the segments (level-major, then cell row).
    int carry = 0;
    for (int base = 0; base < I.seg_count; base += kFinThreads) {
        const int i = base + threadIdx.x;
        const int v = i < I.seg_count ? b.seg_count[I.seg_base + i] : 0;
        int tot;
        const int ex = block_excl_scan<kFinThreads>(v, ws, &tot);
        if (i < I.seg_count) b.seg_off[I.seg_base + i] = carry + ex;
        carry += tot;
    }
    const int S = carry;
    __syncthreads();

    // Canonical position of every survivor; clear the map entries.
    for (int s = threadIdx.x; s < I.slot_count; s += kFinThreads) {
        const int gs = I.slot_base + s;
        const uint32_t key = b.slots[gs];
        if (!key) continue;
        int l = nl - 1;
        while (l > 0 && levs[l].slot_base > gs) --l;
        const LevelDesc &L = levs[l];
        const int rel = gs - L.slot_base;
        const SlotPos p = decode_slot(key, rel, L.cells_x, L.c, k);
        I.map[(size_t)__ldg(L.projy + p.y) * I.W0 + __ldg(L.projx + p.x)] = 0;
        const int rank = b.slot_rank[gs];
        if (rank >= 0) {
            const int cy = rel / (L.cells_x * k);
            b.canon[I.slot_base + b.seg_off[L.seg_base + cy] + rank] = gs;
        }
    }
    __syncthreads();

    // Cap: keep the max_feats largest priorities P = K_l << 27 | K_r << 12 | r,
    // ties at the threshold resolved in canonical order.
    auto prio = [&](int g) -> uint32_t {
        const int gs = b.canon[I.slot_base + g];
        const uint32_t K = b.slot_k[gs];
        return ((K >> 16) << 27) | ((K & 0xFFFFu) << 12) | (b.slots[gs] >> 16);
    };
    for (int g = threadIdx.x; g < min(S, kFinPrioCache); g += kFinThreads) s_prio[g] = prio(g);
    __syncthreads();
    auto prio_c = [&](int g) -> uint32_t { return g < kFinPrioCache ? s_prio[g] : prio(g); };
    const bool capped = S > I.max_feats;
    uint32_t T = 0;
    int quota = 0;
    if (capped) {
        int need = I.max_feats;
        uint32_t prefix = 0, mask = 0;
        for (int sh = 24; sh >= 0; sh -= 8) {
            for (int i = threadIdx.x; i < 256; i += kFinThreads) hist[i] = 0;
            __syncthreads();
            for (int g = threadIdx.x; g < S; g += kFinThreads) {
                const uint32_t P = prio_c(g);
                if ((P & mask) == prefix) atomicAdd(&hist[(P >> sh) & 255u], 1);
            }
            __syncthreads();
            // the largest digit d whose count, added to the counts of the
            // larger digits, reaches `need` (which never exceeds the total):
            // lane l holds digits 255 - 8 l down to 248 - 8 l, a warp scan
            // gives the counts above each lane, and the one lane where the
            // running count crosses `need` walks its eight digits
            if (threadIdx.x < 32) {
                const int lane = threadIdx.x;
                int cnt8[8], s8 = 0;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    cnt8[j] = hist[255 - 8 * lane - j];
                    s8 += cnt8[j];
                }
                int incl = s8;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                    if (lane >= o) incl += y;
                }
                int cum = incl - s8;
                if (cum < need && incl >= need) {
                    int j = 0;
                    for (; j < 7; ++j) {
                        if (cum + cnt8[j] >= need) break;
                        cum += cnt8[j];
                    }
                    sh_digit = 255 - 8 * lane - j;
                    sh_need = need - cum;
                }
            }
            __syncthreads();
            prefix |= (uint32_t)sh_digit << sh;
            mask |= 255u << sh;
            need = sh_need;
            __syncthreads();
        }
        T = prefix;
        quota = need;
    }
    const int keep = capped ? I.max_feats : S;
    if (threadIdx.x <= kMaxLevels) lstart[threadIdx.x] = keep;
    __syncthreads();

    int carry_tie = 0, carry_out = 0;
    const KpOut &o = I.out;
    for (int base = 0; base < S; base += kFinThreads) {
        const int g = base + threadIdx.x;
        const bool valid = g < S;
        const uint32_t P = valid ? prio_c(g) : 0u;
        int tot;
        const int tie_rank = carry_tie + block_excl_scan<kFinThreads>(valid && capped && P == T, ws, &tot);
        carry_tie += tot;
        const bool kept = valid && (!capped || P > T || (P == T && tie_rank < quota));
        const int oi = carry_out + block_excl_scan<kFinThreads>(kept, ws, &tot);
        carry_out += tot;
        if (kept) {
            const int gs = b.canon[I.slot_base + g];
            int l = nl - 1;
            while (l > 0 && levs[l].slot_base > gs) --l;
            const LevelDesc &L = levs[l];
            const uint32_t key = b.slots[gs];
            const SlotPos p = decode_slot(key, gs - L.slot_base, L.cells_x, L.c, k);
            const uint32_t K = b.slot_k[gs];
            o.x[oi] = (uint16_t)p.x;
            o.y[oi] = (uint16_t)p.y;
            o.X[oi] = __ldg(L.projx + p.x);
            o.Y[oi] = __ldg(L.projy + p.y);
            o.level[oi] = (uint8_t)l;
            o.response[oi] = (uint16_t)p.r;
            o.k_levels[oi] = (uint8_t)(K >> 16);
            o.k_resp[oi] = K & 0xFFFFu;
            atomicMin(&lstart[l], oi);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int l = kMaxLevels - 1; l >= 0; --l) lstart[l] = min(lstart[l], lstart[l + 1]);
        for (int l = 0; l <= kMaxLevels; ++l) I.level_start[l] = lstart[l];
        *I.count = keep;
        *I.count_hdr = keep;
    }
    __syncthreads();
    fill_row_index(b.images[img], lstart);
}

cudaError_t launch_pfa_finalize(const Batch &b, cudaStream_t stream)
{
    if (b.n_images == 0) return cudaSuccess;
    k_pfa_finalize<<<b.n_images, kFinThreads, 0, stream>>>(b);
    return cudaGetLastError();
}

}  // namespace jslam
