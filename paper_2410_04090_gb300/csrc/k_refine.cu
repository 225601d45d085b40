// Correlation minimisation of the stereo matches (Sec. III, middle-end
// stereo matching): sub-pixel disparity and depth of every accepted
// descriptor match.
//
// k_refine         one warp per left keypoint.  The (2w+1)^2 left patch and
//                  the (2w+1) x (2w+2L+1) right strip on the keypoint's level
//                  are staged in shared memory (lanes on consecutive
//                  columns); lanes 0..2(2L+1)-1 each sum the centre-normalised
//                  absolute differences of one shift over half of the rows,
//                  a shuffle adds the halves, a warp minimum picks the first
//                  minimum shift, and lane 0 takes the decisions in integers
//                  and computes delta, disparity and depth in float (the
//                  host-side definition's doubles to a few float ulps; the
//                  FP64 pipe is a small fraction of the FP32 rate here).
// k_refine_median  one CTA per pair: the median SAD of the surviving matches
//                  by a three-pass 8-bit radix select, then the matches above
//                  2.1 times it are rejected.
#include "jslam_internal.h"

namespace jslam {

constexpr int kRefW = kRefineMaxW, kRefL = kRefineMaxL;
constexpr int kRefLeft = (2 * kRefW + 1) * (2 * kRefW + 1);
constexpr int kRefRight = (2 * kRefW + 1) * (2 * kRefW + 2 * kRefL + 1);

// WC > 0: the window half-size fixed at compile time (the default 5), so the
// SAD loops unroll; WC == 0: any half-size given at run time.
template <int WC>
__global__ void __launch_bounds__(256) k_refine(Batch b, int w_rt, int L, double bf)
{
    const int w = WC > 0 ? WC : w_rt;
    __shared__ uint8_t s_left[8][kRefLeft];
    __shared__ uint8_t s_right[8][kRefRight];
    const int pair = blockIdx.y;
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const int i = blockIdx.x * 8 + wi;
    const PairDesc &P = b.pairs[pair];
    const ImageDesc &Il = b.images[P.left];
    const ImageDesc &Ir = b.images[P.right];
    if (i >= *Il.count) return;
    const int j = P.match_idx[i];
    float disp_out = -1.0f, depth_out = 0.0f;
    uint32_t sad_out = 0xFFFFFFFFu;
    if (j >= 0) {
        const int n = Il.out.level[i], xi = Il.out.x[i], yi = Il.out.y[i];
        const LevelDesc &A = b.levels[Il.level_base + n];
        const LevelDesc &B = b.levels[Ir.level_base + n];
        const double s = A.zeta;
        // xr0 = floor(X / s + 0.5): in float, |X / s - q| < 2^-10 for X < 2^13,
        // so a q more than 2^-8 away from a half-integer rounds as the double
        // does; closer ones (rare) take the double computation
        const int X = Ir.out.X[j];
        const float q = __fmul_rn((float)X, A.zeta_inv_f);
        const float fr = q - floorf(q);
        int xr0 = (int)floorf(q + 0.5f);
        if (fabsf(fr - 0.5f) < 0x1p-8f) xr0 = (int)floor(__dadd_rn(__ddiv_rn((double)X, s), 0.5));
        const int W = A.W, H = A.H;
        if (xi - w >= 0 && xi + w < W && yi - w >= 0 && yi + w < H && xr0 - L - w >= 0 && xr0 + L + w < W) {
            const int pw = 2 * w + 1, rw = 2 * (w + L) + 1;
            uint8_t *lp = s_left[wi], *rp = s_right[wi];
            const uint8_t *la0 = A.raw + (size_t)(yi - w) * A.pitch + (xi - w);
            const uint8_t *rb0 = B.raw + (size_t)(yi - w) * B.pitch + (xr0 - L - w);
            for (int r = 0; r < pw; ++r) {
                if (lane < pw) lp[r * pw + lane] = la0[(size_t)r * A.pitch + lane];
                for (int c = lane; c < rw; c += 32) rp[r * rw + c] = rb0[(size_t)r * B.pitch + c];
            }
            __syncwarp();
            const int nsh = 2 * L + 1;
            int part = 0;
            if (lane < 2 * nsh) {
                const int k = lane % nsh, half = lane / nsh;  // shift t = k - L
                const int lc = lp[w * pw + w], rc = rp[w * rw + k + w];
                const int r0 = half == 0 ? 0 : w, r1 = half == 0 ? w : pw;  // rows [0, w) and [w, 2w + 1)
                const int cc = lc - rc;  // |(l - lc) - (r - rc)| = |(l - r) - cc|
                if (WC > 0) {
#pragma unroll
                    for (int rr = 0; rr < WC + 1; ++rr) {
                        const int r = r0 + rr;
                        if (r < r1) {
                            const uint8_t *la = lp + r * (2 * WC + 1), *ra = rp + r * rw + k;
#pragma unroll
                            for (int c = 0; c < 2 * WC + 1; ++c) part += abs((int)la[c] - (int)ra[c] - cc);
                        }
                    }
                } else {
                    for (int r = r0; r < r1; ++r) {
                        const uint8_t *la = lp + r * pw, *ra = rp + r * rw + k;
                        for (int c = 0; c < pw; ++c) part += abs((int)la[c] - (int)ra[c] - cc);
                    }
                }
            }
            const int other = __shfl_down_sync(0xFFFFFFFFu, part, nsh);
            const int sad = part + other;  // valid in lanes 0..nsh-1
            unsigned long long key = lane < nsh ? ((unsigned long long)sad << 8) | (unsigned)lane : ~0ull;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const unsigned long long o = __shfl_xor_sync(0xFFFFFFFFu, key, off);
                key = o < key ? o : key;
            }
            const int kb = (int)(key & 0xFFu);
            const long long d2 = (long long)(key >> 8);
            const long long d1 = __shfl_sync(0xFFFFFFFFu, sad, max(kb - 1, 0));
            const long long d3 = __shfl_sync(0xFFFFFFFFu, sad, min(kb + 1, nsh - 1));
            sad_out = (uint32_t)d2;
            const int ts = kb - L;
            if (ts != -L && ts != L) {
                const long long num = d1 - d3, den = 2 * (d1 + d3 - 2 * d2);
                // disparity >= 0 <=> q den >= num; <= max_disp <=> s (q den - num) <= max_disp den
                const long long qi = (long long)xi - xr0 - ts;
                bool ok = den != 0 && (num < 0 ? -num : num) <= den && qi * den >= num;
                if (ok) {
                    // s (q den - num) <= max_disp den, in float unless within a
                    // relative 2^-18 of equality (float error < 2^-21 relative)
                    const float lhs = __fmul_rn(A.zeta_f, (float)(qi * den - num));
                    const float rhs = __fmul_rn((float)b.prm.max_disp, (float)den);
                    if (lhs > rhs * (1.0f + 0x1p-18f)) ok = false;
                    else if (!(lhs < rhs * (1.0f - 0x1p-18f)))
                        ok = !(__dmul_rn(s, (double)(qi * den - num)) > (double)b.prm.max_disp * (double)den);
                }
                if (ok) {
                    const float delta = __fdiv_rn((float)num, (float)den);
                    const float disp = __fmul_rn(A.zeta_f, __fsub_rn((float)qi, delta));
                    disp_out = disp;
                    depth_out = bf > 0.0 ? __fdiv_rn((float)bf, fmaxf(disp, 0.01f)) : 0.0f;
                }
            }
        }
    }
    if (lane == 0) {
        P.sub_disp[i] = disp_out;
        P.depth[i] = depth_out;
        P.corr[i] = sad_out;
    }
}

__global__ void __launch_bounds__(256) k_refine_median(Batch b)
{
    __shared__ uint32_t hist[256];
    __shared__ uint32_t s_prefix, s_rank, s_total;
    const PairDesc &P = b.pairs[blockIdx.x];
    const int n = *b.images[P.left].count;
    if (threadIdx.x == 0) { s_prefix = 0; s_total = 0; }
    __syncthreads();
    uint32_t mine = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) mine += P.sub_disp[i] >= 0.0f;
    atomicAdd(&s_total, mine);
    __syncthreads();
    const uint32_t total = s_total;
    if (total == 0) return;
    if (threadIdx.x == 0) s_rank = total / 2;  // the median is element total/2 of the ascending list
    // three 8-bit passes over the 24-bit SADs (at most 441 x 510 < 2^18)
    for (int pass = 0; pass < 3; ++pass) {
        const int shift = 16 - 8 * pass;
        hist[threadIdx.x] = 0;
        __syncthreads();
        const uint32_t prefix = s_prefix, hi_mask = pass == 0 ? 0u : (0xFFFFFFu << (shift + 8)) & 0xFFFFFFu;
        for (int i = threadIdx.x; i < n; i += blockDim.x)
            if (P.sub_disp[i] >= 0.0f) {
                const uint32_t v = P.corr[i];
                if ((v & hi_mask) == prefix) atomicAdd(&hist[(v >> shift) & 0xFFu], 1u);
            }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t r = s_rank, acc = 0;
            int d = 0;
            for (; d < 256; ++d) {
                if (acc + hist[d] > r) break;
                acc += hist[d];
            }
            s_rank = r - acc;
            s_prefix = prefix | ((uint32_t)d << shift);
        }
        __syncthreads();
    }
    const unsigned long long median = s_prefix;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        if (P.sub_disp[i] >= 0.0f && 10ull * P.corr[i] > 21ull * median) {
            P.sub_disp[i] = -1.0f;
            P.depth[i] = 0.0f;
        }
}

cudaError_t launch_refine(const Batch &b, int w, int L, double bf, cudaStream_t stream)
{
    if (b.n_pairs == 0 || b.max_capacity == 0) return cudaSuccess;
    dim3 grid((b.max_capacity + 7) / 8, b.n_pairs);
    if (w == 5) k_refine<5><<<grid, 256, 0, stream>>>(b, w, L, bf);
    else k_refine<0><<<grid, 256, 0, stream>>>(b, w, L, bf);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_refine_median<<<b.n_pairs, 256, 0, stream>>>(b);
    return cudaGetLastError();
}

}  // namespace jslam
