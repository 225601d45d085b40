// The arc response: the alternative reading of the corner response of
// Sec. III ("sum of absolute differences over the circle", read as over the
// arc that makes the pixel a corner).  For each polarity whose longest
// circular run N of Eq. 1 labels satisfies Eq. 3 (P_min <= N <= P_max), the
// sum of (|d_k| - eps) over the ring positions that lie on a circular run of
// that polarity of length N; the response is the larger of the two sums.
// Every term is at least 1 (the labels are strict), so a corner's response
// lies in [P_min, 16 x 254]; it fits the 16-bit response field and the key
// response << 16 of the culling.
//
// The ring is walked in this library's order (position 0 below the centre,
// image y down); another start or direction around the circle keeps every
// circular run, so the sums are those of any other ordering of the ring.
#pragma once

#include <cstdint>

namespace jslam {

// Longest circular run of set bits of a 16-bit mask (16 for 0xFFFF), and the
// positions lying on a run of that length.
__device__ __forceinline__ uint32_t ring_arc_positions(uint32_t m, int *len)
{
    const uint32_t m32 = m | (m << 16);  // bit i is ring position i mod 16
    uint32_t x = m32;
    int n = 0;
    while (x) {
        x &= x >> 1;
        ++n;
    }
    n = n > 16 ? 16 : n;
    *len = n;
    if (n == 0) return 0u;
    uint32_t starts = m32;  // bit q: positions q .. q + n - 1 all set
    for (int i = 1; i < n; ++i) starts &= m32 >> i;
    starts &= 0xFFFFu;
    uint32_t on = 0;
    for (int j = 0; j < n; ++j) on |= (starts << j) | (starts >> (16 - j));
    return on & 0xFFFFu;
}

// Arc response of the pixel at p (rows rowb bytes apart) for threshold eps
// and run bounds [p_min, p_max]; 0 when neither polarity qualifies.
__device__ __forceinline__ int ring_arc(const uint8_t *p, int rowb, int eps, int p_min, int p_max)
{
    constexpr int DX[16] = { 0, 1, 2, 3, 3, 3, 2, 1, 0, -1, -2, -3, -3, -3, -2, -1 };
    constexpr int DY[16] = { 3, 3, 2, 1, 0, -1, -2, -3, -3, -3, -2, -1, 0, 1, 2, 3 };
    const int ic = p[0];
    int ad[16];
    uint32_t mb = 0, md = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int d = (int)p[DY[k] * rowb + DX[k]] - ic;
        ad[k] = d < 0 ? -d : d;
        mb |= (uint32_t)(d > eps) << k;
        md |= (uint32_t)(d < -eps) << k;
    }
    int best = 0;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        int n;
        const uint32_t on = ring_arc_positions(s ? md : mb, &n);
        if (n < p_min || n > p_max || n == 0) continue;
        int sum = 0;
#pragma unroll
        for (int k = 0; k < 16; ++k)
            if ((on >> k) & 1u) sum += ad[k] - eps;
        best = sum > best ? sum : best;
    }
    return best;
}

}  // namespace jslam
