// Host-built tables of libjslam.  Every floating-point step is plain IEEE
// double with no contraction (compiled with -ffp-contract=off) so that the
// integer tables the kernels consume are reproducible on any host.
#include "tables.h"

#include <cmath>
#include <cstdint>

namespace jslam {

double zeta_pow(float scale, int n)
{
    // zeta^n by repeated multiplication, zeta promoted from the float argument.
    const double z = static_cast<double>(scale);
    double acc = 1.0;
    for (int i = 0; i < n; ++i) acc *= z;
    return acc;
}

Geometry level_geometry(int W0, int H0, int levels, float scale, int cell)
{
    Geometry g;
    g.levels = levels;
    for (int n = 0; n < levels; ++n) {
        const double s = zeta_pow(scale, n);
        g.W[n] = static_cast<int>(std::floor(W0 / s + 0.5));
        g.H[n] = static_cast<int>(std::floor(H0 / s + 0.5));
        const int cn = static_cast<int>(std::floor(cell / s));
        g.c[n] = cn > 0 ? cn : 1;
    }
    return g;
}

// Bilinear source position of output pixel v of a level with scale s: the
// pixel centres are aligned, u = (v + 1/2) s - 1/2, clamped to the source.
uint32_t bilinear_tap(int v, double s, int src_extent)
{
    double u = (static_cast<double>(v) + 0.5) * s - 0.5;
    const double hi = static_cast<double>(src_extent - 1);
    u = u < 0.0 ? 0.0 : (u > hi ? hi : u);
    int base = static_cast<int>(std::floor(u));
    int weight = static_cast<int>(std::floor((u - base) * 256.0 + 0.5));
    if (weight == 256) { ++base; weight = 0; }
    return static_cast<uint32_t>(base) | (static_cast<uint32_t>(weight) << 16);
}

uint16_t project(int v, double s, int extent)
{
    const int p = static_cast<int>(std::floor(v * s + 0.5));
    return static_cast<uint16_t>(p < extent - 1 ? p : extent - 1);
}

int match_band(int level, float scale, int row_band_px)
{
    return static_cast<int>(std::ceil(row_band_px * zeta_pow(scale, level)));
}

void blur_weights(int32_t w[7])
{
    // sigma = 2: g_i = exp(-i^2 / 8), quantised to 1/256, centre absorbs the rest.
    double g[7], total = 0.0;
    for (int i = 0; i < 7; ++i) {
        const int d = i - 3;
        g[i] = std::exp(-static_cast<double>(d * d) / 8.0);
        total += g[i];
    }
    int sum = 0;
    for (int i = 0; i < 7; ++i) {
        w[i] = static_cast<int32_t>(std::floor(256.0 * g[i] / total + 0.5));
        sum += w[i];
    }
    w[3] += 256 - sum;
}

void sector_tables(double *cosb, double *sinb)
{
    const double tau = 6.283185307179586476925286766559;
    for (int b = 0; b < 30; ++b) {
        const double phi = tau * static_cast<double>(b) / 30.0;
        cosb[b] = std::cos(phi);
        sinb[b] = std::sin(phi);
    }
}

namespace {

struct SplitMix64 {
    uint64_t s;
    uint64_t next()
    {
        s += 0x9E3779B97F4A7C15ull;
        uint64_t z = s;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    // Uniform in (0, 1] from the top 53 bits.
    double unit() { return static_cast<double>((next() >> 11) + 1) * (1.0 / 9007199254740992.0); }
    // Standard normal: Box-Muller, cosine branch only.
    double normal()
    {
        const double tau = 6.283185307179586476925286766559;
        const double a = unit();
        const double b = unit();
        const double rad = std::sqrt(-2.0 * std::log(a));
        return rad * std::cos(tau * b);
    }
};

}  // namespace

void brief_pattern(int8_t *base)
{
    SplitMix64 rng{0x4A534C414D31ull};
    const double sigma = 31.0 / 5.0;
    int have = 0;
    while (have < 256) {
        long v[4];
        for (long &e : v) e = std::lround(sigma * rng.normal());
        const bool inside = v[0] * v[0] + v[1] * v[1] <= 169 && v[2] * v[2] + v[3] * v[3] <= 169;
        const bool distinct = v[0] != v[2] || v[1] != v[3];
        if (!inside || !distinct) continue;
        for (int j = 0; j < 4; ++j) base[have * 4 + j] = static_cast<int8_t>(v[j]);
        ++have;
    }
}

void rotated_pattern(int8_t *out)
{
    int8_t base[256 * 4];
    double cosb[30], sinb[30];
    brief_pattern(base);
    sector_tables(cosb, sinb);
    for (int b = 0; b < 30; ++b) {
        for (int i = 0; i < 256; ++i) {
            for (int pt = 0; pt < 2; ++pt) {
                const double x = base[i * 4 + 2 * pt];
                const double y = base[i * 4 + 2 * pt + 1];
                const double rx = cosb[b] * x - sinb[b] * y;
                const double ry = sinb[b] * x + cosb[b] * y;
                int8_t *dst = out + (static_cast<size_t>(b) * 256 + i) * 4 + 2 * pt;
                dst[0] = static_cast<int8_t>(std::lround(rx));
                dst[1] = static_cast<int8_t>(std::lround(ry));
            }
        }
    }
}

// Bit m of the table: the 16-bit ring mask m has its longest circular run of
// set bits in [p_min, p_max] (Eq. 3 on one mask; Sec. III builds such a table).
void corner_table(int p_min, int p_max, uint32_t *bits)
{
    for (int w = 0; w < 2048; ++w) bits[w] = 0;
    for (uint32_t m = 0; m < 65536; ++m) {
        int longest = 0;
        if (m == 0xFFFFu) {
            longest = 16;
        } else {
            // rotate so that bit 15 is clear, then scan linearly
            uint32_t r = m;
            while (r & 0x8000u) r = ((r << 1) | (r >> 15)) & 0xFFFFu;
            int run = 0;
            for (int i = 0; i < 16; ++i) {
                run = (r >> i & 1u) ? run + 1 : 0;
                longest = run > longest ? run : longest;
            }
        }
        if (longest >= p_min && longest <= p_max) bits[m >> 5] |= 1u << (m & 31);
    }
}

}  // namespace jslam
