// Host-built tables of libjslam (pyramid geometry, bilinear taps, s0
// projection, stereo band, blur weights, angle sectors, BRIEF pattern).
#pragma once

#include <cstddef>
#include <cstdint>

namespace jslam {

struct Geometry {
    int levels;
    int W[8], H[8], c[8];
};

double zeta_pow(float scale, int n);
Geometry level_geometry(int W0, int H0, int levels, float scale, int cell);
uint32_t bilinear_tap(int v, double s, int src_extent);
uint16_t project(int v, double s, int extent);
int match_band(int level, float scale, int row_band_px);
void blur_weights(int32_t w[7]);
void sector_tables(double *cosb, double *sinb);
void brief_pattern(int8_t *base);
void rotated_pattern(int8_t *out);
void corner_table(int p_min, int p_max, uint32_t *bits /* 2048 words */);

}  // namespace jslam
