/*
 * jslam_oracle.c -- plain, slow, single-threaded CPU oracle for the stereo
 * frontend hot path of "High-Speed Stereo Visual SLAM for Low-Powered
 * Computing Devices" (Jetson-SLAM, arXiv 2410.04090).
 *
 * TEST INFRASTRUCTURE.  This file exists only to check the CUDA path.  Only
 * the test suite, the package's smoke check and the benchmark's CPU-baseline
 * leg may load it.  It shares no code, header, table or constant generator
 * with the CUDA library: every table it needs (ring offsets, bilinear taps,
 * blur weights, projection, angle bins, the BRIEF pattern) is derived here
 * again from the written definition.
 *
 * Each function follows the paper's steps in the paper's order, as plain
 * nested loops, and cites the passage it implements:
 *   Sec. II-A  Bounded Rectification: Eq. 1 (pixel labels), Eq. 2 (classic
 *              FAST rule), Eq. 3 (bounded rule), the Bresenham ring figure.
 *   Sec. II-C-1 Feature Culling (FC) over the CRF-matrix.
 *   Sec. II-C-2 Pyramidal Feature Aggregation (PFA) and its worked figure.
 *   Sec. III   micro-second FAST (bit masks, SAD response), streamlined
 *              multiscale detection + extraction (Gaussian filter, ORB),
 *              middle-end stereo matching.
 *
 * Where the paper is silent the reading used is stated at the function.
 * Floating point is IEEE double; build with -ffp-contract=off so that no
 * multiply-add is fused (the CUDA path reproduces these roundings exactly).
 *
 * Pins (tests/test_oracle_*.py) tie every function to something other than
 * itself: paper figures (ring layout, all-bright non-corner, PFA example),
 * closed forms (SAD response, blur and bilinear against scipy routines,
 * intensity-centroid angle of ramps), published test vectors (splitmix64)
 * and brute force on tiny inputs (run length, culling, PFA, matching).
 * Parity unpinned: none of the exported functions; the Box-Muller draw and
 * the pattern rejection rule are pinned only statistically (moments and
 * radius bounds).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define OR_MAX_LEVELS 8
#define OR_NBINS 30
#define OR_NPAIRS 256
#define OR_DISK_R 15

typedef struct {
    int32_t levels;        /* number of pyramid levels, 1..8 */
    float scale;           /* scale factor zeta between levels (> 1) */
    int32_t fast_thresh;   /* epsilon of Eq. 1 */
    int32_t fast_thresh_lo;/* fallback epsilon for empty cells, <= 0: off */
    int32_t p_min, p_max;  /* bounds of Eq. 3 */
    int32_t cell;          /* FC cell size at s0 */
    int32_t k_per_cell;    /* corners kept per cell */
    int32_t nms_q;         /* PFA NMS window q (odd) */
    int32_t border;        /* pixels skipped at each edge of a level */
    int32_t max_feats;     /* keypoint cap per image */
    int32_t pfa_rule;      /* 0: dominance on both scores, 1: lexicographic */
    int32_t max_disp;      /* stereo search range in s0 pixels */
    int32_t row_band_px;   /* stereo row band at s0, scaled per level */
    int32_t match_max_dist;/* Hamming acceptance threshold */
    int32_t response_mode; /* 0: SAD over the whole circle (default); 1: the arc reading, see or_arc_response */
    int32_t pyramid_mode;  /* 0: each level resampled from level 0 (default); 1: cascaded, from level n - 1 */
} or_params;

typedef struct {
    int32_t capacity;
    int32_t count;
    uint16_t *x, *y;       /* level coordinates */
    uint16_t *X, *Y;       /* s0 projection */
    uint8_t *level;
    uint16_t *response;    /* SAD response r */
    uint8_t *k_levels;     /* K_l at (X, Y) */
    uint32_t *k_resp;      /* K_r at (X, Y) */
    float *angle;          /* theta, radians, (-pi, pi] */
    uint8_t *angle_bin;    /* 0..29 */
    uint32_t *desc;        /* capacity x 8 words */
    int32_t *m10, *m01;    /* intensity moments (for tests) */
} or_keypoints;

/* ------------------------------------------------------------------ */
/* Level geometry (Sec. III "streamlined multiscale"; cell scaling as in the
 * cell-size ablation: a 32x32 cell at s0 is 8x8 at the 8th scale for
 * zeta = 1.2).  zeta^n is accumulated by repeated multiplication in double,
 * W_n = floor(W0 / zeta^n + 0.5), c_n = max(1, floor(c / zeta^n)).        */

double or_level_scale(float scale, int32_t n)
{
    double s = 1.0;
    for (int32_t i = 0; i < n; ++i) s = s * (double)scale;
    return s;
}

void or_level_geometry(int32_t W0, int32_t H0, int32_t levels, float scale,
                       int32_t cell, int32_t *W, int32_t *H, int32_t *c)
{
    for (int32_t n = 0; n < levels; ++n) {
        double s = or_level_scale(scale, n);
        W[n] = (int32_t)floor((double)W0 / s + 0.5);
        H[n] = (int32_t)floor((double)H0 / s + 0.5);
        int32_t cn = (int32_t)floor((double)cell / s);
        c[n] = cn < 1 ? 1 : cn;
    }
}

/* ------------------------------------------------------------------ */
/* Pyramid (Sec. III; the resampling method is not stated).  Each level n >= 1
 * is resampled directly from L0 by bilinear interpolation at the pixel-centre
 * aligned source position u = (x + 0.5) zeta^n - 0.5, clamped to the image,
 * with Q8 weights.                                                         */

static void bilinear_tap(int32_t x, double s, int32_t W0,
                         int32_t *xa, int32_t *xb, int32_t *a)
{
    double u = ((double)x + 0.5) * s - 0.5;
    if (u < 0.0) u = 0.0;
    if (u > (double)(W0 - 1)) u = (double)(W0 - 1);
    int32_t i = (int32_t)floor(u);
    int32_t w = (int32_t)floor((u - (double)i) * 256.0 + 0.5);
    if (w == 256) { i += 1; w = 0; }
    *xa = i;
    *xb = (i + 1 < W0) ? i + 1 : W0 - 1;
    *a = w;
}

void or_pyramid_level(const uint8_t *L0, int32_t W0, int32_t H0, int32_t pitch0,
                      float scale, int32_t n, uint8_t *out, int32_t Wn, int32_t Hn,
                      int32_t pitch_out)
{
    double s = or_level_scale(scale, n);
    for (int32_t y = 0; y < Hn; ++y) {
        int32_t ya, yb, b;
        bilinear_tap(y, s, H0, &ya, &yb, &b);
        for (int32_t x = 0; x < Wn; ++x) {
            int32_t xa, xb, a;
            bilinear_tap(x, s, W0, &xa, &xb, &a);
            uint32_t p00 = L0[(size_t)ya * pitch0 + xa];
            uint32_t p01 = L0[(size_t)ya * pitch0 + xb];
            uint32_t p10 = L0[(size_t)yb * pitch0 + xa];
            uint32_t p11 = L0[(size_t)yb * pitch0 + xb];
            uint32_t top = (256u - (uint32_t)a) * p00 + (uint32_t)a * p01;
            uint32_t bot = (256u - (uint32_t)a) * p10 + (uint32_t)a * p11;
            uint32_t v = (256u - (uint32_t)b) * top + (uint32_t)b * bot;
            out[(size_t)y * pitch_out + x] = (uint8_t)((v + 32768u) >> 16);
        }
    }
}

/* ------------------------------------------------------------------ */
/* Gaussian filtering before ORB extraction (Sec. III): a 7-tap separable
 * Gaussian with sigma = 2, weights quantised to Q8 with the centre tap
 * absorbing the rounding so that they sum to 256; replicated border.        */

void or_blur_weights(int32_t w[7])
{
    double g[7], sum = 0.0;
    for (int32_t i = -3; i <= 3; ++i) {
        g[i + 3] = exp(-(double)(i * i) / (2.0 * 2.0 * 2.0));
        sum += g[i + 3];
    }
    int32_t total = 0;
    for (int32_t i = 0; i < 7; ++i) {
        w[i] = (int32_t)floor(256.0 * g[i] / sum + 0.5);
        total += w[i];
    }
    w[3] += 256 - total;
}

static int32_t clampi(int32_t v, int32_t lo, int32_t hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

void or_blur(const uint8_t *in, int32_t W, int32_t H, int32_t pitch_in,
             uint8_t *out, int32_t pitch_out)
{
    int32_t w[7];
    or_blur_weights(w);
    uint32_t *h = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)W * (size_t)H);
    for (int32_t y = 0; y < H; ++y)
        for (int32_t x = 0; x < W; ++x) {
            uint32_t acc = 0;
            for (int32_t i = -3; i <= 3; ++i)
                acc += (uint32_t)w[i + 3] * in[(size_t)y * pitch_in + clampi(x + i, 0, W - 1)];
            h[(size_t)y * W + x] = acc;
        }
    for (int32_t y = 0; y < H; ++y)
        for (int32_t x = 0; x < W; ++x) {
            uint32_t acc = 0;
            for (int32_t j = -3; j <= 3; ++j)
                acc += (uint32_t)w[j + 3] * h[(size_t)clampi(y + j, 0, H - 1) * W + x];
            out[(size_t)y * pitch_out + x] = (uint8_t)((acc + 32768u) >> 16);
        }
    free(h);
}

/* ------------------------------------------------------------------ */
/* FAST with Bounded Rectification (Sec. II-A, Eq. 1-3; Sec. III bit masks).
 * Ring: the 16-pixel radius-3 Bresenham circle of the non-corner figure,
 * index 0 directly below the centre (image y grows downward), then in ring
 * order.                                                                   */

static const int32_t RING_DX[16] = { 0, 1, 2, 3, 3, 3, 2, 1, 0, -1, -2, -3, -3, -3, -2, -1 };
static const int32_t RING_DY[16] = { 3, 3, 2, 1, 0, -1, -2, -3, -3, -3, -2, -1, 0, 1, 2, 3 };

void or_ring(int32_t *dx, int32_t *dy)
{
    for (int32_t k = 0; k < 16; ++k) { dx[k] = RING_DX[k]; dy[k] = RING_DY[k]; }
}

/* Longest circular run of set bits of a 16-bit ring mask (N_b or N_d). */
int32_t or_longest_run(uint32_t mask)
{
    int32_t best = 0;
    for (int32_t start = 0; start < 16; ++start) {
        int32_t len = 0;
        while (len < 16 && ((mask >> ((start + len) % 16)) & 1u)) ++len;
        if (len > best) best = len;
    }
    return best;
}

/* Eq. 3 read disjunctively: a conjunction would need N_b + N_d >= 2 P_min > 16. */
int32_t or_corner_from_masks(uint32_t Bb, uint32_t Bd, int32_t p_min, int32_t p_max)
{
    int32_t nb = or_longest_run(Bb), nd = or_longest_run(Bd);
    return (nb >= p_min && nb <= p_max) || (nd >= p_min && nd <= p_max);
}

/* CRF-matrix of one level: corner flag and SAD response for every pixel at
 * least `border` from each edge (0 elsewhere).  Eq. 1: bright when
 * I_p - I_c > eps, dark when I_p - I_c < -eps, similar otherwise (|d| = eps
 * is similar).  Response: sum of |I_c - I_p| over the whole circle.         */
void or_fast(const uint8_t *img, int32_t W, int32_t H, int32_t pitch, int32_t eps,
             int32_t p_min, int32_t p_max, int32_t border,
             uint8_t *corner, uint16_t *resp)
{
    memset(corner, 0, (size_t)W * (size_t)H);
    memset(resp, 0, sizeof(uint16_t) * (size_t)W * (size_t)H);
    for (int32_t y = border; y < H - border; ++y)
        for (int32_t x = border; x < W - border; ++x) {
            int32_t ic = img[(size_t)y * pitch + x];
            uint32_t Bb = 0, Bd = 0;
            int32_t r = 0;
            for (int32_t k = 0; k < 16; ++k) {
                int32_t ip = img[(size_t)(y + RING_DY[k]) * pitch + (x + RING_DX[k])];
                int32_t d = ip - ic;
                if (d > eps) Bb |= 1u << k;
                if (d < -eps) Bd |= 1u << k;
                r += d < 0 ? -d : d;
            }
            corner[(size_t)y * W + x] = (uint8_t)or_corner_from_masks(Bb, Bd, p_min, p_max);
            resp[(size_t)y * W + x] = (uint16_t)r;
        }
}

/* The alternative reading of the response (Sec. III, "sum of absolute
 * differences over the circle", read as over the arc that makes the corner):
 * for each polarity whose longest circular run N satisfies Eq. 3, the sum of
 * (|d_k| - eps) over the ring positions that lie on a circular run of that
 * polarity of length N (for N >= 9 there is one such run); the response is
 * the larger of the two sums (one polarity qualifies when P_min >= 9), 0 when
 * neither qualifies.  Every term is at least 1, so a corner's response is at
 * least P_min and at most 16 x 254.                                         */

/* Bit k set when ring position k lies on a circular run of set bits of
 * `mask` (16 bits) whose length is the longest run's. */
uint32_t or_arc_positions(uint32_t mask)
{
    int32_t n = or_longest_run(mask);
    uint32_t on = 0;
    if (n == 0) return 0;
    for (int32_t start = 0; start < 16; ++start) {
        int32_t len = 0;
        while (len < n && ((mask >> ((start + len) % 16)) & 1u)) ++len;
        if (len == n)
            for (int32_t j = 0; j < n; ++j) on |= 1u << ((start + j) % 16);
    }
    return on;
}

int32_t or_arc_response(const int32_t d[16], uint32_t Bb, uint32_t Bd, int32_t eps, int32_t p_min, int32_t p_max)
{
    int32_t best = 0;
    uint32_t masks[2] = { Bb, Bd };
    for (int32_t s = 0; s < 2; ++s) {
        int32_t n = or_longest_run(masks[s]);
        if (n < p_min || n > p_max) continue;
        uint32_t on = or_arc_positions(masks[s]);
        int32_t sum = 0;
        for (int32_t k = 0; k < 16; ++k)
            if ((on >> k) & 1u) sum += (d[k] < 0 ? -d[k] : d[k]) - eps;
        if (sum > best) best = sum;
    }
    return best;
}

/* CRF-matrix of one level with the arc response (corners as in or_fast). */
void or_fast_arc(const uint8_t *img, int32_t W, int32_t H, int32_t pitch, int32_t eps,
                 int32_t p_min, int32_t p_max, int32_t border,
                 uint8_t *corner, uint16_t *resp)
{
    memset(corner, 0, (size_t)W * (size_t)H);
    memset(resp, 0, sizeof(uint16_t) * (size_t)W * (size_t)H);
    for (int32_t y = border; y < H - border; ++y)
        for (int32_t x = border; x < W - border; ++x) {
            int32_t ic = img[(size_t)y * pitch + x];
            int32_t d[16];
            uint32_t Bb = 0, Bd = 0;
            for (int32_t k = 0; k < 16; ++k) {
                d[k] = (int32_t)img[(size_t)(y + RING_DY[k]) * pitch + (x + RING_DX[k])] - ic;
                if (d[k] > eps) Bb |= 1u << k;
                if (d[k] < -eps) Bd |= 1u << k;
            }
            int32_t is_corner = or_corner_from_masks(Bb, Bd, p_min, p_max);
            corner[(size_t)y * W + x] = (uint8_t)is_corner;
            resp[(size_t)y * W + x] = (uint16_t)(is_corner ? or_arc_response(d, Bb, Bd, eps, p_min, p_max) : 0);
        }
}

/* ------------------------------------------------------------------ */
/* Feature Culling (Sec. II-C-1): non-overlapping c x c cells tiled from the
 * level origin (partial cells at the right and bottom edges count); each
 * cell keeps its strongest corners.  Order within a cell: response
 * descending, then y ascending, then x ascending.  Fallback: a cell with no
 * corner at the primary threshold selects among fallback-threshold corners. */

typedef struct { int32_t x, y, r; } or_cand;

static int cmp_cand(const void *pa, const void *pb)
{
    const or_cand *a = (const or_cand *)pa, *b = (const or_cand *)pb;
    if (a->r != b->r) return a->r > b->r ? -1 : 1;
    if (a->y != b->y) return a->y < b->y ? -1 : 1;
    if (a->x != b->x) return a->x < b->x ? -1 : 1;
    return 0;
}

int32_t or_cull_level(const uint8_t *corner_hi, const uint8_t *corner_lo,
                      const uint16_t *resp, int32_t W, int32_t H, int32_t c, int32_t k,
                      int32_t *out_x, int32_t *out_y, int32_t *out_r, int32_t cap)
{
    int32_t n_out = 0;
    or_cand *buf = (or_cand *)malloc(sizeof(or_cand) * (size_t)c * (size_t)c);
    int32_t cells_x = (W + c - 1) / c, cells_y = (H + c - 1) / c;
    for (int32_t cy = 0; cy < cells_y; ++cy)
        for (int32_t cx = 0; cx < cells_x; ++cx) {
            int32_t y0 = cy * c, x0 = cx * c;
            int32_t y1 = y0 + c < H ? y0 + c : H, x1 = x0 + c < W ? x0 + c : W;
            const uint8_t *flags = corner_hi;
            int32_t any_hi = 0;
            for (int32_t y = y0; y < y1 && !any_hi; ++y)
                for (int32_t x = x0; x < x1; ++x)
                    if (corner_hi[(size_t)y * W + x]) { any_hi = 1; break; }
            if (!any_hi) {
                if (!corner_lo) continue;
                flags = corner_lo;
            }
            int32_t m = 0;
            for (int32_t y = y0; y < y1; ++y)
                for (int32_t x = x0; x < x1; ++x)
                    if (flags[(size_t)y * W + x]) {
                        buf[m].x = x; buf[m].y = y; buf[m].r = resp[(size_t)y * W + x];
                        ++m;
                    }
            qsort(buf, (size_t)m, sizeof(or_cand), cmp_cand);
            for (int32_t i = 0; i < m && i < k; ++i) {
                if (n_out < cap) {
                    out_x[n_out] = buf[i].x; out_y[n_out] = buf[i].y; out_r[n_out] = buf[i].r;
                }
                ++n_out;
            }
        }
    free(buf);
    return n_out;
}

/* ------------------------------------------------------------------ */
/* Pyramidal Feature Aggregation (Sec. II-C-2 and its worked figure).
 * Step 1: project every keypoint to s0 and copy its response into the
 *         N_s x H x W matrix M (zero-initialised).
 * Step 2: K_r = sum of responses across scales, K_l = number of scales with
 *         a keypoint, per s0 pixel.
 * Step 3: sparse q x q NMS around each keypoint: a keypoint is suppressed
 *         when a keypoint in its window has both larger k_r and larger k_l
 *         (rule 0; rule 1 compares (k_l, k_r) lexicographically).
 * The survivors keep their own level and coordinates.                      */

int32_t or_project(int32_t x, int32_t n, float scale, int32_t W0)
{
    double s = or_level_scale(scale, n);
    int32_t X = (int32_t)floor((double)x * s + 0.5);
    return X < W0 - 1 ? X : W0 - 1;
}

void or_pfa_core(int32_t n_cand, const int32_t *lev, const int32_t *X, const int32_t *Y,
                 const int32_t *r, int32_t W0, int32_t H0, int32_t Ns, int32_t q,
                 int32_t rule, int32_t *Kl_out, int32_t *Kr_out, uint8_t *alive)
{
    size_t plane = (size_t)W0 * (size_t)H0;
    int32_t *M = (int32_t *)calloc((size_t)Ns * plane, sizeof(int32_t));
    uint8_t *occ = (uint8_t *)calloc((size_t)Ns * plane, 1);
    int32_t *Kr = (int32_t *)calloc(plane, sizeof(int32_t));
    int32_t *Kl = (int32_t *)calloc(plane, sizeof(int32_t));
    for (int32_t i = 0; i < n_cand; ++i) {
        size_t at = (size_t)lev[i] * plane + (size_t)Y[i] * W0 + X[i];
        M[at] = r[i];
        occ[at] = 1;
    }
    for (int32_t n = 0; n < Ns; ++n)
        for (size_t p = 0; p < plane; ++p) {
            Kr[p] += M[(size_t)n * plane + p];
            Kl[p] += occ[(size_t)n * plane + p];
        }
    int32_t rad = (q - 1) / 2;
    for (int32_t i = 0; i < n_cand; ++i) {
        size_t p = (size_t)Y[i] * W0 + X[i];
        int32_t kl = Kl[p], kr = Kr[p];
        int32_t suppressed = 0;
        for (int32_t dy = -rad; dy <= rad && !suppressed; ++dy)
            for (int32_t dx = -rad; dx <= rad; ++dx) {
                int32_t qy = Y[i] + dy, qx = X[i] + dx;
                if ((dx == 0 && dy == 0) || qy < 0 || qy >= H0 || qx < 0 || qx >= W0) continue;
                size_t qp = (size_t)qy * W0 + qx;
                if (Kl[qp] == 0) continue;
                int32_t dom = rule == 0 ? (Kl[qp] > kl && Kr[qp] > kr)
                                        : (Kl[qp] > kl || (Kl[qp] == kl && Kr[qp] > kr));
                if (dom) { suppressed = 1; break; }
            }
        Kl_out[i] = kl;
        Kr_out[i] = kr;
        alive[i] = (uint8_t)!suppressed;
    }
    free(M); free(occ); free(Kr); free(Kl);
}

/* ------------------------------------------------------------------ */
/* Orientation by intensity centroid (ORB, used by the streamlined
 * extraction of Sec. III) over the radius-15 disk of the raw level, and the
 * angle bin of 30 equal sectors decided by exact-rounding sign tests.       */

void or_bin_tables(double *cosb, double *sinb)
{
    const double two_pi = 6.283185307179586476925286766559;
    for (int32_t b = 0; b < OR_NBINS; ++b) {
        double phi = two_pi * (double)b / (double)OR_NBINS;
        cosb[b] = cos(phi);
        sinb[b] = sin(phi);
    }
}

static int32_t left_of_boundary(int32_t m10, int32_t m01, double cb, double sb)
{
    double t1 = (double)m01 * cb;
    double t2 = (double)m10 * sb;
    double t = t1 - t2;
    return t >= 0.0;
}

void or_orient(const uint8_t *img, int32_t pitch, int32_t x, int32_t y,
               int32_t *m10_out, int32_t *m01_out, double *theta, int32_t *bin)
{
    int32_t m10 = 0, m01 = 0;
    for (int32_t dy = -OR_DISK_R; dy <= OR_DISK_R; ++dy)
        for (int32_t dx = -OR_DISK_R; dx <= OR_DISK_R; ++dx) {
            if (dx * dx + dy * dy > OR_DISK_R * OR_DISK_R) continue;
            int32_t v = img[(size_t)(y + dy) * pitch + (x + dx)];
            m10 += dx * v;
            m01 += dy * v;
        }
    *m10_out = m10;
    *m01_out = m01;
    double cosb[OR_NBINS], sinb[OR_NBINS];
    or_bin_tables(cosb, sinb);
    *bin = 0;
    if (m10 == 0 && m01 == 0) { *theta = 0.0; return; }
    *theta = atan2((double)m01, (double)m10);
    for (int32_t b = 0; b < OR_NBINS; ++b) {
        int32_t nb = (b + 1) % OR_NBINS;
        if (left_of_boundary(m10, m01, cosb[b], sinb[b]) &&
            !left_of_boundary(m10, m01, cosb[nb], sinb[nb])) {
            *bin = b;
            break;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Steered BRIEF pattern.  ORB's learned pattern is third-party data and is
 * not used; this build draws its own: 256 point pairs with i.i.d. Gaussian
 * offsets (sigma = 31/5, as in BRIEF's isotropic sampling), rounded to the
 * nearest integer, redrawn when a point leaves the radius-13 disk or p = q.
 * Random source: splitmix64 (Steele, Lea, Flood 2014) from seed
 * 0x4A534C414D31, Box-Muller (cosine branch) on 53-bit uniforms in (0, 1]. */

uint64_t or_splitmix64_next(uint64_t *state)
{
    *state += 0x9E3779B97F4A7C15ull;
    uint64_t z = *state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double or_std_normal(uint64_t *state)
{
    const double two_pi = 6.283185307179586476925286766559;
    double u1 = (double)((or_splitmix64_next(state) >> 11) + 1) * (1.0 / 9007199254740992.0);
    double u2 = (double)((or_splitmix64_next(state) >> 11) + 1) * (1.0 / 9007199254740992.0);
    double radius = sqrt(-2.0 * log(u1));
    double ang = two_pi * u2;
    return radius * cos(ang);
}

void or_pattern_base(int8_t *out)
{
    uint64_t st = 0x4A534C414D31ull;
    const double sigma = 31.0 / 5.0;
    int32_t got = 0;
    while (got < OR_NPAIRS) {
        int32_t v[4];
        for (int32_t j = 0; j < 4; ++j) {
            double g = or_std_normal(&st);
            double scaled = sigma * g;
            v[j] = (int32_t)lround(scaled);
        }
        if (v[0] * v[0] + v[1] * v[1] > 169) continue;
        if (v[2] * v[2] + v[3] * v[3] > 169) continue;
        if (v[0] == v[2] && v[1] == v[3]) continue;
        for (int32_t j = 0; j < 4; ++j) out[got * 4 + j] = (int8_t)v[j];
        ++got;
    }
}

/* Pattern rotated by phi_b: p' = (round(cos x - sin y), round(sin x + cos y)). */
void or_pattern_rotated(int8_t *out)
{
    int8_t base[OR_NPAIRS * 4];
    double cosb[OR_NBINS], sinb[OR_NBINS];
    or_pattern_base(base);
    or_bin_tables(cosb, sinb);
    for (int32_t b = 0; b < OR_NBINS; ++b)
        for (int32_t i = 0; i < OR_NPAIRS; ++i)
            for (int32_t pt = 0; pt < 2; ++pt) {
                double x = (double)base[i * 4 + pt * 2 + 0];
                double y = (double)base[i * 4 + pt * 2 + 1];
                double cx = cosb[b] * x, sy = sinb[b] * y;
                double sx = sinb[b] * x, cy = cosb[b] * y;
                double xr = cx - sy;
                double yr = sx + cy;
                out[((size_t)b * OR_NPAIRS + i) * 4 + pt * 2 + 0] = (int8_t)lround(xr);
                out[((size_t)b * OR_NPAIRS + i) * 4 + pt * 2 + 1] = (int8_t)lround(yr);
            }
}

/* Bit i = [B(kp + p'_i) < B(kp + q'_i)] on the blurred level; bit i lives in
 * word i / 32 at position i % 32.                                           */
void or_describe(const uint8_t *blur, int32_t pitch, int32_t x, int32_t y,
                 const int8_t *rot_bin, uint32_t *desc)
{
    for (int32_t w = 0; w < 8; ++w) desc[w] = 0;
    for (int32_t i = 0; i < OR_NPAIRS; ++i) {
        int32_t px = rot_bin[i * 4 + 0], py = rot_bin[i * 4 + 1];
        int32_t qx = rot_bin[i * 4 + 2], qy = rot_bin[i * 4 + 3];
        int32_t a = blur[(size_t)(y + py) * pitch + (x + px)];
        int32_t b = blur[(size_t)(y + qy) * pitch + (x + qx)];
        if (a < b) desc[i / 32] |= 1u << (i % 32);
    }
}

/* ------------------------------------------------------------------ */
/* Whole frontend for one image: pyramid, blur, CRF, FC, PFA, cap, ORB.    */

typedef struct {
    int32_t level, x, y, X, Y, r, kl, kr;
} or_kp;

static int cmp_cap(const void *pa, const void *pb)
{
    const or_kp *a = (const or_kp *)pa, *b = (const or_kp *)pb;
    if (a->kl != b->kl) return a->kl > b->kl ? -1 : 1;
    if (a->kr != b->kr) return a->kr > b->kr ? -1 : 1;
    if (a->r != b->r) return a->r > b->r ? -1 : 1;
    if (a->level != b->level) return a->level < b->level ? -1 : 1;
    if (a->y != b->y) return a->y < b->y ? -1 : 1;
    if (a->x != b->x) return a->x < b->x ? -1 : 1;
    return 0;
}

static int cmp_canonical(const void *pa, const void *pb)
{
    const or_kp *a = (const or_kp *)pa, *b = (const or_kp *)pb;
    if (a->level != b->level) return a->level < b->level ? -1 : 1;
    if (a->y != b->y) return a->y < b->y ? -1 : 1;
    if (a->x != b->x) return a->x < b->x ? -1 : 1;
    return 0;
}

int32_t or_check_params(int32_t W0, int32_t H0, const or_params *p)
{
    if (p->levels < 1 || p->levels > OR_MAX_LEVELS) return -1;
    if (!(p->scale > 1.0f)) return -1;
    if (p->fast_thresh < 1 || p->fast_thresh > 254) return -1;
    if (p->fast_thresh_lo > 254) return -1;
    if (p->p_min < 1 || p->p_max > 16 || p->p_min > p->p_max) return -1;
    if (p->cell < 1 || p->cell > 128) return -1;
    if (p->k_per_cell < 1 || p->k_per_cell > 8) return -1;
    if (p->nms_q < 1 || (p->nms_q & 1) == 0 || p->nms_q > 7) return -1;
    if (p->border < 16) return -1;
    if (p->max_feats < 1) return -1;
    if (p->pfa_rule < 0 || p->pfa_rule > 1) return -1;
    if (p->response_mode < 0 || p->response_mode > 1 || p->pyramid_mode < 0 || p->pyramid_mode > 1) return -1;
    if (W0 < 1 || H0 < 1 || W0 > 4096 || H0 > 4096) return -1;
    int32_t W[OR_MAX_LEVELS], H[OR_MAX_LEVELS], c[OR_MAX_LEVELS];
    or_level_geometry(W0, H0, p->levels, p->scale, p->cell, W, H, c);
    for (int32_t n = 0; n < p->levels; ++n)
        if (W[n] < 2 * p->border + 1 || H[n] < 2 * p->border + 1) return -1;
    return 0;
}

int32_t or_extract_image(const uint8_t *L0, int32_t W0, int32_t H0, int32_t pitch0,
                         const or_params *p, or_keypoints *out)
{
    if (or_check_params(W0, H0, p) != 0) return -1;
    int32_t L = p->levels;
    int32_t W[OR_MAX_LEVELS], H[OR_MAX_LEVELS], c[OR_MAX_LEVELS];
    or_level_geometry(W0, H0, L, p->scale, p->cell, W, H, c);

    uint8_t *raw[OR_MAX_LEVELS], *blur[OR_MAX_LEVELS];
    for (int32_t n = 0; n < L; ++n) {
        raw[n] = (uint8_t *)malloc((size_t)W[n] * (size_t)H[n]);
        blur[n] = (uint8_t *)malloc((size_t)W[n] * (size_t)H[n]);
        if (n == 0)
            for (int32_t y = 0; y < H0; ++y) memcpy(raw[0] + (size_t)y * W0, L0 + (size_t)y * pitch0, (size_t)W0);
        else if (p->pyramid_mode == 1)  /* cascaded: level n from level n - 1 by one factor zeta */
            or_pyramid_level(raw[n - 1], W[n - 1], H[n - 1], W[n - 1], p->scale, 1, raw[n], W[n], H[n], W[n]);
        else
            or_pyramid_level(L0, W0, H0, pitch0, p->scale, n, raw[n], W[n], H[n], W[n]);
        or_blur(raw[n], W[n], H[n], W[n], blur[n], W[n]);
    }

    /* CRF + FC per level. */
    size_t cap_all = 0;
    for (int32_t n = 0; n < L; ++n)
        cap_all += (size_t)((W[n] + c[n] - 1) / c[n]) * (size_t)((H[n] + c[n] - 1) / c[n]) * (size_t)p->k_per_cell;
    or_kp *cand = (or_kp *)malloc(sizeof(or_kp) * (cap_all + 1));
    int32_t n_cand = 0;
    for (int32_t n = 0; n < L; ++n) {
        size_t area = (size_t)W[n] * (size_t)H[n];
        uint8_t *hi = (uint8_t *)malloc(area), *lo = NULL;
        uint16_t *resp = (uint16_t *)malloc(area * sizeof(uint16_t));
        or_fast(raw[n], W[n], H[n], W[n], p->fast_thresh, p->p_min, p->p_max, p->border, hi, resp);
        if (p->fast_thresh_lo > 0) {
            uint16_t *resp_lo = (uint16_t *)malloc(area * sizeof(uint16_t));
            lo = (uint8_t *)malloc(area);
            or_fast(raw[n], W[n], H[n], W[n], p->fast_thresh_lo, p->p_min, p->p_max, p->border, lo, resp_lo);
            free(resp_lo);
        }
        if (p->response_mode == 1) {
            /* the arc response depends on the threshold: the corners of a
             * cell with no primary-threshold corner (the only cells whose
             * fallback corners are ranked) take it at the fallback threshold */
            or_fast_arc(raw[n], W[n], H[n], W[n], p->fast_thresh, p->p_min, p->p_max, p->border, hi, resp);
            if (lo) {
                uint8_t *lo_arc = (uint8_t *)malloc(area);
                uint16_t *resp_arc = (uint16_t *)malloc(area * sizeof(uint16_t));
                or_fast_arc(raw[n], W[n], H[n], W[n], p->fast_thresh_lo, p->p_min, p->p_max, p->border, lo_arc,
                            resp_arc);
                for (size_t q = 0; q < area; ++q)
                    if (!hi[q]) resp[q] = resp_arc[q];
                free(lo_arc); free(resp_arc);
            }
        }
        size_t cells = (size_t)((W[n] + c[n] - 1) / c[n]) * (size_t)((H[n] + c[n] - 1) / c[n]) * (size_t)p->k_per_cell;
        int32_t *cx = (int32_t *)malloc(sizeof(int32_t) * (cells + 1));
        int32_t *cy = (int32_t *)malloc(sizeof(int32_t) * (cells + 1));
        int32_t *cr = (int32_t *)malloc(sizeof(int32_t) * (cells + 1));
        int32_t m = or_cull_level(hi, lo, resp, W[n], H[n], c[n], p->k_per_cell, cx, cy, cr, (int32_t)cells);
        for (int32_t i = 0; i < m; ++i) {
            or_kp *k = &cand[n_cand++];
            k->level = n; k->x = cx[i]; k->y = cy[i]; k->r = cr[i];
            k->X = or_project(cx[i], n, p->scale, W0);
            k->Y = or_project(cy[i], n, p->scale, H0);
        }
        free(cx); free(cy); free(cr); free(hi); free(lo); free(resp);
    }

    /* PFA. */
    int32_t *lev = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_cand + 1));
    int32_t *X = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_cand + 1));
    int32_t *Y = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_cand + 1));
    int32_t *R = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_cand + 1));
    int32_t *Kl = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_cand + 1));
    int32_t *Kr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_cand + 1));
    uint8_t *alive = (uint8_t *)malloc((size_t)(n_cand + 1));
    for (int32_t i = 0; i < n_cand; ++i) {
        lev[i] = cand[i].level; X[i] = cand[i].X; Y[i] = cand[i].Y; R[i] = cand[i].r;
    }
    or_pfa_core(n_cand, lev, X, Y, R, W0, H0, L, p->nms_q, p->pfa_rule, Kl, Kr, alive);
    int32_t n_alive = 0;
    for (int32_t i = 0; i < n_cand; ++i)
        if (alive[i]) {
            cand[n_alive] = cand[i];
            cand[n_alive].kl = Kl[i];
            cand[n_alive].kr = Kr[i];
            ++n_alive;
        }
    free(lev); free(X); free(Y); free(R); free(Kl); free(Kr); free(alive);

    /* Cap, then canonical order (level, y, x). */
    int32_t keep = n_alive;
    if (keep > p->max_feats) {
        qsort(cand, (size_t)n_alive, sizeof(or_kp), cmp_cap);
        keep = p->max_feats;
    }
    qsort(cand, (size_t)keep, sizeof(or_kp), cmp_canonical);
    if (keep > out->capacity) keep = out->capacity;

    /* Orientation on the raw level, descriptor on the blurred level. */
    int8_t *rot = (int8_t *)malloc((size_t)OR_NBINS * OR_NPAIRS * 4);
    or_pattern_rotated(rot);
    for (int32_t i = 0; i < keep; ++i) {
        const or_kp *k = &cand[i];
        int32_t m10, m01, bin;
        double theta;
        or_orient(raw[k->level], W[k->level], k->x, k->y, &m10, &m01, &theta, &bin);
        out->x[i] = (uint16_t)k->x; out->y[i] = (uint16_t)k->y;
        out->X[i] = (uint16_t)k->X; out->Y[i] = (uint16_t)k->Y;
        out->level[i] = (uint8_t)k->level;
        out->response[i] = (uint16_t)k->r;
        out->k_levels[i] = (uint8_t)k->kl;
        out->k_resp[i] = (uint32_t)k->kr;
        out->angle[i] = (float)theta;
        out->angle_bin[i] = (uint8_t)bin;
        if (out->m10) out->m10[i] = m10;
        if (out->m01) out->m01[i] = m01;
        or_describe(blur[k->level], W[k->level], k->x, k->y,
                    rot + (size_t)bin * OR_NPAIRS * 4, out->desc + (size_t)i * 8);
    }
    out->count = keep;
    free(rot);
    free(cand);
    for (int32_t n = 0; n < L; ++n) { free(raw[n]); free(blur[n]); }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Stereo matching by descriptor-distance minimisation (Sec. III
 * middle-end).  Rectified pair: for each left keypoint the candidates are
 * right keypoints within one pyramid level, within a row band of
 * ceil(row_band_px * zeta^n) s0 rows, and with 0 <= X_l - X_r <= max_disp.
 * The best candidate minimises (Hamming distance, disparity, index) and is
 * accepted when the distance is at most match_max_dist.                     */

int32_t or_match_band(int32_t n, float scale, int32_t row_band_px)
{
    double s = or_level_scale(scale, n);
    return (int32_t)ceil((double)row_band_px * s);
}

static int32_t popcount32(uint32_t v)
{
    int32_t c = 0;
    while (v) { c += (int32_t)(v & 1u); v >>= 1; }
    return c;
}

void or_match(const or_keypoints *Lk, const or_keypoints *Rk, const or_params *p,
              int32_t *right_idx, int16_t *disparity, uint16_t *dist)
{
    for (int32_t i = 0; i < Lk->count; ++i) {
        int32_t nl = Lk->level[i];
        int32_t band = or_match_band(nl, p->scale, p->row_band_px);
        int32_t best_j = -1, best_d = 0x7fffffff, best_disp = 0x7fffffff;
        for (int32_t j = 0; j < Rk->count; ++j) {
            int32_t nr = Rk->level[j];
            if (nr < nl - 1 || nr > nl + 1) continue;
            int32_t dy = (int32_t)Rk->Y[j] - (int32_t)Lk->Y[i];
            if (dy < -band || dy > band) continue;
            int32_t disp = (int32_t)Lk->X[i] - (int32_t)Rk->X[j];
            if (disp < 0 || disp > p->max_disp) continue;
            int32_t d = 0;
            for (int32_t w = 0; w < 8; ++w)
                d += popcount32(Lk->desc[(size_t)i * 8 + w] ^ Rk->desc[(size_t)j * 8 + w]);
            if (d < best_d || (d == best_d && disp < best_disp)) {
                best_d = d; best_disp = disp; best_j = j;
            }
        }
        if (best_j < 0) {
            right_idx[i] = -1; disparity[i] = 0; dist[i] = 0xFFFF;
        } else if (best_d <= p->match_max_dist) {
            right_idx[i] = best_j; disparity[i] = (int16_t)best_disp; dist[i] = (uint16_t)best_d;
        } else {
            right_idx[i] = -1; disparity[i] = 0; dist[i] = (uint16_t)best_d;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Correlation minimisation (Sec. III, middle-end stereo matching: the SLAM
 * pipeline figure names it beside descriptor-distance minimisation; the
 * text gives no detail).  Reading: the sub-pixel refinement of the stereo
 * SLAM system the paper builds on, restated here.  For each left keypoint i
 * with an accepted descriptor match j, on the left keypoint's level n of
 * both raw pyramids (s = zeta^n):
 *   xr0 = floor(X_j / s + 0.5), the match's s0 column at level n;
 *   for shifts t = -L..L: the (2w+1)^2 patches centred on (x_i, y_i) in the
 *   left level and on (xr0 + t, y_i) in the right level, each minus its own
 *   centre pixel, and SAD(t) = sum of |left - right|; t* = the first
 *   minimum; a window leaving the level rejects (SAD reported as none);
 *   t* = -L or t* = L rejects (a minimum at the end of the search);
 *   d1, d2, d3 = SAD(t* - 1), SAD(t*), SAD(t* + 1); the parabola through
 *   them peaks at delta = (d1 - d3) / (2 (d1 + d3 - 2 d2)); a flat minimum
 *   (d1 + d3 = 2 d2) or |delta| > 1 rejects;
 *   disparity = s (x_i - xr0 - t* - delta) in s0 pixels; outside
 *   [0, max_disp] rejects; depth = bf / max(disparity, 0.01) when bf > 0.
 * Then, over the pair's matches that survived, median = the SAD at index
 * count / 2 of the ascending list; a match with 10 SAD > 21 median (SAD
 * above 2.1 times the median, in integers) is rejected as an outlier.  The
 * decisions use integers; delta, disparity and depth are IEEE double,
 * reported as float.  Outputs per left keypoint: disparity (-1 rejected),
 * depth (0 rejected), SAD(t*) (0xFFFFFFFF when no SAD was computed).      */

static void sp_levels(const uint8_t *L0, int32_t W0, int32_t H0, int32_t pitch0, const or_params *p,
                      uint8_t **lev, int32_t *Wn, int32_t *Hn)
{
    int32_t c[OR_MAX_LEVELS];
    or_level_geometry(W0, H0, p->levels, p->scale, p->cell, Wn, Hn, c);
    for (int32_t n = 0; n < p->levels; ++n) {
        lev[n] = (uint8_t *)malloc((size_t)Wn[n] * (size_t)Hn[n]);
        if (n == 0) {
            for (int32_t y = 0; y < H0; ++y) memcpy(lev[0] + (size_t)y * W0, L0 + (size_t)y * pitch0, (size_t)W0);
        } else {
            or_pyramid_level(L0, W0, H0, pitch0, p->scale, n, lev[n], Wn[n], Hn[n], Wn[n]);
        }
    }
}

static int cmp_u32(const void *a, const void *b)
{
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

void or_subpixel(const uint8_t *left0, const uint8_t *right0, int32_t W0, int32_t H0, int32_t pitch0,
                 const or_keypoints *Lk, const or_keypoints *Rk, const int32_t *right_idx,
                 const or_params *p, int32_t w, int32_t L, double bf,
                 float *disp_out, float *depth_out, uint32_t *sad_out)
{
    uint8_t *lv[OR_MAX_LEVELS], *rv[OR_MAX_LEVELS];
    int32_t Wn[OR_MAX_LEVELS], Hn[OR_MAX_LEVELS];
    sp_levels(left0, W0, H0, pitch0, p, lv, Wn, Hn);
    sp_levels(right0, W0, H0, pitch0, p, rv, Wn, Hn);
    uint32_t *kept = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(Lk->count > 0 ? Lk->count : 1));
    int32_t n_kept = 0;
    for (int32_t i = 0; i < Lk->count; ++i) {
        disp_out[i] = -1.0f;
        depth_out[i] = 0.0f;
        sad_out[i] = 0xFFFFFFFFu;
        int32_t j = right_idx[i];
        if (j < 0) continue;
        int32_t n = Lk->level[i], xi = Lk->x[i], yi = Lk->y[i];
        double s = or_level_scale(p->scale, n);
        int32_t xr0 = (int32_t)floor((double)Rk->X[j] / s + 0.5);
        int32_t W = Wn[n], H = Hn[n];
        if (xi - w < 0 || xi + w >= W || yi - w < 0 || yi + w >= H || xr0 - L - w < 0 || xr0 + L + w >= W)
            continue;
        const uint8_t *A = lv[n], *B = rv[n];
        int32_t lc = A[(size_t)yi * W + xi];
        int64_t sad[2 * 7 + 1] = { 0 };
        int32_t best = 0;
        for (int32_t t = -L; t <= L; ++t) {
            int32_t rc = B[(size_t)yi * W + xr0 + t];
            int64_t acc = 0;
            for (int32_t dy = -w; dy <= w; ++dy)
                for (int32_t dx = -w; dx <= w; ++dx) {
                    int32_t a = (int32_t)A[(size_t)(yi + dy) * W + xi + dx] - lc;
                    int32_t b = (int32_t)B[(size_t)(yi + dy) * W + xr0 + t + dx] - rc;
                    acc += a > b ? a - b : b - a;
                }
            sad[t + L] = acc;
            if (acc < sad[best]) best = t + L;
        }
        int32_t ts = best - L;
        sad_out[i] = (uint32_t)sad[best];
        if (ts == -L || ts == L) continue;
        int64_t d1 = sad[best - 1], d2 = sad[best], d3 = sad[best + 1];
        int64_t num = d1 - d3, den = 2 * (d1 + d3 - 2 * d2);
        if (den == 0) continue;
        if ((num < 0 ? -num : num) > den) continue;
        int64_t q = (int64_t)xi - xr0 - ts;
        /* disparity >= 0  <=>  q den >= num;  disparity <= max_disp  <=>  s (q den - num) <= max_disp den */
        if (q * den < num) continue;
        if (s * (double)(q * den - num) > (double)p->max_disp * (double)den) continue;
        double delta = (double)num / (double)den;
        double disp = s * ((double)q - delta);
        disp_out[i] = (float)disp;
        depth_out[i] = bf > 0.0 ? (float)(bf / (disp > 0.01 ? disp : 0.01)) : 0.0f;
        kept[n_kept++] = (uint32_t)sad[best];
    }
    if (n_kept > 0) {
        qsort(kept, (size_t)n_kept, sizeof(uint32_t), cmp_u32);
        uint64_t median = kept[n_kept / 2];
        for (int32_t i = 0; i < Lk->count; ++i)
            if (disp_out[i] >= 0.0f && 10u * (uint64_t)sad_out[i] > 21u * median) {
                disp_out[i] = -1.0f;
                depth_out[i] = 0.0f;
            }
    }
    free(kept);
    for (int32_t n = 0; n < p->levels; ++n) { free(lv[n]); free(rv[n]); }
}

/* ------------------------------------------------------------------ */
/* Feature tracking by projection (Sec. III, middle-end: feature matching and
 * tracking, with the conic projections of map points; the text gives no
 * detail).  Reading: the caller projects its map points (or the previous
 * frame's keypoints) into the current frame with its own pose or motion
 * model and passes, per query q, the predicted s0 position (u_q, v_q), the
 * predicted level n_q and the 256-bit descriptor.  Candidates are the
 * frame's keypoints k with level in [n_q - 1, n_q + 1] inside the square
 * window |X_k - u_q| <= r_q, |Y_k - v_q| <= r_q, r_q = radius * zeta^n_q.
 * The window test is a floating-point decision, taken in IEEE float like the
 * GPU kernel: r_q = fl(radius * fl(zeta^n_q)), |fl(X_k - u_q)| <= r_q.  The
 * best candidate minimises (Hamming distance, index); it is accepted when
 * its distance is at most max_dist and, if another candidate exists, 10 best
 * <= 9 second (ratio 0.9 against the second-smallest distance, in integers).
 * A predicted level of 8 or more has no candidates.  Outputs: idx (-1 none
 * or rejected) and dist (best distance, 0xFFFF when there is no candidate). */
void or_track(const or_keypoints *Kf, float scale, const float *u, const float *v, const uint8_t *lvl,
              const uint32_t *desc, int32_t n, float radius, int32_t max_dist,
              int32_t *idx_out, uint16_t *dist_out)
{
    for (int32_t q = 0; q < n; ++q) {
        /* the band n - 1 .. n + 1 holds only the frame's levels: a query one
         * level past the deepest still meets that level, deeper ones none */
        float zf = (float)or_level_scale(scale, lvl[q]);
        volatile float r = radius * zf;  /* one float rounding, no contraction */
        int32_t best = -1, bd = 0x7fffffff, sd = 0x7fffffff;
        for (int32_t k = 0; k < Kf->count; ++k) {
            int32_t m = Kf->level[k];
            if (m < (int32_t)lvl[q] - 1 || m > (int32_t)lvl[q] + 1) continue;
            volatile float dx = (float)Kf->X[k] - u[q];
            volatile float dy = (float)Kf->Y[k] - v[q];
            if (fabsf(dx) > r || fabsf(dy) > r) continue;
            int32_t d = 0;
            for (int32_t w = 0; w < 8; ++w)
                d += popcount32(desc[(size_t)q * 8 + w] ^ Kf->desc[(size_t)k * 8 + w]);
            if (d < bd) { sd = bd; bd = d; best = k; }
            else if (d < sd) { sd = d; }
        }
        if (best < 0) { idx_out[q] = -1; dist_out[q] = 0xFFFF; continue; }
        dist_out[q] = (uint16_t)bd;
        int ok = bd <= max_dist && (sd == 0x7fffffff || 10 * bd <= 9 * sd);
        idx_out[q] = ok ? best : -1;
    }
}
