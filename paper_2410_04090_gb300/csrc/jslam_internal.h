// Internal types shared by the host code and the kernels of libjslam.
//
// The whole batch (every image of every stereo pair, every pyramid level) is
// described by three device tables built on the host:
//   ImageDesc[2 * pairs]   one per image (pair p: left = 2p, right = 2p + 1)
//   LevelDesc[sum levels]  one per (image, level), image-major
//   PairDesc[pairs]        stereo matching outputs
// and each kernel's grid is a flat list of work units mapped onto these
// tables through small prefix arrays (tiles per level, segments per level),
// so a batch of mixed image sizes and pyramid depths runs in one launch per
// stage.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace jslam {

constexpr int kMaxLevels = 8;
constexpr int kBins = 30;        // orientation sectors of 12 degrees
constexpr int kPairs = 256;      // BRIEF point pairs
constexpr int kDiskR = 15;       // intensity-centroid disk radius
constexpr int kPatR = 13;        // rotated BRIEF offsets lie in [-13, 13]
constexpr int kPatPitch = 32;    // row pitch of the staged 27 x 27 BRIEF patch (8 aligned words)
constexpr int kMaxSegment = 4096;  // candidate slots per (level, cell row)
constexpr int kMaxImages = 256;    // images per batch (two per stereo pair)

// Pyramid tile (outputs per CTA) and thread count.
constexpr int kPyrTW = 128, kPyrTH = 32, kPyrThreads = 256;
// Detection tile: at most this many pixels a side (host picks cells per CTA).
constexpr int kFastMaxTile = 128, kFastThreads = 256;

// Row stride of the bit-planes in 16-byte units for a tile of nch 32-pixel
// chunks: chunks 0..nch (32 bytes each) and a 16-byte pad, an odd count, so
// that the 128-bit loads of two neighbouring rows fall on the two halves of
// the shared-memory banks.
__host__ __device__ inline int bs_row_units(int nch) { return 2 * (nch + 1) + 1; }
constexpr int kFastMaxCellsPerCta = 2048;  // cells x k per CTA
constexpr int kLutWords = 2048;            // 2^16-entry corner bit table
constexpr int kSkipC = 16;                 // channels of the learned cell-skip net
constexpr int kSkipTileW = 26, kSkipTileH = 12;  // its logits per CTA (grid pitch 26 + 6 = 32)
constexpr int kRefineMaxW = 10, kRefineMaxL = 7;  // correlation window half-size and search radius limits
constexpr int kNmsThreads = 128;
constexpr int kFinThreads = 1024;

// Device error bits (OR-ed into the context's error word).
constexpr uint32_t kErrSegment = 1u << 0;  // a segment was larger than kMaxSegment
constexpr uint32_t kErrDecode = 1u << 1;   // a candidate decoded outside its level
constexpr uint32_t kErrTimeout = 1u << 2;  // a bounded wait for a tile load gave up

struct KpOut {
    uint16_t *x, *y, *X, *Y, *response;
    uint8_t *level, *angle_bin, *k_levels;
    uint32_t *k_resp;
    float *angle;
    uint32_t *desc;  // capacity x 8
    int32_t capacity;
};

struct LevelDesc {
    const uint8_t *raw;      // raw level (level 0: aligned copy of the input)
    uint8_t *raw_w;          // the same buffer, written by the pyramid kernel
    uint8_t *blur;           // blurred level
    const uint32_t *tapx;    // bilinear taps: src index | weight << 16 (levels >= 1)
    const uint32_t *tapy;
    const uint16_t *projx;   // s0 projection of each x / y of the level
    const uint16_t *projy;
    // source of the resampling: nullptr = level 0 (the input image); in the
    // cascaded pyramid the raw level n - 1 (taps then use one factor zeta)
    const uint8_t *src;
    int32_t src_W, src_H, src_pitch;
    int32_t W, H, pitch;     // pitch of raw: width rounded up to 128
    int32_t blur_pitch;
    int32_t c, cells_x, cells_y;
    int32_t bx, by;          // cells per detection tile
    int32_t cinv;            // ceil(2^16 / c): exact division by c for values < 128
    const CUtensorMap *tmap; // TMA map of the raw level (nullptr: tiles loaded with plain loads)
    int32_t box_w, box_h;    // detection tile box: bytes per row (multiple of 16) and rows
    int32_t slot_base;       // first candidate slot of the level
    int32_t seg_base;        // first segment (cell row) of the level
    int32_t image, level;
    int32_t band;            // stereo row band for keypoints of this level
    double zeta;             // zeta^n (repeated multiplication in double)
    float zeta_f, zeta_inv_f; // zeta^n and 1 / zeta^n rounded to float
};

struct ImageDesc {
    int32_t W0, H0;
    int32_t levels, level_base;
    int32_t eps_hi, eps_lo;  // eps_lo <= 0: no fallback
    int32_t max_feats;
    int32_t slot_base, slot_count;
    int32_t seg_base, seg_count;
    uint32_t *map;           // W0 * H0 packed (K_l << 16 | K_r); all zero between runs
    int32_t *count;          // keypoint count written by finalisation
    int32_t *count_hdr;      // the same count in the header of the pair's result block
    int32_t *level_start;    // kMaxLevels + 1 entries
    // row index of the canonical list, per level H0 + 1 entries: entry v is
    // the first index of the level whose Y is >= v (the level's end if none);
    // written by k_pfa_finalize for levels with keypoints, read by k_match
    int32_t *row_first;
    KpOut out;
    // learned cell-skip (skip == nullptr: exact mode)
    float *skip_logits;      // skip_h8 x skip_w8 logits at 1/8 scale
    uint8_t *skip;           // per s0 culling cell: 1 = skipped
    int32_t skip_w8, skip_h8, skip_cells_x, skip_cells_y, skip_c0;
};

// Device copy of the skip net: BF16 weights, FP32 biases.
struct SkipModelDev {
    const uint16_t *w1, *w2, *w3;  // [16][9], [16][16][9], [16][9]
    const float *b1, *b2;          // [16], [16]
    float b3;
};

struct PairDesc {
    int32_t left, right;
    int32_t *match_idx;
    int16_t *disparity;
    uint16_t *dist;
    float *sub_disp;         // correlation minimisation: sub-pixel disparity (-1 rejected)
    float *depth;            //   depth bf / disparity (0 rejected)
    uint32_t *corr;          //   SAD at the best shift (0xFFFFFFFF: none computed)
};

// Parameters fixed for a context.
struct Params {
    int32_t p_min, p_max, k, nms_rad, border, rule;
    int32_t max_disp, max_dist;
    int32_t resp_arc;        // 1: arc response (see ring_response.cuh); 0: sum over the whole circle
};

// Level-0 pixels of every image of the call.  Passed by value as a kernel
// parameter so that a plan (which depends only on the shapes) is reused
// across calls whose input buffers differ.
struct Inputs {
    const uint8_t *ptr[kMaxImages];
    int32_t pitch[kMaxImages];
};

// Everything the kernels of one extraction need.
// One detection tile of the bit-sliced kernel, prepared on the host: the
// tile's place in its level, the level's and image's scalars, and the
// 16-byte-aligned ranges of the level's s0 projection tables that cover the
// tile's columns and rows.  The kernel copies it into shared memory with a
// bulk copy, so no chain of descriptor loads precedes a tile.
constexpr int kPrjBytes = 288;  // staged projection bytes per axis: 2 x 128 + alignment slack, rounded to 16
struct __align__(16) TileRec {
    int32_t ccx0, ccy0, ncx, ncy, x0, y0, tw, th, xs, ys, delta;
    int32_t c, cells_x, W, H, cinv, box_w, box_h, slot_base, pitch;
    int32_t eps_hi, eps_lo, W0, skip_c0, skip_cells_x;
    int32_t prj_bytes_x, prj_bytes_y;  // bulk copy sizes (multiples of 16)
    int32_t prj_off_x, prj_off_y;      // element offset of x0 / y0 in the staged copies
    int32_t image;                     // the tile's image
    const uint8_t *raw;
    const CUtensorMap *tmap;           // nullptr: the box is loaded with plain loads
    const uint16_t *prj_src_x, *prj_src_y;
    uint32_t *map;
    const uint8_t *skip;
};
static_assert(sizeof(TileRec) % 16 == 0, "bulk copies move multiples of 16 bytes");

struct Batch {
    const ImageDesc *images;
    const LevelDesc *levels;
    const PairDesc *pairs;
    const int32_t *pyr_tile_base;   // n_levels + 1
    const int32_t *pyr_tile_level;  // level index of each pyramid tile
    const int32_t *pyr_order;       // pyramid tiles ordered by level number (cascaded pyramid)
    int32_t pyr_pass_first[kMaxLevels + 1];  // first entry of pyr_order of each level number
    int32_t pyr_pass;               // -1: one launch over every tile; n: the tiles of level number n
    const int32_t *fast_tile_base;  // n_levels + 1
    const int32_t *fast_tile_level; // level index of each detection tile
    const int32_t *seg_level;       // level index of each segment
    int32_t n_images, n_levels, n_pairs, n_segments;
    int32_t max_segment;            // largest segment (cells_x x k slots) of the batch
    int32_t pyr_tiles, fast_tiles;
    int32_t max_capacity;           // largest keypoint capacity of any image
    int32_t fast_smem;              // dynamic shared memory of the detection kernel
    int32_t fast_max_box, fast_max_px, fast_max_cells;  // its tile layout maxima
    int32_t fast_max_planes;        // bit-plane bytes of the largest tile box
    int32_t fast_bits;              // 1: bit-sliced ring test (P_min = 9, P_max = 13)
    const TileRec *tile_rec;        // one per detection tile
    const uint32_t *corner_lut;     // bit m: P_min <= longest circular run of m <= P_max
    uint32_t *slots;                // candidate keys per slot
    uint32_t *slot_k;               // PFA scores seen by each slot
    int32_t *slot_rank;             // rank within its segment, -1 if suppressed
    int32_t *seg_count;             // survivors per segment
    int32_t *seg_off;               // exclusive prefix of seg_count per image
    int32_t *canon;                 // slot of each canonical position
    const int8_t *pattern;          // kBins x kPairs x 4
    const uint32_t *pattern_off;    // kBins x kPairs: int16 patch offsets of p | of q << 16 (pitch kPatPitch)
    const double *bin_cos, *bin_sin;
    const float *bin_cosf, *bin_sinf;  // the same tables rounded to float (fast sector test)
    uint32_t *err;
    Params prm;
    int32_t skip_max_tiles, skip_max_cells;  // learned cell-skip launch shape
    int32_t *skip_any;              // learned skip: per image, nonzero once its proposal skipped a cell
    int32_t nms_kernel;             // 0: a warp per segment where segments allow, 1: a CTA per segment
    int32_t fast_ctas_per_sm;       // persistent detection CTAs per SM (0: as many as fit)
    Inputs in;
};

// Kernel launchers (one per stage), all on `stream`.
cudaError_t launch_pyramid(const Batch &b, cudaStream_t stream);
cudaError_t launch_fast_cull(const Batch &b, cudaStream_t stream);
cudaError_t launch_wait_selftest(uint32_t *err, cudaStream_t stream);
cudaError_t launch_pfa_nms(const Batch &b, cudaStream_t stream);
cudaError_t launch_pfa_finalize(const Batch &b, cudaStream_t stream);
cudaError_t launch_orient_desc(const Batch &b, cudaStream_t stream);
cudaError_t launch_match(const Batch &b, cudaStream_t stream);
cudaError_t launch_refine(const Batch &b, int w, int L, double bf, cudaStream_t stream);

// Feature tracking by projection: caller-projected queries against one image's keypoints.
struct TrackArgs {
    int32_t image, n, max_dist;
    float radius;
    float zeta_f[kMaxLevels + 1];  // zeta^n rounded to float, n = 0..kMaxLevels
    const float *u, *v;
    const uint8_t *level;
    const uint32_t *desc;
    int32_t *out_idx;
    uint16_t *out_dist;
};
cudaError_t launch_track(const Batch &b, const TrackArgs &a, cudaStream_t stream);
cudaError_t launch_fc_ablation(const Batch &b, uint16_t *crf, const uint64_t *off, uint32_t *keys,
                               const int *level_blocks, int max_pixels, int max_levels, const int *level_cells_y,
                               const int *level_c, int n_max, cudaStream_t stream, cudaEvent_t mid);
cudaError_t launch_skipnet(const Batch &b, const SkipModelDev &m, float thresh, cudaStream_t stream);
cudaError_t set_blur_weights(const int32_t w[7]);
cudaError_t configure_kernels();
cudaError_t configure_skipnet();
int skipnet_smem_bytes();

}  // namespace jslam
