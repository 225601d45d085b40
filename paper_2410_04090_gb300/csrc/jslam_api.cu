// C ABI of libjslam: context, grow-only device buffers, batch plans and the
// launch sequence of the stereo frontend.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <utility>
#include <vector>

#include <cudaTypedefs.h>
#include <nvtx3/nvToolsExt.h>

#include "jslam.h"
#include "jslam_internal.h"
#include "tables.h"

namespace jslam {
int fast_smem_bytes(int max_box, int max_px, int max_cells, int k, int max_planes);
const void *pyramid_kernel();
cudaError_t detect_ctas_that_fit(const Batch &b, int *per_sm);
}

using namespace jslam;

namespace {

// Host-side NVTX range around each stage's launch, named by stage, so that a
// profiler's timeline shows which launch belongs to which step of the path.
// With no profiler attached the push and pop are no-ops.
const char *const kStageNames[JSLAM_NUM_STAGES] = { "jslam pyramid", "jslam skip proposal", "jslam detect",
                                                     "jslam PFA NMS",  "jslam PFA final",     "jslam ORB",
                                                     "jslam match",    "jslam refine" };
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// cuTensorMapEncodeTiled through the runtime's driver entry point (no
// link-time dependency on the driver library).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        cudaGetLastError();
    }
    return fn;
}

// Detection tile box of a level: rows of box_w bytes (a multiple of 16 that
// covers the tile, its 4-pixel halo on both sides and up to 12 bytes of
// alignment slack on the left) and box_h rows (3-row halo above and below).
void detect_box(int tw, int th, int *box_w, int *box_h)
{
    *box_w = (int)align_up((size_t)(tw + 8 + 12), 16);
    *box_h = th + 6;
}

constexpr size_t kLevelSlack = 256;  // bytes after each level buffer

// Optional allocation-failure injection for host-side fault tests: the
// environment variable JSLAM_FAIL_ALLOC_AFTER=n makes the (n+1)-th device
// allocation of the process report failure.
int g_alloc_budget = -2;

cudaError_t dev_alloc(void **p, size_t bytes)
{
    if (g_alloc_budget == -2) {
        const char *e = std::getenv("JSLAM_FAIL_ALLOC_AFTER");
        g_alloc_budget = e ? std::atoi(e) : -1;
    }
    if (g_alloc_budget == 0) return cudaErrorMemoryAllocation;
    if (g_alloc_budget > 0) --g_alloc_budget;
    return cudaMalloc(p, bytes);
}

// Device buffer that only grows (the Synchronized Shared Memory policy of
// Sec. III: reallocate only when a request exceeds the current size).
struct GrowBuf {
    void *ptr = nullptr;
    size_t cap = 0;
    // Grows to at least `bytes`; *fresh tells whether it was (re)allocated.
    // Zero-filling is ordered on `stream` (synchronous when null).
    cudaError_t ensure(size_t bytes, bool zero, bool *fresh, cudaStream_t stream = nullptr)
    {
        if (fresh) *fresh = false;
        if (bytes <= cap) return cudaSuccess;
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        cap = 0;
        const size_t want = align_up(bytes + bytes / 4, 1 << 20);
        cudaError_t e = dev_alloc(&ptr, want);
        if (e != cudaSuccess) { ptr = nullptr; return e; }
        cap = want;
        if (zero) e = stream ? cudaMemsetAsync(ptr, 0, want, stream) : cudaMemset(ptr, 0, want);
        if (fresh) *fresh = true;
        return e;
    }
    void release()
    {
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        cap = 0;
    }
    template <class T> T *as(size_t byte_off = 0) const
    {
        return reinterpret_cast<T *>(static_cast<char *>(ptr) + byte_off);
    }
};

// Signature of a batch: everything that changes the plan tables (not the
// input buffers, which reach the kernels through Inputs).
struct JobKey {
    int W, H, levels, eps, cell, feats;
    uint32_t scale_bits;
    int mem[2];
    bool operator==(const JobKey &o) const { return std::memcmp(this, &o, sizeof(JobKey)) == 0; }
};

// Byte layout of one image's outputs (capacity C) inside a pair's result block.
struct SideLayout {
    size_t desc, k_resp, angle, x, y, X, Y, response, level, angle_bin, k_levels, end;
};

SideLayout side_layout(int C, size_t base)
{
    SideLayout s;
    size_t o = base;
    auto take = [&](size_t bytes) { size_t at = o; o = align_up(o + bytes, 256); return at; };
    s.desc = take((size_t)C * 32);
    s.k_resp = take((size_t)C * 4);
    s.angle = take((size_t)C * 4);
    s.x = take((size_t)C * 2);
    s.y = take((size_t)C * 2);
    s.X = take((size_t)C * 2);
    s.Y = take((size_t)C * 2);
    s.response = take((size_t)C * 2);
    s.level = take((size_t)C);
    s.angle_bin = take((size_t)C);
    s.k_levels = take((size_t)C);
    s.end = o;
    return s;
}

// A pair's result block starts with a 16-byte header of int32 counts (left
// keypoints, right keypoints, two reserved), written by the finalisation, so
// that a downloaded block describes itself.
constexpr size_t kBlockHeader = 16;
struct PairLayout {
    int capacity;
    SideLayout side[2];
    size_t match_idx, disparity, dist, sub_disp, depth, corr, bytes;
};

PairLayout pair_layout(int max_feats)
{
    PairLayout p;
    p.capacity = (int)align_up((size_t)max_feats, 32);
    p.side[0] = side_layout(p.capacity, align_up(kBlockHeader, 256));
    p.side[1] = side_layout(p.capacity, p.side[0].end);
    size_t o = p.side[1].end;
    p.match_idx = o; o = align_up(o + (size_t)p.capacity * 4, 256);
    p.disparity = o; o = align_up(o + (size_t)p.capacity * 2, 256);
    p.dist = o; o = align_up(o + (size_t)p.capacity * 2, 256);
    p.sub_disp = o; o = align_up(o + (size_t)p.capacity * 4, 256);
    p.depth = o; o = align_up(o + (size_t)p.capacity * 4, 256);
    p.corr = o; o = align_up(o + (size_t)p.capacity * 4, 256);
    p.bytes = o;
    return p;
}

}  // namespace

struct jslam_ctx {
    jslam_config cfg;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    jslam_status status = JSLAM_OK;

    // constant tables
    GrowBuf consts;  // pattern | cos | sin | corner table
    int8_t *d_pattern = nullptr;
    uint32_t *d_pattern_off = nullptr;
    double *d_cos = nullptr, *d_sin = nullptr;
    float *d_cosf = nullptr, *d_sinf = nullptr;
    uint32_t *d_lut = nullptr;

    // per-batch buffers
    GrowBuf plan, levels, maps, scratch, results, staging, counts;
    int32_t *h_counts = nullptr;  // pinned mirror: 2 * max_pairs counts + error word
    bool synced = false;
    bool have_extract = false, have_match = false, have_refine = false;

    // current plan
    std::vector<JobKey> keys;
    std::vector<PairLayout> layouts;
    std::vector<size_t> result_off;
    std::vector<ImageDesc> h_images;
    std::vector<LevelDesc> h_levels;
    std::vector<size_t> staging_off;
    std::vector<float> pair_scale;  // scale factor of each pair of the current plan
    size_t slot_count = 0;          // candidate slots of the current plan
    // feature-culling ablation (the paper's CRF-matrix + MLPT/TEWA kernels)
    GrowBuf abl;
    std::vector<uint64_t> abl_off;
    cudaEvent_t abl_ev[3] = {};
    bool have_ablation = false;
    Batch batch{};
    Params prm{};

    // stage timing: events[0] before the first stage, events[i + 1] after stage i
    bool timing = false;
    cudaEvent_t events[JSLAM_NUM_STAGES + 1] = {};
    bool stage_done[JSLAM_NUM_STAGES] = {};

    // learned cell-skip model
    GrowBuf skipw, skipbuf;
    SkipModelDev skip_model{};
    bool skip_on = false;
    float skip_thresh = 0.0f;
    bool plan_skip = false;  // the current plan has skip buffers

    // launch-shape tuning and the captured graph
    jslam_tuning tune{128, 64, 0, 0, 0};
    jslam_tuning plan_tune{0, 0, 0, 0, 0};  // tuning the current plan was built with (tile fields)
    cudaGraphExec_t graph = nullptr;
    cudaGraph_t graph_src = nullptr;    // the captured graph (its node handles address `graph`)
    // its pyramid launches (one, or one per level in the cascaded pyramid):
    // the kernel that reads the input images, with the batch each got
    std::vector<cudaGraphNode_t> graph_pyr;
    std::vector<cudaKernelNodeParams> graph_pyr_params;
    std::vector<Batch> graph_pyr_batch;
    std::vector<JobKey> graph_keys;     // batch signature of the capture
    uint64_t graph_gen = 0;             // plan generation the graph was captured on
    int graph_pairs = 0;
    bool graph_timed = false;  // the graph records the stage events
    // generation of the plan: bumped whenever build_plan rebuilds the tables
    // or buffers, which invalidates a graph captured on an earlier plan
    uint64_t plan_gen = 0;
    float tune_ms = 0.0f;  // detection stage time of the last autotuned pick
};

namespace {

jslam_status fail(jslam_ctx *ctx, cudaError_t e)
{
    if (e == cudaSuccess) return JSLAM_OK;
    jslam_status s = (e == cudaErrorMemoryAllocation) ? JSLAM_ERR_NOMEM : JSLAM_ERR_CUDA;
    if (ctx && ctx->status == JSLAM_OK) ctx->status = s;
    cudaGetLastError();
    return s;
}

bool image_ok(const jslam_image &im, const jslam_config &cfg)
{
    if (!im.data || im.width < 1 || im.height < 1) return false;
    if (im.pitch < im.width) return false;
    if ((int64_t)im.pitch * im.height > (int64_t)UINT32_MAX) return false;  // kernels take 32-bit offsets
    if (im.width > cfg.max_width || im.height > cfg.max_height) return false;
    if (im.memory != JSLAM_MEM_DEVICE && im.memory != JSLAM_MEM_HOST) return false;
    return true;
}

jslam_status check_job(const jslam_ctx *ctx, const jslam_stereo_job &j)
{
    const jslam_config &cfg = ctx->cfg;
    if (!image_ok(j.left, cfg) || !image_ok(j.right, cfg)) return JSLAM_ERR_ARG;
    if (j.left.width != j.right.width || j.left.height != j.right.height) return JSLAM_ERR_ARG;
    if (j.levels < 1 || j.levels > cfg.max_levels) return JSLAM_ERR_ARG;
    if (!(j.scale > 1.0f) || !(j.scale < 16.0f)) return JSLAM_ERR_ARG;
    if (j.fast_thresh < 1 || j.fast_thresh > 254) return JSLAM_ERR_ARG;
    if (j.cell < 1 || j.cell > 128) return JSLAM_ERR_ARG;
    if (j.max_feats < 1 || j.max_feats > cfg.max_feats) return JSLAM_ERR_ARG;
    const Geometry g = level_geometry(j.left.width, j.left.height, j.levels, j.scale, j.cell);
    for (int n = 0; n < j.levels; ++n) {
        if (g.W[n] < 2 * cfg.border + 1 || g.H[n] < 2 * cfg.border + 1) return JSLAM_ERR_ARG;
        const int cells_x = (g.W[n] + g.c[n] - 1) / g.c[n];
        if (cells_x * cfg.k_per_cell > kMaxSegment) return JSLAM_ERR_ARG;
    }
    return JSLAM_OK;
}

// Cells per detection tile: about tile_w x tile_h pixels (128 x 64 by
// default), capped in cells x k; the tile width is kept a multiple of 4
// pixels where possible so that tiles start on word boundaries.
void fast_block(int c, int k, int tile_w, int tile_h, int *bx, int *by)
{
    int x = tile_w / c > 1 ? tile_w / c : 1;
    for (int cand = x; cand >= 1; --cand)
        if ((cand * c) % 4 == 0) { x = cand; break; }
    int y = tile_h / c > 1 ? tile_h / c : 1;
    while (x * y * k > kFastMaxCellsPerCta) {
        if (y > 1) --y; else --x;
    }
    *bx = x;
    *by = y;
}

// Build (or reuse) the plan of a batch and upload it.
jslam_status build_plan(jslam_ctx *ctx, const jslam_stereo_job *jobs, int n)
{
    const jslam_config &cfg = ctx->cfg;
    std::vector<JobKey> keys(n);
    for (int p = 0; p < n; ++p) {
        JobKey &k = keys[p];
        std::memset(&k, 0, sizeof(k));
        k.W = jobs[p].left.width; k.H = jobs[p].left.height; k.levels = jobs[p].levels;
        k.eps = jobs[p].fast_thresh; k.cell = jobs[p].cell; k.feats = jobs[p].max_feats;
        std::memcpy(&k.scale_bits, &jobs[p].scale, 4);
        const jslam_image *im[2] = { &jobs[p].left, &jobs[p].right };
        for (int s = 0; s < 2; ++s) k.mem[s] = im[s]->memory;
    }
    if (keys == ctx->keys && ctx->plan_tune.tile_w_px == ctx->tune.tile_w_px &&
        ctx->plan_tune.tile_h_px == ctx->tune.tile_h_px && ctx->plan_tune.tile_order == ctx->tune.tile_order &&
        ctx->plan_skip == ctx->skip_on)
        return JSLAM_OK;
    ++ctx->plan_gen;

    const int n_img = 2 * n;
    const int k = cfg.k_per_cell;
    std::vector<Geometry> geo(n);
    std::vector<PairLayout> layouts(n);
    std::vector<size_t> result_off(n);
    size_t result_bytes = 0, level_bytes = 0, map_bytes = 0, staging_bytes = 0, table_bytes = 0;
    int n_levels = 0, n_slots = 0, n_segs = 0, max_cap = 0;
    int max_box = 0, max_px = 0, max_cells = 0, max_planes = 0;
    for (int p = 0; p < n; ++p) {
        geo[p] = level_geometry(jobs[p].left.width, jobs[p].left.height, jobs[p].levels, jobs[p].scale, jobs[p].cell);
        layouts[p] = pair_layout(jobs[p].max_feats);
        result_off[p] = result_bytes;
        result_bytes += layouts[p].bytes;
        max_cap = std::max(max_cap, layouts[p].capacity);
        const Geometry &g = geo[p];
        for (int s = 0; s < 2; ++s) {
            for (int l = 0; l < g.levels; ++l) {
                const size_t pitch = align_up((size_t)g.W[l], 128);
                level_bytes += 2 * align_up(pitch * g.H[l] + kLevelSlack, 256);
                table_bytes += align_up((size_t)(g.W[l] + g.H[l]) * 4, 16);  // taps
                table_bytes += align_up((size_t)(g.W[l] + g.H[l]) * 2, 16);  // projection
                const int cx = (g.W[l] + g.c[l] - 1) / g.c[l], cy = (g.H[l] + g.c[l] - 1) / g.c[l];
                n_slots += cx * cy * k;
                n_segs += cy;
                int bx, by;
                fast_block(g.c[l], k, ctx->tune.tile_w_px, ctx->tune.tile_h_px, &bx, &by);
                const int tw = std::min(bx * g.c[l], g.W[l]), th = std::min(by * g.c[l], g.H[l]);
                int bw, bh;
                detect_box(tw, th, &bw, &bh);
                max_box = std::max(max_box, bw * bh);
                max_planes = std::max(max_planes, bh * bs_row_units((tw + 31) / 32) * 16);
                max_px = std::max(max_px, tw * th);
                max_cells = std::max(max_cells, bx * by);
            }
            n_levels += g.levels;
            map_bytes += align_up((size_t)g.W[0] * g.H[0] * 4, 256);
            staging_bytes += align_up((size_t)align_up(g.W[0], 128) * g.H[0], 256);
        }
    }

    // Device arenas (grow-only).
    cudaError_t e;
    bool fresh = false;  // a fresh score map is zero-filled on the stream
    if ((e = ctx->levels.ensure(level_bytes + 256, false, nullptr)) != cudaSuccess) return fail(ctx, e);
    if ((e = ctx->maps.ensure(map_bytes + 256, true, &fresh, ctx->stream)) != cudaSuccess) return fail(ctx, e);
    if ((e = ctx->results.ensure(result_bytes + 256, true, nullptr, ctx->stream)) != cudaSuccess) return fail(ctx, e);
    bool any_host = false;
    for (int p = 0; p < n; ++p)
        any_host |= jobs[p].left.memory == JSLAM_MEM_HOST || jobs[p].right.memory == JSLAM_MEM_HOST;
    if (any_host && (e = ctx->staging.ensure(staging_bytes + 256, false, nullptr)) != cudaSuccess) return fail(ctx, e);
    // learned cell-skip buffers: logits at 1/8 scale and per-s0-cell flags
    size_t skip_bytes = 0;
    int skip_max_tiles = 0, skip_max_cells = 0;
    if (ctx->skip_on) {
        for (int p = 0; p < n; ++p) {
            const int w8 = (geo[p].W[0] + 7) / 8, h8 = (geo[p].H[0] + 7) / 8;
            const int cx = (geo[p].W[0] + jobs[p].cell - 1) / jobs[p].cell, cy = (geo[p].H[0] + jobs[p].cell - 1) / jobs[p].cell;
            skip_bytes += 2 * (align_up((size_t)w8 * h8 * 4, 256) + align_up((size_t)cx * cy, 256));
            skip_max_tiles = std::max(skip_max_tiles, ((w8 + kSkipTileW - 1) / kSkipTileW) * ((h8 + kSkipTileH - 1) / kSkipTileH));
            skip_max_cells = std::max(skip_max_cells, cx * cy);
        }
        skip_bytes += align_up(sizeof(int32_t) * (size_t)(2 * n), 256);  // per image: any cell skipped
        if ((e = ctx->skipbuf.ensure(skip_bytes + 256, false, nullptr)) != cudaSuccess) return fail(ctx, e);
    }
    size_t skip_off = 0;
    const size_t slot_words = (size_t)n_slots + 64;
    const size_t seg_words = (size_t)n_segs + 64;
    size_t row_words = 64;  // row index of each image's canonical list: levels x (H0 + 1)
    for (int p = 0; p < n; ++p) row_words += 2 * (size_t)geo[p].levels * (geo[p].H[0] + 1);
    const size_t scratch_bytes = slot_words * 4 * 4 + seg_words * 4 * 2 + row_words * 4;
    if ((e = ctx->scratch.ensure(scratch_bytes, false, nullptr)) != cudaSuccess) return fail(ctx, e);

    // Host tables: [images][levels][pairs][pyr base][fast base][seg level][taps/proj ...]
    size_t off = 0;
    auto reserve = [&](size_t bytes) { size_t at = off; off = align_up(off + bytes, 256); return at; };
    const size_t o_images = reserve(sizeof(ImageDesc) * n_img);
    const size_t o_levels = reserve(sizeof(LevelDesc) * n_levels);
    const size_t o_pairs = reserve(sizeof(PairDesc) * n);
    const size_t o_pyr = reserve(sizeof(int32_t) * (n_levels + 1));
    const size_t o_fast = reserve(sizeof(int32_t) * (n_levels + 1));
    const size_t o_seg = reserve(sizeof(int32_t) * (n_segs + 1));
    size_t n_fast_tiles = 0, n_pyr_tiles = 0;
    for (int p = 0; p < n; ++p)
        for (int l = 0; l < geo[p].levels; ++l) {
            n_pyr_tiles += 2 * (size_t)(((geo[p].W[l] + kPyrTW - 1) / kPyrTW) * ((geo[p].H[l] + kPyrTH - 1) / kPyrTH));
            int bx, by;
            fast_block(geo[p].c[l], k, ctx->tune.tile_w_px, ctx->tune.tile_h_px, &bx, &by);
            const int cx = (geo[p].W[l] + geo[p].c[l] - 1) / geo[p].c[l], cy = (geo[p].H[l] + geo[p].c[l] - 1) / geo[p].c[l];
            n_fast_tiles += 2 * (size_t)(((cx + bx - 1) / bx) * ((cy + by - 1) / by));
        }
    const size_t o_ftl = reserve(sizeof(int32_t) * (n_fast_tiles + 1));
    const size_t o_ptl = reserve(sizeof(int32_t) * (n_pyr_tiles + 1));
    const size_t o_porder = reserve(sizeof(int32_t) * (n_pyr_tiles + 1));
    const size_t o_trec = reserve(sizeof(TileRec) * (n_fast_tiles + 1));
    const size_t o_lstart = reserve(sizeof(int32_t) * (kMaxLevels + 1) * n_img);
    const size_t o_tmaps = reserve(sizeof(CUtensorMap) * (size_t)n_levels);
    const size_t o_tables = reserve(table_bytes + 256);
    if ((e = ctx->plan.ensure(off, false, nullptr)) != cudaSuccess) return fail(ctx, e);

    std::vector<char> host(off, 0);
    char *dplan = ctx->plan.as<char>();
    auto images = reinterpret_cast<ImageDesc *>(host.data() + o_images);
    auto levels = reinterpret_cast<LevelDesc *>(host.data() + o_levels);
    auto pairs = reinterpret_cast<PairDesc *>(host.data() + o_pairs);
    auto pyr_base = reinterpret_cast<int32_t *>(host.data() + o_pyr);
    auto fast_base = reinterpret_cast<int32_t *>(host.data() + o_fast);
    auto seg_level = reinterpret_cast<int32_t *>(host.data() + o_seg);
    auto ftile_level = reinterpret_cast<int32_t *>(host.data() + o_ftl);
    auto ptile_level = reinterpret_cast<int32_t *>(host.data() + o_ptl);
    size_t t_off = o_tables, lvl_off = 0, map_off = 0, stage_off = 0, row_off = 0;
    int li = 0, slot = 0, seg = 0, pyr = 0, fast = 0;
    ctx->staging_off.assign(n_img, 0);
    int32_t *dcounts = ctx->counts.as<int32_t>();

    for (int p = 0; p < n; ++p) {
        const Geometry &g = geo[p];
        const PairLayout &pl = layouts[p];
        char *rblock = ctx->results.as<char>(result_off[p]);
        for (int s = 0; s < 2; ++s) {
            const int img = 2 * p + s;
            const jslam_image &im = s == 0 ? jobs[p].left : jobs[p].right;
            ImageDesc &I = images[img];
            if (im.memory == JSLAM_MEM_HOST) {
                ctx->staging_off[img] = stage_off;
                stage_off += align_up(align_up(g.W[0], 128) * g.H[0], 256);
            }
            I.W0 = g.W[0]; I.H0 = g.H[0];
            I.levels = g.levels; I.level_base = li;
            I.eps_hi = jobs[p].fast_thresh; I.eps_lo = cfg.fast_thresh_lo;
            I.max_feats = jobs[p].max_feats;
            I.slot_base = slot; I.seg_base = seg;
            I.map = ctx->maps.as<uint32_t>(map_off);
            map_off += align_up((size_t)g.W[0] * g.H[0] * 4, 256);
            I.count = dcounts + img;
            I.count_hdr = reinterpret_cast<int32_t *>(rblock) + s;
            I.skip = nullptr;
            I.skip_logits = nullptr;
            I.skip_w8 = (g.W[0] + 7) / 8;
            I.skip_h8 = (g.H[0] + 7) / 8;
            I.skip_c0 = jobs[p].cell;
            I.skip_cells_x = (g.W[0] + jobs[p].cell - 1) / jobs[p].cell;
            I.skip_cells_y = (g.H[0] + jobs[p].cell - 1) / jobs[p].cell;
            if (ctx->skip_on) {
                I.skip_logits = ctx->skipbuf.as<float>(skip_off);
                skip_off += align_up((size_t)I.skip_w8 * I.skip_h8 * 4, 256);
                I.skip = ctx->skipbuf.as<uint8_t>(skip_off);
                skip_off += align_up((size_t)I.skip_cells_x * I.skip_cells_y, 256);
            }
            I.level_start = reinterpret_cast<int32_t *>(dplan + o_lstart) + img * (kMaxLevels + 1);
            I.row_first = ctx->scratch.as<int32_t>(4 * (slot_words * 4 + seg_words * 2) + row_off);
            row_off += 4 * (size_t)g.levels * (g.H[0] + 1);
            const SideLayout &sl = pl.side[s];
            I.out.capacity = pl.capacity;
            I.out.desc = reinterpret_cast<uint32_t *>(rblock + sl.desc);
            I.out.k_resp = reinterpret_cast<uint32_t *>(rblock + sl.k_resp);
            I.out.angle = reinterpret_cast<float *>(rblock + sl.angle);
            I.out.x = reinterpret_cast<uint16_t *>(rblock + sl.x);
            I.out.y = reinterpret_cast<uint16_t *>(rblock + sl.y);
            I.out.X = reinterpret_cast<uint16_t *>(rblock + sl.X);
            I.out.Y = reinterpret_cast<uint16_t *>(rblock + sl.Y);
            I.out.response = reinterpret_cast<uint16_t *>(rblock + sl.response);
            I.out.level = reinterpret_cast<uint8_t *>(rblock + sl.level);
            I.out.angle_bin = reinterpret_cast<uint8_t *>(rblock + sl.angle_bin);
            I.out.k_levels = reinterpret_cast<uint8_t *>(rblock + sl.k_levels);

            for (int l = 0; l < g.levels; ++l, ++li) {
                LevelDesc &L = levels[li];
                const double sc = zeta_pow(jobs[p].scale, l);
                L.W = g.W[l]; L.H = g.H[l]; L.c = g.c[l];
                L.cells_x = (L.W + L.c - 1) / L.c;
                L.cells_y = (L.H + L.c - 1) / L.c;
                fast_block(L.c, k, ctx->tune.tile_w_px, ctx->tune.tile_h_px, &L.bx, &L.by);
                L.cinv = (65536 + L.c - 1) / L.c;
                detect_box(std::min(L.bx * L.c, L.W), std::min(L.by * L.c, L.H), &L.box_w, &L.box_h);
                L.image = img; L.level = l;
                L.band = match_band(l, jobs[p].scale, cfg.row_band_px);
                L.zeta = zeta_pow(jobs[p].scale, l);
                L.zeta_f = static_cast<float>(L.zeta);
                L.zeta_inv_f = static_cast<float>(1.0 / L.zeta);
                const size_t pitch = align_up((size_t)L.W, 128);
                // raw and blurred level, each padded so that whole-word and
                // halo reads past the last row stay inside the buffer
                L.blur_pitch = (int)pitch;
                L.pitch = (int)pitch;
                L.raw_w = ctx->levels.as<uint8_t>(lvl_off);
                L.raw = L.raw_w;
                lvl_off += align_up(pitch * L.H + kLevelSlack, 256);
                L.blur = ctx->levels.as<uint8_t>(lvl_off);
                lvl_off += align_up(pitch * L.H + kLevelSlack, 256);
                // taps
                uint32_t *tx = reinterpret_cast<uint32_t *>(host.data() + t_off);
                L.tapx = reinterpret_cast<const uint32_t *>(dplan + t_off);
                L.tapy = L.tapx + L.W;
                // source of the resampling: level 0 by zeta^n, or (cascaded)
                // the level above by one factor zeta
                const bool cascade = cfg.pyramid_mode == 1 && l > 0;
                const LevelDesc *up = cascade ? &levels[li - 1] : nullptr;
                L.src = up ? up->raw : nullptr;
                L.src_W = up ? up->W : g.W[0];
                L.src_H = up ? up->H : g.H[0];
                L.src_pitch = up ? up->pitch : 0;
                const double tap_s = cascade ? zeta_pow(jobs[p].scale, 1) : sc;
                for (int x = 0; x < L.W; ++x) tx[x] = bilinear_tap(x, tap_s, L.src_W);
                for (int y = 0; y < L.H; ++y) tx[L.W + y] = bilinear_tap(y, tap_s, L.src_H);
                t_off += align_up((size_t)(L.W + L.H) * 4, 16);
                uint16_t *px = reinterpret_cast<uint16_t *>(host.data() + t_off);
                L.projx = reinterpret_cast<const uint16_t *>(dplan + t_off);
                L.projy = L.projx + L.W;
                for (int x = 0; x < L.W; ++x) px[x] = project(x, sc, g.W[0]);
                for (int y = 0; y < L.H; ++y) px[L.W + y] = project(y, sc, g.H[0]);
                t_off += align_up((size_t)(L.W + L.H) * 2, 16);

                // TMA map of the raw level when every tile starts on a word
                // boundary (the box x is rounded down to 16 bytes)
                L.tmap = nullptr;
                PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
                if (encode && (L.bx * L.c) % 4 == 0) {
                    CUtensorMap map;  // encoded into an aligned object, then copied into the plan
                    const cuuint64_t dims[2] = { (cuuint64_t)L.W, (cuuint64_t)L.H };
                    const cuuint64_t strides[1] = { (cuuint64_t)L.pitch };
                    const cuuint32_t box[2] = { (cuuint32_t)L.box_w, (cuuint32_t)L.box_h };
                    const cuuint32_t estr[2] = { 1, 1 };
                    if (encode(&map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, L.raw_w, dims, strides, box, estr,
                               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS) {
                        std::memcpy(host.data() + o_tmaps + sizeof(CUtensorMap) * li, &map, sizeof(CUtensorMap));
                        L.tmap = reinterpret_cast<const CUtensorMap *>(dplan + o_tmaps) + li;
                    }
                }
                L.slot_base = slot;
                L.seg_base = seg;
                slot += L.cells_x * L.cells_y * k;
                for (int r = 0; r < L.cells_y; ++r) seg_level[seg + r] = li;
                seg += L.cells_y;
                pyr_base[li] = pyr;
                const int ptiles = ((L.W + kPyrTW - 1) / kPyrTW) * ((L.H + kPyrTH - 1) / kPyrTH);
                for (int q = 0; q < ptiles; ++q) ptile_level[pyr + q] = li;
                pyr += ptiles;
                fast_base[li] = fast;
                const int ftiles = ((L.cells_x + L.bx - 1) / L.bx) * ((L.cells_y + L.by - 1) / L.by);
                for (int q = 0; q < ftiles; ++q) ftile_level[fast + q] = li;
                fast += ftiles;
            }
            I.slot_count = slot - I.slot_base;
            I.seg_count = seg - I.seg_base;
        }
        PairDesc &P = pairs[p];
        P.left = 2 * p; P.right = 2 * p + 1;
        P.match_idx = reinterpret_cast<int32_t *>(rblock + pl.match_idx);
        P.disparity = reinterpret_cast<int16_t *>(rblock + pl.disparity);
        P.dist = reinterpret_cast<uint16_t *>(rblock + pl.dist);
        P.sub_disp = reinterpret_cast<float *>(rblock + pl.sub_disp);
        P.depth = reinterpret_cast<float *>(rblock + pl.depth);
        P.corr = reinterpret_cast<uint32_t *>(rblock + pl.corr);
    }
    pyr_base[n_levels] = pyr;
    fast_base[n_levels] = fast;
    seg_level[n_segs] = n_levels - 1;

    // detection tile records (the device-side tile geometry, evaluated here)
    auto trec = reinterpret_cast<TileRec *>(host.data() + o_trec);
    for (int l = 0; l < n_levels; ++l) {
        const LevelDesc &L = levels[l];
        const ImageDesc &I = images[L.image];
        const int ctas_x = (L.cells_x + L.bx - 1) / L.bx;
        for (int t = fast_base[l]; t < fast_base[l + 1]; ++t) {
            TileRec &R = trec[t];
            const int tt = t - fast_base[l], ty = tt / ctas_x;
            R.ccx0 = (tt - ty * ctas_x) * L.bx;
            R.ccy0 = ty * L.by;
            R.ncx = std::min(L.bx, L.cells_x - R.ccx0);
            R.ncy = std::min(L.by, L.cells_y - R.ccy0);
            R.x0 = R.ccx0 * L.c;
            R.y0 = R.ccy0 * L.c;
            R.tw = std::min(R.ncx * L.c, L.W - R.x0);
            R.th = std::min(R.ncy * L.c, L.H - R.y0);
            R.xs = L.tmap ? ((R.x0 - 4) & ~15) : R.x0 - 4;
            R.ys = R.y0 - 3;
            R.delta = R.x0 - 4 - R.xs;
            R.c = L.c; R.cells_x = L.cells_x; R.W = L.W; R.H = L.H; R.cinv = L.cinv;
            R.box_w = L.box_w; R.box_h = L.box_h; R.slot_base = L.slot_base; R.pitch = L.pitch;
            R.eps_hi = I.eps_hi; R.eps_lo = I.eps_lo; R.W0 = I.W0;
            R.skip_c0 = I.skip_c0; R.skip_cells_x = I.skip_cells_x;
            // projection ranges, widened to 16-byte boundaries (inside the
            // level's table, whose size is rounded up to 16 bytes)
            const uintptr_t ax = reinterpret_cast<uintptr_t>(L.projx + R.x0);
            const uintptr_t ay = reinterpret_cast<uintptr_t>(L.projy + R.y0);
            const uintptr_t bx0 = ax & ~(uintptr_t)15, by0 = ay & ~(uintptr_t)15;
            R.prj_src_x = reinterpret_cast<const uint16_t *>(bx0);
            R.prj_src_y = reinterpret_cast<const uint16_t *>(by0);
            R.prj_off_x = (int)(ax - bx0) / 2;
            R.prj_off_y = (int)(ay - by0) / 2;
            R.prj_bytes_x = (int)align_up((size_t)(ax - bx0) + 2 * (size_t)R.tw, 16);
            R.prj_bytes_y = (int)align_up((size_t)(ay - by0) + 2 * (size_t)R.th, 16);
            R.image = L.image;
            R.raw = L.raw; R.tmap = L.tmap; R.map = I.map; R.skip = I.skip;
        }
    }
    // Tile order 1: the persistent detection CTAs take records t, t + grid,
    // t + 2 grid, ...; ordered by decreasing work (evaluated rows x 32-pixel
    // chunks, the items of a threshold pass) the grid's last rounds hold the
    // smallest tiles.  Each record is self-contained (its tile's geometry,
    // slots and buffers), so the order changes no result; which order is
    // faster depends on the batch (the autotuner measures both).
    if (ctx->tune.tile_order == 1) {
        const int border = cfg.border;
        std::vector<std::pair<int, int>> work(fast);
        for (int t = 0; t < fast; ++t) {
            const TileRec &R = trec[t];
            const int rows = std::max(std::min(R.H - border - R.y0, R.th) - std::max(border - R.y0, 0), 0);
            work[t] = { -rows * ((R.tw + 31) >> 5), t };
        }
        std::stable_sort(work.begin(), work.end(),
                         [](const std::pair<int, int> &a, const std::pair<int, int> &b) { return a.first < b.first; });
        std::vector<TileRec> sorted(fast);
        for (int t = 0; t < fast; ++t) sorted[t] = trec[work[t].second];
        std::copy(sorted.begin(), sorted.end(), trec);
    }

    // pyramid tiles by level number (the cascaded pyramid launches level
    // number n once level n - 1 of every image is complete)
    int pass_first[kMaxLevels + 1] = {};
    {
        auto porder = reinterpret_cast<int32_t *>(host.data() + o_porder);
        int count[kMaxLevels] = {};
        for (int t = 0; t < pyr; ++t) ++count[levels[ptile_level[t]].level];
        for (int d = 0; d < kMaxLevels; ++d) pass_first[d + 1] = pass_first[d] + count[d];
        int fill[kMaxLevels];
        for (int d = 0; d < kMaxLevels; ++d) fill[d] = pass_first[d];
        for (int t = 0; t < pyr; ++t) porder[fill[levels[ptile_level[t]].level]++] = t;
    }
    e = cudaMemcpyAsync(ctx->plan.ptr, host.data(), off, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return fail(ctx, e);

    Batch &b = ctx->batch;
    b.images = reinterpret_cast<const ImageDesc *>(dplan + o_images);
    b.levels = reinterpret_cast<const LevelDesc *>(dplan + o_levels);
    b.pairs = reinterpret_cast<const PairDesc *>(dplan + o_pairs);
    b.pyr_tile_base = reinterpret_cast<const int32_t *>(dplan + o_pyr);
    b.pyr_tile_level = reinterpret_cast<const int32_t *>(dplan + o_ptl);
    b.pyr_order = reinterpret_cast<const int32_t *>(dplan + o_porder);
    b.pyr_pass = cfg.pyramid_mode == 1 ? 0 : -1;
    for (int d = 0; d <= kMaxLevels; ++d) b.pyr_pass_first[d] = pass_first[d];
    b.fast_tile_base = reinterpret_cast<const int32_t *>(dplan + o_fast);
    b.seg_level = reinterpret_cast<const int32_t *>(dplan + o_seg);
    b.fast_tile_level = reinterpret_cast<const int32_t *>(dplan + o_ftl);
    b.tile_rec = reinterpret_cast<const TileRec *>(dplan + o_trec);
    b.n_images = n_img; b.n_levels = n_levels; b.n_pairs = n; b.n_segments = n_segs;
    b.max_segment = 0;
    for (int l = 0; l < n_levels; ++l) b.max_segment = std::max(b.max_segment, levels[l].cells_x * k);
    b.pyr_tiles = pyr; b.fast_tiles = fast; b.max_capacity = max_cap;
    b.fast_max_box = max_box; b.fast_max_px = max_px; b.fast_max_cells = max_cells;
    b.fast_bits = ctx->prm.p_min == 9 && ctx->prm.p_max == 13;
    b.fast_max_planes = max_planes;
    b.fast_smem = fast_smem_bytes(max_box, max_px, max_cells, k, b.fast_bits ? max_planes : 0);
    b.corner_lut = ctx->d_lut;
    b.skip_max_tiles = skip_max_tiles;
    b.skip_any = ctx->skip_on ? ctx->skipbuf.as<int32_t>(skip_off) : nullptr;
    b.skip_max_cells = skip_max_cells;
    uint32_t *sw = ctx->scratch.as<uint32_t>();
    b.slots = sw;
    b.slot_k = sw + slot_words;
    b.slot_rank = reinterpret_cast<int32_t *>(sw + 2 * slot_words);
    b.canon = reinterpret_cast<int32_t *>(sw + 3 * slot_words);
    b.seg_count = reinterpret_cast<int32_t *>(sw + 4 * slot_words);
    b.seg_off = reinterpret_cast<int32_t *>(sw + 4 * slot_words + seg_words);
    b.pattern = ctx->d_pattern;
    b.pattern_off = ctx->d_pattern_off;
    b.bin_cos = ctx->d_cos;
    b.bin_sin = ctx->d_sin;
    b.bin_cosf = ctx->d_cosf;
    b.bin_sinf = ctx->d_sinf;
    b.err = reinterpret_cast<uint32_t *>(dcounts + 2 * cfg.max_pairs);
    b.prm = ctx->prm;

    ctx->keys = keys;
    ctx->plan_tune = ctx->tune;
    ctx->plan_skip = ctx->skip_on;
    ctx->layouts = layouts;
    ctx->result_off = result_off;
    ctx->slot_count = (size_t)n_slots;
    ctx->have_ablation = false;
    ctx->pair_scale.resize(n);
    for (int p = 0; p < n; ++p) ctx->pair_scale[p] = jobs[p].scale;
    ctx->h_images.assign(images, images + n_img);
    ctx->h_levels.assign(levels, levels + n_levels);
    return JSLAM_OK;
}

jslam_status enqueue_counts(jslam_ctx *ctx)
{
    const size_t bytes = sizeof(int32_t) * (2 * (size_t)ctx->cfg.max_pairs + 8);
    return fail(ctx, cudaMemcpyAsync(ctx->h_counts, ctx->counts.ptr, bytes, cudaMemcpyDeviceToHost, ctx->stream));
}

// Signature of one job (see JobKey).
JobKey job_key(const jslam_stereo_job &j)
{
    JobKey k;
    std::memset(&k, 0, sizeof(k));
    k.W = j.left.width; k.H = j.left.height; k.levels = j.levels;
    k.eps = j.fast_thresh; k.cell = j.cell; k.feats = j.max_feats;
    std::memcpy(&k.scale_bits, &j.scale, 4);
    k.mem[0] = j.left.memory;
    k.mem[1] = j.right.memory;
    return k;
}

// Release the captured graph, if any.
void drop_graph(jslam_ctx *ctx)
{
    if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    if (ctx->graph_src) cudaGraphDestroy(ctx->graph_src);
    ctx->graph = nullptr;
    ctx->graph_src = nullptr;
    ctx->graph_pyr.clear();
    ctx->graph_pyr_params.clear();
    ctx->graph_pyr_batch.clear();
    ctx->graph_keys.clear();
}

// Context state after a graph replay (extraction and matching; refinement is
// enqueued separately).
jslam_status graph_launched(jslam_ctx *ctx)
{
    ctx->have_extract = true;
    ctx->have_match = true;
    ctx->have_refine = false;
    ctx->synced = false;
    for (int i = 0; i < JSLAM_NUM_STAGES; ++i)
        ctx->stage_done[i] = i <= JSLAM_STAGE_MATCH && ctx->graph_timed && ctx->timing;
    return JSLAM_OK;
}

jslam_status use_device(jslam_ctx *ctx)
{
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return fail(ctx, cudaErrorInvalidDevice);
    if (cur != ctx->cfg.device) return fail(ctx, cudaSetDevice(ctx->cfg.device));
    return JSLAM_OK;
}

}  // namespace

extern "C" {

void jslam_default_config(jslam_config *cfg)
{
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->device = 0;
    cfg->cuda_stream = nullptr;
    cfg->max_width = 1920;
    cfg->max_height = 1080;
    cfg->max_levels = 8;
    cfg->max_feats = 4000;
    cfg->max_pairs = 64;
    cfg->fast_thresh_lo = 0;
    cfg->p_min = 9;
    cfg->p_max = 13;
    cfg->k_per_cell = 1;
    cfg->nms_q = 3;
    cfg->border = 19;
    cfg->max_disp = 128;
    cfg->row_band_px = 2;
    cfg->match_max_dist = 100;
    cfg->pfa_rule = 0;
    cfg->response_mode = 0;
    cfg->pyramid_mode = 0;
}

jslam_status jslam_create(jslam_ctx **out, const jslam_config *cfg)
{
    if (!out || !cfg) return JSLAM_ERR_ARG;
    *out = nullptr;
    const jslam_config &c = *cfg;
    if (c.max_width < 1 || c.max_width > 4096 || c.max_height < 1 || c.max_height > 4096) return JSLAM_ERR_ARG;
    if (c.max_levels < 1 || c.max_levels > kMaxLevels || c.max_feats < 1 || c.max_feats > (1 << 20)) return JSLAM_ERR_ARG;
    if (c.max_pairs < 1 || 2 * c.max_pairs > kMaxImages) return JSLAM_ERR_ARG;
    if (c.fast_thresh_lo > 254) return JSLAM_ERR_ARG;
    if (c.p_min < 1 || c.p_max > 16 || c.p_min > c.p_max) return JSLAM_ERR_ARG;
    if (c.k_per_cell < 1 || c.k_per_cell > 8) return JSLAM_ERR_ARG;
    if (c.nms_q < 1 || c.nms_q > 7 || (c.nms_q & 1) == 0) return JSLAM_ERR_ARG;
    if (c.border < 16 || c.border > 512) return JSLAM_ERR_ARG;
    if (c.max_disp < 0 || c.max_disp > 4096 || c.row_band_px < 0 || c.row_band_px > 64) return JSLAM_ERR_ARG;
    if (c.match_max_dist < 0 || c.pfa_rule < 0 || c.pfa_rule > 1) return JSLAM_ERR_ARG;
    if (c.response_mode < 0 || c.response_mode > 1 || c.pyramid_mode < 0 || c.pyramid_mode > 1) return JSLAM_ERR_ARG;

    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || c.device < 0 || c.device >= ndev) {
        cudaGetLastError();
        return JSLAM_ERR_CUDA;
    }
    jslam_ctx *ctx = new jslam_ctx();
    ctx->cfg = c;
    ctx->prm.p_min = c.p_min; ctx->prm.p_max = c.p_max; ctx->prm.k = c.k_per_cell;
    ctx->prm.nms_rad = (c.nms_q - 1) / 2; ctx->prm.border = c.border; ctx->prm.rule = c.pfa_rule;
    ctx->prm.resp_arc = c.response_mode;
    ctx->prm.max_disp = c.max_disp; ctx->prm.max_dist = c.match_max_dist;

    jslam_status st = JSLAM_OK;
    cudaError_t e = cudaSetDevice(c.device);
    if (e == cudaSuccess) {
        if (c.cuda_stream) {
            ctx->stream = static_cast<cudaStream_t>(c.cuda_stream);
        } else {
            e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
            ctx->own_stream = e == cudaSuccess;
        }
    }
    if (e == cudaSuccess) e = configure_kernels();
    if (e == cudaSuccess) e = configure_skipnet();
    int32_t w[7];
    blur_weights(w);
    if (e == cudaSuccess) e = set_blur_weights(w);
    const size_t pat_bytes = (size_t)kBins * kPairs * 4;
    const size_t lut_off = pat_bytes + 2 * kBins * sizeof(double);
    const size_t f_off = lut_off + kLutWords * sizeof(uint32_t);
    const size_t po_off = f_off + 2 * kBins * sizeof(float);
    const size_t const_bytes = po_off + (size_t)kBins * kPairs * sizeof(uint32_t);
    if (e == cudaSuccess) e = ctx->consts.ensure(const_bytes + 512, false, nullptr);
    if (e == cudaSuccess) {
        std::vector<char> h(const_bytes, 0);
        rotated_pattern(reinterpret_cast<int8_t *>(h.data()));
        double *cs = reinterpret_cast<double *>(h.data() + pat_bytes);
        sector_tables(cs, cs + kBins);
        corner_table(c.p_min, c.p_max, reinterpret_cast<uint32_t *>(h.data() + lut_off));
        float *cf = reinterpret_cast<float *>(h.data() + f_off);
        for (int i = 0; i < 2 * kBins; ++i) cf[i] = static_cast<float>(cs[i]);
        // the same pattern as offsets into the staged patch (row pitch kPatPitch)
        const int8_t *pt = reinterpret_cast<const int8_t *>(h.data());
        uint32_t *po = reinterpret_cast<uint32_t *>(h.data() + po_off);
        for (int i = 0; i < kBins * kPairs; ++i) {
            const int op = pt[4 * i + 1] * kPatPitch + pt[4 * i + 0];
            const int oq = pt[4 * i + 3] * kPatPitch + pt[4 * i + 2];
            po[i] = (uint32_t)(uint16_t)(int16_t)op | ((uint32_t)(uint16_t)(int16_t)oq << 16);
        }
        e = cudaMemcpy(ctx->consts.ptr, h.data(), h.size(), cudaMemcpyHostToDevice);
        ctx->d_pattern = ctx->consts.as<int8_t>();
        ctx->d_cos = ctx->consts.as<double>(pat_bytes);
        ctx->d_sin = ctx->d_cos + kBins;
        ctx->d_lut = ctx->consts.as<uint32_t>(lut_off);
        ctx->d_cosf = ctx->consts.as<float>(f_off);
        ctx->d_sinf = ctx->d_cosf + kBins;
        ctx->d_pattern_off = ctx->consts.as<uint32_t>(po_off);
    }
    if (e == cudaSuccess) e = ctx->counts.ensure(sizeof(int32_t) * (2 * (size_t)c.max_pairs + 8), true, nullptr);
    if (e == cudaSuccess) {
        e = cudaMallocHost(reinterpret_cast<void **>(&ctx->h_counts), sizeof(int32_t) * (2 * (size_t)c.max_pairs + 8));
        if (e == cudaSuccess) std::memset(ctx->h_counts, 0, sizeof(int32_t) * (2 * (size_t)c.max_pairs + 8));
        else ctx->h_counts = nullptr;
    }
    if (e != cudaSuccess) {
        st = (e == cudaErrorMemoryAllocation) ? JSLAM_ERR_NOMEM : JSLAM_ERR_CUDA;
        cudaGetLastError();
        jslam_destroy(ctx);
        return st;
    }
    *out = ctx;
    return JSLAM_OK;
}

jslam_status jslam_extract_batch(jslam_ctx *ctx, const jslam_stereo_job *jobs, int32_t n)
{
    if (!ctx || !jobs) return JSLAM_ERR_ARG;
    if (ctx->status != JSLAM_OK) return ctx->status;
    if (n < 1) return JSLAM_ERR_ARG;
    if (n > ctx->cfg.max_pairs) return JSLAM_ERR_CAPACITY;
    for (int p = 0; p < n; ++p) {
        const jslam_status s = check_job(ctx, jobs[p]);
        if (s != JSLAM_OK) return s;
    }
    jslam_status st = use_device(ctx);
    if (st != JSLAM_OK) return st;
    st = build_plan(ctx, jobs, n);
    if (st != JSLAM_OK) return st;

    // Level-0 inputs of this call; host images are copied into the staging
    // buffers on the context stream first.  Host images that lie back to
    // back in host memory (each starting where the previous one's pitch x
    // height ends) and whose pitch fits the staging slot go up in ONE copy
    // that keeps their pitch (a copy costs ~6 us of setup, and strided 2-D
    // copies run far below the link rate); other host images use one 2-D
    // copy each into a 128-aligned pitch.
    Batch &b = ctx->batch;
    const int n_img = 2 * n;
    auto image_of = [&](int img) -> const jslam_image & { return img & 1 ? jobs[img >> 1].right : jobs[img >> 1].left; };
    auto fits_slot = [](const jslam_image &im) { return (size_t)im.pitch <= align_up((size_t)im.width, 128); };
    for (int img = 0; img < n_img;) {
        const jslam_image &im = image_of(img);
        if (im.memory != JSLAM_MEM_HOST) {
            b.in.ptr[img] = im.data;
            b.in.pitch[img] = im.pitch;
            ++img;
            continue;
        }
        uint8_t *dst = ctx->staging.as<uint8_t>(ctx->staging_off[img]);
        if (!fits_slot(im)) {
            const int dpitch = (int)align_up((size_t)im.width, 128);
            cudaError_t e = cudaMemcpy2DAsync(dst, dpitch, im.data, im.pitch, im.width, im.height,
                                              cudaMemcpyHostToDevice, ctx->stream);
            if (e != cudaSuccess) return fail(ctx, e);
            b.in.ptr[img] = dst;
            b.in.pitch[img] = dpitch;
            ++img;
            continue;
        }
        int last = img;  // extend the run while the next image continues it in host memory
        while (last + 1 < n_img) {
            const jslam_image &cur = image_of(last), &nxt = image_of(last + 1);
            if (nxt.memory != JSLAM_MEM_HOST || !fits_slot(nxt) ||
                nxt.data != cur.data + (size_t)cur.pitch * (size_t)cur.height)
                break;
            ++last;
        }
        const jslam_image &lim = image_of(last);
        const size_t span = (size_t)(lim.data - im.data) + (size_t)lim.pitch * (size_t)(lim.height - 1) + lim.width;
        cudaError_t e = cudaMemcpyAsync(dst, im.data, span, cudaMemcpyHostToDevice, ctx->stream);
        if (e != cudaSuccess) return fail(ctx, e);
        for (int k = img; k <= last; ++k) {
            const jslam_image &ik = image_of(k);
            b.in.ptr[k] = dst + (ik.data - im.data);
            b.in.pitch[k] = ik.pitch;
        }
        img = last + 1;
    }
    cudaError_t e;
    b.nms_kernel = ctx->tune.nms_kernel;
    b.fast_ctas_per_sm = ctx->tune.detect_ctas_per_sm;
    for (bool &d : ctx->stage_done) d = false;
    if (ctx->timing && (e = cudaEventRecord(ctx->events[0], ctx->stream)) != cudaSuccess) return fail(ctx, e);
    for (int i = 0; i < JSLAM_STAGE_MATCH; ++i) {
        const NvtxRange range(kStageNames[i]);
        switch (i) {
        case JSLAM_STAGE_PYRAMID: e = launch_pyramid(b, ctx->stream); break;
        case JSLAM_STAGE_SKIP:
            e = ctx->skip_on ? launch_skipnet(b, ctx->skip_model, ctx->skip_thresh, ctx->stream) : cudaSuccess;
            break;
        case JSLAM_STAGE_DETECT: e = launch_fast_cull(b, ctx->stream); break;
        case JSLAM_STAGE_PFA_NMS: e = launch_pfa_nms(b, ctx->stream); break;
        case JSLAM_STAGE_PFA_FINAL: e = launch_pfa_finalize(b, ctx->stream); break;
        default: e = launch_orient_desc(b, ctx->stream); break;
        }
        if (e != cudaSuccess) return fail(ctx, e);
        if (ctx->timing) {
            if ((e = cudaEventRecord(ctx->events[i + 1], ctx->stream)) != cudaSuccess) return fail(ctx, e);
            ctx->stage_done[i] = true;
        }
    }
    ctx->have_extract = true;
    ctx->have_match = false;
    ctx->have_refine = false;
    ctx->synced = false;
    return enqueue_counts(ctx);
}

jslam_status jslam_extract(jslam_ctx *ctx, jslam_image left, jslam_image right, int32_t levels, float scale,
                           int32_t fast_thresh, int32_t cell, int32_t max_feats)
{
    jslam_stereo_job j;
    j.left = left; j.right = right; j.levels = levels; j.scale = scale;
    j.fast_thresh = fast_thresh; j.cell = cell; j.max_feats = max_feats;
    return jslam_extract_batch(ctx, &j, 1);
}

jslam_status jslam_match(jslam_ctx *ctx)
{
    if (!ctx) return JSLAM_ERR_ARG;
    if (ctx->status != JSLAM_OK) return ctx->status;
    if (!ctx->have_extract) return JSLAM_ERR_STATE;
    jslam_status st = use_device(ctx);
    if (st != JSLAM_OK) return st;
    cudaError_t e;
    {
        const NvtxRange range(kStageNames[JSLAM_STAGE_MATCH]);
        e = launch_match(ctx->batch, ctx->stream);
    }
    if (e != cudaSuccess) return fail(ctx, e);
    if (ctx->timing && ctx->stage_done[JSLAM_STAGE_ORB]) {
        if ((e = cudaEventRecord(ctx->events[JSLAM_STAGE_MATCH + 1], ctx->stream)) != cudaSuccess) return fail(ctx, e);
        ctx->stage_done[JSLAM_STAGE_MATCH] = true;
    }
    ctx->have_match = true;
    ctx->have_refine = false;
    return JSLAM_OK;
}

jslam_status jslam_refine_matches(jslam_ctx *ctx, int32_t half_window, int32_t search, float bf)
{
    if (!ctx) return JSLAM_ERR_ARG;
    if (ctx->status != JSLAM_OK) return ctx->status;
    if (half_window < 1 || half_window > kRefineMaxW || search < 1 || search > kRefineMaxL || !(bf >= 0.0f))
        return JSLAM_ERR_ARG;
    if (!ctx->have_match) return JSLAM_ERR_STATE;
    jslam_status st = use_device(ctx);
    if (st != JSLAM_OK) return st;
    cudaError_t e;
    {
        const NvtxRange range(kStageNames[JSLAM_STAGE_REFINE]);
        e = launch_refine(ctx->batch, half_window, search, (double)bf, ctx->stream);
    }
    if (e != cudaSuccess) return fail(ctx, e);
    if (ctx->timing && ctx->stage_done[JSLAM_STAGE_MATCH]) {
        if ((e = cudaEventRecord(ctx->events[JSLAM_STAGE_REFINE + 1], ctx->stream)) != cudaSuccess) return fail(ctx, e);
        ctx->stage_done[JSLAM_STAGE_REFINE] = true;
    }
    ctx->have_refine = true;
    return JSLAM_OK;
}

jslam_status jslam_track(jslam_ctx *ctx, int32_t pair, int32_t side, const float *u, const float *v,
                         const uint8_t *level, const uint32_t *desc, int32_t n, float radius, int32_t max_dist,
                         int32_t *out_idx, uint16_t *out_dist)
{
    if (!ctx) return JSLAM_ERR_ARG;
    if (ctx->status != JSLAM_OK) return ctx->status;
    if (n < 0 || side < 0 || side > 1 || !(radius >= 0.0f && radius < 1e6f) || max_dist < 0 || max_dist > 256)
        return JSLAM_ERR_ARG;
    if (n > 0 && (!u || !v || !level || !desc || !out_idx || !out_dist)) return JSLAM_ERR_ARG;
    if (!ctx->have_extract) return JSLAM_ERR_STATE;
    if (pair < 0 || pair >= (int)ctx->layouts.size()) return JSLAM_ERR_ARG;
    if (n == 0) return JSLAM_OK;
    jslam_status st = use_device(ctx);
    if (st != JSLAM_OK) return st;
    TrackArgs a;
    a.image = 2 * pair + side;
    a.n = n;
    a.max_dist = max_dist;
    a.radius = radius;
    for (int l = 0; l <= kMaxLevels; ++l) a.zeta_f[l] = static_cast<float>(zeta_pow(ctx->pair_scale[pair], l));
    a.u = u; a.v = v; a.level = level; a.desc = desc;
    a.out_idx = out_idx; a.out_dist = out_dist;
    const NvtxRange range("jslam track");
    return fail(ctx, launch_track(ctx->batch, a, ctx->stream));
}

jslam_status jslam_fc_ablation(jslam_ctx *ctx, int32_t n_max)
{
    if (!ctx) return JSLAM_ERR_ARG;
    if (ctx->status != JSLAM_OK) return ctx->status;
    if (!ctx->have_extract) return JSLAM_ERR_STATE;
    if (n_max < 1 || ctx->cfg.k_per_cell != 1) return JSLAM_ERR_ARG;
    const std::vector<LevelDesc> &lv = ctx->h_levels;
    int level_c[kMaxLevels] = {}, level_cy[kMaxLevels] = {}, level_bx[kMaxLevels] = {};
    int max_levels = 0, max_pixels = 0;
    ctx->abl_off.assign(lv.size(), 0);
    uint64_t total = 0;
    for (size_t i = 0; i < lv.size(); ++i) {
        const LevelDesc &L = lv[i];
        ctx->abl_off[i] = total;
        total += (uint64_t)L.W * (uint64_t)L.H;
        max_pixels = std::max(max_pixels, L.W * L.H);
        max_levels = std::max(max_levels, L.level + 1);
        level_c[L.level] = std::max(level_c[L.level], L.c);
        level_cy[L.level] = std::max(level_cy[L.level], L.cells_y);
        const int cpb = 128 / L.c;
        level_bx[L.level] = std::max(level_bx[L.level], (L.cells_x + cpb - 1) / cpb);
    }
    for (int l = 0; l < max_levels; ++l)
        if ((level_c[l] + n_max - 1) / n_max > 8) return JSLAM_ERR_ARG;  // 128 x N_t <= 1024 threads
    jslam_status st = use_device(ctx);
    if (st != JSLAM_OK) return st;
    const size_t off_bytes = align_up(lv.size() * sizeof(uint64_t), 256);
    const size_t key_bytes = align_up(ctx->slot_count * sizeof(uint32_t), 256);
    cudaError_t e = ctx->abl.ensure(off_bytes + key_bytes + total * sizeof(uint16_t) + 256, false, nullptr);
    if (e != cudaSuccess) return fail(ctx, e);
    for (cudaEvent_t &ev : ctx->abl_ev)
        if (!ev && (e = cudaEventCreate(&ev)) != cudaSuccess) return fail(ctx, e);
    uint64_t *d_off = ctx->abl.as<uint64_t>();
    uint32_t *d_keys = ctx->abl.as<uint32_t>(off_bytes);
    uint16_t *d_crf = ctx->abl.as<uint16_t>(off_bytes + key_bytes);
    // ctx->abl_off stays alive (and unchanged) until the next call, after this copy ran
    if ((e = cudaMemcpyAsync(d_off, ctx->abl_off.data(), lv.size() * sizeof(uint64_t), cudaMemcpyHostToDevice,
                             ctx->stream)) != cudaSuccess)
        return fail(ctx, e);
    if ((e = cudaEventRecord(ctx->abl_ev[0], ctx->stream)) != cudaSuccess) return fail(ctx, e);
    e = launch_fc_ablation(ctx->batch, d_crf, d_off, d_keys, level_bx, max_pixels, max_levels, level_cy, level_c,
                           n_max, ctx->stream, ctx->abl_ev[1]);
    if (e != cudaSuccess) return fail(ctx, e);
    if ((e = cudaEventRecord(ctx->abl_ev[2], ctx->stream)) != cudaSuccess) return fail(ctx, e);
    ctx->have_ablation = true;
    return JSLAM_OK;
}

jslam_status jslam_fc_ablation_view(jslam_ctx *ctx, int32_t pair, int32_t side, int32_t level,
                                    const uint32_t **ablation_keys, const uint32_t **fused_keys, int32_t *cells_x,
                                    int32_t *cells_y)
{
    if (!ctx || !ablation_keys || !fused_keys || !cells_x || !cells_y) return JSLAM_ERR_ARG;
    if (!ctx->have_ablation) return JSLAM_ERR_STATE;
    if (pair < 0 || pair >= (int)ctx->layouts.size() || side < 0 || side > 1) return JSLAM_ERR_ARG;
    const int img = 2 * pair + side;
    int base = -1, nl = 0;
    for (size_t i = 0; i < ctx->h_levels.size(); ++i)
        if (ctx->h_levels[i].image == img) { if (base < 0) base = (int)i; ++nl; }
    if (level < 0 || level >= nl) return JSLAM_ERR_ARG;
    const LevelDesc &L = ctx->h_levels[base + level];
    const size_t off_bytes = align_up(ctx->h_levels.size() * sizeof(uint64_t), 256);
    *ablation_keys = ctx->abl.as<uint32_t>(off_bytes) + L.slot_base;
    *fused_keys = ctx->batch.slots + L.slot_base;
    *cells_x = L.cells_x;
    *cells_y = L.cells_y;
    return JSLAM_OK;
}

jslam_status jslam_selftest_wait(jslam_ctx *ctx)
{
    if (!ctx) return JSLAM_ERR_ARG;
    if (ctx->status != JSLAM_OK) return ctx->status;
    jslam_status st = use_device(ctx);
    if (st != JSLAM_OK) return st;
    uint32_t *err = reinterpret_cast<uint32_t *>(ctx->counts.as<int32_t>() + 2 * (size_t)ctx->cfg.max_pairs);
    cudaError_t e = launch_wait_selftest(err, ctx->stream);
    if (e != cudaSuccess) return fail(ctx, e);
    return enqueue_counts(ctx);
}

jslam_status jslam_crf_view(jslam_ctx *ctx, int32_t pair, int32_t side, int32_t level, const uint16_t **crf,
                            int32_t *width, int32_t *height)
{
    if (!ctx || !crf || !width || !height) return JSLAM_ERR_ARG;
    if (!ctx->have_ablation) return JSLAM_ERR_STATE;
    if (pair < 0 || pair >= (int)ctx->layouts.size() || side < 0 || side > 1) return JSLAM_ERR_ARG;
    const int img = 2 * pair + side;
    int base = -1, nl = 0;
    for (size_t i = 0; i < ctx->h_levels.size(); ++i)
        if (ctx->h_levels[i].image == img) { if (base < 0) base = (int)i; ++nl; }
    if (level < 0 || level >= nl) return JSLAM_ERR_ARG;
    const LevelDesc &L = ctx->h_levels[base + level];
    const size_t off_bytes = align_up(ctx->h_levels.size() * sizeof(uint64_t), 256);
    const size_t key_bytes = align_up(ctx->slot_count * sizeof(uint32_t), 256);
    *crf = ctx->abl.as<uint16_t>(off_bytes + key_bytes) + ctx->abl_off[base + level];
    *width = L.W;
    *height = L.H;
    return JSLAM_OK;
}

jslam_status jslam_fc_ablation_times(jslam_ctx *ctx, float *crf_ms, float *fc_ms)
{
    if (!ctx || !crf_ms || !fc_ms) return JSLAM_ERR_ARG;
    if (!ctx->have_ablation) return JSLAM_ERR_STATE;
    cudaError_t e = cudaEventElapsedTime(crf_ms, ctx->abl_ev[0], ctx->abl_ev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(fc_ms, ctx->abl_ev[1], ctx->abl_ev[2]);
    return fail(ctx, e);
}

// Keypoint count of `side` in a downloaded result block (its header).
static int32_t block_count(const void *block, int side)
{
    int32_t c;
    std::memcpy(&c, static_cast<const char *>(block) + 4 * side, 4);
    return c;
}

static void refined_views(const PairLayout &pl, const char *b, int32_t count, jslam_refined *out)
{
    out->count = count;
    out->disparity = reinterpret_cast<const float *>(b + pl.sub_disp);
    out->depth = reinterpret_cast<const float *>(b + pl.depth);
    out->sad = reinterpret_cast<const uint32_t *>(b + pl.corr);
}

jslam_status jslam_sync(jslam_ctx *ctx)
{
    if (!ctx) return JSLAM_ERR_ARG;
    if (ctx->status != JSLAM_OK) return ctx->status;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return fail(ctx, e);
    ctx->synced = true;
    const uint32_t err = static_cast<uint32_t>(ctx->h_counts[2 * ctx->cfg.max_pairs]);
    if (err & kErrTimeout) ctx->status = JSLAM_ERR_TIMEOUT;
    else if (err) ctx->status = JSLAM_ERR_CAPACITY;
    return ctx->status;
}

static int32_t synced_count(const jslam_ctx *ctx, int img)
{
    return ctx->synced ? ctx->h_counts[img] : -1;
}

jslam_status jslam_get_keypoints(jslam_ctx *ctx, int32_t pair, int32_t side, jslam_keypoints *out)
{
    if (!ctx || !out) return JSLAM_ERR_ARG;
    if (!ctx->have_extract) return JSLAM_ERR_STATE;
    if (pair < 0 || pair >= (int)ctx->layouts.size() || side < 0 || side > 1) return JSLAM_ERR_ARG;
    const KpOut &o = ctx->h_images[2 * pair + side].out;
    out->count = synced_count(ctx, 2 * pair + side);
    out->capacity = o.capacity;
    out->x = o.x; out->y = o.y; out->X = o.X; out->Y = o.Y;
    out->level = o.level; out->angle_bin = o.angle_bin; out->response = o.response;
    out->k_levels = o.k_levels; out->k_resp = o.k_resp; out->angle = o.angle; out->desc = o.desc;
    return JSLAM_OK;
}

jslam_status jslam_get_matches(jslam_ctx *ctx, int32_t pair, jslam_matches *out)
{
    if (!ctx || !out) return JSLAM_ERR_ARG;
    if (!ctx->have_match) return JSLAM_ERR_STATE;
    if (pair < 0 || pair >= (int)ctx->layouts.size()) return JSLAM_ERR_ARG;
    const PairLayout &pl = ctx->layouts[pair];
    char *rb = ctx->results.as<char>(ctx->result_off[pair]);
    out->count = synced_count(ctx, 2 * pair);
    out->right_idx = reinterpret_cast<const int32_t *>(rb + pl.match_idx);
    out->disparity = reinterpret_cast<const int16_t *>(rb + pl.disparity);
    out->dist = reinterpret_cast<const uint16_t *>(rb + pl.dist);
    return JSLAM_OK;
}

jslam_status jslam_get_refined(jslam_ctx *ctx, int32_t pair, jslam_refined *out)
{
    if (!ctx || !out) return JSLAM_ERR_ARG;
    if (!ctx->have_refine) return JSLAM_ERR_STATE;
    if (pair < 0 || pair >= (int)ctx->layouts.size()) return JSLAM_ERR_ARG;
    refined_views(ctx->layouts[pair], ctx->results.as<char>(ctx->result_off[pair]), synced_count(ctx, 2 * pair), out);
    return JSLAM_OK;
}

jslam_status jslam_result_refined_view(jslam_ctx *ctx, int32_t pair, const void *block, jslam_refined *out)
{
    if (!ctx || !block || !out) return JSLAM_ERR_ARG;
    if (!ctx->have_refine) return JSLAM_ERR_STATE;
    if (pair < 0 || pair >= (int)ctx->layouts.size()) return JSLAM_ERR_ARG;
    refined_views(ctx->layouts[pair], static_cast<const char *>(block), block_count(block, 0), out);
    return JSLAM_OK;
}

jslam_status jslam_get_level(jslam_ctx *ctx, int32_t pair, int32_t side, int32_t level, jslam_level_view *out)
{
    if (!ctx || !out) return JSLAM_ERR_ARG;
    if (!ctx->have_extract) return JSLAM_ERR_STATE;
    if (pair < 0 || pair >= (int)ctx->layouts.size() || side < 0 || side > 1) return JSLAM_ERR_ARG;
    const ImageDesc &I = ctx->h_images[2 * pair + side];
    if (level < 0 || level >= I.levels) return JSLAM_ERR_ARG;
    const LevelDesc &L = ctx->h_levels[I.level_base + level];
    out->width = L.W; out->height = L.H; out->blurred_pitch = L.blur_pitch; out->blurred = L.blur;
    out->raw_pitch = L.pitch;
    out->raw = L.raw;
    return JSLAM_OK;
}

jslam_status jslam_result_bytes(jslam_ctx *ctx, int32_t pair, size_t *bytes)
{
    if (!ctx || !bytes) return JSLAM_ERR_ARG;
    if (!ctx->have_extract) return JSLAM_ERR_STATE;
    if (pair < 0 || pair >= (int)ctx->layouts.size()) return JSLAM_ERR_ARG;
    *bytes = ctx->layouts[pair].bytes;
    return JSLAM_OK;
}

jslam_status jslam_download(jslam_ctx *ctx, int32_t pair, void *dst, size_t bytes)
{
    if (!ctx || !dst) return JSLAM_ERR_ARG;
    if (ctx->status != JSLAM_OK) return ctx->status;
    if (!ctx->have_extract) return JSLAM_ERR_STATE;
    if (pair < 0 || pair >= (int)ctx->layouts.size()) return JSLAM_ERR_ARG;
    if (bytes < ctx->layouts[pair].bytes) return JSLAM_ERR_ARG;
    jslam_status st = use_device(ctx);
    if (st != JSLAM_OK) return st;
    return fail(ctx, cudaMemcpyAsync(dst, ctx->results.as<char>(ctx->result_off[pair]), ctx->layouts[pair].bytes,
                                     cudaMemcpyDeviceToHost, ctx->stream));
}

jslam_status jslam_result_range(jslam_ctx *ctx, int32_t first, int32_t count, size_t *bytes, size_t *offsets)
{
    if (!ctx || !bytes) return JSLAM_ERR_ARG;
    if (!ctx->have_extract) return JSLAM_ERR_STATE;
    if (first < 0 || count < 1 || first + count > (int)ctx->layouts.size()) return JSLAM_ERR_ARG;
    const size_t base = ctx->result_off[first];
    const int end = first + count - 1;
    *bytes = ctx->result_off[end] + ctx->layouts[end].bytes - base;
    if (offsets)
        for (int i = 0; i < count; ++i) offsets[i] = ctx->result_off[first + i] - base;
    return JSLAM_OK;
}

jslam_status jslam_download_range(jslam_ctx *ctx, int32_t first, int32_t count, void *dst, size_t bytes)
{
    if (!ctx || !dst) return JSLAM_ERR_ARG;
    if (ctx->status != JSLAM_OK) return ctx->status;
    size_t need = 0;
    jslam_status st = jslam_result_range(ctx, first, count, &need, nullptr);
    if (st != JSLAM_OK) return st;
    if (bytes < need) return JSLAM_ERR_ARG;
    st = use_device(ctx);
    if (st != JSLAM_OK) return st;
    return fail(ctx, cudaMemcpyAsync(dst, ctx->results.as<char>(ctx->result_off[first]), need, cudaMemcpyDeviceToHost,
                                     ctx->stream));
}

jslam_status jslam_result_view(jslam_ctx *ctx, int32_t pair, const void *block, int32_t side, jslam_keypoints *kp,
                               jslam_matches *m)
{
    if (!ctx || !block || !kp) return JSLAM_ERR_ARG;
    if (!ctx->have_extract) return JSLAM_ERR_STATE;
    if (pair < 0 || pair >= (int)ctx->layouts.size() || side < 0 || side > 1) return JSLAM_ERR_ARG;
    const PairLayout &pl = ctx->layouts[pair];
    const SideLayout &s = pl.side[side];
    const char *b = static_cast<const char *>(block);
    kp->count = block_count(block, side);
    kp->capacity = pl.capacity;
    kp->desc = reinterpret_cast<const uint32_t *>(b + s.desc);
    kp->k_resp = reinterpret_cast<const uint32_t *>(b + s.k_resp);
    kp->angle = reinterpret_cast<const float *>(b + s.angle);
    kp->x = reinterpret_cast<const uint16_t *>(b + s.x);
    kp->y = reinterpret_cast<const uint16_t *>(b + s.y);
    kp->X = reinterpret_cast<const uint16_t *>(b + s.X);
    kp->Y = reinterpret_cast<const uint16_t *>(b + s.Y);
    kp->response = reinterpret_cast<const uint16_t *>(b + s.response);
    kp->level = reinterpret_cast<const uint8_t *>(b + s.level);
    kp->angle_bin = reinterpret_cast<const uint8_t *>(b + s.angle_bin);
    kp->k_levels = reinterpret_cast<const uint8_t *>(b + s.k_levels);
    if (m) {
        m->count = side == 0 && ctx->have_match ? kp->count : -1;
        m->right_idx = reinterpret_cast<const int32_t *>(b + pl.match_idx);
        m->disparity = reinterpret_cast<const int16_t *>(b + pl.disparity);
        m->dist = reinterpret_cast<const uint16_t *>(b + pl.dist);
    }
    return JSLAM_OK;
}

jslam_status jslam_enable_stage_timing(jslam_ctx *ctx, int32_t enable)
{
    if (!ctx) return JSLAM_ERR_ARG;
    if (ctx->status != JSLAM_OK) return ctx->status;
    if (enable && !ctx->events[0]) {
        jslam_status st = use_device(ctx);
        if (st != JSLAM_OK) return st;
        for (cudaEvent_t &ev : ctx->events) {
            cudaError_t e = cudaEventCreate(&ev);
            if (e != cudaSuccess) return fail(ctx, e);
        }
    }
    ctx->timing = enable != 0;
    for (bool &d : ctx->stage_done) d = false;
    return JSLAM_OK;
}

jslam_status jslam_stage_times(jslam_ctx *ctx, float *ms)
{
    if (!ctx || !ms) return JSLAM_ERR_ARG;
    if (ctx->status != JSLAM_OK) return ctx->status;
    if (!ctx->timing || !ctx->stage_done[0]) return JSLAM_ERR_STATE;
    for (int i = 0; i < JSLAM_NUM_STAGES; ++i) {
        ms[i] = 0.0f;
        if (!ctx->stage_done[i]) continue;
        // the match stage follows the ORB stage's event
        cudaError_t e = cudaEventElapsedTime(&ms[i], ctx->events[i], ctx->events[i + 1]);
        if (e != cudaSuccess) return fail(ctx, e);
    }
    return JSLAM_OK;
}

jslam_status jslam_set_skip_model(jslam_ctx *ctx, const void *blob, size_t bytes, float thresh)
{
    if (!ctx) return JSLAM_ERR_ARG;
    if (ctx->status != JSLAM_OK) return ctx->status;
    if (!blob) {
        ctx->skip_on = false;
        return JSLAM_OK;
    }
    constexpr size_t kHeader = 16, kBias = (2 * kSkipC + 1) * sizeof(float);
    constexpr size_t kW1 = kSkipC * 9, kW2 = kSkipC * kSkipC * 9, kW3 = kSkipC * 9;
    constexpr size_t kBytes = kHeader + kBias + 2 * (kW1 + kW2 + kW3);
    const uint8_t *p = static_cast<const uint8_t *>(blob);
    uint32_t hdr[3];
    if (bytes != kBytes || std::memcmp(p, "JSKP", 4) != 0) return JSLAM_ERR_ARG;
    std::memcpy(hdr, p + 4, sizeof(hdr));
    if (hdr[0] != 1 || hdr[1] != (uint32_t)kSkipC || hdr[2] != 8) return JSLAM_ERR_ARG;
    if (!(thresh == thresh)) return JSLAM_ERR_ARG;  // NaN
    jslam_status st = use_device(ctx);
    if (st != JSLAM_OK) return st;
    cudaError_t e = ctx->skipw.ensure(kBytes + 256, false, nullptr);
    if (e != cudaSuccess) return fail(ctx, e);
    // device layout: biases (FP32) first, then the BF16 weights
    e = cudaMemcpy(ctx->skipw.ptr, p + kHeader, kBytes - kHeader, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(ctx, e);
    float b3 = 0.0f;
    std::memcpy(&b3, p + kHeader + 2 * kSkipC * sizeof(float), sizeof(float));
    SkipModelDev &m = ctx->skip_model;
    m.b1 = ctx->skipw.as<float>(0);
    m.b2 = ctx->skipw.as<float>(kSkipC * sizeof(float));
    m.b3 = b3;
    m.w1 = ctx->skipw.as<uint16_t>(kBias);
    m.w2 = m.w1 + kW1;
    m.w3 = m.w2 + kW2;
    ctx->skip_thresh = thresh;
    ctx->skip_on = true;
    return JSLAM_OK;
}

jslam_status jslam_get_skip_view(jslam_ctx *ctx, int32_t pair, int32_t side, jslam_skip_view *out)
{
    if (!ctx || !out) return JSLAM_ERR_ARG;
    if (!ctx->have_extract || !ctx->plan_skip) return JSLAM_ERR_STATE;
    if (pair < 0 || pair >= (int)ctx->layouts.size() || side < 0 || side > 1) return JSLAM_ERR_ARG;
    const ImageDesc &I = ctx->h_images[2 * pair + side];
    out->w8 = I.skip_w8; out->h8 = I.skip_h8;
    out->cells_x = I.skip_cells_x; out->cells_y = I.skip_cells_y;
    out->logits = I.skip_logits; out->skip = I.skip;
    return JSLAM_OK;
}

jslam_status jslam_set_tuning(jslam_ctx *ctx, const jslam_tuning *t)
{
    if (!ctx || !t) return JSLAM_ERR_ARG;
    if (t->tile_w_px < 32 || t->tile_w_px > kFastMaxTile || t->tile_w_px % 4 != 0) return JSLAM_ERR_ARG;
    if (t->tile_h_px < 8 || t->tile_h_px > kFastMaxTile) return JSLAM_ERR_ARG;
    if (t->nms_kernel < 0 || t->nms_kernel > 1 || t->detect_ctas_per_sm < 0 || t->detect_ctas_per_sm > 8)
        return JSLAM_ERR_ARG;
    if (t->tile_order < 0 || t->tile_order > 1) return JSLAM_ERR_ARG;
    ctx->tune = *t;
    return JSLAM_OK;
}

namespace {

// Median-free minimum of a stage's time over `reps` runs of the batch (the
// first run of a new tuning also rebuilds the plan and is not counted).
jslam_status time_stage(jslam_ctx *ctx, const jslam_stereo_job *jobs, int32_t n, int stage, int reps, float *best)
{
    *best = -1.0f;
    for (int rep = 0; rep <= reps; ++rep) {
        jslam_status st = jslam_extract_batch(ctx, jobs, n);
        if (st == JSLAM_OK) st = jslam_sync(ctx);
        float ms[JSLAM_NUM_STAGES];
        if (st == JSLAM_OK) st = jslam_stage_times(ctx, ms);
        if (st != JSLAM_OK) return st;
        if (rep > 0 && (*best < 0 || ms[stage] < *best)) *best = ms[stage];
    }
    return JSLAM_OK;
}

}  // namespace

jslam_status jslam_autotune(jslam_ctx *ctx, const jslam_stereo_job *jobs, int32_t n, jslam_tuning *out)
{
    if (!ctx || !jobs) return JSLAM_ERR_ARG;
    if (ctx->status != JSLAM_OK) return ctx->status;
    static const int tiles[][2] = { { 128, 64 }, { 128, 32 }, { 128, 128 }, { 64, 64 }, { 64, 128 } };
    const bool was_timing = ctx->timing;
    jslam_status st = jslam_enable_stage_timing(ctx, 1);
    if (st != JSLAM_OK) return st;
    jslam_tuning best = ctx->tune;
    best.nms_kernel = 0;
    best.detect_ctas_per_sm = 0;
    best.tile_order = 0;
    // 1. the detection tile
    float best_ms = -1.0f;
    for (const auto &tl : tiles) {
        ctx->tune = best;
        ctx->tune.tile_w_px = tl[0];
        ctx->tune.tile_h_px = tl[1];
        float ms;
        if ((st = time_stage(ctx, jobs, n, JSLAM_STAGE_DETECT, 3, &ms)) != JSLAM_OK) break;
        if (best_ms < 0 || ms < best_ms) {
            best_ms = ms;
            best.tile_w_px = tl[0];
            best.tile_h_px = tl[1];
        }
    }
    // 2. fewer persistent detection CTAs per SM than fit (one less, then two)
    int fit = 0;
    if (st == JSLAM_OK) {
        ctx->tune = best;
        if ((st = jslam_extract_batch(ctx, jobs, n)) == JSLAM_OK) st = jslam_sync(ctx);
        if (st == JSLAM_OK) {
            const cudaError_t e = detect_ctas_that_fit(ctx->batch, &fit);
            if (e != cudaSuccess) st = fail(ctx, e);
        }
    }
    for (int c = fit - 1; st == JSLAM_OK && c >= 1 && c >= fit - 2; --c) {
        ctx->tune = best;
        ctx->tune.detect_ctas_per_sm = c;
        float ms;
        if ((st = time_stage(ctx, jobs, n, JSLAM_STAGE_DETECT, 3, &ms)) != JSLAM_OK) break;
        if (ms < best_ms) { best_ms = ms; best.detect_ctas_per_sm = c; }
    }
    // 3. the NMS kernel, where the warp-per-segment variant applies
    if (st == JSLAM_OK && ctx->batch.max_segment <= 96) {
        float nms_ms[2] = { -1.0f, -1.0f };
        for (int v = 0; v < 2 && st == JSLAM_OK; ++v) {
            ctx->tune = best;
            ctx->tune.nms_kernel = v;
            st = time_stage(ctx, jobs, n, JSLAM_STAGE_PFA_NMS, 3, &nms_ms[v]);
        }
        if (st == JSLAM_OK) best.nms_kernel = nms_ms[1] < nms_ms[0] ? 1 : 0;
    }
    // 4. the tile order (a replan each), against the detection time of the
    // pick so far
    if (st == JSLAM_OK) {
        ctx->tune = best;
        ctx->tune.tile_order = 1;
        float ms;
        if ((st = time_stage(ctx, jobs, n, JSLAM_STAGE_DETECT, 3, &ms)) == JSLAM_OK && ms < best_ms) {
            best_ms = ms;
            best.tile_order = 1;
        }
    }
    ctx->tune = best;
    ctx->tune_ms = best_ms;
    if (st == JSLAM_OK) st = jslam_enable_stage_timing(ctx, was_timing ? 1 : 0);
    if (st == JSLAM_OK && out) *out = best;
    return st;
}

jslam_status jslam_autotune_cached(jslam_ctx *ctx, const jslam_stereo_job *jobs, int32_t n, const char *cache_path,
                                   jslam_tuning *out, int32_t *hit)
{
    if (!ctx || !jobs || !cache_path || n < 1) return JSLAM_ERR_ARG;
    if (ctx->status != JSLAM_OK) return ctx->status;
    if (hit) *hit = 0;
    jslam_status st = use_device(ctx);
    if (st != JSLAM_OK) return st;
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, ctx->cfg.device);
    if (e != cudaSuccess) return fail(ctx, e);
    std::vector<char> key(256 + 96 * (size_t)n);
    st = jslam_tune_key(prop.name, prop.multiProcessorCount, &ctx->cfg, jobs, n, key.data(), key.size());
    if (st != JSLAM_OK) return st;
    jslam_tuning t{};
    int32_t found = 0;
    if ((st = jslam_tune_cache_get(cache_path, key.data(), &t, &found)) != JSLAM_OK) return st;
    if (found) {
        if ((st = jslam_set_tuning(ctx, &t)) != JSLAM_OK) return st;
        if (hit) *hit = 1;
        if (out) *out = t;
        return JSLAM_OK;
    }
    if ((st = jslam_autotune(ctx, jobs, n, &t)) != JSLAM_OK) return st;
    if ((st = jslam_tune_cache_put(cache_path, key.data(), &t, ctx->tune_ms)) != JSLAM_OK) return st;
    if (out) *out = t;
    return JSLAM_OK;
}

jslam_status jslam_graph_capture(jslam_ctx *ctx, const jslam_stereo_job *jobs, int32_t n)
{
    if (!ctx || !jobs) return JSLAM_ERR_ARG;
    if (ctx->status != JSLAM_OK) return ctx->status;
    if (ctx->stream == nullptr || ctx->stream == cudaStreamLegacy) return JSLAM_ERR_STATE;
    jslam_status st = jslam_extract_batch(ctx, jobs, n);  // plan, buffers, tables
    if (st == JSLAM_OK) st = jslam_match(ctx);
    if (st == JSLAM_OK) st = jslam_sync(ctx);
    if (st != JSLAM_OK) return st;
    drop_graph(ctx);
    cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return fail(ctx, e);
    jslam_status cap = jslam_extract_batch(ctx, jobs, n);
    if (cap == JSLAM_OK) cap = jslam_match(ctx);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(ctx->stream, &graph);
    if (cap != JSLAM_OK) { if (graph) cudaGraphDestroy(graph); return cap; }
    if (e != cudaSuccess) return fail(ctx, e);
    // the pyramid launch is the one node that reads the input images: keep
    // its handle (and the graph it belongs to) so that replays can point it
    // at new frames
    size_t n_nodes = 0;
    e = cudaGraphGetNodes(graph, nullptr, &n_nodes);
    std::vector<cudaGraphNode_t> nodes(n_nodes);
    if (e == cudaSuccess && n_nodes) e = cudaGraphGetNodes(graph, nodes.data(), &n_nodes);
    for (size_t i = 0; e == cudaSuccess && i < n_nodes; ++i) {
        cudaGraphNodeType type;
        if ((e = cudaGraphNodeGetType(nodes[i], &type)) != cudaSuccess || type != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams kp{};
        if ((e = cudaGraphKernelNodeGetParams(nodes[i], &kp)) != cudaSuccess) break;
        if (kp.func == pyramid_kernel()) {
            if (!kp.kernelParams || !kp.kernelParams[0]) { e = cudaErrorInvalidValue; break; }
            ctx->graph_pyr.push_back(nodes[i]);
            ctx->graph_pyr_params.push_back(kp);
            ctx->graph_pyr_batch.push_back(*static_cast<const Batch *>(kp.kernelParams[0]));
        }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ctx->graph, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        ctx->graph = nullptr;
        ctx->graph_pyr.clear();
        ctx->graph_pyr_params.clear();
        ctx->graph_pyr_batch.clear();
        return fail(ctx, e);
    }
    ctx->graph_src = graph;
    ctx->graph_keys = ctx->keys;
    ctx->graph_gen = ctx->plan_gen;
    ctx->graph_pairs = n;
    ctx->graph_timed = ctx->timing;
    return JSLAM_OK;
}

jslam_status jslam_graph_launch(jslam_ctx *ctx)
{
    if (!ctx) return JSLAM_ERR_ARG;
    if (ctx->status != JSLAM_OK) return ctx->status;
    if (!ctx->graph || ctx->graph_gen != ctx->plan_gen) return JSLAM_ERR_STATE;
    jslam_status st = use_device(ctx);
    if (st != JSLAM_OK) return st;
    cudaError_t e = cudaGraphLaunch(ctx->graph, ctx->stream);
    if (e != cudaSuccess) return fail(ctx, e);
    return graph_launched(ctx);
}

jslam_status jslam_graph_launch_jobs(jslam_ctx *ctx, const jslam_stereo_job *jobs, int32_t n)
{
    if (!ctx || !jobs) return JSLAM_ERR_ARG;
    if (ctx->status != JSLAM_OK) return ctx->status;
    if (!ctx->graph || ctx->graph_gen != ctx->plan_gen) return JSLAM_ERR_STATE;
    if (n != ctx->graph_pairs || ctx->graph_pyr.empty()) return JSLAM_ERR_ARG;
    for (int p = 0; p < n; ++p) {
        const jslam_status s = check_job(ctx, jobs[p]);
        if (s != JSLAM_OK) return s;
        if (jobs[p].left.memory != JSLAM_MEM_DEVICE || jobs[p].right.memory != JSLAM_MEM_DEVICE)
            return JSLAM_ERR_ARG;
        if (!(job_key(jobs[p]) == ctx->graph_keys[p])) return JSLAM_ERR_ARG;
    }
    jslam_status st = use_device(ctx);
    if (st != JSLAM_OK) return st;
    // each pyramid launch as captured, with this call's frames; the nodes
    // keep copies of their parameters, so `b` may go out of scope after
    Inputs in = ctx->batch.in;
    for (int img = 0; img < 2 * n; ++img) {
        const jslam_image &im = img & 1 ? jobs[img >> 1].right : jobs[img >> 1].left;
        in.ptr[img] = im.data;
        in.pitch[img] = im.pitch;
    }
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; i < ctx->graph_pyr.size() && e == cudaSuccess; ++i) {
        Batch b = ctx->graph_pyr_batch[i];
        b.in = in;
        void *args[] = { &b };
        cudaKernelNodeParams kp = ctx->graph_pyr_params[i];
        kp.kernelParams = args;
        kp.extra = nullptr;
        e = cudaGraphExecKernelNodeSetParams(ctx->graph, ctx->graph_pyr[i], &kp);
    }
    if (e == cudaSuccess) e = cudaGraphLaunch(ctx->graph, ctx->stream);
    if (e != cudaSuccess) return fail(ctx, e);
    ctx->batch.in = in;
    return graph_launched(ctx);
}

void jslam_destroy(jslam_ctx *ctx)
{
    if (!ctx) return;
    int cur = -1;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != ctx->cfg.device) cudaSetDevice(ctx->cfg.device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    ctx->consts.release();
    ctx->plan.release();
    ctx->levels.release();
    ctx->maps.release();
    ctx->scratch.release();
    ctx->results.release();
    ctx->staging.release();
    ctx->counts.release();
    ctx->skipw.release();
    ctx->skipbuf.release();
    ctx->abl.release();
    if (ctx->h_counts) cudaFreeHost(ctx->h_counts);
    for (cudaEvent_t ev : ctx->events)
        if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t ev : ctx->abl_ev)
        if (ev) cudaEventDestroy(ev);
    drop_graph(ctx);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    cudaGetLastError();
    delete ctx;
}

const char *jslam_status_str(jslam_status s)
{
    switch (s) {
    case JSLAM_OK: return "ok";
    case JSLAM_ERR_ARG: return "invalid argument";
    case JSLAM_ERR_CUDA: return "CUDA error";
    case JSLAM_ERR_NOMEM: return "out of memory";
    case JSLAM_ERR_CAPACITY: return "capacity exceeded";
    case JSLAM_ERR_TIMEOUT: return "device wait timed out";
    case JSLAM_ERR_STATE: return "call out of order";
    }
    return "unknown status";
}

void jslam_pattern_table(int8_t *out)
{
    if (out) rotated_pattern(out);
}

jslam_status jslam_level_geometry(int32_t width, int32_t height, int32_t levels, float scale, int32_t cell,
                                  int32_t *w, int32_t *h, int32_t *c)
{
    if (!w || !h || !c || levels < 1 || levels > kMaxLevels || !(scale > 1.0f) || cell < 1) return JSLAM_ERR_ARG;
    const Geometry g = level_geometry(width, height, levels, scale, cell);
    for (int n = 0; n < levels; ++n) { w[n] = g.W[n]; h[n] = g.H[n]; c[n] = g.c[n]; }
    return JSLAM_OK;
}

int32_t jslam_project(int32_t v, int32_t level, float scale, int32_t extent)
{
    return project(v, zeta_pow(scale, level), extent);
}

jslam_status jslam_corner_table(int32_t p_min, int32_t p_max, uint32_t *out)
{
    if (!out || p_min < 1 || p_max > 16 || p_min > p_max) return JSLAM_ERR_ARG;
    corner_table(p_min, p_max, out);
    return JSLAM_OK;
}

int32_t jslam_match_band(int32_t level, float scale, int32_t row_band_px)
{
    return match_band(level, scale, row_band_px);
}

}  // extern "C"
