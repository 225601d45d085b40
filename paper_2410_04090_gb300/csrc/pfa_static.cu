// PFA scores without device allocation.
//
// Some callers cannot allocate device memory: a real-time loop that forbids
// allocation after start-up (allocation can block and fragment), code that
// runs inside another framework's enqueue hook where only the framework may
// allocate, or a process whose device memory is handed out by a fixed pool.
// jslam_pfa_scores_static serves them: it computes, for a caller-supplied
// list of culled corners of one image, the aggregation scores K_l and K_r at
// each corner's s0 pixel and whether the sparse q x q NMS keeps it -- the
// same scores the full extraction reports -- using only a scratch table that
// lives in this file as a statically allocated device array.
//
// The table belongs to every GPU that loads the library, for the life of the
// process, and every call shares it: two calls whose kernels overlap on the
// GPU (different streams, or different host threads) race on it.  Each call
// clears the table before it uses it.
#include <cmath>
#include <mutex>

#include "jslam.h"
#include "jslam_internal.h"
#include "tables.h"

namespace jslam {

constexpr int kStaticMaxCandidates = 16384;              // largest n accepted
constexpr int kStaticSlots = 2 * kStaticMaxCandidates;   // open-addressing table, load <= 1/2
constexpr int kStaticThreads = 1024;

struct StaticPfaScratch {
    uint32_t key[kStaticSlots];  // s0 pixel index + 1; 0 = empty
    uint32_t val[kStaticSlots];  // mask of the levels seen << 16 | K_r (K_l = bits of the mask)
};

// 256 KB of device memory per GPU, reserved when the library is loaded.
static __device__ __align__(256) StaticPfaScratch g_pfa_scratch;

struct LevelScales {
    double s[kMaxLevels];
};

__device__ __forceinline__ uint32_t slot_of(uint32_t key)
{
    return (key * 2654435761u) >> (32 - 15);  // kStaticSlots = 2^15
}

// Entry of `key` (inserted if absent).  The table is at most half full, so
// the probe ends within kStaticSlots steps.
__device__ __forceinline__ int table_insert(StaticPfaScratch *t, uint32_t key)
{
    uint32_t h = slot_of(key);
    for (int probe = 0; probe < kStaticSlots; ++probe, h = (h + 1) & (kStaticSlots - 1)) {
        const uint32_t prev = atomicCAS(&t->key[h], 0u, key);
        if (prev == 0u || prev == key) return (int)h;
    }
    return -1;
}

__device__ __forceinline__ uint32_t table_value(const StaticPfaScratch *t, uint32_t key)
{
    uint32_t h = slot_of(key);
    for (int probe = 0; probe < kStaticSlots; ++probe, h = (h + 1) & (kStaticSlots - 1)) {
        const uint32_t k = t->key[h];
        if (k == key) return t->val[h];
        if (k == 0u) return 0u;
    }
    return 0u;
}

__device__ __forceinline__ int project_s0(int v, double s, int extent)
{
    const int p = (int)floor(__dadd_rn(__dmul_rn((double)v, s), 0.5));
    return p < extent - 1 ? p : extent - 1;
}

// Outputs of a corner that takes no part in the scores: a level outside the
// image's pyramid, a response above the largest SAD (16 x 255), or a repeat
// of a corner already counted.
__device__ __forceinline__ void reject(int i, uint16_t *Xo, uint16_t *Yo, uint8_t *k_levels, uint32_t *k_resp,
                                       uint8_t *alive)
{
    Xo[i] = 0xFFFFu;
    Yo[i] = 0xFFFFu;
    k_levels[i] = 0;
    k_resp[i] = 0u;
    alive[i] = 2;
}

// One CTA: clear, accumulate (K_l, K_r) per s0 pixel, then the NMS test.
// Each thread handles the same corners i in both phases, so the rejections it
// writes in the first are its own to read in the second.
__global__ void __launch_bounds__(kStaticThreads)
k_pfa_scores_static(StaticPfaScratch *t, const uint8_t *level, const uint16_t *x, const uint16_t *y,
                    const uint16_t *response, int n, int W0, int H0, int levels, LevelScales sc, int rad,
                    int rule, uint16_t *Xo, uint16_t *Yo, uint8_t *k_levels, uint32_t *k_resp, uint8_t *alive)
{
    for (int i = threadIdx.x; i < kStaticSlots; i += kStaticThreads) {
        t->key[i] = 0u;
        t->val[i] = 0u;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += kStaticThreads) {
        const int l = level[i];
        const uint32_t r = response[i];
        if (l >= levels || r > 16u * 255u) { reject(i, Xo, Yo, k_levels, k_resp, alive); continue; }
        const int X = project_s0(x[i], sc.s[l], W0), Y = project_s0(y[i], sc.s[l], H0);
        const int h = table_insert(t, (uint32_t)(Y * W0 + X) + 1u);
        // distinct pixels of one level project to distinct s0 pixels (zeta^n
        // >= 1), so a level already in this pixel's mask is a repeated corner
        const uint32_t bit = 1u << (16 + l);
        if (h < 0 || (atomicOr(&t->val[h], bit) & bit)) { reject(i, Xo, Yo, k_levels, k_resp, alive); continue; }
        atomicAdd(&t->val[h], r);  // at most 8 x 4080 < 2^16: never reaches the mask
        Xo[i] = (uint16_t)X;
        Yo[i] = (uint16_t)Y;
        alive[i] = 1;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += kStaticThreads) {
        if (alive[i] == 2) continue;
        const int X = Xo[i], Y = Yo[i];
        const uint32_t own = table_value(t, (uint32_t)(Y * W0 + X) + 1u);
        const uint32_t kl = __popc(own >> 16), kr = own & 0xFFFFu;
        bool dom = false;
        for (int dy = -rad; dy <= rad; ++dy) {
            const int qy = Y + dy;
            if (qy < 0 || qy >= H0) continue;
            for (int dx = -rad; dx <= rad; ++dx) {
                const int qx = X + dx;
                if ((dx | dy) == 0 || qx < 0 || qx >= W0) continue;
                const uint32_t w = table_value(t, (uint32_t)(qy * W0 + qx) + 1u);
                if (!w) continue;
                const uint32_t ql = __popc(w >> 16), qr = w & 0xFFFFu;
                dom |= rule == 0 ? (ql > kl && qr > kr) : (ql > kl || (ql == kl && qr > kr));
            }
        }
        k_levels[i] = (uint8_t)kl;
        k_resp[i] = kr;
        alive[i] = dom ? 0 : 1;
    }
}

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
StaticPfaScratch *g_scratch_ptr[kMaxDevices] = {};

// Device address of the static table on `device` (which must be current).
// Looked up once per device; later calls reuse it.  The address belongs to
// the device's primary context: after cudaDeviceReset the cached value is
// stale, so a process that resets a device must not call the entry point on
// it again.
cudaError_t scratch_on(int device, StaticPfaScratch **out)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_pfa_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[device] = static_cast<StaticPfaScratch *>(p);
    }
    *out = g_scratch_ptr[device];
    return cudaSuccess;
}

}  // namespace
}  // namespace jslam

using namespace jslam;

extern "C" jslam_status jslam_pfa_scores_static(const uint8_t *level, const uint16_t *x, const uint16_t *y,
                                                const uint16_t *response, int32_t n, int32_t width0,
                                                int32_t height0, int32_t levels, float scale, int32_t nms_q,
                                                int32_t pfa_rule, uint16_t *X, uint16_t *Y, uint8_t *k_levels,
                                                uint32_t *k_resp, uint8_t *alive, int32_t device,
                                                void *cuda_stream)
{
    if (n < 0) return JSLAM_ERR_ARG;
    if (n > kStaticMaxCandidates) return JSLAM_ERR_CAPACITY;
    if (width0 < 1 || width0 > 4096 || height0 < 1 || height0 > 4096) return JSLAM_ERR_ARG;
    if (levels < 1 || levels > kMaxLevels || !(scale > 1.0f) || !(scale < 16.0f)) return JSLAM_ERR_ARG;
    if (nms_q < 1 || nms_q > 7 || (nms_q & 1) == 0 || pfa_rule < 0 || pfa_rule > 1) return JSLAM_ERR_ARG;
    if (device < 0 || device >= kMaxDevices) return JSLAM_ERR_ARG;
    if (n > 0 && (!level || !x || !y || !response || !X || !Y || !k_levels || !k_resp || !alive))
        return JSLAM_ERR_ARG;
    if (n == 0) return JSLAM_OK;

    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) { cudaGetLastError(); return JSLAM_ERR_CUDA; }
    if (prev != device && cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return JSLAM_ERR_CUDA; }
    StaticPfaScratch *table = nullptr;
    cudaError_t e = scratch_on(device, &table);
    if (e == cudaSuccess) {
        LevelScales sc;
        for (int l = 0; l < kMaxLevels; ++l) sc.s[l] = zeta_pow(scale, l < levels ? l : levels - 1);
        k_pfa_scores_static<<<1, kStaticThreads, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
            table, level, x, y, response, n, width0, height0, levels, sc, (nms_q - 1) / 2, pfa_rule, X, Y,
            k_levels, k_resp, alive);
        e = cudaGetLastError();
    }
    if (prev != device) cudaSetDevice(prev);
    if (e != cudaSuccess) { cudaGetLastError(); return JSLAM_ERR_CUDA; }
    return JSLAM_OK;
}
