// Persistent cache of autotuner picks: a JSON file mapping a batch signature
// (GPU name and SM count, the context's parameters, the batch's image sizes,
// depths and per-pair parameters) to the launch shapes the tuner chose, so
// that a process that meets the same batch again skips the tuning runs.
//
// File layout (written by this file, read back by the small parser below):
//   {
//     "format": "jslam-tune-cache",
//     "version": 1,
//     "entries": {
//       "<key>": {"tile_w_px": 128, "tile_h_px": 128, "nms_kernel": 0,
//                 "detect_ctas_per_sm": 0, "tile_order": 0, "stage_ms": 0.8612},
//       (an entry without "tile_order" reads as 0)
//       ...
//     }
//   }
// Keys hold no quote or backslash (the key builder replaces them), so the
// parser needs no escapes.  A file that does not parse is treated as empty;
// writes go to a temporary file renamed over the old one, so readers never
// see a half-written file (two writers at once: the last rename wins).
//
// Host code only: no device call, so every function here runs without a GPU.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <unistd.h>

#include "jslam.h"

namespace {

struct Entry {
    jslam_tuning t{};
    double ms = 0.0;
};

bool read_file(const char *path, std::string *out)
{
    FILE *f = std::fopen(path, "rb");
    if (!f) return false;
    char buf[4096];
    size_t got;
    out->clear();
    while ((got = std::fread(buf, 1, sizeof buf, f)) > 0) out->append(buf, got);
    std::fclose(f);
    return true;
}

struct Parser {
    const std::string &s;
    size_t i = 0;
    explicit Parser(const std::string &text) : s(text) {}
    void ws()
    {
        while (i < s.size() && (s[i] == ' ' || s[i] == '\n' || s[i] == '\r' || s[i] == '\t')) ++i;
    }
    bool lit(char c)
    {
        ws();
        if (i < s.size() && s[i] == c) { ++i; return true; }
        return false;
    }
    bool str(std::string *out)
    {
        if (!lit('"')) return false;
        const size_t end = s.find('"', i);
        if (end == std::string::npos) return false;
        out->assign(s, i, end - i);
        if (out->find('\\') != std::string::npos) return false;
        i = end + 1;
        return true;
    }
    bool num(double *v)
    {
        ws();
        const char *start = s.c_str() + i;
        char *stop = nullptr;
        *v = std::strtod(start, &stop);
        if (stop == start) return false;
        i += (size_t)(stop - start);
        return true;
    }
    // Skip one JSON value of the kinds this file holds (string, number, object).
    bool skip_value()
    {
        ws();
        if (i >= s.size()) return false;
        if (s[i] == '"') { std::string t; return str(&t); }
        if (s[i] == '{') {
            ++i;
            if (lit('}')) return true;
            do {
                std::string k;
                if (!str(&k) || !lit(':') || !skip_value()) return false;
            } while (lit(','));
            return lit('}');
        }
        double v;
        return num(&v);
    }
};

bool parse_entry(Parser &p, Entry *e)
{
    if (!p.lit('{')) return false;
    if (p.lit('}')) return true;
    do {
        std::string k;
        double v = 0.0;
        if (!p.str(&k) || !p.lit(':')) return false;
        if (k == "tile_w_px" || k == "tile_h_px" || k == "nms_kernel" || k == "detect_ctas_per_sm" ||
            k == "tile_order" || k == "stage_ms") {
            if (!p.num(&v)) return false;
            if (k == "tile_w_px") e->t.tile_w_px = (int32_t)v;
            else if (k == "tile_h_px") e->t.tile_h_px = (int32_t)v;
            else if (k == "nms_kernel") e->t.nms_kernel = (int32_t)v;
            else if (k == "detect_ctas_per_sm") e->t.detect_ctas_per_sm = (int32_t)v;
            else if (k == "tile_order") e->t.tile_order = (int32_t)v;
            else e->ms = v;
        } else if (!p.skip_value()) {
            return false;
        }
    } while (p.lit(','));
    return p.lit('}');
}

// Entries of the file at `path`; empty when it is missing or does not parse.
std::map<std::string, Entry> load(const char *path)
{
    std::map<std::string, Entry> out;
    std::string text;
    if (!read_file(path, &text)) return out;
    Parser p(text);
    if (!p.lit('{')) return out;
    if (p.lit('}')) return out;
    do {
        std::string k;
        if (!p.str(&k) || !p.lit(':')) return {};
        if (k == "entries") {
            if (!p.lit('{')) return {};
            if (p.lit('}')) continue;
            do {
                std::string key;
                Entry e;
                if (!p.str(&key) || !p.lit(':') || !parse_entry(p, &e)) return {};
                out[key] = e;
            } while (p.lit(','));
            if (!p.lit('}')) return {};
        } else if (!p.skip_value()) {
            return {};
        }
    } while (p.lit(','));
    if (!p.lit('}')) return {};
    return out;
}

bool tuning_ok(const jslam_tuning &t)
{
    return t.tile_w_px >= 32 && t.tile_w_px <= 128 && t.tile_w_px % 4 == 0 && t.tile_h_px >= 8 &&
           t.tile_h_px <= 128 && t.nms_kernel >= 0 && t.nms_kernel <= 1 && t.detect_ctas_per_sm >= 0 &&
           t.detect_ctas_per_sm <= 8 && t.tile_order >= 0 && t.tile_order <= 1;
}

}  // namespace

extern "C" {

jslam_status jslam_tune_key(const char *gpu_name, int32_t sm_count, const jslam_config *cfg,
                            const jslam_stereo_job *jobs, int32_t n, char *buf, size_t len)
{
    if (!gpu_name || !cfg || !jobs || n < 1 || !buf || sm_count < 1) return JSLAM_ERR_ARG;
    std::string k = "gpu=";
    for (const char *c = gpu_name; *c; ++c) k += (*c == '"' || *c == '\\' || (unsigned char)*c < 32) ? '_' : *c;
    char tmp[256];
    std::snprintf(tmp, sizeof tmp, "|sm=%d|p=%d,%d|k=%d|q=%d|b=%d|rule=%d|lo=%d", sm_count, cfg->p_min, cfg->p_max,
                  cfg->k_per_cell, cfg->nms_q, cfg->border, cfg->pfa_rule, cfg->fast_thresh_lo);
    k += tmp;
    k += "|jobs=";
    for (int p = 0; p < n; ++p) {
        const jslam_stereo_job &j = jobs[p];
        uint32_t sbits;
        std::memcpy(&sbits, &j.scale, 4);
        std::snprintf(tmp, sizeof tmp, "%s%dx%d:L%d:s%08x:e%d:c%d:f%d:m%d%d", p ? ";" : "", j.left.width,
                      j.left.height, j.levels, sbits, j.fast_thresh, j.cell, j.max_feats, j.left.memory,
                      j.right.memory);
        k += tmp;
    }
    if (k.size() + 1 > len) return JSLAM_ERR_CAPACITY;
    std::memcpy(buf, k.c_str(), k.size() + 1);
    return JSLAM_OK;
}

jslam_status jslam_tune_cache_get(const char *path, const char *key, jslam_tuning *out, int32_t *found)
{
    if (!path || !key || !out || !found) return JSLAM_ERR_ARG;
    *found = 0;
    const std::map<std::string, Entry> m = load(path);
    const auto it = m.find(key);
    if (it == m.end() || !tuning_ok(it->second.t)) return JSLAM_OK;
    *out = it->second.t;
    *found = 1;
    return JSLAM_OK;
}

jslam_status jslam_tune_cache_put(const char *path, const char *key, const jslam_tuning *t, float stage_ms)
{
    if (!path || !key || !t || !tuning_ok(*t)) return JSLAM_ERR_ARG;
    if (std::strchr(key, '"') || std::strchr(key, '\\')) return JSLAM_ERR_ARG;
    std::map<std::string, Entry> m = load(path);
    Entry &e = m[key];
    e.t = *t;
    e.ms = stage_ms;
    const std::string tmp = std::string(path) + ".tmp" + std::to_string((long)getpid());
    FILE *f = std::fopen(tmp.c_str(), "wb");
    if (!f) return JSLAM_ERR_ARG;
    bool ok = std::fprintf(f, "{\n  \"format\": \"jslam-tune-cache\",\n  \"version\": 1,\n  \"entries\": {") > 0;
    size_t i = 0;
    for (const auto &kv : m) {
        ok = ok && std::fprintf(f,
                                "%s\n    \"%s\": {\"tile_w_px\": %d, \"tile_h_px\": %d, \"nms_kernel\": %d, "
                                "\"detect_ctas_per_sm\": %d, \"tile_order\": %d, \"stage_ms\": %.6f}",
                                i++ ? "," : "", kv.first.c_str(), kv.second.t.tile_w_px, kv.second.t.tile_h_px,
                                kv.second.t.nms_kernel, kv.second.t.detect_ctas_per_sm, kv.second.t.tile_order,
                                kv.second.ms) > 0;
    }
    ok = ok && std::fprintf(f, "\n  }\n}\n") > 0;
    ok = (std::fclose(f) == 0) && ok;
    if (!ok || std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return JSLAM_ERR_ARG;
    }
    return JSLAM_OK;
}

}  // extern "C"
