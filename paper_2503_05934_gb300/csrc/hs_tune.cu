// Batched-form entry points, and the autotuners of the batched form's and
// the single-array merge path's launch plans.
//
// The batched tuner times candidate plans on the caller's own segments: leaf
// network set (leaf size 8, 7, 5 or 4: {6,7,8}, {3,5,7}, {3,4,5}, {3,4}),
// CTA shape (256 threads x four leaves or 512 threads x two leaves) and persistent
// CTAs per SM.  The single-array tuner times the block-sort shape (256 or
// 288 threads) and the merge fan-in (binary or four-way levels) on the
// caller's own array, for its network set.  Every plan produces the same
// bytes; only the time differs.  Winners are cached in-process by device name
// and size buckets and can be saved to / loaded from a small JSON file.
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "hs_networks.cuh"
#include "hs_segsort.h"

namespace hs {

struct TuneEntry {
    std::string device;
    int n_bucket, s_bucket, m_bucket;
    hs_plan plan;
    double ms;
};

static std::mutex g_tune_mu;
static std::vector<TuneEntry> g_tune;

static int log2_bucket(double x) {
    int b = 0;
    while (x >= 2.0 && b < 62) {
        x /= 2.0;
        ++b;
    }
    return b;
}

static hs_status device_name(std::string *out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_cuda(e, "cudaGetDevice");
    cudaDeviceProp prop;
    if ((e = cudaGetDeviceProperties(&prop, dev)) != cudaSuccess)
        return fail_cuda(e, "cudaGetDeviceProperties");
    *out = prop.name;
    return HS_OK;
}

static bool cache_find(const std::string &dev, int nb, int sb, int mb, TuneEntry *out) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const TuneEntry &t : g_tune)
        if (t.device == dev && t.n_bucket == nb && t.s_bucket == sb && t.m_bucket == mb) {
            *out = t;
            return true;
        }
    return false;
}

static size_t cache_size() {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return g_tune.size();
}

static void cache_put(const TuneEntry &e) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (TuneEntry &t : g_tune)
        if (t.device == e.device && t.n_bucket == e.n_bucket && t.s_bucket == e.s_bucket &&
            t.m_bucket == e.m_bucket) {
            t = e;
            return;
        }
    g_tune.push_back(e);
}

size_t autotune_workspace_bytes(size_t n_keys, size_t num_segs) {
    return segsort_workspace_bytes(n_keys, num_segs) + align_up(n_keys * sizeof(int32_t), 256);
}

static hs_status time_plan(int32_t *keys, const int32_t *backup, size_t n_keys,
                           const int64_t *offs, size_t nseg, const hs_plan &p, void *ws,
                           size_t ws_bytes, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1,
                           float *ms) {
    const size_t bytes = n_keys * sizeof(int32_t);
    for (int rep = 0; rep < 2; ++rep) {  // one warm-up, one timed run
        cudaError_t e = cudaMemcpyAsync(keys, backup, bytes, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return fail_cuda(e, "autotune: restore keys");
        if (rep == 1 && (e = cudaEventRecord(e0, st)) != cudaSuccess)
            return fail_cuda(e, "autotune: event");
        hs_status r = segsort(keys, n_keys, offs, nseg, p, ws, ws_bytes, st);
        if (r != HS_OK) return r;
        if (rep == 1 && (e = cudaEventRecord(e1, st)) != cudaSuccess)
            return fail_cuda(e, "autotune: event");
    }
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    if (e != cudaSuccess) return fail_cuda(e, "autotune: timing");
    return HS_OK;
}

hs_status autotune(int32_t *d_keys, size_t n_keys, const int64_t *d_offsets, size_t num_segs,
                   void *d_ws, size_t ws_bytes, cudaStream_t st, hs_plan *best, double *best_ms) {
    if (!best) return fail(HS_ERR_INVALID_ARG, "hs_segsort_autotune: NULL result");
    if (num_segs == 0 || n_keys == 0) {
        *best = default_seg_plan(HS_NETS_6TO8);
        if (best_ms) *best_ms = 0.0;
        return HS_OK;
    }
    const size_t seg_ws = segsort_workspace_bytes(n_keys, num_segs);
    if (!d_ws || ws_bytes < autotune_workspace_bytes(n_keys, num_segs))
        return fail(HS_ERR_INVALID_ARG,
                    "hs_segsort_autotune: workspace smaller than hs_segsort_autotune_workspace_bytes");
    std::string dev;
    hs_status r = device_name(&dev);
    if (r != HS_OK) return r;
    const int nb = log2_bucket((double)n_keys), sb = log2_bucket((double)num_segs),
              mb = log2_bucket((double)n_keys / (double)num_segs);
    TuneEntry hit;
    if (cache_find(dev, nb, sb, mb, &hit)) {
        *best = hit.plan;
        if (best_ms) *best_ms = hit.ms;
        return HS_OK;
    }
    int32_t *backup = reinterpret_cast<int32_t *>(static_cast<char *>(d_ws) + seg_ws);
    const size_t bytes = n_keys * sizeof(int32_t);
    cudaError_t e = cudaMemcpyAsync(backup, d_keys, bytes, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return fail_cuda(e, "autotune: save keys");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return fail_cuda(e, "autotune: events");
    }
    const hs_netset sets[] = {HS_NETS_6TO8, HS_NETS_ODD, HS_NETS_3TO5, HS_NETS_3TO4};
    const int threads[] = {256, 512};
    const int ctas[] = {0, 1, 2};
    float best_t = 1e30f;
    hs_plan best_p = default_seg_plan(HS_NETS_6TO8);
    for (hs_netset s : sets)
        for (int nt : threads)
            for (int c : ctas) {
                hs_plan p = default_seg_plan(s);
                p.block_threads = nt;
                p.ctas_per_sm = c;
                float ms = 0.f;
                r = time_plan(d_keys, backup, n_keys, d_offsets, num_segs, p, d_ws, seg_ws, st, e0,
                              e1, &ms);
                if (r != HS_OK) break;
                if (ms < best_t) {
                    best_t = ms;
                    best_p = p;
                }
            }
    if (r == HS_OK) {
        e = cudaMemcpyAsync(d_keys, backup, bytes, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) r = fail_cuda(e, "autotune: restore keys");
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r != HS_OK) return r;
    cache_put(TuneEntry{dev, nb, sb, mb, best_p, (double)best_t});
    *best = best_p;
    if (best_ms) *best_ms = best_t;
    return HS_OK;
}

// ---------------------------------------------------------------------------
// Single-array merge path.

size_t sort_autotune_workspace_bytes(size_t n) {
    return merge_workspace_bytes(n, 0) + align_up(n * sizeof(int32_t), 256);
}

// One warm-up and two timed sorts of the saved keys under plan p; the
// smaller time.
static hs_status time_sort_plan(int32_t *keys, const int32_t *backup, size_t n, hs_netset s,
                                const SortPlan &p, void *ws, size_t ws_bytes, cudaStream_t st,
                                cudaEvent_t e0, cudaEvent_t e1, float *ms) {
    const size_t bytes = n * sizeof(int32_t);
    struct Force {
        explicit Force(const SortPlan *q) { sort_plan_force(q); }
        ~Force() { sort_plan_force(nullptr); }
    } force(&p);
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        cudaError_t e = cudaMemcpyAsync(keys, backup, bytes, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return fail_cuda(e, "sort autotune: restore keys");
        if ((e = cudaEventRecord(e0, st)) != cudaSuccess) return fail_cuda(e, "sort autotune: event");
        hs_status r = merge_sort(keys, nullptr, n, s, ws, ws_bytes, st);
        if (r != HS_OK) return r;
        if ((e = cudaEventRecord(e1, st)) != cudaSuccess) return fail_cuda(e, "sort autotune: event");
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return fail_cuda(e, "sort autotune: timing");
        float t = 0.f;
        if ((e = cudaEventElapsedTime(&t, e0, e1)) != cudaSuccess)
            return fail_cuda(e, "sort autotune: timing");
        if (rep > 0 && t < best) best = t;
    }
    *ms = best;
    return HS_OK;
}

hs_status sort_autotune(int32_t *d_keys, size_t n, hs_netset s, void *d_ws, size_t ws_bytes,
                        cudaStream_t st, hs_sort_plan *best, double *best_ms) {
    if (!best) return fail(HS_ERR_INVALID_ARG, "hs_sort_autotune: NULL result");
    if (!netset_ok(s))
        return fail(HS_ERR_INVALID_ARG, "hs_sort_autotune: netset is neither a set of sizes 3..8 nor a VarSort configuration");
    if (n > 0 && (!d_keys || !aligned(d_keys, 4)))
        return fail(HS_ERR_INVALID_ARG, "hs_sort_autotune: NULL or unaligned keys with n > 0");
    if (n > (size_t)INT64_MAX / 16) return fail(HS_ERR_INVALID_ARG, "hs_sort_autotune: n too large");
    const int L = leaf_size(s);
    if (n <= 1) {
        *best = hs_sort_plan{256, 2, {0, 0}};
        if (best_ms) *best_ms = 0.0;
        return HS_OK;
    }
    const size_t sort_ws = merge_workspace_bytes(n, 0);
    if (!d_ws || ws_bytes < sort_autotune_workspace_bytes(n))
        return fail(HS_ERR_INVALID_ARG,
                    "hs_sort_autotune: workspace smaller than hs_sort_autotune_workspace_bytes");
    if (!aligned(d_ws, 16)) return fail(HS_ERR_INVALID_ARG, "hs_sort_autotune: workspace not 16-byte aligned");
    std::string dev;
    hs_status r = current_device_name(&dev);
    if (r != HS_OK) return r;
    const int nb = size_bucket((int64_t)n);
    SortPlan hit;
    double hit_ms = 0.0;
    if (sort_plan_cache_get(dev, nb, L, &hit, &hit_ms)) {
        *best = hs_sort_plan{hit.shape == 4 ? 288 : 256, hit.fanin, {0, 0}};
        if (best_ms) *best_ms = hit_ms;
        return HS_OK;
    }
    int32_t *backup = reinterpret_cast<int32_t *>(static_cast<char *>(d_ws) + sort_ws);
    const size_t bytes = n * sizeof(int32_t);
    cudaError_t e = cudaMemcpyAsync(backup, d_keys, bytes, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return fail_cuda(e, "sort autotune: save keys");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return fail_cuda(e, "sort autotune: events");
    }
    const bool four_ok = merge_four_way_possible(d_keys, (int64_t)n);
    float best_t = 1e30f;
    SortPlan best_p{2, 2};
    for (int shape : {2, 4})
        for (int fanin : {2, 4}) {
            if (fanin == 4 && !four_ok) continue;
            const SortPlan p{shape, fanin};
            float ms = 0.f;
            r = time_sort_plan(d_keys, backup, n, s, p, d_ws, sort_ws, st, e0, e1, &ms);
            if (r != HS_OK) break;
            if (ms < best_t) {
                best_t = ms;
                best_p = p;
            }
        }
    // The keys go back as they came, whatever happened above.
    e = cudaMemcpyAsync(d_keys, backup, bytes, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess && r == HS_OK) r = fail_cuda(e, "sort autotune: restore keys");
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r != HS_OK) return r;
    sort_plan_cache_put(dev, nb, L, best_p, (double)best_t);
    *best = hs_sort_plan{best_p.shape == 4 ? 288 : 256, best_p.fanin, {0, 0}};
    if (best_ms) *best_ms = best_t;
    return HS_OK;
}

static void save_sort_entry(void *ctx, const std::string &device, int n_bucket, int leaf,
                            const SortPlan &p, double ms) {
    std::vector<std::string> *out = static_cast<std::vector<std::string> *>(ctx);
    char buf[512];
    std::snprintf(buf, sizeof buf,
                  "  {\"kind\": \"sort\", \"device\": \"%s\", \"n_bucket\": %d, \"leaf\": %d, "
                  "\"blocksort_threads\": %d, \"merge_fanin\": %d, \"ms\": %.6f}",
                  device.c_str(), n_bucket, leaf, p.shape == 4 ? 288 : 256, p.fanin, ms);
    out->push_back(buf);
}

hs_status tune_cache_save(const char *path) {
    std::vector<std::string> lines;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (const TuneEntry &t : g_tune) {
            char buf[512];
            std::snprintf(buf, sizeof buf,
                          "  {\"kind\": \"batched\", \"device\": \"%s\", \"n_bucket\": %d, "
                          "\"s_bucket\": %d, \"m_bucket\": %d, \"netset\": %u, "
                          "\"block_threads\": %d, \"ctas_per_sm\": %d, \"ms\": %.6f}",
                          t.device.c_str(), t.n_bucket, t.s_bucket, t.m_bucket, t.plan.netset,
                          t.plan.block_threads, t.plan.ctas_per_sm, t.ms);
            lines.push_back(buf);
        }
    }
    sort_plan_cache_each(save_sort_entry, &lines);
    FILE *f = std::fopen(path, "w");
    if (!f) return fail(HS_ERR_INVALID_ARG, std::string("hs_tune_cache_save: cannot open ") + path);
    std::fprintf(f, "[\n");
    for (size_t i = 0; i < lines.size(); ++i)
        std::fprintf(f, "%s%s\n", lines[i].c_str(), i + 1 < lines.size() ? "," : "");
    std::fprintf(f, "]\n");
    return std::fclose(f) == 0 ? HS_OK : fail(HS_ERR_INVALID_ARG, "hs_tune_cache_save: write failed");
}

static bool json_int(const std::string &obj, const char *key, long long *v) {
    const std::string k = std::string("\"") + key + "\"";
    size_t p = obj.find(k);
    if (p == std::string::npos) return false;
    p = obj.find(':', p + k.size());
    if (p == std::string::npos) return false;
    return std::sscanf(obj.c_str() + p + 1, " %lld", v) == 1;
}

static bool json_num(const std::string &obj, const char *key, double *v) {
    const std::string k = std::string("\"") + key + "\"";
    size_t p = obj.find(k);
    if (p == std::string::npos) return false;
    p = obj.find(':', p + k.size());
    if (p == std::string::npos) return false;
    return std::sscanf(obj.c_str() + p + 1, " %lf", v) == 1;
}

static bool json_str(const std::string &obj, const char *key, std::string *v) {
    const std::string k = std::string("\"") + key + "\"";
    size_t p = obj.find(k);
    if (p == std::string::npos) return false;
    p = obj.find('"', obj.find(':', p + k.size()) + 1);
    if (p == std::string::npos) return false;
    size_t q = obj.find('"', p + 1);
    if (q == std::string::npos) return false;
    *v = obj.substr(p + 1, q - p - 1);
    return true;
}

// Reads a file written by tune_cache_save.  Entries of kind "sort" are
// single-array plans; entries of kind "batched", or with no kind, batched
// plans.  Nothing is cached unless every entry parses and is valid.
hs_status tune_cache_load(const char *path) {
    FILE *f = std::fopen(path, "r");
    if (!f) return fail(HS_ERR_INVALID_ARG, std::string("hs_tune_cache_load: cannot open ") + path);
    std::string text;
    char buf[4096];
    size_t got;
    while ((got = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, got);
    std::fclose(f);
    struct SortEntry {
        std::string device;
        int n_bucket, leaf;
        SortPlan plan;
        double ms;
    };
    size_t pos = 0;
    std::vector<TuneEntry> parsed;
    std::vector<SortEntry> parsed_sort;
    while ((pos = text.find('{', pos)) != std::string::npos) {
        size_t end = text.find('}', pos);
        if (end == std::string::npos) return fail(HS_ERR_INVALID_ARG, "hs_tune_cache_load: unterminated entry");
        const std::string obj = text.substr(pos, end - pos + 1);
        pos = end + 1;
        std::string kind = "batched";
        if (obj.find("\"kind\"") != std::string::npos && !json_str(obj, "kind", &kind))
            return fail(HS_ERR_INVALID_ARG, "hs_tune_cache_load: malformed kind");
        if (kind == "sort") {
            SortEntry t{};
            long long nb, leaf, bt, fi;
            if (!json_str(obj, "device", &t.device) || !json_int(obj, "n_bucket", &nb) ||
                !json_int(obj, "leaf", &leaf) || !json_int(obj, "blocksort_threads", &bt) ||
                !json_int(obj, "merge_fanin", &fi) || !json_num(obj, "ms", &t.ms))
                return fail(HS_ERR_INVALID_ARG, "hs_tune_cache_load: malformed sort entry");
            if (nb < 0 || nb > 62 || leaf < 1 || leaf > 8 || (bt != 256 && bt != 288) ||
                (fi != 2 && fi != 4))
                return fail(HS_ERR_INVALID_ARG, "hs_tune_cache_load: invalid sort plan");
            t.n_bucket = (int)nb;
            t.leaf = (int)leaf;
            t.plan = SortPlan{bt == 288 ? 4 : 2, (int)fi};
            parsed_sort.push_back(t);
            continue;
        }
        if (kind != "batched") return fail(HS_ERR_INVALID_ARG, "hs_tune_cache_load: unknown kind " + kind);
        TuneEntry t{};
        long long nb, sb, mb, ns, bt, cp;
        if (!json_str(obj, "device", &t.device) || !json_int(obj, "n_bucket", &nb) ||
            !json_int(obj, "s_bucket", &sb) || !json_int(obj, "m_bucket", &mb) ||
            !json_int(obj, "netset", &ns) || !json_int(obj, "block_threads", &bt) ||
            !json_int(obj, "ctas_per_sm", &cp) || !json_num(obj, "ms", &t.ms))
            return fail(HS_ERR_INVALID_ARG, "hs_tune_cache_load: malformed entry");
        t.n_bucket = (int)nb;
        t.s_bucket = (int)sb;
        t.m_bucket = (int)mb;
        t.plan = default_seg_plan((hs_netset)ns);
        t.plan.block_threads = (int32_t)bt;
        t.plan.ctas_per_sm = (int32_t)cp;
        if (check_plan(t.plan) != HS_OK) return fail(HS_ERR_INVALID_ARG, "hs_tune_cache_load: invalid plan");
        parsed.push_back(t);
    }
    for (const TuneEntry &t : parsed) cache_put(t);
    for (const SortEntry &t : parsed_sort) sort_plan_cache_put(t.device, t.n_bucket, t.leaf, t.plan, t.ms);
    return HS_OK;
}

}  // namespace hs

using namespace hs;

extern "C" {

size_t hs_segsort_workspace_bytes(size_t n_keys, size_t num_segs) {
    return segsort_workspace_bytes(n_keys, num_segs);
}

// The plan a NULL plan stands for: the one hs_segsort_autotune cached for
// this device and these size buckets when its network set is s, else s with
// the default shape.
static hs_plan tuned_or_default(size_t n_keys, size_t num_segs, hs_netset s) {
    if (n_keys > 0 && num_segs > 0 && cache_size() > 0) {
        std::string dev;
        if (current_device_name(&dev) == HS_OK) {
            TuneEntry hit;
            if (cache_find(dev, log2_bucket((double)n_keys), log2_bucket((double)num_segs),
                           log2_bucket((double)n_keys / (double)num_segs), &hit) &&
                hit.plan.netset == s)
                return hit.plan;
        } else {
            clear_error();  // no device to match: the default shape
        }
    }
    return default_seg_plan(s);
}

static hs_status plan_from(const hs_plan *plan, hs_netset s, size_t n_keys, size_t num_segs,
                           hs_plan *out) {
    if (plan) {
        if (plan->reserved != 0) return fail(HS_ERR_INVALID_ARG, "plan reserved field must be 0");
        *out = *plan;
    } else {
        if (!netset_ok(s)) return fail(HS_ERR_INVALID_ARG, "netset is neither a set of sizes 3..8 nor a VarSort configuration");
        *out = tuned_or_default(n_keys, num_segs, s);
    }
    return check_plan(*out);
}

hs_status hs_segsort_i32(int32_t *d_keys, size_t n_keys, const int64_t *d_offsets, size_t num_segs,
                         hs_algo a, hs_netset s, const hs_plan *plan, void *d_ws, size_t ws_bytes,
                         hs_stream_t stream) {
    const ApiRange range("hs_segsort_i32");
    clear_error();
    if (a == HS_ALGO_QUICK)
        return fail(HS_ERR_UNSUPPORTED, "hs_segsort_i32: the batched form runs the merge path only");
    if (a != HS_ALGO_MERGE) return fail(HS_ERR_INVALID_ARG, "hs_segsort_i32: unknown algo");
    hs_plan p;
    hs_status r = plan_from(plan, s, n_keys, num_segs, &p);
    if (r != HS_OK) return r;
    return segsort(d_keys, n_keys, d_offsets, num_segs, p, d_ws, ws_bytes, (cudaStream_t)stream);
}

hs_status hs_sort_i32_many(int32_t *d_keys, size_t n_keys, const int64_t *h_offsets,
                           size_t num_segs, hs_algo a, hs_netset s, void *d_ws, size_t ws_bytes,
                           hs_stream_t stream) {
    clear_error();
    if (num_segs > 0 && !h_offsets) return fail(HS_ERR_INVALID_ARG, "hs_sort_i32_many: NULL offsets");
    for (size_t i = 0; i < num_segs; ++i) {
        const int64_t b = h_offsets[i], e = h_offsets[i + 1];
        if (b < 0 || e < b || (size_t)e > n_keys)
            return fail(HS_ERR_INVALID_ARG, "hs_sort_i32_many: malformed offsets");
        hs_status r = hs_sort_i32(d_keys + b, (size_t)(e - b), a, s, d_ws, ws_bytes, stream);
        if (r != HS_OK) return r;
    }
    return HS_OK;
}

hs_status hs_segsort_capture(int32_t *d_keys, size_t n_keys, const int64_t *d_offsets,
                             size_t num_segs, const hs_plan *plan, void *d_ws, size_t ws_bytes,
                             hs_graph **out) {
    clear_error();
    if (!out) return fail(HS_ERR_INVALID_ARG, "hs_segsort_capture: NULL result");
    hs_plan p;
    hs_status r = plan_from(plan, HS_NETS_6TO8, n_keys, num_segs, &p);
    if (r != HS_OK) return r;
    void *h = nullptr;
    r = segsort_capture(d_keys, n_keys, d_offsets, num_segs, p, d_ws, ws_bytes, &h);
    if (r == HS_OK) *out = static_cast<hs_graph *>(h);
    return r;
}

hs_status hs_graph_launch(hs_graph *g, hs_stream_t stream) {
    clear_error();
    return graph_launch(g, (cudaStream_t)stream);
}

void hs_graph_destroy(hs_graph *g) { graph_destroy(g); }

size_t hs_segsort_autotune_workspace_bytes(size_t n_keys, size_t num_segs) {
    return autotune_workspace_bytes(n_keys, num_segs);
}

hs_status hs_segsort_autotune(int32_t *d_keys, size_t n_keys, const int64_t *d_offsets,
                              size_t num_segs, void *d_ws, size_t ws_bytes, hs_stream_t stream,
                              hs_plan *best, double *best_ms) {
    clear_error();
    return autotune(d_keys, n_keys, d_offsets, num_segs, d_ws, ws_bytes, (cudaStream_t)stream, best,
                    best_ms);
}

size_t hs_sort_autotune_workspace_bytes(size_t n) { return sort_autotune_workspace_bytes(n); }

hs_status hs_sort_autotune(int32_t *d_keys, size_t n, hs_netset s, void *d_ws, size_t ws_bytes,
                           hs_stream_t stream, hs_sort_plan *best, double *best_ms) {
    const ApiRange range("hs_sort_autotune");
    clear_error();
    return sort_autotune(d_keys, n, s, d_ws, ws_bytes, (cudaStream_t)stream, best, best_ms);
}

hs_status hs_segsort_plan_for(size_t n_keys, size_t num_segs, hs_netset s, hs_plan *out) {
    clear_error();
    if (!out) return fail(HS_ERR_INVALID_ARG, "hs_segsort_plan_for: NULL result");
    return plan_from(nullptr, s, n_keys, num_segs, out);
}

hs_status hs_sort_plan_for(const int32_t *d_keys, size_t n, hs_netset s, hs_sort_plan *out) {
    clear_error();
    if (!out) return fail(HS_ERR_INVALID_ARG, "hs_sort_plan_for: NULL result");
    if (!netset_ok(s))
        return fail(HS_ERR_INVALID_ARG, "hs_sort_plan_for: netset is neither a set of sizes 3..8 nor a VarSort configuration");
    if (n > (size_t)INT64_MAX / 16) return fail(HS_ERR_INVALID_ARG, "hs_sort_plan_for: n too large");
    const SortPlan p = merge_plan_for(d_keys, (int64_t)n, leaf_size(s));
    *out = hs_sort_plan{p.shape == 4 ? 288 : 256, p.fanin, {0, 0}};
    return HS_OK;
}

void hs_tune_cache_clear(void) {
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune.clear();
    }
    sort_plan_cache_clear();
}

hs_status hs_tune_cache_save(const char *path) {
    clear_error();
    if (!path) return fail(HS_ERR_INVALID_ARG, "hs_tune_cache_save: NULL path");
    return tune_cache_save(path);
}

hs_status hs_tune_cache_load(const char *path) {
    clear_error();
    if (!path) return fail(HS_ERR_INVALID_ARG, "hs_tune_cache_load: NULL path");
    return tune_cache_load(path);
}

}  // extern "C"
