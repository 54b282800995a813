// tune.cu -- autotuner implementation (see tune.h): timing with CUDA events
// and L2 flushes, a process-wide cache of decisions, and its JSON file.
#include <errno.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "tune.h"

namespace stag {

namespace {

struct Entry {
    int choice = 0;
    std::vector<int> candidates;
    std::vector<float> ms;
    bool from_file = false;   // loaded, not timed in this process
};

struct Cache {
    std::mutex mu;
    std::map<std::string, Entry> entries;
    bool loaded = false;
    long long timed = 0, hits = 0;
};

Cache& cache()
{
    static Cache c;
    return c;
}

std::string default_path()
{
    const char* e = getenv("STAG_TUNE_CACHE");
    if (e) return e;   // empty: no file
    const char* x = getenv("XDG_CACHE_HOME");
    if (x && *x) return std::string(x) + "/stag/tune.json";
    const char* h = getenv("HOME");
    if (h && *h) return std::string(h) + "/.cache/stag/tune.json";
    return "";
}

int tune_mode()   // 0 never time, 1 time what is missing, 2 force
{
    const char* e = getenv("STAG_TUNE");
    if (!e || !*e) return 1;
    if (strcmp(e, "0") == 0) return 0;
    if (strcmp(e, "force") == 0) return 2;
    return 1;
}

// ------------------------------------------------------------- JSON file
//
// {"format": "stag-tune-1", "entries": {"<key>": {"choice": 3, "candidates":
// [1, 2, 3], "ms": [0.1, 0.2, 0.3]}, ...}}.  The reader takes what it needs:
// each key string of the entries object and the integer after its "choice".

const char* skip_ws(const char* p)
{
    while (*p == ' ' || *p == '\n' || *p == '\r' || *p == '\t') ++p;
    return p;
}

// Parse the file text into out; returns the number of entries, or -1 if the
// text is not a tuning file of this format.
int parse_text(const std::string& text, std::map<std::string, Entry>& out)
{
    const char* s = text.c_str();
    if (!strstr(s, "\"stag-tune-1\"")) return -1;
    const char* p = strstr(s, "\"entries\"");
    if (!p) return -1;
    p = skip_ws(p + 9);
    if (*p != ':') return -1;
    p = skip_ws(p + 1);
    if (*p != '{') return -1;
    ++p;
    int n = 0;
    for (;;) {
        p = skip_ws(p);
        if (*p == '}') break;
        if (*p == ',') {
            ++p;
            continue;
        }
        if (*p != '"') return -1;
        const char* k0 = ++p;
        while (*p && *p != '"') ++p;
        if (!*p) return -1;
        std::string key(k0, p - k0);
        ++p;
        p = skip_ws(p);
        if (*p != ':') return -1;
        p = skip_ws(p + 1);
        if (*p != '{') return -1;
        const char* end = strchr(p, '}');
        if (!end) return -1;
        const char* c = strstr(p, "\"choice\"");
        if (!c || c > end) return -1;
        c = skip_ws(c + 8);
        if (*c != ':') return -1;
        char* after = nullptr;
        const long v = strtol(c + 1, &after, 10);
        if (after == c + 1) return -1;
        Entry e;
        e.choice = (int)v;
        e.from_file = true;
        const char* cl = strstr(p, "\"candidates\"");
        if (cl && cl < end) {
            cl = strchr(cl, '[');
            const char* ce = cl ? strchr(cl, ']') : nullptr;
            for (const char* q = cl ? cl + 1 : nullptr; q && q < ce;) {
                char* a = nullptr;
                const long w = strtol(q, &a, 10);
                if (a == q) break;
                e.candidates.push_back((int)w);
                q = a;
                while (q < ce && (*q == ',' || *q == ' ')) ++q;
            }
        }
        out[key] = e;
        ++n;
        p = end + 1;
    }
    return n;
}

std::string render_text(const std::map<std::string, Entry>& entries)
{
    std::string s = "{\n \"format\": \"stag-tune-1\",\n \"entries\": {";
    bool first = true;
    char buf[64];
    for (const auto& kv : entries) {
        s += first ? "\n  \"" : ",\n  \"";
        first = false;
        s += kv.first;
        snprintf(buf, sizeof(buf), "\": {\"choice\": %d, \"candidates\": [", kv.second.choice);
        s += buf;
        for (size_t i = 0; i < kv.second.candidates.size(); ++i) {
            snprintf(buf, sizeof(buf), i ? ", %d" : "%d", kv.second.candidates[i]);
            s += buf;
        }
        s += "], \"ms\": [";
        for (size_t i = 0; i < kv.second.ms.size(); ++i) {
            snprintf(buf, sizeof(buf), i ? ", %.5g" : "%.5g", (double)kv.second.ms[i]);
            s += buf;
        }
        s += "]}";
    }
    s += "\n }\n}\n";
    return s;
}

int read_file(const std::string& path, std::string& text)
{
    FILE* f = fopen(path.c_str(), "rb");
    if (!f) return -1;
    char buf[4096];
    size_t n;
    while ((n = fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, n);
    fclose(f);
    return 0;
}

void mkdirs(const std::string& path)
{
    for (size_t i = 1; i < path.size(); ++i)
        if (path[i] == '/') mkdir(path.substr(0, i).c_str(), 0755);
}

// Write the file atomically (temporary file, then rename).
int write_file(const std::string& path, const std::string& text)
{
    mkdirs(path);
    const std::string tmp = path + ".tmp" + std::to_string((long)getpid());
    FILE* f = fopen(tmp.c_str(), "wb");
    if (!f) return -1;
    const bool ok = fwrite(text.data(), 1, text.size(), f) == text.size();
    if (fclose(f) != 0 || !ok) {
        remove(tmp.c_str());
        return -1;
    }
    if (rename(tmp.c_str(), path.c_str()) != 0) {
        remove(tmp.c_str());
        return -1;
    }
    return 0;
}

// Load the default file once (caller holds the lock).
void ensure_loaded(Cache& c)
{
    if (c.loaded) return;
    c.loaded = true;
    const std::string path = default_path();
    std::string text;
    if (path.empty() || read_file(path, text) != 0) return;
    std::map<std::string, Entry> m;
    if (parse_text(text, m) >= 0)
        for (auto& kv : m)
            if (!c.entries.count(kv.first)) c.entries[kv.first] = kv.second;
}

// ------------------------------------------------------------- L2 flush

constexpr size_t FLUSH_BYTES = 256u << 20;   // twice the 129 MB L2 of GB300

__global__ void k_l2_flush(const float4* __restrict__ buf, size_t n, float* sink)
{
    float s = 0.f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float4 v = __ldcg(buf + i);
        s += v.x + v.y + v.z + v.w;
    }
    if (s == 12345.f) *sink = s;   // keeps the loads
}

int flush_l2(stag_ctx ctx)
{
    static std::mutex mu;
    static void* bufs[64] = {};
    std::lock_guard<std::mutex> lock(mu);
    const int dev = ctx->device >= 0 && ctx->device < 64 ? ctx->device : 0;
    if (!bufs[dev]) {
        STAG_CUDA_TRY(cudaMalloc(&bufs[dev], FLUSH_BYTES + 256));
        STAG_CUDA_TRY(cudaMemsetAsync(bufs[dev], 0, FLUSH_BYTES + 256, ctx->stream));
    }
    const size_t n = FLUSH_BYTES / sizeof(float4);
    k_l2_flush<<<ctx->sm_count * 4, 256, 0, ctx->stream>>>((const float4*)bufs[dev], n,
                                                          (float*)((char*)bufs[dev] + FLUSH_BYTES));
    STAG_CUDA_TRY(cudaGetLastError());
    return STAG_OK;
}

}  // namespace

std::string tune_key_string(const char* kernel, const int dims[4], int prec, int recon, int nrhs, const char* gpu)
{
    char buf[256];
    snprintf(buf, sizeof(buf), "%s|%dx%dx%dx%d|p%d|r%d|n%d|", kernel, dims[0], dims[1], dims[2], dims[3], prec, recon,
             nrhs);
    std::string s = buf;
    for (const char* q = gpu; q && *q; ++q) {
        const char ch = *q;
        const bool ok = (ch >= 'a' && ch <= 'z') || (ch >= 'A' && ch <= 'Z') || (ch >= '0' && ch <= '9') ||
                        ch == '_' || ch == '-';
        s += ok ? ch : '_';
    }
    for (char& ch : s)
        if (ch == '"' || ch == '\\') ch = '_';
    return s;
}

std::string tune_key(stag_ctx ctx, const char* kernel, int prec, int recon, int nrhs)
{
    cudaDeviceProp prop;
    const char* name = "gpu";
    if (cudaGetDeviceProperties(&prop, ctx->device) == cudaSuccess) name = prop.name;
    return tune_key_string(kernel, ctx->g.L, prec, recon, nrhs, name);
}

int tune_choice(stag_ctx ctx, const std::string& key, const std::vector<int>& cands, int* choice,
                const std::function<int(int)>& launch)
{
    Cache& c = cache();
    const int mode = tune_mode();
    {
        std::lock_guard<std::mutex> lock(c.mu);
        ensure_loaded(c);
        auto it = c.entries.find(key);
        if (it != c.entries.end() && !(mode == 2 && it->second.from_file) &&
            std::find(cands.begin(), cands.end(), it->second.choice) != cands.end()) {
            *choice = it->second.choice;
            ++c.hits;
            return STAG_OK;
        }
        if (mode == 0 || cands.size() <= 1) {
            if (cands.size() == 1) *choice = cands[0];
            Entry e;
            e.choice = *choice;
            e.candidates = cands;
            c.entries[key] = e;
            return STAG_OK;
        }
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    STAG_CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        set_error("autotuner: cudaEventCreate failed");
        return STAG_ECUDA;
    }
    int best = cands.front(), rc = STAG_OK;
    float best_ms = 1e30f;
    std::vector<float> record;
    for (int cand : cands) {
        if ((rc = launch(cand)) != STAG_OK) break;   // warm-up
        float ts[3];
        for (int r = 0; r < 3 && rc == STAG_OK; ++r) {
            if ((rc = flush_l2(ctx)) != STAG_OK) break;
            cudaEventRecord(e0, ctx->stream);
            rc = launch(cand);
            cudaEventRecord(e1, ctx->stream);
            if (rc == STAG_OK &&
                (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ts[r], e0, e1) != cudaSuccess)) {
                set_error("autotuner timing failed");
                rc = STAG_ECUDA;
            }
        }
        if (rc != STAG_OK) break;
        std::sort(ts, ts + 3);
        record.push_back(ts[1]);
        if (ts[1] < best_ms) {
            best_ms = ts[1];
            best = cand;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != STAG_OK) return rc;
    std::string text, path;
    {
        std::lock_guard<std::mutex> lock(c.mu);
        Entry e;
        e.choice = best;
        e.candidates = cands;
        e.ms = record;
        c.entries[key] = e;
        ++c.timed;
        path = default_path();
        if (!path.empty()) text = render_text(c.entries);
    }
    if (!path.empty()) write_file(path, text);   // best effort: a read-only home only loses the cache
    *choice = best;
    return STAG_OK;
}

void free_tune_cache(stag_ctx) {}

}  // namespace stag

using namespace stag;

extern "C" {

int stag_tune_make_key(const char* kernel, const int dims[4], int prec, int recon, int nrhs, const char* gpu,
                       char* out, int len)
{
    if (!kernel || !dims || !gpu || !out || len < 1) {
        set_error("stag_tune_make_key: NULL argument or len < 1");
        return STAG_EINVAL;
    }
    const std::string k = tune_key_string(kernel, dims, prec, recon, nrhs, gpu);
    if ((int)k.size() >= len) {
        set_error("stag_tune_make_key: buffer of %d bytes too small for %zu", len, k.size() + 1);
        return STAG_EINVAL;
    }
    memcpy(out, k.c_str(), k.size() + 1);
    return (int)k.size();
}

int stag_tune_cache_load(const char* path)
{
    const std::string p = path ? path : default_path();
    std::string text;
    if (p.empty() || read_file(p, text) != 0) {
        set_error("stag_tune_cache_load: cannot read '%s'", p.c_str());
        return STAG_EINVAL;
    }
    std::map<std::string, Entry> m;
    const int n = parse_text(text, m);
    if (n < 0) {
        set_error("stag_tune_cache_load: '%s' is not a tuning cache file", p.c_str());
        return STAG_EINVAL;
    }
    Cache& c = cache();
    std::lock_guard<std::mutex> lock(c.mu);
    c.entries = m;
    c.loaded = true;
    return n;
}

int stag_tune_cache_save(const char* path)
{
    const std::string p = path ? path : default_path();
    if (p.empty()) {
        set_error("stag_tune_cache_save: no cache file (STAG_TUNE_CACHE is empty)");
        return STAG_EINVAL;
    }
    std::string text;
    {
        Cache& c = cache();
        std::lock_guard<std::mutex> lock(c.mu);
        text = render_text(c.entries);
    }
    if (write_file(p, text) != 0) {
        set_error("stag_tune_cache_save: cannot write '%s'", p.c_str());
        return STAG_EINVAL;
    }
    return STAG_OK;
}

int stag_tune_cache_lookup(const char* key, int* choice)
{
    if (!key || !choice) {
        set_error("stag_tune_cache_lookup: NULL argument");
        return STAG_EINVAL;
    }
    Cache& c = cache();
    std::lock_guard<std::mutex> lock(c.mu);
    ensure_loaded(c);
    auto it = c.entries.find(key);
    if (it == c.entries.end()) return 0;
    *choice = it->second.choice;
    return 1;
}

int stag_tune_cache_insert(const char* key, int choice)
{
    if (!key || !*key || strchr(key, '"') || strchr(key, '\\')) {
        set_error("stag_tune_cache_insert: key NULL, empty or with quotes");
        return STAG_EINVAL;
    }
    Cache& c = cache();
    std::lock_guard<std::mutex> lock(c.mu);
    Entry e;
    e.choice = choice;
    c.entries[key] = e;
    return STAG_OK;
}

void stag_tune_cache_clear(void)
{
    Cache& c = cache();
    std::lock_guard<std::mutex> lock(c.mu);
    c.entries.clear();
    c.loaded = true;   // and do not reload the default file
    c.timed = c.hits = 0;
}

int stag_tune_stats(long long* timed, long long* from_cache)
{
    Cache& c = cache();
    std::lock_guard<std::mutex> lock(c.mu);
    if (timed) *timed = c.timed;
    if (from_cache) *from_cache = c.hits;
    return STAG_OK;
}

}  // extern "C"
