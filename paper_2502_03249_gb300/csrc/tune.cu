// tune.cu -- autotuner implementation (see tune.h).
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "tune.h"

namespace stag {

struct TuneCache {
    std::map<std::string, int> best;
    std::map<std::string, std::vector<float>> times;
};

static TuneCache* cache_of(stag_ctx ctx)
{
    if (!ctx->tune) ctx->tune = new TuneCache();
    return (TuneCache*)ctx->tune;
}

int tune_choice(stag_ctx ctx, const char* key, const std::vector<int>& cands, int* choice,
                const std::function<int(int)>& launch)
{
    TuneCache* tc = cache_of(ctx);
    auto it = tc->best.find(key);
    if (it != tc->best.end()) {
        *choice = it->second;
        return STAG_OK;
    }
    const char* env = getenv("STAG_TUNE");
    if (env && strcmp(env, "0") == 0) {
        tc->best[key] = *choice;   // the caller's default
        return STAG_OK;
    }
    cudaEvent_t e0, e1;
    STAG_CUDA_TRY(cudaEventCreate(&e0));
    STAG_CUDA_TRY(cudaEventCreate(&e1));
    int best = cands.front();
    float best_ms = 1e30f;
    std::vector<float> record;
    int rc = STAG_OK;
    for (int c : cands) {
        if ((rc = launch(c)) != STAG_OK) break;
        float ts[3];
        for (int r = 0; r < 3 && rc == STAG_OK; ++r) {
            cudaEventRecord(e0, ctx->stream);
            rc = launch(c);
            cudaEventRecord(e1, ctx->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ts[r], e0, e1) != cudaSuccess) {
                set_error("autotuner timing failed");
                rc = STAG_ECUDA;
            }
        }
        if (rc != STAG_OK) break;
        std::sort(ts, ts + 3);
        record.push_back(ts[1]);
        if (ts[1] < best_ms) {
            best_ms = ts[1];
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != STAG_OK) return rc;
    tc->best[key] = best;
    tc->times[key] = record;
    *choice = best;
    return STAG_OK;
}

void free_tune_cache(stag_ctx ctx)
{
    delete (TuneCache*)ctx->tune;
    ctx->tune = nullptr;
}

}  // namespace stag
