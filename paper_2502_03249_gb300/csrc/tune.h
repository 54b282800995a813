// tune.h -- a small autotuner: times each candidate launch shape with CUDA
// events on the context's stream (one warm-up launch, then the median of three)
// and caches the fastest per context and key.  STAG_TUNE=0 in the environment
// turns timing off and takes the default candidate instead.
#pragma once

#include <functional>
#include <initializer_list>
#include <vector>

#include "ctx.h"

namespace stag {

// Candidates above the smallest power of two >= limit are skipped.  Must not
// be called while the context's stream is being captured.
int tune_choice(stag_ctx ctx, const char* key, const std::vector<int>& candidates, int* choice,
                const std::function<int(int)>& launch);

void free_tune_cache(stag_ctx ctx);

}  // namespace stag
