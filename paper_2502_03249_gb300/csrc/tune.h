// tune.h -- the autotuner: picks a launch configuration per kernel and
// problem shape by timing the candidates, and remembers the choice.
//
// A decision is keyed by the kernel, the lattice extents, the storage
// (precision, compression), the number of right-hand sides and the GPU's name
// (tune_key).  Candidates are timed with CUDA events on the context's stream:
// one warm-up launch, then three launches each preceded by an L2 flush (a
// read of a buffer larger than L2), the median counts.  Choices live in a
// process-wide cache backed by a JSON file, so that later processes on the
// same GPU and shapes skip the timing:
//
//   STAG_TUNE        0: never time (the caller's default candidate);
//                    1 or unset: time what the cache lacks;
//                    force: time every decision once in this process, even
//                    if the file has it (and rewrite the file)
//   STAG_TUNE_CACHE  path of the JSON file; empty: no file (memory only);
//                    unset: $XDG_CACHE_HOME/stag/tune.json or
//                    $HOME/.cache/stag/tune.json
//
// Timing launches the candidates on the caller's buffers, so tune_choice
// must only be called where running the candidate kernel is harmless (its
// outputs are overwritten afterwards) and never while the stream is captured.
#pragma once

#include <functional>
#include <string>
#include <vector>

#include "ctx.h"

namespace stag {

// "kernel|LxxLyxLzxLt|p<prec>|r<recon>|n<nrhs>|<gpu>" (GPU name with every
// character outside [A-Za-z0-9_-] replaced by '_').
std::string tune_key_string(const char* kernel, const int dims[4], int prec, int recon, int nrhs, const char* gpu);
std::string tune_key(stag_ctx ctx, const char* kernel, int prec, int recon, int nrhs);

// *choice: on entry the default candidate (used with STAG_TUNE=0), on return
// the decision.  launch(c) enqueues candidate c on the context's stream.
int tune_choice(stag_ctx ctx, const std::string& key, const std::vector<int>& candidates, int* choice,
                const std::function<int(int)>& launch);

void free_tune_cache(stag_ctx ctx);

}  // namespace stag
