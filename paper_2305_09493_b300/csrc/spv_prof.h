// spv_prof.h -- optional per-kernel CUDA-event timing of library launches.
#pragma once
#include <cuda_runtime.h>

namespace spvprof {
bool enabled();
// returns a token to pass to end(); -1 when profiling is off
int begin(const char *name, cudaStream_t st);
void end(int token, cudaStream_t st);
}  // namespace spvprof

// wraps one kernel launch statement
#define SPV_LAUNCH(name, st, ...)                       \
    do {                                                \
        int _tok = spvprof::begin(name, st);            \
        __VA_ARGS__;                                    \
        spvprof::end(_tok, st);                         \
    } while (0)
