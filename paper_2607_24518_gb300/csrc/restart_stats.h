// Per-restart check quantities of a handle whose k columns hold R restarts
// (column blocks of kb = k / R), k_restart.cu.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace symnmf {

constexpr int kRestartSums = 3;  // sums per restart in launch_restart_stats

// out[3 r] = sum over block r of H .* g, out[3 r + 1] = sum over block r of
// the projected gradient squared (g where H > 0, min(0, g) where H == 0),
// out[3 r + 2] = sum over block r of the accumulator A; H, g and A are
// n x kp row-major over ntiles * 128 rows (rows past n are 0); part holds
// ntiles * 3R doubles of per-tile partials.  FP64, fixed order.
cudaError_t launch_restart_stats(const float *H, const float *g, const float *A, int64_t n, int k,
                                 int kp, int R, double *part, double *out, cudaStream_t s);

}  // namespace symnmf
