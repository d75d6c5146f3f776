// Per-restart check quantities of a handle whose k columns hold R restarts
// (column blocks of kb = k / R), k_restart.cu.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace symnmf {

// out[2 r] = sum over block r of H .* g, out[2 r + 1] = sum over block r of
// the projected gradient squared (g where H > 0, min(0, g) where H == 0);
// H and g are n x kp row-major over ntiles * 128 rows (rows past n are 0);
// part holds ntiles * 2R doubles of per-tile partials.  FP64, fixed order.
cudaError_t launch_restart_stats(const float *H, const float *g, int64_t n, int k, int kp, int R,
                                 double *part, double *out, cudaStream_t s);

}  // namespace symnmf
