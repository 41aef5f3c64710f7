// Refinement loop of continuous templates on the device (the follow-up of the
// loudest events, Sec. V).
#pragma once

#include "stk_internal.cuh"

namespace stk {

// Gradient ascent of n continuous templates' interpolated SNR: `steps` Adam steps
// (lr_f in bins, lr_u in units of tau_max) with f3 and tau updated in place and
// projected onto f in [0, n_f - 1], |tau| <= tau_max; hist (optional) gets
// [steps + 1][n] SNRs.  Scratch: refine_scratch_bytes(n), 16-byte aligned.
// P: threads per template (32, 64, 128; 0 chooses by n).
size_t refine_scratch_bytes(uint64_t n);
cudaError_t launch_refine(const MapDev &m, float *f3, float *tau, uint64_t n, int steps, float lr_f, float lr_u,
                          float tau_max, float *hist, void *scratch, int P, cudaStream_t st);

// launch_interp with P threads per template (32, 64, 128; 0 chooses by n).
cudaError_t launch_interp_tuned(const MapDev &m, const float *f3, const float *tau, const float *g, uint64_t n,
                                float *snr, float *gf3, float *gtau, bool adjoint, int P, cudaStream_t st);

}  // namespace stk
