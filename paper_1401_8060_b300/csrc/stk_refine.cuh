// Refinement loop of continuous templates on the device (the follow-up of the
// loudest events, Sec. V).
#pragma once

#include "stk_internal.cuh"

namespace stk {

// Gradient ascent of n continuous templates' interpolated SNR: `steps` Adam steps
// (lr_f in bins, lr_u in units of tau_max) with f3 and tau updated in place and
// projected onto f in [0, n_f - 1], |tau| <= tau_max; hist (optional) gets
// [steps + 1][n] SNRs.  Scratch: refine_scratch_bytes(steps), 16-byte aligned.
// P: threads per template (32, 64, 128; 0 chooses by n).  One launch for all steps.
size_t refine_scratch_bytes(int steps);
cudaError_t launch_refine(const MapDev &m, float *f3, float *tau, uint64_t n, int steps, float lr_f, float lr_u,
                          float tau_max, float *hist, void *scratch, int P, int *err, cudaStream_t st);

// launch_interp with P threads per template (32, 64, 128; 0 chooses by n).
cudaError_t launch_interp_tuned(const MapDev &m, const float *f3, const float *tau, const float *g, uint64_t n,
                                float *snr, float *gf3, float *gtau, bool adjoint, int P, int *err, cudaStream_t st);

// Discrete follow-up: n templates f3 [n][3] (bins), tau [n] (s), in place; alt_f3 /
// alt_tau (optional) continuous alternatives, rounded and polished too; the better
// of start / polished start / polished alternative by the scorer's SNR is kept
// (snr, which optional outputs).  moves: most +-1 bin moves per climb.
cudaError_t launch_polish(const MapDev &m, uint32_t *f3, double *tau, const float *alt_f3, const float *alt_tau,
                          uint64_t n, double tau_max, int moves, double *snr, int *which, int *err, cudaStream_t st);

}  // namespace stk
