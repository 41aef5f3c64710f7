// Library-private definitions of the opaque handles and error helpers, shared
// by the C-ABI translation units.
#pragma once

#include <string>

#include "stk_internal.cuh"

using stk::MapDev;
using stk::ScorePlan;
using stk::TrackSet;
using stk::Tuning;


struct stk_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    size_t smem_optin = 0;
    bool have_tracks = false;
    TrackSet ts{};
    int *d_err = nullptr;          // device error/flag word
    float *snr_buf = nullptr;      // scratch: one FP32 SNR per template
    size_t snr_cap = 0;
    void *sel_buf = nullptr;       // scratch: selection state
    size_t sel_cap = 0;
    stk_hit *hits_dev = nullptr;   // STK_MAX_K records
    uint32_t *small_dev = nullptr; // track_params: f[3], t[3], tau, bins
    size_t small_cap = 0;
    double *tauq_dev = nullptr;    // delay prior quantiles
    size_t tauq_cap = 0;
    void *stage_y = nullptr;       // host-pointer map uploads: y and sigma staged here
    size_t stage_y_cap = 0;
    void *stage_s = nullptr;
    size_t stage_s_cap = 0;
    void *order_buf = nullptr;     // coherent-order pre-pass of the slab kernel
    size_t order_cap = 0;
    void *refine_buf = nullptr;    // refinement: Adam moments and delay coordinate
    size_t refine_cap = 0;
    int interp_threads = 0;        // continuous templates: threads per template (0: by count)
    Tuning tune{};
    ScorePlan plan{};
    bool profiling = false;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // start, scoring done, selection done, order done
    cudaEvent_t stream_mark = nullptr;  // stk_score_noalloc: marks the context stream's work for other streams
    bool timed = false;
    int last_launches = 0;
    std::string err;
};

struct stk_map {
    stk_ctx *ctx = nullptr;
    MapDev dev{};
    void *rec_buf = nullptr;
    void *w_buf = nullptr;
    size_t rec_bytes = 0;          // bytes of rec_buf and w_buf in use (a debug build's canary follows)
    size_t w_bytes = 0;
    unsigned flags = 0;
};

// Record a formatted message on the context (or the thread's creation message
// when c is NULL) and return code.
int set_err(stk_ctx *c, int code, const char *fmt, ...);

// Read and clear the device error word (synchronises the stream).
int read_err_flags(stk_ctx *c, int *flags);
// Map error bits to a status code (with message).
int flags_to_status(stk_ctx *c, int flags);
// Debug build: check canaries and out-of-range gathers after a call (release: STK_OK).
int debug_verify(stk_ctx *c, const stk_map *m);

#define CUDA_TRY(ctx, call)                                                                                         \
    do {                                                                                                           \
        cudaError_t e_ = (call);                                                                                   \
        if (e_ != cudaSuccess)                                                                                     \
            return set_err((ctx), e_ == cudaErrorMemoryAllocation ? STK_ENOMEM : STK_ECUDA, "%s: %s (%s:%d)", #call, \
                           cudaGetErrorString(e_), __FILE__, __LINE__);                                            \
    } while (0)

