// C ABI of the scorer: contexts, map packing, argument checks and launches.
// The statistic and template definitions are those of Eq. 7 and Sec. III of
// the paper; see stk.h for the contract of each call.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include <cuda_fp16.h>

#include "stk_internal.cuh"
#include "stk_objects.cuh"
#include "stk_refine.cuh"

using namespace stk;

static thread_local std::string g_create_err;

int set_err(stk_ctx *c, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    else g_create_err = buf;
    return code;
}

int read_err_flags(stk_ctx *c, int *flags)
{
    int h = 0;
    CUDA_TRY(c, cudaMemcpyAsync(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
    *flags = h;
    return STK_OK;
}

int flags_to_status(stk_ctx *c, int f)
{
    if (f & ERR_BOUNDS)
        return set_err(c, STK_EBOUNDS, "debug build: a pixel gather outside its template's bins or the map");
    if (f & ERR_TIMEOUT) return set_err(c, STK_ETIMEOUT, "a bounded in-kernel wait for a map slab gave up");
    if (f & ERR_CANCELED) return set_err(c, STK_ECANCELED, "batch cancelled through stk_batch_cancel");
    if (f & ERR_BADTRACK) return set_err(c, STK_EINVAL, "explicit template with a control bin outside [0, n_f)");
    if (f & ERR_BADINPUT)
        return set_err(c, STK_EINVAL, "stk_update_map data: y non-finite at a pixel that is not notched, or sigma "
                                      "<= 0 or NaN");
    if (f & ERR_FP16_RANGE) return set_err(c, STK_EINVAL, "stk_update_map data: |y| / sigma exceeds 65504 (FP16)");
    return STK_OK;
}

namespace {

// Pack y, sigma into polar records z = |z| e^{i arg} with z = y sigma^-2
// (weighted) or y / sigma (paper form), and the weights.  FP32 arithmetic (|z|
// to about 2 ulp; the angle, in radians in [-pi, pi], to about 2 ulp).
__global__ void pack_kernel(const float2 *__restrict__ y, const float *__restrict__ sigma, int per_freq, int n_t,
                            int n_f, int ldr, int ldw, int paper, uint2 *__restrict__ rec, float *__restrict__ wout,
                            int *err)
{
    const float s0 = sigma[0];
    int flags = 0;
    const uint64_t total = (uint64_t)n_t * ldr;
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total;
         p += (uint64_t)gridDim.x * blockDim.x) {
        // row and column: a 32-bit division when the map has fewer than 2^32 records
        const int t = total <= 0xffffffffull ? (int)((uint32_t)p / (uint32_t)ldr) : (int)(p / ldr);
        const int k = (int)(p - (uint64_t)t * ldr);
        if (k >= n_f) {
            rec[p] = make_uint2(0u, 0u);
            continue;
        }
        const size_t q = (size_t)t * n_f + k;
        const float2 v = y[q];
        const float s = per_freq ? sigma[k] : sigma[q];
        if (s != s0) flags |= FLAG_SIGMA_VARIES;
        if (isinf(s) && s > 0.f) {  // notched pixel (sigma = +inf): no data, whatever y holds
            rec[p] = make_uint2(0u, 0u);
            if (wout) {
                const float w = paper ? 1.f : 0.f;
                if (!per_freq) wout[(size_t)t * ldw + k] = w;
                else if (t == 0) wout[k] = w;
            }
            continue;
        }
        if (!isfinite(v.x) || !isfinite(v.y) || !(s > 0.f) || !isfinite(s)) flags |= ERR_BADINPUT;
        const float w = paper ? 1.f : 1.f / (s * s);
        const float h = hypotf(v.x, v.y);
        const float mag = paper ? h / s : h * w;
        rec[p] = make_uint2(__float_as_uint(mag), __float_as_uint(atan2f(v.y, v.x)));
        if (wout) {
            if (!per_freq) wout[(size_t)t * ldw + k] = w;
            else if (t == 0) wout[k] = w;
        }
    }
    if (flags) atomicOr(err, flags);
}

// FP16 storage: record = FP16(|y| / sigma) << 16 | (Q0.16 arg y); weights r = 1/sigma.
__global__ void pack_fp16_kernel(const float2 *__restrict__ y, const float *__restrict__ sigma, int per_freq, int n_t,
                                 int n_f, int ldr, int ldw, uint32_t *__restrict__ rec, float *__restrict__ rout,
                                 int *err)
{
    const float s0 = sigma[0];
    int flags = 0;
    const uint64_t total = (uint64_t)n_t * ldr;
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total;
         p += (uint64_t)gridDim.x * blockDim.x) {
        // row and column: a 32-bit division when the map has fewer than 2^32 records
        const int t = total <= 0xffffffffull ? (int)((uint32_t)p / (uint32_t)ldr) : (int)(p / ldr);
        const int k = (int)(p - (uint64_t)t * ldr);
        if (k >= n_f) {
            rec[p] = 0u;
            continue;
        }
        const size_t q = (size_t)t * n_f + k;
        const float2 v = y[q];
        const float s = per_freq ? sigma[k] : sigma[q];
        if (s != s0) flags |= FLAG_SIGMA_VARIES;
        if (isinf(s) && s > 0.f) {  // notched pixel (sigma = +inf): no data, whatever y holds
            rec[p] = 0u;
            if (rout) {
                if (!per_freq) rout[(size_t)t * ldw + k] = 0.f;
                else if (t == 0) rout[k] = 0.f;
            }
            continue;
        }
        if (!isfinite(v.x) || !isfinite(v.y) || !(s > 0.f) || !isfinite(s)) flags |= ERR_BADINPUT;
        const float h = hypotf(v.x, v.y) / s;
        if (!(h <= 65504.f)) flags |= ERR_FP16_RANGE;
        const float turns = atan2f(v.y, v.x) * 0.159154943091895336f;  // [-1/2, 1/2]
        const uint32_t a16 = (uint32_t)llrintf(turns * 65536.f) & 0xffffu;
        const unsigned short hb = __half_as_ushort(__float2half_rn(h));
        rec[p] = ((uint32_t)hb << 16) | a16;
        if (rout) {
            const float r = 1.f / s;
            if (!per_freq) rout[(size_t)t * ldw + k] = r;
            else if (t == 0) rout[k] = r;
        }
    }
    if (flags) atomicOr(err, flags);
}

// floor(N / d) == umulhi(N, magic) >> shift for every N <= n_max:
// magic = ceil(2^(32+s) / d) < 2^32 and (magic d - 2^(32+s)) n_max < 2^(32+s).
bool find_magic(uint64_t d, uint64_t n_max, uint32_t &magic, int &shift)
{
    if (n_max >= (1ull << 32) || d == 0) return false;
    for (int s = 0; s < 32; ++s) {
        const unsigned __int128 p2 = (unsigned __int128)1 << (32 + s);
        const unsigned __int128 m = (p2 + d - 1) / d;
        if (m >= ((unsigned __int128)1 << 32)) continue;
        const unsigned __int128 e = m * d - p2;
        if (e * n_max < p2) {
            magic = (uint32_t)m;
            shift = s;
            return true;
        }
    }
    return false;
}

// Debug build: every buffer the library allocates ends in kCanaryBytes of
// kCanaryByte, checked after each call (debug_verify); a write past a buffer's
// end changes them.  Release build: no canaries.
constexpr size_t kCanaryBytes = kDebugBounds ? 256 : 0;
constexpr unsigned char kCanaryByte = 0xA5;

cudaError_t canary_set(void *buf, size_t at, cudaStream_t st)
{
    return kCanaryBytes ? cudaMemsetAsync(static_cast<char *>(buf) + at, kCanaryByte, kCanaryBytes, st)
                        : cudaSuccess;
}

int ensure(stk_ctx *c, void **buf, size_t *cap, size_t need)
{
    if (*cap >= need && *buf) return STK_OK;
    if (*buf) {
        cudaStreamSynchronize(c->stream);
        cudaFree(*buf);
        *buf = nullptr;
        *cap = 0;
    }
    cudaError_t e = cudaMalloc(buf, need + kCanaryBytes);
    if (e != cudaSuccess) {
        *buf = nullptr;
        return set_err(c, STK_ENOMEM, "cudaMalloc(%zu bytes): %s", need, cudaGetErrorString(e));
    }
    *cap = need;
    if ((e = canary_set(*buf, need, c->stream)) != cudaSuccess)
        return set_err(c, STK_ECUDA, "canary: %s", cudaGetErrorString(e));
    return STK_OK;
}



int check_general(stk_ctx *c, const stk_map *m)
{
    if (m->dev.n_t > 4096 || m->dev.n_f > 8192)
        return set_err(c, STK_EINVAL, "general templates need n_t <= 4096 and n_f <= 8192 (map is %d x %d)",
                       m->dev.n_t, m->dev.n_f);
    if (c->ts.t_min > m->dev.n_t - 1)
        return set_err(c, STK_EINVAL, "t_min = %d exceeds the map's n_t - 1 = %d", c->ts.t_min, m->dev.n_t - 1);
    return STK_OK;
}

int check_ready(stk_ctx *c, const stk_map *m)
{
    if (!m || m->ctx != c) return set_err(c, STK_EINVAL, "map is NULL or belongs to another context");
    if (!c->have_tracks) return set_err(c, STK_ESTATE, "stk_set_tracks has not been called");
    if (c->ts.general) return check_general(c, m);
    return STK_OK;
}

}  // namespace

// Debug build, after a call: wait, then check every canary of the context (and
// of map m) and the out-of-range gather flag.  Release build: nothing.
int debug_verify(stk_ctx *c, const stk_map *m)
{
#ifndef STK_DEBUG_BOUNDS
    (void)c;
    (void)m;
    return STK_OK;
#else
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    struct Canary {
        const void *buf;
        size_t at;
        const char *what;
    };
    const Canary cs[] = {{m ? m->rec_buf : nullptr, m ? m->rec_bytes : 0, "map records"},
                         {m ? m->w_buf : nullptr, m ? m->w_bytes : 0, "map weights"},
                         {c->snr_buf, c->snr_cap, "SNR scratch"},
                         {c->sel_buf, c->sel_cap, "selection scratch"},
                         {c->order_buf, c->order_cap, "order scratch"},
                         {c->small_dev, c->small_cap, "parameter scratch"},
                         {c->refine_buf, c->refine_cap, "refinement scratch"},
                         {c->hits_dev, sizeof(stk_hit) * STK_MAX_K, "hit records"}};
    unsigned char h[kCanaryBytes];
    for (const Canary &k : cs) {
        if (!k.buf) continue;
        CUDA_TRY(c, cudaMemcpy(h, static_cast<const char *>(k.buf) + k.at, kCanaryBytes, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < kCanaryBytes; ++i)
            if (h[i] != kCanaryByte)
                return set_err(c, STK_EBOUNDS, "debug build: canary after the %s damaged at byte %zu", k.what, i);
    }
    int fl = 0;
    CUDA_TRY(c, cudaMemcpy(&fl, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (fl & ERR_BOUNDS) {
        const int rest = fl & ~ERR_BOUNDS;   // other deferred errors stay for the next stk_sync
        CUDA_TRY(c, cudaMemcpy(c->d_err, &rest, sizeof(int), cudaMemcpyHostToDevice));
        return flags_to_status(c, ERR_BOUNDS);
    }
    return STK_OK;
#endif
}

extern "C" {

int stk_version(void) { return 100; }

int stk_build_flags(void) { return kDebugBounds ? 1 : 0; }

const char *stk_last_error(const stk_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_err.c_str(); }

int stk_create(stk_ctx **out, int device, void *cuda_stream)
{
    if (!out) return set_err(nullptr, STK_EINVAL, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return set_err(nullptr, STK_ECUDA, "cudaGetDeviceCount: %s", cudaGetErrorString(e));
    if (device < 0 || device >= ndev) return set_err(nullptr, STK_EINVAL, "device %d not in [0, %d)", device, ndev);
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return set_err(nullptr, STK_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    stk_ctx *c = new stk_ctx();
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
    c->num_sms = v;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    c->smem_optin = (size_t)v;
    if (cudaMalloc(&c->d_err, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&c->hits_dev, sizeof(stk_hit) * STK_MAX_K + kCanaryBytes) != cudaSuccess ||
        canary_set(c->hits_dev, sizeof(stk_hit) * STK_MAX_K, c->stream) != cudaSuccess) {
        cudaFree(c->d_err);
        delete c;
        return set_err(nullptr, STK_ENOMEM, "context allocation failed");
    }
    cudaMemset(c->d_err, 0, sizeof(int));
    for (auto &ev : c->ev) cudaEventCreate(&ev);
    cudaEventCreateWithFlags(&c->stream_mark, cudaEventDisableTiming);
    // the order's key table (module memory of this device; every context writes the
    // same values, and the synchronisation below completes them before any use)
    if (order_build_tables(c->stream) != cudaSuccess) {
        cudaFree(c->d_err);
        cudaFree(c->hits_dev);
        delete c;
        return set_err(nullptr, STK_ECUDA, "order table build failed");
    }
    cudaDeviceSynchronize();
    *out = c;
    return STK_OK;
}

void stk_destroy(stk_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    cudaFree(c->d_err);
    cudaFree(c->snr_buf);
    cudaFree(c->sel_buf);
    cudaFree(c->hits_dev);
    cudaFree(c->small_dev);
    cudaFree(c->tauq_dev);
    cudaFree(c->stage_y);
    cudaFree(c->stage_s);
    cudaFree(c->order_buf);
    cudaFree(c->refine_buf);
    if (c->stream_mark) cudaEventDestroy(c->stream_mark);
    for (auto &ev : c->ev)
        if (ev) cudaEventDestroy(ev);
    delete c;
}

int stk_set_stream(stk_ctx *c, void *s)
{
    if (!c) return STK_EINVAL;
    c->stream = (cudaStream_t)s;
    return STK_OK;
}

int stk_set_option(stk_ctx *c, int option, int64_t value)
{
    if (!c) return STK_EINVAL;
    switch (option) {
    case STK_OPT_KERNEL:
        if (value < 0 || value > 2) return set_err(c, STK_EINVAL, "kernel option must be 0, 1 or 2");
        c->tune.kernel = (int)value;
        return STK_OK;
    case STK_OPT_THREADS:
        if (value < 0 || value > 1024) return set_err(c, STK_EINVAL, "threads must be in [0, 1024]");
        c->tune.threads = (int)value;
        return STK_OK;
    case STK_OPT_MAX_R:
        if (value < 1 || value > 12) return set_err(c, STK_EINVAL, "templates per thread must be in [1, 12]");
        c->tune.max_R = (int)value;
        return STK_OK;
    case STK_OPT_STAGES:
        if (value < 2 || value > 4) return set_err(c, STK_EINVAL, "stages must be in [2, 4]");
        c->tune.nstage = (int)value;
        return STK_OK;
    case STK_OPT_SMEM_KB:
        if (value < 0 || value > 1024) return set_err(c, STK_EINVAL, "shared-memory budget out of range");
        c->tune.smem_kb = (int)value;
        return STK_OK;
    case STK_OPT_WAIT_MS:
        if (value < 0 || value > 60000) return set_err(c, STK_EINVAL, "wait limit must be in [0, 60000] ms");
        c->tune.wait_ms = (int)value;
        return STK_OK;
    case STK_OPT_ORDER:
        if (value < 0 || value > 1) return set_err(c, STK_EINVAL, "order option must be 0 or 1");
        c->tune.order = (int)value;
        return STK_OK;
    case STK_OPT_WITHHOLD_SLAB:
        if (value < -1 || value > (1 << 30)) return set_err(c, STK_EINVAL, "slab index out of range");
        c->tune.withhold_slab = (int)value;
        return STK_OK;
    case STK_OPT_SELECT_SAMPLE:
        if (value < 0 || value > 49152) return set_err(c, STK_EINVAL, "selection sample must be in [0, 49152]");
        c->tune.select_sample = (int)value;
        return STK_OK;
    case STK_OPT_INTERP_THREADS:
        if (value != 0 && value != 32 && value != 64 && value != 128)
            return set_err(c, STK_EINVAL, "threads per continuous template must be 0, 32, 64 or 128");
        c->interp_threads = (int)value;
        return STK_OK;
    default: return set_err(c, STK_EINVAL, "unknown option %d", option);
    }
}

int stk_last_plan(const stk_ctx *c, int64_t out[9])
{
    if (!c || !out) return STK_EINVAL;
    const ScorePlan &p = c->plan;
    out[0] = p.kernel; out[1] = p.R; out[2] = p.threads; out[3] = p.grid;
    out[4] = p.S; out[5] = p.nstage; out[6] = (int64_t)p.nbatches; out[7] = (int64_t)p.smem;
    out[8] = p.order;
    return STK_OK;
}

// Copy (host pointers: through the context's staging buffers) and pack y, sigma
// into the map's buffers; set the weighting mode and normalisation.  Synchronises,
// unless `deferred`: then the map keeps its weighting mode (per-pixel or
// per-frequency weights, or the paper form, which hold for any sigma), nothing
// waits, and invalid data is reported by the next reader of the deferred errors.
static int pack_into(stk_ctx *c, stk_map *m, const void *y_c64, const float *sigma, unsigned flags,
                     bool deferred = false)
{
    MapDev &d = m->dev;
    const int n_t = d.n_t, n_f = d.n_f;
    const bool host = flags & STK_HOST_PTR, per_freq = flags & STK_SIGMA_PER_FREQ, paper = flags & STK_NORM_PAPER;
    const bool fp16 = flags & STK_FP16;
    const size_t npx = (size_t)n_t * n_f;
    const size_t ybytes = npx * 8, sbytes = (per_freq ? (size_t)n_f : npx) * 4;
    const float2 *ysrc = (const float2 *)y_c64;
    const float *ssrc = sigma;
    if (host) {
        int rc = ensure(c, &c->stage_y, &c->stage_y_cap, ybytes);
        if (rc) return rc;
        rc = ensure(c, &c->stage_s, &c->stage_s_cap, sbytes);
        if (rc) return rc;
        CUDA_TRY(c, cudaMemcpyAsync(c->stage_y, y_c64, ybytes, cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(c, cudaMemcpyAsync(c->stage_s, sigma, sbytes, cudaMemcpyHostToDevice, c->stream));
        ysrc = (const float2 *)c->stage_y;
        ssrc = (const float *)c->stage_s;
    }
    const size_t wbytes = per_freq ? (size_t)d.ldw * 4 : (size_t)n_t * d.ldw * 4;
    CUDA_TRY(c, cudaMemsetAsync(m->w_buf, 0, wbytes, c->stream));
    if (!deferred) CUDA_TRY(c, cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
    const uint64_t total = (uint64_t)n_t * d.ldr;
    const int blocks = (int)std::min<uint64_t>((total + 255) / 256, (uint64_t)c->num_sms * 8);
    if (fp16)
        pack_fp16_kernel<<<blocks, 256, 0, c->stream>>>(ysrc, ssrc, per_freq ? 1 : 0, n_t, n_f, d.ldr, d.ldw,
                                                         (uint32_t *)m->rec_buf, (float *)m->w_buf, c->d_err);
    else
        pack_kernel<<<blocks, 256, 0, c->stream>>>(ysrc, ssrc, per_freq ? 1 : 0, n_t, n_f, d.ldr, d.ldw, d.paper,
                                                    (uint2 *)m->rec_buf, (float *)m->w_buf, c->d_err);
    CUDA_TRY(c, cudaGetLastError());
    if (deferred) return STK_OK;
    int fl = 0;
    int rc = read_err_flags(c, &fl);
    if (rc) return rc;
    if (fl & ERR_BADINPUT)
        return set_err(c, STK_EINVAL, "y has a non-finite value at a pixel that is not notched, or sigma is <= 0 or NaN");
    if (fl & ERR_FP16_RANGE) return set_err(c, STK_EINVAL, "FP16 storage: |y| / sigma exceeds 65504");
    if (paper) {
        d.wmode = WMODE_CONST;
        d.w_const = 1.0f;
    } else if (!(fl & FLAG_SIGMA_VARIES)) {
        d.wmode = WMODE_CONST;
        float w0 = 0.f;
        CUDA_TRY(c, cudaMemcpy(&w0, m->w_buf, sizeof(float), cudaMemcpyDeviceToHost));
        d.w_const = w0;
    } else {
        d.wmode = per_freq ? WMODE_FREQ : WMODE_PIXEL;
    }
    // constant weight: FP32 records hold |y| w0 (SNR = S / sqrt(n_t w0)); FP16 records hold
    // |y| / sigma0 (SNR = S r0 / sqrt(n_t r0^2) = S / sqrt(n_t)); paper form: S / n_t
    if (paper) d.norm = 1.0 / (double)n_t;
    else if (d.wmode == WMODE_CONST) d.norm = fp16 ? 1.0 / std::sqrt((double)n_t)
                                       : (d.w_const > 0.f ? 1.0 / std::sqrt((double)n_t * (double)d.w_const)
                                                           : 0.0);   // every pixel notched: SNR 0
    else d.norm = 0.0;
    d.norm_f = (float)d.norm;
    d.rec = m->rec_buf;
    d.w = d.wmode == WMODE_CONST ? nullptr : (const float *)m->w_buf;
    return STK_OK;
}

int stk_load_map(stk_ctx *c, const void *y_c64, const float *sigma, int n_t, int n_f, double f_min_hz,
                 double df_hz, unsigned flags, stk_map **out)
{
    if (!c) return STK_EINVAL;
    if (!out) return set_err(c, STK_EINVAL, "out is NULL");
    *out = nullptr;
    if (!y_c64 || !sigma) return set_err(c, STK_EINVAL, "y or sigma is NULL");
    if (n_t < 2) return set_err(c, STK_EINVAL, "n_t = %d: a template needs at least 2 columns", n_t);
    if (n_f < 1) return set_err(c, STK_EINVAL, "n_f = %d must be >= 1", n_f);
    if ((uint64_t)n_t * (uint64_t)n_f > (1ull << 34)) return set_err(c, STK_EINVAL, "map too large");
    {
        const unsigned __int128 M = (unsigned __int128)(n_t - 1);
        if (M * M * (2 * (unsigned __int128)n_f) >= ((unsigned __int128)1 << 62))
            return set_err(c, STK_EINVAL, "map shape %d x %d too large for exact 64-bit rasterisation", n_t, n_f);
    }
    if (!std::isfinite(f_min_hz) || !std::isfinite(df_hz) || !(df_hz > 0))
        return set_err(c, STK_EINVAL, "f_min must be finite and df finite and > 0");
    if (flags & ~(STK_HOST_PTR | STK_SIGMA_PER_FREQ | STK_NORM_PAPER | STK_FP16))
        return set_err(c, STK_EINVAL, "unknown flags 0x%x", flags);
    CUDA_TRY(c, cudaSetDevice(c->device));
    const bool per_freq = flags & STK_SIGMA_PER_FREQ, paper = flags & STK_NORM_PAPER;
    const bool fp16 = flags & STK_FP16;

    stk_map *m = new stk_map();
    m->ctx = c;
    m->flags = flags & ~STK_HOST_PTR;
    MapDev &d = m->dev;
    d.n_t = n_t;
    d.n_f = n_f;
    d.prec = fp16 ? PREC_FP16 : PREC_FP32;
    d.ldr = fp16 ? (n_f + 3) / 4 * 4 : (n_f + 1) / 2 * 2;
    d.ldw = (n_f + 3) / 4 * 4;
    d.paper = paper ? 1 : 0;
    d.f_min = f_min_hz;
    d.df = df_hz;
    d.M = (uint32_t)(n_t - 1);
    d.d = 2ull * d.M * d.M;
    const uint64_t n_max = (uint64_t)d.M * d.M * (2ull * (uint64_t)n_f - 1);
    d.fast32 = find_magic(d.d, n_max, d.magic, d.shift) ? 1 : 0;

    cudaError_t e;
    const size_t recbytes = (size_t)n_t * d.ldr * (fp16 ? 4 : 8);
    const size_t wbytes = per_freq ? (size_t)d.ldw * 4 : (size_t)n_t * d.ldw * 4;
    if ((e = cudaMalloc(&m->rec_buf, recbytes + kCanaryBytes)) != cudaSuccess ||
        (e = cudaMalloc(&m->w_buf, wbytes + kCanaryBytes)) != cudaSuccess) {
        cudaFree(m->rec_buf);
        delete m;
        return set_err(c, STK_ENOMEM, "map allocation (%zu bytes): %s", recbytes + wbytes, cudaGetErrorString(e));
    }
    m->rec_bytes = recbytes;
    m->w_bytes = wbytes;
    if ((e = canary_set(m->rec_buf, recbytes, c->stream)) != cudaSuccess ||
        (e = canary_set(m->w_buf, wbytes, c->stream)) != cudaSuccess) {
        cudaFree(m->rec_buf);
        cudaFree(m->w_buf);
        delete m;
        return set_err(c, STK_ECUDA, "canary: %s", cudaGetErrorString(e));
    }
    int rc = pack_into(c, m, y_c64, sigma, flags);
    if (rc) {
        cudaStreamSynchronize(c->stream);
        cudaFree(m->rec_buf);
        cudaFree(m->w_buf);
        delete m;
        return rc;
    }
    *out = m;
    return STK_OK;
}

int stk_update_map(stk_ctx *c, stk_map *m, const void *y_c64, const float *sigma, unsigned flags)
{
    if (!c) return STK_EINVAL;
    if (!m || m->ctx != c) return set_err(c, STK_EINVAL, "map is NULL or belongs to another context");
    if (!y_c64 || !sigma) return set_err(c, STK_EINVAL, "y or sigma is NULL");
    if (flags & ~(STK_HOST_PTR | STK_SIGMA_PER_FREQ | STK_NORM_PAPER | STK_FP16))
        return set_err(c, STK_EINVAL, "unknown flags 0x%x", flags);
    if ((flags & ~STK_HOST_PTR) != m->flags)
        return set_err(c, STK_EINVAL, "flags 0x%x do not match the map's (0x%x, host flag aside)", flags, m->flags);
    CUDA_TRY(c, cudaSetDevice(c->device));
    // varying weights or the paper form stay valid for any new sigma: no wait
    const bool deferred = m->dev.paper || m->dev.wmode != WMODE_CONST;
    return pack_into(c, m, y_c64, sigma, flags, deferred);
}

void stk_free_map(stk_map *m)
{
    if (!m) return;
    if (m->ctx) {
        cudaSetDevice(m->ctx->device);
        cudaStreamSynchronize(m->ctx->stream);
    }
    cudaFree(m->rec_buf);
    cudaFree(m->w_buf);
    delete m;
}

int stk_map_info(const stk_map *m, int *n_t, int *n_f, unsigned *flags)
{
    if (!m) return STK_EINVAL;
    if (n_t) *n_t = m->dev.n_t;
    if (n_f) *n_f = m->dev.n_f;
    if (flags) *flags = m->flags;
    return STK_OK;
}

int stk_set_tracks(stk_ctx *c, uint64_t n_tracks, uint64_t seed, uint64_t counter_offset, double tau_max_s)
{
    if (!c) return STK_EINVAL;
    if (n_tracks < 1) return set_err(c, STK_EINVAL, "n_tracks must be >= 1");
    if (n_tracks > 0xffffffffull) return set_err(c, STK_EINVAL, "n_tracks must be < 2^32 per call; split the range");
    if (!std::isfinite(tau_max_s) || tau_max_s < 0) return set_err(c, STK_EINVAL, "tau_max must be finite and >= 0");
    c->ts.n = n_tracks;
    c->ts.seed = seed;
    c->ts.offset = counter_offset;
    c->ts.tau_max = tau_max_s;
    c->have_tracks = true;
    return STK_OK;
}

static int score_into(stk_ctx *c, const stk_map *m, float *out)
{
    CUDA_TRY(c, cudaSetDevice(c->device));
    void *order = nullptr;
    if (score_wants_order(m->dev, c->ts, c->tune)) {
        int rc = ensure(c, &c->order_buf, &c->order_cap, order_scratch_bytes(c->ts.n, m->dev.n_f, m->dev.n_t,
                                                                           c->ts.general != 0, c->num_sms));
        if (rc) return rc;
        order = c->order_buf;
    }
    if (c->profiling) CUDA_TRY(c, cudaEventRecord(c->ev[0], c->stream));
    cudaError_t e = launch_score_generated(m->dev, c->ts, out, c->d_err, c->tune, c->num_sms, c->smem_optin,
                                           c->stream, &c->plan, order, c->profiling ? c->ev[3] : nullptr);
    if (e != cudaSuccess) return set_err(c, STK_ECUDA, "scoring kernel launch: %s", cudaGetErrorString(e));
    if (c->profiling) CUDA_TRY(c, cudaEventRecord(c->ev[1], c->stream));
    return STK_OK;
}

int stk_score_all(stk_ctx *c, const stk_map *m, double *out_snr_dev)
{
    if (!c) return STK_EINVAL;
    int rc = check_ready(c, m);
    if (rc) return rc;
    if (!out_snr_dev) return set_err(c, STK_EINVAL, "out_snr_dev is NULL");
    rc = ensure(c, (void **)&c->snr_buf, &c->snr_cap, c->ts.n * sizeof(float));
    if (rc) return rc;
    rc = score_into(c, m, c->snr_buf);
    if (rc) return rc;
    cudaError_t e = launch_widen(c->snr_buf, out_snr_dev, c->ts.n, c->stream);
    if (e != cudaSuccess) return set_err(c, STK_ECUDA, "widening launch: %s", cudaGetErrorString(e));
    c->timed = c->profiling;
    c->last_launches = 2 + (c->plan.order ? c->plan.order_launches : 0);
    if (c->profiling) CUDA_TRY(c, cudaEventRecord(c->ev[2], c->stream));
    return debug_verify(c, m);
}

int stk_score(stk_ctx *c, const stk_map *m, int k, stk_hit *out, unsigned flags)
{
    if (!c) return STK_EINVAL;
    int rc = check_ready(c, m);
    if (rc) return rc;
    if (!out) return set_err(c, STK_EINVAL, "out_topk is NULL");
    if (flags & ~STK_OUT_HOST) return set_err(c, STK_EINVAL, "unknown flags 0x%x", flags);
    if (k < 1 || k > STK_MAX_K || (uint64_t)k > c->ts.n)
        return set_err(c, STK_EINVAL, "k = %d must be in [1, min(%d, n_tracks))", k, STK_MAX_K);
    rc = ensure(c, (void **)&c->snr_buf, &c->snr_cap, c->ts.n * sizeof(float));
    if (rc) return rc;
    rc = ensure(c, &c->sel_buf, &c->sel_cap, select_scratch_bytes(c->ts.n, k));
    if (rc) return rc;
    rc = score_into(c, m, c->snr_buf);
    if (rc) return rc;
    stk_hit *dst = (flags & STK_OUT_HOST) ? c->hits_dev : out;
    int nl = 0;
    cudaError_t e = launch_select_topk(c->snr_buf, c->ts.n, k, c->ts, m->dev, c->sel_buf, dst, c->stream, &nl,
                                       (uint32_t)c->tune.select_sample);
    if (e != cudaSuccess) return set_err(c, STK_ECUDA, "selection launch: %s", cudaGetErrorString(e));
    c->last_launches = 1 + nl + (c->plan.order ? c->plan.order_launches : 0);
    c->timed = c->profiling;
    if (c->profiling) CUDA_TRY(c, cudaEventRecord(c->ev[2], c->stream));
    if (flags & STK_OUT_HOST) {
        CUDA_TRY(c, cudaMemcpyAsync(out, c->hits_dev, sizeof(stk_hit) * (size_t)k, cudaMemcpyDeviceToHost, c->stream));
        if ((rc = debug_verify(c, m)) != STK_OK) return rc;
        int fl = 0;
        rc = read_err_flags(c, &fl);
        if (rc) return rc;
        return flags_to_status(c, fl);
    }
    return debug_verify(c, m);
}

int stk_track_params(stk_ctx *c, const stk_map *m, uint64_t g, uint32_t f[3], double *tau, int32_t *bins_host)
{
    if (!c) return STK_EINVAL;
    int rc = check_ready(c, m);
    if (rc) return rc;
    if (!f || !tau) return set_err(c, STK_EINVAL, "f or tau is NULL");
    CUDA_TRY(c, cudaSetDevice(c->device));
    const size_t need = 32 + (size_t)m->dev.n_t * 4;
    rc = ensure(c, (void **)&c->small_dev, &c->small_cap, need);
    if (rc) return rc;
    uint32_t *fd = c->small_dev;                            // 3 bins, 3 times
    double *td = (double *)((char *)c->small_dev + 24);
    int32_t *bd = (int32_t *)((char *)c->small_dev + 32);
    if (c->ts.general && (rc = check_general(c, m)) != STK_OK) return rc;
    cudaError_t e = launch_track_params(m->dev, c->ts, g, fd, td, bins_host ? bd : nullptr, c->stream);
    if (e != cudaSuccess) return set_err(c, STK_ECUDA, "params launch: %s", cudaGetErrorString(e));
    CUDA_TRY(c, cudaMemcpyAsync(f, fd, 12, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(tau, td, 8, cudaMemcpyDeviceToHost, c->stream));
    if (bins_host)
        CUDA_TRY(c, cudaMemcpyAsync(bins_host, bd, (size_t)m->dev.n_t * 4, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return STK_OK;
}

int stk_score_explicit(stk_ctx *c, const stk_map *m, const uint32_t *f3, const double *tau, uint64_t n,
                       double *out)
{
    if (!c) return STK_EINVAL;
    if (!m || m->ctx != c) return set_err(c, STK_EINVAL, "map is NULL or belongs to another context");
    if (n == 0) return STK_OK;
    if (!f3 || !tau || !out) return set_err(c, STK_EINVAL, "NULL pointer");
    CUDA_TRY(c, cudaSetDevice(c->device));
    int rc = ensure(c, (void **)&c->snr_buf, &c->snr_cap, n * sizeof(float));
    if (rc) return rc;
    cudaError_t e = launch_score_explicit(m->dev, f3, tau, n, c->snr_buf, c->d_err, c->stream);
    if (e == cudaSuccess) e = launch_widen(c->snr_buf, out, n, c->stream);
    if (e != cudaSuccess) return set_err(c, STK_ECUDA, "explicit scoring launch: %s", cudaGetErrorString(e));
    return debug_verify(c, m);
}

int stk_set_template_shape(stk_ctx *c, int general, int t_min)
{
    if (!c) return STK_EINVAL;
    if (general && t_min < 1) return set_err(c, STK_EINVAL, "t_min must be >= 1 column for general templates");
    c->ts.general = general ? 1 : 0;
    c->ts.t_min = general ? t_min : 0;
    return STK_OK;
}

int stk_set_tau_prior(stk_ctx *c, const double *q, int n)
{
    if (!c) return STK_EINVAL;
    if (!q || n == 0) {
        c->ts.tau_q = nullptr;
        c->ts.n_q = 0;
        return STK_OK;
    }
    if (n < 2 || n > 65536) return set_err(c, STK_EINVAL, "the delay prior needs 2 .. 65536 quantiles");
    for (int i = 0; i < n; ++i) {
        if (!std::isfinite(q[i])) return set_err(c, STK_EINVAL, "delay quantile %d is not finite", i);
        if (i && q[i] < q[i - 1]) return set_err(c, STK_EINVAL, "delay quantiles must not decrease (at %d)", i);
    }
    CUDA_TRY(c, cudaSetDevice(c->device));
    int rc = ensure(c, (void **)&c->tauq_dev, &c->tauq_cap, sizeof(double) * (size_t)n);
    if (rc) return rc;
    CUDA_TRY(c, cudaMemcpyAsync(c->tauq_dev, q, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->ts.tau_q = c->tauq_dev;
    c->ts.n_q = n;
    return STK_OK;
}

int stk_track_times(stk_ctx *c, const stk_map *m, uint64_t g, uint32_t t[3])
{
    if (!c) return STK_EINVAL;
    if (!t) return set_err(c, STK_EINVAL, "t is NULL");
    uint32_t f[3];
    double tau;
    int rc = stk_track_params(c, m, g, f, &tau, nullptr);
    if (rc) return rc;
    CUDA_TRY(c, cudaMemcpy(t, (char *)c->small_dev + 12, 12, cudaMemcpyDeviceToHost));
    return STK_OK;
}

int stk_score_explicit_general(stk_ctx *c, const stk_map *m, const uint32_t *t3, const uint32_t *f3,
                               const double *tau, uint64_t n, double *out)
{
    if (!c) return STK_EINVAL;
    if (!m || m->ctx != c) return set_err(c, STK_EINVAL, "map is NULL or belongs to another context");
    if (n == 0) return STK_OK;
    if (!t3 || !f3 || !tau || !out) return set_err(c, STK_EINVAL, "NULL pointer");
    if (m->dev.n_t > 4096 || m->dev.n_f > 8192)
        return set_err(c, STK_EINVAL, "general templates need n_t <= 4096 and n_f <= 8192");
    CUDA_TRY(c, cudaSetDevice(c->device));
    int rc = ensure(c, (void **)&c->snr_buf, &c->snr_cap, n * sizeof(float));
    if (rc) return rc;
    cudaError_t e = launch_score_explicit_general(m->dev, t3, f3, tau, n, c->snr_buf, c->d_err, c->stream);
    if (e == cudaSuccess) e = launch_widen(c->snr_buf, out, n, c->stream);
    if (e != cudaSuccess) return set_err(c, STK_ECUDA, "explicit general scoring launch: %s", cudaGetErrorString(e));
    return debug_verify(c, m);
}

int stk_interp_forward(stk_ctx *c, const stk_map *m, const float *f3, const float *tau, uint64_t n, float *snr)
{
    if (!c) return STK_EINVAL;
    if (!m || m->ctx != c) return set_err(c, STK_EINVAL, "map is NULL or belongs to another context");
    if (n == 0) return STK_OK;
    if (!f3 || !tau || !snr) return set_err(c, STK_EINVAL, "NULL pointer");
    CUDA_TRY(c, cudaSetDevice(c->device));
    cudaError_t e = launch_interp_tuned(m->dev, f3, tau, nullptr, n, snr, nullptr, nullptr, false, c->interp_threads, c->d_err,
                                        c->stream);
    if (e != cudaSuccess) return set_err(c, STK_ECUDA, "interpolated forward launch: %s", cudaGetErrorString(e));
    return debug_verify(c, m);
}

int stk_interp_adjoint(stk_ctx *c, const stk_map *m, const float *f3, const float *tau, const float *g, uint64_t n,
                       float *grad_f3, float *grad_tau)
{
    if (!c) return STK_EINVAL;
    if (!m || m->ctx != c) return set_err(c, STK_EINVAL, "map is NULL or belongs to another context");
    if (n == 0) return STK_OK;
    if (!f3 || !tau || !g || !grad_f3 || !grad_tau) return set_err(c, STK_EINVAL, "NULL pointer");
    CUDA_TRY(c, cudaSetDevice(c->device));
    cudaError_t e = launch_interp_tuned(m->dev, f3, tau, g, n, nullptr, grad_f3, grad_tau, true, c->interp_threads, c->d_err,
                                        c->stream);
    if (e != cudaSuccess) return set_err(c, STK_ECUDA, "interpolated adjoint launch: %s", cudaGetErrorString(e));
    return debug_verify(c, m);
}

int stk_refine(stk_ctx *c, const stk_map *m, float *f3, float *tau, uint64_t n, int steps, float lr_bins,
               float lr_tau_frac, float tau_max, float *hist)
{
    if (!c) return STK_EINVAL;
    if (!m || m->ctx != c) return set_err(c, STK_EINVAL, "map is NULL or belongs to another context");
    if (steps < 0) return set_err(c, STK_EINVAL, "steps < 0");
    if (!(tau_max > 0.f) || !std::isfinite(tau_max)) return set_err(c, STK_EINVAL, "tau_max must be > 0 and finite");
    if (!std::isfinite(lr_bins) || !std::isfinite(lr_tau_frac) || lr_bins < 0.f || lr_tau_frac < 0.f)
        return set_err(c, STK_EINVAL, "learning rates must be >= 0 and finite");
    if (n == 0) return STK_OK;
    if (!f3 || !tau) return set_err(c, STK_EINVAL, "NULL pointer");
    CUDA_TRY(c, cudaSetDevice(c->device));
    int rc = ensure(c, &c->refine_buf, &c->refine_cap, refine_scratch_bytes(steps));
    if (rc) return rc;
    cudaError_t e = launch_refine(m->dev, f3, tau, n, steps, lr_bins, lr_tau_frac, tau_max, hist, c->refine_buf,
                                  c->interp_threads, c->d_err, c->stream);
    if (e != cudaSuccess) return set_err(c, STK_ECUDA, "refinement launch: %s", cudaGetErrorString(e));
    return debug_verify(c, m);
}

int stk_polish(stk_ctx *c, const stk_map *m, uint32_t *f3, double *tau, const float *alt_f3, const float *alt_tau,
               uint64_t n, double tau_max, int moves, double *snr, int *which)
{
    if (!c) return STK_EINVAL;
    if (!m || m->ctx != c) return set_err(c, STK_EINVAL, "map is NULL or belongs to another context");
    if (!(tau_max > 0.0) || !std::isfinite(tau_max)) return set_err(c, STK_EINVAL, "tau_max must be > 0 and finite");
    if (moves < 0 || moves > 1024) return set_err(c, STK_EINVAL, "moves = %d outside [0, 1024]", moves);
    if ((alt_f3 == nullptr) != (alt_tau == nullptr)) return set_err(c, STK_EINVAL, "alt_f3 and alt_tau go together");
    if (n == 0) return STK_OK;
    if (!f3 || !tau) return set_err(c, STK_EINVAL, "NULL pointer");
    CUDA_TRY(c, cudaSetDevice(c->device));
    cudaError_t e = launch_polish(m->dev, f3, tau, alt_f3, alt_tau, n, tau_max, moves, snr, which, c->d_err,
                                  c->stream);
    if (e != cudaSuccess) return set_err(c, STK_ECUDA, "polish launch: %s", cudaGetErrorString(e));
    return debug_verify(c, m);
}

int stk_sync(stk_ctx *c)
{
    if (!c) return STK_EINVAL;
    CUDA_TRY(c, cudaSetDevice(c->device));
    int fl = 0;
    int rc = read_err_flags(c, &fl);
    if (rc) return rc;
    return flags_to_status(c, fl);
}

int stk_set_profiling(stk_ctx *c, int enable)
{
    if (!c) return STK_EINVAL;
    c->profiling = enable != 0;
    c->timed = false;
    return STK_OK;
}

int stk_last_timings(stk_ctx *c, double out[4])
{
    if (!c || !out) return STK_EINVAL;
    if (!c->timed) return set_err(c, STK_ESTATE, "no profiled call yet (stk_set_profiling)");
    CUDA_TRY(c, cudaEventSynchronize(c->ev[2]));
    float a = 0.f, b = 0.f, o = 0.f;
    CUDA_TRY(c, cudaEventElapsedTime(&o, c->ev[0], c->ev[3]));
    CUDA_TRY(c, cudaEventElapsedTime(&a, c->ev[3], c->ev[1]));
    CUDA_TRY(c, cudaEventElapsedTime(&b, c->ev[1], c->ev[2]));
    out[0] = a;
    out[1] = b;
    out[2] = c->last_launches;
    out[3] = o;
    return STK_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// No-allocation variant of stk_score (the paper has no counterpart).
//
// Some callers cannot call cudaMalloc at scoring time: code whose device
// memory is owned by another allocator (a framework's caching allocator or a
// fixed memory budget, where an extra allocation can fail or fragment), and
// latency-critical loops that cannot afford cudaFree's device-wide
// synchronisation.  This entry point takes its scratch (one SNR per template
// plus the selection state) from a fixed array in device memory that every
// GPU loading the library holds until the process exits.  It never calls
// cudaMalloc, cudaFree or any allocating routine.
namespace {

constexpr uint64_t kNoAllocMaxTracks = STK_NOALLOC_MAX_TRACKS;
constexpr size_t kNoAllocSnrBytes = kNoAllocMaxTracks * sizeof(float);
constexpr size_t kNoAllocFlagBytes = 256;
constexpr size_t kNoAllocSelBytes = 1024 * 1024;
constexpr int kNoAllocMaxDevices = 64;

// Shared by every call on a device: SNRs | error flag | selection state.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocSnrBytes + kNoAllocFlagBytes + kNoAllocSelBytes];

struct NoAllocDevice {
    void *base = nullptr;  // device address of g_noalloc_scratch on this device
    int num_sms = 0;
    size_t smem_optin = 0;
};
std::mutex g_noalloc_mu;
NoAllocDevice g_noalloc_dev[kNoAllocMaxDevices];

// Once per device, with that device current: resolve the array's device address.
int noalloc_setup(int dev, NoAllocDevice *out)
{
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    NoAllocDevice &d = g_noalloc_dev[dev];
    if (!d.base) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return set_err(nullptr, STK_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
        int v = 0;
        if ((e = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return set_err(nullptr, STK_ECUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(e));
        d.num_sms = v;
        if ((e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
            return set_err(nullptr, STK_ECUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(e));
        d.smem_optin = (size_t)v;
        d.base = p;
    }
    *out = d;
    return STK_OK;
}

// After the selection: on a timeout (some templates' SNRs were not written and
// the array still holds an earlier call's values) or on bad map data reported
// by a deferred pack, every output hit is marked invalid (SNR NaN, index all
// ones); the status word, if given, gets STK_ETIMEOUT, STK_EINVAL or STK_OK.
__global__ void noalloc_finish_kernel(const int *flags, const int *ctx_flags, int k, stk_hit *out, int *status)
{
    const bool timeout = (*flags & ERR_TIMEOUT) != 0;
    const bool bad = (*ctx_flags & (ERR_BADINPUT | ERR_FP16_RANGE)) != 0;
    if (timeout || bad)
        for (int i = threadIdx.x; i < k; i += blockDim.x) {
            out[i].snr = __longlong_as_double(0x7ff8000000000000ll);
            out[i].index = ~0ull;
        }
    if (status && threadIdx.x == 0) *status = timeout ? STK_ETIMEOUT : bad ? STK_EINVAL : STK_OK;
}

}  // namespace

extern "C" int stk_score_noalloc(const stk_map *m, uint64_t n_tracks, uint64_t seed, uint64_t counter_offset,
                                 double tau_max_s, int k, stk_hit *out_topk_dev, int *status_dev,
                                 void *cuda_stream)
{
    if (!m || !m->ctx) return set_err(nullptr, STK_EINVAL, "map is NULL");
    if (!out_topk_dev) return set_err(nullptr, STK_EINVAL, "out_topk_dev is NULL");
    if (n_tracks < 1 || n_tracks > kNoAllocMaxTracks)
        return set_err(nullptr, STK_EINVAL,
                       "n_tracks = %llu outside [1, %llu], the no-allocation scratch limit; split the template "
                       "range over several calls and keep the largest SNRs",
                       (unsigned long long)n_tracks, (unsigned long long)kNoAllocMaxTracks);
    if (k < 1 || k > STK_MAX_K || (uint64_t)k > n_tracks)
        return set_err(nullptr, STK_EINVAL, "k = %d must be in [1, min(%d, n_tracks)]", k, STK_MAX_K);
    if (!std::isfinite(tau_max_s) || tau_max_s < 0) return set_err(nullptr, STK_EINVAL, "tau_max must be finite and >= 0");
    if (select_scratch_bytes(n_tracks, k) > kNoAllocSelBytes)
        return set_err(nullptr, STK_EINVAL, "selection state exceeds the no-allocation scratch");
    const int dev = m->ctx->device;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return set_err(nullptr, STK_EINVAL, "device %d out of range", dev);
    int prev = 0;
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess) return set_err(nullptr, STK_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if ((e = cudaSetDevice(dev)) != cudaSuccess)
        return set_err(nullptr, STK_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    NoAllocDevice d;
    int rc = noalloc_setup(dev, &d);
    if (rc == STK_OK) {
        cudaStream_t st = (cudaStream_t)cuda_stream;
        stk_ctx *c = m->ctx;
        unsigned char *base = (unsigned char *)d.base;
        float *snr = (float *)base;
        int *flags = (int *)(base + kNoAllocSnrBytes);
        void *sel = base + kNoAllocSnrBytes + kNoAllocFlagBytes;
        TrackSet ts{n_tracks, seed, counter_offset, tau_max_s};
        Tuning tu = c->tune;  // launch shape and wait limits; no coherent order (it needs scratch)
        ScorePlan plan{};
        int nl = 0;
        // The map's last load or update may still be packing on the context's
        // stream: this stream waits for it.  The array keeps the previous call's
        // contents: the flag word must start at zero; the selection kernels reset
        // their own state; the scoring kernel writes every SNR unless a bounded wait
        // gives up, and then the finishing kernel marks the hits invalid.
        if ((e = cudaEventRecord(c->stream_mark, c->stream)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(st, c->stream_mark, 0)) != cudaSuccess ||
            (e = cudaMemsetAsync(flags, 0, sizeof(int), st)) != cudaSuccess ||
            (e = launch_score_generated(m->dev, ts, snr, flags, tu, d.num_sms, d.smem_optin, st, &plan)) !=
                cudaSuccess ||
            (e = launch_select_topk(snr, n_tracks, k, ts, m->dev, sel, out_topk_dev, st, &nl)) != cudaSuccess)
            rc = set_err(nullptr, STK_ECUDA, "no-allocation scoring: %s", cudaGetErrorString(e));
        else {
            noalloc_finish_kernel<<<1, 256, 0, st>>>(flags, c->d_err, k, out_topk_dev, status_dev);
            if ((e = cudaGetLastError()) != cudaSuccess)
                rc = set_err(nullptr, STK_ECUDA, "finishing kernel: %s", cudaGetErrorString(e));
        }
    }
    cudaSetDevice(prev);
    return rc;
}
