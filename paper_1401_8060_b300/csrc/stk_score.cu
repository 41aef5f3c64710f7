// Scoring kernels: Eq. 7 of the paper for many templates.
//
//   SNR_tot = sum over the template's pixels of Re[exp(2 pi i f tau) p(t; f)],
//   normalised by sqrt(sum sigma^-2) (weighted) or by N (paper form).
//
// Two kernels compute the same per-template arithmetic in the same order:
//   score_simple  one thread per template, pixels read from the L2-resident map;
//                 used for explicit templates, small jobs and maps whose
//                 rasteriser needs 64-bit numerators or whose phase needs the
//                 64-bit form (n_f > 8192).
//   score_staged  persistent CTAs; each CTA holds a batch of R * blockDim
//                 templates in registers (in coherent order, stk_order.cu) and
//                 streams the map through shared memory in slabs of S time
//                 columns (one bulk copy per slab, two buffers on mbarriers,
//                 refilled by the last warp to finish them), so every gathered
//                 pixel is a shared-memory load.  The map is read from L2 once
//                 per batch.
// Both come in two storage precisions (PREC): 8-byte FP32 polar records, or
// 4-byte records holding |y|/sigma in FP16 and the phase in Q0.16 turns, the
// per-frequency (or per-pixel) scale 1/sigma then doubling as the weight.
// General templates (random control times) have their own one-thread kernel.
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdio>

#include "stk_internal.cuh"
#include "stk_pixel.cuh"

namespace stk {

namespace {

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s per slab wait
constexpr int kMaxThreads = 1024;

// ------------------------------------------------------------------ simple kernel
template <int WMODE, int PREC, bool EXPLICIT, bool FAST32>
__global__ void __launch_bounds__(256) score_simple_kernel(MapDev m, TrackSet ts, const uint32_t *__restrict__ f3,
                                                           const double *__restrict__ tau_in, uint64_t n,
                                                           float *__restrict__ out, int *err)
{
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t f[3];
    double tau;
    if (EXPLICIT) {
        bool bad = false;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            f[k] = f3[3 * i + k];
            if (f[k] >= (uint32_t)m.n_f) { bad = true; f[k] = (uint32_t)m.n_f - 1; }
        }
        if (bad) atomicOr(err, ERR_BADTRACK);
        tau = tau_in[i];
    } else {
        draw_track_ts(ts, ts.offset + i, (uint32_t)m.n_f, f, tau);
    }
    const Phase ph = phase_consts(m.f_min, m.df, tau, m.n_f);
    float acc = 0.f, W = 0.f;
    Raster32 r;
    if (FAST32) r = raster_init(f[0], f[1], f[2], m.M);
    for (int j = 0; j < m.n_t; ++j) {
        uint32_t bin;
        if (FAST32) {
            bin = __umulhi(r.N, m.magic) >> m.shift;
            r.N += r.D;
            r.D += r.D2;
        } else {
            bin = raster_bin_wide(f[0], f[1], f[2], m.M, (uint32_t)j, m.d);
        }
        if (kDebugBounds) bin = checked_bin(bin, j, m.n_t, hull_lo(f), hull_hi(f), err);
        const auto v = Pix<PREC>::load_global(m.rec, (size_t)j * m.ldr + bin);
        float wv = 0.f;
        if (WMODE == WMODE_FREQ) wv = __ldg(m.w + bin);
        if (WMODE == WMODE_PIXEL) wv = __ldg(m.w + (size_t)j * m.ldw + bin);
        accumulate<PREC, WMODE>(v, bin, ph, wv, acc, W);
    }
    out[i] = finalize_snr<WMODE>(acc, W, m);
}

// ------------------------------------------------------------------ general templates
// Templates with random start, middle and end times (Sec. III: six random numbers,
// duration >= t_min): one thread per template, pixels of its own columns t0 .. t2
// only, from the L2-resident map; the exact integer rasteriser (gen_step) moves the
// pixel from column to column.  N = t2 - t0 + 1 pixels.
template <int WMODE, int PREC>
__device__ __forceinline__ float finalize_general(float acc, float W, const MapDev &m, int N)
{
    if (m.paper) return __fdiv_rn(acc, (float)N);
    if (WMODE == WMODE_CONST) {
        const float Wc = PREC == PREC_FP16 ? (float)N : __fmul_rn((float)N, m.w_const);
        return Wc > 0.f ? __fdiv_rn(acc, __fsqrt_rn(Wc)) : 0.f;   // every pixel notched: no data
    }
    return W > 0.f ? __fdiv_rn(acc, __fsqrt_rn(W)) : 0.f;
}

// One thread per template, in coherent order when perm is given (a warp's
// templates then start and end in nearby columns and sit at nearby bins).  The
// L2 gathers make it latency-bound: 64 registers (4 blocks of 256 per SM) run
// 15 % faster than the 80 the compiler takes unbounded.
template <int WMODE, int PREC, bool EXPLICIT>
__global__ void __launch_bounds__(256, 4) score_general_kernel(MapDev m, TrackSet ts, const uint32_t *__restrict__ t3,
                                                            const uint32_t *__restrict__ f3,
                                                            const double *__restrict__ tau_in, uint64_t n,
                                                            float *__restrict__ out, int *err,
                                                            const uint32_t *__restrict__ perm)
{
    const uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const uint64_t i = perm ? (uint64_t)__ldg(perm + p) : p;
    uint32_t f[3], t[3];
    double tau;
    if (EXPLICIT) {
        bool bad = false;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            f[k] = f3[3 * i + k];
            t[k] = t3[3 * i + k];
            if (f[k] >= (uint32_t)m.n_f) { bad = true; f[k] = (uint32_t)m.n_f - 1; }
            if (t[k] >= (uint32_t)m.n_t) { bad = true; t[k] = (uint32_t)m.n_t - 1; }
        }
        if (!(t[0] <= t[1] && t[1] <= t[2] && t[0] < t[2])) {  // not a valid time ordering: use the full span
            bad = true;
            t[0] = 0; t[2] = (uint32_t)m.n_t - 1; t[1] = t[2] / 2;
        }
        if (bad) atomicOr(err, ERR_BADTRACK);
        tau = tau_in[i];
    } else {
        draw_track_ts(ts, ts.offset + i, (uint32_t)m.n_f, f, tau);
        draw_times(ts.seed, ts.offset + i, (uint32_t)m.n_t, (uint32_t)ts.t_min, t);
    }
    const Phase ph = phase_consts(m.f_min, m.df, tau, m.n_f);
    const GenCurve c = gen_curve(t, f);
    const GenFilter gf = gen_filter(c);
    // Two partial sums: pixels the estimate decides, in column order, and pixels
    // within its margin of a rounding boundary (about 2 % of them), also in column
    // order.  Those wait, up to four per lane; the waiting pixels of all lanes then
    // take the long exact test together, so the warp runs it once for every lane
    // rather than once per lane.  Each template's sums do not depend on its
    // neighbours in the warp: when a flush happens changes nothing.
    float acc = 0.f, W = 0.f, acc_x = 0.f, W_x = 0.f;
    const uint32_t h_lo = hull_lo(f), h_hi = hull_hi(f);
    // General-template maps have n_t <= 4096 and n_f <= 8192: 32-bit pixel indices
    // and the narrow phase form (its 64-bit increment term is zero) always apply.
    const uint32_t ldr = (uint32_t)m.ldr, ldw = (uint32_t)m.ldw;
    auto add = [&](int j, int32_t b, float &a_, float &w_) {
        if (kDebugBounds) b = (int32_t)checked_bin((uint32_t)b, j, m.n_t, h_lo, h_hi, err);
        const auto v = Pix<PREC>::load_global(m.rec, (uint32_t)j * ldr + (uint32_t)b);
        float wv = 0.f;
        if (WMODE == WMODE_FREQ) wv = __ldg(m.w + b);
        if (WMODE == WMODE_PIXEL) wv = __ldg(m.w + ((uint32_t)j * ldw + (uint32_t)b));
        pixel_add<PREC, WMODE>(v, template_turn_narrow((uint32_t)b, ph.a, ph.c), wv, a_, w_);
    };
    int np = 0, pj0 = 0, pj1 = 0, pj2 = 0, pj3 = 0;
    int32_t pb0 = 0, pb1 = 0, pb2 = 0, pb3 = 0;
    auto flush = [&]() {
        for (int q = 0; q < np; ++q) {
            const int j = q == 0 ? pj0 : q == 1 ? pj1 : q == 2 ? pj2 : pj3;
            const int32_t b0 = q == 0 ? pb0 : q == 1 ? pb1 : q == 2 ? pb2 : pb3;
            add(j, gen_step(c, j, b0, m.n_f), acc_x, W_x);
        }
        np = 0;
    };
    auto push = [&](int j, int32_t b) {
        if (np == 0) { pj0 = j; pb0 = b; }
        else if (np == 1) { pj1 = j; pb1 = b; }
        else if (np == 2) { pj2 = j; pb2 = b; }
        else { pj3 = j; pb3 = b; }
        ++np;
    };
    // Two columns a step: both estimates, then both gathers in flight together (an
    // estimate's bin is always inside the map, so an undecided pixel's gather is
    // harmless and unused), then the sums in column order.
    using Rec = typename Pix<PREC>::Rec;
    auto gather = [&](int j, int32_t b, Rec &v, float &wv) {
        if (kDebugBounds) b = (int32_t)checked_bin((uint32_t)b, j, m.n_t, 0u, (uint32_t)m.n_f - 1u, err);
        v = Pix<PREC>::load_global(m.rec, (uint32_t)j * ldr + (uint32_t)b);
        wv = 0.f;
        if (WMODE == WMODE_FREQ) wv = __ldg(m.w + b);
        if (WMODE == WMODE_PIXEL) wv = __ldg(m.w + ((uint32_t)j * ldw + (uint32_t)b));
    };
    add((int)t[0], (int32_t)f[0], acc, W);
    const int jend = (int)t[2];
    for (int j = (int)t[0] + 1; j <= jend; j += 2) {
        const bool has1 = j < jend;
        const int j1 = has1 ? j + 1 : j;
        int32_t b0, b1;
        const bool ok0 = gen_estimate(c, gf, j, m.n_f, b0);
        const bool ok1 = gen_estimate(c, gf, j1, m.n_f, b1);
        Rec v0, v1;
        float w0, w1;
        gather(j, b0, v0, w0);
        gather(j1, b1, v1, w1);
        if (ok0) pixel_add<PREC, WMODE>(v0, template_turn_narrow((uint32_t)b0, ph.a, ph.c), w0, acc, W);
        else push(j, b0);
        if (has1) {
            if (ok1) pixel_add<PREC, WMODE>(v1, template_turn_narrow((uint32_t)b1, ph.a, ph.c), w1, acc, W);
            else push(j1, b1);
        }
        if (__any_sync(__activemask(), np >= 3)) flush();  // room for the next step's two
    }
    flush();
    acc += acc_x;
    W += W_x;
    out[i] = finalize_general<WMODE, PREC>(acc, W, m, (int)(t[2] - t[0] + 1));
}

template <int WMODE, int PREC, bool EXPLICIT>
cudaError_t launch_general_W(const MapDev &m, const TrackSet &ts, const uint32_t *t3, const uint32_t *f3,
                             const double *tau, uint64_t n, float *out, int *err, cudaStream_t st,
                             const uint32_t *perm)
{
    const uint64_t blocks = (n + 255) / 256;
    if (blocks > 0x7fffffffull) return cudaErrorInvalidValue;
    score_general_kernel<WMODE, PREC, EXPLICIT>
        <<<(unsigned)blocks, 256, 0, st>>>(m, ts, t3, f3, tau, n, out, err, perm);
    return cudaGetLastError();
}

template <bool EXPLICIT>
cudaError_t launch_general(const MapDev &m, const TrackSet &ts, const uint32_t *t3, const uint32_t *f3,
                           const double *tau, uint64_t n, float *out, int *err, cudaStream_t st,
                           const uint32_t *perm = nullptr)
{
#define STK_GEN(W, P) return launch_general_W<W, P, EXPLICIT>(m, ts, t3, f3, tau, n, out, err, st, perm)
    if (m.prec == PREC_FP16) {
        if (m.wmode == WMODE_CONST) STK_GEN(WMODE_CONST, PREC_FP16);
        if (m.wmode == WMODE_FREQ) STK_GEN(WMODE_FREQ, PREC_FP16);
        STK_GEN(WMODE_PIXEL, PREC_FP16);
    }
    if (m.wmode == WMODE_CONST) STK_GEN(WMODE_CONST, PREC_FP32);
    if (m.wmode == WMODE_FREQ) STK_GEN(WMODE_FREQ, PREC_FP32);
    STK_GEN(WMODE_PIXEL, PREC_FP32);
#undef STK_GEN
}

// ------------------------------------------------------------------ staged kernel
constexpr int kMaxStages = 4;
// shared bytes after the slabs and weight table: full barriers, last issued
// slab and finished-warp count per buffer, abort flag
constexpr size_t kStagedBookkeeping = 128;
static_assert(kMaxStages * (8 + 8 + 4) + 4 <= kStagedBookkeeping, "bookkeeping block too small");

struct StagedArgs {
    int S, nstage, nslabs;
    uint64_t batch, nbatches;
    uint32_t slab_recs;    // S * ldr
    uint32_t slab_ws;      // S * ldw (WMODE_PIXEL)
    uint32_t wtab_floats;  // n_f rounded to 4 (WMODE_FREQ)
    uint64_t wait_ns;      // limit of each slab wait
    uint64_t withhold_q;   // test of the bounded waits: CTA 0 never issues its slab number withhold_q
    const uint32_t *perm;  // scoring order: position p holds template offset + perm[p] (NULL: index order)
};

// Slab pipeline without block-wide barriers: a slab buffer is refilled by the
// warp that finishes it last (a shared counter per buffer elects it), so a warp
// waits only for the slab it needs next and warps may drift by up to nstage - 1
// slabs.  Every wait is bounded; a warp that gives up raises a shared flag and
// the others stop at their next slab.
// Up to 5 templates per thread (6 without a weight sum) fit 64 registers (1024
// threads); more need up to 128 (512 threads).
constexpr int staged_max_threads(int R, int WMODE)
{
    return (R <= 5 || (R == 6 && WMODE == WMODE_CONST)) ? kMaxThreads : 512;
}

template <int R, int WMODE, int PREC>
__global__ void __launch_bounds__(staged_max_threads(R, WMODE), 1)
    score_staged_kernel(MapDev m, TrackSet ts, StagedArgs a, float *__restrict__ out, int *err)
{
    using Rec = typename Pix<PREC>::Rec;
    extern __shared__ __align__(128) unsigned char smem[];
    // bookkeeping first (fixed offsets), then the slab buffers and weight table
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);               // full barrier per buffer
    uint64_t *issued = bars + kMaxStages;                               // last slab issued into each buffer
    uint32_t *done = reinterpret_cast<uint32_t *>(issued + kMaxStages);  // warps finished with each buffer
    int *abort_flag = reinterpret_cast<int *>(done + kMaxStages);
    Rec *srec = reinterpret_cast<Rec *>(smem + kStagedBookkeeping);
    float *sw = reinterpret_cast<float *>(srec + (size_t)a.nstage * a.slab_recs);  // WMODE_PIXEL slabs
    float *swt = sw + (WMODE == WMODE_PIXEL ? (size_t)a.nstage * a.slab_ws : 0);    // WMODE_FREQ table

    const int tid = threadIdx.x;
    const int nthr = blockDim.x;
    const int lane = tid & 31;
    if (blockIdx.x >= a.nbatches) return;
    const uint64_t my_nb = (a.nbatches - blockIdx.x + gridDim.x - 1) / gridDim.x;
    const uint64_t total = my_nb * (uint64_t)a.nslabs;  // slabs this CTA consumes, over all its batches
    const Rec *grec = reinterpret_cast<const Rec *>(m.rec);

    if (tid == 0) {
        for (int s = 0; s < a.nstage; ++s) {
            mbar_init(&bars[s], 1);
            issued[s] = ~0ull;
            done[s] = 0u;
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (WMODE == WMODE_FREQ) {
        for (int k = tid; k < m.n_f; k += nthr) swt[k] = m.w[k];
    }
    __syncthreads();

    // Producer: slab q of this CTA's sequence (slab index sl of a batch) goes to buffer `slot`.
    auto issue = [&](uint64_t q, int slot, int sl) {
        if (blockIdx.x == 0 && q == a.withhold_q) return;  // a copy that never comes: the wait must give up
        const int row0 = sl * a.S;
        const int rows = min(a.S, m.n_t - row0);
        const uint32_t row_bytes = (uint32_t)m.ldr * (uint32_t)sizeof(Rec);
        const uint32_t wrow_bytes = (uint32_t)m.ldw * 4u;
        uint32_t bytes = (uint32_t)rows * row_bytes;
        if (WMODE == WMODE_PIXEL) bytes += (uint32_t)rows * wrow_bytes;
        issued[slot] = q;
        mbar_arrive_expect_tx(&bars[slot], bytes);
        bulk_g2s(srec + (size_t)slot * a.slab_recs, grec + (size_t)row0 * m.ldr, (uint32_t)rows * row_bytes,
                 &bars[slot]);
        if (WMODE == WMODE_PIXEL)
            bulk_g2s(sw + (size_t)slot * a.slab_ws, m.w + (size_t)row0 * m.ldw, (uint32_t)rows * wrow_bytes,
                     &bars[slot]);
    };
    if (tid == 0) {
        const int pre = (int)(total < (uint64_t)a.nstage ? total : (uint64_t)a.nstage);
        for (int q0 = 0; q0 < pre; ++q0) issue((uint64_t)q0, q0, q0 % a.nslabs);
    }

    const uint32_t magic = m.magic;
    const int shift = m.shift;
    const uint32_t srec_a = smem_u32(srec), sw_a = smem_u32(sw), swt_a = smem_u32(swt);
    const uint32_t row_bytes = (uint32_t)m.ldr * (uint32_t)sizeof(Rec);
    const uint32_t wrow_bytes = WMODE == WMODE_PIXEL ? (uint32_t)m.ldw * 4u : 0u;
    const uint32_t slab_bytes = a.slab_recs * (uint32_t)sizeof(Rec);
    const uint32_t wslab_bytes = WMODE == WMODE_PIXEL ? a.slab_ws * 4u : 0u;
    uint64_t q = 0;      // slab sequence number
    int slot = 0;        // q % nstage
    uint32_t parity = 0; // (q / nstage) & 1
    bool failed = false;
    for (uint64_t ib = 0; ib < my_nb && !failed; ++ib) {
        const uint64_t b = blockIdx.x + ib * gridDim.x;
        const uint64_t t0 = b * a.batch;
        const uint64_t tn = (ts.n - t0) < a.batch ? (ts.n - t0) : a.batch;

        uint32_t N[R], D[R], D2[R];
        uint32_t pa[R], pc[R];  // narrow phase form (n_f <= kPhaseNarrowNf)
        float acc[R], W[R];
        uint32_t hlo[kDebugBounds ? R : 1], hhi[kDebugBounds ? R : 1];  // debug build: each template's bins
#pragma unroll
        for (int r = 0; r < R; ++r) {
            uint64_t i = (uint64_t)tid + (uint64_t)r * nthr;
            if (i >= tn) i = tn - 1;  // idle slot: repeat a valid template, result discarded
            const uint64_t rel = a.perm ? (uint64_t)__ldg(a.perm + t0 + i) : t0 + i;
            uint32_t f[3];
            double tau;
            draw_track_ts(ts, ts.offset + rel, (uint32_t)m.n_f, f, tau);
            const Raster32 rs = raster_init(f[0], f[1], f[2], m.M);
            N[r] = rs.N; D[r] = rs.D; D2[r] = rs.D2;
            const Phase ph = phase_consts(m.f_min, m.df, tau, m.n_f);
            pa[r] = ph.a;
            pc[r] = ph.c;
            acc[r] = 0.f;
            W[r] = 0.f;
            if (kDebugBounds) {
                hlo[kDebugBounds ? r : 0] = hull_lo(f);
                hhi[kDebugBounds ? r : 0] = hull_hi(f);
            }
        }

        for (int s = 0; s < a.nslabs; ++s, ++q) {
            const bool ok = __all_sync(0xffffffffu, mbar_wait(&bars[slot], parity, a.wait_ns)) &&
                            !*(volatile int *)abort_flag;
            if (!ok) {
                if (lane == 0) atomicOr(abort_flag, 1);
                failed = true;
                break;
            }
            const int rows = min(a.S, m.n_t - s * a.S);
            uint32_t rb = srec_a + (uint32_t)slot * slab_bytes;  // shared address of the slab's current row
            uint32_t wb = sw_a + (uint32_t)slot * wslab_bytes;   // its weight row (WMODE_PIXEL)
            // One pixel of template r at rasteriser value Nv (row base rb_, weight row wb_).
            auto col = [&](int r, uint32_t Nv, uint32_t rb_, uint32_t wb_, int jcol) {
                uint32_t b = __umulhi(Nv, magic) >> shift;
                if (kDebugBounds)
                    b = checked_bin(b, jcol, m.n_t, hlo[kDebugBounds ? r : 0], hhi[kDebugBounds ? r : 0], err);
                const Rec v = Pix<PREC>::load_shared(rb_ + (b << Pix<PREC>::kLog2Bytes));
                float wv = 0.f;
                if (WMODE == WMODE_FREQ) wv = lds_f32(swt_a + (b << 2));
                if (WMODE == WMODE_PIXEL) wv = lds_f32(wb_ + (b << 2));
                pixel_add<PREC, WMODE>(v, template_turn_narrow(b, pa[r], pc[r]), wv, acc[r], W[r]);
            };
            // Columns in pairs: N_{j+1} = N_j + D_j and N_{j+2} = N_{j+1} + D_j + D2,
            // D_{j+2} = D_j + 2 D2 (three additions per two columns, exact mod 2^32).
            int jj = 0;
            for (; jj + 1 < rows; jj += 2) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const uint32_t Na = N[r], Nb = Na + D[r];
                    col(r, Na, rb, wb, s * a.S + jj);
                    col(r, Nb, rb + row_bytes, wb + wrow_bytes, s * a.S + jj + 1);
                    N[r] = Nb + D[r] + D2[r];
                    D[r] = D[r] + D2[r] + D2[r];
                }
                rb += 2 * row_bytes;
                wb += 2 * wrow_bytes;
            }
            if (jj < rows) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    col(r, N[r], rb, wb, s * a.S + jj);
                    N[r] += D[r];
                    D[r] += D2[r];
                }
            }
            // This warp is done with the buffer; the last warp to finish refills it.
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();
                if (atomicAdd(&done[slot], 1u) == (uint32_t)(nthr >> 5) - 1u) {
                    done[slot] = 0u;
                    __threadfence_block();
                    fence_proxy_async_smem();
                    if (q + a.nstage < total) {
                        int sl = s + a.nstage;
                        while (sl >= a.nslabs) sl -= a.nslabs;
                        issue(q + a.nstage, slot, sl);
                    }
                }
            }
            if (++slot == a.nstage) {
                slot = 0;
                parity ^= 1u;
            }
        }
        if (failed) break;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint64_t i = (uint64_t)tid + (uint64_t)r * nthr;
            if (i < tn) {
                const uint64_t rel = a.perm ? (uint64_t)__ldg(a.perm + t0 + i) : t0 + i;
                out[rel] = finalize_snr<WMODE>(acc[r], W[r], m);
            }
        }
    }
    // Copies already issued must land before the CTA's shared memory goes away
    // (after a timeout some may still be in flight); each wait is bounded.
    __syncthreads();
    if (tid == 0) {
        if (*(volatile int *)abort_flag) atomicOr(err, ERR_TIMEOUT);
        for (int s = 0; s < a.nstage; ++s)
            if (issued[s] != ~0ull) mbar_wait(&bars[s], (uint32_t)((issued[s] / a.nstage) & 1ull), a.wait_ns);
    }
}

template <int R, int WMODE, int PREC>
cudaError_t launch_staged_R(const MapDev &m, const TrackSet &ts, const StagedArgs &sa, int grid, int threads,
                            size_t smem, float *out, int *err, cudaStream_t st)
{
    auto k = score_staged_kernel<R, WMODE, PREC>;
    if (threads > staged_max_threads(R, WMODE)) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, threads, smem, st>>>(m, ts, sa, out, err);
    return cudaGetLastError();
}

template <int WMODE, int PREC>
cudaError_t launch_staged_W(int R, const MapDev &m, const TrackSet &ts, const StagedArgs &sa, int grid, int threads,
                            size_t smem, float *out, int *err, cudaStream_t st)
{
    switch (R) {
    case 1: return launch_staged_R<1, WMODE, PREC>(m, ts, sa, grid, threads, smem, out, err, st);
    case 2: return launch_staged_R<2, WMODE, PREC>(m, ts, sa, grid, threads, smem, out, err, st);
    case 3: return launch_staged_R<3, WMODE, PREC>(m, ts, sa, grid, threads, smem, out, err, st);
    case 4: return launch_staged_R<4, WMODE, PREC>(m, ts, sa, grid, threads, smem, out, err, st);
    case 5: return launch_staged_R<5, WMODE, PREC>(m, ts, sa, grid, threads, smem, out, err, st);
    case 6: return launch_staged_R<6, WMODE, PREC>(m, ts, sa, grid, threads, smem, out, err, st);
    case 7: return launch_staged_R<7, WMODE, PREC>(m, ts, sa, grid, threads, smem, out, err, st);
    case 8: return launch_staged_R<8, WMODE, PREC>(m, ts, sa, grid, threads, smem, out, err, st);
    case 9: return launch_staged_R<9, WMODE, PREC>(m, ts, sa, grid, threads, smem, out, err, st);
    case 10: return launch_staged_R<10, WMODE, PREC>(m, ts, sa, grid, threads, smem, out, err, st);
    case 11: return launch_staged_R<11, WMODE, PREC>(m, ts, sa, grid, threads, smem, out, err, st);
    case 12:
        if (WMODE == WMODE_CONST)
            return launch_staged_R<12, WMODE_CONST, PREC>(m, ts, sa, grid, threads, smem, out, err, st);
        return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
    }
}

template <int PREC>
cudaError_t launch_staged_P(int R, const MapDev &m, const TrackSet &ts, const StagedArgs &sa, int grid, int threads,
                            size_t smem, float *out, int *err, cudaStream_t st)
{
    switch (m.wmode) {
    case WMODE_CONST: return launch_staged_W<WMODE_CONST, PREC>(R, m, ts, sa, grid, threads, smem, out, err, st);
    case WMODE_FREQ: return launch_staged_W<WMODE_FREQ, PREC>(R, m, ts, sa, grid, threads, smem, out, err, st);
    default: return launch_staged_W<WMODE_PIXEL, PREC>(R, m, ts, sa, grid, threads, smem, out, err, st);
    }
}

template <int WMODE, int PREC, bool EXPLICIT>
cudaError_t launch_simple_W(const MapDev &m, const TrackSet &ts, const uint32_t *f3, const double *tau, uint64_t n,
                            float *out, int *err, cudaStream_t st)
{
    const int threads = 256;
    const uint64_t blocks = (n + threads - 1) / threads;
    if (blocks > 0x7fffffffull) return cudaErrorInvalidValue;
    if (m.fast32)
        score_simple_kernel<WMODE, PREC, EXPLICIT, true>
            <<<(unsigned)blocks, threads, 0, st>>>(m, ts, f3, tau, n, out, err);
    else
        score_simple_kernel<WMODE, PREC, EXPLICIT, false>
            <<<(unsigned)blocks, threads, 0, st>>>(m, ts, f3, tau, n, out, err);
    return cudaGetLastError();
}

template <int PREC, bool EXPLICIT>
cudaError_t launch_simple_P(const MapDev &m, const TrackSet &ts, const uint32_t *f3, const double *tau, uint64_t n,
                            float *out, int *err, cudaStream_t st)
{
    switch (m.wmode) {
    case WMODE_CONST: return launch_simple_W<WMODE_CONST, PREC, EXPLICIT>(m, ts, f3, tau, n, out, err, st);
    case WMODE_FREQ: return launch_simple_W<WMODE_FREQ, PREC, EXPLICIT>(m, ts, f3, tau, n, out, err, st);
    default: return launch_simple_W<WMODE_PIXEL, PREC, EXPLICIT>(m, ts, f3, tau, n, out, err, st);
    }
}

template <bool EXPLICIT>
cudaError_t launch_simple(const MapDev &m, const TrackSet &ts, const uint32_t *f3, const double *tau, uint64_t n,
                          float *out, int *err, cudaStream_t st)
{
    if (m.prec == PREC_FP16) return launch_simple_P<PREC_FP16, EXPLICIT>(m, ts, f3, tau, n, out, err, st);
    return launch_simple_P<PREC_FP32, EXPLICIT>(m, ts, f3, tau, n, out, err, st);
}

// ------------------------------------------------------------------ FP32 -> FP64 output
__global__ void __launch_bounds__(256) widen_kernel(const float *__restrict__ in, double *__restrict__ out,
                                                    uint64_t n)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) out[i] = (double)in[i];
}

// ------------------------------------------------------------------ template-params kernel
// f_out[0..2] control bins, f_out[3..5] control times (general templates; else 0, M/2, M),
// *tau_out the delay, bins[n_t] the pixels (-1 outside a general template's span).
__global__ void track_params_kernel(MapDev m, TrackSet ts, uint64_t g, uint32_t *f_out, double *tau_out,
                                    int32_t *bins)
{
    uint32_t f[3], t[3] = {0u, (uint32_t)(m.n_t - 1) / 2, (uint32_t)(m.n_t - 1)};
    double tau;
    draw_track_ts(ts, g, (uint32_t)m.n_f, f, tau);
    if (ts.general) draw_times(ts.seed, g, (uint32_t)m.n_t, (uint32_t)ts.t_min, t);
    if (threadIdx.x == 0) {
        f_out[0] = f[0]; f_out[1] = f[1]; f_out[2] = f[2];
        f_out[3] = t[0]; f_out[4] = t[1]; f_out[5] = t[2];
        *tau_out = tau;
    }
    if (!bins) return;
    if (!ts.general) {
        for (int j = threadIdx.x; j < m.n_t; j += blockDim.x)
            bins[j] = (int32_t)raster_bin_wide(f[0], f[1], f[2], m.M, (uint32_t)j, m.d);
        return;
    }
    for (int j = threadIdx.x; j < m.n_t; j += blockDim.x)
        if (j < (int)t[0] || j > (int)t[2]) bins[j] = -1;
    if (threadIdx.x == 0) {   // the rasteriser walks the columns in order
        const GenCurve c = gen_curve(t, f);
        const GenFilter gf = gen_filter(c);
        int32_t b = (int32_t)f[0];
        for (int j = (int)t[0]; j <= (int)t[2]; ++j) {
            if (j > (int)t[0]) b = gen_pixel(c, gf, j, m.n_f);
            bins[j] = b;
        }
    }
}

}  // namespace

bool score_wants_order(const MapDev &m, const TrackSet &ts, const Tuning &tu)
{
    if (!tu.order) return false;
    if (ts.general) return ts.n * (uint64_t)m.n_t >= (1ull << 22);  // general-template kernel
    if (!m.fast32 || tu.kernel == 1 || m.n_f > kPhaseNarrowNf) return false;
    return tu.kernel == 2 || ts.n * (uint64_t)m.n_t >= (1ull << 24);
}

cudaError_t launch_score_generated(const MapDev &m, const TrackSet &ts, float *out, int *err, const Tuning &tu,
                                   int num_sms, size_t smem_optin, cudaStream_t st, ScorePlan *plan,
                                   void *order_scratch, cudaEvent_t order_done)
{
    ScorePlan p{};
    const uint64_t n = ts.n;
    if (ts.general) {
        p.kernel = 3;
        p.threads = 256;
        p.grid = (int)std::min<uint64_t>((n + 255) / 256, 0x7fffffffull);
        const uint32_t *perm = nullptr;
        if (order_scratch && score_wants_order(m, ts, tu)) {
            cudaError_t e = launch_order(m, ts, order_scratch, num_sms, st, &perm, &p.order_launches);
            if (e != cudaSuccess) return e;
            p.order = 1;
        }
        if (plan) *plan = p;
        if (order_done && cudaEventRecord(order_done, st) != cudaSuccess) return cudaGetLastError();
        return launch_general<false>(m, ts, nullptr, nullptr, nullptr, n, out, err, st, perm);
    }
    const uint64_t work = n * (uint64_t)m.n_t;
    int kernel = tu.kernel;
    if (kernel == 0) kernel = (!m.fast32 || work < (1ull << 24)) ? 1 : 2;
    if (kernel == 2 && (!m.fast32 || m.n_f > kPhaseNarrowNf)) kernel = 1;  // slab kernel: narrow phase form

    if (kernel == 2) {
        const size_t row_bytes = (size_t)m.ldr * (m.prec == PREC_FP16 ? 4 : 8);
        const size_t wrow_bytes = m.wmode == WMODE_PIXEL ? (size_t)m.ldw * 4 : 0;
        const size_t wtab_bytes = m.wmode == WMODE_FREQ ? (size_t)((m.n_f + 3) / 4 * 4) * 4 : 0;
        size_t budget = smem_optin;
        if (tu.smem_kb > 0) budget = std::min(budget, (size_t)tu.smem_kb * 1024);
        const int nstage = std::max(2, std::min(tu.nstage, 4));
        const size_t fixed = wtab_bytes + kStagedBookkeeping;
        long S = budget > fixed ? (long)((budget - fixed) / (nstage * (row_bytes + wrow_bytes))) : 0;
        S = std::min<long>(S, m.n_t);
        if (S < 1) {
            kernel = 1;  // a single map row does not fit in shared memory
        } else {
            // templates held per thread: up to 6 fit 64 registers without a weight sum,
            // 5 with one (1024 threads); 7 to 12 (11 with a weight sum) fit 128 registers
            // (512 threads) and run a few per cent faster, the default
            const int maxR = tu.max_R > 6 ? std::min(tu.max_R, m.wmode == WMODE_CONST ? 12 : 11)
                                          : std::max(1, std::min(tu.max_R, m.wmode == WMODE_CONST ? 6 : 5));
            const int tmax = maxR > 6 ? 512 : kMaxThreads;
            const uint64_t cap = (uint64_t)maxR * tmax;
            const uint64_t G = (uint64_t)std::max(1, num_sms);
            const uint64_t per_cta = (n + G - 1) / G;
            const uint64_t nb_per_cta = std::max<uint64_t>(1, (per_cta + cap - 1) / cap);
            uint64_t nb = G * nb_per_cta;
            uint64_t batch = (n + nb - 1) / nb;
            if (batch < 32) batch = 32;
            nb = (n + batch - 1) / batch;
            int R, threads;
            if (tu.threads > 0) {
                threads = std::min(tmax, (tu.threads + 31) / 32 * 32);
                R = (int)((batch + threads - 1) / threads);
                if (R > maxR) {  // requested block too small for the batch: shrink the batch
                    R = maxR;
                    batch = (uint64_t)R * threads;
                    nb = (n + batch - 1) / batch;
                }
            } else {
                R = (int)std::min<uint64_t>((batch + tmax - 1) / tmax, (uint64_t)maxR);
                threads = (int)(((batch + R - 1) / R + 31) / 32 * 32);
            }
            p.kernel = 2;
            p.R = R;
            p.threads = threads;
            p.grid = (int)std::min<uint64_t>(G, nb);
            p.S = (int)S;
            p.nstage = nstage;
            p.nslabs = (int)((m.n_t + S - 1) / S);
            p.batch = batch;
            p.nbatches = nb;
            p.smem = (size_t)nstage * S * (row_bytes + wrow_bytes) + wtab_bytes + kStagedBookkeeping;
            StagedArgs sa;
            sa.S = (int)S;
            sa.nstage = nstage;
            sa.nslabs = p.nslabs;
            sa.batch = batch;
            sa.nbatches = nb;
            sa.slab_recs = (uint32_t)(S * m.ldr);
            sa.slab_ws = m.wmode == WMODE_PIXEL ? (uint32_t)(S * m.ldw) : 0u;
            sa.wtab_floats = m.wmode == WMODE_FREQ ? (uint32_t)((m.n_f + 3) / 4 * 4) : 0u;
            sa.wait_ns = tu.wait_ms > 0 ? (uint64_t)tu.wait_ms * 1000000ull : kWaitLimitNs;
            sa.withhold_q = tu.withhold_slab >= 0 ? (uint64_t)tu.withhold_slab : ~0ull;
            sa.perm = nullptr;
            if (order_scratch && score_wants_order(m, ts, tu)) {
                cudaError_t e = launch_order(m, ts, order_scratch, num_sms, st, &sa.perm, &p.order_launches);
                if (e != cudaSuccess) return e;
                p.order = 1;
            }
            if (order_done) {
                cudaError_t e = cudaEventRecord(order_done, st);
                if (e != cudaSuccess) return e;
            }
            if (plan) *plan = p;
            if (m.prec == PREC_FP16)
                return launch_staged_P<PREC_FP16>(R, m, ts, sa, p.grid, threads, p.smem, out, err, st);
            return launch_staged_P<PREC_FP32>(R, m, ts, sa, p.grid, threads, p.smem, out, err, st);
        }
    }
    p.kernel = 1;
    p.threads = 256;
    p.grid = (int)std::min<uint64_t>((n + 255) / 256, 0x7fffffffull);
    if (plan) *plan = p;
    if (order_done) {
        cudaError_t e = cudaEventRecord(order_done, st);
        if (e != cudaSuccess) return e;
    }
    return launch_simple<false>(m, ts, nullptr, nullptr, n, out, err, st);
}

cudaError_t launch_score_explicit(const MapDev &m, const uint32_t *f3, const double *tau, uint64_t n, float *out,
                                  int *err, cudaStream_t st)
{
    TrackSet ts{};
    return launch_simple<true>(m, ts, f3, tau, n, out, err, st);
}

cudaError_t launch_score_explicit_general(const MapDev &m, const uint32_t *t3, const uint32_t *f3, const double *tau,
                                          uint64_t n, float *out, int *err, cudaStream_t st)
{
    TrackSet ts{};
    return launch_general<true>(m, ts, t3, f3, tau, n, out, err, st);
}

cudaError_t launch_widen(const float *in, double *out, uint64_t n, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const uint64_t blocks = (n + 255) / 256;
    widen_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(in, out, n);
    return cudaGetLastError();
}

cudaError_t launch_track_params(const MapDev &m, const TrackSet &ts, uint64_t g, uint32_t *f_dev, double *tau_dev,
                                int32_t *bins_dev, cudaStream_t st)
{
    track_params_kernel<<<1, 256, 0, st>>>(m, ts, g, f_dev, tau_dev, bins_dev);
    return cudaGetLastError();
}

}  // namespace stk
