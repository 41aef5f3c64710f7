// Many ft-maps of uneven size scored in one persistent launch.
//
// The paper's searches cut long data into many maps and score each with its
// own template set, recording every map's loudest SNR (Sec. V, Eqs. 9-10: time
// windows and n_ts unphysical time shifts per window).  A batch runs them all
// in one kernel:
//   - the work is a list of tiles (map, block of R * blockDim positions) in
//     schedule order, largest maps first; CTAs take tiles from a global work
//     counter, so ragged maps balance across the GPU;
//   - each tile streams its map through shared memory in slabs (bulk copies on
//     mbarriers with bounded waits, as in the single-map kernel) and keeps its
//     k loudest templates (warp, then block, repeated arg-max);
//   - a second kernel ranks each map's tile candidates and writes its k hits.
// Before taking a tile a CTA reads a cancel flag in host-mapped memory.  The
// launch sequence is captured once in a CUDA graph and replayed.  Every
// template's SNR is computed with the same per-pixel arithmetic as the
// single-map kernels.  The division by 2 M^2 is the map's exact multiply-shift
// when it has one, else a multiply-shift with one correction step (exact for all
// numerators below 2^32).  Each map's templates are scored in coherent
// order (one sort over all maps, run inside the graph before the tiles).
#include <algorithm>
#include <cmath>
#include <vector>

#include "stk_internal.cuh"
#include "stk_objects.cuh"
#include "stk_pixel.cuh"

using namespace stk;

namespace {

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s per slab wait
constexpr int kMaxWarps = 32;
constexpr int kRankChunk = 64;
constexpr int kRankTile = 1024;
constexpr int kBatchStages = 4;            // most slab buffers
constexpr size_t kBatchBookkeeping = 128;  // barriers, last issued slab, finished warps, abort flag
static_assert(kBatchStages * (8 + 8 + 4) + 4 <= kBatchBookkeeping, "bookkeeping block too small");

struct BatchMap {
    MapDev m;
    TrackSet ts;
    uint32_t magic;   // exact multiply-shift (fast), else ceil(2^(32+shift) / d) with one correction
    int shift;
    int fast;
    uint32_t d32;     // 2 M^2
    int S;            // time columns per slab
    int nslabs;
    uint32_t ntiles;  // template blocks of this map
    uint32_t tile0;   // first candidate block of this map (map-major order)
    uint32_t pos0;    // first position of this map in the scoring order
};

struct BatchArgs {
    const BatchMap *maps;
    const uint2 *sched;     // (map, block) in schedule order
    uint32_t ntiles;        // tiles to run (a prefix of the schedule)
    unsigned int *counter;  // work counter, zero before the launch
    const volatile int *cancel;
    int nstage;
    uint32_t slot_bytes;    // bytes per slab buffer: record rows, then weight rows
    uint32_t wtab_floats;   // per-frequency weight table capacity
    uint32_t tile;          // templates per tile = R * blockDim
    int K;
    unsigned long long *cand_key;  // [all tiles][K]
    unsigned int *cand_idx;
    int *err;
    const uint32_t *perm;   // coherent order: position pos0 + p of map i holds its template perm[.] (NULL: index order)
};

// One slab of one tile: rows time columns for the R templates of this thread.
// rb, wb: shared addresses of the slab's first record row and weight row, swt_a
// of the per-frequency weight table.  Columns go in pairs (three rasteriser
// additions per two columns, exact mod 2^32), each template's sums in column order.
// Debug build: hull[r] = the template's bins (lo | hi << 16), j0 the slab's first
// column, n_t the map's columns, err the flag word.
template <int R, int WMODE, int PREC, bool FAST>
__device__ __forceinline__ void batch_slab(uint32_t rb, uint32_t wb, uint32_t swt_a, int rows, uint32_t row_bytes,
                                           uint32_t wrow_bytes, uint32_t magic, int shift, uint32_t d32,
                                           uint32_t (&N)[R], uint32_t (&D)[R], const uint32_t (&D2)[R],
                                           const uint32_t (&pa)[R], const uint32_t (&pc)[R], float (&acc)[R],
                                           float (&W)[R], const uint32_t *hull, int j0, int n_t, int *err)
{
    using Rec = typename Pix<PREC>::Rec;
    auto col = [&](int r, uint32_t Nv, uint32_t rb_, uint32_t wb_, int jcol) {
        uint32_t b = FAST ? __umulhi(Nv, magic) >> shift : div_corrected(Nv, magic, shift, d32);
        if (kDebugBounds) b = checked_bin(b, jcol, n_t, hull[r] & 0xffffu, hull[r] >> 16, err);
        const Rec v = Pix<PREC>::load_shared(rb_ + (b << Pix<PREC>::kLog2Bytes));
        float wv = 0.f;
        if (WMODE == WMODE_FREQ) wv = lds_f32(swt_a + (b << 2));
        if (WMODE == WMODE_PIXEL) wv = lds_f32(wb_ + (b << 2));
        pixel_add<PREC, WMODE>(v, template_turn_narrow(b, pa[r], pc[r]), wv, acc[r], W[r]);
    };
    int jj = 0;
    for (; jj + 1 < rows; jj += 2) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint32_t Na = N[r], Nb = Na + D[r];
            col(r, Na, rb, wb, j0 + jj);
            col(r, Nb, rb + row_bytes, wb + wrow_bytes, j0 + jj + 1);
            N[r] = Nb + D[r] + D2[r];
            D[r] = D[r] + D2[r] + D2[r];
        }
        rb += 2 * row_bytes;
        wb += 2 * wrow_bytes;
    }
    if (jj < rows) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            col(r, N[r], rb, wb, j0 + jj);
            N[r] += D[r];
            D[r] += D2[r];
        }
    }
}

// Up to 5 templates per thread fit 64 registers (1024 threads); 6 to 11 need up
// to 128 (512 threads).
constexpr int batch_max_threads(int R) { return R <= 5 ? 1024 : 512; }

template <int R, int WMODE, int PREC>
__global__ void __launch_bounds__(batch_max_threads(R), 1) score_batch_kernel(BatchArgs a)
{
    using Rec = typename Pix<PREC>::Rec;
    extern __shared__ __align__(128) unsigned char smem[];
    // bookkeeping first (fixed offsets), then slab buffers, weight table, tile candidates
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);                // full barrier per buffer
    uint64_t *issued = bars + kBatchStages;                              // last slab issued into each buffer
    uint32_t *done = reinterpret_cast<uint32_t *>(issued + kBatchStages);  // warps finished with each buffer
    int *abort_flag = reinterpret_cast<int *>(done + kBatchStages);
    unsigned char *slabs = smem + kBatchBookkeeping;
    float *swt = reinterpret_cast<float *>(slabs + (size_t)a.nstage * a.slot_bytes);
    const uint32_t slabs_a = smem_u32(slabs), swt_a = smem_u32(swt);
    unsigned long long *ck = reinterpret_cast<unsigned long long *>(swt + a.wtab_floats);
    unsigned int *ci = reinterpret_cast<unsigned int *>(ck + kMaxWarps * a.K);
    __shared__ unsigned int sh_tile;

    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
    const int K = a.K;
    if (tid == 0) {
        for (int s = 0; s < a.nstage; ++s) {
            mbar_init(&bars[s], 1);
            issued[s] = ~0ull;
            done[s] = 0u;
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();

    uint64_t q = 0;       // slab sequence number over all tiles of this CTA
    int slot = 0;         // q % nstage
    uint32_t parity = 0;  // (q / nstage) & 1
    int cur_map = -1;
    while (true) {
        if (tid == 0) {
            unsigned int t = atomicAdd(a.counter, 1u);
            if (*a.cancel) {
                atomicOr(a.err, ERR_CANCELED);
                t = 0xffffffffu;
            }
            sh_tile = t;
        }
        __syncthreads();
        const unsigned int t = sh_tile;
        if (t >= a.ntiles) break;
        const uint2 tb = a.sched[t];
        // per-map values: the loop's scalars in registers, the rest read where used
        const BatchMap *bm = a.maps + tb.x;
        const int n_t = bm->m.n_t, ldr = bm->m.ldr, ldw = bm->m.ldw;
        const uint32_t magic = bm->magic, d32 = bm->d32;
        const int shift = bm->shift, S = bm->S, nslabs = bm->nslabs;
        const bool fast = bm->fast != 0;
        if (WMODE == WMODE_FREQ && (int)tb.x != cur_map) {
            const int n_f = bm->m.n_f;
            const float *w = bm->m.w;
            for (int k = tid; k < n_f; k += nthr) swt[k] = w[k];
            __syncthreads();
        }
        cur_map = (int)tb.x;
        const uint64_t t0 = (uint64_t)tb.y * a.tile;
        const uint64_t nt_map = bm->ts.n;
        const uint64_t tn = (nt_map - t0) < a.tile ? (nt_map - t0) : a.tile;

        // slab sl of this tile (sequence number qq) into buffer bslot
        auto issue = [&](uint64_t qq, int bslot, int sl) {
            const uint32_t row_bytes = (uint32_t)ldr * (uint32_t)sizeof(Rec);
            const uint32_t wrow_bytes = (uint32_t)ldw * 4u;
            const int row0 = sl * S;
            const int rows = min(S, n_t - row0);
            unsigned char *dst = slabs + (size_t)bslot * a.slot_bytes;
            uint32_t bytes = (uint32_t)rows * row_bytes;
            if (WMODE == WMODE_PIXEL) bytes += (uint32_t)rows * wrow_bytes;
            issued[bslot] = qq;
            mbar_arrive_expect_tx(&bars[bslot], bytes);
            const Rec *grec = reinterpret_cast<const Rec *>(bm->m.rec);
            bulk_g2s(dst, grec + (size_t)row0 * ldr, (uint32_t)rows * row_bytes, &bars[bslot]);
            if (WMODE == WMODE_PIXEL)
                bulk_g2s(dst + (size_t)S * row_bytes, bm->m.w + (size_t)row0 * ldw, (uint32_t)rows * wrow_bytes,
                         &bars[bslot]);
        };
        if (tid == 0) {
            const int pre = min(a.nstage, nslabs);
            int bs = slot;
            for (int s = 0; s < pre; ++s) {
                issue(q + s, bs, s);
                if (++bs == a.nstage) bs = 0;
            }
        }

        uint32_t N[R], D[R], D2[R];
        uint32_t pa[R], pc[R];  // narrow phase form (n_f <= kPhaseNarrowNf)
        float acc[R], W[R];
        uint32_t hull[kDebugBounds ? R : 1];  // debug build: each template's bins, lo | hi << 16
#pragma unroll
        for (int r = 0; r < R; ++r) {
            uint64_t i = (uint64_t)tid + (uint64_t)r * nthr;
            if (i >= tn) i = tn - 1;  // idle slot: repeat a valid template, result discarded
            const uint64_t rel = a.perm ? (uint64_t)__ldg(a.perm + bm->pos0 + t0 + i) : t0 + i;
            uint32_t f[3];
            double tau;
            draw_track(bm->ts.seed, bm->ts.offset + rel, (uint32_t)bm->m.n_f, bm->ts.tau_max, f, tau);
            if (kDebugBounds) hull[kDebugBounds ? r : 0] = hull_lo(f) | (hull_hi(f) << 16);
            const Raster32 rs = raster_init(f[0], f[1], f[2], (uint32_t)(n_t - 1));
            N[r] = rs.N; D[r] = rs.D; D2[r] = rs.D2;
            const Phase ph = phase_consts(bm->m.f_min, bm->m.df, tau, bm->m.n_f);
            pa[r] = ph.a;
            pc[r] = ph.c;
            acc[r] = 0.f;
            W[r] = 0.f;
        }

        for (int s = 0; s < nslabs; ++s, ++q) {
            const bool ok = __all_sync(0xffffffffu, mbar_wait(&bars[slot], parity, kWaitLimitNs)) &&
                            !*(volatile int *)abort_flag;
            if (!ok) {
                if (lane == 0) atomicOr(abort_flag, 1);
                break;
            }
            const int rows = min(S, n_t - s * S);
            const uint32_t row_bytes = (uint32_t)ldr * (uint32_t)sizeof(Rec);
            const uint32_t wrow_bytes = WMODE == WMODE_PIXEL ? (uint32_t)ldw * 4u : 0u;
            const uint32_t rb = slabs_a + (uint32_t)slot * a.slot_bytes;
            const uint32_t wb = rb + (uint32_t)S * row_bytes;
            if (fast)
                batch_slab<R, WMODE, PREC, true>(rb, wb, swt_a, rows, row_bytes, wrow_bytes, magic, shift, d32, N, D,
                                                 D2, pa, pc, acc, W, hull, s * S, n_t, a.err);
            else
                batch_slab<R, WMODE, PREC, false>(rb, wb, swt_a, rows, row_bytes, wrow_bytes, magic, shift, d32, N,
                                                  D, D2, pa, pc, acc, W, hull, s * S, n_t, a.err);
            // This warp is done with the buffer; the last warp to finish refills it.
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();
                if (atomicAdd(&done[slot], 1u) == (uint32_t)nwarps - 1u) {
                    done[slot] = 0u;
                    __threadfence_block();
                    fence_proxy_async_smem();
                    if (s + a.nstage < nslabs) issue(q + a.nstage, slot, s + a.nstage);
                }
            }
            if (++slot == a.nstage) {
                slot = 0;
                parity ^= 1u;
            }
        }
        __syncthreads();
        if (*(volatile int *)abort_flag) break;  // read after the barrier: the same for every thread

        // this tile's K loudest: repeated arg-max, per warp and then over the warps
        unsigned long long key[R];
        unsigned int idx[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint64_t i = (uint64_t)tid + (uint64_t)r * nthr;
            const bool valid = i < tn;
            const uint64_t rel = valid ? (a.perm ? (uint64_t)__ldg(a.perm + bm->pos0 + t0 + i) : t0 + i) : 0ull;
            key[r] = valid ? order_key(finalize_snr<WMODE>(acc[r], W[r], bm->m)) : 0ull;
            idx[r] = valid ? (unsigned int)rel : 0xffffffffu;
        }
        for (int it = 0; it < K; ++it) {
            unsigned long long bk = 0ull;
            unsigned int bi = 0xffffffffu;
            int br = -1;
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (before(key[r], idx[r], bk, bi)) { bk = key[r]; bi = idx[r]; br = r; }
            unsigned long long wk = bk;
            unsigned int wi = bi;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long ok2 = __shfl_xor_sync(0xffffffffu, wk, o);
                const unsigned int oi = __shfl_xor_sync(0xffffffffu, wi, o);
                if (before(ok2, oi, wk, wi)) { wk = ok2; wi = oi; }
            }
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (r == br && key[r] == wk && idx[r] == wi) { key[r] = 0ull; idx[r] = 0xffffffffu; }
            if (lane == 0) {
                ck[warp * K + it] = wk;
                ci[warp * K + it] = wi;
            }
        }
        __syncthreads();
        if (warp == 0) {
            const int ne = nwarps * K;
            const size_t out0 = (size_t)(bm->tile0 + tb.y) * K;
            for (int it = 0; it < K; ++it) {
                unsigned long long bk = 0ull;
                unsigned int bi = 0xffffffffu;
                int bp = -1;
                for (int e = lane; e < ne; e += 32)
                    if (before(ck[e], ci[e], bk, bi)) { bk = ck[e]; bi = ci[e]; bp = e; }
                unsigned long long wk = bk;
                unsigned int wi = bi;
                int wp = bp;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const unsigned long long ok2 = __shfl_xor_sync(0xffffffffu, wk, o);
                    const unsigned int oi = __shfl_xor_sync(0xffffffffu, wi, o);
                    const int op = __shfl_xor_sync(0xffffffffu, wp, o);
                    if (before(ok2, oi, wk, wi)) { wk = ok2; wi = oi; wp = op; }
                }
                if (lane == 0) {
                    a.cand_key[out0 + it] = wk;
                    a.cand_idx[out0 + it] = wi;
                }
                if (wp >= 0 && bp == wp) {
                    ck[wp] = 0ull;
                    ci[wp] = 0xffffffffu;
                }
                __syncwarp();
            }
        }
        // the next tile's fetch barrier orders the reuse of ck / ci and the slab buffers
    }
    // Copies already issued must land before the CTA's shared memory goes away
    // (after a timeout some may still be in flight); each wait is bounded.
    __syncthreads();
    if (tid == 0) {
        if (*(volatile int *)abort_flag) atomicOr(a.err, ERR_TIMEOUT);
        for (int s = 0; s < a.nstage; ++s)
            if (issued[s] != ~0ull)
                mbar_wait(&bars[s], (uint32_t)((issued[s] / (uint64_t)a.nstage) & 1ull), kWaitLimitNs);
    }
}

// Map i's candidates: rank = number of its candidates ordered before; ranks
// below K write hit i*K + rank.  grid = (chunks of 64 candidates, maps).
__global__ void __launch_bounds__(256) batch_rank_kernel(const BatchMap *__restrict__ maps, int K,
                                                         const unsigned long long *__restrict__ cand_key,
                                                         const unsigned int *__restrict__ cand_idx, stk_hit *out)
{
    __shared__ unsigned int part[4][kRankChunk];
    __shared__ unsigned long long tk[kRankTile];
    __shared__ unsigned int ti[kRankTile];
    const BatchMap *bm = maps + blockIdx.y;
    const unsigned int nc = bm->ntiles * (unsigned int)K;
    const size_t base = (size_t)bm->tile0 * K;
    const unsigned int c0 = blockIdx.x * kRankChunk;
    if (c0 >= nc) return;
    const int c = threadIdx.x & (kRankChunk - 1), qd = threadIdx.x / kRankChunk;
    const unsigned int me = c0 + c;
    const bool valid = me < nc;
    const unsigned long long mk = valid ? cand_key[base + me] : 0ull;
    const unsigned int mi = valid ? cand_idx[base + me] : 0xffffffffu;
    unsigned int before_me = 0;
    for (unsigned int t0 = 0; t0 < nc; t0 += kRankTile) {
        const unsigned int tn = min((unsigned int)kRankTile, nc - t0);
        for (unsigned int j = threadIdx.x; j < tn; j += blockDim.x) {
            tk[j] = cand_key[base + t0 + j];
            ti[j] = cand_idx[base + t0 + j];
        }
        __syncthreads();
        for (unsigned int j = qd; j < tn; j += 4) before_me += before(tk[j], ti[j], mk, mi) ? 1u : 0u;
        __syncthreads();
    }
    part[qd][c] = before_me;
    __syncthreads();
    if (qd == 0 && valid && mk != 0ull) {
        const unsigned int rank = part[0][c] + part[1][c] + part[2][c] + part[3][c];
        if (rank < (unsigned int)K) {
            stk_hit h;
            uint32_t f[3];
            double tau;
            draw_track(bm->ts.seed, bm->ts.offset + mi, (uint32_t)bm->m.n_f, bm->ts.tau_max, f, tau);
            h.snr = (double)snr_from_key(mk);  // the SNR back from its order-preserving key
            h.index = bm->ts.offset + mi;
            h.f[0] = f[0]; h.f[1] = f[1]; h.f[2] = f[2];
            h.reserved = 0;
            h.tau = tau;
            out[(size_t)blockIdx.y * K + rank] = h;
        }
    }
}

// set_attr: raise the kernel's dynamic shared-memory limit first (not allowed while
// a stream is being captured, so the capture path relies on an earlier launch).
template <int R, int WMODE, int PREC>
cudaError_t launch_batch_R(const BatchArgs &a, int grid, int threads, size_t smem, bool set_attr, cudaStream_t st)
{
    auto k = score_batch_kernel<R, WMODE, PREC>;
    if (threads > batch_max_threads(R)) return cudaErrorInvalidConfiguration;
    if (set_attr) {
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, k);
        if (e != cudaSuccess) return e;
        int dev = 0, optin = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
            return e;
        if (smem + fa.sharedSizeBytes > (size_t)optin) return cudaErrorInvalidConfiguration;
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<grid, threads, smem, st>>>(a);
    return cudaGetLastError();
}

template <int WMODE, int PREC>
cudaError_t launch_batch_W(int R, const BatchArgs &a, int grid, int threads, size_t smem, bool sa, cudaStream_t st)
{
    switch (R) {
    case 1: return launch_batch_R<1, WMODE, PREC>(a, grid, threads, smem, sa, st);
    case 2: return launch_batch_R<2, WMODE, PREC>(a, grid, threads, smem, sa, st);
    case 3: return launch_batch_R<3, WMODE, PREC>(a, grid, threads, smem, sa, st);
    case 4: return launch_batch_R<4, WMODE, PREC>(a, grid, threads, smem, sa, st);
    case 5: return launch_batch_R<5, WMODE, PREC>(a, grid, threads, smem, sa, st);
    case 6: return launch_batch_R<6, WMODE, PREC>(a, grid, threads, smem, sa, st);
    case 8: return launch_batch_R<8, WMODE, PREC>(a, grid, threads, smem, sa, st);
    case 10: return launch_batch_R<10, WMODE, PREC>(a, grid, threads, smem, sa, st);
    case 11: return launch_batch_R<11, WMODE, PREC>(a, grid, threads, smem, sa, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_batch(int wmode, int prec, int R, const BatchArgs &a, int grid, int threads, size_t smem,
                         bool sa, cudaStream_t st)
{
    if (prec == PREC_FP16) {
        if (wmode == WMODE_CONST) return launch_batch_W<WMODE_CONST, PREC_FP16>(R, a, grid, threads, smem, sa, st);
        if (wmode == WMODE_FREQ) return launch_batch_W<WMODE_FREQ, PREC_FP16>(R, a, grid, threads, smem, sa, st);
        return launch_batch_W<WMODE_PIXEL, PREC_FP16>(R, a, grid, threads, smem, sa, st);
    }
    if (wmode == WMODE_CONST) return launch_batch_W<WMODE_CONST, PREC_FP32>(R, a, grid, threads, smem, sa, st);
    if (wmode == WMODE_FREQ) return launch_batch_W<WMODE_FREQ, PREC_FP32>(R, a, grid, threads, smem, sa, st);
    return launch_batch_W<WMODE_PIXEL, PREC_FP32>(R, a, grid, threads, smem, sa, st);
}

// ceil(2^(32+s) / d) < 2^32 for the largest such s (d >= 2).
bool corrected_magic(uint64_t d, uint32_t &magic, int &shift)
{
    for (int s = 31; s >= 0; --s) {
        const unsigned __int128 p2 = (unsigned __int128)1 << (32 + s);
        const unsigned __int128 mm = (p2 + d - 1) / d;
        if (mm < ((unsigned __int128)1 << 32)) {
            magic = (uint32_t)mm;
            shift = s;
            return true;
        }
    }
    return false;
}

}  // namespace

struct stk_batch {
    stk_ctx *ctx = nullptr;
    int n_maps = 0;
    std::vector<const stk_map *> maps;
    std::vector<BatchMap> hmaps;
    int wmode = 0, prec = 0;
    // launch shape
    int threads = 1024, R = 5, nstage = 2;
    uint32_t tile = 0, slot_bytes = 0, wtab_floats = 0;
    size_t smem = 0;
    uint32_t ntiles_total = 0;
    uint32_t max_ntiles = 0;  // most tiles of any one map
    // device
    BatchMap *d_maps = nullptr;
    uint2 *d_sched = nullptr;
    unsigned int *d_counter = nullptr;
    int *h_cancel = nullptr, *d_cancel = nullptr;
    unsigned long long *d_ckey = nullptr;
    unsigned int *d_cidx = nullptr;
    size_t cand_cap = 0;
    stk_hit *d_hits = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int graph_k = 0;
    // coherent order (one bucket sort over all maps, run in every scoring call)
    bool use_order = false;
    OrderMap *d_omaps = nullptr;
    void *order_buf = nullptr;
    uint64_t total_n = 0, max_n = 0;
    uint32_t order_nc = 0, order_fbits = 0;  // coarse buckets, most fine bits of a map
    const uint32_t *d_perm = nullptr;
};

namespace {

void drop_graph(stk_batch *b)
{
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->gexec = nullptr;
    b->graph = nullptr;
    b->graph_k = 0;
}

// Lay out tiles, slabs and buffers for a launch shape; uploads the map table and schedule.
int configure(stk_batch *b, int threads, int R, int nstage)
{
    stk_ctx *c = b->ctx;
    const size_t rec_bytes = b->prec == PREC_FP16 ? 4 : 8;
    uint32_t max_nf = 0;
    for (auto *m : b->maps) max_nf = std::max<uint32_t>(max_nf, (uint32_t)m->dev.n_f);
    const uint32_t wtab = b->wmode == WMODE_FREQ ? (max_nf + 3) / 4 * 4 : 0;
    // room for the kernel's own static shared memory (the tile index, aligned) and slack
    const size_t fixed = kBatchBookkeeping + (size_t)wtab * 4 + (size_t)kMaxWarps * STK_BATCH_MAX_K * 12 + 1024;
    if (c->smem_optin <= fixed) return set_err(c, STK_EINVAL, "shared memory too small for the batch");
    const uint32_t slot = (uint32_t)((c->smem_optin - fixed) / nstage / 16 * 16);
    const uint32_t tile = (uint32_t)(R * threads);
    uint32_t tile0 = 0;
    std::vector<BatchMap> hm(b->n_maps);
    for (int i = 0; i < b->n_maps; ++i) {
        BatchMap &x = hm[i];
        x = b->hmaps[i];
        const MapDev &m = x.m;
        const size_t rowb = (size_t)m.ldr * rec_bytes + (b->wmode == WMODE_PIXEL ? (size_t)m.ldw * 4 : 0);
        const long S = std::min<long>((long)(slot / rowb), m.n_t);
        if (S < 1) return set_err(c, STK_EINVAL, "map %d: one row (%zu bytes) exceeds a slab buffer", i, rowb);
        x.S = (int)S;
        x.nslabs = (int)((m.n_t + S - 1) / S);
        x.ntiles = (uint32_t)((x.ts.n + tile - 1) / tile);
        x.tile0 = tile0;
        tile0 += x.ntiles;
    }
    // schedule: tiles of the largest maps (most work per tile) first
    std::vector<int> order(b->n_maps);
    for (int i = 0; i < b->n_maps; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int p, int q) { return hm[p].m.n_t > hm[q].m.n_t; });
    std::vector<uint2> sched;
    sched.reserve(tile0);
    for (int i : order)
        for (uint32_t t = 0; t < hm[i].ntiles; ++t) sched.push_back(make_uint2((unsigned)i, t));
    uint32_t max_ntiles = 0;
    for (auto &x : hm) max_ntiles = std::max(max_ntiles, x.ntiles);

    cudaError_t e;
    cudaStreamSynchronize(c->stream);
    cudaFree(b->d_sched);
    b->d_sched = nullptr;
    if ((e = cudaMalloc(&b->d_sched, sizeof(uint2) * sched.size())) != cudaSuccess)
        return set_err(c, STK_ENOMEM, "schedule allocation: %s", cudaGetErrorString(e));
    if (!b->d_maps && (e = cudaMalloc(&b->d_maps, sizeof(BatchMap) * b->n_maps)) != cudaSuccess)
        return set_err(c, STK_ENOMEM, "map table allocation: %s", cudaGetErrorString(e));
    const size_t need = (size_t)tile0 * STK_BATCH_MAX_K;
    if (need > b->cand_cap) {
        cudaFree(b->d_ckey);
        cudaFree(b->d_cidx);
        b->d_ckey = nullptr;
        b->d_cidx = nullptr;
        b->cand_cap = 0;
        if ((e = cudaMalloc(&b->d_ckey, need * 8)) != cudaSuccess ||
            (e = cudaMalloc(&b->d_cidx, need * 4)) != cudaSuccess)
            return set_err(c, STK_ENOMEM, "candidate allocation: %s", cudaGetErrorString(e));
        b->cand_cap = need;
    }
    CUDA_TRY(c, cudaMemcpy(b->d_maps, hm.data(), sizeof(BatchMap) * b->n_maps, cudaMemcpyHostToDevice));
    CUDA_TRY(c, cudaMemcpy(b->d_sched, sched.data(), sizeof(uint2) * sched.size(), cudaMemcpyHostToDevice));
    b->hmaps = hm;
    b->threads = threads;
    b->R = R;
    b->nstage = nstage;
    b->tile = tile;
    b->slot_bytes = slot;
    b->wtab_floats = wtab;
    b->smem = kBatchBookkeeping + (size_t)nstage * slot + (size_t)wtab * 4 + (size_t)kMaxWarps * STK_BATCH_MAX_K * 12;
    b->ntiles_total = tile0;
    b->max_ntiles = max_ntiles;
    drop_graph(b);
    return STK_OK;
}

// The launch sequence: the coherent order (if `order`), zero the work counter,
// run the tiles, merge per map.
cudaError_t enqueue(stk_batch *b, int k, uint32_t ntiles, bool merge, bool set_attr, cudaStream_t st,
                    bool order = true)
{
    if (b->use_order && order) {
        cudaError_t e = launch_order_batch(b->d_omaps, b->n_maps, b->total_n, b->order_nc, b->order_fbits,
                                           b->order_buf, b->ctx->num_sms, st, &b->d_perm, nullptr);
        if (e != cudaSuccess) return e;
    }
    BatchArgs a;
    a.perm = b->use_order ? b->d_perm : nullptr;
    a.maps = b->d_maps;
    a.sched = b->d_sched;
    a.ntiles = ntiles;
    a.counter = b->d_counter;
    a.cancel = b->d_cancel;
    a.nstage = b->nstage;
    a.slot_bytes = b->slot_bytes;
    a.wtab_floats = b->wtab_floats;
    a.tile = b->tile;
    a.K = k;
    a.cand_key = b->d_ckey;
    a.cand_idx = b->d_cidx;
    a.err = b->ctx->d_err;
    cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    e = launch_batch(b->wmode, b->prec, b->R, a, b->ctx->num_sms, b->threads, b->smem, set_attr, st);
    if (e != cudaSuccess || !merge) return e;
    const int chunks = (int)std::max<uint64_t>(1, ((uint64_t)b->max_ntiles * k + kRankChunk - 1) / kRankChunk);
    batch_rank_kernel<<<dim3(chunks, b->n_maps), 256, 0, st>>>(b->d_maps, k, b->d_ckey, b->d_cidx, b->d_hits);
    return cudaGetLastError();
}

int ensure_graph(stk_batch *b, int k)
{
    stk_ctx *c = b->ctx;
    if (b->gexec && b->graph_k == k) return STK_OK;
    drop_graph(b);
    // kernel attributes are set outside the capture
    cudaError_t e = enqueue(b, k, 0, false, true, b->cap_stream, false);
    if (e != cudaSuccess) return set_err(c, STK_ECUDA, "batch warm launch: %s", cudaGetErrorString(e));
    CUDA_TRY(c, cudaStreamSynchronize(b->cap_stream));
    CUDA_TRY(c, cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    e = enqueue(b, k, b->ntiles_total, true, false, b->cap_stream);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return set_err(c, STK_ECUDA, "batch graph capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    b->graph = g;
    CUDA_TRY(c, cudaGraphInstantiate(&b->gexec, g, 0));
    b->graph_k = k;
    return STK_OK;
}

}  // namespace

extern "C" {

int stk_batch_create(stk_ctx *c, const stk_map *const *maps, int n_maps, const uint64_t *n_tracks,
                     const uint64_t *seeds, const uint64_t *offsets, double tau_max_s, stk_batch **out)
{
    if (!c) return STK_EINVAL;
    if (!out) return set_err(c, STK_EINVAL, "out is NULL");
    *out = nullptr;
    if (!maps || !n_tracks || !seeds || !offsets || n_maps < 1)
        return set_err(c, STK_EINVAL, "maps, n_tracks, seeds and offsets must be non-NULL and n_maps >= 1");
    if (!std::isfinite(tau_max_s) || tau_max_s < 0) return set_err(c, STK_EINVAL, "tau_max must be finite and >= 0");
    CUDA_TRY(c, cudaSetDevice(c->device));
    stk_batch *b = new stk_batch();
    b->ctx = c;
    b->n_maps = n_maps;
    b->maps.assign(maps, maps + n_maps);
    b->hmaps.resize(n_maps);
    for (int i = 0; i < n_maps; ++i) {
        const stk_map *m = maps[i];
        if (!m || m->ctx != c) {
            delete b;
            return set_err(c, STK_EINVAL, "map %d is NULL or belongs to another context", i);
        }
        if (i == 0) {
            b->wmode = m->dev.wmode;
            b->prec = m->dev.prec;
        }
        if (m->dev.wmode != b->wmode || m->dev.prec != b->prec || m->dev.paper != maps[0]->dev.paper) {
            delete b;
            return set_err(c, STK_EINVAL, "map %d differs from map 0 in statistic, precision or weighting", i);
        }
        if (n_tracks[i] < 1 || n_tracks[i] > 0xffffffffull) {
            delete b;
            return set_err(c, STK_EINVAL, "n_tracks[%d] must be in [1, 2^32)", i);
        }
        if (m->dev.n_f > kPhaseNarrowNf) {
            delete b;
            return set_err(c, STK_EINVAL, "map %d: n_f = %d exceeds %d (batched scoring)", i, m->dev.n_f,
                           kPhaseNarrowNf);
        }
        const uint64_t M = m->dev.M;
        if ((unsigned __int128)M * M * (2 * (uint64_t)m->dev.n_f - 1) >= ((unsigned __int128)1 << 32)) {
            delete b;
            return set_err(c, STK_EINVAL, "map %d: (n_t - 1)^2 (2 n_f - 1) must be below 2^32", i);
        }
        BatchMap &x = b->hmaps[i];
        x.m = m->dev;
        x.ts = TrackSet{n_tracks[i], seeds[i], offsets[i], tau_max_s};
        x.d32 = (uint32_t)m->dev.d;
        x.pos0 = (uint32_t)b->total_n;
        b->total_n += n_tracks[i];
        b->max_n = std::max<uint64_t>(b->max_n, n_tracks[i]);
        if (b->total_n > 0xffffffffull) {
            delete b;
            return set_err(c, STK_EINVAL, "the batch's templates must number below 2^32 in all");
        }
    }
    // the division by 2 M^2: a map's exact multiply-shift when it has one, else the
    // corrected form
    for (int i = 0; i < n_maps; ++i) {
        BatchMap &x = b->hmaps[i];
        x.fast = maps[i]->dev.fast32 ? 1 : 0;
        if (x.fast) {
            x.magic = maps[i]->dev.magic;
            x.shift = maps[i]->dev.shift;
        } else {
            corrected_magic(maps[i]->dev.d, x.magic, x.shift);
        }
    }
    cudaError_t e;
    if ((e = cudaMalloc(&b->d_counter, sizeof(unsigned int))) != cudaSuccess ||
        (e = cudaMalloc(&b->d_hits, sizeof(stk_hit) * (size_t)n_maps * STK_BATCH_MAX_K)) != cudaSuccess ||
        (e = cudaHostAlloc(&b->h_cancel, sizeof(int), cudaHostAllocMapped)) != cudaSuccess ||
        (e = cudaHostGetDevicePointer(&b->d_cancel, b->h_cancel, 0)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking)) != cudaSuccess) {
        stk_batch_destroy(b);
        return set_err(c, STK_ENOMEM, "batch allocation: %s", cudaGetErrorString(e));
    }
    *b->h_cancel = 0;
    if (c->tune.order && n_maps <= 8192) {
        // coarse buckets: at most 8192 over all maps, so large batches keep fewer key bits per map
        std::vector<OrderMap> om(n_maps);
        for (int i = 0; i < n_maps; ++i) {
            om[i] = OrderMap{};
            om[i].ts = b->hmaps[i].ts;
            om[i].n_f = (uint32_t)b->hmaps[i].m.n_f;
            om[i].n_t = (uint32_t)b->hmaps[i].m.n_t;
            om[i].pos0 = b->hmaps[i].pos0;
        }
        order_plan_maps(om.data(), n_maps, b->order_nc, b->order_fbits);
        const size_t bytes = order_scratch_bytes_maps(b->total_n, b->order_nc, c->num_sms);
        if ((e = cudaMalloc(&b->d_omaps, sizeof(OrderMap) * n_maps)) != cudaSuccess ||
            (e = cudaMalloc(&b->order_buf, bytes)) != cudaSuccess ||
            (e = cudaMemcpy(b->d_omaps, om.data(), sizeof(OrderMap) * n_maps, cudaMemcpyHostToDevice)) !=
                cudaSuccess ||
            (e = order_prepare(b->order_nc, b->order_fbits)) != cudaSuccess) {
            stk_batch_destroy(b);
            return set_err(c, STK_ENOMEM, "batch order scratch (%zu bytes): %s", bytes, cudaGetErrorString(e));
        }
        b->use_order = true;
    }
    int rc = configure(b, 1024, 5, 2);
    if (rc) {
        stk_batch_destroy(b);
        return rc;
    }
    *out = b;
    return STK_OK;
}

void stk_batch_destroy(stk_batch *b)
{
    if (!b) return;
    cudaSetDevice(b->ctx->device);
    cudaStreamSynchronize(b->ctx->stream);
    drop_graph(b);
    cudaFree(b->d_maps);
    cudaFree(b->d_sched);
    cudaFree(b->d_counter);
    cudaFree(b->d_ckey);
    cudaFree(b->d_cidx);
    cudaFree(b->d_hits);
    cudaFree(b->d_omaps);
    cudaFree(b->order_buf);
    if (b->h_cancel) cudaFreeHost(b->h_cancel);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    delete b;
}

int stk_batch_cancel(stk_batch *b, int on)
{
    if (!b) return STK_EINVAL;
    *(volatile int *)b->h_cancel = on ? 1 : 0;
    return STK_OK;
}

int stk_batch_score(stk_batch *b, int k, stk_hit *out, unsigned flags)
{
    if (!b) return STK_EINVAL;
    stk_ctx *c = b->ctx;
    if (!out) return set_err(c, STK_EINVAL, "out is NULL");
    if (flags & ~STK_OUT_HOST) return set_err(c, STK_EINVAL, "unknown flags 0x%x", flags);
    if (k < 1 || k > STK_BATCH_MAX_K) return set_err(c, STK_EINVAL, "k = %d must be in [1, %d]", k, STK_BATCH_MAX_K);
    for (int i = 0; i < b->n_maps; ++i)
        if ((uint64_t)k > b->hmaps[i].ts.n) return set_err(c, STK_EINVAL, "k exceeds n_tracks of map %d", i);
    CUDA_TRY(c, cudaSetDevice(c->device));
    int rc = ensure_graph(b, k);
    if (rc) return rc;
    CUDA_TRY(c, cudaGraphLaunch(b->gexec, c->stream));
    const size_t bytes = sizeof(stk_hit) * (size_t)b->n_maps * k;
    if (kDebugBounds)   // every map's canaries and the out-of-range flag (debug build)
        for (int i = 0; i < b->n_maps; ++i)
            if ((rc = debug_verify(c, b->maps[i])) != STK_OK) return rc;
    if (flags & STK_OUT_HOST) {
        CUDA_TRY(c, cudaMemcpyAsync(out, b->d_hits, bytes, cudaMemcpyDeviceToHost, c->stream));
        int fl = 0;
        rc = read_err_flags(c, &fl);
        if (rc) return rc;
        return flags_to_status(c, fl);
    }
    CUDA_TRY(c, cudaMemcpyAsync(out, b->d_hits, bytes, cudaMemcpyDeviceToDevice, c->stream));
    return STK_OK;
}

int stk_batch_tune(stk_batch *b, int k, int64_t out[4])
{
    if (!b) return STK_EINVAL;
    stk_ctx *c = b->ctx;
    if (k < 1 || k > STK_BATCH_MAX_K) return set_err(c, STK_EINVAL, "k = %d must be in [1, %d]", k, STK_BATCH_MAX_K);
    CUDA_TRY(c, cudaSetDevice(c->device));
    cudaEvent_t e0, e1;
    CUDA_TRY(c, cudaEventCreate(&e0));
    CUDA_TRY(c, cudaEventCreate(&e1));
    // candidate launch shapes: 64-register (up to 1024 threads, R <= 5) and
    // 128-register (512 threads, R 6..11) families, 2 or 3 slab buffers
    struct Shape {
        int threads, R, nstage;
    };
    std::vector<Shape> shapes;
    for (int th : {512, 768, 1024})
        for (int R = 2; R <= 5; ++R)
            for (int ns : {2, 3}) shapes.push_back({th, R, ns});
    for (int R : {6, 8, 10, 11})
        for (int ns : {2, 3}) shapes.push_back({512, R, ns});
    double best_rate = -1.0;
    int bt = b->threads, bR = b->R, bs = b->nstage;
    float best_ms = 0.f;
    int rc = STK_OK;
    for (size_t ci = 0; ci < shapes.size() && rc == STK_OK; ++ci) {
        const int th = shapes[ci].threads, R = shapes[ci].R, ns = shapes[ci].nstage;
        if ((rc = configure(b, th, R, ns)) != STK_OK) break;
        // sample: the first waves of the schedule (largest maps), about 3 tiles per SM
        const uint32_t nt = std::min<uint32_t>(b->ntiles_total, (uint32_t)c->num_sms * 3);
        std::vector<uint2> sched(nt);
        cudaError_t e = cudaMemcpy(sched.data(), b->d_sched, sizeof(uint2) * nt, cudaMemcpyDeviceToHost);
        double px = 0;  // track-pixels in the sampled tiles
        for (auto &sp : sched) {
            const BatchMap &x = b->hmaps[sp.x];
            const uint64_t t0 = (uint64_t)sp.y * b->tile;
            px += (double)std::min<uint64_t>(b->tile, x.ts.n - t0) * x.m.n_t;
        }
        if (e == cudaSuccess) e = enqueue(b, k, nt, false, true, c->stream, ci == 0);  // warm-up (+ order once)
        if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
        if (e == cudaSuccess) e = enqueue(b, k, nt, false, false, c->stream, false);
        if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            rc = set_err(c, STK_ECUDA, "tuning launch: %s", cudaGetErrorString(e));
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double rate = px / (ms > 0 ? ms : 1e-6);
        if (rate > best_rate) {
            best_rate = rate;
            bt = th; bR = R; bs = ns;
            best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int fl = 0;
    read_err_flags(c, &fl);   // the samples' tile candidates are discarded; clear their flags
    if (rc != STK_OK) return rc;
    rc = configure(b, bt, bR, bs);
    if (rc) return rc;
    if (out) {
        out[0] = bt;
        out[1] = bR;
        out[2] = bs;
        out[3] = (int64_t)(best_ms * 1e6);
    }
    return STK_OK;
}

}  // extern "C"
