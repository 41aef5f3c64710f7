// Selection of the k loudest templates (the paper's "most significant
// cluster", Sec. III, kept to k > 1 so runs can be merged, Sec. V).
//
// Exact and deterministic: order by SNR descending, then template index
// ascending.  The FP32 SNRs are mapped to order-preserving keys: 32 bits, in
// the upper half of a 64-bit key (the candidate and batch formats).
//   1. the threshold, a 24-bit key prefix: one block reads the keys of S
//      templates in 4 runs spread over the range (all of them when n <= S) and
//      takes the prefix of the q-th largest sample key, q chosen so that at
//      least k of all n keys reach it except with negligible probability; or,
//      when that would admit more than a quarter of the candidate buffer (k
//      small against n / S), the exact prefix of the k-th largest key from two
//      histogram passes over all keys;
//   2. one pass collects every template whose key prefix is at least that one
//      (the k winners and a few thousand more) into a candidate buffer;
//   3. one block selects exactly: a radix select of the k-th largest key, then
//      (only when more keys tie with it than places are left) of the largest
//      index kept among the ties, and a gather of the k winners.  When at
//      least k were collected (and the buffer did not overflow) it works on
//      the candidates, staged in shared memory: at least k keys reach the
//      prefix, so the k-th largest key does too and the k loudest are all
//      candidates.  Otherwise -- the sample missed, or many templates agree in
//      their top 24 key bits (e.g. a constant map) -- it works on the full SNR
//      array, which is slower;
//   4. many blocks place each winner at the number of winners ordered before it.
// Exactness never rests on the sample.
#include <cmath>
#include <cstdint>

#include "stk_internal.cuh"
#include "stk_pixel.cuh"

namespace stk {

namespace {

constexpr int kPassThreads = 512;
constexpr int kFinalThreads = 1024;
constexpr int kWarps = kFinalThreads / 32;
constexpr int kDigits = 256;                // 8-bit radix digits
constexpr int kBins12 = 4096;               // 12-bit digits of the exact threshold
constexpr uint32_t kCandCap = 65536;        // candidate buffer
constexpr uint32_t kSmemCand = 12288;       // candidates staged in shared memory by the final step
constexpr uint32_t kSampleDefault = 16384;  // keys sampled for the threshold
constexpr uint32_t kSampleMax = 49152;      // the sample lives in shared memory
constexpr uint32_t kSampleRuns = 4;         // runs of consecutive templates in the sample

struct SelState {
    unsigned int prefix;   // the threshold: 24-bit key prefix
    unsigned int ncand;    // candidates collected
    unsigned int overflow; // candidates exceeded kCandCap
    unsigned int d1, krem; // exact threshold: first digit, places left inside it
    unsigned int pad[3];
    unsigned int hist[kBins12];  // exact threshold: digit histogram
};

// Upper half of order_key: unsigned order is SNR order.
__device__ __forceinline__ uint32_t key32(float x) { return (uint32_t)(order_key(x) >> 32); }

// ------------------------------------------------------------------ block radix select
// Shared state of a block-wide radix select over 32-bit values, 8 bits a pass.
// Each warp counts into its own digit histogram (no contention between warps),
// then the histograms are summed and the digit holding the r-th largest value
// is found.
struct Radix {
    unsigned int wh[kWarps][kDigits];
    unsigned int tot[kDigits];
    unsigned int wsum[kDigits / 32];
    unsigned int d, r;
};

// One pass: tot[b] = number of i < n whose digit(i) is b (digit 0xffffffff: none).
template <class Digit>
__device__ void radix_count(Radix &R, uint64_t n, Digit digit)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int b = lane; b < kDigits; b += 32) R.wh[w][b] = 0;
    __syncwarp();
    for (uint64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const unsigned int b = digit(i);
        if (b != 0xffffffffu) atomicAdd(&R.wh[w][b], 1u);
    }
    __syncthreads();
    if (threadIdx.x < kDigits) {
        unsigned int t = 0;
        for (int v = 0; v < kWarps; ++v) t += R.wh[v][threadIdx.x];
        R.tot[threadIdx.x] = t;
    }
    __syncthreads();
}

// R.d = the digit d with above(d) < r <= above(d) + tot[d] (above(d): the count
// in digits > d), R.r = r - above(d).
__device__ void radix_pick(Radix &R, unsigned int r)
{
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t == 0) {  // overwritten below (some digit always qualifies when r <= sum of tot)
        R.d = 0;
        R.r = 1;
    }
    unsigned int c = 0, incl = 0;
    if (t < kDigits) {  // whole warps 0 .. 7
        c = R.tot[t];
        incl = c;  // becomes the sum over digits t .. 32 w + 31
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int y = __shfl_down_sync(0xffffffffu, incl, o);
            if (lane + o < 32) incl += y;
        }
        if (lane == 0) R.wsum[w] = incl;
    }
    __syncthreads();
    if (t < kDigits) {
        unsigned int above = incl - c;
        for (int v = w + 1; v < kDigits / 32; ++v) above += R.wsum[v];
        if (above < r && above + c >= r) {
            R.d = (unsigned int)t;
            R.r = r - above;
        }
    }
    __syncthreads();
}

// The r-th largest (1-based) of the 32-bit values value(i) over the i < n with
// valid(i), resolved to its top 8 * passes bits.  r_left: places left among the
// values sharing that prefix; tied: how many share it.
template <class Valid, class Value>
__device__ uint32_t radix_select(Radix &R, uint64_t n, unsigned int r, int passes, Valid valid, Value value,
                                 unsigned int &r_left, unsigned int &tied)
{
    uint32_t prefix = 0, mask = 0;
    for (int p = 0; p < passes; ++p) {
        const int shift = 24 - 8 * p;
        radix_count(R, n, [&](uint64_t i) -> unsigned int {
            if (!valid(i)) return 0xffffffffu;
            const uint32_t v = value(i);
            return (v & mask) == prefix ? (v >> shift) & 255u : 0xffffffffu;
        });
        radix_pick(R, r);
        const unsigned int d = R.d;
        r = R.r;
        tied = R.tot[d];
        prefix |= d << shift;
        mask |= 255u << shift;
        __syncthreads();  // R is reused by the next pass
    }
    r_left = r;
    return prefix;
}

// ------------------------------------------------------------------ step 1: threshold
// One block: S sample keys in shared memory (kSampleRuns runs of consecutive
// templates spread over the range, coalesced; the templates are independent
// draws, so any run is a random sample of them), then the 24-bit prefix of the
// q-th largest.  Resets the candidate count for step 2.
__global__ void __launch_bounds__(kFinalThreads) sel_threshold(const float *__restrict__ snr, uint64_t n,
                                                               uint32_t S, uint32_t q, SelState *st)
{
    extern __shared__ uint32_t sk[];  // [S]
    __shared__ Radix R;
    const uint32_t L = (S + kSampleRuns - 1) / kSampleRuns;
    constexpr int U = 32;  // loads in flight per thread (the default sample in one round)
    for (uint32_t i0 = 0; i0 < S; i0 += blockDim.x * U) {
        float v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t i = i0 + u * blockDim.x + threadIdx.x;
            const uint32_t c = i / L, j = i - c * L;
            uint64_t pos = n <= (uint64_t)S ? (uint64_t)i : (uint64_t)c * n / kSampleRuns + j;
            if (pos >= n) pos = n - 1;
            v[u] = i < S ? snr[pos] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t i = i0 + u * blockDim.x + threadIdx.x;
            if (i < S) sk[i] = key32(v[u]);
        }
    }
    __syncthreads();
    unsigned int r_left, tied;
    const uint32_t pref = radix_select(
        R, S, q, 3, [](uint64_t) { return true; }, [&](uint64_t i) { return sk[i]; }, r_left, tied);
    if (threadIdx.x == 0) {
        st->prefix = pref >> 8;
        st->ncand = 0;
        st->overflow = 0;
    }
}

// ------------------------------------------------------------------ step 1, exact form
// When a sampled threshold would admit too many candidates (k small against
// n / S), the threshold is instead the exact 24-bit prefix of the k-th largest
// key: a histogram pass over all keys for the digit key[31:20], a pick, a pass
// for key[19:8] among keys with that digit, a pick.  Multi-block passes; lanes
// of a warp holding the same digit merge into one shared atomic.

// Block-wide: given hist[0..nbins), the digit d with above(d) < krem <= above(d) +
// hist[d] (above(d) = sum of bins > d) and krem - above(d), through shared memory.
// nbins must be a multiple of blockDim.x.
__device__ void pick_digit(const unsigned int *hist, int nbins, unsigned int krem, unsigned int *out_d,
                           unsigned int *out_krem)
{
    __shared__ unsigned int warp_sum[32];
    const int per = nbins / blockDim.x;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
    if (t == 0) {  // overwritten below (some digit always qualifies when krem <= the total)
        *out_d = 0;
        *out_krem = 1;
    }
    unsigned int mine = 0;
    for (int i = 0; i < per; ++i) mine += hist[t * per + i];
    unsigned int incl = mine;  // becomes the sum over threads t .. 32 wid + 31
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int v = __shfl_down_sync(0xffffffffu, incl, o);
        if (lane + o < 32) incl += v;
    }
    if (lane == 0) warp_sum[wid] = incl;
    __syncthreads();
    unsigned int above = incl - mine;
    for (int w = wid + 1; w < nw; ++w) above += warp_sum[w];
    for (int i = per - 1; i >= 0; --i) {
        const unsigned int d = (unsigned int)(t * per + i), c = hist[d];
        if (above < krem && above + c >= krem) {
            *out_d = d;
            *out_krem = krem - above;
        }
        above += c;
    }
    __syncthreads();
}

__global__ void sel_init(SelState *st)
{
    for (int i = threadIdx.x; i < kBins12; i += blockDim.x) st->hist[i] = 0;
    if (threadIdx.x == 0) {
        st->ncand = 0;
        st->overflow = 0;
    }
}

// PASS 0: histogram of key[31:20]; PASS 1: of key[19:8] among keys with key[31:20] == d1.
template <int PASS>
__global__ void __launch_bounds__(kPassThreads) sel_hist(const float *__restrict__ snr, uint64_t n, SelState *st)
{
    __shared__ unsigned int h[kBins12];
    for (int i = threadIdx.x; i < kBins12; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const unsigned int d1 = PASS ? st->d1 : 0u;
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const uint64_t w0 = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    for (uint64_t base = w0 * 128; base < n; base += warps * 128) {
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {  // four independent loads in flight per lane
            const uint64_t i = base + u * 32 + lane;
            v[u] = i < n ? snr[i] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            unsigned int bin = 0xffffffffu;  // no bin
            if (base + u * 32 + lane < n) {
                const uint32_t key = key32(v[u]);
                if (PASS == 0) bin = key >> 20;
                else if ((key >> 20) == d1) bin = (key >> 8) & 4095u;
            }
            const unsigned int peers = __match_any_sync(0xffffffffu, bin);
            if (bin != 0xffffffffu && lane == __ffs(peers) - 1) atomicAdd(&h[bin], (unsigned int)__popc(peers));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kBins12; i += blockDim.x)
        if (h[i]) atomicAdd(&st->hist[i], h[i]);
}

template <int PASS>
__global__ void __launch_bounds__(kFinalThreads) sel_pick(SelState *st, unsigned int k)
{
    __shared__ unsigned int d, kr;
    const unsigned int krem = PASS ? st->krem : k;
    pick_digit(st->hist, kBins12, krem, &d, &kr);
    if (threadIdx.x == 0) {
        if (PASS == 0) st->d1 = d;
        else st->prefix = (st->d1 << 12) | d;
        st->krem = kr;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kBins12; i += blockDim.x) st->hist[i] = 0;
}

// ------------------------------------------------------------------ step 2: candidates
// Every key whose 24-bit prefix is at least the threshold becomes a candidate.
__global__ void __launch_bounds__(kPassThreads) sel_collect(const float *__restrict__ snr, uint64_t n, SelState *st,
                                                            unsigned long long *cand_key, unsigned int *cand_idx)
{
    const unsigned int pref = st->prefix;
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const uint64_t w0 = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    for (uint64_t base = w0 * 128; base < n; base += warps * 128) {
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint64_t i = base + u * 32 + lane;
            v[u] = i < n ? snr[i] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint64_t i = base + u * 32 + lane;
            unsigned long long key = 0;
            bool p = false;
            if (i < n) {
                key = order_key(v[u]);
                p = (unsigned int)(key >> 40) >= pref;
            }
            const unsigned int msk = __ballot_sync(0xffffffffu, p);
            if (!msk) continue;
            unsigned int pos0 = 0;
            if (lane == __ffs(msk) - 1) pos0 = atomicAdd(&st->ncand, (unsigned int)__popc(msk));
            pos0 = __shfl_sync(0xffffffffu, pos0, __ffs(msk) - 1);
            if (p) {
                const unsigned int pos = pos0 + __popc(msk & ((1u << lane) - 1u));
                if (pos < kCandCap) {
                    cand_key[pos] = key;
                    cand_idx[pos] = (unsigned int)i;
                } else {
                    st->overflow = 1;
                }
            }
        }
    }
}

// ------------------------------------------------------------------ step 3: exact select
__device__ __forceinline__ void write_hit(const float *snr, unsigned int t, const TrackSet &ts, const MapDev &m,
                                          stk_hit *out)
{
    stk_hit hit;
    hit.snr = (double)snr[t];
    hit.index = ts.offset + t;
    uint32_t f[3];
    double tau;
    draw_track_ts(ts, ts.offset + t, (uint32_t)m.n_f, f, tau);
    hit.f[0] = f[0]; hit.f[1] = f[1]; hit.f[2] = f[2];
    hit.reserved = 0;
    hit.tau = tau;
    *out = hit;
}

// One block: the exact k loudest (SNR descending, then index ascending) of the
// candidates when they hold them (at least k collected, no overflow; up to
// kSmemCand staged in shared memory), else of every SNR.  A radix select finds
// the k-th largest key; only if more keys tie with it than places are left, a
// second one finds the largest index kept among the ties.  The k winners go to
// win[] packed as key << 32 | ~index, so that one unsigned order gives both
// rules (larger SNR, then smaller index), in no particular order.
__global__ void __launch_bounds__(kFinalThreads)
    sel_select(const float *__restrict__ snr, uint64_t n, const SelState *st, const unsigned long long *cand_key,
               const unsigned int *cand_idx, int k, unsigned long long *win)
{
    extern __shared__ uint32_t ck[];  // [kSmemCand] staged keys, then [kSmemCand] indices
    __shared__ Radix R;
    __shared__ unsigned int cnt;
    const unsigned int ncand = st->ncand;
    const bool full = st->overflow || ncand < (unsigned int)k;
    const uint64_t N = full ? n : (uint64_t)ncand;
    const bool staged = !full && ncand <= kSmemCand;
    uint32_t *ci = ck + kSmemCand;
    if (staged) {
        for (unsigned int i = threadIdx.x; i < ncand; i += blockDim.x) {
            ck[i] = (uint32_t)(cand_key[i] >> 32);
            ci[i] = cand_idx[i];
        }
        __syncthreads();
    }
    auto key_of = [&](uint64_t i) -> uint32_t {
        return full ? key32(snr[i]) : (staged ? ck[i] : (uint32_t)(cand_key[i] >> 32));
    };
    auto idx_of = [&](uint64_t i) -> uint32_t { return full ? (uint32_t)i : (staged ? ci[i] : cand_idx[i]); };
    unsigned int r_left, tied;
    const uint32_t kth = radix_select(
        R, N, (unsigned int)k, 4, [](uint64_t) { return true; }, key_of, r_left, tied);
    uint32_t ithr = 0xffffffffu;  // largest index kept among keys equal to kth
    if (tied > r_left) {
        unsigned int r2, t2;
        ithr = ~radix_select(
            R, N, r_left, 4, [&](uint64_t i) { return key_of(i) == kth; }, [&](uint64_t i) { return ~idx_of(i); },
            r2, t2);
    }
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (uint64_t i0 = 0; i0 < N; i0 += blockDim.x) {
        const uint64_t i = i0 + threadIdx.x;
        bool w = false;
        unsigned long long pv = 0;
        if (i < N) {
            const uint32_t kk = key_of(i), ix = idx_of(i);
            w = kk > kth || (kk == kth && ix <= ithr);
            pv = ((unsigned long long)kk << 32) | (uint32_t)~ix;
        }
        const unsigned int msk = __ballot_sync(0xffffffffu, w);
        unsigned int pos0 = 0;
        if (msk && lane == __ffs(msk) - 1) pos0 = atomicAdd(&cnt, (unsigned int)__popc(msk));
        pos0 = __shfl_sync(0xffffffffu, pos0, __ffs(msk ? msk : 1u) - 1);
        if (w) {
            const unsigned int pos = pos0 + __popc(msk & ((1u << lane) - 1u));
            if (pos < (unsigned int)k) win[pos] = pv;
        }
    }
}

// Many blocks: winner i's place is the number of winners above it (the packed
// values are distinct); its hit goes there.  Block b takes winners
// [kPlaceChunk b, kPlaceChunk (b + 1)), four threads each comparing against a
// quarter of every shared-memory tile.
constexpr int kPlaceChunk = 64;
constexpr int kPlaceTile = 1024;

__global__ void __launch_bounds__(256) sel_place(const float *__restrict__ snr, const unsigned long long *win, int k,
                                                 TrackSet ts, MapDev m, stk_hit *out)
{
    __shared__ unsigned long long tv[kPlaceTile];
    __shared__ unsigned int part[4][kPlaceChunk];
    const int c = threadIdx.x & (kPlaceChunk - 1), qd = threadIdx.x / kPlaceChunk;
    const int me = blockIdx.x * kPlaceChunk + c;
    const unsigned long long mv = me < k ? win[me] : 0ull;
    unsigned int above = 0;
    for (int t0 = 0; t0 < k; t0 += kPlaceTile) {
        const int tn = min(kPlaceTile, k - t0);
        for (int j = threadIdx.x; j < tn; j += blockDim.x) tv[j] = win[t0 + j];
        __syncthreads();
        for (int j = qd; j < tn; j += 4) above += tv[j] > mv ? 1u : 0u;
        __syncthreads();
    }
    part[qd][c] = above;
    __syncthreads();
    if (qd == 0 && me < k) {
        const unsigned int place = part[0][c] + part[1][c] + part[2][c] + part[3][c];
        write_hit(snr, ~(uint32_t)mv, ts, m, out + place);
    }
}

constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

size_t select_scratch_bytes(uint64_t /*n*/, int /*k*/)
{
    return align256(sizeof(SelState)) + align256((size_t)kCandCap * 8) + align256((size_t)kCandCap * 4) +
           align256((size_t)STK_MAX_K * 8);
}

uint32_t select_sample_size(uint64_t n, uint32_t sample)
{
    const uint64_t S = sample ? sample : kSampleDefault;
    return (uint32_t)(n < S ? n : S);
}

cudaError_t launch_select_topk(const float *snr, uint64_t n, int k, const TrackSet &ts, const MapDev &m,
                               void *scratch, stk_hit *out, cudaStream_t st, int *launches, uint32_t sample)
{
    if (k <= 0 || (uint64_t)k > n || k > STK_MAX_K || n > 0xffffffffull || sample > kSampleMax)
        return cudaErrorInvalidValue;
    unsigned char *p = (unsigned char *)scratch;
    SelState *ss = (SelState *)p;
    unsigned long long *ckey = (unsigned long long *)(p + align256(sizeof(SelState)));
    unsigned int *cidx = (unsigned int *)(p + align256(sizeof(SelState)) + align256((size_t)kCandCap * 8));
    unsigned long long *win = (unsigned long long *)(p + align256(sizeof(SelState)) + align256((size_t)kCandCap * 8) +
                                                     align256((size_t)kCandCap * 4));
    // lambda = expected sample keys among the k largest; q = lambda + 4 sqrt(lambda) + 8
    // falls short of the k-th largest key only with the probability of a binomial
    // tail beyond 4 standard deviations plus 8 (the final step stays exact
    // regardless, on the full array).  All keys sampled: q = k.
    const uint32_t S = select_sample_size(n, sample);
    uint32_t q = (uint32_t)k;
    if ((uint64_t)S < n) {
        const double lambda = (double)k * (double)S / (double)n;
        const double qd = std::ceil(lambda + 4.0 * std::sqrt(lambda) + 8.0);
        q = qd >= (double)S ? S : (uint32_t)qd;
    }
    const size_t smem_t = (size_t)S * 4, smem_s = (size_t)kSmemCand * 8;
    cudaError_t e = cudaFuncSetAttribute(sel_threshold, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_t);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sel_select, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_s);
    if (e != cudaSuccess) return e;
    const uint64_t blocks = (n + kPassThreads * 8 - 1) / (kPassThreads * 8);
    const int grid = (int)(blocks < 592 ? (blocks < 1 ? 1 : blocks) : 592);
    // expected candidates above the sampled threshold: q n / S; beyond a quarter of the
    // buffer the exact threshold (two full passes) is cheaper than the risk of overflow
    const double expect = (uint64_t)S < n ? (double)q * (double)n / (double)S : (double)k;
    int nl = 3;
    if (expect <= (double)(kCandCap / 4)) {
        sel_threshold<<<1, kFinalThreads, smem_t, st>>>(snr, n, S, q, ss);
        nl += 1;
    } else {
        sel_init<<<1, 1024, 0, st>>>(ss);
        sel_hist<0><<<grid, kPassThreads, 0, st>>>(snr, n, ss);
        sel_pick<0><<<1, kFinalThreads, 0, st>>>(ss, (unsigned int)k);
        sel_hist<1><<<grid, kPassThreads, 0, st>>>(snr, n, ss);
        sel_pick<1><<<1, kFinalThreads, 0, st>>>(ss, (unsigned int)k);
        nl += 5;
    }
    sel_collect<<<grid, kPassThreads, 0, st>>>(snr, n, ss, ckey, cidx);
    sel_select<<<1, kFinalThreads, smem_s, st>>>(snr, n, ss, ckey, cidx, k, win);
    sel_place<<<(k + kPlaceChunk - 1) / kPlaceChunk, 256, 0, st>>>(snr, win, k, ts, m, out);
    if (launches) *launches = nl;
    return cudaGetLastError();
}

}  // namespace stk
