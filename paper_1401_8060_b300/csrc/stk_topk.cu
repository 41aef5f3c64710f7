// Selection of the k loudest templates (the paper's "most significant
// cluster", Sec. III, kept to k > 1 so runs can be merged, Sec. V).
//
// Exact and deterministic: order by SNR descending, then template index
// ascending.  The FP32 SNRs are mapped to order-preserving keys: 32 bits, in
// the upper half of a 64-bit key (the candidate and batch formats).
//   1. two histogram passes over the 12-bit digits key[63:52] and key[51:40]
//      fix the 24-bit prefix of the k-th largest key;
//   2. one pass collects every template whose key prefix is at least that one
//      (the k winners plus the rest of the boundary bucket, usually a few
//      thousand) into a candidate buffer;
//   3. every candidate counts the candidates ordered before it (all pairs, in
//      parallel over many blocks); that count is its rank, and ranks below k
//      write their hit straight to its place.
// When the boundary bucket is too large for that (many templates agreeing in
// their top 24 key bits, e.g. a constant map), step 3 instead runs an exact
// radix select over the keys and then over the indices of the tied keys, in
// one block, on the full SNR array.
#include <cstdint>

#include "stk_internal.cuh"
#include "stk_pixel.cuh"

namespace stk {

namespace {

constexpr int kBins = 4096;           // 12-bit digits
constexpr int kPassThreads = 512;
constexpr int kFinalThreads = 1024;
constexpr uint32_t kCandCap = 65536;  // candidate buffer
constexpr int kRankCap = 16384;       // candidates ranked by all-pairs comparison
constexpr int kRankChunk = 64;        // candidates per ranking block (x 4 comparand lanes)

struct SelState {
    unsigned int hist[kBins];
    unsigned int d1, d2;   // digits of the k-th key's 24-bit prefix
    unsigned int krem;     // places left for keys sharing the prefix being resolved
    unsigned int ncand;    // candidates collected
    unsigned int overflow; // candidates exceeded kCandCap
    unsigned int pad[3];
};

// Block-wide: given hist[0..nbins) in shared or global memory, find the digit d
// with above(d) < krem <= above(d) + hist[d], where above(d) = sum of bins > d.
// Returns d and the places left inside bin d (krem - above(d)) through smem.
// nbins must be a multiple of blockDim.x.
__device__ void pick_digit(const unsigned int *hist, int nbins, unsigned int krem, unsigned int *out_d,
                           unsigned int *out_krem)
{
    __shared__ unsigned int warp_sum[32];
    const int per = nbins / blockDim.x;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
    unsigned int mine = 0;
    for (int i = 0; i < per; ++i) mine += hist[t * per + i];
    // exclusive suffix sum over threads: sum of bins owned by threads > t
    unsigned int incl = mine;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int v = __shfl_down_sync(0xffffffffu, incl, o);
        if (lane + o < 32) incl += v;
    }
    if (lane == 0) warp_sum[wid] = incl;
    __syncthreads();
    unsigned int later_warps = 0;
    for (int w = wid + 1; w < nw; ++w) later_warps += warp_sum[w];
    unsigned int above = later_warps + incl - mine;
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
    for (int i = threadIdx.x; i < kBins; i += blockDim.x) st->hist[i] = 0;
    if (threadIdx.x == 0) {
        st->ncand = 0;
        st->overflow = 0;
    }
}

// PASS 0: histogram of key[63:52]; PASS 1: of key[51:40] among keys with key[63:52] == d1.
// The leading key bits of SNRs fall into few bins, so lanes of a warp holding the
// same bin are merged (__match_any_sync) into one shared-memory atomic.
template <int PASS>
__global__ void __launch_bounds__(kPassThreads) sel_hist(const float *__restrict__ snr, uint64_t n, SelState *st)
{
    __shared__ unsigned int h[kBins];
    for (int i = threadIdx.x; i < kBins; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const unsigned int d1 = PASS ? st->d1 : 0u;
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const uint64_t w0 = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    for (uint64_t base = w0 * 128; base < n; base += warps * 128) {
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {   // four independent loads in flight per lane
            const uint64_t i = base + u * 32 + lane;
            v[u] = i < n ? snr[i] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            unsigned int bin = 0xffffffffu;  // no bin
            if (base + u * 32 + lane < n) {
                const unsigned long long key = order_key(v[u]);
                if (PASS == 0) bin = (unsigned int)(key >> 52);
                else if ((unsigned int)(key >> 52) == d1) bin = (unsigned int)(key >> 40) & 4095u;
            }
            const unsigned int peers = __match_any_sync(0xffffffffu, bin);
            if (bin != 0xffffffffu && lane == __ffs(peers) - 1) atomicAdd(&h[bin], (unsigned int)__popc(peers));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kBins; i += blockDim.x)
        if (h[i]) atomicAdd(&st->hist[i], h[i]);
}

template <int PASS>
__global__ void __launch_bounds__(kFinalThreads) sel_pick(SelState *st, unsigned int k)
{
    __shared__ unsigned int d, kr;
    const unsigned int krem = PASS ? st->krem : k;
    pick_digit(st->hist, kBins, krem, &d, &kr);
    if (threadIdx.x == 0) {
        if (PASS == 0) st->d1 = d;
        else st->d2 = d;
        st->krem = kr;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kBins; i += blockDim.x) st->hist[i] = 0;
}

// Every key whose 24-bit prefix is >= (d1, d2) becomes a candidate.
__global__ void __launch_bounds__(kPassThreads) sel_collect(const float *__restrict__ snr, uint64_t n, SelState *st,
                                                            unsigned long long *cand_key, unsigned int *cand_idx)
{
    const unsigned int pref = (st->d1 << 12) | st->d2;
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

// Bitonic sort of P (power of two) entries in shared memory, "before" first.
__device__ void bitonic_sort(unsigned long long *key, unsigned int *ix, int P)
{
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool up = (i & size) == 0;
                    if (before(key[j], ix[j], key[i], ix[i]) == up) {
                        const unsigned long long tk = key[i]; key[i] = key[j]; key[j] = tk;
                        const unsigned int ti = ix[i]; ix[i] = ix[j]; ix[j] = ti;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Source of (key, index) pairs for the final step.
struct Src {
    const float *snr;
    const unsigned long long *ckey;
    const unsigned int *cidx;
    uint64_t n;
    bool full;  // true: all templates (key from snr[i], index i); false: the candidates
    __device__ __forceinline__ unsigned long long key(uint64_t i) const { return full ? order_key(snr[i]) : ckey[i]; }
    __device__ __forceinline__ unsigned int idx(uint64_t i) const { return full ? (unsigned int)i : cidx[i]; }
};

// Exact k-th largest key, then the largest index among the tied keys that still
// fits, by 8-bit radix passes in one block; then gather the k winners.
// hp: blockDim.x shared counters (the first 256 are the digit histogram).
__device__ void select_generic(const Src &src, int k, unsigned long long *out_key, unsigned int *out_idx,
                               unsigned int *hp, unsigned int *cnt)
{
    __shared__ unsigned int d, kr;
    unsigned long long prefix = 0, mask = 0;
    unsigned int krem = (unsigned int)k;
    for (int shift = 56; shift >= 32; shift -= 8) {  // the lower 32 key bits are zero
        for (int i = threadIdx.x; i < (int)blockDim.x; i += blockDim.x) hp[i] = 0;
        __syncthreads();
        for (uint64_t i = threadIdx.x; i < src.n; i += blockDim.x) {
            const unsigned long long key = src.key(i);
            if ((key & mask) == prefix) atomicAdd(&hp[(key >> shift) & 255u], 1u);
        }
        __syncthreads();
        pick_digit(hp, blockDim.x, krem, &d, &kr);
        prefix |= (unsigned long long)d << shift;
        mask |= 255ull << shift;
        krem = kr;
    }
    const unsigned long long kth = prefix;
    // among keys equal to kth, the krem smallest indices: digits binned in reverse
    unsigned int iprefix = 0, imask = 0, irem = krem;
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int i = threadIdx.x; i < (int)blockDim.x; i += blockDim.x) hp[i] = 0;
        __syncthreads();
        for (uint64_t i = threadIdx.x; i < src.n; i += blockDim.x) {
            if (src.key(i) != kth) continue;
            const unsigned int ix = src.idx(i);
            if ((ix & imask) == iprefix) atomicAdd(&hp[255u - ((ix >> shift) & 255u)], 1u);
        }
        __syncthreads();
        pick_digit(hp, blockDim.x, irem, &d, &kr);
        iprefix |= (255u - d) << shift;
        imask |= 255u << shift;
        irem = kr;
    }
    const unsigned int ithr = iprefix;  // largest index kept among the ties
    if (threadIdx.x == 0) *cnt = 0;
    __syncthreads();
    for (uint64_t i = threadIdx.x; i < src.n; i += blockDim.x) {
        const unsigned long long key = src.key(i);
        const unsigned int ix = src.idx(i);
        if (key > kth || (key == kth && ix <= ithr)) {
            const unsigned int pos = atomicAdd(cnt, 1u);
            if (pos < (unsigned int)k) {
                out_key[pos] = key;
                out_idx[pos] = ix;
            }
        }
    }
    __syncthreads();
}

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

// Rank of each candidate = number of candidates ordered before it; block b
// ranks candidates [64 b, 64 b + 64), four threads per candidate each taking a
// quarter of every shared-memory tile of comparands (all lanes of a warp read
// the same comparand: a broadcast).
constexpr int kRankTile = 1024;

__global__ void __launch_bounds__(256) sel_rank(const float *__restrict__ snr, const SelState *st,
                                                const unsigned long long *__restrict__ cand_key,
                                                const unsigned int *__restrict__ cand_idx, int k, TrackSet ts,
                                                MapDev m, stk_hit *out)
{
    __shared__ unsigned int part[4][kRankChunk];
    __shared__ unsigned long long tk[kRankTile];
    __shared__ unsigned int ti[kRankTile];
    const unsigned int nc = st->ncand;
    if (st->overflow || nc > (unsigned int)kRankCap) return;
    const unsigned int c0 = blockIdx.x * kRankChunk;
    if (c0 >= nc) return;
    const int c = threadIdx.x & (kRankChunk - 1), qd = threadIdx.x / kRankChunk;
    const unsigned int me = c0 + c;
    const bool valid = me < nc;
    const unsigned long long mk = valid ? cand_key[me] : 0ull;
    const unsigned int mi = valid ? cand_idx[me] : 0xffffffffu;
    unsigned int before_me = 0;
    for (unsigned int t0 = 0; t0 < nc; t0 += kRankTile) {
        const unsigned int tn = min((unsigned int)kRankTile, nc - t0);
        for (unsigned int j = threadIdx.x; j < tn; j += blockDim.x) {
            tk[j] = cand_key[t0 + j];
            ti[j] = cand_idx[t0 + j];
        }
        __syncthreads();
        for (unsigned int j = qd; j < tn; j += 4) before_me += before(tk[j], ti[j], mk, mi) ? 1u : 0u;
        __syncthreads();
    }
    part[qd][c] = before_me;
    __syncthreads();
    if (qd == 0 && valid) {
        const unsigned int rank = part[0][c] + part[1][c] + part[2][c] + part[3][c];
        if (rank < (unsigned int)k) write_hit(snr, mi, ts, m, out + rank);
    }
}

// Fallback when the candidates overflowed or exceed kRankCap: exact selection in
// one block (radix select over keys, then over the tied indices), bitonic sort of
// the k winners.  Returns at once otherwise.
__global__ void __launch_bounds__(kFinalThreads)
    sel_generic(const float *__restrict__ snr, uint64_t n, const SelState *st, const unsigned long long *cand_key,
                const unsigned int *cand_idx, int k, TrackSet ts, MapDev m, stk_hit *out)
{
    extern __shared__ unsigned long long sh[];
    __shared__ unsigned int hp[kFinalThreads];
    __shared__ unsigned int cnt;
    const unsigned int ncand = st->ncand;
    if (!st->overflow && ncand <= (unsigned int)kRankCap) return;
    int P = 1;
    while (P < k) P <<= 1;
    unsigned long long *key = sh;
    unsigned int *ix = reinterpret_cast<unsigned int *>(sh + P);
    Src src{snr, cand_key, cand_idx, st->overflow ? n : (uint64_t)ncand, st->overflow != 0};
    select_generic(src, k, key, ix, hp, &cnt);
    for (int i = k + threadIdx.x; i < P; i += blockDim.x) {
        key[i] = 0ull;   // below every real key
        ix[i] = 0xffffffffu;
    }
    __syncthreads();
    bitonic_sort(key, ix, P);
    for (int i = threadIdx.x; i < k; i += blockDim.x) write_hit(snr, ix[i], ts, m, out + i);
}

constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

size_t select_scratch_bytes(uint64_t /*n*/, int /*k*/)
{
    return align256(sizeof(SelState)) + align256((size_t)kCandCap * 8) + align256((size_t)kCandCap * 4);
}

cudaError_t launch_select_topk(const float *snr, uint64_t n, int k, const TrackSet &ts, const MapDev &m,
                               void *scratch, stk_hit *out, cudaStream_t st, int *launches)
{
    if (k <= 0 || (uint64_t)k > n || k > STK_MAX_K || n > 0xffffffffull) return cudaErrorInvalidValue;
    unsigned char *p = (unsigned char *)scratch;
    SelState *ss = (SelState *)p;
    unsigned long long *ckey = (unsigned long long *)(p + align256(sizeof(SelState)));
    unsigned int *cidx = (unsigned int *)(p + align256(sizeof(SelState)) + align256((size_t)kCandCap * 8));
    const uint64_t blocks = (n + kPassThreads * 8 - 1) / (kPassThreads * 8);
    const int grid = (int)(blocks < 592 ? (blocks < 1 ? 1 : blocks) : 592);
    sel_init<<<1, 1024, 0, st>>>(ss);
    sel_hist<0><<<grid, kPassThreads, 0, st>>>(snr, n, ss);
    sel_pick<0><<<1, kFinalThreads, 0, st>>>(ss, (unsigned int)k);
    sel_hist<1><<<grid, kPassThreads, 0, st>>>(snr, n, ss);
    sel_pick<1><<<1, kFinalThreads, 0, st>>>(ss, (unsigned int)k);
    sel_collect<<<grid, kPassThreads, 0, st>>>(snr, n, ss, ckey, cidx);
    sel_rank<<<kRankCap / kRankChunk, 256, 0, st>>>(snr, ss, ckey, cidx, k, ts, m, out);
    const size_t smem = (size_t)STK_MAX_K * 12;
    cudaError_t e = cudaFuncSetAttribute(sel_generic, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    sel_generic<<<1, kFinalThreads, smem, st>>>(snr, n, ss, ckey, cidx, k, ts, m, out);
    if (launches) *launches = 8;
    return cudaGetLastError();
}

}  // namespace stk
