// Selection of the k loudest templates (the paper's "most significant
// cluster", Sec. III, kept to k > 1 so runs can be merged, Sec. V).
//
// Exact and deterministic: order by SNR descending, then template index
// ascending.  Steps, all on the device:
//   1. radix select: eight passes of 8-bit digits over order-preserving 64-bit
//      keys of the FP64 SNRs find the k-th largest key exactly;
//   2. every template with a larger key is collected; of those equal to it, the
//      ones with the smallest indices fill the remaining places (a block-ordered
//      compaction over contiguous chunks keeps index order);
//   3. the k survivors are sorted in shared memory (bitonic) and their
//      parameters regenerated from their indices.
#include <cstdint>

#include "stk_internal.cuh"

namespace stk {

namespace {

constexpr int kHistThreads = 512;
constexpr int kMaxChunks = 1024;

struct SelState {
    unsigned long long prefix;  // digits fixed so far (the k-th key once all passes ran)
    unsigned long long mask;
    unsigned int krem;          // places still to fill from keys equal to the prefix
    unsigned int n_gt;          // keys strictly greater than the k-th, collected
    unsigned int pad0, pad1;
    unsigned int hist[256];
};

__device__ __forceinline__ unsigned long long order_key(double x)
{
    if (x == 0.0) x = 0.0;  // -0 and +0 compare equal: one key
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__global__ void sel_init(SelState *st, unsigned int k)
{
    const int t = threadIdx.x;
    if (t == 0) {
        st->prefix = 0;
        st->mask = 0;
        st->krem = k;
        st->n_gt = 0;
    }
    for (int i = t; i < 256; i += blockDim.x) st->hist[i] = 0;
}

__global__ void __launch_bounds__(kHistThreads) sel_hist(const double *__restrict__ snr, uint64_t n, SelState *st,
                                                         int shift)
{
    __shared__ unsigned int h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const unsigned long long prefix = st->prefix, mask = st->mask;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long key = order_key(snr[i]);
        if ((key & mask) == prefix) atomicAdd(&h[(key >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        if (h[i]) atomicAdd(&st->hist[i], h[i]);
}

// Fix the digit holding the krem-th largest key among those matching the prefix.
__global__ void sel_pick(SelState *st, int shift)
{
    if (threadIdx.x != 0) return;
    unsigned int above = 0, krem = st->krem;
    int d = 255;
    for (; d > 0; --d) {
        const unsigned int c = st->hist[d];
        if (above + c >= krem) break;
        above += c;
    }
    st->krem = krem - above;
    st->prefix |= (unsigned long long)d << shift;
    st->mask |= 255ull << shift;
    for (int i = 0; i < 256; ++i) st->hist[i] = 0;
}

// Collect keys > k-th into out_idx[0 .. n_gt); count keys == k-th per contiguous chunk.
__global__ void __launch_bounds__(kHistThreads) sel_collect(const double *__restrict__ snr, uint64_t n,
                                                            uint64_t chunk, SelState *st, unsigned int *out_idx,
                                                            unsigned int *chunk_eq)
{
    __shared__ unsigned int ceq;
    if (threadIdx.x == 0) ceq = 0;
    __syncthreads();
    const unsigned long long kth = st->prefix;
    const uint64_t lo = (uint64_t)blockIdx.x * chunk;
    const uint64_t hi = lo + chunk < n ? lo + chunk : n;
    unsigned int eq = 0;
    for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const unsigned long long key = order_key(snr[i]);
        if (key > kth) out_idx[atomicAdd(&st->n_gt, 1u)] = (unsigned int)i;
        eq += (key == kth);
    }
    if (eq) atomicAdd(&ceq, eq);
    __syncthreads();
    if (threadIdx.x == 0) chunk_eq[blockIdx.x] = ceq;
}

// Fill the remaining krem places with the lowest-index keys equal to the k-th.
__global__ void __launch_bounds__(kHistThreads) sel_ties(const double *__restrict__ snr, uint64_t n, uint64_t chunk,
                                                         const SelState *st, unsigned int *out_idx,
                                                         const unsigned int *chunk_eq)
{
    __shared__ unsigned int warp_tot[kHistThreads / 32];
    __shared__ unsigned int base_sh;
    const unsigned int krem = st->krem, ngt = st->n_gt;
    const unsigned long long kth = st->prefix;
    // Equal keys before this chunk.
    unsigned int before = 0;
    for (unsigned int b = threadIdx.x; b < blockIdx.x; b += blockDim.x) before += chunk_eq[b];
    for (int o = 16; o; o >>= 1) before += __shfl_xor_sync(0xffffffffu, before, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) warp_tot[wid] = before;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += warp_tot[w];
        base_sh = s;
    }
    __syncthreads();
    unsigned int base = base_sh;
    if (base >= krem || chunk_eq[blockIdx.x] == 0) return;
    const uint64_t lo = (uint64_t)blockIdx.x * chunk;
    const uint64_t hi = lo + chunk < n ? lo + chunk : n;
    for (uint64_t t0 = lo; t0 < hi && base < krem; t0 += blockDim.x) {
        const uint64_t i = t0 + threadIdx.x;
        const bool e = i < hi && order_key(snr[i]) == kth;
        const unsigned int bal = __ballot_sync(0xffffffffu, e);
        __syncthreads();  // warp_tot reuse
        if (lane == 0) warp_tot[wid] = __popc(bal);
        __syncthreads();
        unsigned int wbase = 0, tot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            if (w < wid) wbase += warp_tot[w];
            tot += warp_tot[w];
        }
        if (e) {
            const unsigned int rank = base + wbase + __popc(bal & ((1u << lane) - 1u));
            if (rank < krem) out_idx[ngt + rank] = (unsigned int)i;
        }
        base += tot;
    }
}

__global__ void sel_finalize(const double *__restrict__ snr, const unsigned int *idx, int k, int P, TrackSet ts,
                             MapDev m, stk_hit *out)
{
    extern __shared__ unsigned long long sh[];
    unsigned long long *key = sh;
    unsigned int *ix = reinterpret_cast<unsigned int *>(sh + P);
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        if (i < k) {
            key[i] = order_key(snr[idx[i]]);
            ix[i] = idx[i];
        } else {
            key[i] = 0ull;          // below every real key
            ix[i] = 0xffffffffu;
        }
    }
    __syncthreads();
    // Bitonic sort, "before" = larger key, then smaller index.
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool desc = (i & size) == 0;
                    const bool i_first = key[i] > key[j] || (key[i] == key[j] && ix[i] < ix[j]);
                    if (i_first != desc) {
                        const unsigned long long tk = key[i]; key[i] = key[j]; key[j] = tk;
                        const unsigned int ti = ix[i]; ix[i] = ix[j]; ix[j] = ti;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        const unsigned int t = ix[i];
        stk_hit h;
        h.snr = snr[t];
        h.index = ts.offset + t;
        uint32_t f[3];
        double tau;
        draw_track(ts.seed, ts.offset + t, (uint32_t)m.n_f, ts.tau_max, f, tau);
        h.f[0] = f[0]; h.f[1] = f[1]; h.f[2] = f[2];
        h.reserved = 0;
        h.tau = tau;
        out[i] = h;
    }
}

}  // namespace

size_t select_scratch_bytes(uint64_t /*n*/, int k)
{
    return sizeof(SelState) + ((size_t)k * 4 + 255) / 256 * 256 + (size_t)kMaxChunks * 4;
}

cudaError_t launch_select_topk(const double *snr, uint64_t n, int k, const TrackSet &ts, const MapDev &m,
                               void *scratch, stk_hit *out, cudaStream_t st, int *launches)
{
    if (k <= 0 || (uint64_t)k > n || k > STK_MAX_K || n > 0xffffffffull) return cudaErrorInvalidValue;
    unsigned char *p = (unsigned char *)scratch;
    SelState *ss = (SelState *)p;
    unsigned int *idx = (unsigned int *)(p + sizeof(SelState));
    unsigned int *chunk_eq = (unsigned int *)(p + sizeof(SelState) + ((size_t)k * 4 + 255) / 256 * 256);
    int nl = 0;
    sel_init<<<1, 256, 0, st>>>(ss, (unsigned int)k);
    ++nl;
    const uint64_t hb = (n + kHistThreads - 1) / kHistThreads;
    const int hist_grid = (int)(hb < 1184 ? hb : 1184);
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = 56 - 8 * pass;
        sel_hist<<<hist_grid, kHistThreads, 0, st>>>(snr, n, ss, shift);
        sel_pick<<<1, 32, 0, st>>>(ss, shift);
        nl += 2;
    }
    uint64_t nchunks = (n + kHistThreads * 8 - 1) / (kHistThreads * 8);
    if (nchunks > kMaxChunks) nchunks = kMaxChunks;
    if (nchunks < 1) nchunks = 1;
    const uint64_t chunk = (n + nchunks - 1) / nchunks;
    nchunks = (n + chunk - 1) / chunk;
    sel_collect<<<(unsigned)nchunks, kHistThreads, 0, st>>>(snr, n, chunk, ss, idx, chunk_eq);
    sel_ties<<<(unsigned)nchunks, kHistThreads, 0, st>>>(snr, n, chunk, ss, idx, chunk_eq);
    nl += 2;
    int P = 1;
    while (P < k) P <<= 1;
    const size_t smem = (size_t)P * 12;
    cudaError_t e = cudaFuncSetAttribute(sel_finalize, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    sel_finalize<<<1, 1024, smem, st>>>(snr, idx, k, P, ts, m, out);
    ++nl;
    if (launches) *launches = nl;
    return cudaGetLastError();
}

}  // namespace stk
