// Coherent template order: a scheduling pre-pass for the slab kernel.
//
// Templates are independent draws, and the statistic of each (Eq. 7) does not
// depend on the order in which templates are scored, so the slab kernel may
// give a warp any 32 templates.  Given 32 random templates, the lanes' pixel
// bins in a column are random and their shared-memory gathers collide in banks
// (about 6 wavefronts per warp for 8-byte records and 3.5 for the 4-byte weight
// table, against 2 and 1 without conflicts).  Two templates whose control
// frequencies differ by at most d bins are at most d bins apart in every column
// (the curve is a convex combination of f0, f1, f2 with Bernstein weights), so
// scoring templates in an order that keeps neighbours in (f0, f1, f2) together
// puts each warp's bins in a narrow band, where distinct bins fall in distinct
// banks.
//
// The order is a bucket sort of the template indices by a Morton (Z-order) key
// of the three control bins, each reduced to its 7 leading bits:
//   keys:    key[i] of template offset + i, histogram of the keys (atomics)
//   tiles:   per tile of 4096 buckets, the number of templates
//   scan:    exclusive prefix over buckets (tile base + in-tile scan)
//   scatter: perm[pos] = i, pos taken from the bucket's running offset
// Within a bucket the order is whatever the atomics give; no result depends on
// it (each template's sums run over its own columns in column order).
#include "stk_internal.cuh"

namespace stk {

namespace {

constexpr int kTile = 4096;        // buckets per scan tile
constexpr int kScanThreads = 256;  // 16 buckets per thread

// bits 0..9 of x spread to bits 0, 3, 6, ..., 27 (Morton interleave)
__device__ __forceinline__ uint32_t spread3(uint32_t x)
{
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

__global__ void order_keys_kernel(TrackSet ts, uint32_t n_f, int shift, uint32_t *__restrict__ keys,
                                  uint32_t *__restrict__ hist)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ts.n; i += stride) {
        uint32_t f[3];
        double tau;
        draw_track_ts(ts, ts.offset + i, n_f, f, tau);
        const uint32_t key =
            spread3(f[0] >> shift) | (spread3(f[1] >> shift) << 1) | (spread3(f[2] >> shift) << 2);
        keys[i] = key;
        atomicAdd(&hist[key], 1u);
    }
}

__device__ __forceinline__ uint32_t block_sum(uint32_t v, uint32_t *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    uint32_t t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    return t;
}

__global__ void __launch_bounds__(kScanThreads) order_tiles_kernel(const uint32_t *__restrict__ hist, uint32_t nb,
                                                                   uint32_t *__restrict__ tilesum)
{
    __shared__ uint32_t red[kScanThreads / 32];
    const uint32_t base = blockIdx.x * kTile;
    uint32_t v = 0;
    for (uint32_t k = threadIdx.x; k < kTile && base + k < nb; k += kScanThreads) v += hist[base + k];
    const uint32_t t = block_sum(v, red);
    if (threadIdx.x == 0) tilesum[blockIdx.x] = t;
}

// hist[] (counts) becomes the exclusive prefix over all buckets.
__global__ void __launch_bounds__(kScanThreads) order_scan_kernel(uint32_t *__restrict__ hist, uint32_t nb,
                                                                  const uint32_t *__restrict__ tilesum)
{
    __shared__ uint32_t red[kScanThreads / 32];
    __shared__ uint32_t wsum[kScanThreads / 32];
    uint32_t pre = 0;
    for (uint32_t k = threadIdx.x; k < blockIdx.x; k += kScanThreads) pre += tilesum[k];
    const uint32_t base = block_sum(pre, red);

    constexpr int per = kTile / kScanThreads;
    const uint32_t b0 = blockIdx.x * kTile + threadIdx.x * per;
    uint32_t c[per], run = 0;
#pragma unroll
    for (int q = 0; q < per; ++q) {
        c[q] = (b0 + q < nb) ? hist[b0 + q] : 0u;
        run += c[q];
    }
    // exclusive scan of the threads' totals: warp inclusive scan, then warp bases
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    uint32_t inc = run;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (l >= o) inc += y;
    }
    if (l == 31) wsum[w] = inc;
    __syncthreads();
    uint32_t wb = 0;
    for (int k = 0; k < w; ++k) wb += wsum[k];
    uint32_t acc = base + wb + inc - run;
#pragma unroll
    for (int q = 0; q < per; ++q) {
        if (b0 + q < nb) hist[b0 + q] = acc;
        acc += c[q];
    }
}

__global__ void order_scatter_kernel(const uint32_t *__restrict__ keys, uint64_t n, uint32_t *__restrict__ offs,
                                     uint32_t *__restrict__ perm)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t pos = atomicAdd(&offs[keys[i]], 1u);
        perm[pos] = (uint32_t)i;
    }
}

int bit_length(uint32_t x)
{
    int b = 0;
    while (x) {
        ++b;
        x >>= 1;
    }
    return b;
}

void order_shape(int n_f, int &shift, uint32_t &nb)
{
    const int bits = bit_length((uint32_t)(n_f > 1 ? n_f - 1 : 0));
    const int keep = bits < 7 ? bits : 7;
    shift = bits - keep;
    nb = 1u << (3 * keep);
}

}  // namespace

size_t order_scratch_bytes(uint64_t n, int n_f)
{
    int shift;
    uint32_t nb;
    order_shape(n_f, shift, nb);
    const uint64_t ntiles = (nb + kTile - 1) / kTile;
    return (size_t)(2 * n + nb + ntiles) * sizeof(uint32_t) + 256;
}

cudaError_t launch_order(const MapDev &m, const TrackSet &ts, void *scratch, int num_sms, cudaStream_t st,
                         const uint32_t **perm_out, int *launches)
{
    int shift;
    uint32_t nb;
    order_shape(m.n_f, shift, nb);
    const uint32_t ntiles = (nb + kTile - 1) / kTile;
    const uint64_t n = ts.n;
    uint32_t *keys = reinterpret_cast<uint32_t *>(scratch);
    uint32_t *perm = keys + n;
    uint32_t *hist = perm + n;
    uint32_t *tilesum = hist + nb;
    cudaError_t e = cudaMemsetAsync(hist, 0, (size_t)nb * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    const int threads = 256;
    const uint64_t want = (n + threads - 1) / threads;
    const int grid = (int)std::min<uint64_t>(want, (uint64_t)num_sms * 8);
    order_keys_kernel<<<grid, threads, 0, st>>>(ts, (uint32_t)m.n_f, shift, keys, hist);
    order_tiles_kernel<<<ntiles, kScanThreads, 0, st>>>(hist, nb, tilesum);
    order_scan_kernel<<<ntiles, kScanThreads, 0, st>>>(hist, nb, tilesum);
    order_scatter_kernel<<<grid, threads, 0, st>>>(keys, n, hist, perm);
    *perm_out = perm;
    if (launches) *launches = 5;
    return cudaGetLastError();
}

}  // namespace stk
