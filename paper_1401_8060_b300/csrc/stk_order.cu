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
// of the three control bins, each reduced to its leading bits (7 for one map;
// fewer per map in a batch, where map i owns its own range of buckets and of
// positions).  General templates (random control times) are keyed first by
// their start and end columns, so a warp's templates also cover the same
// columns, then by the bins:
//   keys:    bucket of each template, histogram of the buckets (atomics)
//   tiles:   per tile of 4096 buckets, the number of templates
//   bases:   exclusive prefix of the tile counts (one block)
//   scan:    exclusive prefix over buckets (tile base + in-tile scan)
//   scatter: perm[pos] = i (index within its map), pos from the bucket's offset
// Within a bucket the order is whatever the atomics give; no result depends on
// it (each template's sums run over its own columns in column order).
#include <algorithm>

#include "stk_internal.cuh"

namespace stk {

namespace {

constexpr int kTile = 4096;        // buckets per scan tile
constexpr int kScanThreads = 256;  // 16 buckets per thread
constexpr int kBaseThreads = 1024; // one block scans the tile counts

struct OrderArgs {
    const OrderMap *maps;  // device array (grid.y = map), or NULL: `single`
    OrderMap single;
};

__device__ __forceinline__ const OrderMap &order_map(const OrderArgs &a)
{
    return a.maps ? a.maps[blockIdx.y] : a.single;
}

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

__global__ void order_keys_kernel(OrderArgs a, uint32_t *__restrict__ keys, uint32_t *__restrict__ hist)
{
    const OrderMap &om = order_map(a);
    const TrackSet ts = om.ts;
    const uint32_t n_f = om.n_f, bucket0 = om.bucket0, pos0 = om.pos0;
    const int shift = om.shift;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ts.n; i += stride) {
        uint32_t f[3];
        double tau;
        draw_track_ts(ts, ts.offset + i, n_f, f, tau);
        uint32_t key = spread3(f[0] >> shift) | (spread3(f[1] >> shift) << 1) | (spread3(f[2] >> shift) << 2);
        if (ts.general) {  // start and end column first: a warp's templates cover the same columns
            uint32_t t[3];
            draw_times(ts.seed, ts.offset + i, om.n_t, (uint32_t)ts.t_min, t);
            key |= (((t[0] >> om.tshift) << 4) | (t[2] >> om.tshift)) << 12;
        }
        key += bucket0;
        keys[pos0 + i] = key;
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

// Exclusive scan of each thread's `run` over the block (warp scans, then warp bases).
__device__ __forceinline__ uint32_t block_exclusive(uint32_t run, uint32_t *wsum)
{
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
    return wb + inc - run;
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

// tilesum[] (counts) becomes the exclusive prefix over tiles; one block.
__global__ void __launch_bounds__(kBaseThreads) order_bases_kernel(uint32_t *__restrict__ tilesum, uint32_t ntiles)
{
    __shared__ uint32_t wsum[kBaseThreads / 32];
    const uint32_t per = (ntiles + kBaseThreads - 1) / kBaseThreads;
    const uint32_t b0 = threadIdx.x * per;
    uint32_t run = 0;
    for (uint32_t q = 0; q < per && b0 + q < ntiles; ++q) run += tilesum[b0 + q];
    uint32_t acc = block_exclusive(run, wsum);
    for (uint32_t q = 0; q < per && b0 + q < ntiles; ++q) {
        const uint32_t c = tilesum[b0 + q];
        tilesum[b0 + q] = acc;
        acc += c;
    }
}

// hist[] (counts) becomes the exclusive prefix over all buckets.
__global__ void __launch_bounds__(kScanThreads) order_scan_kernel(uint32_t *__restrict__ hist, uint32_t nb,
                                                                  const uint32_t *__restrict__ tilebase)
{
    __shared__ uint32_t wsum[kScanThreads / 32];
    constexpr int per = kTile / kScanThreads;
    const uint32_t b0 = blockIdx.x * kTile + threadIdx.x * per;
    uint32_t c[per], run = 0;
#pragma unroll
    for (int q = 0; q < per; ++q) {
        c[q] = (b0 + q < nb) ? hist[b0 + q] : 0u;
        run += c[q];
    }
    uint32_t acc = tilebase[blockIdx.x] + block_exclusive(run, wsum);
#pragma unroll
    for (int q = 0; q < per; ++q) {
        if (b0 + q < nb) hist[b0 + q] = acc;
        acc += c[q];
    }
}

__global__ void order_scatter_kernel(OrderArgs a, const uint32_t *__restrict__ keys, uint32_t *__restrict__ offs,
                                     uint32_t *__restrict__ perm)
{
    const OrderMap &om = order_map(a);
    const uint64_t n = om.ts.n;
    const uint32_t pos0 = om.pos0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t pos = atomicAdd(&offs[keys[pos0 + i]], 1u);
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

cudaError_t run_order(const OrderArgs &oa, int n_maps, uint64_t max_n, uint64_t total_n, uint64_t nb,
                      void *scratch, int num_sms, cudaStream_t st, const uint32_t **perm_out, int *launches)
{
    const uint32_t ntiles = (uint32_t)((nb + kTile - 1) / kTile);
    uint32_t *keys = reinterpret_cast<uint32_t *>(scratch);
    uint32_t *perm = keys + total_n;
    uint32_t *hist = perm + total_n;
    uint32_t *tilesum = hist + nb;
    cudaError_t e = cudaMemsetAsync(hist, 0, (size_t)nb * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    const int threads = 256;
    // about 8 blocks per SM over all maps
    const uint64_t want = std::max<uint64_t>(1, std::min<uint64_t>((max_n + threads - 1) / threads,
                                                                    (uint64_t)num_sms * 8 / (uint64_t)n_maps + 1));
    const dim3 grid((unsigned)want, (unsigned)n_maps);
    order_keys_kernel<<<grid, threads, 0, st>>>(oa, keys, hist);
    order_tiles_kernel<<<ntiles, kScanThreads, 0, st>>>(hist, (uint32_t)nb, tilesum);
    order_bases_kernel<<<1, kBaseThreads, 0, st>>>(tilesum, ntiles);
    order_scan_kernel<<<ntiles, kScanThreads, 0, st>>>(hist, (uint32_t)nb, tilesum);
    order_scatter_kernel<<<grid, threads, 0, st>>>(oa, keys, hist, perm);
    *perm_out = perm;
    if (launches) *launches = 6;
    return cudaGetLastError();
}

}  // namespace

void order_shape(int n_f, int max_bits, int &shift, int &bits)
{
    const int b = bit_length((uint32_t)(n_f > 1 ? n_f - 1 : 0));
    bits = b < max_bits ? b : max_bits;
    shift = b - bits;
}

size_t order_scratch_bytes_total(uint64_t total_n, uint64_t total_buckets)
{
    const uint64_t ntiles = (total_buckets + kTile - 1) / kTile;
    return (size_t)(2 * total_n + total_buckets + ntiles) * sizeof(uint32_t) + 256;
}

// Pinned templates: 7 bits per control bin (2^21 buckets).  General templates:
// 4 bits each of the start and end column, then 4 bits per control bin (2^20).
size_t order_scratch_bytes(uint64_t n, int n_f, bool general)
{
    int shift, bits;
    order_shape(n_f, 7, shift, bits);
    // general keys place the time bits at bit 12 whatever the bin bits in use
    return order_scratch_bytes_total(n, general ? (1ull << 20) : (1ull << (3 * bits)));
}

cudaError_t launch_order(const MapDev &m, const TrackSet &ts, void *scratch, int num_sms, cudaStream_t st,
                         const uint32_t **perm_out, int *launches)
{
    OrderArgs oa{};
    oa.maps = nullptr;
    oa.single.ts = ts;
    oa.single.n_f = (uint32_t)m.n_f;
    int bits, tbits;
    order_shape(m.n_f, ts.general ? 4 : 7, oa.single.shift, bits);
    order_shape(m.n_t, 4, oa.single.tshift, tbits);
    oa.single.n_t = (uint32_t)m.n_t;
    oa.single.bucket0 = 0;
    oa.single.pos0 = 0;
    // general keys place the time bits at bit 12 whatever the bin bits in use
    const uint64_t nb = ts.general ? (1ull << 20) : (1ull << (3 * bits));
    return run_order(oa, 1, ts.n, ts.n, nb, scratch, num_sms, st, perm_out, launches);
}

cudaError_t launch_order_batch(const OrderMap *d_maps, int n_maps, uint64_t max_n, uint64_t total_n,
                               uint64_t total_buckets, void *scratch, int num_sms, cudaStream_t st,
                               const uint32_t **perm_out, int *launches)
{
    OrderArgs oa{};
    oa.maps = d_maps;
    return run_order(oa, n_maps, max_n, total_n, total_buckets, scratch, num_sms, st, perm_out, launches);
}

}  // namespace stk
