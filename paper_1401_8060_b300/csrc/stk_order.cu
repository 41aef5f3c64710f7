// Coherent template order: a scheduling pre-pass for the slab, batched and
// general-template kernels.
//
// Templates are independent draws, and the statistic of each (Eq. 7) does not
// depend on the order in which templates are scored, so a kernel may give a
// warp any 32 templates.  Given 32 random templates, the lanes' pixel bins in a
// column are random and their shared-memory gathers collide in banks (about 6
// wavefronts per warp for 8-byte records and 3.5 for the 4-byte weight table,
// against 2 and 1 without conflicts).  Two templates whose control frequencies
// differ by at most d bins are at most d bins apart in every column (the curve
// is a convex combination of f0, f1, f2 with Bernstein weights), so scoring
// templates in an order that keeps neighbours in (f0, f1, f2) together puts
// each warp's bins in a narrow band, where distinct bins fall in distinct banks.
//
// The order sorts template positions by a key: the position along a 3-D Hilbert
// curve of the leading bits of f0, of the middle column's bin (f0 + 2 f1 + f2) / 4
// and of f2 (7 bits each for one map, fewer per map in large batches); general
// templates (random control times) put 6 bits each of the start and end column
// above a Morton (Z-order) interleave of 3 bits per bin, so a warp's templates
// also cover the same columns.  The Hilbert curve keeps consecutive keys in
// adjacent cells (a Z-order curve jumps between distant cells), and the middle
// bin measures the spread of the middle columns more directly than f1: both
// lower the bank conflicts of the slab kernel's gathers (realistic workload:
// 4.51 -> 4.15 shared wavefronts per 32 track-pixels, measured).  Map i of a batch owns its own key range and position range.  The
// sort is two-level; its only global atomic is one ticket counter:
//   keys:    draw each template, write its key, count coarse buckets (the top
//            key bits) per block in shared memory
//   columns: per coarse bucket, the exclusive prefix over blocks and, in the
//            last of its blocks to finish, the exclusive prefix over buckets
//   coarse:  each block places its templates into their coarse buckets (sorted
//            by bucket in shared memory first, when they fit)
//   fine:    one block per coarse bucket sorts it by the remaining key bits
//            (counting sort in shared memory) and writes the positions
// Within a fine bucket the order is whatever the shared atomics give; no result
// depends on it (each template's sums run over its own columns in column order).
#include <algorithm>
#include <vector>

#include "stk_internal.cuh"

namespace stk {

namespace {

constexpr int kKeyThreads = 1024;  // keys and coarse kernels
constexpr int kFineThreads = 256;  // fine kernel
constexpr int kFineCache = 2048;   // fine kernel: bucket sizes held in registers
constexpr int kFineShift = 14;     // stored key = coarse << 14 | fine
constexpr uint32_t kMaxCoarse = 8192;
constexpr int kGenTimeBits = 6;             // general templates: key bits of the start and of the end column
constexpr int kGenBinBits = 3;              // general templates: key bits of each control bin
constexpr uint32_t kStageSmem = 227 * 1024 - 1024;  // staged coarse kernel: dynamic shared memory budget
constexpr int kStagedGridMax = 8192;        // blocks beyond which the unstaged coarse kernel runs

struct OrderArgs {
    const OrderMap *maps;  // device array, or NULL: `single`
    OrderMap single;
    int n_maps;
    uint64_t total_n;
    uint32_t nc;           // coarse buckets
    int grid;              // blocks of the keys and coarse kernels
};

__device__ __forceinline__ const OrderMap &omap(const OrderArgs &a, int i) { return a.maps ? a.maps[i] : a.single; }

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

// The map holding position p (maps are contiguous in position order).
__device__ __forceinline__ int map_of(const OrderArgs &a, uint64_t p)
{
    int lo = 0, hi = a.n_maps - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((uint64_t)omap(a, mid).pos0 <= p) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Block b's share of all positions.
__device__ __forceinline__ void block_range(const OrderArgs &a, uint64_t &p0, uint64_t &p1)
{
    const uint64_t chunk = (a.total_n + a.grid - 1) / a.grid;
    p0 = (uint64_t)blockIdx.x * chunk;
    p1 = p0 + chunk < a.total_n ? p0 + chunk : a.total_n;
}

// Position of (x0, x1, x2), `bits` bits each, along a 3-D Hilbert curve: Skilling's
// transform of the coordinates to the curve's "transposed" index (Gray-code
// inverse and the excess-undo loop), whose bits interleaved with x0's first give
// the index.
__device__ __forceinline__ uint32_t hilbert3(uint32_t x0, uint32_t x1, uint32_t x2, int bits)
{
    if (bits <= 0) return 0u;
    uint32_t X[3] = {x0, x1, x2};
    const uint32_t top = 1u << (bits - 1);
    // Q-th bit set in X[i]: invert the low bits of X[0]; else exchange them with X[i]'s
    // (selects, not branches: the lanes of a warp hold different templates)
    for (uint32_t Q = top; Q > 1; Q >>= 1) {
        const uint32_t P = Q - 1;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const bool set = (X[i] & Q) != 0;
            const uint32_t t = set ? 0u : (X[0] ^ X[i]) & P;
            X[0] ^= set ? P : t;
            if (i) X[i] ^= t;
        }
    }
    X[1] ^= X[0];
    X[2] ^= X[1];
    uint32_t t = 0;
    for (uint32_t Q = top; Q > 1; Q >>= 1) t ^= (X[2] & Q) ? Q - 1 : 0u;
    X[0] ^= t;
    X[1] ^= t;
    X[2] ^= t;
    return (spread3(X[0]) << 2) | (spread3(X[1]) << 1) | spread3(X[2]);
}

// Hilbert indices of every cell at 1..7 bits a coordinate, so the keys kernel
// looks a key up (one 4-byte gather from a 9.6 MB table that stays in L2)
// instead of running the transform: bits b start at hilbert_tab_offset(b), cell
// (x0, x1, x2) at (x0 << 2b) | (x1 << b) | x2.  Filled once per device by
// order_build_tables from hilbert3 itself, so the keys are those of the
// transform.
constexpr int kHilbertTabBits = 7;
__host__ __device__ constexpr uint32_t hilbert_tab_offset(int b)
{
    return (uint32_t)(((1ull << (3 * b)) - 8ull) / 7ull);  // sum of 8^i for i = 1 .. b - 1
}
constexpr uint32_t kHilbertTabEntries = hilbert_tab_offset(kHilbertTabBits + 1);
__device__ uint32_t g_hilbert_tab[kHilbertTabEntries];

__global__ void __launch_bounds__(256) hilbert_table_kernel()
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < kHilbertTabEntries; i += gridDim.x * blockDim.x) {
        int b = 1;
        while (i >= hilbert_tab_offset(b + 1)) ++b;
        const uint32_t c = i - hilbert_tab_offset(b), mask = (1u << b) - 1u;
        g_hilbert_tab[i] = hilbert3(c >> (2 * b), (c >> b) & mask, c & mask, b);
    }
}

// Key of one template: Hilbert index of its control bins (general templates: the
// start and end column above a Morton code of the bins), split into coarse bucket
// and fine bits.
template <bool GENERAL>
__device__ __forceinline__ uint32_t template_key(const TrackSet &ts, uint64_t g, uint32_t n_f, uint32_t n_t, int shift,
                                                 int bbits, int tshift, int tbits, int fbits, uint32_t coarse0)
{
    uint32_t f[3];
    double tau;
    draw_track_ts(ts, g, n_f, f, tau);
    uint32_t key;
    if (GENERAL) {  // start and end column first: a warp's templates cover the same columns
        key = spread3(f[0] >> shift) | (spread3(f[1] >> shift) << 1) | (spread3(f[2] >> shift) << 2);
        uint32_t t[3];
        draw_times(ts.seed, g, n_t, (uint32_t)ts.t_min, t);
        key |= (((t[0] >> tshift) << tbits) | (t[2] >> tshift)) << (3 * kGenBinBits);
    } else {
        const uint32_t mid = (f[0] + 2 * f[1] + f[2]) >> 2;
        key = bbits > 0 ? __ldg(g_hilbert_tab + hilbert_tab_offset(bbits) +
                                (((f[0] >> shift) << (2 * bbits)) | ((mid >> shift) << bbits) | (f[2] >> shift)))
                        : 0u;
    }
    const uint32_t c = coarse0 + (key >> fbits);
    return (c << kFineShift) | (key & ((1u << fbits) - 1u));
}

// MULTI: several maps (else a.single); GENERAL: general templates (else pinned).
template <bool MULTI, bool GENERAL>
__global__ void __launch_bounds__(kKeyThreads, 1) order_keys_kernel(OrderArgs a, uint32_t *__restrict__ keys,
                                                                    uint32_t *__restrict__ blockhist,
                                                                    unsigned int *done)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) *done = 0u;  // the columns kernel's ticket counter
    extern __shared__ uint32_t hc[];  // [nc]
    for (uint32_t c = threadIdx.x; c < a.nc; c += blockDim.x) hc[c] = 0;
    __syncthreads();
    uint64_t p0, p1;  // 64-bit: positions reach 2^32 - 1, the loop steps past them
    block_range(a, p0, p1);
    if (MULTI) {
        if (p0 + threadIdx.x < p1) {
            int mi = map_of(a, p0 + threadIdx.x);
            for (uint64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
                while (mi + 1 < a.n_maps && (uint64_t)a.maps[mi + 1].pos0 <= p) ++mi;
                const OrderMap &om = a.maps[mi];
                const uint32_t k = template_key<GENERAL>(om.ts, om.ts.offset + (p - om.pos0), om.n_f, om.n_t,
                                                         om.shift, om.bbits, om.tshift, om.tbits, om.fbits,
                                                         om.coarse0);
                keys[p] = k;
                atomicAdd(&hc[k >> kFineShift], 1u);
            }
        }
    } else {
        const OrderMap &om = a.single;  // read from the parameters where used
        for (uint64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
            const uint32_t k = template_key<GENERAL>(om.ts, om.ts.offset + p, om.n_f, om.n_t, om.shift, om.bbits,
                                                     om.tshift, om.tbits, om.fbits, 0u);
            keys[p] = k;
            atomicAdd(&hc[k >> kFineShift], 1u);
        }
    }
    __syncthreads();
    for (uint32_t c = threadIdx.x; c < a.nc; c += blockDim.x) blockhist[(size_t)blockIdx.x * a.nc + c] = hc[c];
}

// base[c] = exclusive prefix of total over coarse buckets, by one block.
__device__ void bucket_bases(const uint32_t *total, uint32_t nc, uint32_t *base)
{
    __shared__ uint32_t wsum[32];
    const uint32_t per = (nc + blockDim.x - 1) / blockDim.x;
    const uint32_t c0 = threadIdx.x * per;
    uint32_t run = 0;
    for (uint32_t q = 0; q < per && c0 + q < nc; ++q) run += __ldcg(total + c0 + q);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    uint32_t inc = run;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (l >= o) inc += y;
    }
    if (l == 31) wsum[w] = inc;
    __syncthreads();
    uint32_t acc = inc - run;
    for (int k = 0; k < w; ++k) acc += wsum[k];
    for (uint32_t q = 0; q < per && c0 + q < nc; ++q) {
        base[c0 + q] = acc;
        acc += __ldcg(total + c0 + q);
    }
}

// blockhist[b][c] becomes, for each coarse bucket c, the exclusive prefix over
// blocks b; total[c] the bucket's size; then base[c], the prefix over buckets.  A block takes 32 buckets (one per lane)
// and its 32 warps a share of the blocks each: warp sums, a scan over warps,
// then each warp writes its share's prefixes.
__global__ void __launch_bounds__(1024) order_columns_kernel(uint32_t *__restrict__ blockhist, uint32_t nc,
                                                             int grid, uint32_t *__restrict__ total,
                                                             uint32_t *__restrict__ base, unsigned int *done)
{
    __shared__ bool last;
    __shared__ uint32_t part[32][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t c = blockIdx.x * 32 + lane;
    const int per = (grid + 31) / 32, b0 = w * per, b1 = min(grid, b0 + per);
    uint32_t sum = 0;
    if (c < nc)
        for (int b = b0; b < b1; ++b) sum += blockhist[(size_t)b * nc + c];
    part[w][lane] = sum;
    __syncthreads();
    uint32_t before = 0, all = 0;
    for (int k = 0; k < 32; ++k) {
        const uint32_t v = part[k][lane];
        if (k < w) before += v;
        all += v;
    }
    if (c < nc) {
        for (int b = b0; b < b1; ++b) {
            uint32_t *e = blockhist + (size_t)b * nc + c;
            const uint32_t v = *e;
            *e = before;
            before += v;
        }
        if (w == 0) total[c] = all;
    }
    // the last block to finish (a ticket counter, zeroed by the keys kernel) also
    // takes the prefix over buckets; no block waits for another
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    bucket_bases(total, nc, base);
}

// Each block places its positions into their coarse buckets: tmp[slot] = fine << 32 | position.
__global__ void __launch_bounds__(kKeyThreads) order_coarse_kernel(OrderArgs a, const uint32_t *__restrict__ keys,
                                                                   const uint32_t *__restrict__ blockhist,
                                                                   const uint32_t *__restrict__ base,
                                                                   unsigned long long *__restrict__ tmp)
{
    extern __shared__ uint32_t ctr[];  // [nc]
    for (uint32_t c = threadIdx.x; c < a.nc; c += blockDim.x)
        ctr[c] = base[c] + blockhist[(size_t)blockIdx.x * a.nc + c];
    __syncthreads();
    uint64_t p0, p1;
    block_range(a, p0, p1);
    for (uint64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
        const uint32_t key = keys[p];
        const uint32_t slot = atomicAdd(&ctr[key >> kFineShift], 1u);
        tmp[slot] = ((unsigned long long)(key & ((1u << kFineShift) - 1u)) << 32) | (uint32_t)p;
    }
}

// As order_coarse_kernel, for blocks whose positions fit shared memory: the block
// first sorts its entries by coarse bucket in shared memory, then writes them
// out in that order, so a warp's stores run through consecutive slots of each
// bucket (about four per bucket per block) instead of scattering one by one.
// The block's count per bucket is the next block's prefix minus its own (the
// last block: the bucket's total).
__global__ void __launch_bounds__(kKeyThreads) order_coarse_staged_kernel(OrderArgs a,
                                                                          const uint32_t *__restrict__ keys,
                                                                          const uint32_t *__restrict__ blockhist,
                                                                          const uint32_t *__restrict__ total,
                                                                          const uint32_t *__restrict__ base,
                                                                          unsigned long long *__restrict__ tmp)
{
    extern __shared__ uint32_t sm[];  // cursor[nc], delta[nc], stage[chunk] (8 B), bucket[chunk] (2 B)
    __shared__ uint32_t wsum[kKeyThreads / 32];
    const uint32_t nc = a.nc, b = blockIdx.x;
    const uint64_t chunk = (a.total_n + a.grid - 1) / a.grid;
    uint32_t *cursor = sm, *delta = sm + nc;
    unsigned long long *stage = reinterpret_cast<unsigned long long *>(sm + 2 * nc);
    uint16_t *sbk = reinterpret_cast<uint16_t *>(stage + chunk);
    // exclusive scan of this block's counts over the buckets: each thread a run of them
    const uint32_t per = (nc + blockDim.x - 1) / blockDim.x, c0 = threadIdx.x * per;
    const uint32_t *pre = blockhist + (size_t)b * nc;
    const uint32_t *nxt = blockhist + (size_t)(b + 1) * nc;
    const bool last = (int)b + 1 == a.grid;
    uint32_t run = 0;
    for (uint32_t q = 0; q < per && c0 + q < nc; ++q) run += (last ? total[c0 + q] : nxt[c0 + q]) - pre[c0 + q];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    uint32_t inc = run;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (l >= o) inc += y;
    }
    if (l == 31) wsum[w] = inc;
    __syncthreads();
    uint32_t acc = inc - run;
    for (int k = 0; k < w; ++k) acc += wsum[k];
    for (uint32_t q = 0; q < per && c0 + q < nc; ++q) {
        const uint32_t c = c0 + q;
        cursor[c] = acc;
        delta[c] = base[c] + pre[c] - acc;  // global slot of local position i in bucket c: delta[c] + i
        acc += (last ? total[c] : nxt[c]) - pre[c];
    }
    __syncthreads();
    uint64_t p0, p1;
    block_range(a, p0, p1);
    constexpr int U = 4;  // key loads in flight per thread
    for (uint64_t pb = p0 + threadIdx.x; pb < p1; pb += U * (uint64_t)blockDim.x) {
        uint32_t kk[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t p = pb + (uint64_t)u * blockDim.x;
            kk[u] = p < p1 ? keys[p] : 0u;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t p = pb + (uint64_t)u * blockDim.x;
            if (p < p1) {
                const uint32_t c = kk[u] >> kFineShift;
                const uint32_t i = atomicAdd(&cursor[c], 1u);
                stage[i] = ((unsigned long long)(kk[u] & ((1u << kFineShift) - 1u)) << 32) | (uint32_t)p;
                sbk[i] = (uint16_t)c;
            }
        }
    }
    __syncthreads();
    const uint32_t m = (uint32_t)(p1 > p0 ? p1 - p0 : 0);
    for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) tmp[delta[sbk[i]] + i] = stage[i];
}

// One block per coarse bucket: counting sort by the fine key bits; perm[pos] =
// the template's index within its map.
__global__ void __launch_bounds__(kFineThreads) order_fine_kernel(OrderArgs a,
                                                                  const unsigned long long *__restrict__ tmp,
                                                                  const uint32_t *__restrict__ base,
                                                                  const uint32_t *__restrict__ total,
                                                                  uint32_t *__restrict__ perm)
{
    extern __shared__ uint32_t hf[];  // [2^fbits]
    __shared__ uint32_t wsum[kFineThreads / 32];
    const uint32_t c = blockIdx.x;
    const uint32_t n = total[c];
    if (n == 0) return;
    // the bucket's map: the last one whose first coarse bucket is <= c
    int lo = 0, hi = a.n_maps - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (omap(a, mid).coarse0 <= c) lo = mid;
        else hi = mid - 1;
    }
    const OrderMap &om = omap(a, lo);
    const uint32_t nb = 1u << om.fbits, pos0 = om.pos0, b0 = base[c];
    for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) hf[i] = 0;
    __syncthreads();
    // buckets of up to kFineCache elements stay in registers between the two passes
    constexpr int kPer = kFineCache / kFineThreads;
    const bool cached = n <= (uint32_t)kFineCache;
    unsigned long long r[kPer];
    if (cached) {
#pragma unroll
        for (int u = 0; u < kPer; ++u) {  // every load in flight before the first atomic
            const uint32_t i = threadIdx.x + u * kFineThreads;
            r[u] = i < n ? tmp[b0 + i] : 0ull;
        }
#pragma unroll
        for (int u = 0; u < kPer; ++u)
            if (threadIdx.x + u * kFineThreads < n) atomicAdd(&hf[(uint32_t)(r[u] >> 32)], 1u);
    } else {
        for (uint64_t i = threadIdx.x; i < n; i += blockDim.x)
            atomicAdd(&hf[(uint32_t)(tmp[(uint64_t)b0 + i] >> 32)], 1u);
    }
    __syncthreads();
    // exclusive scan of hf: each thread a contiguous run of bins
    const uint32_t per = (nb + blockDim.x - 1) / blockDim.x;
    const uint32_t f0 = threadIdx.x * per;
    uint32_t run = 0;
    for (uint32_t q = 0; q < per && f0 + q < nb; ++q) run += hf[f0 + q];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    uint32_t inc = run;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (l >= o) inc += y;
    }
    if (l == 31) wsum[w] = inc;
    __syncthreads();
    uint32_t acc = inc - run;
    for (int k = 0; k < w; ++k) acc += wsum[k];
    for (uint32_t q = 0; q < per && f0 + q < nb; ++q) {
        const uint32_t v = hf[f0 + q];
        hf[f0 + q] = acc;
        acc += v;
    }
    __syncthreads();
    if (cached) {
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const uint32_t i = threadIdx.x + u * kFineThreads;
            if (i < n) {
                const uint32_t q = atomicAdd(&hf[(uint32_t)(r[u] >> 32)], 1u);
                perm[b0 + q] = (uint32_t)r[u] - pos0;
            }
        }
        return;
    }
    for (uint64_t i = threadIdx.x; i < n; i += blockDim.x) {  // 64-bit: n may approach 2^32
        const unsigned long long e = tmp[(uint64_t)b0 + i];
        const uint32_t q = atomicAdd(&hf[(uint32_t)(e >> 32)], 1u);
        perm[(uint64_t)b0 + q] = (uint32_t)e - pos0;
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

struct Layout {
    uint32_t *keys, *perm, *blockhist, *total, *base;
    unsigned int *done;
    unsigned long long *tmp;
};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Scratch layout (and its size): tmp[n] u64, keys[n], perm[n], blockhist[grid][nc], total[nc], base[nc],
// the columns kernel's ticket counter.
size_t layout_bytes(uint64_t total_n, uint32_t nc, int grid, Layout *L, void *scratch)
{
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += align256(bytes);
        return o;
    };
    const size_t o_tmp = take(total_n * 8), o_keys = take(total_n * 4), o_perm = take(total_n * 4);
    const size_t o_bh = take((size_t)nc * grid * 4), o_tot = take((size_t)nc * 4), o_base = take((size_t)nc * 4);
    const size_t o_done = take(4);
    if (L) {
        unsigned char *s = static_cast<unsigned char *>(scratch);
        L->tmp = reinterpret_cast<unsigned long long *>(s + o_tmp);
        L->keys = reinterpret_cast<uint32_t *>(s + o_keys);
        L->perm = reinterpret_cast<uint32_t *>(s + o_perm);
        L->blockhist = reinterpret_cast<uint32_t *>(s + o_bh);
        L->total = reinterpret_cast<uint32_t *>(s + o_tot);
        L->base = reinterpret_cast<uint32_t *>(s + o_base);
        L->done = reinterpret_cast<unsigned int *>(s + o_done);
    }
    return off;
}

// Positions per block the staged coarse kernel holds with nc coarse buckets
// (8 bytes of entry and 2 of bucket each, after 8 nc bytes of counters).
uint64_t stage_cap(uint32_t nc) { return (kStageSmem - 8 * (uint64_t)nc) / 10; }

// Blocks of the keys and coarse kernels: twice the SMs when each block's
// positions fit the staged coarse kernel (or when nothing fits within
// kStagedGridMax blocks), else the next multiple of that which fits.
int order_grid(int num_sms, uint64_t total_n, uint32_t nc)
{
    const uint64_t g0 = 2 * (uint64_t)std::max(1, num_sms), cap = stage_cap(nc);
    if ((total_n + g0 - 1) / g0 <= cap) return (int)g0;
    const uint64_t need = (total_n + cap - 1) / cap, g = (need + g0 - 1) / g0 * g0;
    return (int)(g <= (uint64_t)kStagedGridMax ? g : g0);
}

bool staged_ok(uint64_t total_n, int grid, uint32_t nc) { return (total_n + grid - 1) / grid <= stage_cap(nc); }

int staged_smem(uint64_t total_n, int grid, uint32_t nc)
{
    return (int)(8 * (uint64_t)nc + 10 * ((total_n + grid - 1) / grid));
}

cudaError_t run_order(const OrderArgs &oa, uint32_t max_fbits, void *scratch, cudaStream_t st,
                      const uint32_t **perm_out, int *launches)
{
    Layout L;
    layout_bytes(oa.total_n, oa.nc, oa.grid, &L, scratch);
    const size_t smem_c = (size_t)oa.nc * 4, smem_f = (size_t)4 << max_fbits;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return e;
    if (cs == cudaStreamCaptureStatusNone && (e = order_prepare(oa.nc, max_fbits)) != cudaSuccess) return e;
    // batches hold pinned templates only; one map may hold either kind
    if (oa.maps)
        order_keys_kernel<true, false><<<oa.grid, kKeyThreads, smem_c, st>>>(oa, L.keys, L.blockhist, L.done);
    else if (oa.single.ts.general)
        order_keys_kernel<false, true><<<oa.grid, kKeyThreads, smem_c, st>>>(oa, L.keys, L.blockhist, L.done);
    else
        order_keys_kernel<false, false><<<oa.grid, kKeyThreads, smem_c, st>>>(oa, L.keys, L.blockhist, L.done);
    order_columns_kernel<<<(oa.nc + 31) / 32, 1024, 0, st>>>(L.blockhist, oa.nc, oa.grid, L.total, L.base, L.done);
    if (staged_ok(oa.total_n, oa.grid, oa.nc))
        order_coarse_staged_kernel<<<oa.grid, kKeyThreads, staged_smem(oa.total_n, oa.grid, oa.nc), st>>>(
            oa, L.keys, L.blockhist, L.total, L.base, L.tmp);
    else
        order_coarse_kernel<<<oa.grid, kKeyThreads, smem_c, st>>>(oa, L.keys, L.blockhist, L.base, L.tmp);
    order_fine_kernel<<<oa.nc, kFineThreads, smem_f, st>>>(oa, L.tmp, L.base, L.total, L.perm);
    *perm_out = L.perm;
    if (launches) *launches = 4;
    return cudaGetLastError();
}



}  // namespace

cudaError_t order_build_tables(cudaStream_t st)
{
    hilbert_table_kernel<<<(kHilbertTabEntries + 255) / 256, 256, 0, st>>>();
    return cudaGetLastError();
}

// Shared-memory limits of the order kernels on the current device (not while a
// stream is being captured: batches call this before capturing their graph).
cudaError_t order_prepare(uint32_t nc, uint32_t max_fbits)
{
    // the largest any pass may ask for, whatever this one needs: a later pass (or
    // a graph captured later) never finds a limit lowered by an earlier one
    (void)nc;
    (void)max_fbits;
    const int smem_c = (int)kMaxCoarse * 4, smem_f = 4 << kFineShift;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(order_keys_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  smem_c)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(order_keys_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  smem_c)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(order_keys_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  smem_c)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(order_keys_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  smem_c)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(order_coarse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_c)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(order_coarse_staged_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kStageSmem)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(order_fine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_f)) !=
            cudaSuccess)
        return e;
    return cudaSuccess;
}

namespace {

// Single map: the key's top 12 bits (or all, if fewer) are the coarse bucket.
void single_plan(const MapDev &m, const TrackSet &ts, OrderMap &om, uint32_t &nc)
{
    om = OrderMap{};
    om.ts = ts;
    om.n_f = (uint32_t)m.n_f;
    om.n_t = (uint32_t)m.n_t;
    int bits;
    order_shape(m.n_f, ts.general ? kGenBinBits : 7, om.shift, bits);
    om.bbits = bits;
    order_shape(m.n_t, kGenTimeBits, om.tshift, om.tbits);
    // general keys: 2 x 6 bits of start and end column above 3 x 3 bits of the
    // bins (at bit 9 whatever the bin bits in use); the columns group a warp's
    // templates more than the bins do (measured: 1.26 ms with 4 bits for each
    // column and bin, 1.22 ms with 6 and 3 or 6 and 4)
    const int kb = ts.general ? 3 * kGenBinBits + 2 * om.tbits : 3 * bits;
    const int cb = std::min(kb, 12);
    om.fbits = kb - cb;
    om.coarse0 = 0;
    om.pos0 = 0;
    nc = 1u << cb;
}

}  // namespace

void order_shape(int n_f, int max_bits, int &shift, int &bits)
{
    const int b = bit_length((uint32_t)(n_f > 1 ? n_f - 1 : 0));
    bits = b < max_bits ? b : max_bits;
    shift = b - bits;
}

void order_plan_maps(OrderMap *maps, int n_maps, uint32_t &nc, uint32_t &max_fbits)
{
    // coarse bits per map so that all maps together have at most kMaxCoarse
    // buckets; at most 14 fine bits, which bounds the bits per control bin
    int cbits = 12;
    while (cbits > 0 && ((uint64_t)n_maps << cbits) > kMaxCoarse) --cbits;
    const int max_bits = std::min(7, (kFineShift + cbits) / 3);
    nc = 0;
    max_fbits = 0;
    for (int i = 0; i < n_maps; ++i) {
        OrderMap &om = maps[i];
        int bits;
        order_shape((int)om.n_f, om.ts.general ? std::min(kGenBinBits, max_bits) : max_bits, om.shift, bits);
        om.bbits = bits;
        // general keys: time bits limited so that at most kFineShift bits lie below the coarse bucket
        order_shape((int)om.n_t,
                    std::max(0, std::min(kGenTimeBits, (kFineShift + cbits - 3 * kGenBinBits) / 2)), om.tshift,
                    om.tbits);
        const int kb = om.ts.general ? 3 * kGenBinBits + 2 * om.tbits : 3 * bits;
        const int cb = std::min(kb, cbits);
        om.fbits = kb - cb;
        om.coarse0 = nc;
        nc += 1u << cb;
        max_fbits = std::max<uint32_t>(max_fbits, (uint32_t)om.fbits);
    }
}

size_t order_scratch_bytes_maps(uint64_t total_n, uint32_t nc, int num_sms)
{
    return layout_bytes(total_n, nc, order_grid(num_sms, total_n, nc), nullptr, nullptr);
}

size_t order_scratch_bytes(uint64_t n, int n_f, int n_t, bool general, int num_sms)
{
    MapDev m{};
    m.n_f = n_f;
    m.n_t = n_t;
    TrackSet ts{};
    ts.general = general ? 1 : 0;
    OrderMap om;
    uint32_t nc;
    single_plan(m, ts, om, nc);
    return layout_bytes(n, nc, order_grid(num_sms, n, nc), nullptr, nullptr);
}

cudaError_t launch_order(const MapDev &m, const TrackSet &ts, void *scratch, int num_sms, cudaStream_t st,
                         const uint32_t **perm_out, int *launches)
{
    OrderArgs oa{};
    oa.maps = nullptr;
    single_plan(m, ts, oa.single, oa.nc);
    oa.n_maps = 1;
    oa.total_n = ts.n;
    oa.grid = order_grid(num_sms, oa.total_n, oa.nc);
    return run_order(oa, (uint32_t)oa.single.fbits, scratch, st, perm_out, launches);
}

cudaError_t launch_order_batch(const OrderMap *d_maps, int n_maps, uint64_t total_n, uint32_t nc, uint32_t max_fbits,
                               void *scratch, int num_sms, cudaStream_t st, const uint32_t **perm_out,
                               int *launches)
{
    OrderArgs oa{};
    oa.maps = d_maps;
    oa.n_maps = n_maps;
    oa.total_n = total_n;
    oa.nc = nc;
    oa.grid = order_grid(num_sms, oa.total_n, oa.nc);
    return run_order(oa, max_fbits, scratch, st, perm_out, launches);
}

}  // namespace stk
