// Internal declarations shared by the library's translation units.
//
// Notation follows the paper (Thrane & Coughlin, all-sky seedless clustering):
// a template is a quadratic Bezier curve through control frequencies f0, f1,
// f2 (Sec. III) with a random delay tau (Sec. III, after Eq. 6); its statistic
// is Eq. 7, the sum over its pixels of Re[exp(2 pi i f tau) p(t; f)].
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "../../include/stk.h"

namespace stk {

// ---------------------------------------------------------------- packed map
// Each pixel is stored once, in polar form.  FP32 storage: an 8-byte record
//   .x = bits of |z| (FP32), .y = bits of arg z in radians (FP32, [-pi, pi]),
// where z = y sigma^-2 (weighted statistic) or z = y / sigma (STK_NORM_PAPER);
// the weight array holds w = sigma^-2.  FP16 storage: a 4-byte record, low
// half arg(y) in Q0.16 turns, high half the FP16 value of |y| / sigma (the
// per-frequency or per-pixel scaling); the weight array then holds r = 1/sigma,
// so |z| = (|y|/sigma) r in the weighted form and the weight is r^2.
// Re[e^{i theta} z] = |z| cos(theta + arg z): one cosine per pixel.
enum Prec : int {
    PREC_FP32 = 0,
    PREC_FP16 = 1,
};

enum WMode : int {
    WMODE_CONST = 0,  // every pixel has the same weight (w_const), or paper mode
    WMODE_FREQ = 1,   // weight depends on frequency only: table w[n_f]
    WMODE_PIXEL = 2,  // weight per pixel: plane w[n_t][ldw]
};

struct MapDev {
    int n_t, n_f;
    int prec;         // PREC_FP32 or PREC_FP16
    int ldr;          // records per row: n_f rounded up so rows are 16-byte multiples
    int ldw;          // floats per weight row (WMODE_PIXEL): n_f rounded up to a multiple of 4
    int wmode;
    int paper;        // 1: SNR = S / n_t
    float w_const;    // WMODE_CONST weight (sigma^-2), 1 in paper mode
    double f_min, df; // Hz
    double norm;      // 1 / n_t (paper form) or 1 / sqrt(n_t w_const) (WMODE_CONST); else unused
    float norm_f;     // norm rounded to FP32
    const void *rec;  // [n_t][ldr] records (uint2 for FP32, uint32 for FP16)
    const float *w;   // [n_f] (WMODE_FREQ) or [n_t][ldw] (WMODE_PIXEL), else null: sigma^-2 or 1/sigma
    // Rasteriser: column j of template (f0, f1, f2) sits at bin floor(N_j / d) with
    // N_j = 2 num_j + M^2, num_j = (M-j)^2 f0 + 2 (M-j) j f1 + j^2 f2, d = 2 M^2.
    uint32_t M;       // n_t - 1
    uint64_t d;       // 2 M^2
    uint32_t magic;   // floor(N / d) = umulhi(N, magic) >> shift for all N <= N_max (when fast32)
    int shift;
    int fast32;       // N_max = M^2 (2 n_f - 1) < 2^32 and the magic pair is exact up to N_max
};

struct TrackSet {
    uint64_t n, seed, offset;
    double tau_max;
    const double *tau_q = nullptr;  // delay prior: n_q quantiles (tau at probability i/(n_q-1)); null: uniform
    int n_q = 0;
    int general = 0;                // 1: random start / middle / end times (six random numbers)
    int t_min = 0;                  // general templates: end - start >= t_min columns
};

// ---------------------------------------------------------------- error bits (device flag)
enum : int {
    ERR_TIMEOUT = 1,   // a bounded mbarrier wait gave up
    ERR_BADTRACK = 2,  // explicit template with a control bin >= n_f
    ERR_BADINPUT = 4,  // map packing saw a non-finite y or a bad sigma
    FLAG_SIGMA_VARIES = 8,  // map packing saw more than one sigma value
    ERR_FP16_RANGE = 16,    // |y| / sigma beyond the FP16 range
    ERR_CANCELED = 32,      // a batch kernel saw its cancel flag
    ERR_BOUNDS = 64,        // debug build: a gather outside its template's bins or the map
};

// ---------------------------------------------------------------- debug build checks
// Built with STK_DEBUG_BOUNDS (libstk_debug.so), every pixel gather checks its
// column against [0, n_t) and its bin against [lo, hi]: the convex hull of the
// template's control bins (the Bezier curve lies inside it), within [0, n_f).
// A bin outside is reported (ERR_BOUNDS, read by the next deferred-error check)
// and replaced by lo, so the check can only report, never read out of range or
// trap.  The release build compiles the checks away.
#ifdef STK_DEBUG_BOUNDS
constexpr bool kDebugBounds = true;
#else
constexpr bool kDebugBounds = false;
#endif

__device__ __forceinline__ uint32_t checked_bin(uint32_t b, int j, int n_t, uint32_t lo, uint32_t hi, int *err)
{
    if (kDebugBounds && (b < lo || b > hi || j < 0 || j >= n_t)) {
        atomicOr(err, ERR_BOUNDS);
        return lo;
    }
    return b;
}

__host__ __device__ __forceinline__ uint32_t hull_lo(const uint32_t f[3])
{
    return f[0] < f[1] ? (f[0] < f[2] ? f[0] : f[2]) : (f[1] < f[2] ? f[1] : f[2]);
}

__host__ __device__ __forceinline__ uint32_t hull_hi(const uint32_t f[3])
{
    return f[0] > f[1] ? (f[0] > f[2] ? f[0] : f[2]) : (f[1] > f[2] ? f[1] : f[2]);
}

// ---------------------------------------------------------------- Philox4x64-10
// Counter-based generator of Salmon, Moraes, Dror and Shaw (SC'11): ten
// rounds of two 64x64->128 multiplies by fixed odd multipliers, with the key
// bumped by two Weyl increments between rounds.
__host__ __device__ __forceinline__ void mul64_hilo(uint64_t a, uint64_t b, uint64_t &hi, uint64_t &lo)
{
#ifdef __CUDA_ARCH__
    hi = __umul64hi(a, b);
    lo = a * b;
#else
    unsigned __int128 p = (unsigned __int128)a * b;
    hi = (uint64_t)(p >> 64);
    lo = (uint64_t)p;
#endif
}

__host__ __device__ __forceinline__ void philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                                       uint64_t k0, uint64_t k1, uint64_t out[4])
{
    const uint64_t kMul0 = 0xD2E7470EE14C6C93ULL, kMul1 = 0xCA5A826395121157ULL;
    const uint64_t kWeyl0 = 0x9E3779B97F4A7C15ULL, kWeyl1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint64_t h0, l0, h1, l1;
        mul64_hilo(kMul0, c0, h0, l0);
        mul64_hilo(kMul1, c2, h1, l1);
        const uint64_t n0 = h1 ^ c1 ^ k0, n2 = h0 ^ c3 ^ k1;
        c0 = n0; c1 = l1; c2 = n2; c3 = l0;
        k0 += kWeyl0; k1 += kWeyl1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Template g (Sec. III): counter (g, 0, 0, 0), key (seed, 0).  Control bins
// are floor(u * n_f / 2^64) of words 0..2; the delay is
// tau_max * ((2 (u3 >> 12) + 1) 2^-52 - 1), exact before the one multiply.
__host__ __device__ __forceinline__ void draw_track(uint64_t seed, uint64_t g, uint32_t n_f, double tau_max,
                                                    uint32_t f[3], double &tau)
{
    uint64_t u[4];
    philox4x64_10(g, 0, 0, 0, seed, 0, u);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        uint64_t hi, lo;
        mul64_hilo(u[k], (uint64_t)n_f, hi, lo);
        f[k] = (uint32_t)hi;
    }
    // tau = tau_max ((2 v + 1) 2^-52 - 1), v = u3 >> 12.  The bracket is exactly
    // m 2^-52 with m = 2 v + 1 - 2^52 (|m| < 2^52), so tau = m (tau_max 2^-52) rounds
    // the same real number once: one conversion and one multiply.
    const int64_t m = (int64_t)(2 * (u[3] >> 12) + 1) - (int64_t)(1ull << 52);
    const double scaled = tau_max * 0x1p-52;
    if (scaled >= 0x1p-1000 || scaled == 0.0)
        tau = (double)m * scaled;
    else  // tau_max so small that tau_max 2^-52 would lose bits
        tau = tau_max * ((double)m * 0x1p-52);
}

// Delay from the prior's quantile table: q = (u >> 11) 2^-53 (n_q - 1), then linear
// interpolation between quantiles floor(q) and floor(q) + 1.  Every step is one
// IEEE operation, written out so no compiler fuses two of them.
__host__ __device__ __forceinline__ double tau_from_prior(uint64_t u, const double *tq, int n_q)
{
#ifdef __CUDA_ARCH__
    const double q = __dmul_rn((double)(u >> 11) * 0x1p-53, (double)(n_q - 1));
    int i = (int)floor(q);
    if (i > n_q - 2) i = n_q - 2;
    const double fr = __dsub_rn(q, (double)i);
    return __dadd_rn(tq[i], __dmul_rn(fr, __dsub_rn(tq[i + 1], tq[i])));
#else
    volatile double q = (double)(u >> 11) * 0x1p-53 * (double)(n_q - 1);
    int i = (int)floor(q);
    if (i > n_q - 2) i = n_q - 2;
    volatile double fr = q - (double)i;
    volatile double d = tq[i + 1] - tq[i];
    volatile double p = fr * d;
    return tq[i] + p;
#endif
}

// Template with a delay prior: as draw_track, with tau from the quantile table.
__host__ __device__ __forceinline__ void draw_track_ts(const TrackSet &ts, uint64_t g, uint32_t n_f, uint32_t f[3],
                                                       double &tau)
{
    if (ts.n_q < 2) {
        draw_track(ts.seed, g, n_f, ts.tau_max, f, tau);
        return;
    }
    uint64_t u[4];
    philox4x64_10(g, 0, 0, 0, ts.seed, 0, u);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        uint64_t hi, lo;
        mul64_hilo(u[k], (uint64_t)n_f, hi, lo);
        f[k] = (uint32_t)hi;
    }
    tau = tau_from_prior(u[3], ts.tau_q, ts.n_q);
}

// ---------------------------------------------------------------- general templates
// Sec. III: three time-frequency control points P_k = (t_k, f_k) from six random
// numbers, the curve persisting at least t_min.  Integer times t0 <= t1 <= t2,
// t2 - t0 >= t_min: Philox block (g, 1, 0, 0) gives the duration d = t2 - t0
// uniform on [t_min, n_t - 1], the start uniform on [0, n_t - 1 - d] and t1
// uniform on [t0, t2]; frequencies and delay come from block (g, 0, 0, 0) as for
// the pinned templates.
__host__ __device__ __forceinline__ void draw_times(uint64_t seed, uint64_t g, uint32_t n_t, uint32_t t_min,
                                                    uint32_t t[3])
{
    uint64_t v[4];
    philox4x64_10(g, 1, 0, 0, seed, 0, v);
    const uint64_t M = n_t - 1;
    uint64_t hi, lo;
    mul64_hilo(v[0], M - t_min + 1, hi, lo);
    const uint64_t d = t_min + hi;
    mul64_hilo(v[1], M - d + 1, hi, lo);
    t[0] = (uint32_t)hi;
    t[2] = (uint32_t)(hi + d);
    mul64_hilo(v[2], d + 1, hi, lo);
    t[1] = (uint32_t)(t[0] + hi);
}

// The curve t(xi) = A xi^2 + B xi + t0, f(xi) = F xi^2 + G xi + f0 (integer
// coefficients).  Column j in [t0, t2] sits at the xi_j in [0, 1] with t(xi_j) = j:
// xi_j = 2 (j - t0) / (sqrt(Delta_j) + B), Delta_j = B^2 + 4 A (j - t0) >= 0.  Its
// pixel is the nearest bin to f(xi_j), halves rounded up: the largest b with
// f(xi_j) >= b - 1/2.  With u = 2 (j - t0), s = sqrt(Delta_j), D = s + B and
// E = 2 f0 - 2 b + 1:
//   (2 f(xi_j) - (2b - 1)) D^2 = P + Q s,
//   P = 2 F u^2 + 2 G u B + E (Delta_j + B^2),  Q = 2 G u + 2 E B,
// whose sign is decided exactly in integers (|P| < 2^44, |Q| < 2^30 for
// n_t <= 4096, n_f <= 8192; the squares compared need 128 bits).
struct GenCurve {
    int32_t t0, t2, A, B, F, G, f0;
};

__host__ __device__ __forceinline__ GenCurve gen_curve(const uint32_t t[3], const uint32_t f[3])
{
    GenCurve c;
    c.t0 = (int32_t)t[0];
    c.t2 = (int32_t)t[2];
    c.A = (int32_t)t[0] - 2 * (int32_t)t[1] + (int32_t)t[2];
    c.B = 2 * ((int32_t)t[1] - (int32_t)t[0]);
    c.F = (int32_t)f[0] - 2 * (int32_t)f[1] + (int32_t)f[2];
    c.G = 2 * ((int32_t)f[1] - (int32_t)f[0]);
    c.f0 = (int32_t)f[0];
    return c;
}

// x^2 (x < 2^63 in magnitude) and x * y (x, y >= 0) as 128-bit (hi, lo).
__host__ __device__ __forceinline__ void umul128(uint64_t x, uint64_t y, uint64_t &hi, uint64_t &lo)
{
    mul64_hilo(x, y, hi, lo);
}

// f(xi_j) >= b - 1/2 ?  (j in (t0, t2])
__host__ __device__ __forceinline__ bool gen_ge(const GenCurve &c, int64_t j, int64_t b)
{
    const int64_t du = j - c.t0;
    const int64_t u = 2 * du;
    const int64_t B = c.B;
    const int64_t Dl = B * B + 4 * (int64_t)c.A * du;
    const int64_t E = 2 * (int64_t)c.f0 - 2 * b + 1;
    const int64_t P = 2 * (int64_t)c.F * u * u + 2 * (int64_t)c.G * u * B + E * (Dl + B * B);
    const int64_t Q = 2 * (int64_t)c.G * u + 2 * E * B;
    if (P >= 0 && Q >= 0) return true;
    if (P <= 0 && Q <= 0) return P == 0 && Q == 0;
    const uint64_t aP = (uint64_t)(P < 0 ? -P : P), aQ = (uint64_t)(Q < 0 ? -Q : Q);
    uint64_t ph, pl, rh, rl;
    umul128(aP, aP, ph, pl);                       // P^2
    umul128(aQ * aQ, (uint64_t)Dl, rh, rl);        // Q^2 Delta  (Q^2 < 2^60)
    const bool p_ge = ph > rh || (ph == rh && pl >= rl);
    const bool r_ge = rh > ph || (rh == ph && rl >= pl);
    return P > 0 ? p_ge : r_ge;                    // P > 0 > Q: P >= |Q| s;  Q > 0 > P: Q s >= |P|
}

// Pixel of column j given the previous column's pixel (bins move a few per column).
__host__ __device__ __forceinline__ int32_t gen_step(const GenCurve &c, int64_t j, int32_t prev, int32_t n_f)
{
    int32_t b = prev;
    while (b + 1 < n_f && gen_ge(c, j, b + 1)) ++b;
    while (b > 0 && !gen_ge(c, j, b)) --b;
    return b;
}

// Filtered pixel: an FP32 estimate of f(xi_j) decides the bin when it lies
// farther than `margin` from a rounding boundary; otherwise the exact test does.
// Error of the estimate (IEEE sqrt and divide, FMA evaluation): Delta_j < 2^27 is
// rounded once (2^-24), s = sqrt once more, D = s + B and xi = u / D each add one
// rounding, so |d xi| <= 4 2^-24 xi <= 4 2^-24.  f' = G + 2 F xi is linear, so on [0, 1]
// |f'| <= Gmax = max(|G|, |G + 2F|); f is a convex combination of the control bins, so
// f and xi (G + F xi) = f - f0 lie in [-fmax, fmax], fmax = max(f0, f1, f2).  The inner
// FMA (G + F xi) and the outer one (f0 + xi inner) each round once, f + 1/2 once more:
// the estimate of f + 1/2 errs by at most 2^-24 (4.01 (Gmax + 1) + 3.01 (fmax + 1) + 1)
// < 2.4e-7 (Gmax + 1) + 1.8e-7 (fmax + 1) + 6e-8.  The margin takes twice that.
struct GenFilter {
    float F, G, f0, B, margin;
};

__host__ __device__ __forceinline__ GenFilter gen_filter(const GenCurve &c)
{
    GenFilter g;
    g.F = (float)c.F;
    g.G = (float)c.G;
    g.f0 = (float)c.f0;
    g.B = (float)c.B;
    const int32_t f1 = c.f0 + c.G / 2, f2 = c.f0 + c.G + c.F;  // G = 2 (f1 - f0), F = f0 - 2 f1 + f2
    const int32_t aG = c.G < 0 ? -c.G : c.G, aG2 = c.G + 2 * c.F < 0 ? -(c.G + 2 * c.F) : c.G + 2 * c.F;
    const float gmax = (float)(aG > aG2 ? aG : aG2);
    const int32_t f12 = f1 > f2 ? f1 : f2;
    const float fmax = (float)(c.f0 > f12 ? c.f0 : f12);
    g.margin = 2.f * (2.4e-7f * (gmax + 1.f) + 1.8e-7f * (fmax + 1.f) + 6e-8f) + 1e-6f;
    return g;
}

// The filter alone: the estimated bin in b, and whether it is certain (else the
// exact test must decide, starting from b).
__device__ __forceinline__ bool gen_estimate(const GenCurve &c, const GenFilter &g, int64_t j, int32_t n_f,
                                             int32_t &b)
{
    const int32_t du = (int32_t)(j - c.t0);
    const int32_t Dl = c.B * c.B + 4 * c.A * du;   // exact, < 2^27
    const float s = __fsqrt_rn((float)Dl);
    const float xi = __fdiv_rn((float)(2 * du), __fadd_rn(s, g.B));
    const float fx = fmaf(xi, fmaf(g.F, xi, g.G), g.f0);
    const float h = fx + 0.5f;
    const float k = floorf(h);
    const float d = h - k;
    b = (int32_t)k;
    b = b < 0 ? 0 : (b > n_f - 1 ? n_f - 1 : b);
    return d > g.margin && d < 1.f - g.margin;
}

__device__ __forceinline__ int32_t gen_pixel(const GenCurve &c, const GenFilter &g, int64_t j, int32_t n_f)
{
    int32_t b;
    if (gen_estimate(c, g, j, n_f, b)) return b;
    return gen_step(c, j, b, n_f);                 // near a boundary: exact
}

// ---------------------------------------------------------------- phase in turns
// theta_j / 2 pi = (f_min + bin_j df) tau = B + bin_j A  (mod 1), with A =
// frac(df tau) and B = frac(f_min tau) exact 64-bit fractions (Q0.64).  A pixel
// needs its turn as Q0.32.  Two forms, both turn = bin a + hi32(bin a_lo) + c + arg
// (mod 2^32):
//   narrow maps (n_f <= kPhaseNarrowNf): a = A rounded to 32 bits, a_lo = 0 and c
//     chosen so the turn is exact at the centre bin n_f / 2; the error is at most
//     |bin - n_f/2| 2^-33 + 2^-33 turn (<= 4.8e-7 turn = 3.0e-6 rad at n_f = 8192);
//   wider maps: a:a_lo = A (64 bits), c = B rounded; error below 2^-32 turn.
// The slab and batched kernels take the narrow form without the hi32 term.
constexpr int kPhaseNarrowNf = 8192;

struct Phase {
    uint32_t a, c, a_lo;
};

// frac(x * y) * 2^64 (unsigned, value - floor(value)), from the exact product of
// two doubles in integer arithmetic: x = mx 2^ex, y = my 2^ey, x y = P 2^e with
// P = mx my < 2^106.  Truncated to 2^-64 (negative products: within 2^-64).
__host__ __device__ __forceinline__ uint64_t frac_prod_q64(double x, double y)
{
#ifdef __CUDA_ARCH__
    const uint64_t bx = (uint64_t)__double_as_longlong(x), by = (uint64_t)__double_as_longlong(y);
#else
    uint64_t bx, by;
    memcpy(&bx, &x, 8);
    memcpy(&by, &y, 8);
#endif
    const int fx = (int)((bx >> 52) & 0x7ff), fy = (int)((by >> 52) & 0x7ff);
    uint64_t mx = bx & 0xFFFFFFFFFFFFFull, my = by & 0xFFFFFFFFFFFFFull;
    if (fx) mx |= 1ull << 52;
    if (fy) my |= 1ull << 52;
    if (mx == 0 || my == 0) return 0;
    const int e = (fx ? fx : 1) - 1075 + (fy ? fy : 1) - 1075;
    if (e >= 0) return 0;                       // an integer
    uint64_t hi, lo;
    mul64_hilo(mx, my, hi, lo);
    const int s = -e;                           // value = P / 2^s
    uint64_t q;
    if (s < 64) q = lo << (64 - s);
    else if (s == 64) q = lo;
    else if (s < 128) q = (lo >> (s - 64)) | (hi << (128 - s));
    else if (s < 192) q = hi >> (s - 128);
    else q = 0;
    if (((bx ^ by) >> 63) && q) q = 0 - q;      // frac(-v) = 1 - frac(v)
    return q;
}

__host__ __device__ __forceinline__ Phase phase_consts(double f_min, double df, double tau, int n_f)
{
    Phase p;
    const uint64_t A = frac_prod_q64(df, tau);
    const uint64_t B = frac_prod_q64(f_min, tau);
    if (n_f <= kPhaseNarrowNf) {
        const uint32_t bc = (uint32_t)(n_f / 2);
        p.a = (uint32_t)((A + 0x80000000ull) >> 32);                       // mod 2^32: A near 1 wraps to 0
        const uint32_t t_c = (uint32_t)(((uint64_t)bc * A + B + 0x80000000ull) >> 32);  // exact turn at bc
        p.c = t_c - bc * p.a;
        p.a_lo = 0u;
    } else {
        p.a = (uint32_t)(A >> 32);
        p.a_lo = (uint32_t)A;
        p.c = (uint32_t)((B + 0x80000000ull) >> 32);
    }
    return p;
}

// The template's phase at a bin, T = frac((f_min + bin df) tau) as Q0.32 turns
// (read as signed: [-1/2, 1/2)).  A pixel's angle is then 2 pi T + arg z, with
// the integer-to-float conversion of T rounding to 24 significant bits (at most
// 2^-26 turn) and 2 pi / 2^32 rounded to FP32 (2^-24 relative).
constexpr float kTurnToRad = 1.46291807926715968e-9f;  // 2 pi / 2^32

__device__ __forceinline__ uint32_t template_turn(uint32_t bin, const Phase &p)
{
    return bin * p.a + __umulhi(bin, p.a_lo) + p.c;
}

// The narrow form (a_lo = 0): slab and batched kernels, n_f <= kPhaseNarrowNf.
__device__ __forceinline__ uint32_t template_turn_narrow(uint32_t bin, uint32_t a, uint32_t c)
{
    return bin * a + c;
}

// ---------------------------------------------------------------- rasteriser state
// Second-order forward differences of N_j (exact modulo 2^32; every N_j lies in
// [0, N_max] < 2^32 when fast32 holds):
//   N_0 = (2 f0 + 1) M^2,  D_0 = 4 M (f1 - f0) + 2 (f0 - 2 f1 + f2),  D2 = 4 (f0 - 2 f1 + f2).
struct Raster32 {
    uint32_t N, D, D2;
};

__device__ __forceinline__ Raster32 raster_init(uint32_t f0, uint32_t f1, uint32_t f2, uint32_t M)
{
    const int64_t M2 = (int64_t)M * M;
    const int64_t c2 = (int64_t)f0 - 2 * (int64_t)f1 + (int64_t)f2;
    Raster32 r;
    r.N = (uint32_t)((2 * (int64_t)f0 + 1) * M2);
    r.D = (uint32_t)(4 * (int64_t)M * ((int64_t)f1 - (int64_t)f0) + 2 * c2);
    r.D2 = (uint32_t)(4 * c2);
    return r;
}

// Wide form for maps where N_max does not fit 32 bits: num_j directly in 64-bit.
__device__ __forceinline__ uint32_t raster_bin_wide(uint32_t f0, uint32_t f1, uint32_t f2, uint32_t M, uint32_t j,
                                                    uint64_t d)
{
    const uint64_t a = (uint64_t)(M - j), b = (uint64_t)j, M2 = (uint64_t)M * M;
    const uint64_t num = a * a * f0 + 2 * a * b * f1 + b * b * f2;
    return (uint32_t)((2 * num + M2) / d);
}

// ---------------------------------------------------------------- mbarrier + bulk copy
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Loads from shared memory at a 32-bit shared-window address.
__device__ __forceinline__ uint2 lds_u64(uint32_t a)
{
    uint2 v;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a));
    return v;
}

__device__ __forceinline__ uint32_t lds_u32(uint32_t a)
{
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}

__device__ __forceinline__ float lds_f32(uint32_t a)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Order this thread's earlier shared-memory accesses (generic proxy) before
// later bulk copies into shared memory (async proxy).
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One-dimensional bulk copy global -> shared, completing `bytes` on `bar`.
// dst, src and bytes must be multiples of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase with the given parity to complete; gives up after
// `limit_ns` nanoseconds and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns)
{
    const uint32_t a = smem_u32(bar);
    uint32_t done = 0;
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                 : "=r"(done)
                 : "r"(a), "r"(parity)
                 : "memory");
    if (done) return true;
    const uint64_t t0 = global_ns();
    while (true) {
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                     : "=r"(done)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (done) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// ---------------------------------------------------------------- host-side launchers
struct ScorePlan {
    int kernel;       // 1 simple, 2 staged, 3 general templates
    int R;            // templates per thread (staged)
    int threads;      // threads per block
    int grid;
    int S;            // rows per slab (staged)
    int nstage;       // slab buffers (staged)
    int nslabs;
    uint64_t batch;   // templates per batch (staged)
    uint64_t nbatches;
    size_t smem;
    int order;           // 1: templates scored in coherent (Z-order) order, 0: index order
    int order_launches;  // launches of the ordering pre-pass
};

struct Tuning {
    int kernel = 0;      // 0 auto
    int threads = 0;     // 0 auto
    int max_R = 12;      // capped per weight mode by the launcher
    int nstage = 2;
    int smem_kb = 0;     // 0 auto
    int wait_ms = 0;     // slab wait limit, 0: 2000 ms
    int withhold_slab = -1;  // test of the bounded waits: CTA 0 withholds this slab copy (-1: off)
    int order = 1;       // slab kernel: score templates in coherent order (1) or index order (0)
    int select_sample = 0;  // selection: keys sampled for the threshold (0: default)
};

// Launch the scoring kernel for generated templates; writes n FP32 SNRs to out.
// order_scratch (order_scratch_bytes(n, n_f) bytes, or NULL for index order)
// holds the coherent-order pre-pass of the slab kernel; order_done, if given,
// is recorded between that pre-pass and the scoring kernel.
cudaError_t launch_score_generated(const MapDev &m, const TrackSet &ts, float *out, int *err, const Tuning &tu,
                                   int num_sms, size_t smem_optin, cudaStream_t st, ScorePlan *plan_out,
                                   void *order_scratch = nullptr, cudaEvent_t order_done = nullptr);
// Whether launch_score_generated would use order scratch for this call.
bool score_wants_order(const MapDev &m, const TrackSet &ts, const Tuning &tu);

// Coherent-order pre-pass (stk_order.cu).  One map: the key is 7 bits per
// control bin (general templates: 6 bits each of the start and end column, 3 of
// each bin); *perm_out = the scoring order inside scratch (perm[p] =
// template index relative to the range's offset).
size_t order_scratch_bytes(uint64_t n, int n_f, int n_t, bool general, int num_sms);
cudaError_t launch_order(const MapDev &m, const TrackSet &ts, void *scratch, int num_sms, cudaStream_t st,
                         const uint32_t **perm_out, int *launches);
// Many maps: map i's templates take positions pos0 .. pos0 + n - 1 of perm
// (values relative to its offset) and coarse buckets from coarse0.
struct OrderMap {
    TrackSet ts;       // with ts.general: key = (t0, t2, Z-order of the bins), tbits + tbits + 9 bits
    uint32_t n_f;
    uint32_t n_t;
    int shift;         // control bins >> shift form the key
    int bbits;         // bits of each key coordinate (pinned templates)
    int tshift;        // general templates: control times >> tshift (tbits bits each)
    int tbits;
    int fbits;         // key bits below the coarse bucket
    uint32_t coarse0;  // first coarse bucket
    uint32_t pos0;     // first position
};
void order_shape(int n_f, int max_bits, int &shift, int &bits);
// Fill shift, tshift, fbits and coarse0 of maps (ts, n_f, n_t, pos0 given); nc = coarse buckets in all.
void order_plan_maps(OrderMap *maps, int n_maps, uint32_t &nc, uint32_t &max_fbits);
size_t order_scratch_bytes_maps(uint64_t total_n, uint32_t nc, int num_sms);
cudaError_t order_prepare(uint32_t nc, uint32_t max_fbits);
// Fills the order's Hilbert key table on the current device (every context, before
// its first order pass; the values never change).
cudaError_t order_build_tables(cudaStream_t st);
cudaError_t launch_order_batch(const OrderMap *d_maps, int n_maps, uint64_t total_n, uint32_t nc, uint32_t max_fbits,
                               void *scratch, int num_sms, cudaStream_t st, const uint32_t **perm_out,
                               int *launches);
// Explicit templates f3[n][3], tau[n] (FP32 SNRs to out).
cudaError_t launch_score_explicit(const MapDev &m, const uint32_t *f3, const double *tau, uint64_t n, float *out,
                                  int *err, cudaStream_t st);
// Explicit general templates: t3[n][3] control times, f3[n][3] control bins.
cudaError_t launch_score_explicit_general(const MapDev &m, const uint32_t *t3, const uint32_t *f3, const double *tau,
                                          uint64_t n, float *out, int *err, cudaStream_t st);
// Parameters (f_dev: 3 bins then 3 times), delay and bins of one template (device buffers).
cudaError_t launch_track_params(const MapDev &m, const TrackSet &ts, uint64_t g, uint32_t *f_dev, double *tau_dev,
                                int32_t *bins_dev, cudaStream_t st);

// out[i] = (double)in[i], i < n.
cudaError_t launch_widen(const float *in, double *out, uint64_t n, cudaStream_t st);

// Interpolated statistic of continuous templates (forward: snr; adjoint: g * gradient).
cudaError_t launch_interp(const MapDev &m, const float *f3, const float *tau, const float *g, uint64_t n, float *snr,
                          float *gf3, float *gtau, bool adjoint, int *err, cudaStream_t st);

// Top-k selection over the FP32 snr[0..n): hits get (snr widened to FP64, offset + i, params).  Scratch
// is caller-provided: see select_scratch_bytes.  sample: keys sampled for the candidate
// threshold (0: the default, 16384; at most 49152); the result does not depend on it.
size_t select_scratch_bytes(uint64_t n, int k);
uint32_t select_sample_size(uint64_t n, uint32_t sample);
cudaError_t launch_select_topk(const float *snr, uint64_t n, int k, const TrackSet &ts, const MapDev &m,
                               void *scratch, stk_hit *out_dev, cudaStream_t st, int *launches,
                               uint32_t sample = 0);

}  // namespace stk
