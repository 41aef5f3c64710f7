// Per-pixel and per-template device code shared by the scoring kernels
// (single map and batched): pixel record decoding, the Eq. 7 accumulation,
// the normalisation, and the order used for selection.
#pragma once

#include <cuda_fp16.h>

#include "stk_internal.cuh"

namespace stk {

// ------------------------------------------------------------------ pixel records
template <int PREC>
struct Pix;

template <>
struct Pix<PREC_FP32> {  // {FP32 |z|, FP32 arg z in radians}; the weight array holds w = sigma^-2
    using Rec = uint2;
    __device__ static __forceinline__ float mag(Rec v) { return __uint_as_float(v.x); }
    __device__ static __forceinline__ float arg_rad(Rec v) { return __uint_as_float(v.y); }
    __device__ static __forceinline__ Rec load_global(const void *p, size_t i) { return __ldg((const uint2 *)p + i); }
    __device__ static __forceinline__ Rec load_shared(uint32_t a) { return lds_u64(a); }
    static constexpr int kLog2Bytes = 3;
};

template <>
struct Pix<PREC_FP16> {  // low half: arg in Q0.16 turns; high half: FP16 |y|/sigma; weights hold r = 1/sigma
    using Rec = uint32_t;
    __device__ static __forceinline__ float mag(Rec v)
    {
        __half2 h;
        memcpy(&h, &v, sizeof h);
        return __high2float(h);
    }
    __device__ static __forceinline__ float arg_rad(Rec v) { return (float)(int32_t)(v << 16) * kTurnToRad; }
    __device__ static __forceinline__ Rec load_global(const void *p, size_t i)
    {
        return __ldg((const unsigned int *)p + i);
    }
    __device__ static __forceinline__ Rec load_shared(uint32_t a) { return lds_u32(a); }
    static constexpr int kLog2Bytes = 2;
};

// One pixel of Eq. 7 given the template's phase turn T at the pixel's bin:
// acc += |z| cos(2 pi T + arg z), W += weight.  FP32 records: the angle is one
// fused multiply-add of the converted turn and the stored FP32 angle (|angle| <
// 2 pi), |z| and w = sigma^-2 as stored.  FP16 records: the Q0.16 angle joins
// the turn in integer arithmetic (exact mod 1 turn); the record holds |y|/sigma
// and wv = 1/sigma, so |z| = mag wv and the weight is wv^2.
// pixel_term forms the pixel's factors (|z|, cosine), pixel_sum adds them and the
// weight; pixel_add is the two in a row.
template <int PREC, int WMODE>
__device__ __forceinline__ void pixel_term(typename Pix<PREC>::Rec v, uint32_t T, float wv, float &mg, float &c)
{
    if constexpr (PREC == PREC_FP32) {
        c = __cosf(fmaf((float)(int32_t)T, kTurnToRad, Pix<PREC_FP32>::arg_rad(v)));
        mg = Pix<PREC_FP32>::mag(v);
    } else {
        const uint32_t t = T + ((uint32_t)v << 16);
        c = __cosf((float)(int32_t)t * kTurnToRad);
        mg = Pix<PREC_FP16>::mag(v);
        if (WMODE != WMODE_CONST) mg *= wv;
    }
}

template <int PREC, int WMODE>
__device__ __forceinline__ void pixel_sum(float mg, float c, float wv, float &acc, float &W)
{
    acc = fmaf(mg, c, acc);
    if (WMODE != WMODE_CONST) W = PREC == PREC_FP32 ? W + wv : fmaf(wv, wv, W);
}

template <int PREC, int WMODE>
__device__ __forceinline__ void pixel_add(typename Pix<PREC>::Rec v, uint32_t T, float wv, float &acc, float &W)
{
    float mg, c;
    pixel_term<PREC, WMODE>(v, T, wv, mg, c);
    pixel_sum<PREC, WMODE>(mg, c, wv, acc, W);
}

// The same pixel for a template phase given in full (64-bit increment for wide maps).
template <int PREC, int WMODE>
__device__ __forceinline__ void accumulate(typename Pix<PREC>::Rec v, uint32_t bin, const Phase &ph, float wv,
                                           float &acc, float &W)
{
    pixel_add<PREC, WMODE>(v, template_turn(bin, ph), wv, acc, W);
}

// Normalisation (Eq. 7 with the weighting of the footnote to Eq. 5) in FP32.
// Weighted form with varying weights: S / sqrt(W), the square root and the
// division each rounded to nearest, so the result is within 2^-23 (1.2e-7)
// relative of S / sqrt(W) for the FP32 sums S and W.  Constant weight or paper
// form: S times the constant rounded to FP32 (within 2^-23 relative).  No FP64
// arithmetic: this GPU issues FP64 operations at a small fraction of the FP32
// rate, and a per-template FP64 normalisation cost 4.5 % of the scoring kernel.
// A template whose pixels are all notched (sigma = +inf: W = 0) has no data and scores 0.
template <int WMODE>
__device__ __forceinline__ float finalize_snr(float acc, float W, const MapDev &m)
{
    if (WMODE == WMODE_CONST || m.paper) return acc * m.norm_f;
    return W > 0.f ? __fdiv_rn(acc, __fsqrt_rn(W)) : 0.f;
}

// ------------------------------------------------------------------ selection order
// Order-preserving key of an FP32 SNR in the upper 32 bits of a 64-bit key
// (-0 and +0 share one key; the lower 32 bits are zero).
__device__ __forceinline__ unsigned long long order_key(float x)
{
    uint32_t b = __float_as_uint(x);
    if ((b << 1) == 0u) b = 0u;
    const uint32_t k = (b >> 31) ? ~b : (b | 0x80000000u);
    return (unsigned long long)k << 32;
}

// The SNR back from its key.
__device__ __forceinline__ float snr_from_key(unsigned long long key)
{
    const uint32_t k = (uint32_t)(key >> 32);
    return __uint_as_float((k >> 31) ? (k & 0x7fffffffu) : ~k);
}

// "a before b": larger key, then smaller index.
__device__ __forceinline__ bool before(unsigned long long ka, unsigned int ia, unsigned long long kb, unsigned int ib)
{
    return ka > kb || (ka == kb && ia < ib);
}

// floor(N / d) for N < 2^32 from magic = ceil(2^(32+shift) / d) < 2^32: the
// multiply-shift estimate is floor(N / d) or one more, and one compare fixes it.
__device__ __forceinline__ uint32_t div_corrected(uint32_t N, uint32_t magic, int shift, uint32_t d)
{
    uint32_t q = __umulhi(N, magic) >> shift;
    q -= (q * d > N) ? 1u : 0u;
    return q;
}

}  // namespace stk
