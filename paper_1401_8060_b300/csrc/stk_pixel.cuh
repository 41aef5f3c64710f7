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
struct Pix<PREC_FP32> {  // {float |z|, Q0.32 arg z}; the weight array holds w = sigma^-2
    using Rec = uint2;
    __device__ static __forceinline__ float mag(Rec v) { return __uint_as_float(v.x); }
    __device__ static __forceinline__ uint32_t arg(Rec v) { return v.y; }
    __device__ static __forceinline__ Rec load_global(const void *p, size_t i) { return __ldg((const uint2 *)p + i); }
};

template <>
struct Pix<PREC_FP16> {  // low half: FP16 |y|/sigma; high half: arg in Q0.16 turns; weights hold r = 1/sigma
    using Rec = uint32_t;
    __device__ static __forceinline__ float mag(Rec v)
    {
        return __half2float(__ushort_as_half((unsigned short)(v & 0xffffu)));
    }
    __device__ static __forceinline__ uint32_t arg(Rec v) { return v & 0xffff0000u; }
    __device__ static __forceinline__ Rec load_global(const void *p, size_t i)
    {
        return __ldg((const unsigned int *)p + i);
    }
};

// One pixel of Eq. 7: acc += |z| cos(theta + 2 pi arg z), W += weight.
// FP32 records carry |z| and wv = sigma^-2; FP16 records carry |y|/sigma and
// wv = 1/sigma, so |z| = mag wv and the weight is wv^2.
template <int PREC, int WMODE>
__device__ __forceinline__ void accumulate_turn(typename Pix<PREC>::Rec v, uint32_t turn, float wv, float &acc,
                                                float &W)
{
    const float c = cos_turn(turn);
    float mg = Pix<PREC>::mag(v);
    if (PREC == PREC_FP16 && WMODE != WMODE_CONST) mg *= wv;
    acc = fmaf(mg, c, acc);
    if (WMODE != WMODE_CONST) W = (PREC == PREC_FP16) ? fmaf(wv, wv, W) : W + wv;
}

// Packed pairs of FP32 operations (Blackwell .f32x2): each lane rounds to
// nearest exactly as the scalar operation does, two results per instruction.
__device__ __forceinline__ void fma2(float &d0, float &d1, float a0, float a1, float b0, float b1)
{
    asm("{ .reg .b64 ra, rb, rc; mov.b64 ra, {%2, %3}; mov.b64 rb, {%4, %5}; mov.b64 rc, {%0, %1};"
        " fma.rn.f32x2 rc, ra, rb, rc; mov.b64 {%0, %1}, rc; }"
        : "+f"(d0), "+f"(d1)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}

__device__ __forceinline__ void add2(float &d0, float &d1, float a0, float a1)
{
    asm("{ .reg .b64 ra, rc; mov.b64 ra, {%2, %3}; mov.b64 rc, {%0, %1};"
        " add.rn.f32x2 rc, rc, ra; mov.b64 {%0, %1}, rc; }"
        : "+f"(d0), "+f"(d1)
        : "f"(a0), "f"(a1));
}

__device__ __forceinline__ void mul2(float &d0, float &d1, float a0, float a1)
{
    asm("{ .reg .b64 ra, rc; mov.b64 ra, {%2, %3}; mov.b64 rc, {%0, %1};"
        " mul.rn.f32x2 rc, rc, ra; mov.b64 {%0, %1}, rc; }"
        : "+f"(d0), "+f"(d1)
        : "f"(a0), "f"(a1));
}

// accumulate_turn for two templates' pixels at once, bit for bit the same.
template <int PREC, int WMODE>
__device__ __forceinline__ void accumulate_turn2(typename Pix<PREC>::Rec v0, typename Pix<PREC>::Rec v1,
                                                 uint32_t t0, uint32_t t1, float w0, float w1, float &acc0,
                                                 float &acc1, float &W0, float &W1)
{
    float x0 = (float)(int32_t)t0, x1 = (float)(int32_t)t1;
    mul2(x0, x1, kTurnToRad, kTurnToRad);
    const float c0 = __cosf(x0), c1 = __cosf(x1);
    float m0 = Pix<PREC>::mag(v0), m1 = Pix<PREC>::mag(v1);
    if (PREC == PREC_FP16 && WMODE != WMODE_CONST) mul2(m0, m1, w0, w1);
    fma2(acc0, acc1, m0, m1, c0, c1);
    if (WMODE != WMODE_CONST) {
        if (PREC == PREC_FP16) fma2(W0, W1, w0, w1, w0, w1);
        else add2(W0, W1, w0, w1);
    }
}

template <int PREC, int WMODE>
__device__ __forceinline__ void accumulate(typename Pix<PREC>::Rec v, uint32_t bin, const Phase &ph, float wv,
                                           float &acc, float &W)
{
    accumulate_turn<PREC, WMODE>(v, pixel_turn(bin, ph, Pix<PREC>::arg(v)), wv, acc, W);
}

// Normalisation (Eq. 7 with the weighting of the footnote to Eq. 5) in FP32.
// Weighted form with varying weights: S / sqrt(W), the square root and the
// division each rounded to nearest, so the result is within 2^-23 (1.2e-7)
// relative of S / sqrt(W) for the FP32 sums S and W.  Constant weight or paper
// form: S times the constant rounded to FP32 (within 2^-23 relative).  No FP64
// arithmetic: this GPU issues FP64 operations at a small fraction of the FP32
// rate, and a per-template FP64 normalisation cost 4.5 % of the scoring kernel.
template <int WMODE>
__device__ __forceinline__ float finalize_snr(float acc, float W, const MapDev &m)
{
    if (WMODE == WMODE_CONST || m.paper) return acc * m.norm_f;
    return __fdiv_rn(acc, __fsqrt_rn(W));
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
