// Continuous templates for refining loud templates by gradient ascent (the
// follow-up of the loudest events, Sec. V).
//
// A template's control frequencies f0, f1, f2 become real numbers (bins) and its
// delay tau stays continuous.  Column j of the curve sits at
//   x_j = ((M-j)^2 f0 + 2 (M-j) j f1 + j^2 f2) / M^2   (bins, clamped to [0, n_f - 1]);
// the map is interpolated linearly in frequency between bins k = floor(x_j) and
// k + 1, and the phase uses the continuous frequency f_min + x_j df:
//   S = sum_j Re[exp(2 pi i (f_min + x_j df) tau) z(j, x_j)],  W = sum_j w(j, x_j),
//   SNR = S / sqrt(W) (weighted) or S / N (paper form) -- Eq. 7 at integer bins.
// The forward kernel returns SNR; the adjoint kernel returns g * dSNR/d(f0, f1,
// f2, tau) for an upstream gradient g, differentiating each of those steps.
// One block of 128 threads per template: thread l takes the columns j = l (mod
// 128) in order; the lanes' partial sums meet in a fixed shuffle tree and the
// four warps' sums are added in warp order (deterministic).  Sums and
// the pixel arithmetic are FP32; the curve position x_j and the phase argument are
// FP64, since FP32 resolves x_j ~ 10^3 only to 6e-5 bins.  FP64 is a slow pipe on
// this GPU, so x_j advances by forward differences and only the position, its
// split into bin and fraction, and the phase's turns use it.
#include <cuda_fp16.h>

#include <cmath>

#include "stk_internal.cuh"
#include "stk_pixel.cuh"
#include "stk_refine.cuh"

namespace stk {

namespace {

// Cartesian pixel value and weight at (column j, bin k) from the packed map.
// FP32 records: z = |z| e^{2 pi i arg}, weight w.  FP16 records: |z| = h r with
// r = 1/sigma (weight r^2), or h alone when the weight is constant.
template <int WMODE, int PREC>
__device__ __forceinline__ void pixel_at(const MapDev &m, int j, int k, float &zr, float &zi, float &w, int *err)
{
    if (kDebugBounds) k = (int)checked_bin((uint32_t)k, j, m.n_t, 0u, (uint32_t)m.n_f - 1u, err);
    const typename Pix<PREC>::Rec v = Pix<PREC>::load_global(m.rec, (size_t)j * m.ldr + k);
    float mag = Pix<PREC>::mag(v);
    float wv = 0.f;
    if (WMODE == WMODE_FREQ) wv = __ldg(m.w + k);
    if (WMODE == WMODE_PIXEL) wv = __ldg(m.w + (size_t)j * m.ldw + k);
    if (PREC == PREC_FP16 && WMODE != WMODE_CONST) {
        mag *= wv;
        wv *= wv;
    }
    const float ang = Pix<PREC>::arg_rad(v);
    float s, c;
    __sincosf(ang, &s, &c);
    zr = mag * c;
    zi = mag * s;
    w = wv;
}

constexpr int kInterpBlock = 128;

// Per-launch constants of the curve and the map (host-computed, so no thread
// repeats the FP64 divisions).
struct InterpConst {
    double M, inv_M2, df, f_min;
    float inv_Mf, df_f, fmin_f;
    int *err;  // deferred error flags (debug build: out-of-range gathers)
};

// Fused Adam step (refinement): the template's thread 0 takes the step from the
// gradient it has just summed.  mom == nullptr: no step.
struct AdamStep {
    float *u;          // tau / tau_max, the ascent's delay coordinate
    float4 *mom;       // first and second moments of (f0, f1, f2, u), two float4 a template
    float step_f, step_u, sbc2, tau_max, f_hi;
};

// One Adam step of the gradient ascent of a template's SNR (Adam with betas 0.9,
// 0.999 and eps 1e-8 on the loss -SNR, in torch's arithmetic order), then the
// projection onto f in [0, n_f - 1] and |u| <= 1.  step_f = lr_f / (1 - 0.9^t),
// step_u likewise, sbc2 = sqrt(1 - 0.999^t), from the host.
__device__ __forceinline__ void adam_update(const AdamStep &ad, uint64_t i, float *f3, float *tau, const float gs[4])
{
    const float w1 = 0.1f, b2 = 0.999f, w2 = 0.001f, eps = 1e-8f;
    float4 m = ad.mom[2 * i], v = ad.mom[2 * i + 1];
    float p[4] = {f3[3 * i], f3[3 * i + 1], f3[3 * i + 2], ad.u[i]};
    float *mm = &m.x, *vv = &v.x;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float g = -gs[q];                                   // d(-SNR)/d(f, u)
        mm[q] = mm[q] + w1 * (g - mm[q]);
        vv[q] = vv[q] * b2 + w2 * g * g;
        const float denom = __fsqrt_rn(vv[q]) / ad.sbc2 + eps;
        p[q] = p[q] - (q < 3 ? ad.step_f : ad.step_u) * (mm[q] / denom);
    }
    ad.mom[2 * i] = m;
    ad.mom[2 * i + 1] = v;
#pragma unroll
    for (int q = 0; q < 3; ++q) f3[3 * i + q] = fminf(fmaxf(p[q], 0.f), ad.f_hi);
    const float uu = fminf(fmaxf(p[3], -1.f), 1.f);
    ad.u[i] = uu;
    tau[i] = uu * ad.tau_max;
}

// P threads per template (32, 64 or 128), kInterpBlock / P templates a block.
// MODE 0: forward (snr); 1: adjoint (g * gradient to gf3, gtau; snr too when
// snr_out is given); 2: adjoint with g = 1 and the fused Adam step, parameters
// updated in place (each template's parameters are read by its own threads
// before the reduction and written by its thread 0 after it).
template <int WMODE, int PREC, int MODE, int P>
__global__ void __launch_bounds__(kInterpBlock) interp_kernel(MapDev m, InterpConst k, const float *f3,
                                                              const float *tau_in, const float *__restrict__ g,
                                                              uint64_t n, float *__restrict__ snr_out,
                                                              float *__restrict__ gf3, float *__restrict__ gtau,
                                                              AdamStep ad)
{
    constexpr bool ADJOINT = MODE != 0;
    constexpr int TPB = kInterpBlock / P;  // templates a block
    constexpr int WPT = P / 32;            // warps a template
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int t = tid % P;                  // thread within the template
    const uint64_t i_raw = (uint64_t)blockIdx.x * TPB + tid / P;
    const bool valid = i_raw < n;           // no early return: the block meets at a barrier below
    const uint64_t i = valid ? i_raw : n - 1;
    const double f0 = f3[3 * i], f1 = f3[3 * i + 1], f2 = f3[3 * i + 2];
    const double tau = tau_in[i];
    const int n_t = m.n_t, n_f = m.n_f;
    const double M = k.M, inv_M2 = k.inv_M2;
    const double a2 = f0 - 2.0 * f1 + f2, a1 = 2.0 * M * (f1 - f0), a0 = M * M * f0;
    const double fa = k.df * tau, fb = k.f_min * tau;     // turns per bin, turns at bin 0
    const float two_pi = 6.28318530717958647692f;
    // Column j, j + P, ... of this thread by forward differences (x(j + P) - x(j) =
    // (a2 (2 P j + P^2) + a1 P) / M^2, second difference 2 P^2 a2 / M^2), in fixed
    // point so the column loop has no FP64 arithmetic (a slow pipe on this GPU):
    // the position X = x 2^32 (Q32.32) and the phase T = frac(fb + fa x) 2^64
    // (Q0.64, wrapping), each a quadratic in j, advance by exact integer additions.
    // The position's differences are rounded once from FP64, so after s steps it is
    // within about s^2 2^-33 bins (s <= n_t / P); the phase is exact given its
    // coefficients, each within 2^-64 turn.  |x| <= max |f| by the convex hull, so |f| < 2^30 keeps X in range;
    // larger or non-finite control frequencies give NaN.
    const bool finite = fabs(f0) < 1073741824.0 && fabs(f1) < 1073741824.0 && fabs(f2) < 1073741824.0 &&
                        fabs(tau) < 1e30;
    const double jl = (double)t, Pd = (double)P;
    const double x_t = finite ? ((a2 * jl + a1) * jl + a0) * inv_M2 : 0.0;
    const double dx = finite ? (a2 * (2.0 * Pd * jl + Pd * Pd) + a1 * Pd) * inv_M2 : 0.0;
    const double ddx = finite ? 2.0 * Pd * Pd * a2 * inv_M2 : 0.0;
    const double two32 = 4294967296.0;
    int64_t X = __double2ll_rn(x_t * two32), DX = __double2ll_rn(dx * two32);
    const int64_t DDX = __double2ll_rn(ddx * two32);
    // The phase is a quadratic in j modulo one turn: T(j) = tau0 + tau1 j + tau2 j^2
    // with tau0 = frac(fb + fa C0), tau1 = frac(fa C1), tau2 = frac(fa C2) and
    // x(j) = C0 + C1 j + C2 j^2.  The template's thread 0 converts them to Q0.64
    // (FP64, once a template); every thread's start value and differences follow
    // in wrapping 64-bit integer arithmetic, exact given the three coefficients.
    __shared__ uint64_t tq[TPB][5];  // tau0, tau1, tau2, and the phases at the band edges
    const int tl = tid / P;
    if (t == 0) {
        auto q64 = [](double turns) {                      // frac(turns) as Q0.64
            const double fr = turns - floor(turns);        // [0, 1]
            return (uint64_t)__double2ll_rn(ldexp(fr - rint(fr), 63)) << 1;  // signed [-1/2, 1/2] turn
        };
        tq[tl][0] = finite ? q64(fb + fa * (a0 * inv_M2)) : 0;
        tq[tl][1] = finite ? q64(fa * (a1 * inv_M2)) : 0;
        tq[tl][2] = finite ? q64(fa * (a2 * inv_M2)) : 0;
        tq[tl][3] = finite ? q64(fb) : 0;
        tq[tl][4] = finite ? q64(fb + fa * (double)(n_f - 1)) : 0;
    }
    if (WPT > 1) __syncthreads();
    else __syncwarp();  // one warp a template: its lane 0 wrote, its lanes read
    const uint64_t tau1 = tq[tl][1], tau2 = tq[tl][2], T_lo = tq[tl][3], T_hi = tq[tl][4];
    const uint64_t tt = (uint64_t)t, PP = (uint64_t)P;
    uint64_t T = tq[tl][0] + tau1 * tt + tau2 * (tt * tt);
    uint64_t DT = tau1 * PP + tau2 * (2 * PP * tt + PP * PP);
    const uint64_t DDT = tau2 * (2 * PP * PP);
    const int64_t X_hi = (int64_t)(n_f - 1) << 32;
    float S = 0.f, W = 0.f;
    float dS0 = 0.f, dS1 = 0.f, dS2 = 0.f, dS3 = 0.f, dW0 = 0.f, dW1 = 0.f, dW2 = 0.f;
    for (int j = t; j < n_t; j += P) {
        int64_t Xc = X;
        uint64_t Tc = T;
        X += DX;
        DX += DDX;
        T += DT;
        DT += DDT;
        bool clamped = false;
        if (Xc < 0) { Xc = 0; Tc = T_lo; clamped = true; }
        if (Xc > X_hi) { Xc = X_hi; Tc = T_hi; clamped = true; }
        int kb = (int)(Xc >> 32);
        float a = (float)(uint32_t)Xc * 2.3283064365386963e-10f;  // fraction of the bin, 2^-32
        if (kb > n_f - 2) { a += (float)(kb - (n_f - 2)); kb = n_f - 2; }  // x = n_f - 1: the top knot
        if (n_f < 2) { kb = 0; a = 0.f; }
        float z0r, z0i, w0, z1r, z1i, w1;
        pixel_at<WMODE, PREC>(m, j, kb, z0r, z0i, w0, k.err);
        if (n_f > 1) pixel_at<WMODE, PREC>(m, j, kb + 1, z1r, z1i, w1, k.err);
        else { z1r = z0r; z1i = z0i; w1 = w0; }
        const float dzr = z1r - z0r, dzi = z1i - z0i, dw = w1 - w0;
        const float zr = fmaf(a, dzr, z0r), zi = fmaf(a, dzi, z0i), w = fmaf(a, dw, w0);
        float sn, cs;
        __sincosf((float)(int32_t)(Tc >> 32) * (two_pi * 2.3283064365386963e-10f), &sn, &cs);
        const float re = cs * zr - sn * zi, im = sn * zr + cs * zi;
        S += re;
        W += w;
        if (ADJOINT) {
            // d re/dx = -im 2 pi df tau + Re[e^{i phi} dz/dx]; d re/dtau = -im 2 pi f
            const float dre_dx = clamped ? 0.f : fmaf(-im, two_pi * (float)fa, cs * dzr - sn * dzi);
            const float dw_dx = clamped ? 0.f : dw;
            const float u = (float)j * k.inv_Mf, c0 = (1.f - u) * (1.f - u), c1 = 2.f * (1.f - u) * u, c2 = u * u;
            dS0 = fmaf(dre_dx, c0, dS0);
            dS1 = fmaf(dre_dx, c1, dS1);
            dS2 = fmaf(dre_dx, c2, dS2);
            dW0 = fmaf(dw_dx, c0, dW0);
            dW1 = fmaf(dw_dx, c1, dW1);
            dW2 = fmaf(dw_dx, c2, dW2);
            dS3 = fmaf(-im, two_pi * fmaf((float)kb + a, k.df_f, k.fmin_f), dS3);
        }
    }
    constexpr int NV = ADJOINT ? 9 : 2;
    float v[NV];
    v[0] = S;
    v[1] = W;
    if (ADJOINT) {
        v[2 % NV] = dS0; v[3 % NV] = dS1; v[4 % NV] = dS2; v[5 % NV] = dS3;
        v[6 % NV] = dW0; v[7 % NV] = dW1; v[8 % NV] = dW2;
    }
#pragma unroll
    for (int q = 0; q < NV; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    if (WPT > 1) {
        // the template's warps' sums, added in warp order by its thread 0
        __shared__ float red[kInterpBlock / 32][NV];
        if (lane == 0)
#pragma unroll
            for (int q = 0; q < NV; ++q) red[warp][q] = v[q];
        __syncthreads();
        if (t == 0)
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                float a = red[warp][q];
                for (int w = 1; w < WPT; ++w) a += red[warp + w][q];
                v[q] = a;
            }
    }
    if (t != 0 || !valid) return;
    if (!finite)
#pragma unroll
        for (int q = 0; q < NV; ++q) v[q] = __int_as_float(0x7fc00000);  // NaN
    S = v[0];
    W = v[1];
    const bool varying = WMODE != WMODE_CONST && !m.paper;
    const float scale = varying ? (W > 0.f ? rsqrtf(W) : 0.f) : (float)m.norm;   // W = 0: all notched
    if (MODE == 0 || snr_out) snr_out[i] = S * scale;
    if (!ADJOINT) return;
    const float gi = MODE == 2 ? 1.f : (g ? g[i] : 1.f);
    float gr[4];
    if (varying) {
        const float h = 0.5f * S * scale * scale * scale;
        gr[0] = gi * (v[2 % NV] * scale - h * v[6 % NV]);
        gr[1] = gi * (v[3 % NV] * scale - h * v[7 % NV]);
        gr[2] = gi * (v[4 % NV] * scale - h * v[8 % NV]);
    } else {
        gr[0] = gi * v[2 % NV] * scale;
        gr[1] = gi * v[3 % NV] * scale;
        gr[2] = gi * v[4 % NV] * scale;
    }
    gr[3] = gi * v[5 % NV] * scale;
    if (MODE == 2) {
        const float gs[4] = {gr[0], gr[1], gr[2], gr[3] * ad.tau_max};  // dSNR/d(f0, f1, f2, u)
        adam_update(ad, i, const_cast<float *>(f3), const_cast<float *>(tau_in), gs);
        return;
    }
    gf3[3 * i] = gr[0];
    gf3[3 * i + 1] = gr[1];
    gf3[3 * i + 2] = gr[2];
    gtau[i] = gr[3];
}

InterpConst interp_const(const MapDev &m, int *err)
{
    InterpConst k;
    k.err = err;
    k.M = (double)(m.n_t - 1);
    k.inv_M2 = 1.0 / (k.M * k.M);
    k.df = m.df;
    k.f_min = m.f_min;
    k.inv_Mf = 1.f / (float)k.M;
    k.df_f = (float)m.df;
    k.fmin_f = (float)m.f_min;
    return k;
}

// Threads per template: 0 picks by the template count.  More threads per template
// fill the GPU when templates are few; each thread also repeats part of the
// template's setup, so with many templates one warp each is fastest (50 ascent
// steps on the 500 x 1600 map, ms, for 32 / 64 / 128 threads: 256 templates
// 0.78 / 0.69 / 0.57, 1024: 0.98 / 0.98 / 0.98, 4096: 1.93 / 2.19 / 3.00,
// 16384: 5.43 / 7.13 / 10.5).
int interp_threads(uint64_t n, int P)
{
    if (P == 32 || P == 64 || P == 128) return P;
    if (n <= 512) return 128;
    if (n <= 1536) return 64;
    return 32;
}

template <int MODE, int P>
cudaError_t launch_interp_P(const MapDev &m, const float *f3, const float *tau, const float *g, uint64_t n,
                            float *snr, float *gf3, float *gtau, const AdamStep &ad, int *err, cudaStream_t st)
{
    constexpr uint64_t TPB = kInterpBlock / P;
    const uint64_t blocks = (n + TPB - 1) / TPB;
    if (blocks > 0x7fffffffull) return cudaErrorInvalidValue;
    const unsigned b = (unsigned)blocks;
    const InterpConst k = interp_const(m, err);
#define STK_INTERP(W, PR) \
    interp_kernel<W, PR, MODE, P><<<b, kInterpBlock, 0, st>>>(m, k, f3, tau, g, n, snr, gf3, gtau, ad)
    if (m.prec == PREC_FP16) {
        if (m.wmode == WMODE_CONST) STK_INTERP(WMODE_CONST, PREC_FP16);
        else if (m.wmode == WMODE_FREQ) STK_INTERP(WMODE_FREQ, PREC_FP16);
        else STK_INTERP(WMODE_PIXEL, PREC_FP16);
    } else {
        if (m.wmode == WMODE_CONST) STK_INTERP(WMODE_CONST, PREC_FP32);
        else if (m.wmode == WMODE_FREQ) STK_INTERP(WMODE_FREQ, PREC_FP32);
        else STK_INTERP(WMODE_PIXEL, PREC_FP32);
    }
#undef STK_INTERP
    return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_interp_M(const MapDev &m, const float *f3, const float *tau, const float *g, uint64_t n,
                            float *snr, float *gf3, float *gtau, const AdamStep &ad, int P, int *err, cudaStream_t st)
{
    switch (interp_threads(n, P)) {
    case 128: return launch_interp_P<MODE, 128>(m, f3, tau, g, n, snr, gf3, gtau, ad, err, st);
    case 64: return launch_interp_P<MODE, 64>(m, f3, tau, g, n, snr, gf3, gtau, ad, err, st);
    default: return launch_interp_P<MODE, 32>(m, f3, tau, g, n, snr, gf3, gtau, ad, err, st);
    }
}

__global__ void __launch_bounds__(256) refine_init_kernel(const float *__restrict__ tau, float *__restrict__ u,
                                                          float4 *__restrict__ st, uint64_t n, float tau_max)
{
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    u[i] = tau[i] / tau_max;
    st[2 * i] = make_float4(0.f, 0.f, 0.f, 0.f);
    st[2 * i + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// ------------------------------------------------------------------ discrete follow-up
// The refined continuous templates are judged by the discrete statistic (Eq. 7
// on whole pixels).  The polish climbs that statistic directly, one warp per
// template: the delay is set to the nearest maximum of SNR(tau) at the
// template's fixed pixels (W does not depend on tau; S(tau) = sum_j |z_j|
// cos(2 pi f_j tau + arg z_j) is smooth, so safeguarded Newton steps on S find
// it), then each control bin moves by +-1 while a move, with its delay again
// maximised, raises the SNR.  The climb compares warp sums (any summation
// order); the choice among the start, the polished start and the polished
// alternative uses the scorer's own sequential sum, so it never returns a
// template that scores below the start.
constexpr int kPolishBlock = 128;   // 4 warps, one template each
constexpr int kPolishNewton = 4;    // Newton steps per delay search

struct PolishSums {
    float S, dS, d2S, W;
};

// S, dS/dtau, d2S/dtau2 and W of template f at delay tau, summed over the warp's
// lanes (lane l takes columns l, l + 32, ...), the same value in every lane.
template <int WMODE, int PREC>
__device__ __forceinline__ PolishSums polish_eval(const MapDev &m, const uint32_t f[3], double tau, int lane, int *err)
{
    const Phase ph = phase_consts(m.f_min, m.df, tau, m.n_f);
    const float two_pi = 6.28318530717958647692f, fmin_f = (float)m.f_min, df_f = (float)m.df;
    float S = 0.f, dS = 0.f, d2S = 0.f, W = 0.f;
    for (int j = lane; j < m.n_t; j += 32) {
        uint32_t b = raster_bin_wide(f[0], f[1], f[2], m.M, (uint32_t)j, m.d);
        if (kDebugBounds) b = checked_bin(b, j, m.n_t, hull_lo(f), hull_hi(f), err);
        const typename Pix<PREC>::Rec v = Pix<PREC>::load_global(m.rec, (size_t)j * m.ldr + b);
        float wv = 0.f;
        if (WMODE == WMODE_FREQ) wv = __ldg(m.w + b);
        if (WMODE == WMODE_PIXEL) wv = __ldg(m.w + (size_t)j * m.ldw + b);
        const uint32_t T = template_turn(b, ph);
        float x, mg = Pix<PREC>::mag(v);
        if constexpr (PREC == PREC_FP32) {
            x = fmaf((float)(int32_t)T, kTurnToRad, Pix<PREC>::arg_rad(v));
        } else {
            x = (float)(int32_t)(T + ((uint32_t)v << 16)) * kTurnToRad;
            if (WMODE != WMODE_CONST) mg *= wv;
        }
        float sn, cs;
        __sincosf(x, &sn, &cs);
        const float om = two_pi * fmaf((float)b, df_f, fmin_f);   // d angle / d tau
        S = fmaf(mg, cs, S);
        dS = fmaf(-mg * sn, om, dS);
        d2S = fmaf(-mg * cs, om * om, d2S);
        W += PREC == PREC_FP32 ? wv : wv * wv;
    }
    float v4[4] = {S, dS, d2S, W};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        for (int o = 16; o > 0; o >>= 1) v4[q] += __shfl_xor_sync(0xffffffffu, v4[q], o);
        v4[q] = __shfl_sync(0xffffffffu, v4[q], 0);   // lane 0's sum for every lane: uniform decisions
    }
    return {v4[0], v4[1], v4[2], v4[3]};
}

template <int WMODE>
__device__ __forceinline__ float polish_snr(const PolishSums &s, const MapDev &m)
{
    if (WMODE == WMODE_CONST || m.paper) return s.S * m.norm_f;
    return s.W > 0.f ? s.S * rsqrtf(s.W) : 0.f;
}

// The delay maximising SNR near tau, within [-tau_max, tau_max]: Newton steps on
// S where it is concave, else a step towards increasing S, each at most a tenth
// of the shortest period in the band and kept only when the SNR rises (else
// halved, twice).  Returns the SNR at the returned delay.
template <int WMODE, int PREC>
__device__ __forceinline__ float polish_delay(const MapDev &m, const uint32_t f[3], double &tau, double tau_max, int lane,
                                              int *err)
{
    PolishSums cur = polish_eval<WMODE, PREC>(m, f, tau, lane, err);
    float snr = polish_snr<WMODE>(cur, m);
    const double f_top = m.f_min + (m.n_f - 1) * m.df;
    const double dmax = 0.1 / fabs(f_top);
    for (int it = 0; it < kPolishNewton; ++it) {
        double step;
        if (cur.d2S < 0.f) step = -(double)cur.dS / (double)cur.d2S;
        else step = cur.dS > 0.f ? dmax : (cur.dS < 0.f ? -dmax : 0.0);
        step = fmin(fmax(step, -dmax), dmax);
        if (!(step != 0.0)) break;
        bool moved = false;
        for (int h = 0; h < 3 && !moved; ++h, step *= 0.5) {
            const double t = fmin(fmax(tau + step, -tau_max), tau_max);
            if (t == tau) break;
            const PolishSums nx = polish_eval<WMODE, PREC>(m, f, t, lane, err);
            const float sn = polish_snr<WMODE>(nx, m);
            if (sn > snr) {
                tau = t;
                cur = nx;
                snr = sn;
                moved = true;
            }
        }
        if (!moved) break;
    }
    return snr;
}

// Hill climb from (f, tau): delay first, then +-1 moves of the control bins.
template <int WMODE, int PREC>
__device__ __forceinline__ void polish_climb(const MapDev &m, uint32_t f[3], double &tau, double tau_max, int moves, int lane,
                                             int *err)
{
    float snr = polish_delay<WMODE, PREC>(m, f, tau, tau_max, lane, err);
    for (int mv = 0; mv < moves; ++mv) {
        uint32_t bf[3] = {f[0], f[1], f[2]};
        double bt = tau;
        float bs = snr;
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int d = -1; d <= 1; d += 2) {
                if ((d < 0 && f[k] == 0) || (d > 0 && f[k] + 1 >= (uint32_t)m.n_f)) continue;
                uint32_t g[3] = {f[0], f[1], f[2]};
                g[k] += (uint32_t)d;
                double t = tau;
                const float sn = polish_delay<WMODE, PREC>(m, g, t, tau_max, lane, err);
                if (sn > bs) {
                    bf[0] = g[0]; bf[1] = g[1]; bf[2] = g[2];
                    bt = t;
                    bs = sn;
                }
            }
        if (!(bs > snr)) break;
        f[0] = bf[0]; f[1] = bf[1]; f[2] = bf[2];
        tau = bt;
        snr = bs;
    }
}

// The scorer's SNR of one template: columns in order, one thread, the same
// per-pixel arithmetic and normalisation as stk_score_explicit (bit-identical).
template <int WMODE, int PREC>
__device__ __forceinline__ float polish_canonical(const MapDev &m, const uint32_t f[3], double tau, int *err)
{
    const Phase ph = phase_consts(m.f_min, m.df, tau, m.n_f);
    float acc = 0.f, W = 0.f;
    for (int j = 0; j < m.n_t; ++j) {
        uint32_t b = raster_bin_wide(f[0], f[1], f[2], m.M, (uint32_t)j, m.d);
        if (kDebugBounds) b = checked_bin(b, j, m.n_t, hull_lo(f), hull_hi(f), err);
        const typename Pix<PREC>::Rec v = Pix<PREC>::load_global(m.rec, (size_t)j * m.ldr + b);
        float wv = 0.f;
        if (WMODE == WMODE_FREQ) wv = __ldg(m.w + b);
        if (WMODE == WMODE_PIXEL) wv = __ldg(m.w + (size_t)j * m.ldw + b);
        accumulate<PREC, WMODE>(v, b, ph, wv, acc, W);
    }
    return finalize_snr<WMODE>(acc, W, m);
}

template <int WMODE, int PREC>
__global__ void __launch_bounds__(kPolishBlock) polish_kernel(MapDev m, uint32_t *__restrict__ f3,
                                                              double *__restrict__ tau,
                                                              const float *__restrict__ alt_f3,
                                                              const float *__restrict__ alt_tau, uint64_t n,
                                                              double tau_max, int moves, double *__restrict__ snr_out,
                                                              int *__restrict__ which_out, int *err)
{
    const uint64_t i = (uint64_t)blockIdx.x * (kPolishBlock / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= n) return;   // whole warps leave together
    const uint32_t fs[3] = {min(f3[3 * i], (uint32_t)m.n_f - 1), min(f3[3 * i + 1], (uint32_t)m.n_f - 1),
                            min(f3[3 * i + 2], (uint32_t)m.n_f - 1)};
    const double ts = tau[i];
    uint32_t fa[3] = {fs[0], fs[1], fs[2]};
    double ta = fmin(fmax(ts, -tau_max), tau_max);
    polish_climb<WMODE, PREC>(m, fa, ta, tau_max, moves, lane, err);
    uint32_t fb[3] = {fa[0], fa[1], fa[2]};
    double tb = ta;
    if (alt_f3) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float x = alt_f3[3 * i + k];
            const float r = rintf(fminf(fmaxf(x == x ? x : 0.f, 0.f), (float)(m.n_f - 1)));
            fb[k] = (uint32_t)r;
        }
        const double t = (double)alt_tau[i];
        tb = t == t ? fmin(fmax(t, -tau_max), tau_max) : ta;
        polish_climb<WMODE, PREC>(m, fb, tb, tau_max, moves, lane, err);
    }
    if (lane != 0) return;
    // the choice, by the scorer's own sums: the start unless a polished form beats it
    const float s0 = polish_canonical<WMODE, PREC>(m, fs, ts, err);
    const float s1 = polish_canonical<WMODE, PREC>(m, fa, ta, err);
    const float s2 = alt_f3 ? polish_canonical<WMODE, PREC>(m, fb, tb, err) : s1;
    int w = 0;
    float best = s0;
    if (s1 > best) { w = 1; best = s1; }
    if (alt_f3 && s2 > best) { w = 2; best = s2; }
    const uint32_t *fo = w == 0 ? fs : (w == 1 ? fa : fb);
    f3[3 * i] = fo[0];
    f3[3 * i + 1] = fo[1];
    f3[3 * i + 2] = fo[2];
    tau[i] = w == 0 ? ts : (w == 1 ? ta : tb);
    if (snr_out) snr_out[i] = (double)best;
    if (which_out) which_out[i] = w;
}

}  // namespace

size_t refine_scratch_bytes(uint64_t n)
{
    return (size_t)n * (sizeof(float4) * 2 + sizeof(float));  // moments, u
}

cudaError_t launch_refine(const MapDev &m, float *f3, float *tau, uint64_t n, int steps, float lr_f, float lr_u,
                          float tau_max, float *hist, void *scratch, int P, int *err, cudaStream_t st)
{
    if (n == 0 || steps < 0) return cudaSuccess;
    AdamStep ad{};
    ad.mom = static_cast<float4 *>(scratch);
    ad.u = reinterpret_cast<float *>(ad.mom + 2 * n);
    ad.tau_max = tau_max;
    ad.f_hi = (float)(m.n_f - 1);
    refine_init_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(tau, ad.u, ad.mom, n, tau_max);
    cudaError_t e = cudaGetLastError();
    for (int t = 1; t <= steps && e == cudaSuccess; ++t) {
        // the step's SNR (history row t - 1), its gradient and the update, in one launch
        const double bc1 = 1.0 - std::pow(0.9, t), bc2 = 1.0 - std::pow(0.999, t);
        ad.step_f = (float)(lr_f / bc1);
        ad.step_u = (float)(lr_u / bc1);
        ad.sbc2 = (float)std::sqrt(bc2);
        e = launch_interp_M<2>(m, f3, tau, nullptr, n, hist ? hist + (size_t)(t - 1) * n : nullptr, nullptr,
                               nullptr, ad, P, err, st);
    }
    if (e == cudaSuccess && hist)
        e = launch_interp_M<0>(m, f3, tau, nullptr, n, hist + (size_t)steps * n, nullptr, nullptr, AdamStep{}, P,
                               err, st);
    return e;
}

cudaError_t launch_interp_tuned(const MapDev &m, const float *f3, const float *tau, const float *g, uint64_t n,
                                float *snr, float *gf3, float *gtau, bool adjoint, int P, int *err, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    return adjoint ? launch_interp_M<1>(m, f3, tau, g, n, snr, gf3, gtau, AdamStep{}, P, err, st)
                   : launch_interp_M<0>(m, f3, tau, g, n, snr, gf3, gtau, AdamStep{}, P, err, st);
}

cudaError_t launch_polish(const MapDev &m, uint32_t *f3, double *tau, const float *alt_f3, const float *alt_tau,
                          uint64_t n, double tau_max, int moves, double *snr, int *which, int *err, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    constexpr uint64_t TPB = kPolishBlock / 32;
    const uint64_t blocks = (n + TPB - 1) / TPB;
    if (blocks > 0x7fffffffull) return cudaErrorInvalidValue;
    const unsigned b = (unsigned)blocks;
#define STK_POLISH(W, PR) \
    polish_kernel<W, PR><<<b, kPolishBlock, 0, st>>>(m, f3, tau, alt_f3, alt_tau, n, tau_max, moves, snr, which, err)
    if (m.prec == PREC_FP16) {
        if (m.wmode == WMODE_CONST) STK_POLISH(WMODE_CONST, PREC_FP16);
        else if (m.wmode == WMODE_FREQ) STK_POLISH(WMODE_FREQ, PREC_FP16);
        else STK_POLISH(WMODE_PIXEL, PREC_FP16);
    } else {
        if (m.wmode == WMODE_CONST) STK_POLISH(WMODE_CONST, PREC_FP32);
        else if (m.wmode == WMODE_FREQ) STK_POLISH(WMODE_FREQ, PREC_FP32);
        else STK_POLISH(WMODE_PIXEL, PREC_FP32);
    }
#undef STK_POLISH
    return cudaGetLastError();
}

cudaError_t launch_interp(const MapDev &m, const float *f3, const float *tau, const float *g, uint64_t n, float *snr,
                          float *gf3, float *gtau, bool adjoint, int *err, cudaStream_t st)
{
    return launch_interp_tuned(m, f3, tau, g, n, snr, gf3, gtau, adjoint, 0, err, st);
}

}  // namespace stk
