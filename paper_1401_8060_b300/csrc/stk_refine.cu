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
// P = 32, 64 or 128 threads per template: thread l takes the columns j = l (mod
// P) in order; the lanes' partial sums meet in a fixed shuffle tree and the
// template's warps' sums are added in warp order (deterministic).  Sums and the
// pixel arithmetic are FP32.  The curve position x_j and the phase need more than
// FP32 (which resolves x_j ~ 10^3 only to 6e-5 bins): a template's quadratic
// coefficients are formed once per evaluation in FP64 (a slow pipe on this GPU,
// so eight lanes share the work), and each thread's positions and phases follow
// from them by exact fixed-point integer arithmetic.  The ascent runs all its
// steps in one launch, each template's parameters and Adam moments held by its
// thread 0.
#include <cuda_fp16.h>

#include <cmath>

#include "stk_internal.cuh"
#include <vector>

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

// One template's curve and phase coefficients for one evaluation, set up by
// eight lanes of the block's first warp, one value a lane (FP64 is a slow pipe
// on this GPU, so no other thread repeats it), and read by the template's threads
// from shared memory:
//   x(j) = C0 + C1 j + C2 j^2 bins, (C0, C1, C2) = (a0, a1, a2) / M^2, each a
//     Q32.96 two's complement integer (lo, hi words), so that every thread's start
//     position and forward differences follow in exact 128-bit integer arithmetic;
//   phase(j) = tau0 + tau1 j + tau2 j^2 turns (mod 1), each Q0.64, with the phases
//     at the band edges, where the clamped curve sits.
struct TplSetup {
    uint64_t ph[5];  // tau0, tau1, tau2, phase at bin 0, phase at bin n_f - 1
    uint64_t c[6];   // C0, C1, C2 as (lo, hi)
    float fa;        // turns per bin, df tau
    int finite;      // control frequencies and delay within range
};

// Lane q (0..7) of a template's setup: value q of TplSetup (0-4 the phase
// coefficients, 5-7 C0..C2) from the template's control bins and delay (s).
// |f| < 2^29 keeps C 2^32 within int64 and the positions within Q32.32 (|x| <=
// max |f| by the convex hull); larger or non-finite control frequencies, or a
// non-finite delay, mark the template, whose results are then NaN.
__device__ __forceinline__ void setup_lane(const InterpConst &k, int n_f, float f0f, float f1f, float f2f,
                                           float tauf, int q, TplSetup &su)
{
    const float lim = 536870912.f;  // 2^29
    const bool finite = fabsf(f0f) < lim && fabsf(f1f) < lim && fabsf(f2f) < lim && fabsf(tauf) < 1e30f;
    const double f0 = f0f, f1 = f1f, f2 = f2f, tau = tauf;
    const double M = k.M;
    const double a2 = f0 - 2.0 * f1 + f2, a1 = 2.0 * M * (f1 - f0), a0 = M * M * f0;
    const double fa = k.df * tau, fb = k.f_min * tau;  // turns per bin, turns at bin 0
    const double base = (q == 0 || q == 5 ? a0 : (q == 1 || q == 6 ? a1 : a2)) * k.inv_M2;
    if (q < 5) {
        // tau0 = frac(fb + fa C0), tau1 = frac(fa C1), tau2 = frac(fa C2), then the
        // phases at bins 0 and n_f - 1; signed [-1/2, 1/2] turn, as Q0.64
        const double mul = q == 3 ? 0.0 : (q == 4 ? (double)(n_f - 1) : base);
        const double add = q == 1 || q == 2 ? 0.0 : fb;
        const double turns = add + fa * mul;
        const double fr = turns - floor(turns);
        su.ph[q] = finite ? (uint64_t)__double2ll_rn((fr - rint(fr)) * 9223372036854775808.0) << 1 : 0;
    } else {
        // C 2^96 = floor(C 2^32) 2^64 + frac(C 2^32) 2^64 (both parts exact)
        const double sc = base * 4294967296.0;
        const double h = floor(sc);
        su.c[2 * (q - 5)] = finite ? __double2ull_rz((sc - h) * 18446744073709551616.0) : 0;
        su.c[2 * (q - 5) + 1] = finite ? (uint64_t)__double2ll_rn(h) : 0;
    }
    if (q == 0) {
        su.fa = (float)fa;
        su.finite = finite;
    }
}

// The template's setup by the first 8 TPB threads of the block, then a barrier.
template <int TPB, typename Params>
__device__ __forceinline__ void setup_block(const InterpConst &k, int n_f, TplSetup *su, Params params)
{
    const int tid = threadIdx.x;
    if (tid < 8 * TPB) {
        float f0, f1, f2, tau;
        params(tid >> 3, f0, f1, f2, tau);
        setup_lane(k, n_f, f0, f1, f2, tau, tid & 7, su[tid >> 3]);
    }
    __syncthreads();
}

typedef unsigned __int128 u128;

__device__ __forceinline__ u128 q96(const uint64_t *c) { return ((u128)c[1] << 64) | c[0]; }

// Q32.96 to Q32.32, rounded (two's complement, wrapping).
__device__ __forceinline__ uint64_t q96_to_q32(u128 v) { return (uint64_t)((v + ((u128)1 << 63)) >> 64); }

// One evaluation of a template by its P threads (thread t takes the columns
// j = t (mod P) in order; the lanes' partial sums meet in a fixed shuffle tree,
// the template's warps' sums are added in warp order: deterministic).  Every
// thread of the block calls it (it has a barrier when P > 32).  Returns true on
// the template's thread 0, with snr and, when ADJOINT, gi * dSNR/d(f0, f1, f2, tau).
template <int WMODE, int PREC, bool ADJOINT, int P>
__device__ __forceinline__ bool interp_step(const MapDev &m, const InterpConst &k, const TplSetup &su, int t,
                                            float gi, float &snr, float gr[4])
{
    constexpr int WPT = P / 32;  // warps a template
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n_t = m.n_t, n_f = m.n_f;
    const float two_pi = 6.28318530717958647692f;
    // Columns j, j + P, ... of this thread by forward differences in fixed point,
    // so the column loop has no FP64 arithmetic: the position X = x 2^32 (Q32.32)
    // and the phase T = phase 2^64 (Q0.64, wrapping) advance by integer additions.
    // The start x(t) and the differences x(t + P) - x(t) = C1 P + C2 (2 P t + P^2)
    // and 2 P^2 C2 are exact in Q32.96 and rounded once to Q32.32, so after s steps
    // the position is within about s^2 2^-33 bins (s <= n_t / P); the phase is exact
    // given its coefficients, each within 2^-64 turn.
    const u128 C0 = q96(su.c), C1 = q96(su.c + 2), C2 = q96(su.c + 4);
    const uint64_t tt = (uint64_t)t, PP = (uint64_t)P;
    uint64_t X = q96_to_q32(C0 + C1 * tt + C2 * (tt * tt));
    uint64_t DX = q96_to_q32(C1 * PP + C2 * (2 * PP * tt + PP * PP));
    const uint64_t DDX = q96_to_q32(C2 * (2 * PP * PP));
    const uint64_t tau1 = su.ph[1], tau2 = su.ph[2], T_lo = su.ph[3], T_hi = su.ph[4];
    uint64_t T = su.ph[0] + tau1 * tt + tau2 * (tt * tt);
    uint64_t DT = tau1 * PP + tau2 * (2 * PP * tt + PP * PP);
    const uint64_t DDT = tau2 * (2 * PP * PP);
    const float fa = su.fa;
    const int64_t X_hi = (int64_t)(n_f - 1) << 32;
    float S = 0.f, W = 0.f;
    float dS0 = 0.f, dS1 = 0.f, dS2 = 0.f, dS3 = 0.f, dW0 = 0.f, dW1 = 0.f, dW2 = 0.f;
    for (int j = t; j < n_t; j += P) {
        int64_t Xc = (int64_t)X;
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
            const float dre_dx = clamped ? 0.f : fmaf(-im, two_pi * fa, cs * dzr - sn * dzi);
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
    if (!ADJOINT) {
#pragma unroll
        for (int q = 0; q < NV; ++q)
            for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    } else {
        // The same butterfly (lane l adds lane l ^ o at o = 16, 8, 4, 2, 1, so every
        // lane ends with the same sums), transposed: each level sends half of the
        // values still held, and the lanes with bit o set keep the upper half.  Value
        // q ends in lanes 2q and 2q + 1, from where lane 0 fetches it: 25 shuffles
        // instead of 45.
        float u[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) u[q] = q < NV ? v[q % NV] : 0.f;
#pragma unroll
        for (int o = 16, h = 8; o > 1; o >>= 1, h >>= 1) {
            const bool up = (lane & o) != 0;
#pragma unroll
            for (int q = 0; q < h; ++q) {
                const float send = up ? u[q] : u[q + h];
                const float keep = up ? u[q + h] : u[q];
                u[q] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
        u[0] += __shfl_xor_sync(0xffffffffu, u[0], 1);
#pragma unroll
        for (int q = 0; q < NV; ++q) v[q] = __shfl_sync(0xffffffffu, u[0], 2 * q);
    }
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
    if (t != 0) return false;
    if (!su.finite)
#pragma unroll
        for (int q = 0; q < NV; ++q) v[q] = __int_as_float(0x7fc00000);  // NaN
    S = v[0];
    W = v[1];
    const bool varying = WMODE != WMODE_CONST && !m.paper;
    const float scale = varying ? (W > 0.f ? rsqrtf(W) : 0.f) : (float)m.norm;   // W = 0: all notched
    snr = S * scale;
    if (ADJOINT) {
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
    }
    return true;
}

// P threads per template (32, 64 or 128), kInterpBlock / P templates a block.
// MODE 0: forward (snr); 1: adjoint (g * gradient to gf3, gtau; snr too when
// snr_out is given).
template <int WMODE, int PREC, int MODE, int P>
__global__ void __launch_bounds__(kInterpBlock) interp_kernel(MapDev m, InterpConst k, const float *__restrict__ f3,
                                                              const float *__restrict__ tau,
                                                              const float *__restrict__ g, uint64_t n,
                                                              float *__restrict__ snr_out, float *__restrict__ gf3,
                                                              float *__restrict__ gtau)
{
    constexpr int TPB = kInterpBlock / P;
    constexpr bool ADJOINT = MODE != 0;
    __shared__ TplSetup su[TPB];
    const uint64_t first = (uint64_t)blockIdx.x * TPB;
    setup_block<TPB>(k, m.n_f, su, [&](int tl, float &f0, float &f1, float &f2, float &tv) {
        const uint64_t i = first + tl < n ? first + tl : n - 1;  // the last block's spare slots repeat one
        f0 = f3[3 * i];
        f1 = f3[3 * i + 1];
        f2 = f3[3 * i + 2];
        tv = tau[i];
    });
    const int tl = threadIdx.x / P, t = threadIdx.x % P;
    const uint64_t i = first + tl;
    const float gi = ADJOINT && g && t == 0 && i < n ? g[i] : 1.f;
    float snr, gr[4];
    if (!interp_step<WMODE, PREC, ADJOINT, P>(m, k, su[tl], t, gi, snr, gr) || i >= n) return;
    if (!ADJOINT || snr_out) snr_out[i] = snr;
    if (ADJOINT) {
        gf3[3 * i] = gr[0];
        gf3[3 * i + 1] = gr[1];
        gf3[3 * i + 2] = gr[2];
        gtau[i] = gr[3];
    }
}

// Step sizes of one Adam step and the projection's bounds.
struct AdamStep {
    float step_f, step_u, sbc2, tau_max, f_hi;
};

// One Adam step of the gradient ascent of a template's SNR (Adam with betas 0.9,
// 0.999 and eps 1e-8 on the loss -SNR, in torch's arithmetic order) on p = (f0,
// f1, f2, u = tau / tau_max) with moments mo, ve, then the projection onto f in
// [0, n_f - 1] and |u| <= 1.  step_f = lr_f / (1 - 0.9^t), step_u likewise, sbc2
// = sqrt(1 - 0.999^t), from the host.
__device__ __forceinline__ void adam_update(const AdamStep &ad, float p[4], float mo[4], float ve[4],
                                            const float gs[4])
{
    const float w1 = 0.1f, b2 = 0.999f, w2 = 0.001f, eps = 1e-8f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float g = -gs[q];                                   // d(-SNR)/d(f, u)
        mo[q] = mo[q] + w1 * (g - mo[q]);
        ve[q] = ve[q] * b2 + w2 * g * g;
        const float denom = __fsqrt_rn(ve[q]) / ad.sbc2 + eps;
        p[q] = p[q] - (q < 3 ? ad.step_f : ad.step_u) * (mo[q] / denom);
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) p[q] = fminf(fmaxf(p[q], 0.f), ad.f_hi);
    p[3] = fminf(fmaxf(p[3], -1.f), 1.f);
}

// The whole ascent in one launch.  Templates are independent, so each block runs
// every step for its own: the template's thread 0 keeps the parameters and Adam's
// moments in registers and publishes (f0, f1, f2, tau) in shared memory for the
// next step's setup; a barrier ends each step.  step_consts[s] = (lr_f / (1 -
// 0.9^(s+1)), lr_u / (1 - 0.9^(s+1)), sqrt(1 - 0.999^(s+1))), from the host.
// hist (optional): [steps + 1][n] SNRs, row s before step s + 1, row steps after
// the last.
template <int WMODE, int PREC, int P>
__global__ void __launch_bounds__(kInterpBlock) refine_kernel(MapDev m, InterpConst k, float *__restrict__ f3,
                                                              float *__restrict__ tau, uint64_t n, int steps,
                                                              const float3 *__restrict__ step_consts, AdamStep ad,
                                                              float *__restrict__ hist)
{
    constexpr int TPB = kInterpBlock / P;
    __shared__ TplSetup su[TPB];
    __shared__ float par[TPB][4];  // f0, f1, f2, tau of each template's current step
    const int tl = threadIdx.x / P, t = threadIdx.x % P;
    const uint64_t i_raw = (uint64_t)blockIdx.x * TPB + tl;
    const bool valid = i_raw < n;
    const uint64_t i = valid ? i_raw : n - 1;  // the last block's spare slots repeat one, writing nothing
    float p[4] = {0.f, 0.f, 0.f, 0.f}, mo[4] = {0.f, 0.f, 0.f, 0.f}, ve[4] = {0.f, 0.f, 0.f, 0.f};
    if (t == 0) {
        const float tv = tau[i];
        p[0] = f3[3 * i];
        p[1] = f3[3 * i + 1];
        p[2] = f3[3 * i + 2];
        p[3] = tv / ad.tau_max;
        par[tl][0] = p[0];
        par[tl][1] = p[1];
        par[tl][2] = p[2];
        par[tl][3] = tv;
    }
    __syncthreads();
    auto params = [&](int sl, float &f0, float &f1, float &f2, float &tv) {
        f0 = par[sl][0];
        f1 = par[sl][1];
        f2 = par[sl][2];
        tv = par[sl][3];
    };
    float snr, gr[4];
    for (int s = 0; s < steps; ++s) {
        // the step's SNR (history row s), its gradient and the update
        setup_block<TPB>(k, m.n_f, su, params);
        if (interp_step<WMODE, PREC, true, P>(m, k, su[tl], t, 1.f, snr, gr)) {
            if (hist && valid) hist[(size_t)s * n + i] = snr;
            const float3 c = step_consts[s];
            AdamStep st = ad;
            st.step_f = c.x;
            st.step_u = c.y;
            st.sbc2 = c.z;
            const float gs[4] = {gr[0], gr[1], gr[2], gr[3] * ad.tau_max};  // dSNR/d(f0, f1, f2, u)
            adam_update(st, p, mo, ve, gs);
            par[tl][0] = p[0];
            par[tl][1] = p[1];
            par[tl][2] = p[2];
            par[tl][3] = p[3] * ad.tau_max;
        }
        __syncthreads();
    }
    if (t == 0 && valid && steps > 0) {
        f3[3 * i] = par[tl][0];
        f3[3 * i + 1] = par[tl][1];
        f3[3 * i + 2] = par[tl][2];
        tau[i] = par[tl][3];
    }
    if (!hist) return;
    setup_block<TPB>(k, m.n_f, su, params);
    if (interp_step<WMODE, PREC, false, P>(m, k, su[tl], t, 1.f, snr, gr) && valid)
        hist[(size_t)steps * n + i] = snr;
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
// fill the GPU when templates are few; with many, one warp each is fastest (50
// ascent steps on the 500 x 1600 map with history, ms, for 32 / 64 / 128 threads:
// 256 templates 0.47 / 0.30 / 0.23, 1024: 0.52 / 0.37 / 0.31, 2048: 0.56 / 0.66 /
// 0.57, 3072: 0.66 / 0.74 / 0.84, 4096: 0.73 / 1.00 / 1.09, 16384: 2.64 / 3.31 /
// 4.04).
int interp_threads(uint64_t n, int P)
{
    if (P == 32 || P == 64 || P == 128) return P;
    return n <= 1536 ? 128 : 32;
}

template <int MODE, int P>
cudaError_t launch_interp_P(const MapDev &m, const float *f3, const float *tau, const float *g, uint64_t n,
                            float *snr, float *gf3, float *gtau, int *err, cudaStream_t st)
{
    constexpr uint64_t TPB = kInterpBlock / P;
    const uint64_t blocks = (n + TPB - 1) / TPB;
    if (blocks > 0x7fffffffull) return cudaErrorInvalidValue;
    const unsigned b = (unsigned)blocks;
    const InterpConst k = interp_const(m, err);
#define STK_INTERP(W, PR) \
    interp_kernel<W, PR, MODE, P><<<b, kInterpBlock, 0, st>>>(m, k, f3, tau, g, n, snr, gf3, gtau)
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
                            float *snr, float *gf3, float *gtau, int P, int *err, cudaStream_t st)
{
    switch (interp_threads(n, P)) {
    case 128: return launch_interp_P<MODE, 128>(m, f3, tau, g, n, snr, gf3, gtau, err, st);
    case 64: return launch_interp_P<MODE, 64>(m, f3, tau, g, n, snr, gf3, gtau, err, st);
    default: return launch_interp_P<MODE, 32>(m, f3, tau, g, n, snr, gf3, gtau, err, st);
    }
}

// ------------------------------------------------------------------ discrete follow-up
// The refined continuous templates are judged by the discrete statistic (Eq. 7
// on whole pixels).  The polish climbs that statistic directly: the delay is set
// to the nearest maximum of SNR(tau) at the template's fixed pixels (W does not
// depend on tau; S(tau) = sum_j |z_j| cos(2 pi f_j tau + arg z_j) is smooth, so
// safeguarded Newton steps on S find it), then each control bin moves by +-1
// while a move, with its delay again maximised, raises the SNR.  One block a
// template: two groups of six warps climb from the start and from the
// alternative side by side, and within a group each warp tries one of the six
// moves (3 control bins x +-1), so a move costs one delay search instead of six.
// The climb compares warp sums (any summation order); the choice among the
// start, the polished start and the polished alternative uses the scorer's own
// sequential sum, so it never returns a template that scores below the start.
constexpr int kPolishWarps = 6;                       // a climb's warps: one per move
constexpr int kPolishBlock = 2 * kPolishWarps * 32;   // the two climbs
constexpr int kPolishNewton = 4;                      // Newton steps per delay search

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
// halved, twice).  One warp; returns the SNR at the returned delay.
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

struct PolishSlot {
    double tau;
    float snr;
};

// Barrier of one climb's six warps (named barrier 1 + group).
__device__ __forceinline__ void group_sync(int group)
{
    asm volatile("bar.sync %0, %1;" ::"r"(1 + group), "r"(kPolishWarps * 32) : "memory");
}

// Hill climb from (f, tau) by one group (warp gw of six): the delay first (warp
// 0), then rounds of the six +-1 moves, one a warp, each with its delay
// maximised; the first strictly best of them in the order (bin 0, -1), (bin 0,
// +1), (bin 1, -1), ... is taken while it beats the current SNR.  f and tau end
// the same in every thread of the group.
template <int WMODE, int PREC>
__device__ __forceinline__ void polish_climb(const MapDev &m, uint32_t f[3], double &tau, double tau_max, int moves,
                                             int group, int gw, int lane, PolishSlot *slot, int *err)
{
    if (gw == 0) {
        double t = tau;
        const float s = polish_delay<WMODE, PREC>(m, f, t, tau_max, lane, err);
        if (lane == 0) {
            slot[0].tau = t;
            slot[0].snr = s;
        }
    }
    group_sync(group);
    float snr = slot[0].snr;
    tau = slot[0].tau;
    group_sync(group);  // read before the slots are reused
    const int k = gw >> 1;
    const uint32_t d = (gw & 1) ? 1u : ~0u;  // +1 or -1 (selects below keep f and g in registers)
    for (int mv = 0; mv < moves; ++mv) {
        float sn = -INFINITY;
        double t = tau;
        const uint32_t fk = k == 0 ? f[0] : (k == 1 ? f[1] : f[2]);
        if (!((gw & 1) == 0 && fk == 0) && !((gw & 1) && fk + 1 >= (uint32_t)m.n_f)) {
            const uint32_t g[3] = {f[0] + (k == 0 ? d : 0u), f[1] + (k == 1 ? d : 0u), f[2] + (k == 2 ? d : 0u)};
            sn = polish_delay<WMODE, PREC>(m, g, t, tau_max, lane, err);
        }
        if (lane == 0) {
            slot[gw].tau = t;
            slot[gw].snr = sn;
        }
        group_sync(group);
        int best = -1;
        float bs = snr;
#pragma unroll
        for (int q = 0; q < kPolishWarps; ++q)
            if (slot[q].snr > bs) {
                bs = slot[q].snr;
                best = q;
            }
        const double bt = best >= 0 ? slot[best].tau : tau;
        group_sync(group);
        if (best < 0) break;
#pragma unroll
        for (int q = 0; q < 3; ++q) f[q] += (best >> 1) == q ? ((best & 1) ? 1u : ~0u) : 0u;
        tau = bt;
        snr = bs;
    }
}

// The scorer's SNR of one template, bit-identical to stk_score_explicit: the
// warp's lanes form the pixels' factors 32 columns at a time and every lane adds
// them in column order, as the scorer's single thread does.
template <int WMODE, int PREC>
__device__ __forceinline__ float polish_canonical(const MapDev &m, const uint32_t f[3], double tau, int lane, int *err)
{
    const Phase ph = phase_consts(m.f_min, m.df, tau, m.n_f);
    float acc = 0.f, W = 0.f;
    for (int j0 = 0; j0 < m.n_t; j0 += 32) {
        const int j = j0 + lane;
        float mg = 0.f, c = 0.f, wv = 0.f;
        if (j < m.n_t) {
            uint32_t b = raster_bin_wide(f[0], f[1], f[2], m.M, (uint32_t)j, m.d);
            if (kDebugBounds) b = checked_bin(b, j, m.n_t, hull_lo(f), hull_hi(f), err);
            const typename Pix<PREC>::Rec v = Pix<PREC>::load_global(m.rec, (size_t)j * m.ldr + b);
            if (WMODE == WMODE_FREQ) wv = __ldg(m.w + b);
            if (WMODE == WMODE_PIXEL) wv = __ldg(m.w + (size_t)j * m.ldw + b);
            pixel_term<PREC, WMODE>(v, template_turn(b, ph), wv, mg, c);
        }
        const int cnt = min(32, m.n_t - j0);
        for (int q = 0; q < cnt; ++q)
            pixel_sum<PREC, WMODE>(__shfl_sync(0xffffffffu, mg, q), __shfl_sync(0xffffffffu, c, q),
                                   __shfl_sync(0xffffffffu, wv, q), acc, W);
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
    __shared__ PolishSlot slots[2][kPolishWarps];
    __shared__ uint32_t cf[3][3];   // candidates: start, polished start, polished alternative
    __shared__ double ct[3];
    __shared__ float cs[3];
    const uint64_t i = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int group = warp / kPolishWarps, gw = warp % kPolishWarps;
    const uint32_t fs[3] = {min(f3[3 * i], (uint32_t)m.n_f - 1), min(f3[3 * i + 1], (uint32_t)m.n_f - 1),
                            min(f3[3 * i + 2], (uint32_t)m.n_f - 1)};
    const double ts = tau[i];
    const double ts_c = fmin(fmax(ts, -tau_max), tau_max);
    if (group == 0 || alt_f3) {
        uint32_t f[3] = {fs[0], fs[1], fs[2]};
        double t = ts_c;
        if (group == 1) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float x = alt_f3[3 * i + k];
                f[k] = (uint32_t)rintf(fminf(fmaxf(x == x ? x : 0.f, 0.f), (float)(m.n_f - 1)));
            }
            const double ta = (double)alt_tau[i];
            if (ta == ta) t = fmin(fmax(ta, -tau_max), tau_max);   // NaN: the start's delay
        }
        polish_climb<WMODE, PREC>(m, f, t, tau_max, moves, group, gw, lane, slots[group], err);
        if (gw == 0 && lane == 0) {
            cf[1 + group][0] = f[0];
            cf[1 + group][1] = f[1];
            cf[1 + group][2] = f[2];
            ct[1 + group] = t;
        }
    }
    if (threadIdx.x == 0) {
        cf[0][0] = fs[0];
        cf[0][1] = fs[1];
        cf[0][2] = fs[2];
        ct[0] = ts;
    }
    __syncthreads();
    // the choice, by the scorer's own sums: the start unless a polished form beats it
    const int nc = alt_f3 ? 3 : 2;
    if (warp < nc) {
        const float s = polish_canonical<WMODE, PREC>(m, cf[warp], ct[warp], lane, err);
        if (lane == 0) cs[warp] = s;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    int w = 0;
    float best = cs[0];
    if (cs[1] > best) { w = 1; best = cs[1]; }
    if (alt_f3 && cs[2] > best) { w = 2; best = cs[2]; }
    f3[3 * i] = cf[w][0];
    f3[3 * i + 1] = cf[w][1];
    f3[3 * i + 2] = cf[w][2];
    tau[i] = ct[w];
    if (snr_out) snr_out[i] = (double)best;
    if (which_out) which_out[i] = w;
}

}  // namespace

size_t refine_scratch_bytes(int steps)
{
    return (size_t)(steps > 0 ? steps : 1) * sizeof(float3);  // the steps' step sizes
}

namespace {

template <int P>
cudaError_t launch_refine_P(const MapDev &m, float *f3, float *tau, uint64_t n, int steps, const float3 *consts,
                            const AdamStep &ad, float *hist, int *err, cudaStream_t st)
{
    constexpr uint64_t TPB = kInterpBlock / P;
    const uint64_t blocks = (n + TPB - 1) / TPB;
    if (blocks > 0x7fffffffull) return cudaErrorInvalidValue;
    const unsigned b = (unsigned)blocks;
    const InterpConst k = interp_const(m, err);
#define STK_REFINE(W, PR) \
    refine_kernel<W, PR, P><<<b, kInterpBlock, 0, st>>>(m, k, f3, tau, n, steps, consts, ad, hist)
    if (m.prec == PREC_FP16) {
        if (m.wmode == WMODE_CONST) STK_REFINE(WMODE_CONST, PREC_FP16);
        else if (m.wmode == WMODE_FREQ) STK_REFINE(WMODE_FREQ, PREC_FP16);
        else STK_REFINE(WMODE_PIXEL, PREC_FP16);
    } else {
        if (m.wmode == WMODE_CONST) STK_REFINE(WMODE_CONST, PREC_FP32);
        else if (m.wmode == WMODE_FREQ) STK_REFINE(WMODE_FREQ, PREC_FP32);
        else STK_REFINE(WMODE_PIXEL, PREC_FP32);
    }
#undef STK_REFINE
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_refine(const MapDev &m, float *f3, float *tau, uint64_t n, int steps, float lr_f, float lr_u,
                          float tau_max, float *hist, void *scratch, int P, int *err, cudaStream_t st)
{
    if (n == 0 || steps < 0) return cudaSuccess;
    AdamStep ad{};
    ad.tau_max = tau_max;
    ad.f_hi = (float)(m.n_f - 1);
    float3 *consts = static_cast<float3 *>(scratch);
    if (steps > 0) {
        // bias-corrected step sizes of every step, in FP64 on the host (Adam, betas 0.9 and 0.999)
        std::vector<float3> hc((size_t)steps);
        for (int t = 1; t <= steps; ++t) {
            const double bc1 = 1.0 - std::pow(0.9, t), bc2 = 1.0 - std::pow(0.999, t);
            hc[t - 1] = make_float3((float)(lr_f / bc1), (float)(lr_u / bc1), (float)std::sqrt(bc2));
        }
        // pageable source: the call returns once the data are staged
        const cudaError_t e = cudaMemcpyAsync(consts, hc.data(), sizeof(float3) * (size_t)steps,
                                              cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;
    }
    switch (interp_threads(n, P)) {
    case 128: return launch_refine_P<128>(m, f3, tau, n, steps, consts, ad, hist, err, st);
    case 64: return launch_refine_P<64>(m, f3, tau, n, steps, consts, ad, hist, err, st);
    default: return launch_refine_P<32>(m, f3, tau, n, steps, consts, ad, hist, err, st);
    }
}

cudaError_t launch_interp_tuned(const MapDev &m, const float *f3, const float *tau, const float *g, uint64_t n,
                                float *snr, float *gf3, float *gtau, bool adjoint, int P, int *err, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    return adjoint ? launch_interp_M<1>(m, f3, tau, g, n, snr, gf3, gtau, P, err, st)
                   : launch_interp_M<0>(m, f3, tau, g, n, snr, gf3, gtau, P, err, st);
}

cudaError_t launch_polish(const MapDev &m, uint32_t *f3, double *tau, const float *alt_f3, const float *alt_tau,
                          uint64_t n, double tau_max, int moves, double *snr, int *which, int *err, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    if (n > 0x7fffffffull) return cudaErrorInvalidValue;
    const unsigned b = (unsigned)n;  // one block a template
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
