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
__device__ __forceinline__ void pixel_at(const MapDev &m, int j, int k, float &zr, float &zi, float &w)
{
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
        pixel_at<WMODE, PREC>(m, j, kb, z0r, z0i, w0);
        if (n_f > 1) pixel_at<WMODE, PREC>(m, j, kb + 1, z1r, z1i, w1);
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
    const float scale = varying ? rsqrtf(W) : (float)m.norm;
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

InterpConst interp_const(const MapDev &m)
{
    InterpConst k;
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
                            float *snr, float *gf3, float *gtau, const AdamStep &ad, cudaStream_t st)
{
    constexpr uint64_t TPB = kInterpBlock / P;
    const uint64_t blocks = (n + TPB - 1) / TPB;
    if (blocks > 0x7fffffffull) return cudaErrorInvalidValue;
    const unsigned b = (unsigned)blocks;
    const InterpConst k = interp_const(m);
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
                            float *snr, float *gf3, float *gtau, const AdamStep &ad, int P, cudaStream_t st)
{
    switch (interp_threads(n, P)) {
    case 128: return launch_interp_P<MODE, 128>(m, f3, tau, g, n, snr, gf3, gtau, ad, st);
    case 64: return launch_interp_P<MODE, 64>(m, f3, tau, g, n, snr, gf3, gtau, ad, st);
    default: return launch_interp_P<MODE, 32>(m, f3, tau, g, n, snr, gf3, gtau, ad, st);
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

}  // namespace

size_t refine_scratch_bytes(uint64_t n)
{
    return (size_t)n * (sizeof(float4) * 2 + sizeof(float));  // moments, u
}

cudaError_t launch_refine(const MapDev &m, float *f3, float *tau, uint64_t n, int steps, float lr_f, float lr_u,
                          float tau_max, float *hist, void *scratch, int P, cudaStream_t st)
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
                               nullptr, ad, P, st);
    }
    if (e == cudaSuccess && hist)
        e = launch_interp_M<0>(m, f3, tau, nullptr, n, hist + (size_t)steps * n, nullptr, nullptr, AdamStep{}, P,
                               st);
    return e;
}

cudaError_t launch_interp_tuned(const MapDev &m, const float *f3, const float *tau, const float *g, uint64_t n,
                                float *snr, float *gf3, float *gtau, bool adjoint, int P, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    return adjoint ? launch_interp_M<1>(m, f3, tau, g, n, snr, gf3, gtau, AdamStep{}, P, st)
                   : launch_interp_M<0>(m, f3, tau, g, n, snr, gf3, gtau, AdamStep{}, P, st);
}

cudaError_t launch_interp(const MapDev &m, const float *f3, const float *tau, const float *g, uint64_t n, float *snr,
                          float *gf3, float *gtau, bool adjoint, cudaStream_t st)
{
    return launch_interp_tuned(m, f3, tau, g, n, snr, gf3, gtau, adjoint, 0, st);
}

}  // namespace stk
