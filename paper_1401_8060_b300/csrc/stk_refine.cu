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
// One warp per template: lane l takes the columns j = l (mod 32) in order, then
// the lanes' partial sums meet in a fixed shuffle tree (deterministic).  Sums and
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
    const float ang = (float)(int32_t)Pix<PREC>::arg(v) * 1.4629180792671596e-09f;  // 2 pi / 2^32
    float s, c;
    __sincosf(ang, &s, &c);
    zr = mag * c;
    zi = mag * s;
    w = wv;
}

template <int WMODE, int PREC, bool ADJOINT>
__global__ void __launch_bounds__(128) interp_kernel(MapDev m, const float *__restrict__ f3,
                                                     const float *__restrict__ tau_in, const float *__restrict__ g,
                                                     uint64_t n, float *__restrict__ snr_out,
                                                     float *__restrict__ gf3, float *__restrict__ gtau)
{
    const uint64_t i = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;  // the same for a whole warp
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const double f0 = f3[3 * i], f1 = f3[3 * i + 1], f2 = f3[3 * i + 2];
    const double tau = tau_in[i];
    const int n_t = m.n_t, n_f = m.n_f;
    const double M = (double)(n_t - 1), inv_M2 = 1.0 / (M * M);
    const double a2 = f0 - 2.0 * f1 + f2, a1 = 2.0 * M * (f1 - f0), a0 = M * M * f0;
    const double fa = m.df * tau, fb = m.f_min * tau;      // turns per bin, turns at bin 0
    const float two_pi = 6.28318530717958647692f;
    const float inv_Mf = 1.f / (float)M, df_f = (float)m.df, fmin_f = (float)m.f_min;
    // x_j by forward differences along the lane's columns j, j + 32, ...: two FP64
    // additions a column (the quadratic's second difference is constant)
    const double jl = (double)lane;
    double x_next = ((a2 * jl + a1) * jl + a0) * inv_M2;
    double dx = (a2 * (64.0 * jl + 1024.0) + 32.0 * a1) * inv_M2;
    const double ddx = 2048.0 * a2 * inv_M2;
    float S = 0.f, W = 0.f;
    float dS0 = 0.f, dS1 = 0.f, dS2 = 0.f, dS3 = 0.f, dW0 = 0.f, dW1 = 0.f, dW2 = 0.f;
    for (int j = lane; j < n_t; j += 32) {
        double x = x_next;
        x_next += dx;
        dx += ddx;
        bool clamped = false;
        if (x < 0.0) { x = 0.0; clamped = true; }
        if (x > (double)(n_f - 1)) { x = (double)(n_f - 1); clamped = true; }
        int k = (int)floor(x);
        if (k > n_f - 2) k = n_f - 2;
        if (k < 0) k = 0;
        const float a = n_f > 1 ? (float)(x - (double)k) : 0.f;
        float z0r, z0i, w0, z1r, z1i, w1;
        pixel_at<WMODE, PREC>(m, j, k, z0r, z0i, w0);
        if (n_f > 1) pixel_at<WMODE, PREC>(m, j, k + 1, z1r, z1i, w1);
        else { z1r = z0r; z1i = z0i; w1 = w0; }
        const float dzr = z1r - z0r, dzi = z1i - z0i, dw = w1 - w0;
        const float zr = fmaf(a, dzr, z0r), zi = fmaf(a, dzi, z0i), w = fmaf(a, dw, w0);
        double turns = fb + x * fa;
        turns -= rint(turns);                                // [-1/2, 1/2]
        float s, c;
        __sincosf(two_pi * (float)turns, &s, &c);
        const float re = c * zr - s * zi, im = s * zr + c * zi;
        S += re;
        W += w;
        if (ADJOINT) {
            // d re/dx = -im 2 pi df tau + Re[e^{i phi} dz/dx]; d re/dtau = -im 2 pi f
            const float dre_dx = clamped ? 0.f : fmaf(-im, two_pi * (float)fa, c * dzr - s * dzi);
            const float dw_dx = clamped ? 0.f : dw;
            const float u = (float)j * inv_Mf, c0 = (1.f - u) * (1.f - u), c1 = 2.f * (1.f - u) * u, c2 = u * u;
            dS0 = fmaf(dre_dx, c0, dS0);
            dS1 = fmaf(dre_dx, c1, dS1);
            dS2 = fmaf(dre_dx, c2, dS2);
            dW0 = fmaf(dw_dx, c0, dW0);
            dW1 = fmaf(dw_dx, c1, dW1);
            dW2 = fmaf(dw_dx, c2, dW2);
            dS3 = fmaf(-im, two_pi * fmaf((float)x, df_f, fmin_f), dS3);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        S += __shfl_xor_sync(0xffffffffu, S, o);
        W += __shfl_xor_sync(0xffffffffu, W, o);
        if (ADJOINT) {
            dS0 += __shfl_xor_sync(0xffffffffu, dS0, o);
            dS1 += __shfl_xor_sync(0xffffffffu, dS1, o);
            dS2 += __shfl_xor_sync(0xffffffffu, dS2, o);
            dS3 += __shfl_xor_sync(0xffffffffu, dS3, o);
            dW0 += __shfl_xor_sync(0xffffffffu, dW0, o);
            dW1 += __shfl_xor_sync(0xffffffffu, dW1, o);
            dW2 += __shfl_xor_sync(0xffffffffu, dW2, o);
        }
    }
    if (lane != 0) return;
    const bool varying = WMODE != WMODE_CONST && !m.paper;
    const float scale = varying ? rsqrtf(W) : (float)m.norm;
    if (!ADJOINT || snr_out) snr_out[i] = S * scale;
    if (!ADJOINT) return;
    const float gi = g ? g[i] : 1.f;
    if (varying) {
        const float h = 0.5f * S * scale * scale * scale;
        gf3[3 * i] = gi * (dS0 * scale - h * dW0);
        gf3[3 * i + 1] = gi * (dS1 * scale - h * dW1);
        gf3[3 * i + 2] = gi * (dS2 * scale - h * dW2);
    } else {
        gf3[3 * i] = gi * dS0 * scale;
        gf3[3 * i + 1] = gi * dS1 * scale;
        gf3[3 * i + 2] = gi * dS2 * scale;
    }
    gtau[i] = gi * dS3 * scale;
}

template <bool ADJ>
cudaError_t launch_interp_A(const MapDev &m, const float *f3, const float *tau, const float *g, uint64_t n,
                            float *snr, float *gf3, float *gtau, cudaStream_t st)
{
    const int threads = 128;                                  // 4 templates (warps) per block
    const uint64_t blocks = (n * 32 + threads - 1) / threads;
    if (blocks > 0x7fffffffull) return cudaErrorInvalidValue;
    const unsigned b = (unsigned)blocks;
#define STK_INTERP(W, P) interp_kernel<W, P, ADJ><<<b, threads, 0, st>>>(m, f3, tau, g, n, snr, gf3, gtau)
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

// One Adam step of the gradient ascent of every template's SNR (Adam with betas
// 0.9, 0.999 and eps 1e-8 on the loss -SNR, in torch's arithmetic order), then the
// projection onto f in [0, n_f - 1] and |u| <= 1, u = tau / tau_max.  st[2i] and
// st[2i+1] hold the first and second moments of (f0, f1, f2, u).  The bias
// corrections come from the host: step_f = lr_f / (1 - 0.9^t), step_u likewise,
// sbc2 = sqrt(1 - 0.999^t).
__global__ void __launch_bounds__(256) adam_kernel(float *__restrict__ f3, float *__restrict__ u,
                                                   float *__restrict__ tau, const float *__restrict__ gf3,
                                                   const float *__restrict__ gtau, float4 *__restrict__ st,
                                                   uint64_t n, float step_f, float step_u, float sbc2,
                                                   float tau_max, float f_hi)
{
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float w1 = 0.1f, b2 = 0.999f, w2 = 0.001f, eps = 1e-8f;
    float4 m = st[2 * i], v = st[2 * i + 1];
    const float g[4] = {-gf3[3 * i], -gf3[3 * i + 1], -gf3[3 * i + 2], -gtau[i] * tau_max};  // d(-SNR)/d(f, u)
    float p[4] = {f3[3 * i], f3[3 * i + 1], f3[3 * i + 2], u[i]};
    float *mm = &m.x, *vv = &v.x;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        mm[q] = mm[q] + w1 * (g[q] - mm[q]);
        vv[q] = vv[q] * b2 + w2 * g[q] * g[q];
        const float denom = __fsqrt_rn(vv[q]) / sbc2 + eps;
        p[q] = p[q] - (q < 3 ? step_f : step_u) * (mm[q] / denom);
    }
    st[2 * i] = m;
    st[2 * i + 1] = v;
#pragma unroll
    for (int q = 0; q < 3; ++q) f3[3 * i + q] = fminf(fmaxf(p[q], 0.f), f_hi);
    const float uu = fminf(fmaxf(p[3], -1.f), 1.f);
    u[i] = uu;
    tau[i] = uu * tau_max;
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
    return (size_t)n * (sizeof(float4) * 2 + sizeof(float) * 5);  // moments, u, gradients (f3, tau)
}

cudaError_t launch_refine(const MapDev &m, float *f3, float *tau, uint64_t n, int steps, float lr_f, float lr_u,
                          float tau_max, float *hist, void *scratch, cudaStream_t st)
{
    if (n == 0 || steps < 0) return cudaSuccess;
    float4 *mom = static_cast<float4 *>(scratch);
    float *u = reinterpret_cast<float *>(mom + 2 * n), *gf3 = u + n, *gtau = gf3 + 3 * n;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    refine_init_kernel<<<blocks, 256, 0, st>>>(tau, u, mom, n, tau_max);
    cudaError_t e = cudaGetLastError();
    const float f_hi = (float)(m.n_f - 1);
    for (int t = 1; t <= steps && e == cudaSuccess; ++t) {
        // the step's SNR (history row t - 1) and its gradient, then the update
        e = launch_interp(m, f3, tau, nullptr, n, hist ? hist + (size_t)(t - 1) * n : nullptr, gf3, gtau, true, st);
        if (e != cudaSuccess) break;
        const double bc1 = 1.0 - std::pow(0.9, t), bc2 = 1.0 - std::pow(0.999, t);
        adam_kernel<<<blocks, 256, 0, st>>>(f3, u, tau, gf3, gtau, mom, n, (float)(lr_f / bc1), (float)(lr_u / bc1),
                                            (float)std::sqrt(bc2), tau_max, f_hi);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && hist)
        e = launch_interp(m, f3, tau, nullptr, n, hist + (size_t)steps * n, nullptr, nullptr, false, st);
    return e;
}

cudaError_t launch_interp(const MapDev &m, const float *f3, const float *tau, const float *g, uint64_t n, float *snr,
                          float *gf3, float *gtau, bool adjoint, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    return adjoint ? launch_interp_A<true>(m, f3, tau, g, n, snr, gf3, gtau, st)
                   : launch_interp_A<false>(m, f3, tau, g, n, snr, gf3, gtau, st);
}

}  // namespace stk
