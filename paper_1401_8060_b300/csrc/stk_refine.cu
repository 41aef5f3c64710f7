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
// One thread per template.  Sums and the pixel arithmetic are FP32; the curve
// position x_j and the phase argument are FP64, since FP32 resolves x_j ~ 10^3
// only to 6e-5 bins.
#include <cuda_fp16.h>

#include "stk_internal.cuh"
#include "stk_pixel.cuh"

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
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double f0 = f3[3 * i], f1 = f3[3 * i + 1], f2 = f3[3 * i + 2];
    const double tau = tau_in[i];
    const int n_t = m.n_t, n_f = m.n_f;
    const double M = (double)(n_t - 1), inv_M2 = 1.0 / (M * M);
    const double a2 = f0 - 2.0 * f1 + f2, a1 = 2.0 * M * (f1 - f0), a0 = M * M * f0;
    const double fa = m.df * tau, fb = m.f_min * tau;      // turns per bin, turns at bin 0
    const float two_pi = 6.28318530717958647692f;
    float S = 0.f, W = 0.f;
    float dS0 = 0.f, dS1 = 0.f, dS2 = 0.f, dS3 = 0.f, dW0 = 0.f, dW1 = 0.f, dW2 = 0.f;
    for (int j = 0; j < n_t; ++j) {
        const double jd = (double)j;
        double x = ((a2 * jd + a1) * jd + a0) * inv_M2;
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
            const float u = (float)(jd / M), c0 = (1.f - u) * (1.f - u), c1 = 2.f * (1.f - u) * u, c2 = u * u;
            dS0 = fmaf(dre_dx, c0, dS0);
            dS1 = fmaf(dre_dx, c1, dS1);
            dS2 = fmaf(dre_dx, c2, dS2);
            dW0 = fmaf(dw_dx, c0, dW0);
            dW1 = fmaf(dw_dx, c1, dW1);
            dW2 = fmaf(dw_dx, c2, dW2);
            dS3 = fmaf(-im, two_pi * (float)(m.f_min + x * m.df), dS3);
        }
    }
    const bool varying = WMODE != WMODE_CONST && !m.paper;
    const float scale = varying ? rsqrtf(W) : (float)m.norm;
    if (!ADJOINT) {
        snr_out[i] = S * scale;
        return;
    }
    const float gi = g[i];
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
    const int threads = 128;
    const uint64_t blocks = (n + threads - 1) / threads;
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

}  // namespace

cudaError_t launch_interp(const MapDev &m, const float *f3, const float *tau, const float *g, uint64_t n, float *snr,
                          float *gf3, float *gtau, bool adjoint, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    return adjoint ? launch_interp_A<true>(m, f3, tau, g, n, snr, gf3, gtau, st)
                   : launch_interp_A<false>(m, f3, tau, g, n, snr, gf3, gtau, st);
}

}  // namespace stk
