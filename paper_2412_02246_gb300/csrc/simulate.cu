// Visibility simulator (Sec. 3): the flat-sky map times the primary beam
// (Eq. beam, the MWA tile's sinc^2 pattern, or Eq. A_G, its Gaussian
// approximation), then the direct DFT of Eq. vis at every baseline, with
// Q = 1 (visibilities in map units):
//
//   V(U) = sum over pixels of dtheta^2 A(theta) T(theta) exp(+i 2 pi U.theta),
//   pixel (row b, column a) at theta = ((a - m/2) dtheta, (b - m/2) dtheta).
//
// One thread per visibility; the weighted map is staged through shared memory
// in tiles that every thread of the block walks in the same order.  The phase
// U.theta is formed in FP64 and reduced to its fractional cycle before the
// FP32 sine and cosine (baselines of hundreds of wavelengths times angles of
// a radian are hundreds of cycles), and the FP32 terms are folded into FP64
// sums every 64 pixels.
#include "abs_internal.cuh"

namespace absk {
namespace {

constexpr int SIM_T = 256;       // visibilities per CTA
constexpr int SIM_TILE = 4096;   // map pixels staged per pass
constexpr int SIM_FOLD = 64;

__global__ void k_sky_weights(int m, double dth, const float *__restrict__ sky, int beam, double bp,
                              float *__restrict__ W) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (int64_t)m * m) return;
    const int b = (int)(p / m), a = (int)(p - (int64_t)b * m);
    const double tx = (a - m / 2) * dth, ty = (b - m / 2) * dth;
    double A = 1.0;
    if (beam == ABS_BEAM_MWA_TILE) {
        const double x = bp * tx, y = bp * ty;   // sinc(x) = sin(pi x) / (pi x)
        const double sx = x == 0.0 ? 1.0 : sinpi(x) / (M_PI * x);
        const double sy = y == 0.0 ? 1.0 : sinpi(y) / (M_PI * y);
        A = sx * sx * sy * sy;
    } else if (beam == ABS_BEAM_GAUSS) {
        A = exp(-(tx * tx + ty * ty) / (bp * bp));
    }
    W[p] = (float)(dth * dth * A * (double)sky[p]);
}

__global__ void __launch_bounds__(SIM_T) k_dft(int m, double dth, const float *__restrict__ W, int64_t n_vis,
                                               const float2 *__restrict__ uv, float2 *__restrict__ vis) {
    __shared__ float ws[SIM_TILE];
    const int64_t e = (int64_t)blockIdx.x * SIM_T + threadIdx.x;
    const bool on = e < n_vis;
    const float2 U = on ? uv[e] : make_float2(0.f, 0.f);
    const double u = U.x, v = U.y, th0 = -(m / 2) * dth;
    const int64_t npix = (int64_t)m * m;
    double re = 0.0, im = 0.0;
    float fr = 0.f, fi = 0.f;
    int a = 0, b = 0, nf = 0;
    double vy = v * (th0 + b * dth);
    for (int64_t p0 = 0; p0 < npix; p0 += SIM_TILE) {
        const int np = (int)min((int64_t)SIM_TILE, npix - p0);
        __syncthreads();
        for (int i = threadIdx.x; i < np; i += SIM_T) ws[i] = W[p0 + i];
        __syncthreads();
        for (int i = 0; i < np; ++i) {
            const double ph = fma(u, th0 + a * dth, vy);      // cycles
            const float f = (float)(2.0 * (ph - rint(ph)));
            float s, c;
            sincospif(f, &s, &c);
            const float w = ws[i];
            fr = fmaf(w, c, fr);
            fi = fmaf(w, s, fi);
            if (++nf == SIM_FOLD) {
                re += fr;
                im += fi;
                fr = fi = 0.f;
                nf = 0;
            }
            if (++a == m) {
                a = 0;
                ++b;
                vy = v * (th0 + b * dth);
            }
        }
    }
    re += fr;
    im += fi;
    if (on) vis[e] = make_float2((float)re, (float)im);
}

}  // namespace

abs_status launch_simulate_vis(abs_ctx *ctx, int32_t m, double dtheta, const float *d_sky, int32_t beam,
                               double beam_param, int64_t n_vis, const float *d_uv, float *d_vis) {
    const int64_t npix = (int64_t)m * m;
    float *W = (float *)workspace(ctx, "sim.weights", sizeof(float) * (size_t)npix);
    if (!W) return fail(ctx, ABS_ERR_OOM, "simulator workspace");
    StageTimer timer(ctx, "simulate_vis");
    k_sky_weights<<<(unsigned)cdiv(npix, 256), 256, 0, ctx->stream>>>(m, dtheta, d_sky, beam, beam_param, W);
    if (n_vis > 0)
        k_dft<<<(unsigned)cdiv(n_vis, SIM_T), SIM_T, 0, ctx->stream>>>(m, dtheta, W, n_vis, (const float2 *)d_uv,
                                                                       (float2 *)d_vis);
    return check_launch(ctx, "visibility simulator");
}

}  // namespace absk
