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
// U.theta (hundreds of cycles for baselines of hundreds of wavelengths over a
// radian) is carried as a double-float pair and reduced to its fractional
// cycle before the FP32 sine and cosine (the SFU's), at the start of every run
// of 16 pixels of a row; the run's other terms are rotated by one column's
// phase (sine and cosine to a few ulp).
// The FP32 terms are folded into double-float sums every 64 pixels.
#include "abs_internal.cuh"

namespace absk {
namespace {

constexpr int SIM_T = 256;       // visibilities per CTA
constexpr int SIM_TILE = 4096;   // map pixels staged per pass
constexpr int SIM_FOLD = 64;     // pixels summed in FP32 before each double-float fold

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

// x + y for double-float pairs (hi, lo): TwoSum of the high parts, low parts added.
__device__ __forceinline__ void df_add(float xh, float xl, float yh, float yl, float &zh, float &zl) {
    const float s = __fadd_rn(xh, yh);
    const float bp = __fsub_rn(s, xh);
    const float e = __fadd_rn(__fsub_rn(xh, __fsub_rn(s, bp)), __fsub_rn(yh, bp));
    const float t = __fadd_rn(e, __fadd_rn(xl, yl));
    zh = __fadd_rn(s, t);
    zl = __fsub_rn(t, __fsub_rn(zh, s));
}

// k x (hi, lo) for a small integer k, as a double-float pair.
__device__ __forceinline__ void df_scale(float h, float l, float k, float &zh, float &zl) {
    const float p = __fmul_rn(h, k);
    const float e = fmaf(h, k, -p);
    const float t = fmaf(l, k, e);
    zh = __fadd_rn(p, t);
    zl = __fsub_rn(t, __fsub_rn(zh, p));
}

// exp(i 2 pi phi) for a double-float phase phi in cycles, from its fractional cycle f
// (|f| <= 1/2).  fast: the SFU's __sincosf of 2 pi f (absolute error about 4e-7 over
// [-pi, pi]); else sincospif (a few ulp, but slow here: it keeps the FP64 pipe busy).
__device__ __forceinline__ float2 cis_cycles(float h, float l, bool fast) {
    const float f = __fadd_rn(__fsub_rn(h, rintf(h)), l);
    float s, c;
    if (fast) __sincosf(6.28318531f * f, &s, &c);
    else sincospif(2.0f * f, &s, &c);
    return make_float2(c, s);
}

// The phase u theta_x(a) + v theta_y(b) in cycles is exact (double-float) at the
// first pixel of every run of SIM_RUN in a row; in between, the term is rotated
// by exp(i 2 pi u dtheta) (a complex multiply), so a run's rounding drift is a
// few units in the last place.
constexpr int SIM_RUN = 16;

__global__ void __launch_bounds__(SIM_T) k_dft(int m, double dth, const float *__restrict__ W, int64_t n_vis,
                                               const float2 *__restrict__ uv, float2 *__restrict__ vis) {
    __shared__ float ws[SIM_TILE];
    const int64_t e = (int64_t)blockIdx.x * SIM_T + threadIdx.x;
    const bool on = e < n_vis;
    const float2 U = on ? uv[e] : make_float2(0.f, 0.f);
    // u dtheta and v dtheta as double-float pairs (from the FP64 products), and the phase
    // of pixel (0, 0): (u + v) theta_0
    const double th0 = -(double)(m / 2) * dth;
    const double cu = (double)U.x * dth, cv = (double)U.y * dth, c0 = ((double)U.x + (double)U.y) * th0;
    const float cuh = (float)cu, cul = (float)(cu - (double)cuh);
    const float cvh = (float)cv, cvl = (float)(cv - (double)cvh);
    float rh = (float)c0, rl = (float)(c0 - (double)rh);   // the row's phase at a = 0
    const float2 w = cis_cycles(cuh, cul, false);          // one column's rotation (accurate: it compounds)
    const int64_t npix = (int64_t)m * m;
    float reh = 0.f, rel = 0.f, imh = 0.f, iml = 0.f;   // double-float sums of the folded blocks
    float fr = 0.f, fi = 0.f;
    float2 z = make_float2(1.f, 0.f);
    int a = 0, nf = 0;
    for (int64_t p0 = 0; p0 < npix; p0 += SIM_TILE) {
        const int np = (int)min((int64_t)SIM_TILE, npix - p0);
        __syncthreads();
        for (int i = threadIdx.x; i < np; i += SIM_T) ws[i] = W[p0 + i];
        __syncthreads();
        for (int i = 0; i < np; ++i) {
            if (a % SIM_RUN == 0) {
                float ph, pl, qh, ql;
                df_scale(cuh, cul, (float)a, ph, pl);
                df_add(rh, rl, ph, pl, qh, ql);
                z = cis_cycles(qh, ql, true);
            } else {
                z = make_float2(fmaf(z.x, w.x, -z.y * w.y), fmaf(z.x, w.y, z.y * w.x));
            }
            const float wt = ws[i];
            fr = fmaf(wt, z.x, fr);
            fi = fmaf(wt, z.y, fi);
            if (++nf == SIM_FOLD) {
                df_add(reh, rel, fr, 0.f, reh, rel);
                df_add(imh, iml, fi, 0.f, imh, iml);
                fr = fi = 0.f;
                nf = 0;
            }
            if (++a == m) {
                a = 0;
                df_add(rh, rl, cvh, cvl, rh, rl);
            }
        }
    }
    df_add(reh, rel, fr, 0.f, reh, rel);
    df_add(imh, iml, fi, 0.f, imh, iml);
    if (on) vis[e] = make_float2(__fadd_rn(reh, rel), __fadd_rn(imh, iml));
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
