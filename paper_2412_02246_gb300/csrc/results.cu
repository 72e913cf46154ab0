// Results layer (Sec. 4): the binned bispectrum in the (l1, mu, t) shape form
// and its ensemble statistics over realisations.
//
// A canonical triplet (i <= j <= k, rings ascending in l) is the paper's
// l1 >= l2 >= l3 as (k, j, i), each side its ring's mean l.  Its shape is
// mu = (l1^2 + l2^2 - l3^2) / (2 l1 l2) and t = l2 / l1 (both in [0.5, 1] for
// closed triangles), computed with correctly rounded, unfused FP64 operations
// in that order, so that the bin decision is reproducible.  A cell is
// (ring of l1, mu bin, t bin) with equal bins over [0.5, 1] (shapes just
// outside, from ring means, clamped to the edge bins).  Per realisation r:
// B_r(c) = sum T B_r / sum T over the cell's triplets with T > 0 and finite B;
// over realisations: mean and sigma^2 = <B_r(c)^2> - mean^2.  The sums use
// FP64 atomics (their order, and so the last bits, may vary run to run).
#include "abs_internal.cuh"

namespace absk {
namespace {

__device__ __forceinline__ int shape_bin(double x, int n) {
    const double v = floor(__dmul_rn(__dsub_rn(x, 0.5), 2.0 * (double)n));
    if (!isfinite(v) || v < 0.0) return 0;
    return v > (double)(n - 1) ? n - 1 : (int)v;
}

__global__ void k_rebin_accum(int n_real, int n_trip, int nb, int n_mu, int n_t, const double *__restrict__ B,
                              const int64_t *__restrict__ T, const double *__restrict__ ellbar,
                              const int32_t *__restrict__ ijk, double *__restrict__ num, double *__restrict__ den) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n_real * n_trip) return;
    const int r = (int)(e / n_trip), q = (int)(e - (int64_t)r * n_trip);
    const int64_t w = T[q];
    const double b = B[(size_t)r * n_trip + q];
    if (w <= 0 || !isfinite(b)) return;
    const int i = ijk[3 * q], j = ijk[3 * q + 1], k = ijk[3 * q + 2];
    if (i < 0 || j < i || k < j || k >= nb) return;
    const double l3 = ellbar[i], l2 = ellbar[j], l1 = ellbar[k];
    const double mu = __ddiv_rn(__dsub_rn(__dadd_rn(__dmul_rn(l1, l1), __dmul_rn(l2, l2)), __dmul_rn(l3, l3)),
                                __dmul_rn(__dmul_rn(2.0, l1), l2));
    const double t = __ddiv_rn(l2, l1);
    const int c = (k * n_mu + shape_bin(mu, n_mu)) * n_t + shape_bin(t, n_t);
    const int cells = nb * n_mu * n_t;
    atomicAdd(&num[(size_t)r * cells + c], (double)w * b);
    if (r == 0) atomicAdd(&den[c], (double)w);
}

__global__ void k_rebin_finish(int n_real, int cells, const double *__restrict__ num, const double *__restrict__ den,
                               double *__restrict__ mean, double *__restrict__ sigma, double *__restrict__ weight) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cells) return;
    const double d = den[c];
    double m = nan(""), sg = nan("");
    if (d > 0.0) {
        double s1 = 0.0, s2 = 0.0;
        for (int r = 0; r < n_real; ++r) {
            const double v = num[(size_t)r * cells + c] / d;
            s1 += v;
            s2 += v * v;
        }
        m = s1 / n_real;
        const double var = s2 / n_real - m * m;
        sg = sqrt(var > 0.0 ? var : 0.0);
    }
    if (mean) mean[c] = m;
    if (sigma) sigma[c] = sg;
    if (weight) weight[c] = d;
}

}  // namespace

abs_status launch_rebin(abs_ctx *ctx, const Setup &s, int32_t n_real, int32_t n_trip, const double *d_B,
                        const int64_t *d_count, const double *d_ellbar, const int32_t *d_ijk, int32_t n_mu,
                        int32_t n_t, double *d_mean, double *d_sigma, double *d_weight) {
    const int cells = s.nb * n_mu * n_t;
    double *num = (double *)workspace(ctx, "rebin.num", sizeof(double) * (size_t)n_real * cells);
    double *den = (double *)workspace(ctx, "rebin.den", sizeof(double) * (size_t)cells);
    if (!num || !den) return fail(ctx, ABS_ERR_OOM, "rebin workspace");
    StageTimer timer(ctx, "rebin");
    cudaMemsetAsync(num, 0, sizeof(double) * (size_t)n_real * cells, ctx->stream);
    cudaMemsetAsync(den, 0, sizeof(double) * (size_t)cells, ctx->stream);
    const int64_t work = (int64_t)n_real * n_trip;
    if (work > 0)
        k_rebin_accum<<<(unsigned)cdiv(work, 256), 256, 0, ctx->stream>>>(n_real, n_trip, s.nb, n_mu, n_t, d_B, d_count,
                                                                           d_ellbar, d_ijk, num, den);
    k_rebin_finish<<<(unsigned)cdiv(cells, 256), 256, 0, ctx->stream>>>(n_real, cells, num, den, d_mean, d_sigma,
                                                                         d_weight);
    return check_launch(ctx, "rebin");
}

}  // namespace absk
