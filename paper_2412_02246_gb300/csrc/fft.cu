// Stage 2: ring-restricted transforms, Eqs. iFT and iFT_I (Sec. 2).
//
// For ring m, X_m(g) = V_g / sum w on the filled cells of a_m, zero elsewhere,
// and D_m(p) = sum_g X_m(g) exp(-2 pi i g.p / N) on the N x N sky grid.
// Because X_m is Hermitian, D_m is real, so two rings a, b are transformed at
// once as Z = X_a + i X_b, giving D_a = Re FFT(Z) and D_b = Im FFT(Z).
//
// The 2D transform is a row pass then a column pass.  Only the rows
// |g_y| <= R_b of a ring pair are nonzero, so the row pass transforms just
// those (2 R_b + 1 of N) rows into a compact intermediate [2R_b+1][N]; the
// column pass reads CW adjacent columns of it (coalesced), expands each to
// length N with the zero rows, and writes CW columns of both fields.
//
// Both passes are radix-2/3/4/5 Stockham transforms in shared memory (the
// autosort form: pass with span p and radix R reads x[i + q N/R], applies
// the twiddle exp(-2 pi i q (i mod p) / (p R)), and writes the R outputs at
// (i div p) p R + (i mod p) + s p).  Twiddles come from a table of
// exp(-2 pi i t / N) evaluated in double on the host.
#include "abs_internal.cuh"

namespace absk {
namespace {

constexpr int MAXRAD = 16;

struct FftPlan {
    int N, nrad;
    int rad[MAXRAD];
};

struct RingGeom {
    int n, half, nb, N, Rmax;
};

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmul_mi(float2 a) { return make_float2(a.y, -a.x); }  // a * (-i)
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// One Stockham pass over `lines` transforms of length N stored line-major.
__device__ __forceinline__ void stockham_pass(const float2 *__restrict__ in, float2 *__restrict__ out,
                                              int N, int R, int p, int lines,
                                              const float2 *__restrict__ tw) {
    const int T = N / R;
    const int tstep = N / (p * R);
    const int nb = lines * T;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const int l = b / T, i = b - l * T;
        const int k = i % p;
        const float2 *src = in + (size_t)l * N + i;
        float2 *dst = out + (size_t)l * N + (i - k) * R + k;
        float2 x[5];
        x[0] = src[0];
        for (int q = 1; q < R; ++q) {
            const float2 v = src[q * T];
            x[q] = k ? cmul(v, __ldg(&tw[q * k * tstep])) : v;
        }
        if (R == 4) {
            const float2 a0 = cadd(x[0], x[2]), a1 = csub(x[0], x[2]);
            const float2 b0 = cadd(x[1], x[3]), b1 = cmul_mi(csub(x[1], x[3]));
            dst[0] = cadd(a0, b0);
            dst[p] = cadd(a1, b1);
            dst[2 * p] = csub(a0, b0);
            dst[3 * p] = csub(a1, b1);
        } else if (R == 2) {
            dst[0] = cadd(x[0], x[1]);
            dst[p] = csub(x[0], x[1]);
        } else if (R == 3) {
            const float s3 = 0.866025403784438646763723f;  // sin(2 pi / 3)
            const float2 t = cadd(x[1], x[2]);
            const float2 m = make_float2(x[0].x - 0.5f * t.x, x[0].y - 0.5f * t.y);
            const float2 dd = cscale(cmul_mi(csub(x[1], x[2])), s3);
            dst[0] = cadd(x[0], t);
            dst[p] = cadd(m, dd);
            dst[2 * p] = csub(m, dd);
        } else {  // R == 5
            const float c1 = 0.309016994374947424102293f;   // cos(2 pi / 5)
            const float c2 = -0.809016994374947424102293f;  // cos(4 pi / 5)
            const float s1 = 0.951056516295153572116439f;   // sin(2 pi / 5)
            const float s2 = 0.587785252292473129168706f;   // sin(4 pi / 5)
            const float2 t1 = cadd(x[1], x[4]), t2 = cadd(x[2], x[3]);
            const float2 t3 = csub(x[1], x[4]), t4 = csub(x[2], x[3]);
            const float2 a1 = make_float2(x[0].x + c1 * t1.x + c2 * t2.x, x[0].y + c1 * t1.y + c2 * t2.y);
            const float2 a2 = make_float2(x[0].x + c2 * t1.x + c1 * t2.x, x[0].y + c2 * t1.y + c1 * t2.y);
            const float2 b1 = make_float2(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y);
            const float2 b2 = make_float2(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y);
            dst[0] = cadd(x[0], cadd(t1, t2));
            dst[p] = cadd(a1, cmul_mi(b1));
            dst[4 * p] = csub(a1, cmul_mi(b1));
            dst[2 * p] = cadd(a2, cmul_mi(b2));
            dst[3 * p] = csub(a2, cmul_mi(b2));
        }
    }
}

// Transforms `lines` lines in buffer a (scratch b); returns the buffer holding the result.
__device__ float2 *fft_lines(float2 *a, float2 *b, int lines, const FftPlan &P,
                             const float2 *__restrict__ tw) {
    int p = 1;
    for (int s = 0; s < P.nrad; ++s) {
        __syncthreads();
        stockham_pass(a, b, P.N, P.rad[s], p, lines, tw);
        p *= P.rad[s];
        float2 *t = a;
        a = b;
        b = t;
    }
    __syncthreads();
    return a;
}

__device__ __forceinline__ int bin_lookup(int64_t r2, int a, int b, const int64_t *__restrict__ q) {
    // 0: ring a, 1: ring b, -1: neither
    if (r2 >= q[a] && r2 < q[a + 1]) return 0;
    if (b >= 0 && r2 >= q[b] && r2 < q[b + 1]) return 1;
    return -1;
}

// Row pass: one CTA per (row y, ring pair).  W[pair][y + Rmax][N].
__global__ void __launch_bounds__(256) k_fft_rows(RingGeom G, FftPlan P, const int64_t *__restrict__ q,
                                                  const int32_t *__restrict__ Rm,
                                                  const float2 *__restrict__ grid,
                                                  const float *__restrict__ wsum,
                                                  const uint8_t *__restrict__ mask,
                                                  const float2 *__restrict__ tw,
                                                  float2 *__restrict__ W) {
    extern __shared__ float2 sbuf[];
    const int pair = blockIdx.y;
    const int a = 2 * pair, b = a + 1 < G.nb ? a + 1 : -1;
    const int Rp = max(Rm[a], b >= 0 ? Rm[b] : -1);
    const int y = (int)blockIdx.x - G.Rmax;
    if (Rp < 0 || y < -Rp || y > Rp) return;
    float2 *l0 = sbuf, *l1 = sbuf + G.N;
    for (int i = threadIdx.x; i < G.N; i += blockDim.x) l0[i] = make_float2(0.f, 0.f);
    __syncthreads();
    if (y >= -G.half && y <= G.half) {
        for (int x = -Rp + (int)threadIdx.x; x <= Rp; x += blockDim.x) {
            if (x < -G.half || x > G.half) continue;
            const int64_t r2 = (int64_t)x * x + (int64_t)y * y;
            const int which = bin_lookup(r2, a, b, q);
            if (which < 0) continue;
            const int64_t cell = (int64_t)(y < 0 ? y + G.n : y) * G.n + (x < 0 ? x + G.n : x);
            if (!mask[cell]) continue;
            const float2 g = grid[cell];
            const float w = wsum[cell];
            const float2 v = make_float2(__fdiv_rn(g.x, w), __fdiv_rn(g.y, w));
            // Z = X_a + i X_b
            l0[x < 0 ? x + G.N : x] = which == 0 ? v : make_float2(-v.y, v.x);
        }
    }
    float2 *res = fft_lines(l0, l1, 1, P, tw);
    float2 *dst = W + ((size_t)pair * (2 * G.Rmax + 1) + (y + G.Rmax)) * G.N;
    for (int i = threadIdx.x; i < G.N; i += blockDim.x) dst[i] = res[i];
}

// Column pass: one CTA per (CW-column tile, ring pair).
__global__ void __launch_bounds__(256) k_fft_cols(RingGeom G, FftPlan P, int CW,
                                                  const int32_t *__restrict__ Rm,
                                                  const float2 *__restrict__ W,
                                                  const float2 *__restrict__ tw,
                                                  float *__restrict__ fields) {
    extern __shared__ float2 sbuf[];
    const int pair = blockIdx.y;
    const int a = 2 * pair, b = a + 1 < G.nb ? a + 1 : -1;
    const int Rp = max(Rm[a], b >= 0 ? Rm[b] : -1);
    const int x0 = blockIdx.x * CW;
    const int cw = min(CW, G.N - x0);
    const size_t P2 = (size_t)G.N * G.N;
    if (Rp < 0) {  // both rings empty: zero fields
        for (int i = threadIdx.x; i < G.N * cw; i += blockDim.x) {
            const int py = i / cw, c = i - py * cw;
            fields[(size_t)a * P2 + (size_t)py * G.N + x0 + c] = 0.f;
            if (b >= 0) fields[(size_t)b * P2 + (size_t)py * G.N + x0 + c] = 0.f;
        }
        return;
    }
    float2 *l0 = sbuf, *l1 = sbuf + (size_t)CW * G.N;
    for (int i = threadIdx.x; i < CW * G.N; i += blockDim.x) l0[i] = make_float2(0.f, 0.f);
    __syncthreads();
    const int rows = 2 * Rp + 1;
    const float2 *src = W + (size_t)pair * (2 * G.Rmax + 1) * G.N;
    for (int i = threadIdx.x; i < rows * cw; i += blockDim.x) {
        const int row = i / cw, c = i - row * cw;
        const int y = row - Rp;
        l0[(size_t)c * G.N + (y < 0 ? y + G.N : y)] = src[(size_t)(y + G.Rmax) * G.N + x0 + c];
    }
    float2 *res = fft_lines(l0, l1, CW, P, tw);
    for (int i = threadIdx.x; i < G.N * cw; i += blockDim.x) {
        const int py = i / cw, c = i - py * cw;
        const float2 v = res[(size_t)c * G.N + py];
        fields[(size_t)a * P2 + (size_t)py * G.N + x0 + c] = v.x;
        if (b >= 0) fields[(size_t)b * P2 + (size_t)py * G.N + x0 + c] = v.y;
    }
}

FftPlan make_plan(const Setup &s) {
    FftPlan P;
    P.N = s.N;
    P.nrad = (int)s.radices.size();
    for (int i = 0; i < P.nrad && i < MAXRAD; ++i) P.rad[i] = s.radices[i];
    return P;
}

}  // namespace

abs_status launch_filter_fft(abs_ctx *ctx, const Setup &s, const float *d_grid, const float *d_wsum,
                             const uint8_t *d_mask, float *d_fields) {
    if ((int)s.radices.size() > MAXRAD) return fail(ctx, ABS_ERR_UNSUPPORTED, "FFT radix plan too long");
    RingGeom G{s.n, s.half, s.nb, s.N, s.R};
    const FftPlan P = make_plan(s);
    const int npairs = (s.nb + 1) / 2;
    const size_t wbytes = sizeof(float2) * (size_t)npairs * (2 * s.R + 1) * s.N;
    float2 *W = (float2 *)workspace(ctx, "fft.rows", wbytes);
    if (!W) return fail(ctx, ABS_ERR_OOM, "FFT row workspace");
    cudaStream_t st = ctx->stream;
    const size_t row_smem = sizeof(float2) * 2 * s.N;
    int CW = 32;
    while (CW > 1 && sizeof(float2) * 2 * (size_t)CW * s.N > 96 * 1024) CW >>= 1;
    const size_t col_smem = sizeof(float2) * 2 * (size_t)CW * s.N;
    static bool attr_set[64] = {};
    if (ctx->device < 64 && !attr_set[ctx->device]) {
        cudaFuncSetAttribute(k_fft_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
        cudaFuncSetAttribute(k_fft_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
        attr_set[ctx->device] = true;
    }
    {
        StageTimer timer(ctx, "fft_rows");
        k_fft_rows<<<dim3(2 * s.R + 1, npairs), 256, row_smem, st>>>(
            G, P, s.d_q, s.d_Rm, (const float2 *)d_grid, d_wsum, d_mask, s.d_tw, W);
    }
    {
        StageTimer timer(ctx, "fft_cols");
        k_fft_cols<<<dim3((unsigned)cdiv(s.N, CW), npairs), 256, col_smem, st>>>(G, P, CW, s.d_Rm, W,
                                                                               s.d_tw, d_fields);
    }
    return check_launch(ctx, "filter+FFT");
}

}  // namespace absk
