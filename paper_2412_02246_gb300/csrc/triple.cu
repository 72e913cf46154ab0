// Stage 3 (FP32 form) and stage 5: sky-plane triple sums, Eq. estimator_t.
//
// S_ijk = N^-2 sum_p D_i(p) D_j(p) D_k(p) for every listed triplet.
//
// A CTA owns a contiguous range of pixels, staged in shared memory for all
// rings (coalesced loads, rows padded so that lanes on different rings read
// different banks).  Lane <-> triplet: each warp takes 32 consecutive
// triplets and every lane walks the staged pixels four at a time, forming
// (D_i D_j) D_k with packed FP32x2 multiplies and fused multiply-adds into a
// float2 partial sum, folded every FOLD steps into a double-float (FP32
// pair, TwoSum) accumulator.  No
// cross-lane reduction is needed.  Per-CTA partial sums go to
// [split][triplet] as double-float pairs and a second kernel adds the splits
// in double-float in a fixed order (so the result does not depend on
// scheduling), then applies N^-2 in FP64.
//
// B_ijk = S_ijk / (A T_ijk) is then formed in FP64 (NaN for T = 0).
#include <mutex>

#include "abs_internal.cuh"

namespace absk {
namespace {

constexpr int FOLD = 8;        // 4-pixel steps per FP32 block before the FP64 fold
constexpr unsigned FULL = 0xffffffffu;

struct TripleGeom {
    int nb;
    int64_t P;                 // pixels
    int PC;                    // pixels staged per pass (multiple of 4)
    int stride;                // staged row stride in floats (odd number of float4s)
    int64_t per_split;         // pixels per split (multiple of PC)
    int n_trip;
    int rounds;                // triplet rounds per CTA (<= 4): blockDim.x triplets each
    int vec4;                  // fields rows are 16-byte aligned (P % 4 == 0, aligned base)
};

// a += (x y) z over four pixels, with packed FP32x2 arithmetic.
__device__ __forceinline__ void step4(float4 x, float4 y, float4 z, float2 &a) {
    const float2 p01 = __fmul2_rn(make_float2(x.x, x.y), make_float2(y.x, y.y));
    const float2 p23 = __fmul2_rn(make_float2(x.z, x.w), make_float2(y.z, y.w));
    a = __ffma2_rn(p01, make_float2(z.x, z.y), a);
    a = __ffma2_rn(p23, make_float2(z.z, z.w), a);
}

__global__ void k_triple_fp32(TripleGeom G, const float *__restrict__ fields, const int32_t *__restrict__ ijk,
                              double *__restrict__ partial) {
    extern __shared__ __align__(16) uint8_t smem[];
    float *F = (float *)smem;                                    // [nb][stride]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int64_t p_begin = (int64_t)blockIdx.x * G.per_split;
    const int64_t p_end = min(G.P, p_begin + G.per_split);
    // this CTA's triplets: [t_base, t_base + rounds * blockDim.x)
    const int t_base = blockIdx.y * G.rounds * blockDim.x;
    const int rounds = G.rounds;
    // this lane's triplet in each round (at most 4 rounds), as double-float
    // sums hi + lo: GB300's FP64 pipe is too narrow for a per-block FP64 add
    float Sh[4] = {0.f, 0.f, 0.f, 0.f}, Sl[4] = {0.f, 0.f, 0.f, 0.f};
    for (int64_t pc = p_begin; pc < p_end; pc += G.PC) {
        const int np = (int)min((int64_t)G.PC, p_end - pc);
        const int np4 = (np + 3) >> 2;
        __syncthreads();
        // stage fields[m][pc .. pc+np), zero-padded to a multiple of 4
        if (G.vec4 && (np & 3) == 0) {
            for (int e = threadIdx.x; e < G.nb * np4; e += blockDim.x) {
                const int m = e / np4, v = e - m * np4;
                ((float4 *)(F + (size_t)m * G.stride))[v] =
                    __ldg((const float4 *)(fields + (size_t)m * G.P + pc) + v);
            }
        } else {
            for (int e = threadIdx.x; e < G.nb * np4 * 4; e += blockDim.x) {
                const int m = e / (np4 * 4), v = e - m * (np4 * 4);
                F[(size_t)m * G.stride + v] = v < np ? fields[(size_t)m * G.P + pc + v] : 0.f;
            }
        }
        __syncthreads();
#pragma unroll
        for (int rd = 0; rd < 4; ++rd) {
            if (rd >= rounds) break;
            const int t = t_base + ((rd * nwarps + warp) << 5) + lane;
            if (t >= G.n_trip) continue;
            const int i = ijk[3 * t], j = ijk[3 * t + 1], k = ijk[3 * t + 2];
            if (i < 0 || i >= G.nb || j < 0 || j >= G.nb || k < 0 || k >= G.nb) continue;   // contributes nothing
            const float4 *Fi = (const float4 *)(F + (size_t)i * G.stride);
            const float4 *Fj = (const float4 *)(F + (size_t)j * G.stride);
            const float4 *Fk = (const float4 *)(F + (size_t)k * G.stride);
            float sh = Sh[rd], sl = Sl[rd];
            for (int q0 = 0; q0 < np4; q0 += FOLD) {
                float2 a = make_float2(0.f, 0.f);
                if (q0 + FOLD <= np4) {   // full block: all loads issued back to back
#pragma unroll
                    for (int u = 0; u < FOLD; ++u) step4(Fi[q0 + u], Fj[q0 + u], Fk[q0 + u], a);
                } else {
                    for (int q = q0; q < np4; ++q) step4(Fi[q], Fj[q], Fk[q], a);
                }
                const float v = __fadd_rn(a.x, a.y);
                const float t = __fadd_rn(sh, v);             // TwoSum(sh, v)
                const float bp = __fsub_rn(t, sh);
                sl = __fadd_rn(sl, __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bp)), __fsub_rn(v, bp)));
                sh = t;
            }
            Sh[rd] = sh;
            Sl[rd] = sl;
        }
    }
#pragma unroll
    for (int rd = 0; rd < 4; ++rd) {
        const int t = t_base + ((rd * nwarps + warp) << 5) + lane;
        if (rd < rounds && t < G.n_trip)
            ((float2 *)partial)[(size_t)blockIdx.x * G.n_trip + t] = make_float2(Sh[rd], Sl[rd]);
    }
}

// Launch shape of k_triple_fp32: pixel splits (about one CTA per SM, or
// fewer when max_split caps them) x triplet groups of up to 4096 (one warp per
// 32 triplets, at most 1024 threads, walked in at most four rounds), and the
// staged chunk.
struct TriplePlan {
    TripleGeom G;
    int64_t nsplit;
    int tgroups;
    int threads;
    size_t smem;
};

bool triple_plan(int nb, int64_t P, int n_trip, int sms, int64_t max_split, const float *d_fields, TriplePlan &tp) {
    TripleGeom &G = tp.G;
    G.nb = nb;
    G.P = P;
    G.n_trip = n_trip;
    const int ngroups = (int)cdiv(n_trip, 32);
    const int warps = std::min(32, ngroups);
    tp.threads = 32 * warps;
    G.rounds = (int)std::min<int64_t>(4, cdiv(ngroups, warps));
    tp.tgroups = (int)cdiv(n_trip, (int64_t)G.rounds * tp.threads);
    int64_t target = std::max<int64_t>(1, std::min<int64_t>(cdiv((int64_t)sms, tp.tgroups), max_split));
    int64_t per = cdiv(cdiv(G.P, target), 4) * 4;
    const int64_t pc_max = std::max<int64_t>(4, ((96 * 1024) / (4 * (int64_t)nb) - 4) / 4 * 4);
    G.PC = (int)std::min<int64_t>(per, pc_max);
    G.stride = 4 * ((G.PC / 4) | 1);   // an odd number of float4: rows start on different banks
    G.vec4 = (G.P % 4 == 0) && (((uintptr_t)d_fields & 15) == 0);
    G.per_split = cdiv(per, G.PC) * G.PC;
    tp.nsplit = cdiv(G.P, G.per_split);
    while (tp.nsplit > max_split) {   // rounding can leave one split too many
        per += G.PC;
        G.per_split = cdiv(per, G.PC) * G.PC;
        tp.nsplit = cdiv(G.P, G.per_split);
    }
    tp.smem = (size_t)nb * G.stride * 4;
    return true;
}

// x + y for double-float pairs (TwoSum of the high parts, low parts added).
__device__ __forceinline__ float2 df2_add(float2 x, float2 y) {
    const float s = __fadd_rn(x.x, y.x);
    const float bp = __fsub_rn(s, x.x);
    const float e = __fadd_rn(__fsub_rn(x.x, __fsub_rn(s, bp)), __fsub_rn(y.x, bp));
    const float t = __fadd_rn(e, __fadd_rn(x.y, y.y));
    const float h = __fadd_rn(s, t);
    return make_float2(h, __fsub_rn(t, __fsub_rn(h, s)));
}

// S[t] = inv_p * sum over splits of partial[split][t] (double-float pairs, stored
// as float2 in the 8 bytes of each entry): one warp per triplet, lane l adds
// splits l, l + 32, ... in double-float (GB300's FP64 pipe is narrow) and a
// fixed butterfly combines the lanes (the order never depends on scheduling, so
// results are reproducible); the total is widened to FP64 once.  With B != nullptr
// also B[t] = S[t] / (A T[t]) (NaN for T = 0).
__global__ void __launch_bounds__(256) k_triple_reduce(int n_trip, int nsplit, double inv_p,
                                                       const double *__restrict__ partial,
                                                       double *__restrict__ S, const int64_t *__restrict__ T,
                                                       double norm_A, double *__restrict__ B) {
    const int lane = threadIdx.x & 31;
    const int t = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (t >= n_trip) return;
    const float2 *pf = (const float2 *)partial;
    float2 s = make_float2(0.f, 0.f);
    for (int k = lane; k < nsplit; k += 32) s = df2_add(s, pf[(size_t)k * n_trip + t]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        s = df2_add(s, make_float2(__shfl_xor_sync(FULL, s.x, o), __shfl_xor_sync(FULL, s.y, o)));
    if (lane == 0) {
        const double v = ((double)s.x + (double)s.y) * inv_p;
        S[t] = v;
        if (B) {
            const int64_t c = T[t];
            B[t] = c > 0 ? v / (norm_A * (double)c) : nan("");
        }
    }
}

__global__ void k_normalise(int n_trip, double norm_A, const double *__restrict__ S,
                            const int64_t *__restrict__ T, double *__restrict__ B) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_trip) return;
    const int64_t c = T[t];
    B[t] = c > 0 ? S[t] / (norm_A * (double)c) : nan("");
}

__global__ void k_normalise_w(int n_trip, double norm_A, const double *__restrict__ S,
                              const double *__restrict__ SW, double *__restrict__ B) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_trip) return;
    const double w = SW[t];
    B[t] = w != 0.0 ? S[t] / (norm_A * w) : nan("");
}

// The sums of the discretely sampled prediction (Sec. 4): per triplet, over the
// pixels, P_i P_j I_k + P_j P_k I_i + P_k P_i I_j from fields P (of C(l_g)) and I
// (of the unit mask): the ordered closed triangles' C1 C2 + C2 C3 + C3 C1, times
// N^2.  Layout and accumulation as k_triple_fp32, with the P rows and then the
// I rows staged (G.nb rings each).
__global__ void k_triple_bana(TripleGeom G, const float *__restrict__ Pf, const float *__restrict__ If,
                              const int32_t *__restrict__ ijk, double *__restrict__ partial) {
    extern __shared__ __align__(16) uint8_t smem[];
    float *F = (float *)smem;                                    // [2 nb][stride]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int64_t p_begin = (int64_t)blockIdx.x * G.per_split;
    const int64_t p_end = min(G.P, p_begin + G.per_split);
    const int t_base = blockIdx.y * G.rounds * blockDim.x;
    const int rounds = G.rounds;
    float Sh[4] = {0.f, 0.f, 0.f, 0.f}, Sl[4] = {0.f, 0.f, 0.f, 0.f};
    const int rows = 2 * G.nb;
    for (int64_t pc = p_begin; pc < p_end; pc += G.PC) {
        const int np = (int)min((int64_t)G.PC, p_end - pc);
        const int np4 = (np + 3) >> 2;
        __syncthreads();
        for (int e = threadIdx.x; e < rows * np4 * 4; e += blockDim.x) {
            const int m = e / (np4 * 4), v = e - m * (np4 * 4);
            const float *src = m < G.nb ? Pf + (size_t)m * G.P : If + (size_t)(m - G.nb) * G.P;
            F[(size_t)m * G.stride + v] = v < np ? src[pc + v] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int rd = 0; rd < 4; ++rd) {
            if (rd >= rounds) break;
            const int t = t_base + ((rd * nwarps + warp) << 5) + lane;
            if (t >= G.n_trip) continue;
            const int i = ijk[3 * t], j = ijk[3 * t + 1], k = ijk[3 * t + 2];
            if (i < 0 || i >= G.nb || j < 0 || j >= G.nb || k < 0 || k >= G.nb) continue;
            const float4 *Pi = (const float4 *)(F + (size_t)i * G.stride);
            const float4 *Pj = (const float4 *)(F + (size_t)j * G.stride);
            const float4 *Pk = (const float4 *)(F + (size_t)k * G.stride);
            const float4 *Ii = (const float4 *)(F + (size_t)(G.nb + i) * G.stride);
            const float4 *Ij = (const float4 *)(F + (size_t)(G.nb + j) * G.stride);
            const float4 *Ik = (const float4 *)(F + (size_t)(G.nb + k) * G.stride);
            float sh = Sh[rd], sl = Sl[rd];
            for (int q0 = 0; q0 < np4; q0 += FOLD) {
                float2 a = make_float2(0.f, 0.f);
                const int qe = min(np4, q0 + FOLD);
                for (int q = q0; q < qe; ++q) {
                    step4(Pi[q], Pj[q], Ik[q], a);
                    step4(Pj[q], Pk[q], Ii[q], a);
                    step4(Pk[q], Pi[q], Ij[q], a);
                }
                const float v = __fadd_rn(a.x, a.y);
                const float tt = __fadd_rn(sh, v);             // TwoSum(sh, v)
                const float bp = __fsub_rn(tt, sh);
                sl = __fadd_rn(sl, __fadd_rn(__fsub_rn(sh, __fsub_rn(tt, bp)), __fsub_rn(v, bp)));
                sh = tt;
            }
            Sh[rd] = sh;
            Sl[rd] = sl;
        }
    }
#pragma unroll
    for (int rd = 0; rd < 4; ++rd) {
        const int t = t_base + ((rd * nwarps + warp) << 5) + lane;
        if (rd < rounds && t < G.n_trip)
            ((float2 *)partial)[(size_t)blockIdx.x * G.n_trip + t] = make_float2(Sh[rd], Sl[rd]);
    }
}

__global__ void k_check_triplets(int nb, int n_trip, const int32_t *__restrict__ ijk,
                                 int32_t *__restrict__ err) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_trip) return;
    const int i = ijk[3 * t], j = ijk[3 * t + 1], k = ijk[3 * t + 2];
    if (i < 0 || j < i || k < j || k >= nb) atomicCAS(err, 0, DERR_TRIPLET_BIN);
    if (t > 0) {
        const int pi = ijk[3 * t - 3], pj = ijk[3 * t - 2], pk = ijk[3 * t - 1];
        const bool ordered = pi < i || (pi == i && (pj < j || (pj == j && pk < k)));
        if (!ordered) atomicCAS(err, 0, DERR_TRIPLET_ORDER);
    }
}

}  // namespace

abs_status launch_check_triplets(abs_ctx *ctx, const Setup &s, int32_t n_trip, const int32_t *d_ijk) {
    if (n_trip == 0) return ABS_OK;
    StageTimer timer(ctx, "check_triplets");
    k_check_triplets<<<(int)cdiv(n_trip, 256), 256, 0, ctx->stream>>>(s.nb, n_trip, d_ijk, ctx->d_err);
    return check_launch(ctx, "triplet check");
}

abs_status launch_triple_sums(abs_ctx *ctx, const Setup &s, const float *d_fields, int32_t n_trip,
                              const int32_t *d_ijk, double *d_sum, const int64_t *d_count, double *d_B,
                              cudaEvent_t wait_before_b) {
    if (n_trip == 0) {
        if (wait_before_b) cudaStreamWaitEvent(ctx->stream, wait_before_b, 0);
        return ABS_OK;
    }
    if (s.precision == ABS_SPLIT_BF16) {
        const abs_status st = launch_triple_tc(ctx, s, d_fields, n_trip, d_ijk, d_sum);
        if (wait_before_b) cudaStreamWaitEvent(ctx->stream, wait_before_b, 0);
        if (st != ABS_OK || !d_B) return st;
        return launch_normalise(ctx, s, n_trip, d_sum, d_count, d_B);
    }
    TriplePlan tp;
    if (!triple_plan(s.nb, s.P, n_trip, ctx->sm_count, INT64_MAX, d_fields, tp))
        return fail(ctx, ABS_ERR_UNSUPPORTED, "FP32 triple-sum tiling");
    const int64_t nsplit = tp.nsplit;
    double *partial = (double *)workspace(ctx, "triple.partial", sizeof(double) * nsplit * n_trip);
    if (!partial) return fail(ctx, ABS_ERR_OOM, "triple-sum workspace");
    allow_smem(k_triple_fp32, tp.smem);
    {
        StageTimer timer(ctx, "triple_fp32");
        k_triple_fp32<<<dim3((unsigned)nsplit, tp.tgroups), tp.threads, tp.smem, ctx->stream>>>(tp.G, d_fields,
                                                                                             d_ijk, partial);
    }
    if (wait_before_b) cudaStreamWaitEvent(ctx->stream, wait_before_b, 0);
    StageTimer timer(ctx, "triple_reduce");
    k_triple_reduce<<<(int)cdiv(n_trip, 8), 256, 0, ctx->stream>>>(
        n_trip, (int)nsplit, 1.0 / (double)s.P, partial, d_sum, d_count, s.norm_A,
        d_B && d_count ? d_B : nullptr);
    return check_launch(ctx, "triple sums");
}

abs_status launch_bana_sums(abs_ctx *ctx, const Setup &s, const float *d_P, const float *d_I, int32_t n_trip,
                            const int32_t *d_ijk, const int64_t *d_count, double fs, double *d_out) {
    if (n_trip == 0) return ABS_OK;
    TriplePlan tp;   // sized for both field sets in shared memory
    if (!triple_plan(2 * s.nb, s.P, n_trip, ctx->sm_count, INT64_MAX, d_P, tp))
        return fail(ctx, ABS_ERR_UNSUPPORTED, "prediction triple-sum tiling");
    tp.G.nb = s.nb;
    const int64_t nsplit = tp.nsplit;
    double *partial = (double *)workspace(ctx, "bana.partial", sizeof(double) * nsplit * n_trip);
    double *sum = (double *)workspace(ctx, "bana.sum", sizeof(double) * n_trip);
    if (!partial || !sum) return fail(ctx, ABS_ERR_OOM, "prediction workspace");
    allow_smem(k_triple_bana, tp.smem);
    StageTimer timer(ctx, "bana_sums");
    k_triple_bana<<<dim3((unsigned)nsplit, tp.tgroups), tp.threads, tp.smem, ctx->stream>>>(tp.G, d_P, d_I, d_ijk,
                                                                                         partial);
    // out = sum / (N^2 A T) with A = 1 / (2 fs)
    k_triple_reduce<<<(int)cdiv(n_trip, 8), 256, 0, ctx->stream>>>(
        n_trip, (int)nsplit, 1.0 / (double)s.P, partial, sum, d_count, 1.0 / (2.0 * fs), d_out);
    return check_launch(ctx, "prediction sums");
}

// ------------------------------------------------------------------ allocation-free variant
// Partial sums of abs_triple_sums_static: one fixed array per device, looked up
// once per device with that device current.
static __device__ __align__(256) double g_static_partial[ABS_STATIC_SCRATCH_BYTES / sizeof(double)];
static double *g_static_ptr[64];
static std::mutex g_static_mu;

static abs_status static_scratch(int dev, double **out) {
    if (dev < 0 || dev >= 64) return ABS_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_partial) != cudaSuccess || !p) {
            cudaGetLastError();
            return ABS_ERR_CUDA;
        }
        g_static_ptr[dev] = (double *)p;
    }
    *out = g_static_ptr[dev];
    return ABS_OK;
}

abs_status launch_normalise_w(abs_ctx *ctx, const Setup &s, int32_t n_trip, const double *d_sum,
                              const double *d_sumw, double *d_B) {
    if (n_trip == 0 || !d_B) return ABS_OK;
    StageTimer timer(ctx, "normalise");
    k_normalise_w<<<(int)cdiv(n_trip, 256), 256, 0, ctx->stream>>>(n_trip, s.norm_A, d_sum, d_sumw, d_B);
    return check_launch(ctx, "normalise");
}

abs_status launch_normalise(abs_ctx *ctx, const Setup &s, int32_t n_trip, const double *d_sum,
                            const int64_t *d_count, double *d_B) {
    if (n_trip == 0) return ABS_OK;
    StageTimer timer(ctx, "normalise");
    k_normalise<<<(int)cdiv(n_trip, 256), 256, 0, ctx->stream>>>(n_trip, s.norm_A, d_sum, d_count, d_B);
    return check_launch(ctx, "normalise");
}

}  // namespace absk

extern "C" abs_status abs_triple_sums_static(const abs_config *cfg, const float *d_fields, int32_t n_trip,
                                             const int32_t *d_ijk, double *d_sum, void *cuda_stream) {
    using namespace absk;
    int64_t q[ABS_MAX_BINS + 1];
    int Rm[ABS_MAX_BINS];
    int R = 0, N = 0;
    const char *msg = "";
    const abs_status st = derive_grid(cfg, q, Rm, &R, &N, &msg);
    if (st != ABS_OK) return st;
    const int64_t cap = ABS_STATIC_SCRATCH_BYTES / sizeof(double);
    if (n_trip < 0 || n_trip > cap) return ABS_ERR_INVALID_ARG;
    if (n_trip == 0) return ABS_OK;
    if (!d_fields || !d_ijk || !d_sum) return ABS_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return ABS_ERR_CUDA;
    }
    double *partial = nullptr;
    const abs_status ss = static_scratch(dev, &partial);
    if (ss != ABS_OK) return ss;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    // same tiling as launch_triple_sums, with the number of pixel splits capped
    // so that [split][triplet] fits the fixed array
    TriplePlan tp;
    if (!triple_plan(cfg->n_bins, (int64_t)N * N, n_trip, sms, std::max<int64_t>(1, cap / n_trip), d_fields, tp))
        return ABS_ERR_UNSUPPORTED;
    const int64_t nsplit = tp.nsplit;
    if (!allow_smem(k_triple_fp32, tp.smem)) return ABS_ERR_CUDA;
    // each launch's own status (an error left over from the caller's earlier work is not ours to report)
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)nsplit, tp.tgroups);
    lc.blockDim = dim3(tp.threads);
    lc.dynamicSmemBytes = tp.smem;
    lc.stream = stream;
    if (cudaLaunchKernelEx(&lc, k_triple_fp32, tp.G, d_fields, d_ijk, partial) != cudaSuccess) {
        cudaGetLastError();
        return ABS_ERR_CUDA;
    }
    lc.gridDim = dim3((unsigned)cdiv(n_trip, 8));
    lc.blockDim = dim3(256);
    lc.dynamicSmemBytes = 0;
    const double *cpartial = partial;
    if (cudaLaunchKernelEx(&lc, k_triple_reduce, (int)n_trip, (int)nsplit, 1.0 / ((double)N * (double)N), cpartial,
                           d_sum, (const int64_t *)nullptr, 1.0, (double *)nullptr) != cudaSuccess) {
        cudaGetLastError();
        return ABS_ERR_CUDA;
    }
    return ABS_OK;
}
