// Stage 3 (FP32 form) and stage 5: sky-plane triple sums, Eq. estimator_t.
//
// S_ijk = N^-2 sum_p D_i(p) D_j(p) D_k(p) for every listed triplet.  Triplets
// sharing (i, j) form a row; the product D_i D_j is formed once per pixel and
// row and multiplied into each D_k of the row (the contraction
// C[(i,j), k] = sum_p (D_i D_j)(p) D_k(p)).
//
// A CTA owns a group of up to TG consecutive triplets and a contiguous range
// of pixels.  It stages the fields of PC pixels at a time in shared memory
// (all rings, coalesced float4 loads); each warp takes a row segment of the
// group and accumulates 8 triplets at a time over the staged pixels (lane ->
// pixel, FP32), reduces across the warp, and adds the result into an FP64
// per-triplet accumulator in shared memory.  Per-CTA partial sums go to
// [split][triplet] and a second kernel adds the splits in a fixed order (so
// the result does not depend on scheduling) and applies N^-2 in FP64.
//
// B_ijk = S_ijk / (A T_ijk) is then formed in FP64 (NaN for T = 0).
#include <mutex>

#include "abs_internal.cuh"

namespace absk {
namespace {

constexpr int TG = 1024;       // triplets per CTA group
constexpr int TT = 512;        // threads per CTA
constexpr int KB = 8;          // triplets per warp pass
constexpr unsigned FULL = 0xffffffffu;

struct TripleGeom {
    int nb;
    int64_t P;                 // pixels
    int PC;                    // pixels staged per pass (multiple of 128)
    int64_t per_split;         // pixels per split (multiple of PC)
    int n_trip;
    int vec4;                  // fields rows are 16-byte aligned (P % 4 == 0, aligned base)
};

__global__ void __launch_bounds__(TT) k_triple_fp32(TripleGeom G, const float *__restrict__ fields,
                                                    const int32_t *__restrict__ ijk,
                                                    double *__restrict__ partial) {
    extern __shared__ __align__(16) uint8_t smem[];
    float *F = (float *)smem;                                    // [nb][PC]
    double *acc = (double *)(F + (size_t)G.nb * G.PC);           // [TG]
    int *seg = (int *)(acc + TG);                                 // [TG + 1] row starts
    int *kk = seg + TG + 1;                                       // [TG] k of each triplet
    uint8_t *flag = (uint8_t *)(kk + TG);                         // [TG] row-start flags
    __shared__ int nseg_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int t0 = blockIdx.y * TG;
    const int nt = min(TG, G.n_trip - t0);
    const int64_t p_begin = (int64_t)blockIdx.x * G.per_split;
    const int64_t p_end = min(G.P, p_begin + G.per_split);
    // row segments of this group: flag row starts, then compact with one warp
    for (int t = threadIdx.x; t < TG; t += blockDim.x) {
        uint8_t f = 0;
        if (t < nt) {
            acc[t] = 0.0;
            const int k = ijk[3 * (t0 + t) + 2];
            kk[t] = (k >= 0 && k < G.nb) ? k : -1;   // out-of-range bins contribute nothing
            const int i = ijk[3 * (t0 + t)], j = ijk[3 * (t0 + t) + 1];
            f = (t == 0 || i != ijk[3 * (t0 + t - 1)] || j != ijk[3 * (t0 + t - 1) + 1]) ? 1 : 0;
        }
        flag[t] = f;
    }
    __syncthreads();
    if (warp == 0) {
        const int base = lane * (TG / 32);
        int c = 0;
        for (int e = 0; e < TG / 32; ++e) c += flag[base + e];
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
        }
        int pos = incl - c;
        for (int e = 0; e < TG / 32; ++e)
            if (flag[base + e]) seg[pos++] = base + e;
        if (lane == 31) {
            seg[incl] = nt;
            nseg_s = incl;
        }
    }
    __syncthreads();
    const int nseg = nseg_s;
    for (int64_t pc = p_begin; pc < p_end; pc += G.PC) {
        const int np = (int)min((int64_t)G.PC, p_end - pc);
        __syncthreads();
        // stage fields[m][pc .. pc+np) (np is a multiple of 4 except possibly at the very end)
        const int nv4 = G.vec4 ? np / 4 : 0;
        for (int e = threadIdx.x; e < G.nb * nv4; e += blockDim.x) {
            const int m = e / nv4, v = e - m * nv4;
            ((float4 *)(F + (size_t)m * G.PC))[v] =
                __ldg((const float4 *)(fields + (size_t)m * G.P + pc) + v);
        }
        for (int e = threadIdx.x; e < G.nb * G.PC; e += blockDim.x) {
            const int m = e / G.PC, v = e - m * G.PC;
            if (v >= nv4 * 4) F[(size_t)m * G.PC + v] = v < np ? fields[(size_t)m * G.P + pc + v] : 0.f;
        }
        __syncthreads();
        for (int sgi = warp; sgi < nseg; sgi += nwarps) {
            const int ta = seg[sgi], tb = seg[sgi + 1];
            const int i = ijk[3 * (t0 + ta)], j = ijk[3 * (t0 + ta) + 1];
            if (i < 0 || i >= G.nb || j < 0 || j >= G.nb) continue;
            const float *Fi = F + (size_t)i * G.PC, *Fj = F + (size_t)j * G.PC;
            for (int tq = ta; tq < tb; tq += KB) {
                const float *Fk[KB];
                float a[KB];
#pragma unroll
                for (int b = 0; b < KB; ++b) {
                    Fk[b] = F + (size_t)max(kk[min(tq + b, tb - 1)], 0) * G.PC;
                    a[b] = 0.f;
                }
                for (int p = lane; p < G.PC; p += 32) {
                    const float dij = Fi[p] * Fj[p];
#pragma unroll
                    for (int b = 0; b < KB; ++b) a[b] = fmaf(dij, Fk[b][p], a[b]);
                }
#pragma unroll
                for (int b = 0; b < KB; ++b) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) a[b] += __shfl_xor_sync(FULL, a[b], o);
                }
                if (lane == 0) {
#pragma unroll
                    for (int b = 0; b < KB; ++b)
                        if (tq + b < tb && kk[tq + b] >= 0) acc[tq + b] += (double)a[b];
                }
            }
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nt; t += blockDim.x)
        partial[(size_t)blockIdx.x * G.n_trip + t0 + t] = acc[t];
}

// S[t] = inv_p * sum over splits of partial[split][t]: 32 triplets per block,
// 8 lanes of splits per triplet, summed in a fixed order (deterministic).
__global__ void __launch_bounds__(256) k_triple_reduce(int n_trip, int nsplit, double inv_p,
                                                       const double *__restrict__ partial,
                                                       double *__restrict__ S) {
    __shared__ double sh[8][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int t = blockIdx.x * 32 + tx;
    double s = 0.0;
    if (t < n_trip)
        for (int k = ty; k < nsplit; k += 8) s += partial[(size_t)k * n_trip + t];
    sh[ty][tx] = s;
    __syncthreads();
    if (ty == 0 && t < n_trip) {
        double a = 0.0;
        for (int k = 0; k < 8; ++k) a += sh[k][tx];
        S[t] = a * inv_p;
    }
}

__global__ void k_normalise(int n_trip, double norm_A, const double *__restrict__ S,
                            const int64_t *__restrict__ T, double *__restrict__ B) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_trip) return;
    const int64_t c = T[t];
    B[t] = c > 0 ? S[t] / (norm_A * (double)c) : nan("");
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
                              const int32_t *d_ijk, double *d_sum) {
    if (n_trip == 0) return ABS_OK;
    if (s.precision == ABS_SPLIT_BF16) return launch_triple_tc(ctx, s, d_fields, n_trip, d_ijk, d_sum);
    TripleGeom G;
    G.nb = s.nb;
    G.P = (int64_t)s.N * s.N;
    G.n_trip = n_trip;
    // staged pixels: keep the field tile within ~96 KB, and make enough
    // chunks for about four CTAs per SM
    // one pixel range per CTA, about two CTAs per SM overall; each range is
    // staged in chunks of PC pixels (a multiple of 32 whose fields fit ~96 KB)
    const int groups = (int)cdiv(n_trip, TG);
    const int64_t target = std::max<int64_t>(1, cdiv(2 * ctx->sm_count, groups));
    const int64_t per = cdiv(cdiv(G.P, target), 32) * 32;
    const int64_t pc_max = std::max<int64_t>(32, ((96 * 1024) / (4 * (int64_t)G.nb)) / 32 * 32);
    const int PC = (int)std::min<int64_t>(per, pc_max);
    G.PC = PC;
    G.vec4 = (G.P % 4 == 0) && (((uintptr_t)d_fields & 15) == 0);
    G.per_split = cdiv(per, PC) * PC;
    const int64_t nsplit = cdiv(G.P, G.per_split);
    double *partial = (double *)workspace(ctx, "triple.partial", sizeof(double) * nsplit * n_trip);
    if (!partial) return fail(ctx, ABS_ERR_OOM, "triple-sum workspace");
    const size_t smem = (size_t)G.nb * PC * 4 + TG * 8 + (2 * TG + 1) * 4 + TG;
    cudaFuncSetAttribute(k_triple_fp32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    {
        StageTimer timer(ctx, "triple_fp32");
        k_triple_fp32<<<dim3((unsigned)nsplit, groups), TT, smem, ctx->stream>>>(G, d_fields, d_ijk, partial);
    }
    StageTimer timer(ctx, "triple_reduce");
    k_triple_reduce<<<(int)cdiv(n_trip, 32), 256, 0, ctx->stream>>>(
        n_trip, (int)nsplit, 1.0 / ((double)s.N * (double)s.N), partial, d_sum);
    return check_launch(ctx, "triple sums");
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
    TripleGeom G;
    G.nb = cfg->n_bins;
    G.P = (int64_t)N * N;
    G.n_trip = n_trip;
    const int groups = (int)cdiv(n_trip, TG);
    int64_t target = std::max<int64_t>(1, cdiv(2 * sms, groups));
    target = std::min<int64_t>(target, std::max<int64_t>(1, cap / n_trip));
    int64_t per = cdiv(cdiv(G.P, target), 32) * 32;
    const int64_t pc_max = std::max<int64_t>(32, ((96 * 1024) / (4 * (int64_t)G.nb)) / 32 * 32);
    const int PC = (int)std::min<int64_t>(per, pc_max);
    G.PC = PC;
    G.vec4 = (G.P % 4 == 0) && (((uintptr_t)d_fields & 15) == 0);
    G.per_split = cdiv(per, PC) * PC;
    int64_t nsplit = cdiv(G.P, G.per_split);
    while (nsplit * n_trip > cap) {   // rounding can leave one split too many
        per += PC;
        G.per_split = cdiv(per, PC) * PC;
        nsplit = cdiv(G.P, G.per_split);
    }
    const size_t smem = (size_t)G.nb * PC * 4 + TG * 8 + (2 * TG + 1) * 4 + TG;
    cudaFuncSetAttribute(k_triple_fp32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_triple_fp32<<<dim3((unsigned)nsplit, groups), TT, smem, stream>>>(G, d_fields, d_ijk, partial);
    k_triple_reduce<<<(int)cdiv(n_trip, 32), 256, 0, stream>>>(n_trip, (int)nsplit,
                                                               1.0 / ((double)N * (double)N), partial, d_sum);
    return cudaGetLastError() == cudaSuccess ? ABS_OK : ABS_ERR_CUDA;
}
