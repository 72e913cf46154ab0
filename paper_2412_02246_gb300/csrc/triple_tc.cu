// Stage 3, precision form: triple sums as a split-BF16 contraction on the
// 5th-generation tensor cores (tcgen05), Eq. estimator_t numerator.
//
// C[r, k] = sum_p A[r, p] B[k, p],  r = (i, j) row of the triplet list,
//   A[r, p] = D_i(p) D_j(p),  B[k, p] = D_k(p),
// and S_ijk = N^-2 C[(i,j), k].  Each FP32 operand x is split into
// x_hi = bf16(x) and x_lo = bf16(x - x_hi) (x - x_hi is exact in FP32, so the
// pair carries 16 significant bits), and three BF16 products are accumulated
// in FP32 in tensor memory: C = Ah Bh^T + Ah Bl^T + Al Bh^T (the Al Bl^T term
// is below FP32 resolution of the result).
//
// One CTA owns a tile of 128 rows and a range of pixels; per chunk of 64
// pixels the 8 warps stage the fields in shared memory, form the four BF16
// operand tiles in the canonical K-major no-swizzle layout (8-row x 16-byte
// core matrices; K-adjacent core matrices 128 B apart, 8-row groups 256 B
// apart, one 16-column K slab after the other), and one thread issues the 12
// MMAs (4 K-steps x 3 products, M = 128, N = rings rounded up to 16, K = 16)
// and commits them to the chunk buffer's mbarrier.  Two buffers alternate, so
// forming chunk c+1 overlaps the MMAs of chunk c.  At the end the accumulator
// is read back with tcgen05.ld and each row writes the partial sums of its
// triplets; a second kernel adds the pixel ranges in FP64 in a fixed order.
//
// Every mbarrier wait is bounded; on timeout the kernel latches an error,
// waits (bounded) for its own MMAs, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include "abs_internal.cuh"

namespace absk {
namespace {

constexpr int TM = 128;          // rows per tile (MMA M)
constexpr int KC = 64;           // pixels per chunk (4 MMA K-steps)
constexpr int NT = 256;          // threads per CTA
constexpr int FPAD = 4;          // field row padding (floats)
constexpr unsigned FULL = 0xffffffffu;
constexpr uint32_t WAIT_LIMIT = 1u << 22;

struct TcGeom {
    int nb, NP;                  // rings, MMA N (rings rounded up to 16)
    int tmem_cols;               // power of two >= max(32, NP)
    int64_t P;                   // pixels
    int64_t per_split;           // pixels per CTA (multiple of KC)
    int n_trip;
    int a_bytes, b_bytes;        // one operand tile (hi or lo) in bytes
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start, leading (K) and stride (8-row group)
// byte offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t make_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFF) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        ::"r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                 ::"r"(mbar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok) : "r"(mbar), "r"(parity) : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (uint32_t it = 0; it < WAIT_LIMIT; ++it)
        if (mbar_try(mbar, parity)) return true;
    return false;
}

__device__ __forceinline__ void store_split8(uint8_t *hi_tile, uint8_t *lo_tile, int off, const float *v) {
    __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        h[e] = __float2bfloat16_rn(v[e]);
        l[e] = __float2bfloat16_rn(v[e] - __bfloat162float(h[e]));
    }
    *(uint4 *)(hi_tile + off) = *(const uint4 *)h;
    *(uint4 *)(lo_tile + off) = *(const uint4 *)l;
}

// Byte offset of (row r, 8-column group g) of a K-major tile with rows8 8-row groups.
__device__ __forceinline__ int core_off(int r, int g, int rows8) {
    const int slab = g >> 1, cb = g & 1;
    return slab * rows8 * 256 + (r >> 3) * 256 + cb * 128 + (r & 7) * 16;
}

__global__ void __launch_bounds__(NT, 1) k_triple_tc(TcGeom G, const float *__restrict__ fields,
                                                     const int4 *__restrict__ rows,
                                                     const int *__restrict__ n_rows_p,
                                                     const int32_t *__restrict__ ijk,
                                                     double *__restrict__ partial,
                                                     int32_t *__restrict__ err) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_holder;
    __shared__ int rowi[TM], rowj[TM];
    __shared__ int abort_s;
    const int n_rows = *n_rows_p;
    const int r0 = blockIdx.x * TM;
    if (r0 >= n_rows) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // layout: [buf 0: Ah Al Bh Bl][buf 1: Ah Al Bh Bl][fields nb x (KC + FPAD)]
    const int buf_bytes = 2 * G.a_bytes + 2 * G.b_bytes;
    float *F = (float *)(smem + 2 * buf_bytes);
    const int fstride = KC + FPAD;
    if (threadIdx.x < TM) {
        const int r = r0 + threadIdx.x;
        int i = -1, j = -1;
        if (r < n_rows) {
            const int4 R = rows[r];
            i = R.x;
            j = R.y;
        }
        rowi[threadIdx.x] = i;
        rowj[threadIdx.x] = j;
    }
    if (threadIdx.x == 0) {
        abort_s = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     ::"r"(smem_u32(&tmem_holder)), "r"(G.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_holder;
    const uint32_t idesc = make_idesc(TM, G.NP);
    const int64_t p_begin = (int64_t)blockIdx.y * G.per_split;
    const int64_t p_end = min(G.P, p_begin + G.per_split);
    const int nchunks = (int)cdiv(p_end - p_begin, KC);
    const int rows8_a = TM / 8, rows8_b = G.NP / 8;
    uint32_t phase[2] = {0u, 0u};
    bool ok = true;
    for (int c = 0; c < nchunks && ok; ++c) {
        const int bsel = c & 1;
        uint8_t *Ah = smem + bsel * buf_bytes, *Al = Ah + G.a_bytes;
        uint8_t *Bh = Al + G.a_bytes, *Bl = Bh + G.b_bytes;
        if (c >= 2) {   // MMAs that read this buffer two chunks ago must be done
            if (threadIdx.x == 0 && !mbar_wait(smem_u32(&mbar[bsel]), phase[bsel] ^ 1u)) abort_s = 1;
        }
        __syncthreads();
        if (abort_s) {
            ok = false;
            break;
        }
        // stage fields of this chunk (zero beyond the last pixel)
        const int64_t pc = p_begin + (int64_t)c * KC;
        for (int e = threadIdx.x; e < G.nb * KC; e += NT) {
            const int m = e / KC, px = e - m * KC;
            F[m * fstride + px] = pc + px < p_end ? __ldg(&fields[(size_t)m * G.P + pc + px]) : 0.f;
        }
        __syncthreads();
        // A: 128 rows x 64 pixels as 128 x 8 groups of 8; lane -> (row within 8, group)
        for (int u = threadIdx.x; u < TM * (KC / 8); u += NT) {
            const int rg = u >> 6, rem = u & 63;        // 8-row group, (group, row) inside
            const int g = rem >> 3, r = rg * 8 + (rem & 7);
            const int i = rowi[r], j = rowj[r];
            float v[8];
            if (i >= 0) {
                const float *fi = F + i * fstride + g * 8, *fj = F + j * fstride + g * 8;
#pragma unroll
                for (int e = 0; e < 8; ++e) v[e] = fi[e] * fj[e];
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e) v[e] = 0.f;
            }
            store_split8(Ah, Al, core_off(r, g, rows8_a), v);
        }
        // B: NP rings x 64 pixels
        for (int u = threadIdx.x; u < G.NP * (KC / 8); u += NT) {
            const int rg = u >> 6, rem = u & 63;
            const int g = rem >> 3, k = rg * 8 + (rem & 7);
            float v[8];
            if (k < G.nb) {
                const float *fk = F + k * fstride + g * 8;
#pragma unroll
                for (int e = 0; e < 8; ++e) v[e] = fk[e];
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e) v[e] = 0.f;
            }
            store_split8(Bh, Bl, core_off(k, g, rows8_b), v);
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
            for (int ks = 0; ks < KC / 16; ++ks) {
                const uint64_t ah = make_desc(smem_u32(Ah + ks * rows8_a * 256), 128, 256);
                const uint64_t al = make_desc(smem_u32(Al + ks * rows8_a * 256), 128, 256);
                const uint64_t bh = make_desc(smem_u32(Bh + ks * rows8_b * 256), 128, 256);
                const uint64_t bl = make_desc(smem_u32(Bl + ks * rows8_b * 256), 128, 256);
                mma_bf16(tmem, ah, bh, idesc, (c > 0 || ks > 0) ? 1u : 0u);
                mma_bf16(tmem, ah, bl, idesc, 1u);
                mma_bf16(tmem, al, bh, idesc, 1u);
            }
            mma_commit(smem_u32(&mbar[bsel]));
        }
        phase[bsel] ^= 1u;
    }
    // wait for the last commit of each used buffer
    if (threadIdx.x == 0) {
        for (int b = 0; b < 2; ++b) {
            const int uses = nchunks > b ? (nchunks - b + 1) / 2 : 0;
            if (uses > 0 && !mbar_wait(smem_u32(&mbar[b]), (uint32_t)((uses - 1) & 1))) {
                abort_s = 1;
            }
        }
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (!ok || abort_s) {
        if (threadIdx.x == 0) atomicCAS(err, 0, DERR_TIMEOUT);
    } else {
        // epilogue: TMEM -> shared [128][NP] (reuse buffer 0) -> per-triplet partials
        float *D = (float *)smem;
        const int lane_base = (warp & 3) * 32;
        const int r = lane_base + lane;
        for (int col = (warp >> 2) * 16; col < G.NP; col += 32) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)lane_base << 16) + (uint32_t)col;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
                "%11, %12, %13, %14, %15}, [%16];\n"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                  "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                  "=r"(v[14]), "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
            for (int e = 0; e < 16; ++e) D[r * (G.NP + 1) + col + e] = __uint_as_float(v[e]);
        }
        __syncthreads();
        if (threadIdx.x < TM && r0 + (int)threadIdx.x < n_rows) {
            const int4 R = rows[r0 + threadIdx.x];
            for (int t = R.z; t < R.w; ++t) {
                const int k = ijk[3 * t + 2];
                if (k >= 0 && k < G.nb)
                    partial[(size_t)blockIdx.y * G.n_trip + t] = (double)D[threadIdx.x * (G.NP + 1) + k];
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(G.tmem_cols));
}

// Row table: one entry (i, j, first triplet, end) per run of equal (i, j).
__global__ void __launch_bounds__(1024) k_rows(int n_trip, const int32_t *__restrict__ ijk,
                                               int4 *__restrict__ rows, int *__restrict__ n_rows) {
    __shared__ int wsum[32];
    __shared__ int carry_s;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int b = 0; b < n_trip; b += blockDim.x) {
        const int t = b + threadIdx.x;
        bool start = false;
        if (t < n_trip)
            start = t == 0 || ijk[3 * t] != ijk[3 * t - 3] || ijk[3 * t + 1] != ijk[3 * t - 2];
        const unsigned bal = __ballot_sync(FULL, start);
        if (lane == 0) wsum[warp] = __popc(bal);
        __syncthreads();
        int before = 0, tot = 0;
        for (int w = 0; w < 32; ++w) {
            if (w < warp) before += wsum[w];
            tot += wsum[w];
        }
        if (start) {
            const int pos = carry_s + before + __popc(bal & ((1u << lane) - 1u));
            int e = t + 1;
            while (e < n_trip && ijk[3 * e] == ijk[3 * t] && ijk[3 * e + 1] == ijk[3 * t + 1]) ++e;
            rows[pos] = make_int4(ijk[3 * t], ijk[3 * t + 1], t, e);
        }
        __syncthreads();
        if (threadIdx.x == 0) carry_s += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *n_rows = carry_s;
}

// S[t] = inv_p * sum over splits of partial[split][t]: 32 triplets per block,
// 8 lanes of splits per triplet, summed in a fixed order (deterministic).
__global__ void __launch_bounds__(256) k_tc_reduce(int n_trip, int nsplit, double inv_p,
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

}  // namespace

abs_status launch_triple_tc(abs_ctx *ctx, const Setup &s, const float *d_fields, int32_t n_trip,
                            const int32_t *d_ijk, double *d_sum) {
    if (n_trip == 0) return ABS_OK;
    TcGeom G;
    G.nb = s.nb;
    G.NP = (int)cdiv(std::max(s.nb, 16), 16) * 16;
    if (G.NP > 256) return fail(ctx, ABS_ERR_UNSUPPORTED, "split-BF16 path supports at most 256 rings");
    G.tmem_cols = 32;
    while (G.tmem_cols < G.NP) G.tmem_cols <<= 1;
    G.P = (int64_t)s.N * s.N;
    G.n_trip = n_trip;
    G.a_bytes = TM * KC * 2;
    G.b_bytes = G.NP * KC * 2;
    const int max_rows = std::min<int64_t>(n_trip, (int64_t)s.nb * (s.nb + 1) / 2);
    const int tiles = (int)cdiv(max_rows, TM);
    // pixel ranges: enough CTAs for about one wave, at most 4096 pixels each
    // (bounds the FP32 accumulation length inside the tensor core)
    int64_t per = cdiv(cdiv(G.P, std::max<int64_t>(1, cdiv(ctx->sm_count, tiles))), KC) * KC;
    per = std::min<int64_t>(per, 4096);
    G.per_split = per;
    const int64_t nsplit = cdiv(G.P, per);
    int4 *rows = (int4 *)workspace(ctx, "tc.rows", sizeof(int4) * std::max(max_rows, 1));
    int *n_rows = (int *)workspace(ctx, "tc.n_rows", sizeof(int));
    double *partial = (double *)workspace(ctx, "tc.partial", sizeof(double) * nsplit * n_trip);
    if (!rows || !n_rows || !partial) return fail(ctx, ABS_ERR_OOM, "split-BF16 workspace");
    cudaStream_t st = ctx->stream;
    const size_t buf = 2 * (size_t)G.a_bytes + 2 * (size_t)G.b_bytes;
    const size_t smem = std::max(2 * buf + (size_t)G.nb * (KC + FPAD) * 4, (size_t)TM * (G.NP + 1) * 4);
    if (smem > 220 * 1024) return fail(ctx, ABS_ERR_UNSUPPORTED, "split-BF16 tile does not fit shared memory");
    cudaFuncSetAttribute(k_triple_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    {
        StageTimer timer(ctx, "tc_rows");
        cudaMemsetAsync(partial, 0, sizeof(double) * nsplit * n_trip, st);
        k_rows<<<1, 1024, 0, st>>>(n_trip, d_ijk, rows, n_rows);
    }
    {
        StageTimer timer(ctx, "triple_tc");
        k_triple_tc<<<dim3(tiles, (unsigned)nsplit), NT, smem, st>>>(G, d_fields, rows, n_rows, d_ijk, partial,
                                                                    ctx->d_err);
    }
    {
        StageTimer timer(ctx, "triple_reduce");
        k_tc_reduce<<<(int)cdiv(n_trip, 32), 256, 0, st>>>(n_trip, (int)nsplit,
                                                             1.0 / ((double)s.N * (double)s.N), partial, d_sum);
    }
    return check_launch(ctx, "split-BF16 triple sums");
}

}  // namespace absk
