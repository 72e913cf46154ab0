// Stage 3, precision form: triple sums as a split-BF16 contraction on the
// 5th-generation tensor cores (tcgen05), Eq. estimator_t numerator.
//
// C[r, k] = sum_p A[r, p] B[k, p],  r = (i, j) row of the triplet list,
//   A[r, p] = D_i(p) D_j(p),  B[k, p] = D_k(p),
// and S_ijk = N^-2 C[(i,j), k].  Each FP32 operand x is split into
// x_hi = bf16(x) and x_lo = bf16(x - x_hi) (x - x_hi is exact in FP32, so the
// pair carries 16 significant bits), and three BF16 products are accumulated
// in FP32 in tensor memory: C = Ah Bh^T + Ah Bl^T + Al Bh^T (the Al Bl^T term
// is below FP32 resolution of the result).  Bh and Bl are stacked into one
// operand [Bh; Bl], so one MMA gives Ah Bh^T and Ah Bl^T side by side and Ah
// is read from shared memory once per K-step; the three FP32 accumulators
// are added in the epilogue.
//
// Rows are ordered by j (then i) and cut into tiles of 128.  A row (i, j)
// only meets the rings k in [j, k_max(i, j)] (the triangle condition), so a
// tile of neighbouring j meets a narrow band of rings: the tile's MMA N is
// that band rounded up to 16, not every ring.
//
// Tiles are grouped so that a group's accumulators (3 x band columns per
// tile) fit the 512 columns of tensor memory.  One CTA owns a group of row
// tiles and a range of pixels, so each field chunk is brought in once for
// every tile of the group.  The range is streamed in chunks of 64-128 pixels by
// three roles through two rings of shared-memory stages, one of field chunks
// (deep, so loads run well ahead) and one of operand tiles (one step per
// chunk and tile):
//   loader warp    copies the chunk's fields, all rings x 68 pixels (the
//                  padded row keeps the producers' reads off one bank), with
//                  one 2-D TMA tensor copy (zero fill past the last pixel)
//                  into a field stage, completion counted on f_full,
//   producer warps form the four BF16 operand tiles (A = D_i D_j and the
//                  band of B = D_k, hi and lo) in the canonical K-major
//                  no-swizzle layout (8-row x 16-byte core matrices, K-adjacent
//                  ones 128 B apart, 8-row groups 256 B apart, one 16-column K
//                  slab after the other) in an operand stage, arrive on
//                  ab_full and release the field stage (f_empty),
//   MMA warp       issues the MMAs of a step (per 16-pixel K-step Ah [Bh; Bl]
//                  and Al Bh, M = 128, N = 2 band and band, K = 16) into the
//                  tile's accumulator columns and commits them to ab_empty,
//                  which frees the operand stage.
// At the end the accumulator is read back with tcgen05.ld and each row writes
// the partial sums of its triplets; a second kernel adds the pixel ranges in
// FP64 in a fixed order.
//
// Every mbarrier wait is bounded; on timeout the kernel latches an error,
// every role leaves its loop, the CTA waits (bounded) for its own copies and
// MMAs in flight, frees its tensor memory and returns.  Where the fields
// cannot be described as a TMA tensor (rows not 16-byte aligned), the loader
// warp copies them with plain loads.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <map>

#include "abs_internal.cuh"

namespace absk {
namespace {

constexpr int TM = 128;          // rows per tile (MMA M)
constexpr int NPW = 16;          // producer warps
constexpr int LOADER = NPW, ISSUER = NPW + 1;   // the two control warps
constexpr int NT = (NPW + 2) * 32;

// The chunk: KC pixels (KC / 16 MMA K-steps), the widest of 128, 96, 64 whose
// stages fit shared memory (wider chunks spread the per-step costs, barrier
// round trips and the MMA commit, over more work).
template <int KC>
struct Chunk {
    static_assert(KC % 32 == 0 && KC <= 128, "whole 16-pixel K-steps; 8-pixel groups; TMA box <= 256");
    static constexpr int GPR = KC / 8;                       // 8-pixel groups per row of a chunk
    static constexpr int KA = TM * GPR / (NPW * 32);         // A units (row, 8 pixels) per producer thread
    static constexpr int KB = 256 * GPR / (NPW * 32);        // B units per producer thread at most (band <= 256)
    static constexpr int FS = KC + 4;   // field row in a stage (floats, a multiple of 4): the TMA box width
    static_assert(KA * NPW * 32 == TM * GPR, "A units split evenly over the producers");
};
constexpr int MAX_AB = 3, MAX_F = 8;   // operand and field stages
constexpr int GMAX = 10;         // row tiles per group (3 x 16 accumulator columns each at least)
constexpr int TMEM_COLS = 512;
constexpr unsigned FULL = 0xffffffffu;
constexpr uint32_t WAIT_LIMIT = 1u << 22;

struct TcGeom {
    int nb, NP;                  // rings, largest MMA N (rings rounded up to 16)
    int tmem_cols;               // columns allocated (the group's accumulators fit them)
    int64_t P;                   // pixels
    int64_t per_split;           // pixels per CTA (multiple of the chunk)
    int n_trip;
    int sf, sa;                  // field and operand stages
    int f_bytes, ab_bytes;       // one field stage [nb][KC + 4] floats; one operand stage [Ah][Al][Bh; Bl]
    int a_bytes, b_bytes;        // one A tile (hi or lo); the stacked B tile (2 NP rows)
    int tma;                     // fields by TMA tensor copy (else plain loads by the loader warp)
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

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(mbar), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];\n" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;\n"
                 ::"r"(mbar), "r"(bytes) : "memory");
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

// Bounded wait for the phase of the given parity; false on timeout, or once
// another role has given up (abort set).
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, const volatile int *abort_flag) {
    for (uint32_t it = 0; it < WAIT_LIMIT; ++it) {
        if (mbar_try(mbar, parity)) return true;
        if ((it & 255u) == 255u && *abort_flag) return false;
    }
    return false;
}

// Bounded wait for work already in flight (copies, MMAs), whatever the abort flag says.
__device__ __forceinline__ bool mbar_drain(uint32_t mbar, uint32_t parity) {
    for (uint32_t it = 0; it < WAIT_LIMIT; ++it)
        if (mbar_try(mbar, parity)) return true;
    return false;
}

// 2-D tensor copy of the box at (x, y) into shared memory, counted on mbar.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n"
        ::"r"(dst), "l"((uint64_t)map), "r"(x), "r"(y), "r"(mbar) : "memory");
}

// Eight FP32 values (four pairs) as their BF16 hi parts and BF16 residuals,
// stored as one 16-byte core-matrix row each.
__device__ __forceinline__ void store_split8(uint8_t *hi_tile, uint8_t *lo_tile, int off, const float2 *v) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const __nv_bfloat162 hb = __float22bfloat162_rn(v[e]);
        const float2 hf = __bfloat1622float2(hb);
        const float2 r = __ffma2_rn(hf, make_float2(-1.f, -1.f), v[e]);   // v - hi, exact in FP32
        const __nv_bfloat162 lb = __float22bfloat162_rn(r);
        h[e] = *(const uint32_t *)&hb;
        l[e] = *(const uint32_t *)&lb;
    }
    *(uint4 *)(hi_tile + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *(uint4 *)(lo_tile + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// Byte offset of (row r, 8-column group g) of a K-major tile with rows8 8-row groups.
__device__ __forceinline__ int core_off(int r, int g, int rows8) {
    const int slab = g >> 1, cb = g & 1;
    return slab * rows8 * 256 + (r >> 3) * 256 + cb * 128 + (r & 7) * 16;
}

// Eight consecutive field values at f (16-byte aligned), as four pairs.
__device__ __forceinline__ void ld8(const float *f, float2 *v) {
    const float4 a = *(const float4 *)f;
    const float4 b = *(const float4 *)(f + 4);
    v[0] = make_float2(a.x, a.y);
    v[1] = make_float2(a.z, a.w);
    v[2] = make_float2(b.x, b.y);
    v[3] = make_float2(b.z, b.w);
}

// Zero the pixels of group g at or past `valid` (the end of the pixel range).
__device__ __forceinline__ void mask_tail(float2 *v, int g, int valid) {
    if (g * 8 + 8 <= valid) return;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        if (g * 8 + 2 * e >= valid) v[e].x = 0.f;
        if (g * 8 + 2 * e + 1 >= valid) v[e].y = 0.f;
    }
}

template <int KC>
__global__ void __launch_bounds__(NT, 1) k_triple_tc(TcGeom G, const __grid_constant__ CUtensorMap fmap,
                                                     const float *__restrict__ fields,
                                                     const int4 *__restrict__ rows,
                                                     const int2 *__restrict__ tiles,
                                                     const int2 *__restrict__ groups,
                                                     const int *__restrict__ ctl,
                                                     const int32_t *__restrict__ ijk,
                                                     double *__restrict__ partial,
                                                     int32_t *__restrict__ err) {
    constexpr int GPR = Chunk<KC>::GPR, KA = Chunk<KC>::KA, KB = Chunk<KC>::KB, FS = Chunk<KC>::FS;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t f_full[MAX_F], f_empty[MAX_F], ab_full[MAX_AB], ab_empty[MAX_AB];
    // stages on a 1024-byte boundary (TMA destinations want 128; the launch adds 1 KB of slack)
    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    __shared__ uint32_t tmem_holder;
    __shared__ int16_t rowi[GMAX][TM], rowj[GMAX][TM];
    __shared__ int t_klo[GMAX], t_nb[GMAX], t_col[GMAX];
    __shared__ volatile int abort_s;
    const int n_rows = ctl[0], n_groups = ctl[1];
    if ((int)blockIdx.x >= n_groups) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int2 grp = groups[blockIdx.x];            // (first tile, tiles)
    const int t0 = grp.x, NG = grp.y;
    if (threadIdx.x < GMAX) {
        const int t = threadIdx.x;
        int lo = 0, w = 16;
        if (t < NG) {
            const int2 band = tiles[t0 + t];        // (first ring of the band, band width)
            lo = band.x;
            w = band.y;
        }
        t_klo[t] = lo;
        t_nb[t] = w;
    }
    for (int e = threadIdx.x; e < GMAX * TM; e += blockDim.x) {
        const int t = e / TM, rr = e - t * TM;
        const int r = (t0 + t) * TM + rr;
        int i = -1, j = -1;
        if (t < NG && r < n_rows) {
            const int4 R = rows[r];
            i = R.x;
            j = R.y;
        }
        rowi[t][rr] = (int16_t)i;
        rowj[t][rr] = (int16_t)j;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        abort_s = 0;
        int col = 0;
        for (int t = 0; t < GMAX; ++t) {   // accumulator columns of each tile: [Ah Bh | Ah Bl | Al Bh]
            t_col[t] = col;
            if (t < NG) col += 3 * t_nb[t];
        }
        for (int s = 0; s < G.sf; ++s) {
            mbar_init(smem_u32(&f_full[s]), 1);
            mbar_init(smem_u32(&f_empty[s]), NPW);
        }
        for (int s = 0; s < G.sa; ++s) {
            mbar_init(smem_u32(&ab_full[s]), NPW);
            mbar_init(smem_u32(&ab_empty[s]), 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == ISSUER) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     ::"r"(smem_u32(&tmem_holder)), "r"(G.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_holder;
    const int64_t p_begin = (int64_t)blockIdx.y * G.per_split;
    const int64_t p_end = min(G.P, p_begin + G.per_split);
    const int nchunks = (int)cdiv(p_end - p_begin, KC);
    const int nsteps = nchunks * NG;                // step = chunk x tile
    const int rows8_a = TM / 8;
    uint8_t *fbase = smem, *abase = smem + (size_t)G.sf * G.f_bytes;

    if (warp == LOADER) {
        // ---------------- loader: a field chunk (every ring) per field stage
        int issued = 0;
        for (int c = 0; c < nchunks; ++c) {
            const int s = c % G.sf, use = c / G.sf;
            bool ok = true;
            if (use > 0) {   // the producers are done with chunk c - sf
                if (lane == 0) ok = mbar_wait(smem_u32(&f_empty[s]), (uint32_t)((use - 1) & 1), &abort_s);
                ok = __shfl_sync(FULL, ok, 0);
            }
            if (!ok) {
                abort_s = 1;
                break;
            }
            float *F = (float *)(fbase + (size_t)s * G.f_bytes);
            const int64_t pc = p_begin + (int64_t)c * KC;
            if (G.tma) {
                if (lane == 0) {
                    mbar_arrive_tx(smem_u32(&f_full[s]), (uint32_t)(G.nb * FS * 4));
                    tma_load_2d(smem_u32(F), &fmap, (int)pc, 0, smem_u32(&f_full[s]));
                }
            } else {
                for (int e = lane; e < G.nb * FS; e += 32) {
                    const int m = e / FS, px = e - m * FS;
                    F[e] = pc + px < G.P ? __ldg(&fields[(size_t)m * G.P + pc + px]) : 0.f;
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&f_full[s]));
            }
            ++issued;
        }
        // copies still in flight land before the CTA moves on
        if (lane == 0 && G.tma)
            for (int s = 0; s < G.sf && s < issued; ++s) {
                const int uses = (issued - s + G.sf - 1) / G.sf;
                if (!mbar_drain(smem_u32(&f_full[s]), (uint32_t)((uses - 1) & 1))) abort_s = 1;
            }
    } else if (warp == ISSUER) {
        // ---------------- MMA issue: one thread, one step (chunk, tile) per operand stage
        if (lane == 0) {
            int committed = 0, c = 0, t = 0, s = 0, use = 0;   // step = (chunk c, tile t), stage s, its use
            int NB = t_nb[0];
            uint32_t acc_t = tmem + (uint32_t)t_col[0];
            for (int st = 0; st < nsteps; ++st) {
                if (!mbar_wait(smem_u32(&ab_full[s]), (uint32_t)(use & 1), &abort_s)) {
                    abort_s = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const int rows8_b = 2 * NB / 8;                 // B: [Bh; Bl], 2 NB rows
                const bool stacked = 2 * NB <= 256;             // one MMA for Ah [Bh; Bl] (N <= 256)
                const uint32_t id2 = make_idesc(TM, 2 * NB), id1 = make_idesc(TM, NB);
                uint8_t *Ah = abase + (size_t)s * G.ab_bytes, *Al = Ah + G.a_bytes;
                uint8_t *Bs = Al + G.a_bytes;
#pragma unroll
                for (int ks = 0; ks < KC / 16; ++ks) {
                    const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
                    const uint64_t ah = make_desc(smem_u32(Ah + ks * rows8_a * 256), 128, 256);
                    const uint64_t al = make_desc(smem_u32(Al + ks * rows8_a * 256), 128, 256);
                    const uint32_t bslab = smem_u32(Bs + ks * rows8_b * 256);
                    const uint64_t bh = make_desc(bslab, 128, 256);                // rows [0, NB): Bh
                    if (stacked) {
                        mma_bf16(acc_t, ah, bh, id2, acc);                           // cols [0, 2 NB)
                    } else {
                        const uint64_t bl = make_desc(bslab + (NB / 8) * 256, 128, 256);   // rows [NB, 2 NB): Bl
                        mma_bf16(acc_t, ah, bh, id1, acc);
                        mma_bf16(acc_t + (uint32_t)NB, ah, bl, id1, acc);
                    }
                    mma_bf16(acc_t + (uint32_t)(2 * NB), al, bh, id1, acc);     // cols [2 NB, 3 NB)
                }
                mma_commit(smem_u32(&ab_empty[s]));
                ++committed;
                if (++s == G.sa) {
                    s = 0;
                    ++use;
                }
                if (++t == NG) {
                    t = 0;
                    ++c;
                }
                if (NG > 1) {
                    NB = t_nb[t];
                    acc_t = tmem + (uint32_t)t_col[t];
                }
            }
            // every MMA issued is done before tensor memory is read or freed
            if (committed > 0) {
                const int st = committed - 1, s2 = st % G.sa, u2 = st / G.sa;
                if (!mbar_drain(smem_u32(&ab_empty[s2]), (uint32_t)(u2 & 1))) abort_s = 1;
            }
            if (committed < nsteps) abort_s = 1;
        }
    } else {
        // ---------------- producers: the operand tiles of a step.  A thread's
        // (row, 8-pixel group) units and band units are the same for every
        // chunk and tile: their tile offsets are worked out once.  Unit u =
        // (8-row group, 8 rows x GPR groups); a warp's 32 units are 8 rows x 4
        // groups (conflict-free 16-byte stores)
        const int p = threadIdx.x;
        int a_r[KA], a_g[KA], a_so[KA];
#pragma unroll
        for (int k = 0; k < KA; ++k) {
            const int u = p + k * NPW * 32;
            const int rg = u / (8 * GPR), rem = u % (8 * GPR);
            a_g[k] = rem >> 3;
            a_r[k] = rg * 8 + (rem & 7);
            a_so[k] = core_off(a_r[k], a_g[k], rows8_a);
        }
        int b_kk[KB], b_g[KB];
#pragma unroll
        for (int k = 0; k < KB; ++k) {
            const int u = p + k * NPW * 32;
            const int rg = u / (8 * GPR), rem = u % (8 * GPR);
            b_g[k] = rem >> 3;
            b_kk[k] = rg * 8 + (rem & 7);
        }
        // a step's field offsets (ring x FS + group x 8) and band, loaded one step ahead
        // so that no field load waits on a shared-memory lookup
        int fi[KA], fj[KA], nfi[KA], nfj[KA];
        auto row_offsets = [&](int t, int *oi, int *oj) {
#pragma unroll
            for (int k = 0; k < KA; ++k) {
                const int i = rowi[t][a_r[k]], j = rowj[t][a_r[k]];
                oi[k] = i >= 0 ? i * FS + a_g[k] * 8 : -1;
                oj[k] = j * FS + a_g[k] * 8;
            }
        };
        row_offsets(0, fi, fj);
        int nb_cur = t_nb[0], klo_cur = t_klo[0];
        int sa = 0, ua = 0, sf = 0, uf = 0;   // operand stage and its use; field stage and its use
        for (int c = 0; c < nchunks; ++c) {
            if (!mbar_wait(smem_u32(&f_full[sf]), (uint32_t)(uf & 1), &abort_s)) {
                abort_s = 1;
                break;
            }
            const float *F = (const float *)(fbase + (size_t)sf * G.f_bytes);
            const int64_t pc = p_begin + (int64_t)c * KC;
            const int valid = (int)min((int64_t)KC, p_end - pc);
            bool ok = true;
            for (int t = 0; t < NG; ++t) {
                if (ua > 0 && !mbar_wait(smem_u32(&ab_empty[sa]), (uint32_t)((ua - 1) & 1), &abort_s)) {
                    ok = false;
                    break;
                }
                uint8_t *Ah = abase + (size_t)sa * G.ab_bytes, *Al = Ah + G.a_bytes;
                uint8_t *Bs = Al + G.a_bytes;
                const int NB = nb_cur, klo = klo_cur, rows8_b = 2 * NB / 8;
                const int bl_off = (NB / 8) * 256;   // row NB of the stacked tile
                const int tn = t + 1 < NG ? t + 1 : 0;   // the next step's tile
                int nb_next = nb_cur, klo_next = klo_cur;
                if (NG > 1) {
                    row_offsets(tn, nfi, nfj);
                    nb_next = t_nb[tn];
                    klo_next = t_klo[tn];
                }
#pragma unroll
                for (int k = 0; k < KA; ++k) {
                    float2 v[4];
                    if (fi[k] >= 0) {
                        float2 x[4], y[4];
                        ld8(F + fi[k], x);
                        ld8(F + fj[k], y);
#pragma unroll
                        for (int e = 0; e < 4; ++e) v[e] = __fmul2_rn(x[e], y[e]);
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; ++e) v[e] = make_float2(0.f, 0.f);
                    }
                    if (valid < KC) mask_tail(v, a_g[k], valid);
                    store_split8(Ah, Al, a_so[k], v);
                }
#pragma unroll
                for (int k = 0; k < KB; ++k) {
                    if (p + k * NPW * 32 >= NB * GPR) break;   // past the band
                    const int ring = klo + b_kk[k];
                    float2 v[4];
                    if (ring < G.nb) {
                        ld8(F + ring * FS + b_g[k] * 8, v);
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; ++e) v[e] = make_float2(0.f, 0.f);
                    }
                    if (valid < KC) mask_tail(v, b_g[k], valid);
                    const int so = core_off(b_kk[k], b_g[k], rows8_b);   // Bh row kk; Bl row NB + kk
                    store_split8(Bs, Bs + bl_off, so, v);
                }
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&ab_full[sa]));
                if (++sa == G.sa) {
                    sa = 0;
                    ++ua;
                }
                if (NG > 1) {
#pragma unroll
                    for (int k = 0; k < KA; ++k) {
                        fi[k] = nfi[k];
                        fj[k] = nfj[k];
                    }
                    nb_cur = nb_next;
                    klo_cur = klo_next;
                }
            }
            if (!ok) {
                abort_s = 1;
                break;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&f_empty[sf]));   // every tile of the chunk is formed
            if (++sf == G.sf) {
                sf = 0;
                ++uf;
            }
        }
    }
    // every role is done: MMAs and copies have landed (or the CTA gave up)
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (abort_s) {
        if (threadIdx.x == 0) atomicCAS(err, 0, DERR_TIMEOUT);
    } else {
        // epilogue, tile by tile: TMEM -> shared [128][3 NB + 1] (over the stages) ->
        // per-triplet partials, (Ah Bh + Ah Bl) + Al Bh
        float *D = (float *)smem;
        for (int t = 0; t < NG; ++t) {
            const int NB = t_nb[t], klo = t_klo[t], dw = 3 * NB + 1;
            if (warp < 4) {   // warp w reads tensor-memory lanes 32 w .. 32 w + 31
                const int lane_base = warp * 32;
                const int r = lane_base + lane;
                for (int col = 0; col < 3 * NB; col += 16) {
                    uint32_t v[16];
                    const uint32_t taddr = tmem + ((uint32_t)lane_base << 16) + (uint32_t)(t_col[t] + col);
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
                        "%11, %12, %13, %14, %15}, [%16];\n"
                        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                          "=r"(v[14]), "=r"(v[15])
                        : "r"(taddr));
                    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
                    for (int e = 0; e < 16; ++e) D[r * dw + col + e] = __uint_as_float(v[e]);
                }
            }
            __syncthreads();
            const int r = (t0 + t) * TM + (int)threadIdx.x;
            if (threadIdx.x < TM && r < n_rows) {
                const int4 R = rows[r];
                for (int q = R.z; q < R.w; ++q) {
                    const int kk = ijk[3 * q + 2] - klo;
                    if (kk >= 0 && kk < NB) {
                        const float *d = D + threadIdx.x * dw + kk;
                        // (hh + hl) + lh as an exact double-float pair (TwoSum), stored in the entry's 8 bytes
                        const float x = d[0] + d[NB], y = d[2 * NB];
                        const float sm = __fadd_rn(x, y), bp = __fsub_rn(sm, x);
                        const float er = __fadd_rn(__fsub_rn(x, __fsub_rn(sm, bp)), __fsub_rn(y, bp));
                        ((float2 *)partial)[(size_t)blockIdx.y * G.n_trip + q] = make_float2(sm, er);
                    }
                }
            }
            __syncthreads();
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == ISSUER)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(G.tmem_cols));
}

// Row table of a (canonical, sorted) triplet list: one entry (i, j, first
// triplet, end) per run of equal (i, j), ordered by (j, i); then per tile of
// TM rows its band of rings (first k, width rounded up to 16, at most np);
// then groups of consecutive tiles whose accumulators (3 x band columns
// each) fit TMEM_COLS, at most gmax tiles and about as many tiles in each
// (gmax = 1: a group per tile).  ctl[0] = rows, ctl[1] = groups.
// One block of 1024 threads; dynamic shared memory: nb x ceil(nb / 32) words
// of presence bits, (j, i) of every row.
__global__ void __launch_bounds__(1024) k_rows(int n_trip, int nb, int np, int gmax,
                                               const int32_t *__restrict__ ijk, int4 *__restrict__ rows,
                                               int *__restrict__ ctl, int2 *__restrict__ tiles,
                                               int2 *__restrict__ groups) {
    int *n_rows = ctl;
    extern __shared__ uint32_t presence[];
    __shared__ int jstart[ABS_MAX_BINS + 1];
    __shared__ int wsum[32];
    __shared__ int nr_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int words = (nb + 31) / 32;
    auto row_start = [&](int t, int &i, int &j) {
        i = ijk[3 * t];
        j = ijk[3 * t + 1];
        const bool start = t == 0 || i != ijk[3 * t - 3] || j != ijk[3 * t - 2];
        return start && i >= 0 && i <= j && j < nb;   // a checked list has nothing else
    };
    for (int e = threadIdx.x; e < nb * words; e += blockDim.x) presence[e] = 0u;
    for (int e = threadIdx.x; e <= nb; e += blockDim.x) jstart[e] = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < n_trip; t += blockDim.x) {
        int i, j;
        if (row_start(t, i, j)) atomicOr(&presence[j * words + (i >> 5)], 1u << (i & 31));
    }
    __syncthreads();
    // rows per j (distinct (i, j) pairs), exclusive prefix over j (nb <= 1024: one pass)
    int cnt = 0;
    if (threadIdx.x < nb)
        for (int w = 0; w < words; ++w) cnt += __popc(presence[threadIdx.x * words + w]);
    int x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < 32; ++w) {
        if (w < warp) before += wsum[w];
        total += wsum[w];
    }
    if (threadIdx.x < nb) jstart[threadIdx.x] = before + x - cnt;
    if (threadIdx.x == 0) {
        nr_s = total;
        *n_rows = total;
    }
    __syncthreads();
    // every row at (rows of smaller j) + (rows of its j with smaller i)
    for (int t = threadIdx.x; t < n_trip; t += blockDim.x) {
        int i, j;
        if (row_start(t, i, j)) {
            int below = 0;
            for (int w = 0; w < (i >> 5); ++w) below += __popc(presence[j * words + w]);
            below += __popc(presence[j * words + (i >> 5)] & ((1u << (i & 31)) - 1u));
            int e = t + 1;
            while (e < n_trip && ijk[3 * e] == i && ijk[3 * e + 1] == j) ++e;
            rows[jstart[j] + below] = make_int4(i, j, t, e);
        }
    }
    __syncthreads();
    // bands: one warp per tile
    const int nr = nr_s;
    const int ntiles = (nr + TM - 1) / TM;
    for (int tl = warp; tl < ntiles; tl += blockDim.x / 32) {
        int lo = 1 << 30, hi = -1;
        for (int r = tl * TM + lane; r < min(nr, tl * TM + TM); r += 32) {
            const int4 R = rows[r];
            lo = min(lo, ijk[3 * R.z + 2]);
            hi = max(hi, ijk[3 * (R.w - 1) + 2]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = min(lo, __shfl_xor_sync(FULL, lo, o));
            hi = max(hi, __shfl_xor_sync(FULL, hi, o));
        }
        if (lane == 0) {
            lo = max(0, min(lo, nb - 1));
            int w = ((max(hi - lo + 1, 1) + 15) / 16) * 16;
            if (w > np) {   // only for a list that fails its check; stay inside the operand tile
                w = np;
                lo = 0;
            }
            tiles[tl] = make_int2(lo, w);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // greedy groups of consecutive tiles; then again with at most ceil(tiles / groups)
        // tiles a group, so that the groups carry about the same work
        int cap = gmax, ng = 0;
        for (int pass = 0; pass < 2; ++pass) {
            ng = 0;
            for (int t = 0; t < ntiles;) {
                const int first = t;
                int cols = 0;
                while (t < ntiles && t - first < cap && cols + 3 * tiles[t].y <= TMEM_COLS) cols += 3 * tiles[t++].y;
                if (t == first) ++t;   // cannot happen: a band is at most np <= TMEM_COLS / 3
                if (pass == 1) groups[ng] = make_int2(first, t - first);
                ++ng;
            }
            cap = min(gmax, (ntiles + ng - 1) / max(ng, 1));
        }
        ctl[1] = ng;
    }
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

// S[t] = inv_p * sum over splits of partial[split][t] (double-float pairs stored as
// float2): 32 triplets per block, 8 lanes of splits per triplet, summed in
// double-float in a fixed order (deterministic; GB300's FP64 pipe is narrow), the
// total widened to FP64 once.
__global__ void __launch_bounds__(256) k_tc_reduce(int n_trip, int nsplit, double inv_p,
                                                       const double *__restrict__ partial,
                                                       double *__restrict__ S) {
    __shared__ float2 sh[8][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int t = blockIdx.x * 32 + tx;
    const float2 *pf = (const float2 *)partial;
    float2 s = make_float2(0.f, 0.f);
    if (t < n_trip)
        for (int k = ty; k < nsplit; k += 8) s = df2_add(s, pf[(size_t)k * n_trip + t]);
    sh[ty][tx] = s;
    __syncthreads();
    if (ty == 0 && t < n_trip) {
        float2 a = make_float2(0.f, 0.f);
        for (int k = 0; k < 8; ++k) a = df2_add(a, sh[k][tx]);
        S[t] = ((double)a.x + (double)a.y) * inv_p;
    }
}

}  // namespace

// cuTensorMapEncodeTiled from the driver, looked up once (no link against libcuda).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        cudaGetLastError();
    }
    return fn;
}

// Tile groups of the canonical triplet list, worked out on the host the way
// k_rows does on the device (rows by (j, i), 128 a tile, bands rounded to 16,
// greedy groups): sizes the grid.  Lists given by the caller use the tile count.
static int canonical_groups(const Setup &s, int np, int gmax) {
    std::map<std::pair<int, int>, std::pair<int, int>> kr;   // (j, i) -> (first k, last k)
    for (size_t t = 0; t + 2 < s.ijk.size(); t += 3) {
        const auto key = std::make_pair(s.ijk[t + 1], s.ijk[t]);
        auto it = kr.find(key);
        if (it == kr.end()) kr[key] = {s.ijk[t + 2], s.ijk[t + 2]};
        else it->second.second = s.ijk[t + 2];
    }
    std::vector<int> w;
    int n = 0, lo = 1 << 30, hi = -1;
    for (const auto &e : kr) {
        lo = std::min(lo, e.second.first);
        hi = std::max(hi, e.second.second);
        if (++n == TM) {
            w.push_back(std::min(np, ((hi - lo + 1 + 15) / 16) * 16));
            n = 0, lo = 1 << 30, hi = -1;
        }
    }
    if (n > 0) w.push_back(std::min(np, ((hi - lo + 1 + 15) / 16) * 16));
    const int ntiles = (int)w.size();
    int cap = gmax, ng = 0;
    for (int pass = 0; pass < 2; ++pass) {   // as k_rows: greedy, then balanced
        ng = 0;
        for (int t = 0; t < ntiles;) {
            const int first = t;
            int cols = 0;
            while (t < ntiles && t - first < cap && cols + 3 * w[t] <= TMEM_COLS) cols += 3 * w[t++];
            if (t == first) ++t;
            ++ng;
        }
        cap = std::min(gmax, (ntiles + ng - 1) / std::max(ng, 1));
    }
    return std::max(ng, 1);
}

// One launch shape of the kernel: the chunk width and whether a CTA owns a
// group of row tiles (the field chunks brought in once for all of them) or a
// single tile; everything else follows from these and the problem.
struct TcLaunch {
    TcGeom G;
    int KC = 0;
    bool grouped = false;
    int groups = 0, gmax = 1;
    size_t smem = 0;
};

// Shared-memory stages for chunk width kc: at least two of each ring (three
// field stages for the wider chunks), three operand stages if the field ring
// keeps its stages, then as many field stages as fit.  False if they do not fit.
static bool tc_stages(TcGeom &G, int kc, int nb, size_t &smem) {
    const int64_t budget = 215 * 1024;   // dynamic shared memory, below the 227 KB per CTA with the static part
    const size_t epi = (size_t)TM * (3 * G.NP + 1) * 4;
    const int min_f = kc > 64 ? 3 : 2;
    G.a_bytes = TM * kc * 2;
    G.b_bytes = 2 * G.NP * kc * 2;
    G.f_bytes = (int)(cdiv((int64_t)nb * (kc + 4) * 4, 1024) * 1024);
    G.ab_bytes = (int)(cdiv(2 * G.a_bytes + G.b_bytes, 1024) * 1024);
    G.sa = MAX_AB;
    while (G.sa > 2 && budget - (int64_t)G.sa * G.ab_bytes < min_f * (int64_t)G.f_bytes) --G.sa;
    G.sf = (int)std::min<int64_t>(MAX_F, (budget - (int64_t)G.sa * G.ab_bytes) / G.f_bytes);
    if (G.sf < min_f || (int64_t)epi > budget) return false;
    smem = 1024 + std::max((size_t)G.sf * G.f_bytes + (size_t)G.sa * G.ab_bytes, epi);
    return true;
}

// The pixel range of a CTA: whole waves of CTAs, at most 4096 pixels (which
// bounds the FP32 accumulation length in the tensor core), a multiple of kc.
static int64_t tc_range(int64_t P, int kc, int groups, int sm_count) {
    for (int waves = 1;; ++waves) {
        const int64_t ranges = std::max<int64_t>(1, (int64_t)sm_count * waves / groups);
        const int64_t per = cdiv(cdiv(P, ranges), kc) * kc;
        if (per <= 4096) return per;
    }
}

static bool tc_shape(const TcGeom &base, int kc, bool grouped, int tiles, int tc_groups, int nb, int sm_count,
                     TcLaunch &L) {
    L.G = base;
    L.KC = kc;
    if (!tc_stages(L.G, kc, nb, L.smem)) return false;
    L.grouped = grouped && tc_groups < tiles;
    L.groups = L.grouped ? tc_groups : tiles;
    L.gmax = L.grouped ? GMAX : 1;
    L.G.per_split = tc_range(base.P, kc, L.groups, sm_count);
    return true;
}

// k_rows and the kernel for one shape, with events around the kernel when given.
static abs_status tc_run(abs_ctx *ctx, const Setup &s, const TcLaunch &L, const float *d_fields, int32_t n_trip,
                         const int32_t *d_ijk, int max_rows, int tiles, double *partial, cudaEvent_t e0,
                         cudaEvent_t e1) {
    TcGeom G = L.G;
    const int KC = L.KC;
    // the field chunk as one TMA box (KC + 4 pixels x every ring) of the [nb][P] FP32 array; the
    // row pitch P x 4 bytes and the array must be 16-byte aligned, else the loader warp copies
    CUtensorMap fmap;
    memset(&fmap, 0, sizeof fmap);
    G.tma = 0;
    PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (encode && G.P % 4 == 0 && ((uintptr_t)d_fields & 15) == 0) {
        const cuuint64_t dims[2] = {(cuuint64_t)G.P, (cuuint64_t)s.nb};
        const cuuint64_t strides[1] = {(cuuint64_t)G.P * 4};
        const cuuint32_t box[2] = {(cuuint32_t)(KC + 4), (cuuint32_t)s.nb};
        const cuuint32_t estr[2] = {1, 1};
        G.tma = encode(&fmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)d_fields, dims, strides, box, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
    const int64_t nsplit = cdiv(G.P, G.per_split);
    int4 *rows = (int4 *)workspace(ctx, "tc.rows", sizeof(int4) * std::max(max_rows, 1));
    int2 *tl = (int2 *)workspace(ctx, "tc.tiles", sizeof(int2) * std::max(tiles, 1));
    int2 *gr = (int2 *)workspace(ctx, "tc.groups", sizeof(int2) * std::max(tiles, 1));
    int *ctl = (int *)workspace(ctx, "tc.ctl", sizeof(int) * 2);
    if (!rows || !tl || !gr || !ctl) return fail(ctx, ABS_ERR_OOM, "split-BF16 workspace");
    cudaStream_t st = ctx->stream;
    auto kern = KC == 128 ? k_triple_tc<128> : KC == 96 ? k_triple_tc<96> : k_triple_tc<64>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
    {
        StageTimer timer(ctx, e0 ? nullptr : "tc_rows");
        const size_t psmem = sizeof(uint32_t) * (size_t)s.nb * ((s.nb + 31) / 32);
        k_rows<<<1, 1024, psmem, st>>>(n_trip, s.nb, G.NP, L.gmax, d_ijk, rows, ctl, tl, gr);
    }
    StageTimer timer(ctx, e0 ? nullptr : "triple_tc");
    if (e0) cudaEventRecord(e0, st);
    kern<<<dim3(L.groups, (unsigned)nsplit), NT, L.smem, st>>>(G, fmap, d_fields, rows, tl, gr, ctl, d_ijk, partial,
                                                               ctx->d_err);
    if (e1) cudaEventRecord(e1, st);
    return check_launch(ctx, "split-BF16 triple sums");
}

abs_status launch_triple_tc(abs_ctx *ctx, const Setup &s, const float *d_fields, int32_t n_trip,
                            const int32_t *d_ijk, double *d_sum) {
    if (n_trip == 0) return ABS_OK;
    TcGeom G;
    G.nb = s.nb;
    G.NP = (int)cdiv(std::max(s.nb, 16), 16) * 16;
    if (3 * G.NP > TMEM_COLS) return fail(ctx, ABS_ERR_UNSUPPORTED, "split-BF16 accumulators exceed tensor memory");
    G.tmem_cols = TMEM_COLS;
    G.P = (int64_t)s.N * s.N;
    G.n_trip = n_trip;
    const int max_rows = (int)std::min<int64_t>(n_trip, (int64_t)s.nb * (s.nb + 1) / 2);
    const int tiles = (int)cdiv(max_rows, TM);
    Setup &ms = const_cast<Setup &>(s);
    const bool canonical = d_ijk == s.d_ijk;
    if (canonical && ms.tc_groups < 0) ms.tc_groups = canonical_groups(s, G.NP, GMAX);
    const int tc_groups = canonical ? ms.tc_groups : tiles;   // lists given by the caller are not grouped
    // the candidate shapes: every chunk width that fits, each with a tile per CTA and grouped
    std::vector<TcLaunch> cand;
    for (int kc : {128, 96, 64})
        for (bool grp : {false, true}) {
            TcLaunch L;
            if ((!grp || tc_groups < tiles) && tc_shape(G, kc, grp, tiles, tc_groups, s.nb, ctx->sm_count, L))
                cand.push_back(L);
        }
    if (cand.empty()) return fail(ctx, ABS_ERR_UNSUPPORTED, "split-BF16 stages do not fit shared memory");
    int64_t max_split = 1;
    for (const TcLaunch &L : cand) max_split = std::max<int64_t>(max_split, cdiv(G.P, L.G.per_split));
    double *partial = (double *)workspace(ctx, "tc.partial", sizeof(double) * max_split * n_trip);
    if (!partial) return fail(ctx, ABS_ERR_OOM, "split-BF16 workspace");
    // The shape: measured on this configuration's first eager call (autotuner), else
    // the model: the widest chunk, grouped or one tile a CTA by a count of CTA waves x
    // work per CTA in tenths of a tile's chunk step (per chunk 10 per tile plus 3 for
    // bringing the chunk in, 80 per tile for its epilogue; fitted to same-GPU timings).
    auto model = [&]() {
        const TcLaunch *one = nullptr, *grp = nullptr;
        for (const TcLaunch &L : cand) {
            if (L.KC != cand[0].KC) continue;
            (L.grouped ? grp : one) = &L;
        }
        auto makespan = [&](const TcLaunch &L) {
            const int per_group = (int)cdiv(tiles, L.groups);
            const int64_t ctas = L.groups * cdiv(G.P, L.G.per_split);
            return cdiv(ctas, ctx->sm_count) * (cdiv(L.G.per_split, L.KC) * (10 * per_group + 3) + 80 * per_group);
        };
        if (grp && (!one || makespan(*grp) < makespan(*one))) return *grp;
        return *one;
    };
    abs_ctx *root = ctx->parent ? ctx->parent : ctx;
    const TcLaunch *pick = nullptr;
    if (canonical) {
        auto it = root->tc_shapes.find(s.key);
        if (it != root->tc_shapes.end())
            for (const TcLaunch &L : cand)
                if (L.KC == it->second.kc && L.grouped == it->second.grouped) pick = &L;
    }
    TcLaunch chosen;
    if (pick) {
        chosen = *pick;
    } else {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(ctx->stream, &cs);
        const bool tune = canonical && root->autotune && !ctx->profiling && cs == cudaStreamCaptureStatusNone &&
                          ctx->stream != nullptr && cand.size() > 1;
        chosen = model();
        if (tune) {
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            float best = 1e30f;
            if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
                for (const TcLaunch &L : cand) {
                    float ms_min = 1e30f;
                    for (int rep = 0; rep < 2; ++rep) {   // the first run warms caches and the code
                        const abs_status rs = tc_run(ctx, s, L, d_fields, n_trip, d_ijk, max_rows, tiles, partial,
                                                     e0, e1);
                        if (rs != ABS_OK) {
                            cudaEventDestroy(e0);
                            cudaEventDestroy(e1);
                            return rs;
                        }
                        float t = 0.f;
                        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
                            cudaGetLastError();
                            t = 1e30f;
                        }
                        ms_min = std::min(ms_min, t);
                    }
                    if (ms_min < best) {
                        best = ms_min;
                        chosen = L;
                    }
                }
            }
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
            cudaGetLastError();
        }
        if (canonical && (tune || !root->autotune || cand.size() == 1)) {
            abs_ctx::TcShape &c = root->tc_shapes[s.key];
            c.kc = chosen.KC;
            c.grouped = chosen.grouped;
            c.measured = tune;
        }
    }
    const abs_status rs = tc_run(ctx, s, chosen, d_fields, n_trip, d_ijk, max_rows, tiles, partial, nullptr, nullptr);
    if (rs != ABS_OK) return rs;
    const int64_t nsplit = cdiv(G.P, chosen.G.per_split);
    {
        StageTimer timer(ctx, "triple_reduce");
        k_tc_reduce<<<(int)cdiv(n_trip, 32), 256, 0, ctx->stream>>>(n_trip, (int)nsplit,
                                                                   1.0 / ((double)s.N * (double)s.N), partial,
                                                                   d_sum);
    }
    return check_launch(ctx, "split-BF16 triple sums");
}

}  // namespace absk
