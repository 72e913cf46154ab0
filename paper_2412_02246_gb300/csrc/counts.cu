// Stage 4: exact triangle counts, the denominator of Eq. estimator_t.
//
// With unit-mask fields I_m (X = 1 on the filled cells of a_m) the sum
// N^-2 sum_p I_i I_j I_k is the number T_ijk of ordered closed triangles
// (g1 in a_i, g2 in a_j, g3 in a_k, all filled, g1 + g2 + g3 = 0).  FP32 or
// even FP64 pixel sums cannot return that integer exactly at these sizes, so
// it is counted directly in integers:
//
//   T_ijk = 2 #{ (g1, g2) : g1 in F_i upper half plane, g2 in F_j, g1 + g2 in F_k }
//
// (F_m = filled cells of ring m.  F_k is symmetric under g -> -g, so the
// third vertex -(g1+g2) is in F_k iff g1 + g2 is; negating a triangle maps
// g1 to the other half plane, hence the factor 2; the origin is in no ring.)
//
// Ring lists are built row-major, so the upper half plane of each ring is
// the second half of its list.  A byte map holds 1 + ring id of every filled
// ring cell (0 elsewhere), indexed by |lin(h)| with lin(g) = g_y W + g_x,
// W = 4R + 1: lin is linear and odd, so lin(g1 + g2) = lin(g1) + lin(g2) and
// |lin(h)| = lin(+-h) picks the upper-half-plane representative of h, whose
// ring and filled state are those of h.  A pair is then classified by one
// add, one abs and one byte load, with no bounds test, from a map half the
// size of [-2R, 2R]^2.  One CTA per (i, j,
// chunk of g1) streams all of F_j through shared memory; each thread keeps
// run-length state for its g1 cells (consecutive g2 in row order usually
// land in the same ring) and adds finished runs into a lane-private
// shared-memory histogram over k, which is reduced into an int64 (i, j, k)
// table at the end.  Of the two sets of a pair (upper half of F_i, all of
// F_j) the larger is spread over the threads and the smaller is streamed, so
// that no thread idles through a pass over a large ring.
#include "abs_internal.cuh"

namespace absk {
namespace {

constexpr int G1 = 4;            // g1 cells per thread
constexpr int CT = 256;          // threads per counting CTA (max)
constexpr int STAGE = 2048;      // inner cells staged per pass
constexpr int INNER = 512;       // inner cells per work item (bounds the work of one item)
constexpr unsigned FULL = 0xffffffffu;

struct CountGeom {
    int n, half, nb, R, W;       // W = 4R + 1
    int64_t base;                // 2R W + 2R
};

__device__ __forceinline__ int64_t cell_index(int n, int gx, int gy) {
    return (int64_t)(gy < 0 ? gy + n : gy) * n + (gx < 0 ? gx + n : gx);
}

__device__ __forceinline__ int64_t isqrt_dev(int64_t v) {
    if (v <= 0) return 0;
    int64_t r = (int64_t)sqrt((double)v);
    while (r * r > v) --r;
    while ((r + 1) * (r + 1) <= v) ++r;
    return r;
}

// Cells of ring m in row y (|y| <= R): x in [-x1, -x0] and [x0, x1] clipped to
// the grid (x0 = 0 contributes the single column x = 0 once).
struct RowSpan {
    int x0, x1;
    bool ok;
};
__device__ __forceinline__ RowSpan row_span(const CountGeom &G, int64_t q0, int64_t q1, int y) {
    RowSpan r{0, -1, false};
    if (y < -G.half || y > G.half) return r;
    const int64_t y2 = (int64_t)y * y;
    const int64_t hi = q1 - 1 - y2;
    if (hi < 0) return r;
    const int64_t lo = q0 - y2;
    int64_t x0 = lo <= 0 ? 0 : isqrt_dev(lo - 1) + 1;   // smallest x >= 0 with x^2 >= lo
    int64_t x1 = isqrt_dev(hi);
    if (x1 > G.half) x1 = G.half;
    if (x0 > x1) return r;
    r.x0 = (int)x0;
    r.x1 = (int)x1;
    r.ok = true;
    return r;
}

// x of the t-th cell of the row span (left part -x1..-x0, then x0..x1).
__device__ __forceinline__ int span_x(const RowSpan &sp, int t) {
    if (sp.x0 == 0) return -sp.x1 + t;
    const int n1 = sp.x1 - sp.x0 + 1;
    return t < n1 ? -sp.x1 + t : sp.x0 + (t - n1);
}
__device__ __forceinline__ int span_len(const RowSpan &sp) {
    if (!sp.ok) return 0;
    return sp.x0 == 0 ? 2 * sp.x1 + 1 : 2 * (sp.x1 - sp.x0 + 1);
}

// Pass 1 (one warp per (ring, row)): filled cells and FP64 sum of |g|.
__global__ void k_ring_rows(CountGeom G, const int64_t *__restrict__ q, const uint8_t *__restrict__ mask,
                            uint32_t *__restrict__ rowcnt, double *__restrict__ rowlen) {
    const int rows = 2 * G.R + 1;
    const int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (e >= G.nb * rows) return;
    const int m = e / rows, y = e - m * rows - G.R;
    const RowSpan sp = row_span(G, q[m], q[m + 1], y);
    const int len = span_len(sp);
    uint32_t c = 0;
    double sum = 0.0;
    for (int t0 = 0; t0 < len; t0 += 32) {
        const int t = t0 + lane;
        bool on = false;
        int x = 0;
        if (t < len) {
            x = span_x(sp, t);
            on = mask[cell_index(G.n, x, y)] != 0;
        }
        c += __popc(__ballot_sync(FULL, on));
        if (on) sum += sqrt((double)x * x + (double)y * y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(FULL, sum, o);
    if (lane == 0) {
        rowcnt[e] = c;
        rowlen[e] = sum;
    }
}

// Pass 2 (one warp per (ring, row)): write the cells in x order and the byte map.
__global__ void k_ring_write(CountGeom G, const int64_t *__restrict__ q, const uint8_t *__restrict__ mask,
                             const uint32_t *__restrict__ rowoff, short2 *__restrict__ lists,
                             uint8_t *__restrict__ binmap) {
    const int rows = 2 * G.R + 1;
    const int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (e >= G.nb * rows) return;
    const int m = e / rows, y = e - m * rows - G.R;
    const RowSpan sp = row_span(G, q[m], q[m + 1], y);
    const int len = span_len(sp);
    uint32_t pos = rowoff[e];
    for (int t0 = 0; t0 < len; t0 += 32) {
        const int t = t0 + lane;
        bool on = false;
        int x = 0;
        if (t < len) {
            x = span_x(sp, t);
            on = mask[cell_index(G.n, x, y)] != 0;
        }
        const unsigned bal = __ballot_sync(FULL, on);
        if (on) {
            lists[pos + __popc(bal & ((1u << lane) - 1u))] = make_short2((short)x, (short)y);
            const int lin = y * G.W + x;
            if (lin > 0) binmap[lin] = (uint8_t)(m + 1);
        }
        pos += __popc(bal);
    }
}

// Pass 3 (one warp per ring): ring offsets, counts and mean l (fixed-order sums).
__global__ void k_ring_finish(CountGeom G, float du, const uint32_t *__restrict__ rowoff,
                              const uint32_t *__restrict__ rowcnt, const double *__restrict__ rowlen,
                              int64_t *__restrict__ ring_off, int32_t *__restrict__ counts,
                              double *__restrict__ ellbar) {
    const int m = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (m >= G.nb) return;
    const int rows = 2 * G.R + 1;
    const int64_t e0 = (int64_t)m * rows, e1 = e0 + rows;
    const uint32_t start = rowoff[e0];
    const uint32_t c = rowoff[e1 - 1] + rowcnt[e1 - 1] - start;
    double len = 0.0;
    for (int64_t e = e0 + lane; e < e1; e += 32) len += rowlen[e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) len += __shfl_xor_sync(FULL, len, o);
    if (lane == 0) {
        ring_off[m] = start;
        counts[m] = (int32_t)c;
        if (m == G.nb - 1) ring_off[G.nb] = start + c;
        if (ellbar) ellbar[m] = c > 0 ? 2.0 * 3.14159265358979323846 * (double)du * len / (double)c : nan("");
    }
}

// One block: the (i, j, first g1) work items for every distinct (i, j) row of
// the triplet list.  A list that is not canonical latches an error.
__global__ void __launch_bounds__(1024) k_count_items(int nb, int32_t n_trip,
                                                      const int32_t *__restrict__ ijk,
                                                      const int32_t *__restrict__ counts, int chunk,
                                                      int4 *__restrict__ items, int cap,
                                                      int *__restrict__ n_items,
                                                      int32_t *__restrict__ err) {
    __shared__ int32_t wsum[32];
    __shared__ int32_t carry_s;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int b = 0; b < n_trip; b += blockDim.x) {
        const int t = b + threadIdx.x;
        int nchunks = 0, i = 0, j = 0, n_in = 0, n_oc = 0, n_ic = 1;
        bool outer_i = false;
        if (t < n_trip) {
            i = ijk[3 * t];
            j = ijk[3 * t + 1];
            const int k = ijk[3 * t + 2];
            if (i < 0 || j < i || k < j || k >= nb) atomicCAS(err, 0, DERR_TRIPLET_BIN);
            bool row_start = true;
            if (t > 0) {
                const int pi = ijk[3 * t - 3], pj = ijk[3 * t - 2], pk = ijk[3 * t - 1];
                const bool same = pi == i && pj == j;
                row_start = !same;
                const bool ordered = pi < i || (pi == i && (pj < j || (pj == j && pk < k)));
                if (!ordered) atomicCAS(err, 0, DERR_TRIPLET_ORDER);
            }
            if (row_start && i >= 0 && i < nb && j >= 0 && j < nb) {
                const int half_i = counts[i] / 2, cj = counts[j];
                outer_i = half_i >= cj;
                n_in = outer_i ? cj : half_i;
                n_oc = ((outer_i ? half_i : cj) + chunk - 1) / chunk;
                n_ic = (n_in + INNER - 1) / INNER;
                nchunks = n_oc * n_ic;
            }
        }
        // block exclusive scan of nchunks (small values; warp-level then serial over warps)
        int x = nchunks;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        int before = 0, tot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            if (w < warp) before += wsum[w];
            tot += wsum[w];
        }
        const int pos = carry_s + before + x - nchunks;
        for (int c = 0; c < nchunks; ++c) {
            const int oc = c / n_ic, ic = c - oc * n_ic;
            if (pos + c < cap)
                items[pos + c] = make_int4(i, j, oc * chunk, (ic * INNER) | (outer_i ? (int)0x80000000u : 0));
        }
        __syncthreads();
        if (threadIdx.x == 0) carry_s += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *n_items = min(carry_s, cap);
}

template <bool MAP_IN_SMEM>
__global__ void __launch_bounds__(CT) k_count_pairs(CountGeom G, const int4 *__restrict__ items,
                                                    const int *__restrict__ n_items,
                                                    const short2 *__restrict__ lists,
                                                    const int64_t *__restrict__ ring_off,
                                                    const int32_t *__restrict__ counts,
                                                    const uint8_t *__restrict__ binmap_g,
                                                    unsigned long long *__restrict__ Td,
                                                    int *__restrict__ next_item) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int nwarps = blockDim.x >> 5;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int hs = G.nb + 1;                       // histogram slots (0 = no ring)
    uint32_t *hist = (uint32_t *)smem;             // [nwarps][hs][32]
    int32_t *stage = (int32_t *)(hist + (size_t)nwarps * hs * 32);   // [STAGE]
    uint8_t *map_s = (uint8_t *)(stage + STAGE);
    const uint8_t *map = MAP_IN_SMEM ? map_s : binmap_g;
    if (MAP_IN_SMEM) {
        const int64_t mb = G.base + 1;
        const int64_t nv = mb / 16;
        for (int64_t i = threadIdx.x; i < nv; i += blockDim.x)
            ((uint4 *)map_s)[i] = ((const uint4 *)binmap_g)[i];
        for (int64_t i = nv * 16 + threadIdx.x; i < mb; i += blockDim.x) map_s[i] = binmap_g[i];
    }
    for (int i = threadIdx.x; i < nwarps * hs * 32; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    uint32_t *myhist = hist + (size_t)warp * hs * 32 + lane;
    __shared__ int it_s;
    const int ni = *n_items;
    for (;;) {
        if (threadIdx.x == 0) it_s = atomicAdd(next_item, 1);   // dynamic: items differ in size
        __syncthreads();
        const int it = it_s;
        if (it >= ni) break;
        const int4 I = items[it];
        const int i = I.x, j = I.y;
        const bool outer_i = (I.w & 0x80000000) != 0;
        const int in0 = I.w & 0x7fffffff;
        const int ci = counts[i], cj = counts[j];
        const short2 *Fi = lists + ring_off[i] + ci / 2;   // upper half plane of ring i
        const short2 *Fj = lists + ring_off[j];
        const int nh = ci / 2;
        // outer set: spread over the threads; inner set: streamed through shared memory
        const short2 *Fo = outer_i ? Fi : Fj;
        const short2 *Fin = (outer_i ? Fj : Fi) + in0;
        const int no = outer_i ? nh : cj;
        const int nin = min(INNER, (outer_i ? cj : nh) - in0);
        int lin1[G1];
        bool v1[G1];
#pragma unroll
        for (int q = 0; q < G1; ++q) {
            const int a = I.z + q * blockDim.x + threadIdx.x;
            v1[q] = a < no;
            const short2 g = v1[q] ? Fo[a] : make_short2(0, 0);
            lin1[q] = g.y * G.W + g.x;
        }
        int cur[G1];
        uint32_t cnt[G1];
#pragma unroll
        for (int q = 0; q < G1; ++q) {
            cur[q] = 0;
            cnt[q] = 0;
        }
        for (int s0 = 0; s0 < nin; s0 += STAGE) {
            const int ns = min(STAGE, nin - s0);
            __syncthreads();
            for (int a = threadIdx.x; a < ns; a += blockDim.x) {
                const short2 g = Fin[s0 + a];
                stage[a] = g.y * G.W + g.x;
            }
            __syncthreads();
            for (int a = 0; a < ns; ++a) {
                const int l2 = stage[a];
#pragma unroll
                for (int q = 0; q < G1; ++q) {
                    const int k = v1[q] ? (int)map[abs(lin1[q] + l2)] : 0;
                    if (k != cur[q]) {
                        myhist[(size_t)cur[q] * 32] += cnt[q];
                        cur[q] = k;
                        cnt[q] = 0;
                    }
                    ++cnt[q];
                }
            }
        }
#pragma unroll
        for (int q = 0; q < G1; ++q) myhist[(size_t)cur[q] * 32] += cnt[q];
        __syncthreads();
        // reduce lanes and warps; slot 0 (no ring) is dropped
        for (int k = 1 + warp; k < hs; k += nwarps) {
            uint64_t s = 0;
            for (int w = 0; w < nwarps; ++w) s += hist[((size_t)w * hs + k) * 32 + lane];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
            if (lane == 0 && s)
                atomicAdd(&Td[((size_t)i * G.nb + j) * G.nb + (k - 1)], (unsigned long long)s);
        }
        __syncthreads();
        for (int a = threadIdx.x; a < nwarps * hs * 32; a += blockDim.x) hist[a] = 0u;
        __syncthreads();
    }
}

__global__ void k_count_gather(int nb, int32_t n_trip, const int32_t *__restrict__ ijk,
                               const unsigned long long *__restrict__ Td, int64_t *__restrict__ T) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_trip) return;
    const int i = ijk[3 * t], j = ijk[3 * t + 1], k = ijk[3 * t + 2];
    if (i < 0 || j < 0 || k < 0 || i >= nb || j >= nb || k >= nb) {
        T[t] = 0;
        return;
    }
    T[t] = 2 * (int64_t)Td[((size_t)i * nb + j) * nb + k];
}

CountGeom cgeom(const Setup &s) {
    CountGeom G;
    G.n = s.n;
    G.half = s.half;
    G.nb = s.nb;
    G.R = s.R;
    G.W = 4 * s.R + 1;
    G.base = (int64_t)2 * s.R * G.W + 2 * s.R;   // largest |lin| of a pair sum
    return G;
}

struct RingBufs {
    short2 *lists;
    int32_t *counts;
    int64_t *ring_off;
    uint8_t *binmap;
};

abs_status ring_tables(abs_ctx *ctx, const Setup &s, const uint8_t *d_mask, RingBufs &rb,
                       double *d_ellbar) {
    const CountGeom G = cgeom(s);
    const int64_t ncell = std::max<int64_t>(s.lat_off.back(), 1);
    const int64_t nrow = (int64_t)s.nb * (2 * s.R + 1);
    rb.lists = (short2 *)workspace(ctx, "ring.lists", sizeof(short2) * ncell);
    rb.counts = (int32_t *)workspace(ctx, "ring.counts", sizeof(int32_t) * s.nb);
    rb.ring_off = (int64_t *)workspace(ctx, "ring.off", sizeof(int64_t) * (s.nb + 1));
    const int64_t mb = G.base + 1;
    rb.binmap = (uint8_t *)workspace(ctx, "ring.binmap", (size_t)cdiv(mb, 16) * 16);
    uint32_t *rowcnt = (uint32_t *)workspace(ctx, "ring.rowcnt", sizeof(uint32_t) * nrow);
    uint32_t *rowoff = (uint32_t *)workspace(ctx, "ring.rowoff", sizeof(uint32_t) * nrow);
    double *rowlen = (double *)workspace(ctx, "ring.rowlen", sizeof(double) * nrow);
    uint32_t *bsum = (uint32_t *)workspace(ctx, "ring.bsum", sizeof(uint32_t) * (cdiv(nrow, 4096) + 1));
    if (!rb.lists || !rb.counts || !rb.ring_off || !rb.binmap || !rowcnt || !rowoff || !rowlen || !bsum)
        return fail(ctx, ABS_ERR_OOM, "ring table workspace");
    StageTimer timer(ctx, "ring_lists");
    cudaStream_t st = ctx->stream;
    cudaMemsetAsync(rb.binmap, 0, (size_t)cdiv(mb, 16) * 16, st);
    const int nbk = (int)cdiv(nrow * 32, 256);
    k_ring_rows<<<nbk, 256, 0, st>>>(G, s.d_q, d_mask, rowcnt, rowlen);
    scan_u32(st, rowcnt, nrow, rowoff, bsum);
    k_ring_write<<<nbk, 256, 0, st>>>(G, s.d_q, d_mask, rowoff, rb.lists, rb.binmap);
    k_ring_finish<<<(int)cdiv((int64_t)s.nb * 32, 256), 256, 0, st>>>(G, s.du, rowoff, rowcnt, rowlen,
                                                                       rb.ring_off, rb.counts, d_ellbar);
    return check_launch(ctx, "ring lists");
}

}  // namespace

abs_status launch_counts(abs_ctx *ctx, const Setup &s, const uint8_t *d_mask, int32_t n_trip,
                         const int32_t *d_ijk, int64_t *d_count, double *d_ellbar) {
    RingBufs rb;
    abs_status st = ring_tables(ctx, s, d_mask, rb, d_ellbar);
    if (st != ABS_OK) return st;
    if (n_trip == 0 || !d_count) return ABS_OK;
    const CountGeom G = cgeom(s);
    // threads per CTA: lane-private histograms must fit next to the map
    const int hs = s.nb + 1;
    const int64_t map_bytes = cdiv(G.base + 1, 16) * 16;
    const size_t hist_budget = 96 * 1024;
    int nwarps = (int)std::min<size_t>(CT / 32, hist_budget / ((size_t)hs * 32 * 4));
    if (nwarps < 1) return fail(ctx, ABS_ERR_UNSUPPORTED, "too many rings for the count kernel");
    const int64_t cta_bytes = map_bytes + (int64_t)nwarps * hs * 32 * 4 + STAGE * 4;
    const bool map_smem = cta_bytes <= 220 * 1024;
    const int per_sm = map_smem ? std::max<int>(1, (int)std::min<int64_t>(4, (226 * 1024) / (cta_bytes + 1024))) : 2;
    const int threads = nwarps * 32;
    const int chunk = threads * G1;
    const size_t smem = (size_t)nwarps * hs * 32 * 4 + STAGE * 4 + (map_smem ? map_bytes : 0);
    // work items: one per (row, chunk of the upper half of ring i)
    int64_t max_ring = 0;
    for (int m = 0; m < s.nb; ++m) max_ring = std::max<int64_t>(max_ring, s.lat[m]);
    const int64_t max_rows = std::min<int64_t>(n_trip, (int64_t)s.nb * (s.nb + 1) / 2);
    const int64_t mr = std::max<int64_t>(max_ring, 1);
    const int cap = (int)std::min<int64_t>(max_rows * cdiv(mr, chunk) * cdiv(mr, INNER), 1 << 26);
    int4 *items = (int4 *)workspace(ctx, "count.items", sizeof(int4) * cap);
    int *n_items = (int *)workspace(ctx, "count.n_items", sizeof(int) * 2);   // [count, next]
    const size_t td_bytes = sizeof(unsigned long long) * (size_t)s.nb * s.nb * s.nb;
    unsigned long long *Td = (unsigned long long *)workspace(ctx, "count.table", td_bytes);
    if (!items || !n_items || !Td) return fail(ctx, ABS_ERR_OOM, "count workspace");
    cudaStream_t stm = ctx->stream;
    {
        StageTimer timer(ctx, "count_items");
        cudaMemsetAsync(Td, 0, td_bytes, stm);
        cudaMemsetAsync(n_items, 0, sizeof(int) * 2, stm);
        k_count_items<<<1, 1024, 0, stm>>>(s.nb, n_trip, d_ijk, rb.counts, chunk, items, cap, n_items,
                                           ctx->d_err);
    }
    {
    StageTimer timer(ctx, "count_pairs");
    const int blocks = ctx->sm_count * per_sm;
    if (map_smem) {
        cudaFuncSetAttribute(k_count_pairs<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_count_pairs<true><<<blocks, threads, smem, stm>>>(G, items, n_items, rb.lists, rb.ring_off,
                                                            rb.counts, rb.binmap, Td, n_items + 1);
    } else {
        cudaFuncSetAttribute(k_count_pairs<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_count_pairs<false><<<blocks, threads, smem, stm>>>(G, items, n_items, rb.lists, rb.ring_off,
                                                             rb.counts, rb.binmap, Td, n_items + 1);
    }
    }
    {
        StageTimer t2(ctx, "count_gather");
        k_count_gather<<<(int)cdiv(n_trip, 256), 256, 0, stm>>>(s.nb, n_trip, d_ijk, Td, d_count);
    }
    return check_launch(ctx, "counts");
}

abs_status launch_ellbar(abs_ctx *ctx, const Setup &s, const uint8_t *d_mask, double *d_ellbar) {
    RingBufs rb;
    return ring_tables(ctx, s, d_mask, rb, d_ellbar);
}

}  // namespace absk
