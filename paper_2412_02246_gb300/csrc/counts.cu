// Stage 4: exact triangle counts, the denominator of Eq. estimator_t.
//
// With unit-mask fields I_m (X = 1 on the filled cells of a_m) the sum
// N^-2 sum_p I_i I_j I_k is the number T_ijk of ordered closed triangles
// (g1 in a_i, g2 in a_j, g3 in a_k, all filled, g1 + g2 + g3 = 0).  FP32 or
// even FP64 pixel sums cannot return that integer exactly at these sizes, so
// it is counted in integers.  For symmetric cell sets X, Y, Z (closed under
// g -> -g; the origin is in no ring)
//
//   T(X_i, Y_j, Z_k) = 2 #{ (g1, g2) : g1 in X_i upper half plane, g2 in Y_j, g1 + g2 in Z_k }
//
// (the third vertex -(g1+g2) is in Z_k iff g1 + g2 is; negating a triangle
// moves g1 to the other half plane, hence the factor 2).
//
// With A = every cell of the annuli on the grid, F = the filled ones and
// H = A \ F the holes, splitting g1, then g2, then g3 into filled and hole gives
//
//   T(F,F,F) = T(A,A,A) - T(H,A,A) - T(F,H,A) - T(F,F,H),
//
// where T(A,A,A) depends only on the ring geometry (computed once per
// configuration and kept by the context) and every other term has a hole
// among the enumerated pair, so its cost is |H| x ring size instead of
// ring size squared.  T(F,F,H) is enumerated as (g1 in F_i, g3 in H_k) with
// g2 = -(g1+g3) looked up in F.  A device-side estimate picks this route or
// the direct enumeration of T(F,F,F), whichever visits fewer pairs; both are
// exact.
//
// Ring lists are built row-major, so the upper half plane of each ring is
// the second half of its list.  A byte map holds 1 + ring id of every cell of
// a family (0 elsewhere), indexed by |lin(h)| with lin(g) = g_y W + g_x,
// W = 2R + 1: lin is linear and odd, so lin(g1 + g2) = lin(g1) + lin(g2) and
// |lin(h)| = lin(+-h) picks the upper-half-plane representative of h, whose
// ring and membership are those of h.  A pair sum with |h_x| > R is in no ring;
// for |h_x| <= R and |h_y| <= 2R, lin is one-to-one, so a pair is classified
// by one add and compare on x, one add, one abs and one byte load (a map of
// about 4R^2 bytes, in shared memory up to R of about 230).  One CTA per work item
// (pair of rings, chunk of the larger set spread over the threads, chunk of
// the smaller set streamed through shared memory); each thread keeps
// run-length state (consecutive cells in row order usually land in the same
// ring) and adds finished runs into a lane-private shared-memory histogram
// of 16-bit counters (an item adds at most INNER x G1 to one counter)
// over the third ring, reduced into an int64 table at the end.
#include "abs_internal.cuh"

namespace absk {
namespace {

#ifndef ABS_COUNT_G1
#define ABS_COUNT_G1 4
#endif
#ifndef ABS_COUNT_KU
#define ABS_COUNT_KU 4
#endif
constexpr int G1 = ABS_COUNT_G1;   // g1 cells per thread
constexpr int KU = ABS_COUNT_KU;   // inner cells whose map loads are issued together
constexpr int CT = 256;          // threads per counting CTA (max)
constexpr int INNER = 512;       // inner cells per work item (bounds the work of one item)
constexpr unsigned FULL = 0xffffffffu;

struct CountGeom {
    int n, half, nb, R, W;       // W = 2R + 1
    int64_t base;                // 2R W + R: the largest |lin| of a pair sum with |h_x| <= R
};

__device__ __forceinline__ int64_t cell_index(int n, int gx, int gy) {
    return (int64_t)(gy < 0 ? gy + n : gy) * n + (gx < 0 ? gx + n : gx);
}

// floor(sqrt(v)) for 0 <= v < 2^53: an FP32 estimate corrected in integers
// (v here is below 2^26, where the estimate is off by at most one).
__device__ __forceinline__ int64_t isqrt_dev(int64_t v) {
    if (v <= 0) return 0;
    int64_t r = (int64_t)sqrtf((float)v);
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

// Cell families of the ring tables.
enum { FAM_F = 0, FAM_H = 1, FAM_A = 2, NFAM = 3 };
// Pair-count jobs: (set of g1 [upper half], set of g2, map looked up), table.
enum { JOB_DIRECT = 0, JOB_E1 = 1, JOB_E2 = 2, JOB_E3 = 3, JOB_FULL = 4, NJOB = 5 };
__host__ __device__ constexpr int job_x(int j) { return j == JOB_E1 ? FAM_H : j == JOB_FULL ? FAM_A : FAM_F; }
__host__ __device__ constexpr int job_y(int j) {
    return j == JOB_DIRECT ? FAM_F : (j == JOB_E1 || j == JOB_FULL) ? FAM_A : FAM_H;
}
__host__ __device__ constexpr bool job_map_a(int j) { return j == JOB_E1 || j == JOB_E2 || j == JOB_FULL; }

struct Fams {
    const short2 *lists;
    const int64_t *off;   // [NFAM][nb + 1]
    const int32_t *cnt;   // [NFAM][nb]
};

// sqrt(v) of a non-negative integer v < 2^31 as a double-float pair h + l
// (relative error about 2^-46), with 32-bit arithmetic only: GB300's FP64 pipe
// (which also converts 64-bit integers) is too narrow for a square root per
// cell.  v = vf + vr exactly; h is the correctly rounded sqrtf(vf), whose
// residual vf - h^2 one FMA gives exactly; l = (v - h^2) / (2h) is the
// first-order (Newton) correction.
__device__ __forceinline__ void df_sqrt_int(int32_t v, float &h, float &l) {
    const float vf = (float)v;
    const float vr = (float)(v - (int32_t)vf);     // exact: |v - vf| <= ulp(vf) / 2 <= 64
    h = sqrtf(vf);
    if (h == 0.f) {
        l = 0.f;
        return;
    }
    const float r = __fadd_rn(fmaf(-h, h, vf), vr);
    l = __fdiv_rn(r, __fmul_rn(2.f, h));
}

// (sh, sl) += (h, l) in double-float (TwoSum of the high parts, then the low parts).
__device__ __forceinline__ void df_add(float &sh, float &sl, float h, float l) {
    const float t = __fadd_rn(sh, h);
    const float bp = __fsub_rn(t, sh);
    const float e = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bp)), __fsub_rn(h, bp));
    const float lo = __fadd_rn(e, __fadd_rn(sl, l));
    sh = __fadd_rn(t, lo);                          // Fast2Sum renormalisation (|t| >= |lo|)
    sl = __fsub_rn(lo, __fsub_rn(sh, t));
}

// One warp per (ring, row y >= 0): the ring's cells of the upper half plane
// (y > 0, or y = 0 and x > 0) in that row, split into filled (F), hole (H)
// and annulus (A) cells.  Each family list of a ring holds only its upper
// half plane (its lower half is the negation, since every family is closed
// under g -> -g), at a static offset with room for the whole upper half of the
// ring's lattice; a warp reserves its place with one atomic per family and
// batch of 32 cells, so rows land in any order (the counts do not depend on
// it).  Also writes the byte maps of F and A (at lin > 0) and the row's sum of
// |g| over filled cells in double-float.
__global__ void k_ring_cells(CountGeom G, const int64_t *__restrict__ q, const uint8_t *__restrict__ mask,
                             const unsigned long long *__restrict__ accw,
                             const int64_t *__restrict__ ring_off, int32_t *__restrict__ cnt_up,
                             short2 *__restrict__ lists, uint8_t *__restrict__ mapF, uint8_t *__restrict__ mapA,
                             double *__restrict__ rowlen) {
    const int rows = G.R + 1;
    const int64_t nrow = (int64_t)G.nb * rows;
    const int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (e >= nrow) return;
    const int m = e / rows, y = e - m * rows;
    const RowSpan sp = row_span(G, q[m], q[m + 1], y);
    const int len = span_len(sp);
    const unsigned below = (1u << lane) - 1u;
    short2 *LF = lists + ring_off[FAM_F * (G.nb + 1) + m];
    short2 *LH = lists + ring_off[FAM_H * (G.nb + 1) + m];
    short2 *LA = lists + ring_off[FAM_A * (G.nb + 1) + m];
    float sh = 0.f, sl = 0.f;
    for (int t0 = 0; t0 < len; t0 += 32) {
        const int t = t0 + lane;
        int x = 0;
        bool in = t < len;
        if (in) {
            x = span_x(sp, t);
            in = y > 0 || x > 0;
        }
        // filled: the mask, or (accw given) a nonzero weight sum at g or -g
        bool on = false;
        if (in) {
            if (accw) on = accw[cell_index(G.n, x, y)] != 0ull || accw[cell_index(G.n, -x, -y)] != 0ull;
            else on = mask[cell_index(G.n, x, y)] != 0;
        }
        const unsigned bf = __ballot_sync(FULL, on), bh = __ballot_sync(FULL, in && !on);
        const unsigned ba = __ballot_sync(FULL, in);
        int pf = 0, ph = 0, pa = 0;
        if (lane == 0) {
            if (bf) pf = atomicAdd(&cnt_up[FAM_F * G.nb + m], __popc(bf));
            if (bh) ph = atomicAdd(&cnt_up[FAM_H * G.nb + m], __popc(bh));
            if (ba) pa = atomicAdd(&cnt_up[FAM_A * G.nb + m], __popc(ba));
        }
        pf = __shfl_sync(FULL, pf, 0);
        ph = __shfl_sync(FULL, ph, 0);
        pa = __shfl_sync(FULL, pa, 0);
        if (in) {
            const short2 g = make_short2((short)x, (short)y);
            LA[pa + __popc(ba & below)] = g;
            if (on) LF[pf + __popc(bf & below)] = g;
            else LH[ph + __popc(bh & below)] = g;
            const int lin = y * G.W + x;   // > 0 in the upper half plane
            mapA[lin] = (uint8_t)(m + 1);
            if (on) mapF[lin] = (uint8_t)(m + 1);
        }
        if (on) {
            float h, l;
            df_sqrt_int(x * x + y * y, h, l);   // |x|, |y| <= n/2 <= 4096
            df_add(sh, sl, h, l);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(FULL, sh, o), ol = __shfl_xor_sync(FULL, sl, o);
        df_add(sh, sl, oh, ol);
    }
    if (lane == 0) rowlen[e] = (double)sh + (double)sl;
}

// One block: choose the route (direct or holes) from the pair counts it would
// visit, and write the work items of every job it needs: one per (pair a <= b,
// chunk of the larger set, chunk of the smaller set).  Items of jobs that look
// Ring pair (a <= b) of pair index pr = a nb - a (a - 1) / 2 + (b - a): a from the
// quadratic's root in FP32, corrected by whole steps.
__device__ __forceinline__ void pair_of(int pr, int nb, int &a, int &b) {
    const float B = 2.f * (float)nb + 1.f;
    a = (int)((B - sqrtf(fmaxf(B * B - 8.f * (float)pr, 0.f))) * 0.5f);
    a = max(0, min(a, nb - 1));
    while (a > 0 && a * nb - a * (a - 1) / 2 > pr) --a;
    while (a + 1 < nb && (a + 1) * nb - (a + 1) * a / 2 <= pr) ++a;
    b = a + (pr - (a * nb - a * (a - 1) / 2));
}

// up the filled map go to list 0, the annulus map to list 1.
// item = (a, b, outer start, inner start | job << 27 | outer-is-x << 31)
__device__ void count_items_block(int nb, const int32_t *__restrict__ counts, int chunk, int need_full,
                                  int4 *__restrict__ items0, int4 *__restrict__ items1, int cap,
                                  int *__restrict__ ctl, int32_t *__restrict__ err) {
    __shared__ unsigned long long wdir_s, wexc_s;
    __shared__ int use_holes_s;
    __shared__ int wsum[32];
    __shared__ int carry_s[2];
    const int npair = nb * (nb + 1) / 2;
    __shared__ int32_t cs[3 * ABS_MAX_BINS];   // the counts, written by other blocks: read once via L2
    for (int i = threadIdx.x; i < 3 * nb; i += blockDim.x) cs[i] = __ldcg(counts + i);
    const int32_t *cF = cs, *cH = cs + nb, *cA = cs + 2 * nb;
    if (threadIdx.x == 0) {
        wdir_s = 0;
        wexc_s = 0;
        carry_s[0] = carry_s[1] = 0;
    }
    __syncthreads();
    unsigned long long wd = 0, we = 0;
    for (int pr = threadIdx.x; pr < npair; pr += blockDim.x) {
        int a, b;
        pair_of(pr, nb, a, b);
        wd += (unsigned long long)(cF[a] / 2) * cF[b];
        we += (unsigned long long)(cH[a] / 2) * cA[b] + 2ull * (cF[a] / 2) * cH[b];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {   // one shared-memory add per warp, not per thread
        wd += __shfl_xor_sync(FULL, wd, o);
        we += __shfl_xor_sync(FULL, we, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&wdir_s, wd);
        atomicAdd(&wexc_s, we);
    }
    __syncthreads();
    if (threadIdx.x == 0) use_holes_s = wexc_s < wdir_s ? 1 : 0;
    __syncthreads();
    const int use_holes = use_holes_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int jobs[4], nj = 0;
    if (use_holes) {
        jobs[nj++] = JOB_E1;
        jobs[nj++] = JOB_E2;
        jobs[nj++] = JOB_E3;
    } else {
        jobs[nj++] = JOB_DIRECT;
    }
    if (need_full) jobs[nj++] = JOB_FULL;
    // per batch of 1024 pairs: chunk counts, their prefix, then every thread
    // writes items of the batch (pair found by binary search over the prefix)
    __shared__ int b_pos[1025];
    __shared__ int b_ab[1024], b_nic[1024];
    for (int jj = 0; jj < nj; ++jj) {
        const int job = jobs[jj];
        const int lst = job_map_a(job) ? 1 : 0;
        const int32_t *cx = cs + job_x(job) * nb, *cy = cs + job_y(job) * nb;
        // PPT consecutive pairs a thread, blockDim.x * PPT pairs a batch (b_pos holds 1024 + 1)
        constexpr int PPT = 4;
        const int per_batch = (int)blockDim.x * PPT;
        for (int p0 = 0; p0 < npair; p0 += per_batch) {
            int nch[PPT], x = 0;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                const int slot = threadIdx.x * PPT + k, pr = p0 + slot;
                int a = 0, b = 0, n_ic = 1, nchunks = 0;
                bool outer_x = false;
                if (pr < npair) {
                    pair_of(pr, nb, a, b);
                    const int hx = cx[a] / 2, ny = cy[b];
                    outer_x = hx >= ny;
                    const int no = outer_x ? hx : ny, ni = outer_x ? ny : hx;
                    const int n_oc = (no + chunk - 1) / chunk;
                    n_ic = (ni + INNER - 1) / INNER;
                    nchunks = ni > 0 ? n_oc * n_ic : 0;
                }
                nch[k] = nchunks;
                x += nchunks;
                b_ab[slot] = a | b << 8 | (outer_x ? 1 << 16 : 0);
                b_nic[slot] = n_ic;
            }
            const int mine = x;
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
            int run = before + x - mine;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                b_pos[threadIdx.x * PPT + k] = run;
                run += nch[k];
            }
            if (threadIdx.x == 0) b_pos[per_batch] = tot;
            __syncthreads();
            const int base = carry_s[lst];
            int4 *items = lst ? items1 : items0;
            for (int t = threadIdx.x; t < tot; t += blockDim.x) {
                int lo = 0, hi = per_batch - 1;   // last pair q with b_pos[q] <= t
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (b_pos[mid] <= t) lo = mid;
                    else hi = mid - 1;
                }
                const int c = t - b_pos[lo], nic = b_nic[lo], ab = b_ab[lo];
                const int oc = c / nic, ic = c - oc * nic;
                if (base + t < cap)
                    items[base + t] = make_int4(ab & 255, (ab >> 8) & 255, oc * chunk,
                                                (ic * INNER) | (job << 27) | ((ab >> 16) ? (int)0x80000000u : 0));
            }
            __syncthreads();
            if (threadIdx.x == 0) carry_s[lst] += tot;
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        if (carry_s[0] > cap || carry_s[1] > cap) atomicCAS(err, 0, DERR_CAPACITY);
        ctl[0] = min(carry_s[0], cap);   // items in list 0
        ctl[1] = min(carry_s[1], cap);   // items in list 1
        ctl[2] = 0;                      // next item of list 0
        ctl[3] = 0;                      // next item of list 1
        ctl[4] = use_holes;
    }
}

// One warp per (family, ring): full counts (twice the upper half plane) and
// the mean l of the filled cells (the upper half plane has the same mean;
// fixed-order sums over the rows).  With items0 given, every block also
// clears a slice of the pair-count tables, and the last block to finish
// (ticket) chooses the route and writes the work items (count_items_block).
struct ItemArgs {
    int chunk, need_full, cap;
    int4 *items0, *items1;
    int *ctl;
    int32_t *err;
    unsigned *ticket;
    unsigned long long *tabs;   // [4][nb^3], cleared
    unsigned long long *full;   // [nb^3], cleared when need_full
};

__global__ void k_ring_finish(CountGeom G, float du, const int32_t *__restrict__ cnt_up,
                              const double *__restrict__ rowlen, int32_t *__restrict__ counts,
                              double *__restrict__ ellbar, ItemArgs ia) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (ia.items0) {
        const int64_t tw = (int64_t)G.nb * G.nb * G.nb;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 4 * tw;
             i += (int64_t)gridDim.x * blockDim.x) {
            ia.tabs[i] = 0ull;
            if (ia.need_full && i < tw) ia.full[i] = 0ull;
        }
    }
    if (w < NFAM * G.nb) {
        const int fam = w / G.nb, m = w - fam * G.nb;
        const int rows = G.R + 1;
        const int32_t c = cnt_up[fam * G.nb + m];
        double len = 0.0;
        if (fam == FAM_F)
            for (int y = lane; y < rows; y += 32) len += rowlen[(int64_t)m * rows + y];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) len += __shfl_xor_sync(FULL, len, o);
        if (lane == 0) {
            counts[fam * G.nb + m] = 2 * c;
            if (fam == FAM_F && ellbar)
                ellbar[m] = c > 0 ? 2.0 * 3.14159265358979323846 * (double)du * len / (double)c : nan("");
        }
    }
    if (!ia.items0) return;
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ia.ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    count_items_block(G.nb, counts, ia.chunk, ia.need_full, ia.items0, ia.items1, ia.cap, ia.ctl, ia.err);
    if (threadIdx.x == 0) *ia.ticket = 0u;
}

struct GatherArgs {   // T_ijk for the listed triplets, by the last CTA to finish (T == nullptr: none)
    int32_t n_trip;
    const int32_t *ijk;
    const int *ctl;
    int64_t *T;
    unsigned *ticket;
};

template <bool MAP_IN_SMEM>
__global__ void __launch_bounds__(CT) k_count_pairs(CountGeom G, const int4 *__restrict__ items,
                                                    const int *__restrict__ n_items,
                                                    int *__restrict__ next_item, Fams fam,
                                                    const uint8_t *__restrict__ map_g,
                                                    unsigned long long *__restrict__ t0,
                                                    unsigned long long *__restrict__ t1,
                                                    unsigned long long *__restrict__ t2,
                                                    unsigned long long *__restrict__ t3,
                                                    unsigned long long *__restrict__ t4, GatherArgs ga) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int nwarps = blockDim.x >> 5;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int hs = G.nb + 1;                       // histogram slots (0 = none)
    uint16_t *hist = (uint16_t *)smem;             // [nwarps][hs][32]
    uint32_t *hist32 = (uint32_t *)smem;           // the same, as pairs of counters (clearing)
    const int hwords = nwarps * hs * 16;
    int32_t *stage = (int32_t *)(hist + (size_t)nwarps * hs * 32);   // [INNER] lin of the inner cells
    int32_t *stage_x = stage + INNER;                                 // [INNER] their x
    uint8_t *map_s = (uint8_t *)(stage_x + INNER);
    const uint8_t *map = MAP_IN_SMEM ? map_s : map_g;
    const int ni = *n_items;
    if (MAP_IN_SMEM && ni > 0) {
        const int64_t mb = G.base + 1;
        const int64_t nv = mb / 16;
        for (int64_t i = threadIdx.x; i < nv; i += blockDim.x) ((uint4 *)map_s)[i] = ((const uint4 *)map_g)[i];
        for (int64_t i = nv * 16 + threadIdx.x; i < mb; i += blockDim.x) map_s[i] = map_g[i];
    }
    if (ni > 0) {   // nothing to clear when there are no items (a grid without holes)
        for (int i = threadIdx.x; i < hwords; i += blockDim.x) hist32[i] = 0u;
        __syncthreads();
    }
    uint16_t *myhist = hist + (size_t)warp * hs * 32 + lane;
    __shared__ int it_s;
    for (; ni > 0;) {
        if (threadIdx.x == 0) it_s = atomicAdd(next_item, 1);   // dynamic: items differ in size
        __syncthreads();
        const int it = it_s;
        if (it >= ni) break;
        const int4 I = items[it];
        const int a = I.x, b = I.y;
        const bool outer_x = (I.w & 0x80000000) != 0;
        const int job = (I.w >> 27) & 7;
        const int in0 = I.w & 0x07ffffff;
        const int fx = job_x(job), fy = job_y(job);
        const int cxa = fam.cnt[fx * G.nb + a], cyb = fam.cnt[fy * G.nb + b];
        // X_a: its upper half plane; Y_b: whole, as its upper half then its negation
        const short2 *X = fam.lists + fam.off[fx * (G.nb + 1) + a];
        const short2 *Yu = fam.lists + fam.off[fy * (G.nb + 1) + b];
        const int nx = cxa / 2, hy = cyb / 2;
        const int no = outer_x ? nx : cyb;
        const int nin = min(INNER, (outer_x ? cyb : nx) - in0);
        int lin1[G1], xr1[G1];   // lin and x + R of this thread's outer cells
        bool v1[G1];
#pragma unroll
        for (int q = 0; q < G1; ++q) {
            const int k = I.z + q * blockDim.x + threadIdx.x;
            v1[q] = k < no;
            int l = 0, x = 0;
            if (v1[q]) {
                const short2 g = outer_x ? X[k] : Yu[k < hy ? k : k - hy];
                l = g.y * G.W + g.x;
                x = g.x;
                if (!outer_x && k >= hy) {
                    l = -l;
                    x = -x;
                }
            }
            lin1[q] = l;
            // an empty slot fails the x-range test of every lookup (|x2| <= R), so the lookups
            // need no separate validity test
            xr1[q] = v1[q] ? x + G.R : 0x40000000;
        }
        const uint32_t span = 2u * (uint32_t)G.R;   // |x1 + x2| <= R  <=>  x1 + R + x2 in [0, 2R]
        int cur[G1];
        uint32_t cnt[G1];
#pragma unroll
        for (int q = 0; q < G1; ++q) {
            cur[q] = 0;
            cnt[q] = 0;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < nin; k += blockDim.x) {
            const int kk = in0 + k;
            int l, x;
            if (outer_x) {
                const short2 g = Yu[kk < hy ? kk : kk - hy];
                l = g.y * G.W + g.x;
                x = g.x;
                if (kk >= hy) {
                    l = -l;
                    x = -x;
                }
            } else {
                const short2 g = X[kk];
                l = g.y * G.W + g.x;
                x = g.x;
            }
            stage[k] = l;
            stage_x[k] = x;
        }
        __syncthreads();
        // the map loads of KU inner cells are issued before their run-length updates,
        // which never feed a load: KU x G1 lookups in flight per thread
        int k = 0;
        for (; k + KU <= nin; k += KU) {
            int rr[KU][G1];
#pragma unroll
            for (int u = 0; u < KU; ++u) {
                const int l2 = stage[k + u], x2 = stage_x[k + u];
#pragma unroll
                for (int q = 0; q < G1; ++q)
                    rr[u][q] = ((uint32_t)(xr1[q] + x2) <= span) ? (int)map[abs(lin1[q] + l2)] : 0;
            }
#pragma unroll
            for (int u = 0; u < KU; ++u) {
#pragma unroll
                for (int q = 0; q < G1; ++q) {
                    if (rr[u][q] != cur[q]) {
                        myhist[(size_t)cur[q] * 32] += (uint16_t)cnt[q];
                        cur[q] = rr[u][q];
                        cnt[q] = 0;
                    }
                    ++cnt[q];
                }
            }
        }
        for (; k < nin; ++k) {
            const int l2 = stage[k], x2 = stage_x[k];
#pragma unroll
            for (int q = 0; q < G1; ++q) {
                const int r = ((uint32_t)(xr1[q] + x2) <= span) ? (int)map[abs(lin1[q] + l2)] : 0;
                if (r != cur[q]) {
                    myhist[(size_t)cur[q] * 32] += (uint16_t)cnt[q];
                    cur[q] = r;
                    cnt[q] = 0;
                }
                ++cnt[q];
            }
        }
#pragma unroll
        for (int q = 0; q < G1; ++q) myhist[(size_t)cur[q] * 32] += (uint16_t)cnt[q];
        __syncthreads();
        unsigned long long *T = job == JOB_DIRECT ? t0 : job == JOB_E1 ? t1 : job == JOB_E2 ? t2
                                : job == JOB_E3 ? t3 : t4;
        for (int k = 1 + warp; k < hs; k += nwarps) {
            uint64_t sacc = 0;
            for (int w = 0; w < nwarps; ++w) sacc += hist[((size_t)w * hs + k) * 32 + lane];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(FULL, sacc, o);
            if (lane == 0 && sacc)
                atomicAdd(&T[((size_t)a * G.nb + b) * G.nb + (k - 1)], (unsigned long long)sacc);
        }
        __syncthreads();
        for (int k = threadIdx.x; k < hwords; k += blockDim.x) hist32[k] = 0u;
        __syncthreads();
    }
    if (!ga.T) return;
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ga.ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int nb = G.nb;
    const bool holes = __ldcg(ga.ctl + 4) != 0;
    for (int t = threadIdx.x; t < ga.n_trip; t += blockDim.x) {
        const int i = ga.ijk[3 * t], j = ga.ijk[3 * t + 1], k = ga.ijk[3 * t + 2];
        if (i < 0 || j < i || k < j || k >= nb) {
            ga.T[t] = 0;
            continue;
        }
        const size_t ijkx = ((size_t)i * nb + j) * nb + k;
        if (holes) {
            const size_t ikj = ((size_t)i * nb + k) * nb + j;
            ga.T[t] = 2 * ((int64_t)__ldcg(t4 + ijkx) - (int64_t)__ldcg(t1 + ijkx) - (int64_t)__ldcg(t2 + ijkx) -
                           (int64_t)__ldcg(t3 + ikj));
        } else {
            ga.T[t] = 2 * (int64_t)__ldcg(t0 + ijkx);
        }
    }
    if (threadIdx.x == 0) *ga.ticket = 0u;
}

CountGeom cgeom(const Setup &s) {
    CountGeom G;
    G.n = s.n;
    G.half = s.half;
    G.nb = s.nb;
    G.R = s.R;
    G.W = 2 * s.R + 1;
    G.base = (int64_t)2 * s.R * G.W + s.R;   // largest |lin| of a pair sum with |h_x| <= R
    return G;
}

struct RingBufs {
    short2 *lists;
    int32_t *counts;      // [NFAM][nb]
    int64_t *ring_off;    // [NFAM][nb + 1]
    uint8_t *mapF, *mapA;
};

abs_status ring_tables(abs_ctx *ctx, const Setup &s, const uint8_t *d_mask, const double *d_accw, RingBufs &rb,
                       double *d_ellbar, const ItemArgs *ia) {
    const CountGeom G = cgeom(s);
    const int64_t U = std::max<int64_t>(s.up_off.back(), 1);   // upper-half lattice cells, all rings
    const int64_t nrow = (int64_t)s.nb * (s.R + 1);
    rb.lists = (short2 *)workspace(ctx, "ring.lists", sizeof(short2) * NFAM * U);
    rb.counts = (int32_t *)workspace(ctx, "ring.counts", sizeof(int32_t) * NFAM * s.nb);
    rb.ring_off = s.d_ring_off;
    const int64_t mb = cdiv(G.base + 1, 16) * 16;
    // byte maps of F and A, then the upper-half-plane counters: cleared together
    uint8_t *maps = (uint8_t *)workspace(ctx, "ring.maps", (size_t)2 * mb + sizeof(int32_t) * NFAM * s.nb);
    double *rowlen = (double *)workspace(ctx, "ring.rowlen", sizeof(double) * nrow);
    if (!rb.lists || !rb.counts || !maps || !rowlen) return fail(ctx, ABS_ERR_OOM, "ring table workspace");
    rb.mapF = maps;
    rb.mapA = maps + mb;
    int32_t *cnt_up = (int32_t *)(maps + 2 * mb);
    StageTimer timer(ctx, "ring_lists");
    cudaStream_t st = ctx->stream;
    cudaMemsetAsync(maps, 0, (size_t)2 * mb + sizeof(int32_t) * NFAM * s.nb, st);
    k_ring_cells<<<(int)cdiv(nrow * 32, 256), 256, 0, st>>>(G, s.d_q, d_mask, (const unsigned long long *)d_accw,
                                                            rb.ring_off, cnt_up, rb.lists,
                                                            rb.mapF, rb.mapA, rowlen);
    ItemArgs none{};
    int blocks = (int)cdiv((int64_t)NFAM * s.nb * 32, 256);
    if (ia) {   // enough blocks to clear the pair-count tables quickly
        const int64_t tw = (int64_t)s.nb * s.nb * s.nb;
        blocks = (int)std::max<int64_t>(blocks, std::min<int64_t>(cdiv(4 * tw, 256 * 8), ctx->sm_count));
    }
    k_ring_finish<<<blocks, 256, 0, st>>>(G, s.du, cnt_up, rowlen, rb.counts, d_ellbar, ia ? *ia : none);
    return check_launch(ctx, "ring lists");
}

template <bool SMEM>
void launch_pairs(abs_ctx *ctx, const CountGeom &G, int blocks, int threads, size_t smem, const int4 *items,
                  const int *n_items, int *next, const Fams &fam, const uint8_t *map,
                  unsigned long long *const *tab, const GatherArgs &ga) {
    allow_smem(k_count_pairs<SMEM>, smem);
    k_count_pairs<SMEM><<<blocks, threads, smem, ctx->stream>>>(G, items, n_items, next, fam, map, tab[0], tab[1],
                                                               tab[2], tab[3], tab[4], ga);
}

}  // namespace

abs_status launch_counts(abs_ctx *ctx, const Setup &s, const uint8_t *d_mask, int32_t n_trip,
                         const int32_t *d_ijk, int64_t *d_count, double *d_ellbar, const double *d_accw) {
    if (n_trip == 0 || !d_count) {
        RingBufs rb;
        return ring_tables(ctx, s, d_mask, d_accw, rb, d_ellbar, nullptr);
    }
    const CountGeom G = cgeom(s);
    const int hs = s.nb + 1;
    const int64_t map_bytes = cdiv(G.base + 1, 16) * 16;
    const size_t hist_budget = 96 * 1024;
    int nwarps = (int)std::min<size_t>(CT / 32, hist_budget / ((size_t)hs * 32 * 2));
    if (nwarps < 1) return fail(ctx, ABS_ERR_UNSUPPORTED, "too many rings for the count kernel");
    const int threads = nwarps * 32;
    const int chunk = threads * G1;
    const int64_t hist_bytes = (int64_t)nwarps * hs * 32 * 2;
    const bool map_smem = map_bytes + hist_bytes + INNER * 8 <= 220 * 1024;
    const size_t smem = (size_t)hist_bytes + INNER * 8 + (map_smem ? map_bytes : 0);
    // resident CTAs an SM (shared memory, threads and registers), for the persistent grid
    int per_sm = 1;
    if (map_smem) {
        allow_smem(k_count_pairs<true>, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_count_pairs<true>, threads, smem);
    } else {
        allow_smem(k_count_pairs<false>, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_count_pairs<false>, threads, smem);
    }
    per_sm = std::max(per_sm, 1);
    int64_t max_ring = 0;
    for (int m = 0; m < s.nb; ++m) max_ring = std::max<int64_t>(max_ring, s.lat[m]);
    const int64_t npair = (int64_t)s.nb * (s.nb + 1) / 2;
    const int64_t mr = std::max<int64_t>(max_ring, 1);
    const int cap = (int)std::min<int64_t>(4 * npair * cdiv(mr, chunk) * cdiv(mr, INNER), 1 << 26);
    int4 *items0 = (int4 *)workspace(ctx, "count.items0", sizeof(int4) * cap);
    int4 *items1 = (int4 *)workspace(ctx, "count.items1", sizeof(int4) * cap);
    int *ctl = (int *)workspace(ctx, "count.ctl", sizeof(int) * 8);
    unsigned *tickets = (unsigned *)workspace_zeroed(ctx, "count.tickets", 2 * sizeof(unsigned));
    const size_t tb = sizeof(unsigned long long) * (size_t)s.nb * s.nb * s.nb;
    unsigned long long *tabs = (unsigned long long *)workspace(ctx, "count.tables", 4 * tb);
    // full-annulus counts: a property of the ring geometry, kept per configuration
    Setup &ms = const_cast<Setup &>(s);
    if (!ms.d_full_counts) {
        if (cudaMalloc(&ms.d_full_counts, tb) != cudaSuccess) {
            cudaGetLastError();
            ms.d_full_counts = nullptr;
        }
    }
    if (!items0 || !items1 || !ctl || !tickets || !tabs || !ms.d_full_counts)
        return fail(ctx, ABS_ERR_OOM, "count workspace");
    const int need_full = ms.full_counts_ready ? 0 : 1;
    unsigned long long *tab[NJOB] = {tabs, tabs + tb / 8, tabs + 2 * (tb / 8), tabs + 3 * (tb / 8), ms.d_full_counts};
    // ring tables; their last block also clears the tables and writes the work items
    RingBufs rb;
    const ItemArgs ia{chunk, need_full, cap, items0, items1, ctl, ctx->d_err, tickets, tabs, ms.d_full_counts};
    abs_status st = ring_tables(ctx, s, d_mask, d_accw, rb, d_ellbar, &ia);
    if (st != ABS_OK) return st;
    Fams fam{rb.lists, rb.ring_off, rb.counts};
    {
        // pairs against each byte map; the last CTA of the second launch gathers T
        StageTimer timer(ctx, "count_pairs");
        const int blocks = ctx->sm_count * per_sm;
        const GatherArgs g0{0, nullptr, nullptr, nullptr, nullptr};
        const GatherArgs g1{n_trip, d_ijk, ctl, d_count, tickets + 1};
        if (map_smem) {
            launch_pairs<true>(ctx, G, blocks, threads, smem, items0, ctl + 0, ctl + 2, fam, rb.mapF, tab, g0);
            launch_pairs<true>(ctx, G, blocks, threads, smem, items1, ctl + 1, ctl + 3, fam, rb.mapA, tab, g1);
        } else {
            launch_pairs<false>(ctx, G, blocks, threads, smem, items0, ctl + 0, ctl + 2, fam, rb.mapF, tab, g0);
            launch_pairs<false>(ctx, G, blocks, threads, smem, items1, ctl + 1, ctl + 3, fam, rb.mapA, tab, g1);
        }
    }
    ms.full_counts_ready = true;
    return check_launch(ctx, "counts");
}

abs_status launch_ellbar(abs_ctx *ctx, const Setup &s, const uint8_t *d_mask, double *d_ellbar) {
    RingBufs rb;
    return ring_tables(ctx, s, d_mask, nullptr, rb, d_ellbar, nullptr);
}

}  // namespace absk
