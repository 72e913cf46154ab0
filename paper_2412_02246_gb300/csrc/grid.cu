// Stage 1: gridding of visibilities, Eq. vg (Sec. 2).
//
// V_g = sum_i w(U_g - U_i) V(U_i) over the (2r+1)^2 cells around each
// visibility's nearest grid point, every visibility also entered at -U_i with
// V*.  The mirror is applied after accumulation (G(g) + conj G(-g)), which is
// the same sum.
//
// Plan (per baseline set): key every visibility by its 16x16-cell uv tile and
// its cell in the tile, stable-sort by that key (LSD radix, two passes up to
// about 2040^2 cells, three beyond), and write the sorted positions and
// original indices; the sorted order is cut into work units of UMAX records.
//
// Accumulation (per realisation): one CTA per unit stages the unit in shared
// memory, forms the 1-D Gaussian weights and cuts it into runs of
// visibilities that share a cell (and at every CHUNK-th record); a warp sums
// the (2r+1)^2 footprint cells of a run (lane per pair of footprint cells,
// compensated FP32, input order) and adds them to an FP64 grid.  A final pass
// applies the Hermitian mirror and writes the FP32 outputs.
//
// Weights: w = exp(-(dx - fx)^2 s) exp(-(dy - fy)^2 s), s = 1/(2 sigma^2),
// with the fractional offset f = u/dU - c carried as a float pair (the exact
// division residual) and the exponent argument formed in double-float, so
// that the only sizeable error is that of expf itself.
#include <algorithm>

#include "abs_internal.cuh"

namespace absk {
namespace {

constexpr int TS = 16;                       // tile side in cells
constexpr int UMAX = 512;                    // visibilities per work unit
constexpr unsigned FULL = 0xffffffffu;

struct GridGeom {
    int n, half, r, ks, tt, off, kernel;
    float du, inv_du, s_hi, s_lo;
};

// The key space of the plan: every nearest cell whose footprint can reach the grid
// (|c| <= half + r), or, with rings_only (the estimate), only those whose footprint can
// reach a ring cell (|c| <= R + r, R the largest |g_x| of a ring cell): a visibility
// outside adds to no cell the estimate reads, and the smaller key space sorts in fewer
// or narrower passes.  Cells keep their place in the full n x n accumulators either way.
GridGeom geom(const Setup &s, bool rings_only = false) {
    GridGeom g;
    g.n = s.n;
    g.half = s.half;
    g.r = s.kernel == ABS_KERNEL_NGP ? 0 : s.r;
    const int reach = rings_only ? std::min(s.half, std::max(s.R, 0)) : s.half;
    g.ks = 2 * (reach + g.r) + 1;
    g.tt = (int)cdiv(g.ks, TS);
    g.off = reach + g.r;
    g.kernel = s.kernel;
    g.du = s.du;
    g.inv_du = (float)(1.0 / (double)s.du);
    g.s_hi = s.s_hi;
    g.s_lo = s.s_lo;
    return g;
}

__device__ __forceinline__ int64_t cell_index(int n, int gx, int gy) {
    const int ix = gx < 0 ? gx + n : gx;
    const int iy = gy < 0 ? gy + n : gy;
    return (int64_t)iy * n + ix;
}

// exp(-(s_hi + s_lo) (d - f_hi - f_lo)^2) with the argument in double-float.
__device__ __forceinline__ float wexp(float d, float f_hi, float f_lo, float s_hi, float s_lo) {
    const float t = __fsub_rn(d, f_hi);                 // TwoSum(d, -f_hi)
    const float bp = __fsub_rn(t, d);
    const float e = __fadd_rn(__fsub_rn(d, __fsub_rn(t, bp)), __fsub_rn(-f_hi, bp));
    const float a_hi = t, a_lo = __fsub_rn(e, f_lo);
    const float p = __fmul_rn(a_hi, a_hi);
    const float pe = fmaf(a_hi, a_hi, -p);              // exact square error
    const float qq = fmaf(2.0f * a_hi, a_lo, pe);
    const float arg_hi = __fmul_rn(-s_hi, p);
    const float arg_e = fmaf(-s_hi, p, -arg_hi);        // exact product error
    const float arg_lo = arg_e - s_hi * qq - s_lo * p;
    return expf(arg_hi) * (1.0f + arg_lo);
}

// ------------------------------------------------------------------ plan kernels
// The plan is a stable counting sort of the visibilities by (uv tile, cell in
// the tile): LSD radix with digits of up to DMAX bits (two passes up to about
// 2040^2 cells, three beyond), so a tile's visibilities are grouped by cell
// whatever the input order (baseline-major tracks or time-major snapshots)
// and keep their input order inside a cell: the gridded sums are reproducible
// run to run.  A pass is per-chunk digit histograms (digit-major) -> exclusive
// scan -> order-preserving scatter.
constexpr int RT = 4096;               // visibilities per sort chunk (256 threads x 16)
constexpr int DMAX = 11;               // widest digit: 2048 bins
constexpr int CB = 8;                  // key bits of the cell inside its tile (TS x TS = 2^CB)
static_assert(TS * TS == 1 << CB, "tile cells must fill CB bits");

// Key of position p given its quotients q = (u / dU, v / dU) in binary32, round to nearest.
__device__ __forceinline__ uint32_t key_from_q(const GridGeom &G, float2 p, float2 q, uint32_t key_none) {
    if (!(isfinite(p.x) && isfinite(p.y))) return key_none;
    if (!(fabsf(q.x) < 1.0e7f && fabsf(q.y) < 1.0e7f)) return key_none;
    const int cx = (int)floorf(__fadd_rn(q.x, 0.5f));
    const int cy = (int)floorf(__fadd_rn(q.y, 0.5f));
    const int kx = cx + G.off, ky = cy + G.off;
    if (kx < 0 || kx >= G.ks || ky < 0 || ky >= G.ks) return key_none;
    const uint32_t tile = (uint32_t)((ky / TS) * G.tt + kx / TS);
    return tile << CB | (uint32_t)((ky % TS) * TS + kx % TS);
}

__device__ __forceinline__ float2 quotients(const GridGeom &G, float2 p) {
    return make_float2(__fdiv_rn(p.x, G.du), __fdiv_rn(p.y, G.du));
}

__device__ __forceinline__ uint32_t cell_key(const GridGeom &G, float2 p, uint32_t key_none) {
    return key_from_q(G, p, quotients(G, p), key_none);
}

// One CTA per chunk: the (tile, cell) key of every visibility (key_none for
// non-finite or off-grid positions) and the chunk's histogram of the first
// digit (nbins bins; digit = key & dmask), added once per distinct digit in a
// warp.  1024 threads, RT / 1024 visibilities each, all loads in flight.
constexpr int KT = 1024;
__global__ void __launch_bounds__(KT) k_plan_keys(GridGeom G, int64_t n_vis, const float2 *__restrict__ uv,
                                                  uint32_t *__restrict__ keys, uint32_t key_none,
                                                  int nbins, uint32_t dmask, int nchunks,
                                                  uint32_t *__restrict__ rhist) {
    __shared__ uint32_t h[1 << DMAX];
    const int lane = threadIdx.x & 31;
    for (int d = threadIdx.x; d < nbins; d += KT) h[d] = 0;
    __syncthreads();
    const int64_t c0 = (int64_t)blockIdx.x * RT;
    float2 pv[RT / KT];
#pragma unroll
    for (int k = 0; k < RT / KT; ++k) {
        const int64_t i = c0 + k * KT + threadIdx.x;
        pv[k] = i < n_vis ? uv[i] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < RT / KT; ++k) {
        const int64_t i = c0 + k * KT + threadIdx.x;
        const bool on = i < n_vis;
        uint32_t key = 0xffffffffu;
        if (on) {
            key = cell_key(G, pv[k], key_none);
            keys[i] = key;
        }
        const uint32_t dig = on ? key & dmask : 0x10000000u + lane;
        const unsigned peers = __match_any_sync(FULL, dig);
        if (on && lane == __ffs(peers) - 1) atomicAdd(&h[dig], (uint32_t)__popc(peers));
    }
    __syncthreads();
    for (int d = threadIdx.x; d < nbins; d += KT) rhist[(int64_t)d * nchunks + blockIdx.x] = h[d];
}

// Block-wide exclusive scan of one value per thread (blockDim.x a multiple of 32, at most 1024).
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *sh, uint32_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w += y;
        }
        sh[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    const uint32_t warp_base = warp ? sh[warp - 1] : 0u;
    total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return warp_base + x - v;
}

// Order-preserving scatter of one chunk (RT items, ST_W warps; warp w owns
// the contiguous [w RT/ST_W, (w+1) RT/ST_W) of the chunk).  One sweep ranks
// every item among the warp's earlier items of its digit (__match_any_sync,
// lower lanes first) and counts the warp's digits; a prefix over (digit,
// warp) then gives every item its place in the chunk ordered by digit, where
// it is staged in shared memory, and the staged chunk is written out in that
// order: each digit's run goes to consecutive addresses, starting where the
// scanned histogram puts this chunk's part of the digit (local scan + its
// block's offset).  vin == nullptr means the identity (first pass); on the
// last pass (uv_out != nullptr) the sorted original indices and positions
// are written instead of keys.  Before the last pass, the next pass's
// per-chunk digit histogram (digit at shift + dw of every placed key, chunk
// = position / RT) is counted into nhist, which must hold zeros: one global
// add per distinct (digit, chunk) in a warp.
constexpr int ST_W = 16;                 // warps per scatter CTA
constexpr int ST_T = ST_W * 32;
constexpr int ST_R = RT / ST_T;          // items per thread
constexpr int ST_D = (1 << DMAX) / ST_T; // digits per thread at most
__host__ __device__ constexpr int scatter_row(int nbins) { return (nbins + 7) & ~7; }
__host__ __device__ constexpr size_t scatter_smem(int nbins) {
    return sizeof(uint32_t) * (2 * RT + 2 * (size_t)scatter_row(nbins)) +
           sizeof(uint16_t) * ST_W * (size_t)scatter_row(nbins);
}
__global__ void __launch_bounds__(ST_T, 2) k_radix_scatter(const uint32_t *__restrict__ kin,
                                                        const uint32_t *__restrict__ vin, int64_t n,
                                                        int shift, int nbins, uint32_t dmask, int nchunks,
                                                        const uint32_t *__restrict__ offs,
                                                        const uint32_t *__restrict__ bsum,
                                                        uint32_t *__restrict__ kout,
                                                        uint32_t *__restrict__ vout,
                                                        const float2 *__restrict__ uv,
                                                        float2 *__restrict__ uv_out, int dw,
                                                        uint32_t *__restrict__ nhist) {
    extern __shared__ __align__(16) uint8_t ssm[];
    const int row = scatter_row(nbins);                  // nbins rounded up to 8 (16-byte rows)
    uint32_t *skey = (uint32_t *)ssm;                    // [RT] the chunk ordered by digit
    uint32_t *sval = skey + RT;                          // [RT]
    uint32_t *gbase = sval + RT;                         // [row] global position of local 0 for the digit
    uint32_t *lstart = gbase + row;                      // [row] the digit's first local position
    uint16_t *wcnt = (uint16_t *)(lstart + row);         // [ST_W][row] per-warp counts, then offsets
    __shared__ uint32_t sh[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t c0 = (int64_t)blockIdx.x * RT;
    const int64_t w0 = c0 + warp * (RT / ST_W);
    const int nloc = (int)min((int64_t)RT, n - c0);
    // every load in flight at once: keys, values, this thread's digit offsets
    uint32_t kv[ST_R], vv[ST_R];
#pragma unroll
    for (int k = 0; k < ST_R; ++k) {
        const int64_t e = w0 + k * 32 + lane;
        kv[k] = e < n ? kin[e] : 0u;
        vv[k] = vin ? (e < n ? vin[e] : 0u) : (uint32_t)e;
    }
    const int d0 = threadIdx.x * ST_D;   // this thread's digits [d0, d0 + ST_D)
#pragma unroll
    for (int j = 0; j < ST_D; ++j) {
        const int64_t e = (int64_t)(d0 + j) * nchunks + blockIdx.x;
        if (d0 + j < nbins) gbase[d0 + j] = offs[e] + bsum[e / 4096];
    }
    for (int i = threadIdx.x; i < ST_W * row / 8; i += ST_T) ((uint4 *)wcnt)[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    // rank of every item among its warp's earlier items of the same digit
    // (below 256: two 16-bit ranks to a register)
    uint32_t rk[ST_R / 2];
#pragma unroll
    for (int k = 0; k < ST_R; ++k) {
        const bool on = w0 + k * 32 + lane < n;
        const uint32_t d = on ? (kv[k] >> shift) & dmask : 0x10000u + lane;
        const unsigned peers = __match_any_sync(FULL, d);
        uint32_t before = 0;
        if (on) before = wcnt[warp * row + d];
        const uint32_t rank = before + (uint32_t)__popc(peers & lt);
        if (k % 2 == 0) rk[k / 2] = rank;
        else rk[k / 2] |= rank << 16;
        __syncwarp();
        if (on && lane == __ffs(peers) - 1) wcnt[warp * row + d] = (uint16_t)(before + __popc(peers));
        __syncwarp();
    }
    __syncthreads();
    // per digit: offsets of the warps inside its run; the runs' local starts
    uint32_t cnt[ST_D], mine = 0;
#pragma unroll
    for (int j = 0; j < ST_D; ++j) {
        const int d = d0 + j;
        uint32_t run = 0;
        if (d < nbins) {
#pragma unroll
            for (int w = 0; w < ST_W; ++w) {
                const uint32_t c = wcnt[w * row + d];
                wcnt[w * row + d] = (uint16_t)run;
                run += c;
            }
        }
        cnt[j] = run;
        mine += run;
    }
    uint32_t total;
    uint32_t ls = block_exclusive_scan(mine, sh, total);
#pragma unroll
    for (int j = 0; j < ST_D; ++j) {
        const int d = d0 + j;
        if (d < nbins) {
            lstart[d] = ls;
            gbase[d] -= ls;   // global position = gbase[d] + local position
        }
        ls += cnt[j];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < ST_R; ++k) {
        if (w0 + k * 32 + lane < n) {
            const uint32_t d = (kv[k] >> shift) & dmask;
            const uint32_t L = lstart[d] + wcnt[warp * row + d] + ((rk[k / 2] >> (16 * (k % 2))) & 0xffffu);
            skey[L] = kv[k];
            sval[L] = vv[k];
        }
    }
    __syncthreads();
    // write-out in digit order: consecutive threads, consecutive addresses within a run
    if (uv_out) {
        float2 pv[ST_R];
        uint32_t gp[ST_R], vl[ST_R];
#pragma unroll
        for (int k = 0; k < ST_R; ++k) {
            const int L = k * ST_T + threadIdx.x;
            if (L < nloc) {
                const uint32_t key = skey[L];
                vl[k] = sval[L];
                gp[k] = gbase[(key >> shift) & dmask] + (uint32_t)L;
                pv[k] = uv[vl[k]];
            }
        }
#pragma unroll
        for (int k = 0; k < ST_R; ++k) {
            if (k * ST_T + (int)threadIdx.x < nloc) {
                vout[gp[k]] = vl[k];
                uv_out[gp[k]] = pv[k];
            }
        }
        return;
    }
#pragma unroll
    for (int k = 0; k < ST_R; ++k) {
        const int L = k * ST_T + threadIdx.x;
        const bool on = L < nloc;
        uint32_t key = 0, pos = 0;
        if (on) {
            key = skey[L];
            pos = gbase[(key >> shift) & dmask] + (uint32_t)L;
            kout[pos] = key;
            vout[pos] = sval[L];
        }
        if (nhist) {   // (next digit, destination chunk): below 2^11 x 2^20 for valid lanes
            const uint32_t d2 = (key >> (shift + dw)) & (uint32_t)((1 << dw) - 1);
            const uint32_t h2 = on ? d2 << 20 | pos / RT : 0x80000000u + lane;
            const unsigned p2 = __match_any_sync(FULL, h2);
            if (on && lane == __ffs(p2) - 1)
                atomicAdd(&nhist[(int64_t)d2 * nchunks + pos / RT], (uint32_t)__popc(p2));
        }
    }
}

// Exclusive scan of len values, 4096 per 1024-thread block: every block scans
// its part into out and writes its total; the last block to finish (ticket)
// scans the totals in place into block offsets (so element e's exclusive
// prefix is out[e] + bsum[e / 4096]) and re-arms the ticket.  zero_in, when
// given, is the input array itself, cleared once read (the next radix pass
// counts into it).
__global__ void __launch_bounds__(1024) k_scan(const uint32_t *in, int64_t len,
                                               uint32_t *__restrict__ out, uint32_t *__restrict__ bsum,
                                               unsigned *__restrict__ ticket, uint32_t *zero_in) {
    __shared__ uint32_t sh[32];
    __shared__ bool last;
    const int64_t base = (int64_t)blockIdx.x * 4096 + threadIdx.x * 4;
    uint32_t v[4];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k] = base + k < len ? in[base + k] : 0u;
        s += v[k];
    }
    if (zero_in) {   // the same array as in
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (base + k < len) zero_in[base + k] = 0u;
    }
    uint32_t total;
    uint32_t pre = block_exclusive_scan(s, sh, total);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (base + k < len) out[base + k] = pre;
        pre += v[k];
    }
    if (threadIdx.x == 0) {
        bsum[blockIdx.x] = total;
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    uint32_t carry = 0;
    for (int64_t b = 0; b < gridDim.x; b += 1024) {
        const int64_t i = b + threadIdx.x;
        const uint32_t x = i < gridDim.x ? __ldcg(bsum + i) : 0u;
        uint32_t t;
        const uint32_t p = block_exclusive_scan(x, sh, t);
        if (i < gridDim.x) bsum[i] = carry + p;
        carry += t;
    }
    if (threadIdx.x == 0) *ticket = 0u;
}

__global__ void k_scan_add(uint32_t *__restrict__ out, int64_t len,
                           const uint32_t *__restrict__ block_sums) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) out[i] += block_sums[i / 4096];
}

// ------------------------------------------------------------------ accumulation
// One CTA per work unit: UMAX consecutive visibilities of the sorted order,
// so a unit's visibilities come grouped by cell (any number of cells and
// tiles).  Each visibility's 2 (2r+1) one-dimensional weights are formed
// once and staged in shared memory, and the unit is cut into tasks: runs of
// one cell, also cut at every CHUNK-th item of the unit, so a task holds at
// most CHUNK visibilities.  A warp takes a task; lane (dy, q) owns the
// footprint cells (2q, dy) and (2q+1, dy) of the (2r+1)^2 around the run's
// cell and sums w = wx wy, w Re V, w Im V over the run with packed FP32x2
// arithmetic (plain blocks of GFOLD, as two interleaved chains, folded into
// Kahan sums; a fixed order), then adds its cells to the FP64 grid.  No
// shared accumulators: runs never wait on one another, whether the cell is
// dense (long runs) or sparse.
//
// Staged record of a visibility (RS floats): wx[0..7] (zero beyond 2r),
// (wy[d], wy[d]) for d = 0..6, two pad floats, (Re V, Re V, Im V, Im V).
constexpr int GT = 256;          // threads per gridding CTA (8 warps x UMAX/8 items)
// What the third (and fourth) accumulator plane of a cell holds: the weight sum
// (GW_SUM), the number N_g of visibilities entered (GW_COUNT, Eq. vg), or the
// weight sum and the sum of squared weights (GW_SUM_SQ).
enum { GW_SUM = 0, GW_COUNT = 1, GW_SUM_SQ = 2 };
constexpr int RS = 28;           // floats per staged record
constexpr int R_WY = 8, R_V = 24;
constexpr int GFOLD = 16;
constexpr int CHUNK = 128;       // visibilities per task at most
static_assert(UMAX == 8 * 64, "each of 8 warps holds two rounds of 32 items of a unit");
static_assert(UMAX % CHUNK == 0 && UMAX <= 65535, "task starts are 16-bit unit offsets");
constexpr size_t GRID_SMEM = UMAX * sizeof(float) * RS + sizeof(uint32_t) * UMAX + sizeof(uint16_t) * (UMAX + 8);

// The double with the value of x, built with integer operations only (GB300's
// FP64 pipe is narrow: one hardware conversion per flushed value is what kept
// it busy).  Exact for normal, infinite and NaN x; subnormal x (|x| < 2^-126)
// become a zero of the same sign.
__device__ __forceinline__ double widen(float x) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t e = (b >> 23) & 255u;
    const uint32_t sign = b & 0x80000000u;
    const uint32_t eh = e == 255u ? 2047u : e + (1023u - 127u);
    const uint32_t hi = e == 0u ? sign : sign | (eh << 20) | ((b >> 3) & 0xFFFFFu);
    const uint32_t lo = e == 0u ? 0u : b << 29;
    return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ void kahan_add2(float2 &s, float2 &c, float2 x) {
    const float2 m1 = make_float2(-1.f, -1.f);
    const float2 y = __ffma2_rn(c, m1, x);                   // x - c
    const float2 t = __fadd2_rn(s, y);
    c = __ffma2_rn(y, m1, __ffma2_rn(s, m1, t));             // (t - s) - y
    s = t;
}

// One staged visibility (record at offset o) into this lane's two footprint
// cells: w = (wx[2q], wx[2q+1]) * wy[dy], re += w Re V, im += w Im V, sum w.
template <int WM>
__device__ __forceinline__ void grid_acc(const float *lw, const float *lwy, const float *lv, int o, float2 &re,
                                         float2 &im, float2 &ws, float2 &ws2) {
    const float2 wxp = *(const float2 *)(lw + o);
    const float2 wyy = *(const float2 *)(lwy + o);
    const float4 vv = *(const float4 *)(lv + o);
    const float2 w = __fmul2_rn(wxp, wyy);
    re = __ffma2_rn(w, make_float2(vv.x, vv.y), re);
    im = __ffma2_rn(w, make_float2(vv.z, vv.w), im);
    if (WM != GW_COUNT) ws = __fadd2_rn(w, ws);
    if (WM == GW_SUM_SQ) ws2 = __ffma2_rn(w, w, ws2);
}

// Inputs of one unit as thread (warp, lane) sees them: items t = 64 warp +
// 32 h + lane, h = 0, 1, in sorted order.
struct UnitIn {
    int cnt;
    float2 p[2];
    uint32_t idx[2];
};

__device__ __forceinline__ void load_unit(UnitIn &in, int64_t u, int64_t nu, int64_t n_vis,
                                          const float2 *__restrict__ s_uv, const uint32_t *__restrict__ s_idx,
                                          int warp, int lane) {
    if (u >= nu) return;
    const int64_t b = u * UMAX;
    in.cnt = n_vis - b < UMAX ? (int)(n_vis - b) : UMAX;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int t = warp * 64 + h * 32 + lane;
        if (t < in.cnt) {
            in.p[h] = s_uv[b + t];
            in.idx[h] = s_idx[b + t];
        }
    }
}

template <int WM>
__global__ void __launch_bounds__(GT, 3) k_grid(GridGeom G, int64_t n_vis, uint32_t key_none,
                                             const float2 *__restrict__ s_uv,
                                             const uint32_t *__restrict__ s_idx,
                                             const float2 *__restrict__ vis,
                                             double *__restrict__ acc_re,
                                             double *__restrict__ acc_im,
                                             double *__restrict__ acc_w,
                                             double *__restrict__ acc_w2) {
    extern __shared__ __align__(16) uint8_t dsm[];
    float *st = (float *)dsm;                                          // [UMAX][RS] staged records
    uint32_t *skey = (uint32_t *)(st + UMAX * RS);                     // [UMAX] key of every item
    uint16_t *tstart = (uint16_t *)(skey + UMAX);                      // [UMAX + 1] first item of each task
    __shared__ uint32_t wsum_s[8], wvalid_s[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = GT / 32;
    const int r = G.r, fw = 2 * r + 1;
    const bool gauss = G.kernel == ABS_KERNEL_GAUSS;
    // this lane's footprint cells: (2q, dy) and (2q + 1, dy)
    const int dy = lane >> 2, q2 = 2 * (lane & 3);
    const bool on_a = lane < 28 && dy < fw && q2 < fw, on_b = on_a && q2 + 1 < fw;
    const int64_t nu = cdiv(n_vis, UMAX);
    UnitIn nxt;
    load_unit(nxt, blockIdx.x, nu, n_vis, s_uv, s_idx, warp, lane);
    float2 vn[2];   // the next unit's visibilities, gathered one unit ahead
#pragma unroll
    for (int h = 0; h < 2; ++h)
        if (blockIdx.x < nu && warp * 64 + h * 32 + lane < nxt.cnt) vn[h] = vis[nxt.idx[h]];
    for (int64_t u = blockIdx.x; u < nu; u += gridDim.x) {
        const UnitIn cur = nxt;
        const int total = cur.cnt;
        const float2 v[2] = {vn[0], vn[1]};   // this unit's visibilities
        load_unit(nxt, u + gridDim.x, nu, n_vis, s_uv, s_idx, warp, lane);   // in flight during this unit
        __syncthreads();   // previous unit done with the staging buffers
        // keys (the plan's, recomputed from the same positions); invalid items sort last
        float2 q[2];   // u/dU, v/dU of this thread's items
        bool valid[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int t = warp * 64 + h * 32 + lane;
            valid[h] = false;
            if (t < total) {
                q[h] = quotients(G, cur.p[h]);
                const uint32_t key = key_from_q(G, cur.p[h], q[h], key_none);
                skey[t] = key;
                valid[h] = key != key_none;
            }
        }
        __syncthreads();
        // task starts: a valid item that begins a cell run or sits at a multiple of CHUNK
        bool ts[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int t = warp * 64 + h * 32 + lane;
            ts[h] = valid[h] && (t % CHUNK == 0 || skey[t] != skey[t - 1]);
        }
        const unsigned b0 = __ballot_sync(FULL, ts[0]), b1 = __ballot_sync(FULL, ts[1]);
        const unsigned nv0 = __ballot_sync(FULL, valid[0]), nv1 = __ballot_sync(FULL, valid[1]);
        if (lane == 0) {
            wsum_s[warp] = (uint32_t)(__popc(b0) + __popc(b1));
            wvalid_s[warp] = (uint32_t)(__popc(nv0) + __popc(nv1));
        }
        __syncthreads();
        uint32_t wbase = 0, ntask = 0, nvalid = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            wbase += w < warp ? wsum_s[w] : 0u;
            ntask += wsum_s[w];
            nvalid += wvalid_s[w];
        }
        const unsigned lt = (1u << lane) - 1u;
        if (ts[0]) tstart[wbase + __popc(b0 & lt)] = (uint16_t)(warp * 64 + lane);
        if (ts[1]) tstart[wbase + __popc(b0) + __popc(b1 & lt)] = (uint16_t)(warp * 64 + 32 + lane);
        if (threadIdx.x == 0) tstart[ntask] = (uint16_t)nvalid;
        // staging: weights and visibility of every valid item, in place
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int t = warp * 64 + h * 32 + lane;
            if (valid[h]) {
                const float2 p = cur.p[h], qq = q[h];
                const float cxf = floorf(__fadd_rn(qq.x, 0.5f)), cyf = floorf(__fadd_rn(qq.y, 0.5f));
                const float fxh = __fsub_rn(qq.x, cxf), fyh = __fsub_rn(qq.y, cyf);
                // the division residual (exact by FMA) over dU: a correction of
                // relative size 2^-24, so one rounding of its own does not matter
                const float fxl = __fmul_rn(fmaf(-qq.x, G.du, p.x), G.inv_du);
                const float fyl = __fmul_rn(fmaf(-qq.y, G.du, p.y), G.inv_du);
                float *rec = st + t * RS;
                float wx[8], wy[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    wx[k] = wy[k] = 0.f;
                    if (k < fw) {
                        const float d = (float)(k - r);
                        wx[k] = gauss ? wexp(d, fxh, fxl, G.s_hi, G.s_lo) : 1.f;
                        wy[k] = gauss ? wexp(d, fyh, fyl, G.s_hi, G.s_lo) : 1.f;
                    }
                }
                ((float4 *)rec)[0] = make_float4(wx[0], wx[1], wx[2], wx[3]);
                ((float4 *)rec)[1] = make_float4(wx[4], wx[5], wx[6], wx[7]);
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    ((float4 *)(rec + R_WY))[k] = make_float4(wy[2 * k], wy[2 * k], wy[2 * k + 1], wy[2 * k + 1]);
                ((float2 *)(rec + R_WY))[6] = make_float2(wy[6], wy[6]);
                ((float4 *)(rec + R_V))[0] = make_float4(v[h].x, v[h].x, v[h].y, v[h].y);
            }
        }
        // the next unit's visibilities: its indices have arrived by now
#pragma unroll
        for (int h = 0; h < 2; ++h)
            if (u + gridDim.x < nu && warp * 64 + h * 32 + lane < nxt.cnt) vn[h] = vis[nxt.idx[h]];
        __syncthreads();
        if (on_a) {   // lanes without a footprint cell take no part in the sums
            for (int tk = warp; tk < (int)ntask; tk += nwarps) {
                const int j_begin = tstart[tk], j_end = tstart[tk + 1];
                const float2 z = make_float2(0.f, 0.f);
                float2 sre = z, cre = z, sim = z, cim = z, sw = z, cw = z, sw2 = z, cw2 = z;
                const float *lw = st + q2, *lwy = st + R_WY + 2 * dy, *lv = st + R_V;
                for (int j0 = j_begin; j0 < j_end; j0 += GFOLD) {   // plain blocks of GFOLD, folded into Kahan sums
                    float2 bre = z, bim = z, bw = z, bw2 = z;
                    if (j0 + GFOLD <= j_end) {
                        // a full block: unrolled, two independent chains (even, odd visibilities)
                        float2 bre1 = z, bim1 = z, bw1 = z, bw21 = z;
#pragma unroll
                        for (int k = 0; k < GFOLD; k += 2) {
                            grid_acc<WM>(lw, lwy, lv, (j0 + k) * RS, bre, bim, bw, bw2);
                            grid_acc<WM>(lw, lwy, lv, (j0 + k + 1) * RS, bre1, bim1, bw1, bw21);
                        }
                        bre = __fadd2_rn(bre, bre1);
                        bim = __fadd2_rn(bim, bim1);
                        if (WM != GW_COUNT) bw = __fadd2_rn(bw, bw1);
                        if (WM == GW_SUM_SQ) bw2 = __fadd2_rn(bw2, bw21);
                    } else {
                        for (int j = j0; j < j_end; ++j) grid_acc<WM>(lw, lwy, lv, j * RS, bre, bim, bw, bw2);
                    }
                    kahan_add2(sre, cre, bre);
                    kahan_add2(sim, cim, bim);
                    if (WM != GW_COUNT) kahan_add2(sw, cw, bw);
                    if (WM == GW_SUM_SQ) kahan_add2(sw2, cw2, bw2);
                }
                // the run's cell from its key: tile (kx / TS, ky / TS), cell in the tile
                const uint32_t key = skey[j_begin];
                const int tile = (int)(key >> CB), loc = (int)(key & (uint32_t)(TS * TS - 1));
                const int kx = (tile % G.tt) * TS + (loc & (TS - 1)), ky = (tile / G.tt) * TS + (loc >> 4);
                const int gy = ky - G.off + dy - r;
                const int gxa = kx - G.off + q2 - r;
                if (gy < -G.half || gy > G.half) continue;
                // the run's sums s - c, rounded once to FP32 (relative 2^-24 of the run)
                const float2 m1 = make_float2(-1.f, -1.f);
                const float2 vre = __ffma2_rn(cre, m1, sre), vim = __ffma2_rn(cim, m1, sim);
                const float2 vw = __ffma2_rn(cw, m1, sw), vw2 = __ffma2_rn(cw2, m1, sw2);
                const double run = (double)(j_end - j_begin);   // visibilities the run enters at the cell
                if (gxa >= -G.half && gxa <= G.half) {
                    const int64_t pidx = cell_index(G.n, gxa, gy);
                    atomicAdd(&acc_re[pidx], widen(vre.x));
                    atomicAdd(&acc_im[pidx], widen(vim.x));
                    atomicAdd(&acc_w[pidx], WM == GW_COUNT ? run : widen(vw.x));
                    if (WM == GW_SUM_SQ) atomicAdd(&acc_w2[pidx], widen(vw2.x));
                }
                if (on_b && gxa + 1 >= -G.half && gxa + 1 <= G.half) {
                    const int64_t pidx = cell_index(G.n, gxa + 1, gy);
                    atomicAdd(&acc_re[pidx], widen(vre.y));
                    atomicAdd(&acc_im[pidx], widen(vim.y));
                    atomicAdd(&acc_w[pidx], WM == GW_COUNT ? run : widen(vw.y));
                    if (WM == GW_SUM_SQ) atomicAdd(&acc_w2[pidx], widen(vw2.y));
                }
            }
        }
    }
}

// Hermitian mirror and FP32 outputs: G(g) + conj G(-g), W(g) + W(-g).
__global__ void k_grid_finalize(int n, const double *__restrict__ acc_re,
                                const double *__restrict__ acc_im,
                                const double *__restrict__ acc_w,
                                float2 *__restrict__ grid, float *__restrict__ wsum,
                                uint8_t *__restrict__ mask) {
    const int64_t cells = (int64_t)n * n;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < cells;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(p % n), iy = (int)(p / n);
        if (ix == n / 2 || iy == n / 2) {
            grid[p] = make_float2(0.f, 0.f);
            wsum[p] = 0.f;
            mask[p] = 0;
            continue;
        }
        const int mx = ix == 0 ? 0 : n - ix, my = iy == 0 ? 0 : n - iy;
        const int64_t pm = (int64_t)my * n + mx;
        grid[p] = make_float2((float)(acc_re[p] + acc_re[pm]), (float)(acc_im[p] - acc_im[pm]));
        wsum[p] = (float)(acc_w[p] + acc_w[pm]);
        mask[p] = (acc_w[p] > 0.0 || acc_w[pm] > 0.0) ? 1 : 0;   // a filled cell has weight > 0
    }
}


// Filled mask only, for the estimate path (which transforms straight from the
// FP64 accumulators): a cell is filled when it or its mirror has a nonzero
// weight sum (sums of positive weights, never -0), tested on the bits.
__global__ void k_grid_mask(int n, const double *__restrict__ acc_w, uint8_t *__restrict__ mask) {
    const int64_t cells = (int64_t)n * n;
    const unsigned long long *wb = (const unsigned long long *)acc_w;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < cells;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(p % n), iy = (int)(p / n);
        const int mx = ix == 0 ? 0 : n - ix, my = iy == 0 ? 0 : n - iy;
        const int64_t pm = (int64_t)my * n + mx;
        mask[p] = (ix != n / 2 && iy != n / 2 && (wb[p] != 0ull || wb[pm] != 0ull)) ? 1 : 0;
    }
}

struct PlanBufs {
    uint32_t *keys, *k2, *v2, *k3, *v3, *rhist, *roffs;
    uint32_t *s_idx;      // sorted original indices
    float2 *s_uv;         // sorted positions
    int64_t n_vis;
    int ntiles, nchunks;
};

bool plan_bufs(abs_ctx *ctx, const GridGeom &G, int64_t n_vis, PlanBufs &b) {
    b.ntiles = G.tt * G.tt;
    b.n_vis = n_vis;
    const int64_t nv = n_vis > 0 ? n_vis : 1;
    b.nchunks = (int)cdiv(nv, RT);
    b.keys = (uint32_t *)workspace(ctx, "plan.keys", sizeof(uint32_t) * nv);
    b.k2 = (uint32_t *)workspace(ctx, "plan.k2", sizeof(uint32_t) * nv);
    b.v2 = (uint32_t *)workspace(ctx, "plan.v2", sizeof(uint32_t) * nv);
    b.k3 = b.v3 = nullptr;   // the middle pass of a three-pass sort only
    b.rhist = (uint32_t *)workspace(ctx, "plan.rhist", sizeof(uint32_t) * ((size_t)1 << DMAX) * b.nchunks);
    b.roffs = (uint32_t *)workspace(ctx, "plan.roffs", sizeof(uint32_t) * ((size_t)1 << DMAX) * b.nchunks);
    b.s_idx = (uint32_t *)workspace(ctx, "plan.s_idx", sizeof(uint32_t) * nv);
    b.s_uv = (float2 *)workspace(ctx, "plan.s_uv", sizeof(float2) * nv);
    return b.keys && b.k2 && b.v2 && b.rhist && b.roffs && b.s_idx && b.s_uv;
}

}  // namespace

// Exclusive scan of len uint32 values (2 kernels; bsum needs cdiv(len, 4096) + 1 entries).
bool scan_u32(abs_ctx *ctx, const uint32_t *in, int64_t len, uint32_t *out, uint32_t *bsum) {
    unsigned *ticket = (unsigned *)workspace_zeroed(ctx, "scan.ticket", sizeof(unsigned));
    if (!ticket) return false;
    const int nblk = (int)cdiv(len, 4096);
    if (nblk == 0) return true;
    k_scan<<<nblk, 1024, 0, ctx->stream>>>(in, len, out, bsum, ticket, nullptr);
    k_scan_add<<<(int)cdiv(len, 256), 256, 0, ctx->stream>>>(out, len, bsum);
    return true;
}

// The key of an invalid visibility: above every (tile, cell) key.
static uint32_t plan_key_none(const PlanBufs &b) { return (uint32_t)b.ntiles << CB; }

abs_status launch_grid_plan(abs_ctx *ctx, const Setup &s, int64_t n_vis, const float *d_uv, bool rings_only) {
    const GridGeom G = geom(s, rings_only);
    PlanBufs b;
    if (!plan_bufs(ctx, G, n_vis, b)) return fail(ctx, ABS_ERR_OOM, "grid plan workspace");
    if ((uint64_t)b.ntiles << CB >= 0x7fffffffull) return fail(ctx, ABS_ERR_UNSUPPORTED, "uv grid too large");
    if (n_vis == 0) return ABS_OK;   // no visibilities: no units
    const uint32_t key_none = plan_key_none(b);     // invalid visibilities sort last
    int bits = 1;
    while (((uint64_t)1 << bits) <= (uint64_t)key_none) ++bits;
    const int passes = (bits + DMAX - 1) / DMAX;
    const int dw = (bits + passes - 1) / passes;
    if (passes == 3) {
        b.k3 = (uint32_t *)workspace(ctx, "plan.k3", sizeof(uint32_t) * n_vis);
        b.v3 = (uint32_t *)workspace(ctx, "plan.v3", sizeof(uint32_t) * n_vis);
        if (!b.k3 || !b.v3) return fail(ctx, ABS_ERR_OOM, "grid plan workspace");
    }
    // one pass: the digit is the key itself, so exactly key_none + 1 bins
    const int nbins0 = passes == 1 ? (int)key_none + 1 : 1 << dw;
    const int64_t rlen = (int64_t)std::max(nbins0, 1 << dw) * b.nchunks;
    uint32_t *bsum = (uint32_t *)workspace(ctx, "plan.bsum", sizeof(uint32_t) * (cdiv(rlen, 4096) + 1));
    unsigned *ticket = (unsigned *)workspace_zeroed(ctx, "scan.ticket", sizeof(unsigned));
    if (!bsum || !ticket) return fail(ctx, ABS_ERR_OOM, "grid plan workspace");
    cudaStream_t st = ctx->stream;
    StageTimer timer(ctx, "grid_plan");
    const size_t ssmem0 = scatter_smem(nbins0), ssmem = scatter_smem(1 << dw);
    allow_smem(k_radix_scatter, std::max(ssmem0, ssmem));
    const uint32_t dmask = passes == 1 ? 0xffffffffu : (uint32_t)((1 << dw) - 1);
    k_plan_keys<<<b.nchunks, KT, 0, st>>>(G, n_vis, (const float2 *)d_uv, b.keys, key_none, nbins0, dmask,
                                          b.nchunks, b.rhist);
    // stable sort of (key, index): keys -> (k2, v2) [-> (k3, v3)] -> (s_idx, s_uv).
    // Every scan clears the histogram it read, and every scatter but the last
    // counts the next pass's histogram into it.
    const uint32_t *ki = b.keys, *vi = nullptr;
    for (int ps = 0; ps < passes; ++ps) {
        const bool last = ps == passes - 1;
        const int nbins = ps == 0 ? nbins0 : 1 << dw;
        const int64_t len = (int64_t)nbins * b.nchunks;
        k_scan<<<(int)cdiv(len, 4096), 1024, 0, st>>>(b.rhist, len, b.roffs, bsum, ticket,
                                                      last ? nullptr : b.rhist);
        uint32_t *ko = ps % 2 == 0 ? b.k2 : b.k3, *vo = ps % 2 == 0 ? b.v2 : b.v3;
        k_radix_scatter<<<b.nchunks, ST_T, ps == 0 ? ssmem0 : ssmem, st>>>(
            ki, vi, n_vis, dw * ps, nbins, dmask, b.nchunks, b.roffs, bsum, last ? nullptr : ko,
            last ? b.s_idx : vo, (const float2 *)d_uv, last ? b.s_uv : nullptr, dw, last ? nullptr : b.rhist);
        ki = ko;
        vi = vo;
    }
    return check_launch(ctx, "grid plan");
}

int grid_acc_planes(const Setup &s) { return s.weight_mode == ABS_W_NOISE ? 4 : 3; }

void grid_acc_buffers(abs_ctx *ctx, const Setup &s, double **acc) {
    const int64_t cells = (int64_t)s.n * s.n;
    *acc = (double *)workspace(ctx, "grid.acc", sizeof(double) * grid_acc_planes(s) * cells);
}

abs_status launch_grid_accumulate(abs_ctx *ctx, const Setup &s, int64_t n_vis, const float *d_vis,
                                  float *d_grid, float *d_wsum, uint8_t *d_mask, bool acc_zeroed) {
    // the estimate path (no FP32 outputs; its plan was made with rings_only) accumulates what
    // its weighting needs
    const bool estimate = !d_grid && !d_wsum;
    const GridGeom G = geom(s, estimate);
    PlanBufs b;
    if (!plan_bufs(ctx, G, n_vis, b)) return fail(ctx, ABS_ERR_OOM, "grid plan workspace");
    const int64_t cells = (int64_t)s.n * s.n;
    const int wm = !estimate ? GW_SUM
                   : s.weight_mode == ABS_W_PAPER_LITERAL ? GW_COUNT
                   : s.weight_mode == ABS_W_NOISE ? GW_SUM_SQ : GW_SUM;
    const int planes = wm == GW_SUM_SQ ? 4 : 3;
    double *acc = (double *)workspace(ctx, "grid.acc", sizeof(double) * planes * cells);
    if (!acc) return fail(ctx, ABS_ERR_OOM, "grid accumulation workspace");
    cudaStream_t st = ctx->stream;
    if (!acc_zeroed) {
        StageTimer timer(ctx, "grid_zero");
        cudaMemsetAsync(acc, 0, sizeof(double) * planes * cells, st);
    }
    if (n_vis > 0) {
        StageTimer timer(ctx, "grid");
        const int blocks = (int)std::min<int64_t>(cdiv(n_vis, UMAX), ctx->sm_count * 3);
        auto run = [&](auto kern) {
            allow_smem(kern, GRID_SMEM);
            kern<<<blocks, GT, GRID_SMEM, st>>>(G, n_vis, plan_key_none(b), b.s_uv, b.s_idx, (const float2 *)d_vis,
                                                acc, acc + cells, acc + 2 * cells, acc + 3 * cells);
        };
        if (wm == GW_COUNT)
            run(k_grid<GW_COUNT>);
        else if (wm == GW_SUM_SQ)
            run(k_grid<GW_SUM_SQ>);
        else
            run(k_grid<GW_SUM>);
    }
    if (!d_grid && !d_wsum) {   // estimate path: the mask alone, if asked for
        if (d_mask) {
            StageTimer timer(ctx, "grid_mask");
            const int fb = (int)std::min<int64_t>(cdiv(cells, 256), ctx->sm_count * 8);
            k_grid_mask<<<fb, 256, 0, st>>>(s.n, acc + 2 * cells, d_mask);
        }
        return check_launch(ctx, "grid accumulate");
    }
    {
        StageTimer timer(ctx, "grid_finalize");
        const int fb = (int)std::min<int64_t>(cdiv(cells, 256), ctx->sm_count * 8);
        k_grid_finalize<<<fb, 256, 0, st>>>(s.n, acc, acc + cells, acc + 2 * cells,
                                            (float2 *)d_grid, d_wsum, d_mask);
    }
    return check_launch(ctx, "grid accumulate");
}

}  // namespace absk
