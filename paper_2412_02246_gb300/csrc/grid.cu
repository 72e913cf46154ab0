// Stage 1: gridding of visibilities, Eq. vg (Sec. 2).
//
// V_g = sum_i w(U_g - U_i) V(U_i) over the (2r+1)^2 cells around each
// visibility's nearest grid point, every visibility also entered at -U_i with
// V*.  The mirror is applied after accumulation (G(g) + conj G(-g)), which is
// the same sum.
//
// Plan (per baseline set): key every visibility by its 16x16-cell uv tile,
// stable-sort by tile (one radix pass while there are fewer than 2048 tiles,
// about 700 cells a side; two beyond), write the sorted positions and original
// indices, and cut every tile's run into work units of at most UMAX
// visibilities.
//
// Accumulation (per realisation): one CTA per unit stages the unit in shared
// memory, sorts it by cell (stable), forms the 1-D Gaussian weights and cuts
// it into runs of visibilities that share a cell; a warp sums the (2r+1)^2
// footprint cells of a run (lane per footprint cell, compensated FP32, input
// order) and adds them to an FP64 grid.  A final pass applies the Hermitian
// mirror and writes the FP32 outputs.
//
// Weights: w = exp(-(dx - fx)^2 s) exp(-(dy - fy)^2 s), s = 1/(2 sigma^2),
// with the fractional offset f = u/dU - c carried as a float pair (the exact
// division residual) and the exponent argument formed in double-float, so
// that the only sizeable error is that of expf itself.
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

GridGeom geom(const Setup &s) {
    GridGeom g;
    g.n = s.n;
    g.half = s.half;
    g.r = s.kernel == ABS_KERNEL_NGP ? 0 : s.r;
    g.ks = s.n - 1 + 2 * g.r;
    g.tt = (int)cdiv(g.ks, TS);
    g.off = s.half + g.r;
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
// The plan is a stable counting sort of the visibilities by uv tile: LSD radix
// with digits of up to DMAX bits (one pass while the tile count fits 2^DMAX,
// two for the largest grids), so every tile's visibilities keep their input
// order and the gridded sums are reproducible run to run.  A pass is per-chunk
// digit histograms (digit-major) -> exclusive scan -> order-preserving scatter.
constexpr int RT = 4096;               // visibilities per sort chunk (256 threads x 16)
constexpr int DMAX = 11;               // widest digit: 2048 bins

__device__ __forceinline__ uint32_t tile_key(const GridGeom &G, float2 p, uint32_t key_none) {
    if (!(isfinite(p.x) && isfinite(p.y))) return key_none;
    const float qx = __fdiv_rn(p.x, G.du), qy = __fdiv_rn(p.y, G.du);
    if (!(fabsf(qx) < 1.0e7f && fabsf(qy) < 1.0e7f)) return key_none;
    const int cx = (int)floorf(__fadd_rn(qx, 0.5f));
    const int cy = (int)floorf(__fadd_rn(qy, 0.5f));
    const int kx = cx + G.off, ky = cy + G.off;
    if (kx < 0 || kx >= G.ks || ky < 0 || ky >= G.ks) return key_none;
    return (uint32_t)((ky / TS) * G.tt + kx / TS);
}

// One CTA per chunk: the tile key of every visibility (key_none for non-finite
// or off-grid positions), per-tile totals and the chunk's histogram of the
// first digit (nbins bins; digit = key & dmask).  Counts are added once per
// distinct key in a warp (consecutive visibilities of a baseline usually share
// a tile).  1024 threads, RT / 1024 visibilities each, all loads in flight.
constexpr int KT = 1024;
__global__ void __launch_bounds__(KT) k_plan_keys(GridGeom G, int64_t n_vis, const float2 *__restrict__ uv,
                                                  uint32_t *__restrict__ keys,
                                                  uint32_t *__restrict__ tile_hist, uint32_t key_none,
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
            key = tile_key(G, pv[k], key_none);
            keys[i] = key;
        }
        const unsigned peers = __match_any_sync(FULL, key);
        if (on && lane == __ffs(peers) - 1) {
            const uint32_t c = (uint32_t)__popc(peers);
            if (tile_hist && key != key_none) atomicAdd(&tile_hist[key], c);
            atomicAdd(&h[key & dmask], c);
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < nbins; d += KT) rhist[(int64_t)d * nchunks + blockIdx.x] = h[d];
}

// Digit histogram of one chunk for the passes after the first.
__global__ void __launch_bounds__(256) k_radix_hist(const uint32_t *__restrict__ keys, int64_t n, int shift,
                                                    int dw, int nchunks, uint32_t *__restrict__ rhist) {
    __shared__ uint32_t h[1 << DMAX];
    const int nb = 1 << dw, lane = threadIdx.x & 31;   // passes after the first use full dw-bit digits
    for (int d = threadIdx.x; d < nb; d += 256) h[d] = 0;
    __syncthreads();
    const int64_t c0 = (int64_t)blockIdx.x * RT;
    for (int k = 0; k < RT / 256; ++k) {
        const int64_t i = c0 + k * 256 + threadIdx.x;
        const bool on = i < n;
        const uint32_t d = on ? (keys[i] >> shift) & (uint32_t)(nb - 1) : 0x10000u + lane;
        const unsigned peers = __match_any_sync(FULL, d);
        if (on && lane == __ffs(peers) - 1) atomicAdd(&h[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    for (int d = threadIdx.x; d < nb; d += 256) rhist[(int64_t)d * nchunks + blockIdx.x] = h[d];
}

// Order-preserving scatter of one chunk.  Warp w owns the contiguous
// [w RT/ST_W, (w+1) RT/ST_W) of the chunk: a first sweep counts its digits, a
// prefix over warps gives every warp its place inside the chunk's run of each
// digit, and a second sweep places the items (rank among equal digits from
// __match_any_sync, lower lanes first).  The chunk's start of each digit is
// the scanned histogram (local scan + its block's offset).  vin == nullptr
// means the identity (first pass); on the last pass (uv_out != nullptr) the
// sorted original indices and positions are written instead of keys.
constexpr int ST_W = 16;                 // warps per scatter CTA
constexpr int ST_R = RT / ST_W / 32;     // rounds per warp
__global__ void __launch_bounds__(ST_W * 32) k_radix_scatter(const uint32_t *__restrict__ kin,
                                                             const uint32_t *__restrict__ vin, int64_t n,
                                                             int shift, int nbins, uint32_t dmask, int nchunks,
                                                             const uint32_t *__restrict__ offs,
                                                             const uint32_t *__restrict__ bsum,
                                                             uint32_t *__restrict__ kout,
                                                             uint32_t *__restrict__ vout,
                                                             const float2 *__restrict__ uv,
                                                             float2 *__restrict__ uv_out) {
    extern __shared__ __align__(16) uint8_t ssm[];
    uint32_t *base = (uint32_t *)ssm;                    // [nbins]
    uint16_t *wloc = (uint16_t *)(base + nbins);         // [ST_W][nbins]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < nbins; d += blockDim.x) {
        const int64_t e = (int64_t)d * nchunks + blockIdx.x;
        base[d] = offs[e] + bsum[e / 4096];
#pragma unroll
        for (int w = 0; w < ST_W; ++w) wloc[w * nbins + d] = 0;
    }
    __syncthreads();
    const int64_t w0 = (int64_t)blockIdx.x * RT + warp * (RT / ST_W);
    uint32_t kv[ST_R];                // the warp's keys, loaded once with all loads in flight
#pragma unroll
    for (int k = 0; k < ST_R; ++k) {
        const int64_t e = w0 + k * 32 + lane;
        kv[k] = e < n ? kin[e] : 0u;
    }
#pragma unroll
    for (int k = 0; k < ST_R; ++k) {
        const int64_t e = w0 + k * 32 + lane;
        const bool on = e < n;
        const uint32_t d = on ? (kv[k] >> shift) & dmask : 0x10000u + lane;
        const unsigned peers = __match_any_sync(FULL, d);
        if (on && lane == __ffs(peers) - 1) wloc[warp * nbins + d] += (uint16_t)__popc(peers);
        __syncwarp();
    }
    __syncthreads();
    for (int d = threadIdx.x; d < nbins; d += blockDim.x) {
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < ST_W; ++w) {
            const uint32_t c = wloc[w * nbins + d];
            wloc[w * nbins + d] = (uint16_t)run;
            run += c;
        }
    }
    __syncthreads();
    uint32_t vv[ST_R];
#pragma unroll
    for (int k = 0; k < ST_R; ++k) {
        const int64_t e = w0 + k * 32 + lane;
        vv[k] = vin ? (e < n ? vin[e] : 0u) : (uint32_t)e;
    }
    float2 pv[ST_R];
    if (uv_out) {
#pragma unroll
        for (int k = 0; k < ST_R; ++k) pv[k] = w0 + k * 32 + lane < n ? uv[vv[k]] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < ST_R; ++k) {
        const int64_t e = w0 + k * 32 + lane;
        const bool on = e < n;
        const uint32_t key = kv[k];
        const uint32_t d = on ? (key >> shift) & dmask : 0x10000u + lane;
        const unsigned peers = __match_any_sync(FULL, d);
        if (on) {
            const uint32_t pos = base[d] + wloc[warp * nbins + d] + (uint32_t)__popc(peers & ((1u << lane) - 1u));
            vout[pos] = vv[k];
            if (uv_out) uv_out[pos] = pv[k];
            else kout[pos] = key;
        }
        __syncwarp();
        if (on && lane == __ffs(peers) - 1) wloc[warp * nbins + d] += (uint16_t)__popc(peers);
        __syncwarp();
    }
}

// Block-wide exclusive scan of one value per thread (blockDim.x == 1024).
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

// Cut every tile's run of sorted visibilities into units of <= UMAX (one
// block).  Tile totals come from hist, or, when hist is null (a one-pass sort
// whose digit is the tile), from the scanned digit histogram itself: tile t
// starts at the exclusive prefix of entry t * nchunks (out + bsum).
__device__ void cut_units(const uint32_t *__restrict__ hist, const uint32_t *__restrict__ out,
                          const uint32_t *__restrict__ bsum, int nchunks, int ntiles, int4 *__restrict__ units,
                          int *__restrict__ n_units, int cap, uint32_t *__restrict__ n_valid_out, uint32_t *sh) {
    auto tile_start = [&](int t) {
        const int64_t e = (int64_t)t * nchunks;
        return __ldcg(out + e) + __ldcg(bsum + e / 4096);
    };
    uint32_t carry = 0, base = 0;
    for (int b = 0; b < ntiles; b += blockDim.x) {
        const int t = b + threadIdx.x;
        uint32_t c = 0u;
        if (t < ntiles) c = hist ? __ldcg(hist + t) : tile_start(t + 1) - tile_start(t);
        uint32_t ctot;
        const uint32_t start = base + block_exclusive_scan(c, sh, ctot);   // tile offset in sorted order
        const uint32_t nu = (c + UMAX - 1) / UMAX;
        uint32_t total;
        const uint32_t pre = block_exclusive_scan(nu, sh, total);
        for (uint32_t k = 0; k < nu; ++k) {
            const uint32_t u = carry + pre + k;
            if ((int)u < cap) {
                const uint32_t s0 = start + k * UMAX;
                units[u] = make_int4(t, (int)s0, (int)min(start + c, s0 + UMAX), 0);
            }
        }
        carry += total;
        base += ctot;
    }
    if (threadIdx.x == 0) {
        *n_units = min((int)carry, cap);
        *n_valid_out = base;
    }
}

// One block: the gridding units of a one-pass sort, cut from its scanned tile
// histogram (run on the side stream beside the scatter).
__global__ void __launch_bounds__(1024) k_units_scan(const uint32_t *__restrict__ out,
                                                     const uint32_t *__restrict__ bsum, int nchunks, int ntiles,
                                                     int4 *__restrict__ units, int *__restrict__ n_units, int cap,
                                                     uint32_t *__restrict__ n_valid_out) {
    __shared__ uint32_t sh[32];
    cut_units(nullptr, out, bsum, nchunks, ntiles, units, n_units, cap, n_valid_out, sh);
}

// Exclusive scan of len values, 4096 per 1024-thread block: every block scans
// its part into out and writes its total; the last block to finish (ticket)
// scans the totals in place into block offsets (so element e's exclusive
// prefix is out[e] + bsum[e / 4096]), optionally cuts the gridding units (from
// tile_hist, or with tile_hist null from this scan of a tile-digit histogram
// with ntiles + 1 bins), and re-arms the ticket.
__global__ void __launch_bounds__(1024) k_scan(const uint32_t *__restrict__ in, int64_t len,
                                               uint32_t *__restrict__ out, uint32_t *__restrict__ bsum,
                                               unsigned *__restrict__ ticket,
                                               const uint32_t *__restrict__ tile_hist, int ntiles,
                                               int4 *__restrict__ units, int *__restrict__ n_units, int cap,
                                               uint32_t *__restrict__ n_valid_out) {
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
    if (units) cut_units(tile_hist, out, bsum, ntiles ? (int)(len / (ntiles + 1)) : 0, ntiles, units, n_units, cap,
                         n_valid_out, sh);
    if (threadIdx.x == 0) *ticket = 0u;
}

__global__ void k_scan_add(uint32_t *__restrict__ out, int64_t len,
                           const uint32_t *__restrict__ block_sums) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) out[i] += block_sums[i / 4096];
}

// ------------------------------------------------------------------ accumulation
// One CTA per work unit (<= UMAX visibilities of one 16x16-cell tile, in input
// order).  The unit is staged in shared memory and stably sorted by cell
// (per-warp counts, prefix over (cell, warp), ranked placement), each
// visibility's 2 (2r+1) one-dimensional weights are formed once, and the
// unit is cut into tasks: runs of at most CHUNK visibilities that share a
// cell.  A warp takes a task; lane (dy, q) owns the footprint cells
// (2q, dy) and (2q+1, dy) of the (2r+1)^2 around the run's cell and sums
// w = wx wy, w Re V, w Im V over the run with packed FP32x2 arithmetic
// (plain blocks of GFOLD, as two interleaved chains, folded into Kahan sums;
// a fixed order), then adds its cells to the FP64 grid.  No shared accumulators: runs never wait on one
// another, whether the tile is dense (long runs) or sparse.
//
// Staged record of a visibility (RS floats): wx[0..7] (zero beyond 2r),
// (wy[d], wy[d]) for d = 0..6, two pad floats, (Re V, Re V, Im V, Im V).
constexpr int GT = 256;          // threads per gridding CTA (8 warps x UMAX/8 items)
constexpr int RS = 28;           // floats per staged record
constexpr int R_WY = 8, R_V = 24;
constexpr int GFOLD = 16;
constexpr int CHUNK = 128;       // visibilities per task at most
constexpr int MAXTASK = UMAX / CHUNK + 256;   // sum over cells of ceil(run / CHUNK)
static_assert(UMAX == 8 * 64, "the in-unit sort gives each of 8 warps two rounds of 32 items");
constexpr size_t GRID_SMEM = UMAX * sizeof(float) * RS + sizeof(int2) * MAXTASK + sizeof(uint16_t) * 8 * 256 +
                             sizeof(uint32_t) * 260 + 2 * UMAX;

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
__device__ __forceinline__ void grid_acc(const float *lw, const float *lwy, const float *lv, int o, float2 &re,
                                         float2 &im, float2 &ws) {
    const float2 wxp = *(const float2 *)(lw + o);
    const float2 wyy = *(const float2 *)(lwy + o);
    const float4 vv = *(const float4 *)(lv + o);
    const float2 w = __fmul2_rn(wxp, wyy);
    re = __ffma2_rn(w, make_float2(vv.x, vv.y), re);
    im = __ffma2_rn(w, make_float2(vv.z, vv.w), im);
    ws = __fadd2_rn(w, ws);
}

// Inputs of one unit as thread (warp, lane) sees them: items t = 64 warp +
// 32 h + lane, h = 0, 1, in input order.
struct UnitIn {
    int4 U;
    float2 p[2];
    uint32_t idx[2];
};

__device__ __forceinline__ void load_unit(UnitIn &in, int u, int nu, const int4 *__restrict__ units,
                                          const float2 *__restrict__ s_uv, const uint32_t *__restrict__ s_idx,
                                          int warp, int lane) {
    if (u >= nu) return;
    in.U = units[u];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int t = warp * 64 + h * 32 + lane;
        if (t < in.U.z - in.U.y) {
            in.p[h] = s_uv[in.U.y + t];
            in.idx[h] = s_idx[in.U.y + t];
        }
    }
}

__global__ void __launch_bounds__(GT) k_grid(GridGeom G, const int4 *__restrict__ units,
                                             const int *__restrict__ n_units,
                                             const float2 *__restrict__ s_uv,
                                             const uint32_t *__restrict__ s_idx,
                                             const float2 *__restrict__ vis,
                                             double *__restrict__ acc_re,
                                             double *__restrict__ acc_im,
                                             double *__restrict__ acc_w) {
    extern __shared__ __align__(16) uint8_t dsm[];
    float *st = (float *)dsm;                                          // [UMAX][RS] staged records
    int2 *task = (int2 *)(st + UMAX * RS);                             // [MAXTASK] (first, end)
    uint16_t *wloc = (uint16_t *)(task + MAXTASK);                     // [8][256] per-warp cell counts
    uint32_t *cstart = (uint32_t *)(wloc + 8 * 256);                   // [257] first item of each cell
    uint8_t *in_c = (uint8_t *)(cstart + 260);                         // [UMAX] cell, input order
    uint8_t *st_c = in_c + UMAX;                                       // [UMAX] cell, sorted order
    __shared__ uint32_t sh_scan[32];
    __shared__ int ntask_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = GT / 32;
    const int r = G.r, fw = 2 * r + 1;
    const bool gauss = G.kernel == ABS_KERNEL_GAUSS;
    // this lane's footprint cells: (2q, dy) and (2q + 1, dy)
    const int dy = lane >> 2, q2 = 2 * (lane & 3);
    const bool on_a = lane < 28 && dy < fw && q2 < fw, on_b = on_a && q2 + 1 < fw;
    const int nu = *n_units;
    UnitIn nxt;
    load_unit(nxt, blockIdx.x, nu, units, s_uv, s_idx, warp, lane);
    for (int u = blockIdx.x; u < nu; u += gridDim.x) {
        const UnitIn cur = nxt;
        const int4 U = cur.U;
        const int total = U.z - U.y;
        const int tile = U.x, tx = tile % G.tt, ty = tile / G.tt;
        float2 v[2];   // this unit's visibilities: gathered now, used at placement
#pragma unroll
        for (int h = 0; h < 2; ++h)
            if (warp * 64 + h * 32 + lane < total) v[h] = vis[cur.idx[h]];
        load_unit(nxt, u + gridDim.x, nu, units, s_uv, s_idx, warp, lane);   // in flight during this unit
        __syncthreads();   // previous unit done with the staging buffers
        // cells, and per-warp counts over the warp's 64 items (input order)
        for (int k = lane; k < 256; k += 32) wloc[warp * 256 + k] = 0;
        __syncwarp();
        float2 q[2];   // u/dU, v/dU of this thread's items
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int t = warp * 64 + h * 32 + lane;
            const bool on = t < total;
            uint32_t c = 0x10000u + lane;
            if (on) {
                q[h] = make_float2(__fdiv_rn(cur.p[h].x, G.du), __fdiv_rn(cur.p[h].y, G.du));
                const int kx = (int)floorf(__fadd_rn(q[h].x, 0.5f)) + G.off;
                const int ky = (int)floorf(__fadd_rn(q[h].y, 0.5f)) + G.off;
                c = (uint32_t)((ky - ty * TS) * TS + (kx - tx * TS));
                in_c[t] = (uint8_t)c;
            }
            const unsigned peers = __match_any_sync(FULL, c);
            if (on && lane == __ffs(peers) - 1) wloc[warp * 256 + c] += (uint16_t)__popc(peers);
            __syncwarp();
        }
        __syncthreads();
        {   // cell threadIdx.x: its start, and each warp's place inside its run
            const int c = threadIdx.x;
            uint32_t cnt = 0;
#pragma unroll
            for (int w = 0; w < 8; ++w) cnt += wloc[w * 256 + c];
            uint32_t tot;
            const uint32_t start = block_exclusive_scan(cnt, sh_scan, tot);
            cstart[c] = start;
            if (c == 255) cstart[256] = start + cnt;
            uint32_t run = start;
#pragma unroll
            for (int w = 0; w < 8; ++w) {
                const uint32_t x = wloc[w * 256 + c];
                wloc[w * 256 + c] = (uint16_t)run;
                run += x;
            }
        }
        __syncthreads();
        // placement in cell order: weights, visibility and cell of every item
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int t = warp * 64 + h * 32 + lane;
            const bool on = t < total;
            const uint32_t c = on ? (uint32_t)in_c[t] : 0x10000u + lane;
            const unsigned peers = __match_any_sync(FULL, c);
            if (on) {
                const int pos = (int)wloc[warp * 256 + c] + __popc(peers & ((1u << lane) - 1u));
                const float2 p = cur.p[h], qq = q[h];
                const float cxf = floorf(__fadd_rn(qq.x, 0.5f)), cyf = floorf(__fadd_rn(qq.y, 0.5f));
                const float fxh = __fsub_rn(qq.x, cxf), fyh = __fsub_rn(qq.y, cyf);
                // the division residual (exact by FMA) over dU: a correction of
                // relative size 2^-24, so one rounding of its own does not matter
                const float fxl = __fmul_rn(fmaf(-qq.x, G.du, p.x), G.inv_du);
                const float fyl = __fmul_rn(fmaf(-qq.y, G.du, p.y), G.inv_du);
                float *rec = st + pos * RS;
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
                st_c[pos] = (uint8_t)c;
            }
            __syncwarp();
            if (on && lane == __ffs(peers) - 1) wloc[warp * 256 + c] += (uint16_t)__popc(peers);
            __syncwarp();
        }
        __syncthreads();
        if (warp == 0) {   // tasks: every cell's run cut into chunks of <= CHUNK
            uint32_t nt[8], run = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int c = lane * 8 + k;
                const uint32_t n = cstart[c + 1] - cstart[c];
                nt[k] = (n + CHUNK - 1) / CHUNK;
                run += nt[k];
            }
            uint32_t incl = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += y;
            }
            uint32_t pos = incl - run;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int c = lane * 8 + k;
                const int j0 = (int)cstart[c], j1 = (int)cstart[c + 1];
                for (uint32_t qn = 0; qn < nt[k]; ++qn, ++pos) {
                    const int a = j0 + (int)qn * CHUNK;
                    task[pos] = make_int2(a, min(j1, a + CHUNK));
                }
            }
            if (lane == 31) ntask_s = (int)incl;
        }
        __syncthreads();
        const int ntask = ntask_s;
        const int gx0 = tx * TS - G.off, gy0 = ty * TS - G.off;
        if (on_a) {   // lanes without a footprint cell take no part in the sums
            for (int tk = warp; tk < ntask; tk += nwarps) {
                const int2 T = task[tk];
                const float2 z = make_float2(0.f, 0.f);
                float2 sre = z, cre = z, sim = z, cim = z, sw = z, cw = z;
                const float *lw = st + q2, *lwy = st + R_WY + 2 * dy, *lv = st + R_V;
                for (int j0 = T.x; j0 < T.y; j0 += GFOLD) {   // plain blocks of GFOLD, folded into Kahan sums
                    float2 bre = z, bim = z, bw = z;
                    if (j0 + GFOLD <= T.y) {
                        // a full block: unrolled, two independent chains (even, odd visibilities)
                        float2 bre1 = z, bim1 = z, bw1 = z;
#pragma unroll
                        for (int u = 0; u < GFOLD; u += 2) {
                            grid_acc(lw, lwy, lv, (j0 + u) * RS, bre, bim, bw);
                            grid_acc(lw, lwy, lv, (j0 + u + 1) * RS, bre1, bim1, bw1);
                        }
                        bre = __fadd2_rn(bre, bre1);
                        bim = __fadd2_rn(bim, bim1);
                        bw = __fadd2_rn(bw, bw1);
                    } else {
                        for (int j = j0; j < T.y; ++j) grid_acc(lw, lwy, lv, j * RS, bre, bim, bw);
                    }
                    kahan_add2(sre, cre, bre);
                    kahan_add2(sim, cim, bim);
                    kahan_add2(sw, cw, bw);
                }
                const int cell = st_c[T.x];
                const int gy = gy0 + (cell >> 4) + dy - r;
                const int gxa = gx0 + (cell & (TS - 1)) + q2 - r;
                if (gy < -G.half || gy > G.half) continue;
                // the run's sums s - c, rounded once to FP32 (relative 2^-24 of the run)
                const float2 m1 = make_float2(-1.f, -1.f);
                const float2 vre = __ffma2_rn(cre, m1, sre), vim = __ffma2_rn(cim, m1, sim);
                const float2 vw = __ffma2_rn(cw, m1, sw);
                if (gxa >= -G.half && gxa <= G.half) {
                    const int64_t pidx = cell_index(G.n, gxa, gy);
                    atomicAdd(&acc_re[pidx], widen(vre.x));
                    atomicAdd(&acc_im[pidx], widen(vim.x));
                    atomicAdd(&acc_w[pidx], widen(vw.x));
                }
                if (on_b && gxa + 1 >= -G.half && gxa + 1 <= G.half) {
                    const int64_t pidx = cell_index(G.n, gxa + 1, gy);
                    atomicAdd(&acc_re[pidx], widen(vre.y));
                    atomicAdd(&acc_im[pidx], widen(vim.y));
                    atomicAdd(&acc_w[pidx], widen(vw.y));
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
    uint32_t *keys, *tile_hist, *k2, *v2, *rhist, *roffs, *n_valid;
    uint32_t *s_idx;      // sorted original indices
    float2 *s_uv;         // sorted positions
    int4 *units;
    int *n_units;
    int64_t n_vis;
    int ntiles, units_cap, nchunks;
};

bool plan_bufs(abs_ctx *ctx, const GridGeom &G, int64_t n_vis, PlanBufs &b) {
    b.ntiles = G.tt * G.tt;
    b.n_vis = n_vis;
    b.units_cap = (int)(b.ntiles + cdiv(n_vis, UMAX) + 1);
    const int64_t nv = n_vis > 0 ? n_vis : 1;
    b.nchunks = (int)cdiv(nv, RT);
    b.keys = (uint32_t *)workspace(ctx, "plan.keys", sizeof(uint32_t) * nv);
    b.tile_hist = (uint32_t *)workspace(ctx, "plan.tile_hist", sizeof(uint32_t) * b.ntiles);
    b.k2 = (uint32_t *)workspace(ctx, "plan.k2", sizeof(uint32_t) * nv);
    b.v2 = (uint32_t *)workspace(ctx, "plan.v2", sizeof(uint32_t) * nv);
    b.rhist = (uint32_t *)workspace(ctx, "plan.rhist", sizeof(uint32_t) * ((size_t)1 << DMAX) * b.nchunks);
    b.roffs = (uint32_t *)workspace(ctx, "plan.roffs", sizeof(uint32_t) * ((size_t)1 << DMAX) * b.nchunks);
    b.n_valid = (uint32_t *)workspace(ctx, "plan.n_valid", sizeof(uint32_t));
    b.s_idx = (uint32_t *)workspace(ctx, "plan.s_idx", sizeof(uint32_t) * nv);
    b.s_uv = (float2 *)workspace(ctx, "plan.s_uv", sizeof(float2) * nv);
    b.units = (int4 *)workspace(ctx, "plan.units", sizeof(int4) * b.units_cap);
    b.n_units = (int *)workspace(ctx, "plan.n_units", sizeof(int));
    return b.keys && b.tile_hist && b.k2 && b.v2 && b.rhist && b.roffs && b.n_valid && b.s_idx &&
           b.s_uv && b.units && b.n_units;
}

}  // namespace

// Exclusive scan of len uint32 values (2 kernels; bsum needs cdiv(len, 4096) + 1 entries).
bool scan_u32(abs_ctx *ctx, const uint32_t *in, int64_t len, uint32_t *out, uint32_t *bsum) {
    unsigned *ticket = (unsigned *)workspace_zeroed(ctx, "scan.ticket", sizeof(unsigned));
    if (!ticket) return false;
    const int nblk = (int)cdiv(len, 4096);
    if (nblk == 0) return true;
    k_scan<<<nblk, 1024, 0, ctx->stream>>>(in, len, out, bsum, ticket, nullptr, 0, nullptr, nullptr, 0, nullptr);
    k_scan_add<<<(int)cdiv(len, 256), 256, 0, ctx->stream>>>(out, len, bsum);
    return true;
}

abs_status launch_grid_plan(abs_ctx *ctx, const Setup &s, int64_t n_vis, const float *d_uv) {
    const GridGeom G = geom(s);
    PlanBufs b;
    if (!plan_bufs(ctx, G, n_vis, b)) return fail(ctx, ABS_ERR_OOM, "grid plan workspace");
    const uint32_t key_none = (uint32_t)b.ntiles;     // invalid visibilities sort last
    int bits = 1;
    while (((uint64_t)1 << bits) <= (uint64_t)key_none) ++bits;
    const int passes = (bits + DMAX - 1) / DMAX;
    if (passes > 2) return fail(ctx, ABS_ERR_UNSUPPORTED, "uv tile count beyond two radix passes");
    const int dw = (bits + passes - 1) / passes;
    // one pass: the digit is the key itself, so exactly ntiles + 1 bins
    const int nbins0 = passes == 1 ? b.ntiles + 1 : 1 << dw;
    const int64_t rlen = (int64_t)(1 << dw) * b.nchunks;
    uint32_t *bsum = (uint32_t *)workspace(ctx, "plan.bsum", sizeof(uint32_t) * (cdiv(rlen, 4096) + 1));
    unsigned *ticket = (unsigned *)workspace_zeroed(ctx, "scan.ticket", sizeof(unsigned));
    if (!bsum || !ticket) return fail(ctx, ABS_ERR_OOM, "grid plan workspace");
    cudaStream_t st = ctx->stream;
    StageTimer timer(ctx, "grid_plan");
    // one pass: the tile totals are read off the scanned histogram; two: counted by atomics
    uint32_t *tile_hist = passes == 1 ? nullptr : b.tile_hist;
    if (tile_hist) cudaMemsetAsync(tile_hist, 0, sizeof(uint32_t) * b.ntiles, st);
    if (n_vis == 0) {
        // no visibilities: no units
        cudaMemsetAsync(b.tile_hist, 0, sizeof(uint32_t) * b.ntiles, st);
        k_scan<<<1, 1024, 0, st>>>(b.rhist, 0, b.roffs, bsum, ticket, b.tile_hist, b.ntiles, b.units, b.n_units,
                                   b.units_cap, b.n_valid);
        return check_launch(ctx, "grid plan");
    }
    const size_t ssmem0 = (size_t)nbins0 * (4 + 2 * ST_W), ssmem = (size_t)(1 << dw) * (4 + 2 * ST_W);
    cudaFuncSetAttribute(k_radix_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)std::max(ssmem0, ssmem));
    k_plan_keys<<<b.nchunks, KT, 0, st>>>(G, n_vis, (const float2 *)d_uv, b.keys, tile_hist, key_none, nbins0,
                                          passes == 1 ? 0xffffffffu : (uint32_t)((1 << dw) - 1), b.nchunks,
                                          b.rhist);
    // stable sort of (tile, index): keys -> (k2, v2) -> (s_idx, s_uv).  Units:
    // one pass, cut from the scanned histogram by one block on the side stream
    // while the scatter runs (by the scan's last block while profiling); two
    // passes, from the tile totals by the last scan's last block
    const bool fork = passes == 1 && !ctx->profiling && ctx->side;
    const uint32_t *ki = b.keys, *vi = nullptr;
    for (int ps = 0; ps < passes; ++ps) {
        const bool last = ps == passes - 1;
        const int nbins = ps == 0 ? nbins0 : 1 << dw;
        const uint32_t dmask = passes == 1 ? 0xffffffffu : (uint32_t)((1 << dw) - 1);
        if (ps > 0) k_radix_hist<<<b.nchunks, 256, 0, st>>>(ki, n_vis, dw * ps, dw, b.nchunks, b.rhist);
        const int64_t len = (int64_t)nbins * b.nchunks;
        const bool cut = !fork && (passes == 1 || last);
        k_scan<<<(int)cdiv(len, 4096), 1024, 0, st>>>(b.rhist, len, b.roffs, bsum, ticket, tile_hist, b.ntiles,
                                                      cut ? b.units : nullptr, b.n_units, b.units_cap, b.n_valid);
        if (fork) {
            cudaEventRecord(ctx->ev_fork2, st);
            cudaStreamWaitEvent(ctx->side, ctx->ev_fork2, 0);
            k_units_scan<<<1, 1024, 0, ctx->side>>>(b.roffs, bsum, b.nchunks, b.ntiles, b.units, b.n_units,
                                                    b.units_cap, b.n_valid);
            cudaEventRecord(ctx->ev_join2, ctx->side);
        }
        k_radix_scatter<<<b.nchunks, ST_W * 32, ps == 0 ? ssmem0 : ssmem, st>>>(
            ki, vi, n_vis, dw * ps, nbins, dmask, b.nchunks, b.roffs, bsum, last ? nullptr : b.k2,
            last ? b.s_idx : b.v2, (const float2 *)d_uv, last ? b.s_uv : nullptr);
        ki = b.k2;
        vi = b.v2;
    }
    if (fork) cudaStreamWaitEvent(st, ctx->ev_join2, 0);
    return check_launch(ctx, "grid plan");
}

void grid_acc_buffers(abs_ctx *ctx, const Setup &s, double **acc) {
    const int64_t cells = (int64_t)s.n * s.n;
    *acc = (double *)workspace(ctx, "grid.acc", sizeof(double) * 3 * cells);
}

abs_status launch_grid_accumulate(abs_ctx *ctx, const Setup &s, int64_t n_vis, const float *d_vis,
                                  float *d_grid, float *d_wsum, uint8_t *d_mask, bool acc_zeroed) {
    const GridGeom G = geom(s);
    PlanBufs b;
    if (!plan_bufs(ctx, G, n_vis, b)) return fail(ctx, ABS_ERR_OOM, "grid plan workspace");
    const int64_t cells = (int64_t)s.n * s.n;
    double *acc = (double *)workspace(ctx, "grid.acc", sizeof(double) * 3 * cells);
    if (!acc) return fail(ctx, ABS_ERR_OOM, "grid accumulation workspace");
    cudaStream_t st = ctx->stream;
    if (!acc_zeroed) {
        StageTimer timer(ctx, "grid_zero");
        cudaMemsetAsync(acc, 0, sizeof(double) * 3 * cells, st);
    }
    if (n_vis > 0) {
        StageTimer timer(ctx, "grid");
        const int blocks = std::min(b.units_cap, ctx->sm_count * 3);
        cudaFuncSetAttribute(k_grid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GRID_SMEM);
        k_grid<<<blocks, GT, GRID_SMEM, st>>>(G, b.units, b.n_units, b.s_uv, b.s_idx, (const float2 *)d_vis, acc,
                                           acc + cells, acc + 2 * cells);
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
