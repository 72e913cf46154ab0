// Stage 1: gridding of visibilities, Eq. vg (Sec. 2).
//
// V_g = sum_i w(U_g - U_i) V(U_i) over the (2r+1)^2 cells around each
// visibility's nearest grid point, every visibility also entered at -U_i with
// V*.  The mirror is applied after accumulation (G(g) + conj G(-g)), which is
// the same sum.
//
// Plan (per baseline set): key every visibility by its 16x16-cell uv tile,
// stable-sort by tile (LSD radix), cut every tile's run into work units of at
// most UMAX visibilities, sort each unit by cell (stable) and form the 1-D
// Gaussian weights of every visibility once.
//
// Accumulation (per realisation): one CTA per unit stages the unit in shared
// memory and cuts it into runs of visibilities that share a cell; a warp sums
// the (2r+1)^2 footprint cells of a run (lane per footprint cell, compensated
// FP32, fixed order) and adds them to an FP64 grid.  A final pass applies the
// Hermitian mirror and writes the FP32 outputs.
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
constexpr int FWMAX = 2 * ABS_MAX_RADIUS + 1;
constexpr unsigned FULL = 0xffffffffu;

struct GridGeom {
    int n, half, r, ks, tt, off, kernel;
    float du, s_hi, s_lo;
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

__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

// ------------------------------------------------------------------ plan kernels

__global__ void k_plan_keys(GridGeom G, int64_t n_vis, const float2 *__restrict__ uv,
                            uint32_t *__restrict__ keys, uint32_t *__restrict__ vals,
                            uint32_t *__restrict__ hist, uint32_t key_none) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_vis;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float2 p = uv[i];
        uint32_t key = key_none;
        if (isfinite(p.x) && isfinite(p.y)) {
            const float qx = __fdiv_rn(p.x, G.du), qy = __fdiv_rn(p.y, G.du);
            if (fabsf(qx) < 1.0e7f && fabsf(qy) < 1.0e7f) {
                const int cx = (int)floorf(__fadd_rn(qx, 0.5f));
                const int cy = (int)floorf(__fadd_rn(qy, 0.5f));
                const int kx = cx + G.off, ky = cy + G.off;
                if (kx >= 0 && kx < G.ks && ky >= 0 && ky < G.ks)
                    key = (uint32_t)((ky / TS) * G.tt + kx / TS);   // 16x16-cell uv tile
            }
        }
        keys[i] = key;
        // one atomic per distinct tile in the warp (consecutive visibilities of a
        // baseline usually share a tile)
        const unsigned active = __activemask();
        const unsigned peers = __match_any_sync(active, key);
        const int lane = threadIdx.x & 31;
        if (key != key_none && lane == __ffs(peers) - 1) atomicAdd(&hist[key], (uint32_t)__popc(peers));
        vals[i] = (uint32_t)i;
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

// Exclusive scan, level 1: 4096 elements per 1024-thread block.
__global__ void __launch_bounds__(1024) k_scan_local(const uint32_t *__restrict__ in, int64_t len,
                                                     uint32_t *__restrict__ out,
                                                     uint32_t *__restrict__ block_sums) {
    __shared__ uint32_t sh[32];
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
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

// Level 2: one block scans the block sums in place (any length).
__global__ void __launch_bounds__(1024) k_scan_top(uint32_t *__restrict__ sums, int64_t len) {
    __shared__ uint32_t sh[32];
    uint32_t carry = 0;
    for (int64_t b = 0; b < len; b += 1024) {
        const int64_t i = b + threadIdx.x;
        const uint32_t v = i < len ? sums[i] : 0u;
        uint32_t total;
        const uint32_t pre = block_exclusive_scan(v, sh, total);
        if (i < len) sums[i] = carry + pre;
        carry += total;
    }
}

__global__ void k_scan_add(uint32_t *__restrict__ out, int64_t len,
                           const uint32_t *__restrict__ block_sums) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) out[i] += block_sums[i / 4096];
}

// Stable LSD radix sort of (key, original index) pairs, 8-bit digits, so
// that every cell's visibilities keep their input order and the gridded sums
// are reproducible run to run.  Pass = per-tile digit histograms (digit-major)
// -> exclusive scan -> order-preserving scatter.
constexpr int RTILE = 2048;            // items per tile (256 threads x 8 rounds)

__global__ void __launch_bounds__(256) k_radix_hist(const uint32_t *__restrict__ keys, int64_t n, int shift,
                                                    int ntiles, uint32_t *__restrict__ hist) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t t0 = (int64_t)blockIdx.x * RTILE;
    for (int r = 0; r < RTILE / 256; ++r) {
        const int64_t e = t0 + r * 256 + threadIdx.x;
        if (e < n) atomicAdd(&h[(keys[e] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(256) k_radix_scatter(const uint32_t *__restrict__ kin,
                                                       const uint32_t *__restrict__ vin, int64_t n,
                                                       int shift, int ntiles,
                                                       const uint32_t *__restrict__ offs,
                                                       uint32_t *__restrict__ kout,
                                                       uint32_t *__restrict__ vout) {
    __shared__ uint32_t wcount[8][256];
    __shared__ uint32_t wbase[8][256];
    __shared__ uint32_t base[256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    base[threadIdx.x] = offs[(int64_t)threadIdx.x * ntiles + blockIdx.x];
    for (int w = 0; w < 8; ++w) wcount[w][threadIdx.x] = 0;
    __syncthreads();
    const int64_t t0 = (int64_t)blockIdx.x * RTILE;
    for (int r = 0; r < RTILE / 256; ++r) {
        const int64_t e = t0 + r * 256 + threadIdx.x;
        const bool on = e < n;
        const uint32_t key = on ? kin[e] : 0u;
        const uint32_t val = on ? vin[e] : 0u;
        const uint32_t d = on ? ((key >> shift) & 255u) : 256u + lane;   // unique for idle lanes
        const unsigned peers = __match_any_sync(FULL, d);
        const unsigned rank = __popc(peers & ((1u << lane) - 1u));
        if (on && rank == 0) wcount[warp][d] = __popc(peers);
        __syncthreads();
        {   // digit threadIdx.x: prefix over warps in order
            uint32_t run = base[threadIdx.x];
            for (int w = 0; w < 8; ++w) {
                const uint32_t c = wcount[w][threadIdx.x];
                wbase[w][threadIdx.x] = run;
                run += c;
                wcount[w][threadIdx.x] = 0;
            }
            base[threadIdx.x] = run;
        }
        __syncthreads();
        if (on) {
            const uint32_t pos = wbase[warp][d] + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
    }
}

// Per work unit (<= UMAX visibilities of one uv tile, in input order after the
// stable tile sort): stable sort by cell within the tile, and the 2 x (2r+1)
// one-dimensional weights of every visibility, w(d) = exp(-s (d - f)^2) with
// f = u/dU - c carried as a float pair (the exact division residual).  Writes
// s_key = tile << 8 | cell in tile, s_idx and s_w [16] = (wx[0..6], -, wy[0..6], -)
// in cell order.  One CTA per unit, 128 threads.
constexpr int PT = 128;
constexpr int WREC = 16;   // floats per weight record

__global__ void __launch_bounds__(PT) k_plan_units(GridGeom G, const int4 *__restrict__ units,
                                                   const int *__restrict__ n_units,
                                                   const float2 *__restrict__ uv,
                                                   const uint32_t *__restrict__ t_idx,
                                                   uint32_t *__restrict__ s_key,
                                                   uint32_t *__restrict__ s_idx,
                                                   float4 *__restrict__ s_w) {
    __shared__ float4 wst[UMAX][WREC / 4];
    __shared__ uint32_t ist[UMAX];
    __shared__ uint8_t cst[UMAX];
    __shared__ uint32_t cnt[256], base[256];
    __shared__ uint32_t wcnt[PT / 32][256], wpre[PT / 32][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = G.r, fw = 2 * r + 1;
    const int nu = *n_units;
    for (int u = blockIdx.x; u < nu; u += gridDim.x) {
        const int4 U = units[u];
        const int total = U.z - U.y;
        const uint32_t tile = (uint32_t)U.x;
        for (int c = threadIdx.x; c < 256; c += PT) cnt[c] = 0;
        __syncthreads();
        for (int t = threadIdx.x; t < total; t += PT) {
            const uint32_t idx = t_idx[U.y + t];
            const float2 p = uv[idx];
            const float qx = __fdiv_rn(p.x, G.du), qy = __fdiv_rn(p.y, G.du);
            const int cx = (int)floorf(__fadd_rn(qx, 0.5f)), cy = (int)floorf(__fadd_rn(qy, 0.5f));
            const int kx = cx + G.off, ky = cy + G.off;
            const int lc = (ky % TS) * TS + kx % TS;
            const float fxh = __fsub_rn(qx, (float)cx), fyh = __fsub_rn(qy, (float)cy);
            const float fxl = __fdiv_rn(fmaf(-qx, G.du, p.x), G.du);
            const float fyl = __fdiv_rn(fmaf(-qy, G.du, p.y), G.du);
            float w[WREC];
#pragma unroll
            for (int k = 0; k < WREC; ++k) w[k] = 0.f;
#pragma unroll
            for (int k = 0; k < FWMAX; ++k) {
                if (k < fw) {
                    const float d = (float)(k - r);
                    w[k] = G.kernel == ABS_KERNEL_GAUSS ? wexp(d, fxh, fxl, G.s_hi, G.s_lo) : 1.f;
                    w[8 + k] = G.kernel == ABS_KERNEL_GAUSS ? wexp(d, fyh, fyl, G.s_hi, G.s_lo) : 1.f;
                }
            }
#pragma unroll
            for (int k = 0; k < WREC / 4; ++k) wst[t][k] = make_float4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
            ist[t] = idx;
            cst[t] = (uint8_t)lc;
            atomicAdd(&cnt[lc], 1u);
        }
        __syncthreads();
        if (warp == 0) {   // exclusive scan of the 256 cell counts
            uint32_t v[8], run = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                v[k] = cnt[lane * 8 + k];
                run += v[k];
            }
            uint32_t incl = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += y;
            }
            uint32_t b0 = incl - run;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                base[lane * 8 + k] = b0;
                b0 += v[k];
            }
        }
        __syncthreads();
        // stable placement: items in input order, rounds of PT
        for (int r0 = 0; r0 < total; r0 += PT) {
            const int t = r0 + threadIdx.x;
            const bool on = t < total;
            const uint32_t c = on ? cst[t] : 256u + lane;
            const unsigned peers = __match_any_sync(FULL, c);
            const unsigned rank = __popc(peers & ((1u << lane) - 1u));
            for (int w = 0; w < PT / 32; ++w) wcnt[w][threadIdx.x] = 0;   // PT >= ... 256 cells: loop below
            for (int cc = threadIdx.x + PT; cc < 256; cc += PT)
                for (int w = 0; w < PT / 32; ++w) wcnt[w][cc] = 0;
            __syncthreads();
            if (on && rank == 0) wcnt[warp][c] = __popc(peers);
            __syncthreads();
            for (int cc = threadIdx.x; cc < 256; cc += PT) {
                uint32_t run = base[cc];
                for (int w = 0; w < PT / 32; ++w) {
                    wpre[w][cc] = run;
                    run += wcnt[w][cc];
                }
                base[cc] = run;
            }
            __syncthreads();
            if (on) {
                const int pos = U.y + (int)(wpre[warp][c] + rank);
                s_key[pos] = tile << 8 | c;
                s_idx[pos] = ist[t];
#pragma unroll
                for (int k = 0; k < WREC / 4; ++k) s_w[(size_t)pos * (WREC / 4) + k] = wst[t][k];
            }
            __syncthreads();
        }
    }
}

// One block: cut every tile's run of sorted visibilities into units of <= UMAX.
__global__ void __launch_bounds__(1024) k_units(const uint32_t *__restrict__ hist, int ntiles,
                                                int4 *__restrict__ units, int *__restrict__ n_units,
                                                int cap, uint32_t *__restrict__ n_valid_out) {
    __shared__ uint32_t sh[32];
    uint32_t carry = 0, base = 0;
    for (int b = 0; b < ntiles; b += 1024) {
        const int t = b + threadIdx.x;
        const uint32_t c = t < ntiles ? hist[t] : 0u;
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

// ------------------------------------------------------------------ accumulation

// ------------------------------------------------------------------ accumulation
// One CTA per work unit (<= UMAX visibilities of one 16x16-cell tile, sorted by
// cell).  The unit is staged in shared memory (1-D weights from the plan, the
// visibilities gathered) and cut into tasks: runs of at most CHUNK
// visibilities that share a cell.  A warp takes a task; lane k owns footprint
// cells k and k + 32 of the (2r+1)^2 around the run's cell and sums
// w = wx[dx] wy[dy] times V over the run (plain FP32 blocks of 8 folded into
// Kahan sums, fixed order), then adds its cells to the FP64 grid.  No shared
// accumulators: runs never wait on one another, whether the tile is dense
// (long runs) or sparse (short ones).
constexpr int WST = 17;          // floats per staged weight record (odd: spreads banks)
constexpr int GT = 256;          // threads per gridding CTA
constexpr int GFOLD = 8;
constexpr int CHUNK = 64;        // visibilities per task at most
constexpr int MAXTASK = UMAX + 256;
constexpr size_t GRID_SMEM = UMAX * (sizeof(float) * WST + sizeof(float2) + 1) + sizeof(uint32_t) * 257 +
                             sizeof(int2) * MAXTASK;

__global__ void __launch_bounds__(GT) k_grid(GridGeom G, const int4 *__restrict__ units,
                                             const int *__restrict__ n_units,
                                             const float4 *__restrict__ s_w,
                                             const uint32_t *__restrict__ s_idx,
                                             const uint32_t *__restrict__ s_key,
                                             const float2 *__restrict__ vis,
                                             double *__restrict__ acc_re,
                                             double *__restrict__ acc_im,
                                             double *__restrict__ acc_w,
                                             uint8_t *__restrict__ hit) {
    extern __shared__ __align__(16) uint8_t dsm[];
    float *st_w = (float *)dsm;                                        // [UMAX][WST] 1-D weights
    float2 *st_v = (float2 *)(st_w + UMAX * WST);                      // [UMAX] visibilities
    int2 *task = (int2 *)(st_v + UMAX);                                // [MAXTASK] (first, end)
    uint32_t *cstart = (uint32_t *)(task + MAXTASK);                   // [257] first item of each cell
    uint8_t *st_c = (uint8_t *)(cstart + 257);                         // [UMAX] cell in tile
    __shared__ int ntask_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = GT / 32;
    const int r = G.r, fw = 2 * r + 1, nfp = fw * fw;
    // this lane's two footprint cells
    const int k1 = lane, k2 = lane + 32;
    const bool on1 = k1 < nfp, on2 = k2 < nfp;
    const int dx1 = on1 ? k1 % fw : 0, dy1 = on1 ? k1 / fw : 0;
    const int dx2 = on2 ? k2 % fw : 0, dy2 = on2 ? k2 / fw : 0;
    const int nu = *n_units;
    for (int u = blockIdx.x; u < nu; u += gridDim.x) {
        const int4 U = units[u];
        const int total = U.z - U.y;
        __syncthreads();   // previous unit done with the staging buffers
        for (int e = threadIdx.x; e < total * (WREC / 4); e += GT) {
            const int t = e >> 2, k = e & 3;
            const float4 q = s_w[(size_t)(U.y + t) * (WREC / 4) + k];
            float *d = st_w + t * WST + 4 * k;
            d[0] = q.x;
            d[1] = q.y;
            d[2] = q.z;
            d[3] = q.w;
        }
        for (int t = threadIdx.x; t < total; t += GT) {
            st_c[t] = (uint8_t)(s_key[U.y + t] & 255u);
            st_v[t] = vis[s_idx[U.y + t]];
        }
        __syncthreads();
        for (int c = threadIdx.x; c <= 256; c += GT) {   // first item of each cell (unit is cell-sorted)
            int lo = 0, hi = total;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if ((int)st_c[mid] < c) lo = mid + 1;
                else hi = mid;
            }
            cstart[c] = (uint32_t)lo;
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
                for (uint32_t q = 0; q < nt[k]; ++q, ++pos) {
                    const int a = j0 + (int)q * CHUNK;
                    task[pos] = make_int2(a, min(j1, a + CHUNK));
                }
            }
            if (lane == 31) ntask_s = (int)incl;
        }
        __syncthreads();
        const int ntask = ntask_s;
        const int tile = U.x, tx = tile % G.tt, ty = tile / G.tt;
        const int gx0 = tx * TS - G.off, gy0 = ty * TS - G.off;
        for (int tk = warp; tk < ntask; tk += nwarps) {
            const int2 T = task[tk];
            float b1[3] = {0.f, 0.f, 0.f}, s1[3] = {0.f, 0.f, 0.f}, c1[3] = {0.f, 0.f, 0.f};
            float b2[3] = {0.f, 0.f, 0.f}, s2[3] = {0.f, 0.f, 0.f}, c2[3] = {0.f, 0.f, 0.f};
            int nblk = 0;
            for (int j = T.x; j < T.y; ++j) {
                const float *w = st_w + j * WST;
                const float2 v = st_v[j];
                const float wa = w[dx1] * w[8 + dy1];
                const float wb = w[dx2] * w[8 + dy2];
                b1[0] = fmaf(wa, v.x, b1[0]);
                b1[1] = fmaf(wa, v.y, b1[1]);
                b1[2] += wa;
                b2[0] = fmaf(wb, v.x, b2[0]);
                b2[1] = fmaf(wb, v.y, b2[1]);
                b2[2] += wb;
                if (++nblk == GFOLD) {
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        kahan_add(s1[k], c1[k], b1[k]);
                        kahan_add(s2[k], c2[k], b2[k]);
                        b1[k] = b2[k] = 0.f;
                    }
                    nblk = 0;
                }
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                kahan_add(s1[k], c1[k], b1[k]);
                kahan_add(s2[k], c2[k], b2[k]);
            }
            const int cell = st_c[T.x];
            const int cx = gx0 + (cell & (TS - 1)), cy = gy0 + (cell >> 4);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (h == 0 ? !on1 : !on2) continue;
                const int gx = cx + (h == 0 ? dx1 : dx2) - r, gy = cy + (h == 0 ? dy1 : dy2) - r;
                if (gx < -G.half || gx > G.half || gy < -G.half || gy > G.half) continue;
                const float *S = h == 0 ? s1 : s2;
                const float *C = h == 0 ? c1 : c2;
                const int64_t pidx = cell_index(G.n, gx, gy);
                atomicAdd(&acc_re[pidx], (double)S[0] - (double)C[0]);
                atomicAdd(&acc_im[pidx], (double)S[1] - (double)C[1]);
                atomicAdd(&acc_w[pidx], (double)S[2] - (double)C[2]);
                hit[pidx] = 1;
            }
        }
    }
}

// Hermitian mirror and FP32 outputs: G(g) + conj G(-g), W(g) + W(-g).
__global__ void k_grid_finalize(int n, const double *__restrict__ acc_re,
                                const double *__restrict__ acc_im,
                                const double *__restrict__ acc_w, const uint8_t *__restrict__ hit,
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
        mask[p] = (hit[p] | hit[pm]) ? 1 : 0;
    }
}

struct PlanBufs {
    uint32_t *keys, *hist, *offs, *bsum;
    float4 *s_w;          // [n][4] weight records
    uint32_t *s_idx, *s_key;
    uint32_t *k2, *v2, *vals, *rhist, *roffs, *n_valid;
    int4 *units;
    int *n_units;
    int64_t nkeys, n_vis;
    int ntiles, units_cap, rtiles;
};

bool plan_bufs(abs_ctx *ctx, const GridGeom &G, int64_t n_vis, PlanBufs &b) {
    b.ntiles = G.tt * G.tt;
    b.nkeys = b.ntiles;
    b.n_vis = n_vis;
    b.units_cap = (int)(b.ntiles + cdiv(n_vis, UMAX) + 1);
    const int64_t nv = n_vis > 0 ? n_vis : 1;
    b.keys = (uint32_t *)workspace(ctx, "plan.keys", sizeof(uint32_t) * nv);
    b.hist = (uint32_t *)workspace(ctx, "plan.hist", sizeof(uint32_t) * b.nkeys);
    b.offs = (uint32_t *)workspace(ctx, "plan.offs", sizeof(uint32_t) * b.nkeys);
    b.bsum = (uint32_t *)workspace(ctx, "plan.bsum", sizeof(uint32_t) * (cdiv(b.nkeys, 4096) + 1));
    b.s_w = (float4 *)workspace(ctx, "plan.s_w", sizeof(float4) * 4 * nv);
    b.s_idx = (uint32_t *)workspace(ctx, "plan.s_idx", sizeof(uint32_t) * nv);
    b.s_key = (uint32_t *)workspace(ctx, "plan.s_key", sizeof(uint32_t) * nv);
    b.units = (int4 *)workspace(ctx, "plan.units", sizeof(int4) * b.units_cap);
    b.n_units = (int *)workspace(ctx, "plan.n_units", sizeof(int));
    b.rtiles = (int)cdiv(nv, RTILE);
    b.k2 = (uint32_t *)workspace(ctx, "plan.k2", sizeof(uint32_t) * nv);
    b.v2 = (uint32_t *)workspace(ctx, "plan.v2", sizeof(uint32_t) * nv);
    b.vals = (uint32_t *)workspace(ctx, "plan.vals", sizeof(uint32_t) * nv);
    b.rhist = (uint32_t *)workspace(ctx, "plan.rhist", sizeof(uint32_t) * 256 * b.rtiles);
    b.roffs = (uint32_t *)workspace(ctx, "plan.roffs", sizeof(uint32_t) * 256 * b.rtiles);
    b.n_valid = (uint32_t *)workspace(ctx, "plan.n_valid", sizeof(uint32_t));
    return b.keys && b.hist && b.offs && b.bsum && b.s_w && b.s_idx && b.s_key && b.units &&
           b.n_units && b.k2 && b.v2 && b.vals && b.rhist && b.roffs && b.n_valid;
}

}  // namespace

// Exclusive scan of len uint32 values (3 kernels; bsum needs cdiv(len, 4096) + 1 entries).
void scan_u32(cudaStream_t st, const uint32_t *in, int64_t len, uint32_t *out, uint32_t *bsum) {
    const int nblk = (int)cdiv(len, 4096);
    k_scan_local<<<nblk, 1024, 0, st>>>(in, len, out, bsum);
    k_scan_top<<<1, 1024, 0, st>>>(bsum, nblk);
    k_scan_add<<<(int)cdiv(len, 256), 256, 0, st>>>(out, len, bsum);
}

abs_status launch_grid_plan(abs_ctx *ctx, const Setup &s, int64_t n_vis, const float *d_uv) {
    const GridGeom G = geom(s);
    PlanBufs b;
    if (!plan_bufs(ctx, G, n_vis, b)) return fail(ctx, ABS_ERR_OOM, "grid plan workspace");
    const int64_t rlen = (int64_t)256 * b.rtiles;
    const int64_t scan_len = std::max<int64_t>(b.nkeys, rlen);
    uint32_t *bsum = (uint32_t *)workspace(ctx, "plan.bsum2", sizeof(uint32_t) * (cdiv(scan_len, 4096) + 1));
    if (!bsum) return fail(ctx, ABS_ERR_OOM, "grid plan workspace");
    cudaStream_t st = ctx->stream;
    StageTimer timer(ctx, "grid_plan");
    cudaMemsetAsync(b.hist, 0, sizeof(uint32_t) * b.nkeys, st);
    const int grid_v = (int)std::min<int64_t>(cdiv(std::max<int64_t>(n_vis, 1), 256), ctx->sm_count * 16);
    const uint32_t key_none = (uint32_t)b.nkeys;     // invalid visibilities sort last
    if (n_vis > 0)
        k_plan_keys<<<grid_v, 256, 0, st>>>(G, n_vis, (const float2 *)d_uv, b.keys, b.vals, b.hist, key_none);
    k_units<<<1, 1024, 0, st>>>(b.hist, b.ntiles, b.units, b.n_units, b.units_cap, b.n_valid);
    if (n_vis > 0) {
        // stable sort of (tile, index); ping-pong keys/vals <-> k2/v2, result in k2/v2
        // or keys/vals; k_plan_units then sorts each unit by cell into s_key/s_idx
        int bits = 1;
        while (((uint64_t)1 << bits) <= (uint64_t)key_none) ++bits;
        const int passes = (bits + 7) / 8;
        uint32_t *ki = b.keys, *vi = b.vals, *ko = b.k2, *vo = b.v2;
        for (int ps = 0; ps < passes; ++ps) {
            k_radix_hist<<<b.rtiles, 256, 0, st>>>(ki, n_vis, 8 * ps, b.rtiles, b.rhist);
            scan_u32(st, b.rhist, rlen, b.roffs, bsum);
            k_radix_scatter<<<b.rtiles, 256, 0, st>>>(ki, vi, n_vis, 8 * ps, b.rtiles, b.roffs, ko, vo);
            if (ps == 0) {
                ki = b.k2;
                vi = b.v2;
                ko = b.keys;
                vo = b.vals;
            } else {
                std::swap(ki, ko);
                std::swap(vi, vo);
            }
        }
        // ki/vi now hold the tile-sorted (tile, index) pairs
        const int ub = std::min(b.units_cap, ctx->sm_count * 8);
        k_plan_units<<<ub, PT, 0, st>>>(G, b.units, b.n_units, (const float2 *)d_uv, vi, b.s_key, b.s_idx, b.s_w);
    }
    return check_launch(ctx, "grid plan");
}

void grid_acc_buffers(abs_ctx *ctx, const Setup &s, double **acc, uint8_t **hit) {
    const int64_t cells = (int64_t)s.n * s.n;
    *acc = (double *)workspace(ctx, "grid.acc", sizeof(double) * 3 * cells);
    *hit = (uint8_t *)workspace(ctx, "grid.hit", cells);
}

abs_status launch_grid_accumulate(abs_ctx *ctx, const Setup &s, int64_t n_vis, const float *d_vis,
                                  float *d_grid, float *d_wsum, uint8_t *d_mask) {
    const GridGeom G = geom(s);
    PlanBufs b;
    if (!plan_bufs(ctx, G, n_vis, b)) return fail(ctx, ABS_ERR_OOM, "grid plan workspace");
    const int64_t cells = (int64_t)s.n * s.n;
    double *acc = (double *)workspace(ctx, "grid.acc", sizeof(double) * 3 * cells);
    uint8_t *hit = (uint8_t *)workspace(ctx, "grid.hit", cells);
    if (!acc || !hit) return fail(ctx, ABS_ERR_OOM, "grid accumulation workspace");
    cudaStream_t st = ctx->stream;
    {
        StageTimer timer(ctx, "grid_zero");
        cudaMemsetAsync(acc, 0, sizeof(double) * 3 * cells, st);
        cudaMemsetAsync(hit, 0, cells, st);
    }
    if (n_vis > 0) {
        StageTimer timer(ctx, "grid");
        const int blocks = std::min(b.units_cap, ctx->sm_count * 4);
        k_grid<<<blocks, GT, GRID_SMEM, st>>>(G, b.units, b.n_units, b.s_w, b.s_idx, b.s_key,
                                           (const float2 *)d_vis, acc, acc + cells,
                                           acc + 2 * cells, hit);
    }
    {
        StageTimer timer(ctx, "grid_finalize");
        const int fb = (int)std::min<int64_t>(cdiv(cells, 256), ctx->sm_count * 8);
        k_grid_finalize<<<fb, 256, 0, st>>>(s.n, acc, acc + cells, acc + 2 * cells, hit,
                                            (float2 *)d_grid, d_wsum, d_mask);
    }
    return check_launch(ctx, "grid accumulate");
}

}  // namespace absk
