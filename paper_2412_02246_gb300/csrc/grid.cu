// Stage 1: gridding of visibilities, Eq. vg (Sec. 2).
//
// V_g = sum_i w(U_g - U_i) V(U_i) over the (2r+1)^2 cells around each
// visibility's nearest grid point, every visibility also entered at -U_i with
// V*.  The mirror is applied after accumulation (G(g) + conj G(-g)), which is
// the same sum.
//
// Plan (per baseline set): key every visibility by (16x16-cell uv tile, cell
// within the tile), counting-sort by key, and cut every tile's run into work
// units of at most UMAX visibilities.
//
// Accumulation (per realisation): a persistent kernel takes one unit per CTA
// pass.  Each warp has 4 slots of 8 lanes; a slot walks a contiguous run of
// the sorted visibilities, lane dx of the slot owning footprint column dx and
// keeping the 2r+1 cells of that column in registers (Kahan-compensated FP32)
// for as long as consecutive visibilities share a nearest cell.  When the cell
// changes the run is added into the warp's shared-memory halo tile
// (compensated FP32); at the end of the unit the warps' tiles are summed in
// FP64 and added to an FP64 grid with one atomic per touched cell.  A final
// pass applies the Hermitian mirror and writes the FP32 outputs.
//
// Weights: w = exp(-(dx - fx)^2 s) exp(-(dy - fy)^2 s), s = 1/(2 sigma^2),
// with the fractional offset f = u/dU - c carried as a float pair (the exact
// division residual) and the exponent argument formed in double-float, so
// that the only sizeable error is that of expf itself.
#include "abs_internal.cuh"

namespace absk {
namespace {

constexpr int TS = 16;                       // tile side in cells
constexpr int SLOTS = 4;                     // slots per warp, 8 lanes each
constexpr int GW = 4;                        // warps per CTA
constexpr int UMAX = 1024;                   // visibilities per work unit
constexpr int HS_MAX = TS + 2 * ABS_MAX_RADIUS;
constexpr int HC = HS_MAX * HS_MAX;          // halo-tile cells
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
                if (kx >= 0 && kx < G.ks && ky >= 0 && ky < G.ks) {
                    const int tx = kx / TS, ty = ky / TS;
                    key = (uint32_t)((ty * G.tt + tx) * (TS * TS) + (ky - ty * TS) * TS +
                                     (kx - tx * TS));
                }
            }
        }
        keys[i] = key;
        // one atomic per distinct key in the warp (consecutive visibilities of a
        // baseline usually share a cell)
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

// Fractional offset f = u/dU - c of every sorted visibility from its nearest
// cell, as a float pair (hi = fl(u/dU) - c exactly, lo = the exact division
// residual over dU): (fx_hi, fx_lo, fy_hi, fy_lo).
__global__ void k_plan_offsets(GridGeom G, int64_t n_valid_max, const uint32_t *__restrict__ n_valid_p,
                               const float2 *__restrict__ uv, const uint32_t *__restrict__ s_idx,
                               const uint32_t *__restrict__ s_key, float4 *__restrict__ s_f) {
    const uint32_t nv = *n_valid_p;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv && i < n_valid_max;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float2 p = uv[s_idx[i]];
        const uint32_t key = s_key[i];
        const int tile = (int)(key >> 8), tx = tile % G.tt, ty = tile / G.tt;
        const int cx = tx * TS + (int)(key & (TS - 1)) - G.off;
        const int cy = ty * TS + (int)((key >> 4) & (TS - 1)) - G.off;
        const float qx = __fdiv_rn(p.x, G.du), qy = __fdiv_rn(p.y, G.du);
        s_f[i] = make_float4(__fsub_rn(qx, (float)cx), __fdiv_rn(fmaf(-qx, G.du, p.x), G.du),
                             __fsub_rn(qy, (float)cy), __fdiv_rn(fmaf(-qy, G.du, p.y), G.du));
    }
}

// One block: cut every tile's run of sorted visibilities into units of <= UMAX.
__global__ void __launch_bounds__(1024) k_units(const uint32_t *__restrict__ offs,
                                                const uint32_t *__restrict__ hist, int64_t nkeys,
                                                int ntiles, int4 *__restrict__ units,
                                                int *__restrict__ n_units, int cap,
                                                uint32_t *__restrict__ n_valid_out) {
    __shared__ uint32_t sh[32];
    const uint32_t n_valid = offs[nkeys - 1] + hist[nkeys - 1];
    if (threadIdx.x == 0) *n_valid_out = n_valid;
    uint32_t carry = 0;
    for (int b = 0; b < ntiles; b += 1024) {
        const int t = b + threadIdx.x;
        uint32_t start = 0, end = 0, nu = 0;
        if (t < ntiles) {
            start = offs[(int64_t)t * (TS * TS)];
            end = t + 1 < ntiles ? offs[(int64_t)(t + 1) * (TS * TS)] : n_valid;
            nu = (end - start + UMAX - 1) / UMAX;
        }
        uint32_t total;
        const uint32_t pre = block_exclusive_scan(nu, sh, total);
        for (uint32_t k = 0; k < nu; ++k) {
            const uint32_t u = carry + pre + k;
            if ((int)u < cap) {
                const uint32_t s0 = start + k * UMAX;
                units[u] = make_int4(t, (int)s0, (int)min(end, s0 + UMAX), 0);
            }
        }
        carry += total;
    }
    if (threadIdx.x == 0) *n_units = min((int)carry, cap);
}

// ------------------------------------------------------------------ accumulation

// Per-lane accumulators of one slot lane: footprint column dx, rows dy, for
// (re, im, w).  blk: plain FP32 sums of up to FOLD visibilities; s, c: Kahan
// sum and compensation of the folded blocks.
constexpr int FOLD = 4;
struct SlotAcc {
    float blk[3][FWMAX], s[3][FWMAX], c[3][FWMAX];
};

__device__ __forceinline__ void acc_zero(SlotAcc &A) {
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int q = 0; q < FWMAX; ++q) A.blk[k][q] = A.s[k][q] = A.c[k][q] = 0.f;
}

__device__ __forceinline__ void acc_fold(SlotAcc &A) {
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int q = 0; q < FWMAX; ++q) {
            kahan_add(A.s[k][q], A.c[k][q], A.blk[k][q]);
            A.blk[k][q] = 0.f;
        }
}

__device__ __forceinline__ void slot_flush(float (*sm)[HC], SlotAcc &A, int hx0, int hy0, int HS,
                                           int fw, uint8_t *shit) {
    acc_fold(A);
#pragma unroll
    for (int dyi = 0; dyi < FWMAX; ++dyi) {
        if (dyi < fw) {
            const int ci = (hy0 + dyi) * HS + hx0;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                float ss = sm[2 * k][ci], cc = sm[2 * k + 1][ci];
                kahan_add(ss, cc, A.s[k][dyi] - A.c[k][dyi]);
                sm[2 * k][ci] = ss;
                sm[2 * k + 1][ci] = cc;
            }
            shit[ci] = 1;
        }
    }
}

constexpr size_t GRID_SMEM = sizeof(float) * GW * 6 * HC + UMAX * (sizeof(float4) + sizeof(float2) + 1) + HC;

__global__ void __launch_bounds__(GW * 32) k_grid(GridGeom G, const int4 *__restrict__ units,
                                                  const int *__restrict__ n_units,
                                                  const float4 *__restrict__ s_f,
                                                  const uint32_t *__restrict__ s_idx,
                                                  const uint32_t *__restrict__ s_key,
                                                  const float2 *__restrict__ vis,
                                                  double *__restrict__ acc_re,
                                                  double *__restrict__ acc_im,
                                                  double *__restrict__ acc_w,
                                                  uint8_t *__restrict__ hit) {
    extern __shared__ __align__(16) uint8_t dsm[];
    float(*sm)[6][HC] = (float(*)[6][HC])dsm;                          // [GW][6][HC]
    float4 *st_f = (float4 *)(dsm + sizeof(float) * GW * 6 * HC);      // [UMAX] offsets
    float2 *st_v = (float2 *)(st_f + UMAX);                            // [UMAX] visibilities
    uint8_t *st_c = (uint8_t *)(st_v + UMAX);                          // [UMAX] cell in tile
    uint8_t *shit = st_c + UMAX;                                       // [HC] touched cells
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int slot = lane >> 3, l8 = lane & 7;
    const int r = G.r, fw = 2 * r + 1, HS = TS + 2 * r;
    const bool lane_on = l8 < fw;
    const float d = (float)(l8 - r);
    const int nu = *n_units;
    for (int u = blockIdx.x; u < nu; u += gridDim.x) {
        const int4 U = units[u];
        const int total = U.z - U.y;
        for (int i = threadIdx.x; i < GW * 6 * HC; i += blockDim.x) (&sm[0][0][0])[i] = 0.f;
        for (int i = threadIdx.x; i < HC; i += blockDim.x) shit[i] = 0;
        for (int t = threadIdx.x; t < total; t += blockDim.x) {   // stage the unit
            st_f[t] = s_f[U.y + t];
            st_c[t] = (uint8_t)(s_key[U.y + t] & 255u);
            st_v[t] = vis[s_idx[U.y + t]];
        }
        __syncthreads();
        const int tile = U.x, tx = tile % G.tt, ty = tile / G.tt;
        const int gx0 = tx * TS - G.off, gy0 = ty * TS - G.off;
        const int nslots = GW * SLOTS;
        const int per = (total + nslots - 1) / nslots;
        const int sid = warp * SLOTS + slot;
        const int my0 = min(total, sid * per), my1 = min(total, (sid + 1) * per);
        int trips = my1 - my0;
        trips = max(trips, __shfl_xor_sync(FULL, trips, 8));
        trips = max(trips, __shfl_xor_sync(FULL, trips, 16));
        SlotAcc A;
        acc_zero(A);
        int run_c = -1, nblk = 0;
        for (int it = 0; it < trips; ++it) {
            const int idx = my0 + it;
            const bool act = idx < my1;
            float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
            float2 v = make_float2(0.f, 0.f);
            int cc = run_c;
            if (act) {
                f = st_f[idx];
                v = st_v[idx];
                cc = st_c[idx];
            }
            const bool need = act && run_c >= 0 && cc != run_c;
            if (__any_sync(FULL, need)) {
                for (int s = 0; s < SLOTS; ++s) {
                    if (slot == s && need && lane_on)
                        slot_flush(sm[warp], A, (run_c & (TS - 1)) + l8, run_c >> 4, HS, fw, shit);
                    __syncwarp();
                }
                if (need) {
                    acc_zero(A);
                    nblk = 0;
                }
            }
            if (act) run_c = cc;
            float wx = 1.f, wyl = 1.f;
            if (G.kernel == ABS_KERNEL_GAUSS) {
                wx = wexp(d, f.x, f.y, G.s_hi, G.s_lo);
                wyl = wexp(d, f.z, f.w, G.s_hi, G.s_lo);
            }
            const int sbase = slot * 8;
#pragma unroll
            for (int dyi = 0; dyi < FWMAX; ++dyi) {
                const float wy = __shfl_sync(FULL, wyl, sbase + dyi);
                if (dyi < fw && act && lane_on) {
                    const float w = wx * wy;
                    A.blk[0][dyi] = fmaf(w, v.x, A.blk[0][dyi]);
                    A.blk[1][dyi] = fmaf(w, v.y, A.blk[1][dyi]);
                    A.blk[2][dyi] += w;
                }
            }
            if (act && ++nblk == FOLD) {
                acc_fold(A);
                nblk = 0;
            }
        }
        for (int s = 0; s < SLOTS; ++s) {
            if (slot == s && run_c >= 0 && lane_on)
                slot_flush(sm[warp], A, (run_c & (TS - 1)) + l8, run_c >> 4, HS, fw, shit);
            __syncwarp();
        }
        __syncthreads();
        for (int i = threadIdx.x; i < HS * HS; i += blockDim.x) {
            if (!shit[i]) continue;
            const int hx = i % HS, hy = i / HS;
            const int gx = gx0 - r + hx, gy = gy0 - r + hy;
            if (gx < -G.half || gx > G.half || gy < -G.half || gy > G.half) continue;
            double re = 0.0, im = 0.0, w = 0.0;
#pragma unroll
            for (int wv = 0; wv < GW; ++wv) {
                re += (double)sm[wv][0][i] - (double)sm[wv][1][i];
                im += (double)sm[wv][2][i] - (double)sm[wv][3][i];
                w += (double)sm[wv][4][i] - (double)sm[wv][5][i];
            }
            const int64_t pidx = cell_index(G.n, gx, gy);
            atomicAdd(&acc_re[pidx], re);
            atomicAdd(&acc_im[pidx], im);
            atomicAdd(&acc_w[pidx], w);
            hit[pidx] = 1;
        }
        __syncthreads();
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
    float4 *s_f;
    uint32_t *s_idx, *s_key;
    uint32_t *k2, *v2, *vals, *rhist, *roffs, *n_valid;
    int4 *units;
    int *n_units;
    int64_t nkeys, n_vis;
    int ntiles, units_cap, rtiles;
};

bool plan_bufs(abs_ctx *ctx, const GridGeom &G, int64_t n_vis, PlanBufs &b) {
    b.ntiles = G.tt * G.tt;
    b.nkeys = (int64_t)b.ntiles * TS * TS;
    b.n_vis = n_vis;
    b.units_cap = (int)(b.ntiles + cdiv(n_vis, UMAX) + 1);
    const int64_t nv = n_vis > 0 ? n_vis : 1;
    b.keys = (uint32_t *)workspace(ctx, "plan.keys", sizeof(uint32_t) * nv);
    b.hist = (uint32_t *)workspace(ctx, "plan.hist", sizeof(uint32_t) * b.nkeys);
    b.offs = (uint32_t *)workspace(ctx, "plan.offs", sizeof(uint32_t) * b.nkeys);
    b.bsum = (uint32_t *)workspace(ctx, "plan.bsum", sizeof(uint32_t) * (cdiv(b.nkeys, 4096) + 1));
    b.s_f = (float4 *)workspace(ctx, "plan.s_f", sizeof(float4) * nv);
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
    return b.keys && b.hist && b.offs && b.bsum && b.s_f && b.s_idx && b.s_key && b.units &&
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
    scan_u32(st, b.hist, b.nkeys, b.offs, bsum);
    k_units<<<1, 1024, 0, st>>>(b.offs, b.hist, b.nkeys, b.ntiles, b.units, b.n_units, b.units_cap,
                                b.n_valid);
    if (n_vis > 0) {
        // stable sort of (key, index); ping-pong keys/vals <-> k2/v2, result in s_key/s_idx
        int bits = 1;
        while (((uint64_t)1 << bits) <= (uint64_t)key_none) ++bits;
        const int passes = (bits + 7) / 8;
        uint32_t *ki = b.keys, *vi = b.vals, *ko = b.k2, *vo = b.v2;
        for (int ps = 0; ps < passes; ++ps) {
            if (ps == passes - 1) {
                ko = b.s_key;
                vo = b.s_idx;
            }
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
        k_plan_offsets<<<grid_v, 256, 0, st>>>(G, n_vis, b.n_valid, (const float2 *)d_uv, b.s_idx, b.s_key,
                                               b.s_f);
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
        const int blocks = std::min(b.units_cap, ctx->sm_count * 3);
        cudaFuncSetAttribute(k_grid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GRID_SMEM);
        k_grid<<<blocks, GW * 32, GRID_SMEM, st>>>(G, b.units, b.n_units, b.s_f, b.s_idx, b.s_key,
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
