// Multi-frequency (3-D) form of the estimator: a reading of the generalisation
// to the three-dimensional bispectrum that Sec. 1 and Sec. 5 name as future
// work (the paper gives no formula for it; the reading follows the route the
// paper cites for the power spectrum: the single-frequency statistic first,
// then a transform along frequency).
//
//   channels      every channel c = 0 .. n_chan-1 is gridded on the same uv
//                 grid (Eq. vg, the 2-D path's plan and gridder);
//   common cells  a cell enters only if it is filled in every channel;
//   delay modes   Xt(g, t) = sum_c X_c(g) exp(-2 pi i c t / n_chan) on those
//                 cells, |t| <= t_max with 2 t_max < n_chan (double-float);
//   bins          voxel (g, t) lies in bin u = m n_dbins + a when g is in ring
//                 a_m and tau_a <= |t| < tau_{a+1} (symmetric in t, so every
//                 3-D field is real);
//   fields        D_u(z, p) = sum over bin u of Xt(g, t) exp(-2 pi i (t z / N_z
//                 + g.p / N)) on an N_z x N x N grid: the 2-D ring transforms of
//                 the delay modes (k_fft_cols_delay and the row pass give F1, F2
//                 with FFT(Xt(., +-t)) = F1 +- i F2), then a direct length-N_z
//                 transform along z (k_cube_zexpand):
//                 D_u = F1_0 [0 in a] + sum_{t > 0 in a} 2 (F1_t cos + F2_t sin)(2 pi t z / N_z);
//   sums          S_uvw = (N^2 N_z)^-1 sum over voxels of D_u D_v D_w by the 2-D
//                 path's triple-sum kernels (FP32 or split-BF16) over N_z N^2
//                 points (on the split-BF16 path with the canonical list the
//                 line-of-sight pass writes that kernel's split planes itself):
//                 the sum over voxel triangles closed in g and in t, with no wrap
//                 when N >= 3R + 1 and N_z >= 3 t_max + 1;
//   counts        the voxel triangles close in g and t independently and the
//                 common mask does not depend on t, so T_uvw = T2(rings) x
//                 T1(delay bins): the 2-D exact counts on the common mask times
//                 the integer delay count (a table of the binning);
//   estimate      B_uvw = Re S_uvw / (A T_uvw), NaN where T = 0.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "abs_internal.cuh"

namespace absk {
namespace {

// One channel's weighted means on the region |gx|, |gy| <= Rr (mirror applied, the sums and
// the quotient X = (re_g + re_-g, im_g - im_-g) / (w_g + w_-g) in FP64 on filled cells), stored
// as packed double-float complex (re.hi, im.hi, re.lo, im.lo), and the channel's filled flag of
// every region cell.
__global__ void k_cube_take(int n, int Rr, int64_t cells, const double *__restrict__ acc, float4 *__restrict__ xc,
                            uint8_t *__restrict__ filled) {
    const int side = 2 * Rr + 1;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= side * side) return;
    const int y = idx / side - Rr, x = idx - (idx / side) * side - Rr;
    const int64_t cell = (int64_t)(y < 0 ? y + n : y) * n + (x < 0 ? x + n : x);
    const int64_t mcell = (int64_t)(y > 0 ? n - y : -y) * n + (x > 0 ? n - x : -x);
    const double ww = acc[2 * cells + cell] + acc[2 * cells + mcell];
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (ww > 0.0) {
        const double re = (acc[cell] + acc[mcell]) / ww, im = (acc[cells + cell] - acc[cells + mcell]) / ww;
        v.x = __double2float_rn(re);
        v.y = __double2float_rn(im);
        v.z = __double2float_rn(re - (double)v.x);
        v.w = __double2float_rn(im - (double)v.y);
    }
    xc[idx] = v;
    filled[idx] = ww > 0.0 ? 1 : 0;
}

// Double-float arithmetic (a value is hi + lo, two FP32 numbers): Knuth's TwoSum of the high
// parts with the low parts added, Dekker's product with the FMA remainder, both renormalised.
struct dfl {
    float h, l;
};
__device__ __forceinline__ dfl dfl_add(dfl a, dfl b) {
    const float s = __fadd_rn(a.h, b.h);
    const float bb = __fsub_rn(s, a.h);
    float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
    e = __fadd_rn(e, __fadd_rn(a.l, b.l));
    const float h = __fadd_rn(s, e);
    return {h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ dfl dfl_mul(dfl a, dfl b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    const float h = __fadd_rn(p, e);
    return {h, __fsub_rn(e, __fsub_rn(h, p))};
}

// Delay modes t = blockIdx.y of every region cell filled in all n_chan channels: the sum over
// the channels of X_c times exp(-2 pi i e / n_chan), e = c t mod n_chan, in double-float
// (GB300's FP64 pipe is narrow; about 2^-44 relative per product), stored as packed
// double-float complex; zero on the other cells.  The first delay also writes the common
// filled mask of the n x n grid (region cells only).
__global__ void k_cube_los(int n, int Rr, int n_chan, const float4 *__restrict__ xc, const uint8_t *__restrict__ filled,
                           const float4 *__restrict__ tw, float4 *__restrict__ xt, uint8_t *__restrict__ mask) {
    const int side = 2 * Rr + 1, side2 = side * side;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= side2) return;
    const int t = blockIdx.y;
    bool common = true;
    for (int c = 0; c < n_chan; ++c) common = common && filled[(size_t)c * side2 + idx];
    dfl sr = {0.f, 0.f}, si = {0.f, 0.f};
    if (common) {
        int e = 0;   // c t mod n_chan, advanced by t per channel
        for (int c = 0; c < n_chan; ++c) {
            const float4 w = __ldg(tw + e), x = xc[(size_t)c * side2 + idx];   // (re.hi, im.hi, re.lo, im.lo)
            const dfl xr = {x.x, x.z}, xi = {x.y, x.w}, wr = {w.x, w.z}, wi = {w.y, w.w};
            const dfl ni = dfl_mul(xi, wi);
            sr = dfl_add(sr, dfl_add(dfl_mul(xr, wr), {-ni.h, -ni.l}));
            si = dfl_add(si, dfl_add(dfl_mul(xr, wi), dfl_mul(xi, wr)));
            e += t;
            if (e >= n_chan) e -= n_chan;
        }
    }
    xt[(size_t)t * side2 + idx] = make_float4(sr.h, si.h, sr.l, si.l);
    if (t == 0) {
        const int y = idx / side - Rr, x = idx - (idx / side) * side - Rr;
        mask[(int64_t)(y < 0 ? y + n : y) * n + (x < 0 ? x + n : x)] = common ? 1 : 0;
    }
}

// Where k_cube_zexpand puts voxel v of bin u: FP32 fields [u][v], or the split-BF16 kernel's
// three planes (the layout SplitOut describes: [P_pad / 64][nbp][64], each 64-point row in the
// 128-byte swizzle of the tensor-core operand, 16-byte units XOR-permuted by u & 7), each value
// split once into hi = bf16(x) and lo = bf16(x - hi) beside its FP32 copy.
struct VoxelFields {
    float *D;
    int64_t P;
    __device__ void put(int u, int64_t v, float x) const { D[(size_t)u * P + v] = x; }
};
struct VoxelPlanes {
    SplitOut o;
    __device__ void put(int u, int64_t v, float x) const {
        const int w = (int)(v & 63), key = u & 7;
        const size_t row = ((size_t)(v >> 6) * o.nbp + u) * 64;
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        const __nv_bfloat16 l = __float2bfloat16_rn(__fsub_rn(x, __bfloat162float(h)));   // exact in FP32
        const size_t ob = row + (size_t)((((w >> 3) ^ key) << 3) | (w & 7));
        ((__nv_bfloat16 *)o.hi)[ob] = h;
        ((__nv_bfloat16 *)o.lo)[ob] = l;
        o.f32[row + (size_t)((((w >> 2) ^ key) << 2) | (w & 3))] = x;
    }
};

// The direct transform along the line of sight: for ring m = blockIdx.y and pixel p, voxel
// z N^2 + p of bin m na + a is the sum over t >= 0 in delay bin a of F1_t(p) c_tz + F2_t(p) s_tz,
// with (c, s) = (cos, sin)(2 pi t z / N_z) times 1 for t = 0 and 2 for t > 0 (the table
// ztw [t1][N_z], staged in shared memory).  Eight z a pass, so each F value is loaded once per
// pass.
constexpr int ZB = 8;
template <class Out>
__global__ void __launch_bounds__(256) k_cube_zexpand(int64_t P2, int t1, int na, const int32_t *__restrict__ tau,
                                                     int Nz, const float *__restrict__ F,
                                                     const float2 *__restrict__ ztw, const Out out) {
    extern __shared__ float2 stw[];
    for (int i = threadIdx.x; i < t1 * Nz; i += blockDim.x) stw[i] = ztw[i];
    __syncthreads();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P2) return;
    const int m = blockIdx.y;
    const float *Fm = F + (size_t)2 * m * t1 * P2;
    for (int a = 0; a < na; ++a) {
        const int ta = tau[a], tb = min(tau[a + 1], t1);
        const int u = m * na + a;
        for (int z0 = 0; z0 < Nz; z0 += ZB) {
            float acc[ZB];
#pragma unroll
            for (int k = 0; k < ZB; ++k) acc[k] = 0.f;
            for (int t = ta; t < tb; ++t) {
                const float f1 = Fm[(size_t)(2 * t) * P2 + p], f2 = Fm[(size_t)(2 * t + 1) * P2 + p];
                const float2 *row = stw + (size_t)t * Nz;
#pragma unroll
                for (int k = 0; k < ZB; ++k) {
                    if (z0 + k < Nz) {
                        const float2 w = row[z0 + k];
                        acc[k] = fmaf(f1, w.x, fmaf(f2, w.y, acc[k]));
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < ZB; ++k)
                if (z0 + k < Nz) out.put(u, (int64_t)(z0 + k) * P2 + p, acc[k]);
        }
    }
}

// T_uvw = T2(sorted rings of u, v, w) x T1(delay bins of u, v, w); T2 of a ring triplet
// outside the 2-D canonical list (idx2d = -1) is 0.  Out-of-range bins give 0 (the
// triplet check latches the error).
__global__ void k_cube_counts(int n_trip, int nb, int na, const int32_t *__restrict__ uvw,
                              const int32_t *__restrict__ idx2d, const int64_t *__restrict__ T2,
                              const int64_t *__restrict__ T1, int64_t *__restrict__ T3) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n_trip) return;
    const int nb3 = nb * na;
    const int u = uvw[3 * x], v = uvw[3 * x + 1], w = uvw[3 * x + 2];
    if (u < 0 || v < 0 || w < 0 || u >= nb3 || v >= nb3 || w >= nb3) {
        T3[x] = 0;
        return;
    }
    int r0 = u / na, r1 = v / na, r2 = w / na;
    if (r0 > r1) { const int tt = r0; r0 = r1; r1 = tt; }
    if (r1 > r2) { const int tt = r1; r1 = r2; r2 = tt; }
    if (r0 > r1) { const int tt = r0; r0 = r1; r1 = tt; }
    const int i2 = idx2d[((size_t)r0 * nb + r1) * nb + r2];
    const int64_t t2 = i2 >= 0 ? T2[i2] : 0;
    T3[x] = t2 * T1[((size_t)(u % na) * na + (v % na)) * na + (w % na)];
}

template <class T>
T *upload_vec(const std::vector<T> &v) {
    T *d = nullptr;
    const size_t bytes = sizeof(T) * std::max<size_t>(v.size(), 1);
    if (cudaMalloc(&d, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (!v.empty() && cudaMemcpy(d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(d);
        return nullptr;
    }
    return d;
}

}  // namespace

CubeSetup::~CubeSetup() {
    cudaFree(st.d_ijk);
    cudaFree(d_idx2d);
    cudaFree(d_rm2);
    cudaFree(d_tau);
    cudaFree(d_T1);
    cudaFree(d_los_tw);
    cudaFree(d_ztw);
}

abs_status derive_cube(const abs_config3d *cfg, const Setup &s2, int &t_max, int &Nz, std::vector<int64_t> &T1,
                       std::vector<int32_t> &uvw, const char **err) {
    if (!cfg) { *err = "NULL config"; return ABS_ERR_INVALID_ARG; }
    if (cfg->base.weight_mode != ABS_W_MEAN_UNITMASK) {
        *err = "the multi-frequency form takes the unit-mask weighting only";
        return ABS_ERR_UNSUPPORTED;
    }
    if (cfg->n_chan < 1 || cfg->n_chan > ABS_MAX_CHAN) { *err = "n_chan must be in [1, ABS_MAX_CHAN]"; return ABS_ERR_INVALID_ARG; }
    const int na = cfg->n_dbins;
    if (na < 1 || !cfg->delay_edges) { *err = "n_dbins must be >= 1 with delay_edges given"; return ABS_ERR_INVALID_ARG; }
    const int32_t *tau = cfg->delay_edges;
    if (tau[0] < 0) { *err = "delay_edges[0] must be >= 0"; return ABS_ERR_INVALID_ARG; }
    for (int a = 0; a < na; ++a)
        if (tau[a + 1] <= tau[a]) { *err = "delay_edges must be strictly ascending"; return ABS_ERR_INVALID_ARG; }
    t_max = tau[na] - 1;
    if (t_max > ABS_MAX_DELAY) { *err = "delay_edges[n_dbins] - 1 exceeds ABS_MAX_DELAY"; return ABS_ERR_UNSUPPORTED; }
    if (2 * t_max >= cfg->n_chan) { *err = "delay_edges[n_dbins] - 1 must be below n_chan / 2"; return ABS_ERR_INVALID_ARG; }
    if ((int64_t)s2.nb * na > ABS_MAX_BINS) { *err = "n_bins x n_dbins exceeds ABS_MAX_BINS"; return ABS_ERR_UNSUPPORTED; }
    if ((int64_t)s2.nb * (t_max + 1) > 65535) { *err = "n_bins x (delay_edges[n_dbins]) exceeds 65535"; return ABS_ERR_UNSUPPORTED; }
    Nz = cfg->n_z == 0 ? 3 * t_max + 1 : cfg->n_z;
    if (Nz < 3 * t_max + 1 || Nz > 4 * ABS_MAX_DELAY + 4) {
        *err = "n_z must be 0 or in [3 t_max + 1, 4 ABS_MAX_DELAY + 4]";
        return ABS_ERR_INVALID_ARG;
    }
    // delay counts of the binning: ordered (t1, t2, t3), |t| <= t_max, t1 + t2 + t3 = 0
    auto bin_of = [&](int t) {
        const int at = t < 0 ? -t : t;
        for (int a = 0; a < na; ++a)
            if (at >= tau[a] && at < tau[a + 1]) return a;
        return -1;
    };
    T1.assign((size_t)na * na * na, 0);
    for (int ta = -t_max; ta <= t_max; ++ta)
        for (int tb = -t_max; tb <= t_max; ++tb) {
            const int tc = -(ta + tb);
            if (tc < -t_max || tc > t_max) continue;
            const int a = bin_of(ta), b = bin_of(tb), c = bin_of(tc);
            if (a >= 0 && b >= 0 && c >= 0) T1[((size_t)a * na + b) * na + c] += 1;
        }
    // canonical bin triplets: rings (sorted) in the 2-D closing list, delay count > 0
    const int nb = s2.nb;
    std::vector<uint8_t> ring_ok((size_t)nb * nb * nb, 0);
    for (size_t t = 0; t < s2.ijk.size() / 3; ++t)
        ring_ok[((size_t)s2.ijk[3 * t] * nb + s2.ijk[3 * t + 1]) * nb + s2.ijk[3 * t + 2]] = 1;
    const int nb3 = nb * na;
    uvw.clear();
    for (int u = 0; u < nb3; ++u)
        for (int v = u; v < nb3; ++v)
            for (int w = v; w < nb3; ++w) {
                int r[3] = {u / na, v / na, w / na};
                std::sort(r, r + 3);
                if (!ring_ok[((size_t)r[0] * nb + r[1]) * nb + r[2]]) continue;
                if (T1[((size_t)(u % na) * na + (v % na)) * na + (w % na)] == 0) continue;
                uvw.push_back(u);
                uvw.push_back(v);
                uvw.push_back(w);
            }
    return ABS_OK;
}

static std::string cube_key(const abs_config3d *c) {
    std::string k;
    auto put = [&k](const void *p, size_t n) { k.append((const char *)p, n); };
    put(&c->n_chan, sizeof c->n_chan);
    put(&c->n_dbins, sizeof c->n_dbins);
    put(c->delay_edges, sizeof(int32_t) * (c->n_dbins + 1));
    put(&c->n_z, sizeof c->n_z);
    return k;
}

const CubeSetup *get_cube_setup(abs_ctx *ctx, const abs_config3d *cfg, abs_status &st) {
    if (!cfg || cfg->n_dbins < 1 || !cfg->delay_edges) {
        st = fail(ctx, ABS_ERR_INVALID_ARG, "invalid multi-frequency config (n_dbins / delay_edges)");
        return nullptr;
    }
    const Setup *s2 = get_setup(ctx, &cfg->base, st);
    if (!s2) return nullptr;
    const std::string key = s2->key + "|cube|" + cube_key(cfg);
    auto it = ctx->cubes.find(key);
    if (it != ctx->cubes.end()) {
        st = ABS_OK;
        return it->second.get();
    }
    std::unique_ptr<CubeSetup> c(new CubeSetup);
    const char *msg = "";
    std::vector<int32_t> uvw;
    st = derive_cube(cfg, *s2, c->t_max, c->Nz, c->T1, uvw, &msg);
    if (st != ABS_OK) {
        fail(ctx, st, msg);
        return nullptr;
    }
    c->s2 = s2;
    c->n_chan = cfg->n_chan;
    c->na = cfg->n_dbins;
    c->tau.assign(cfg->delay_edges, cfg->delay_edges + cfg->n_dbins + 1);
    // the triple stage: bins u = m n_dbins + a, N_z N^2 points, the canonical list
    Setup &t = c->st;
    t.n = s2->n;
    t.half = s2->half;
    t.nb = s2->nb * c->na;
    t.N = s2->N;
    t.P = (int64_t)s2->N * s2->N * c->Nz;
    t.precision = s2->precision;
    t.norm_A = s2->norm_A;
    t.weight_mode = s2->weight_mode;
    t.ijk = uvw;
    t.key = key;
    // tables: 2-D triplet index of every sorted ring triple, per-pair ring extent, twiddles
    const int nb = s2->nb, t1 = c->t_max + 1;
    std::vector<int32_t> idx2d((size_t)nb * nb * nb, -1);
    for (size_t x = 0; x < s2->ijk.size() / 3; ++x)
        idx2d[((size_t)s2->ijk[3 * x] * nb + s2->ijk[3 * x + 1]) * nb + s2->ijk[3 * x + 2]] = (int32_t)x;
    std::vector<int32_t> rm2((size_t)2 * nb * t1);
    for (int m = 0; m < nb; ++m)
        for (int d = 0; d < t1; ++d) rm2[2 * ((size_t)m * t1 + d)] = rm2[2 * ((size_t)m * t1 + d) + 1] = s2->Rm[m];
    std::vector<float4> los(c->n_chan);   // exp(-2 pi i e / n_chan) as double-float (re.hi, im.hi, re.lo, im.lo)
    for (int e = 0; e < c->n_chan; ++e) {
        const double a = -2.0 * M_PI * (double)e / (double)c->n_chan;
        const double cr = std::cos(a), ci = std::sin(a);
        const float rh = (float)cr, ih = (float)ci;
        los[e] = make_float4(rh, ih, (float)(cr - (double)rh), (float)(ci - (double)ih));
    }
    std::vector<float2> ztw((size_t)t1 * c->Nz);
    for (int d = 0; d < t1; ++d)
        for (int z = 0; z < c->Nz; ++z) {
            const double a = 2.0 * M_PI * (double)(((int64_t)d * z) % c->Nz) / (double)c->Nz;
            const double f = d == 0 ? 1.0 : 2.0;
            ztw[(size_t)d * c->Nz + z] = make_float2((float)(f * std::cos(a)), (float)(f * std::sin(a)));
        }
    t.d_ijk = upload_vec(t.ijk);
    c->d_idx2d = upload_vec(idx2d);
    c->d_rm2 = upload_vec(rm2);
    c->d_tau = upload_vec(c->tau);
    c->d_T1 = upload_vec(c->T1);
    c->d_los_tw = upload_vec(los);
    c->d_ztw = upload_vec(ztw);
    if (!t.d_ijk || !c->d_idx2d || !c->d_rm2 || !c->d_tau || !c->d_T1 || !c->d_los_tw || !c->d_ztw) {
        st = fail(ctx, ABS_ERR_OOM, "multi-frequency setup tables");
        return nullptr;
    }
    CubeSetup *raw = c.get();
    ctx->cubes[key] = std::move(c);
    st = ABS_OK;
    return raw;
}

abs_status launch_cube_estimate(abs_ctx *ctx, const CubeSetup &c, int64_t n_vis, const float *d_uv,
                                const float *d_vis, int32_t n_trip, const int32_t *d_uvw, double *d_B,
                                int64_t *d_count, double *d_ellbar) {
    const Setup &s2 = *c.s2;
    const Setup &st = c.st;
    const int Rr = s2.R, side = 2 * Rr + 1, side2 = side * side, t1 = c.t_max + 1;
    const int64_t cells = (int64_t)s2.n * s2.n, P2 = (int64_t)s2.N * s2.N;
    const int n_trip2 = (int)(s2.ijk.size() / 3);
    float4 *xc = (float4 *)workspace(ctx, "cube.xc", sizeof(float4) * (size_t)c.n_chan * side2);
    uint8_t *filled = (uint8_t *)workspace(ctx, "cube.filled", (size_t)c.n_chan * side2);
    float4 *xt = (float4 *)workspace(ctx, "cube.xt", sizeof(float4) * (size_t)t1 * side2);
    uint8_t *mask = (uint8_t *)workspace(ctx, "cube.mask", (size_t)cells);
    float *F = (float *)workspace(ctx, "cube.F", sizeof(float) * (size_t)2 * s2.nb * t1 * P2);
    // split-BF16 sums over the canonical list: the line-of-sight transform writes the tensor-core
    // kernel's planes directly, and no FP32 voxel fields are kept
    const bool to_planes = st.precision == ABS_SPLIT_BF16 && d_uvw == st.d_ijk && n_trip > 0;
    SplitOut planes{};
    if (to_planes) ABS_CHECK(tc_split_target(ctx, st, planes));
    float *D = to_planes ? nullptr : (float *)workspace(ctx, "cube.D", sizeof(float) * (size_t)st.nb * st.P);
    double *sum = (double *)workspace(ctx, "cube.sum", sizeof(double) * std::max(n_trip, 1));
    int64_t *t2 = (int64_t *)workspace(ctx, "cube.t2", sizeof(int64_t) * std::max(n_trip2, 1));
    int64_t *count = d_count ? d_count : (int64_t *)workspace(ctx, "cube.count", sizeof(int64_t) * std::max(n_trip, 1));
    if (!xc || !filled || !xt || !mask || !F || (!D && !to_planes) || !sum || !t2 || !count)
        return fail(ctx, ABS_ERR_OOM, "multi-frequency workspace");
    cudaStream_t s = ctx->stream;
    if (d_uvw != st.d_ijk) ABS_CHECK(launch_check_triplets(ctx, st, n_trip, d_uvw));
    cudaMemsetAsync(mask, 0, (size_t)cells, s);
    // every channel: the 2-D gridding plan and accumulation, then its means on the region; the
    // channels run round-robin over the context's lanes (concurrent streams with workspaces of
    // their own), forked from and joined back to its stream, except while the stage profiler runs
    // or on the legacy default stream
    const int K = (ctx->profiling || !s || c.n_chan < 2) ? 1 : std::min(ABS_BATCH_LANES, c.n_chan);
    if (K > 1) {
        ABS_CHECK(ensure_lanes(ctx, K));
        cudaEventRecord(ctx->ev_fork, s);
        for (int l = 0; l < K; ++l) cudaStreamWaitEvent(ctx->lanes[l]->stream, ctx->ev_fork, 0);
    }
    abs_status cst = ABS_OK;
    for (int ch = 0; ch < c.n_chan && cst == ABS_OK; ++ch) {
        abs_ctx *lc = K > 1 ? ctx->lanes[ch % K] : ctx;
        cst = launch_grid_plan(lc, s2, n_vis, d_uv + (size_t)ch * 2 * n_vis, true);
        if (cst == ABS_OK) cst = launch_grid_accumulate(lc, s2, n_vis, d_vis + (size_t)ch * 2 * n_vis, nullptr, nullptr, nullptr);
        double *acc = nullptr;
        if (cst == ABS_OK) {
            grid_acc_buffers(lc, s2, &acc);
            if (!acc) cst = fail(lc, ABS_ERR_OOM, "grid accumulation workspace");
        }
        if (cst == ABS_OK) {
            StageTimer timer(lc, "cube_take");
            k_cube_take<<<(int)cdiv(side2, 256), 256, 0, lc->stream>>>(s2.n, Rr, cells, acc, xc + (size_t)ch * side2,
                                                                       filled + (size_t)ch * side2);
            cst = check_launch(lc, "channel means");
        }
        if (cst != ABS_OK && lc != ctx) ctx->last_error = "channel " + std::to_string(ch) + ": " + lc->last_error;
    }
    if (K > 1)   // join: the context's stream waits for every lane
        for (int l = 0; l < K; ++l) {
            cudaEventRecord(ctx->lanes[l]->ev_lane, ctx->lanes[l]->stream);
            cudaStreamWaitEvent(s, ctx->lanes[l]->ev_lane, 0);
        }
    if (cst != ABS_OK) return cst;
    {
        StageTimer timer(ctx, "cube_los");
        k_cube_los<<<dim3((unsigned)cdiv(side2, 128), t1), 128, 0, s>>>(s2.n, Rr, c.n_chan, xc, filled, c.d_los_tw,
                                                                       xt, mask);
    }
    ABS_CHECK(check_launch(ctx, "delay modes"));
    // exact counts: 2-D counts on the common mask (and the rings' mean l), times the delay counts
    ABS_CHECK(launch_counts(ctx, s2, mask, n_trip2, s2.d_ijk, t2, d_ellbar));
    if (n_trip > 0) {
        StageTimer timer(ctx, "cube_counts");
        k_cube_counts<<<(int)cdiv(n_trip, 256), 256, 0, s>>>(n_trip, s2.nb, c.na, d_uvw, c.d_idx2d, t2, c.d_T1,
                                                             count);
    }
    ABS_CHECK(launch_filter_fft_delay(ctx, s2, c.t_max, xt, c.d_rm2, F));
    {
        const size_t zsm = sizeof(float2) * (size_t)t1 * c.Nz;
        const dim3 grid((unsigned)cdiv(P2, 256), s2.nb);
        StageTimer timer(ctx, "cube_zexpand");
        if (to_planes) {
            if (!allow_smem(k_cube_zexpand<VoxelPlanes>, zsm))
                return fail(ctx, ABS_ERR_UNSUPPORTED, "line-of-sight twiddles do not fit shared memory");
            k_cube_zexpand<VoxelPlanes><<<grid, 256, zsm, s>>>(P2, t1, c.na, c.d_tau, c.Nz, F, c.d_ztw,
                                                              VoxelPlanes{planes});
        } else {
            if (!allow_smem(k_cube_zexpand<VoxelFields>, zsm))
                return fail(ctx, ABS_ERR_UNSUPPORTED, "line-of-sight twiddles do not fit shared memory");
            k_cube_zexpand<VoxelFields><<<grid, 256, zsm, s>>>(P2, t1, c.na, c.d_tau, c.Nz, F, c.d_ztw,
                                                              VoxelFields{D, st.P});
        }
    }
    ABS_CHECK(check_launch(ctx, "line-of-sight transform"));
    if (n_trip == 0) return ABS_OK;
    return launch_triple_sums(ctx, st, D, n_trip, d_uvw, sum, count, d_B);
}

}  // namespace absk
