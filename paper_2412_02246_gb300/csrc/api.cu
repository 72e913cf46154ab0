// C ABI of libabs: context, argument validation, host-side setup, and the
// orchestration of the stage kernels (grid.cu, fft.cu, counts.cu, triple.cu).
#include <algorithm>
#include <cmath>
#include <functional>
#include <map>
#include <cstdio>
#include <cstring>

#include "abs_internal.cuh"

namespace absk {

// ------------------------------------------------------------------ host arithmetic

// Q_m = ceil((l_m / (2 pi dU))^2): the smallest integer |g|^2 of ring m, whose
// cells satisfy l_m <= 2 pi |g| dU (Eq. iFT, l_g = 2 pi U_g).
int64_t ring_threshold(double ell, float du) {
    const double t = ell / (2.0 * M_PI * (double)du);
    return (int64_t)std::ceil(t * t);
}

static int64_t isqrt64(int64_t v) {
    if (v <= 0) return 0;
    int64_t r = (int64_t)std::sqrt((double)v);
    while (r * r > v) --r;
    while ((r + 1) * (r + 1) <= v) ++r;
    return r;
}

static int64_t ceil_sqrt64(int64_t v) {
    if (v <= 0) return 0;
    const int64_t r = isqrt64(v);
    return r * r == v ? r : r + 1;
}

// i <= j <= k that can close: sqrt(Q_k) <= sqrt(Q_{i+1}-1) + sqrt(Q_{j+1}-1).
void closing_triplets(const std::vector<int64_t> &q, std::vector<int32_t> &ijk) {
    const int nb = (int)q.size() - 1;
    ijk.clear();
    for (int i = 0; i < nb; ++i)
        for (int j = i; j < nb; ++j)
            for (int k = j; k < nb; ++k) {
                const int64_t a = q[i + 1] - 1, b = q[j + 1] - 1;
                const int64_t l = q[k] - a - b;
                const bool closes = a >= 0 && b >= 0 && (l <= 0 || l * l <= 4 * a * b);
                if (!closes) continue;
                ijk.push_back(i);
                ijk.push_back(j);
                ijk.push_back(k);
            }
}

static bool smooth235(int v) {
    if (v < 1) return false;
    for (int p : {2, 3, 5})
        while (v % p == 0) v /= p;
    return v == 1;
}

// Radices of the transform passes for a 2,3,5-smooth N: the fewest passes with
// radices from the in-register DFTs (2, 3, 4, 5 and their products up to 16),
// ties going to the plan whose smallest radix is largest (fewer idle threads
// in its widest pass).
static std::vector<int> radix_plan(int N) {
    static const int menu[] = {16, 15, 12, 10, 9, 8, 6, 5, 4, 3, 2};
    std::map<int, std::vector<int>> best;   // by remaining length
    std::function<const std::vector<int> &(int)> plan = [&](int n) -> const std::vector<int> & {
        auto it = best.find(n);
        if (it != best.end()) return it->second;
        std::vector<int> b;
        if (n > 1) {
            bool have = false;
            for (int r : menu) {
                if (n % r) continue;
                std::vector<int> c = plan(n / r);
                if (c.empty() && n / r != 1) continue;
                c.insert(c.begin(), r);
                const int cmin = *std::min_element(c.begin(), c.end());
                const int bmin = have ? *std::min_element(b.begin(), b.end()) : 0;
                if (!have || c.size() < b.size() || (c.size() == b.size() && cmin > bmin)) {
                    b = c;
                    have = true;
                }
            }
        }
        return best[n] = b;
    };
    return plan(N);
}

// Validates cfg and derives the ring thresholds q[0..nb], the largest |g_x| of
// a ring cell on the grid per ring (Rm[0..nb-1], -1 for an empty ring), their
// maximum R and the sky-grid side N, in caller-provided storage only (no heap
// or device allocation).  *err points at a static message on failure.
abs_status derive_grid(const abs_config *cfg, int64_t *q, int *Rm, int *R_out, int *N_out, const char **err) {
    if (!cfg) { *err = "cfg is NULL"; return ABS_ERR_INVALID_ARG; }
    if (cfg->n_grid < 8 || cfg->n_grid > 8192 || (cfg->n_grid & 1)) {
        *err = "n_grid must be even and in [8, 8192]";
        return ABS_ERR_INVALID_ARG;
    }
    const float du = (float)cfg->du;
    if (!(cfg->du > 0.0) || !std::isfinite(cfg->du) || !(du > 0.f) || !std::isfinite(du)) {
        *err = "du must be finite and > 0 in binary32";
        return ABS_ERR_INVALID_ARG;
    }
    if (cfg->kernel != ABS_KERNEL_GAUSS && cfg->kernel != ABS_KERNEL_NGP) {
        *err = "kernel must be ABS_KERNEL_GAUSS or ABS_KERNEL_NGP";
        return ABS_ERR_INVALID_ARG;
    }
    if (cfg->kernel == ABS_KERNEL_GAUSS) {
        if (!(cfg->sigma_cells > 0.25) || !std::isfinite(cfg->sigma_cells)) {
            *err = "sigma_cells must be finite and > 0.25";
            return ABS_ERR_INVALID_ARG;
        }
        if (cfg->radius_cells < 0 || cfg->radius_cells > ABS_MAX_RADIUS) {
            *err = "radius_cells must be in [0, 3]";
            return ABS_ERR_INVALID_ARG;
        }
        if (!(cfg->radius_cells + 0.5 < 9.0 * cfg->sigma_cells)) {
            *err = "sigma_cells must exceed (radius_cells + 0.5) / 9 (footprint weights stay normal FP32)";
            return ABS_ERR_INVALID_ARG;
        }
    }
    if (cfg->n_bins < 1 || cfg->n_bins > ABS_MAX_BINS) { *err = "n_bins must be in [1, 254]"; return ABS_ERR_INVALID_ARG; }
    if (!cfg->ell_edges) { *err = "ell_edges is NULL"; return ABS_ERR_INVALID_ARG; }
    for (int m = 0; m <= cfg->n_bins; ++m) {
        const double e = cfg->ell_edges[m];
        if (!std::isfinite(e) || !(e > 0.0) || (m > 0 && !(e > cfg->ell_edges[m - 1]))) {
            *err = "ell_edges must be finite, > 0 and strictly ascending";
            return ABS_ERR_INVALID_ARG;
        }
    }
    if (cfg->precision != ABS_FP32 && cfg->precision != ABS_SPLIT_BF16) {
        *err = "precision must be ABS_FP32 or ABS_SPLIT_BF16";
        return ABS_ERR_INVALID_ARG;
    }
    if (!(cfg->norm_A > 0.0) || !std::isfinite(cfg->norm_A)) { *err = "norm_A must be finite and > 0"; return ABS_ERR_INVALID_ARG; }
    if (cfg->weight_mode != ABS_W_MEAN_UNITMASK && cfg->weight_mode != ABS_W_PAPER_LITERAL &&
        cfg->weight_mode != ABS_W_NOISE) {
        *err = "weight_mode must be ABS_W_MEAN_UNITMASK, ABS_W_PAPER_LITERAL or ABS_W_NOISE";
        return ABS_ERR_INVALID_ARG;
    }
    const int nb = cfg->n_bins, half = cfg->n_grid / 2 - 1;
    for (int m = 0; m <= nb; ++m) q[m] = ring_threshold(cfg->ell_edges[m], du);
    if (q[nb] > (int64_t)1 << 40) { *err = "l range too large for the uv grid spacing"; return ABS_ERR_INVALID_ARG; }
    int R = 0;
    for (int m = 0; m < nb; ++m) {
        Rm[m] = -1;
        const int64_t lo = q[m], hi = q[m + 1] - 1;
        if (hi < lo) continue;
        for (int64_t x = std::min<int64_t>(half, isqrt64(hi)); x >= 0; --x) {
            const int64_t ylo = ceil_sqrt64(lo - x * x);
            const int64_t yhi = std::min<int64_t>(half, isqrt64(hi - x * x));
            if (hi - x * x >= 0 && ylo <= yhi) {
                Rm[m] = (int)x;
                break;
            }
        }
        R = std::max(R, Rm[m]);
    }
    const int Nmin = std::max(3 * R + 1, 8);
    int N = cfg->n_fft;
    if (N == 0) {
        N = Nmin;
        while (!smooth235(N)) ++N;
    } else if (!smooth235(N) || N < Nmin) {
        *err = "n_fft must be a 2^a 3^b 5^c value >= 3R+1 (R = largest |g_x| of a ring cell)";
        return ABS_ERR_INVALID_ARG;
    }
    if (N > ABS_MAX_FFT) { *err = "sky grid side N exceeds 4096 (reduce the l range or coarsen du)"; return ABS_ERR_UNSUPPORTED; }
    *R_out = R;
    *N_out = N;
    return ABS_OK;
}

abs_status make_setup(const abs_config *cfg, Setup &s, std::string &err) {
    const int nb = cfg && cfg->n_bins >= 1 && cfg->n_bins <= ABS_MAX_BINS ? cfg->n_bins : 1;
    s.q.assign(nb + 1, 0);
    s.Rm.assign(nb, -1);
    const char *msg = "";
    const abs_status st = derive_grid(cfg, s.q.data(), s.Rm.data(), &s.R, &s.N, &msg);
    if (st != ABS_OK) {
        err = msg;
        return st;
    }
    s.n = cfg->n_grid;
    s.half = s.n / 2 - 1;
    s.du = (float)cfg->du;
    s.kernel = cfg->kernel;
    s.r = cfg->kernel == ABS_KERNEL_NGP ? 0 : cfg->radius_cells;
    if (cfg->kernel == ABS_KERNEL_GAUSS) {
        const double sc = 1.0 / (2.0 * cfg->sigma_cells * cfg->sigma_cells);
        s.s_hi = (float)sc;
        s.s_lo = (float)(sc - (double)s.s_hi);
    }
    s.nb = cfg->n_bins;
    s.radices = radix_plan(s.N);
    s.P = (int64_t)s.N * s.N;
    // lattice cells per ring on the grid (capacity of the ring lists)
    s.lat.assign(s.nb, 0);
    for (int y = -s.R; y <= s.R; ++y)
        for (int x = -s.R; x <= s.R; ++x) {
            const int64_t r2 = (int64_t)x * x + (int64_t)y * y;
            if (r2 < s.q[0] || r2 >= s.q[s.nb]) continue;
            int m = 0;
            while (r2 >= s.q[m + 1]) ++m;
            s.lat[m]++;
        }
    s.lat_off.assign(s.nb + 1, 0);
    for (int m = 0; m < s.nb; ++m) s.lat_off[m + 1] = s.lat_off[m] + s.lat[m];
    // the lattice is closed under g -> -g and misses the origin: lat is even
    s.up_off.assign(s.nb + 1, 0);
    for (int m = 0; m < s.nb; ++m) s.up_off[m + 1] = s.up_off[m] + s.lat[m] / 2;
    closing_triplets(s.q, s.ijk);
    s.precision = cfg->precision;
    s.norm_A = cfg->norm_A;
    s.weight_mode = cfg->weight_mode;
    return ABS_OK;
}

// ------------------------------------------------------------------ context helpers

abs_status fail(abs_ctx *ctx, abs_status st, const std::string &msg) {
    if (ctx) ctx->last_error = msg;
    return st;
}

abs_status check_launch(abs_ctx *ctx, const char *what) {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ctx, ABS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return ABS_OK;
}

void drop_graphs(abs_ctx *ctx) {
    for (auto &kv : ctx->graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    ctx->graphs.clear();
    if (ctx->parent) drop_graphs(ctx->parent);   // the parent's graphs hold this lane's buffers
}

void *workspace(abs_ctx *ctx, const char *name, size_t bytes) {
    if (bytes == 0) bytes = 16;
    Workspace &w = ctx->ws[name];
    if (w.bytes >= bytes) return w.p;
    if (w.p) {
        cudaStreamSynchronize(ctx->stream);
        drop_graphs(ctx);   // they refer to the buffer freed here
        cudaFree(w.p);
        w.p = nullptr;
        w.bytes = 0;
    }
    const size_t want = bytes + bytes / 8;   // some headroom against regrowth
    if (ctx->fail_allocs > 0) {              // injected failure (abs_inject_alloc_failures)
        --ctx->fail_allocs;
        return nullptr;
    }
    if (cudaMalloc(&w.p, want) != cudaSuccess) {
        cudaGetLastError();
        w.p = nullptr;
        return nullptr;
    }
    w.bytes = want;
    return w.p;
}

void *workspace_zeroed(abs_ctx *ctx, const char *name, size_t bytes) {
    Workspace &w = ctx->ws[name];
    const bool fresh = w.bytes < (bytes == 0 ? 16 : bytes);
    void *p = workspace(ctx, name, bytes);
    if (p && fresh) cudaMemsetAsync(p, 0, ctx->ws[name].bytes, ctx->stream);
    return p;
}

static std::string setup_key(const abs_config *c) {
    std::string k;
    auto put = [&k](const void *p, size_t n) { k.append((const char *)p, n); };
    put(&c->n_grid, sizeof c->n_grid);
    put(&c->du, sizeof c->du);
    put(&c->kernel, sizeof c->kernel);
    put(&c->sigma_cells, sizeof c->sigma_cells);
    put(&c->radius_cells, sizeof c->radius_cells);
    put(&c->n_bins, sizeof c->n_bins);
    put(c->ell_edges, sizeof(double) * (c->n_bins + 1));
    put(&c->n_fft, sizeof c->n_fft);
    put(&c->precision, sizeof c->precision);
    put(&c->norm_A, sizeof c->norm_A);
    put(&c->weight_mode, sizeof c->weight_mode);
    return k;
}

template <class T>
static T *upload(const std::vector<T> &v) {
    T *d = nullptr;
    const size_t bytes = sizeof(T) * std::max<size_t>(v.size(), 1);
    if (cudaMalloc(&d, bytes) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    if (!v.empty() && cudaMemcpy(d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(d);
        return nullptr;
    }
    return d;
}

static void free_setup(Setup &s) {
    cudaFree(s.d_q);
    cudaFree(s.d_lat_off);
    cudaFree(s.d_ring_off);
    s.d_ring_off = nullptr;
    cudaFree(s.d_ijk);
    cudaFree(s.d_tw);
    cudaFree(s.d_Rm);
    cudaFree(s.d_full_counts);
    s.d_full_counts = nullptr;
    s.tc_plan.reset();
    s.full_counts_ready = false;
    s.d_q = nullptr;
    s.d_lat_off = nullptr;
    s.d_ijk = nullptr;
    s.d_tw = nullptr;
    s.d_Rm = nullptr;
}

const Setup *get_setup(abs_ctx *ctx, const abs_config *cfg, abs_status &st) {
    std::string err;
    if (!cfg || !cfg->ell_edges || cfg->n_bins < 1 || cfg->n_bins > ABS_MAX_BINS) {
        st = fail(ctx, ABS_ERR_INVALID_ARG, "invalid config (ell_edges / n_bins)");
        return nullptr;
    }
    const std::string key = setup_key(cfg);
    auto it = ctx->setups.find(key);
    if (it != ctx->setups.end()) {
        st = ABS_OK;
        return it->second.get();
    }
    std::unique_ptr<Setup> s(new Setup);
    st = make_setup(cfg, *s, err);
    s->key = key;
    if (st != ABS_OK) {
        fail(ctx, st, err);
        return nullptr;
    }
    // twiddles laid out for the packed (re, im) complex multiply of the transforms:
    // double-float pairs [2t], [2t + 1], then the FP32 ones [2N + t]
    std::vector<float4> tw(3 * (size_t)s->N);
    for (int t = 0; t < s->N; ++t) {
        const double a = 2.0 * M_PI * (double)t / (double)s->N;
        const double c = std::cos(a), sn = -std::sin(a);
        const float ch = (float)c, sh = (float)sn;
        const float cl = (float)(c - (double)ch), sl = (float)(sn - (double)sh);
        tw[2 * t] = make_float4(ch, ch, cl, cl);
        tw[2 * t + 1] = make_float4(-sh, sh, -sl, sl);
        tw[2 * (size_t)s->N + t] = make_float4(ch, ch, -sh, sh);
    }
    s->d_q = upload(s->q);
    s->d_lat_off = upload(s->lat_off);
    {
        std::vector<int64_t> ro(3 * (size_t)(s->nb + 1));
        for (int f = 0; f < 3; ++f)
            for (int m = 0; m <= s->nb; ++m) ro[(size_t)f * (s->nb + 1) + m] = f * s->up_off[s->nb] + s->up_off[m];
        s->d_ring_off = upload(ro);
    }
    s->d_ijk = upload(s->ijk);
    s->d_tw = upload(tw);
    s->d_Rm = upload(std::vector<int32_t>(s->Rm.begin(), s->Rm.end()));
    if (!s->d_q || !s->d_lat_off || !s->d_ring_off || !s->d_ijk || !s->d_tw || !s->d_Rm) {
        free_setup(*s);
        st = fail(ctx, ABS_ERR_OOM, "setup tables");
        return nullptr;
    }
    Setup *raw = s.get();
    ctx->setups[key] = std::move(s);
    st = ABS_OK;
    return raw;
}

static cudaEvent_t pool_get(abs_ctx *ctx) {
    if (!ctx->event_pool.empty()) {
        cudaEvent_t e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

StageTimer::StageTimer(abs_ctx *c, const char *n) : ctx(c), name(n) {
    if (!ctx->profiling || !n) return;
    a = pool_get(ctx);
    b = pool_get(ctx);
    if (a) cudaEventRecord(a, ctx->stream);
}

StageTimer::~StageTimer() {
    if (!a || !b) return;
    cudaEventRecord(b, ctx->stream);
    ctx->pending.push_back({name, a, b});
}

static void profile_drain(abs_ctx *ctx) {
    for (auto &p : ctx->pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            auto &t = ctx->stage_totals[p.name];
            t.first += ms;
            t.second += 1;
        }
        cudaGetLastError();
        ctx->event_pool.push_back(p.a);
        ctx->event_pool.push_back(p.b);
    }
    ctx->pending.clear();
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace absk

using namespace absk;



extern "C" {

abs_status abs_create(abs_ctx **out, int32_t device, void *cuda_stream) {
    if (!out) return ABS_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return ABS_ERR_INVALID_ARG;
    }
    DeviceGuard g(device);
    abs_ctx *ctx = new abs_ctx;
    ctx->device = device;
    ctx->stream = (cudaStream_t)cuda_stream;
    cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (cudaMalloc(&ctx->d_err, sizeof(int32_t)) != cudaSuccess ||
        cudaMemset(ctx->d_err, 0, sizeof(int32_t)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return ABS_ERR_OOM;
    }
    *out = ctx;
    return ABS_OK;
}

// Everything a context (or a lane) owns; the device error word only when it is not a lane.
static void release_ctx(abs_ctx *ctx) {
    for (abs_ctx *l : ctx->lanes) release_ctx(l);
    ctx->lanes.clear();
    cudaStreamSynchronize(ctx->stream);
    if (ctx->side) cudaStreamSynchronize(ctx->side);
    drop_graphs(ctx);
    for (auto &kv : ctx->ws) cudaFree(kv.second.p);
    ctx->cubes.clear();
    for (auto &kv : ctx->setups) free_setup(*kv.second);
    if (!ctx->parent) cudaFree(ctx->d_err);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    if (ctx->owns_stream) cudaStreamDestroy(ctx->stream);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->ev_lane) cudaEventDestroy(ctx->ev_lane);
    for (auto &p : ctx->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : ctx->event_pool) cudaEventDestroy(e);
    delete ctx;
}

abs_status abs_destroy(abs_ctx *ctx) {
    if (!ctx || ctx->parent) return ABS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    release_ctx(ctx);
    return ABS_OK;
}

const char *abs_last_error(const abs_ctx *ctx) { return ctx ? ctx->last_error.c_str() : "no context"; }

abs_status abs_sync(abs_ctx *ctx) {
    if (!ctx) return ABS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess)
        return fail(ctx, ABS_ERR_CUDA, std::string("stream: ") + cudaGetErrorString(cudaGetLastError()));
    int32_t e = 0;
    if (cudaMemcpy(&e, ctx->d_err, sizeof e, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(ctx, ABS_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
    if (e == DERR_NONE) return ABS_OK;
    cudaMemset(ctx->d_err, 0, sizeof(int32_t));
    if (e == DERR_TIMEOUT) return fail(ctx, ABS_ERR_TIMEOUT, "a bounded device wait gave up");
    if (e == DERR_TRIPLET_ORDER) return fail(ctx, ABS_ERR_DEVICE, "triplet list is not in canonical order");
    if (e == DERR_CAPACITY) return fail(ctx, ABS_ERR_UNSUPPORTED, "problem too large for an internal work list");
    return fail(ctx, ABS_ERR_DEVICE, "triplet list holds a bin outside 0 <= i <= j <= k < n_bins");
}

abs_status abs_profile(abs_ctx *ctx, int32_t on) {
    if (!ctx) return ABS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    profile_drain(ctx);
    ctx->stage_totals.clear();
    ctx->profiling = on != 0;
    return ABS_OK;
}

abs_status abs_rebin(abs_ctx *ctx, const abs_config *cfg, int32_t n_real, int32_t n_trip, const double *d_B,
                     const int64_t *d_count, const double *d_ellbar, const int32_t *d_ijk, int32_t n_mu,
                     int32_t n_t, double *d_mean, double *d_sigma, double *d_weight) {
    if (!ctx) return ABS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    abs_status st;
    const Setup *s = get_setup(ctx, cfg, st);
    if (!s) return st;
    if (n_real < 1 || n_trip < 0) return fail(ctx, ABS_ERR_INVALID_ARG, "n_real must be >= 1 and n_trip >= 0");
    if (n_mu < 1 || n_mu > 64 || n_t < 1 || n_t > 64) return fail(ctx, ABS_ERR_INVALID_ARG, "n_mu, n_t must be in [1, 64]");
    if (n_trip > 0 && (!d_B || !d_count || !d_ellbar))
        return fail(ctx, ABS_ERR_INVALID_ARG, "d_B, d_count and d_ellbar are required");
    if (!d_ijk) {
        if (n_trip != (int32_t)(s->ijk.size() / 3))
            return fail(ctx, ABS_ERR_INVALID_ARG, "n_trip must equal the canonical triplet count when d_ijk is NULL");
        d_ijk = s->d_ijk;
    }
    return launch_rebin(ctx, *s, n_real, n_trip, d_B, d_count, d_ellbar, d_ijk, n_mu, n_t, d_mean, d_sigma,
                        d_weight);
}

abs_status abs_bana_d(abs_ctx *ctx, const abs_config *cfg, const double *d_C, const uint8_t *d_mask,
                      int32_t n_trip, const int32_t *d_ijk, const int64_t *d_count, double f_over_sigma,
                      double *d_out) {
    if (!ctx) return ABS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    abs_status st;
    const Setup *s = get_setup(ctx, cfg, st);
    if (!s) return st;
    if (n_trip < 0) return fail(ctx, ABS_ERR_INVALID_ARG, "n_trip < 0");
    if (!d_C || !d_mask || (n_trip > 0 && (!d_count || !d_out)))
        return fail(ctx, ABS_ERR_INVALID_ARG, "d_C, d_mask, d_count and d_out are required");
    if (!std::isfinite(f_over_sigma)) return fail(ctx, ABS_ERR_INVALID_ARG, "f_over_sigma must be finite");
    if (!d_ijk) {
        if (n_trip != (int32_t)(s->ijk.size() / 3))
            return fail(ctx, ABS_ERR_INVALID_ARG, "n_trip must equal the canonical triplet count when d_ijk is NULL");
        d_ijk = s->d_ijk;
    } else {
        ABS_CHECK(launch_check_triplets(ctx, *s, n_trip, d_ijk));
    }
    const size_t fb = sizeof(float) * (size_t)s->nb * s->N * s->N;
    float *P = (float *)workspace(ctx, "bana.P", fb);
    float *I = (float *)workspace(ctx, "bana.I", fb);
    if (!P || !I) return fail(ctx, ABS_ERR_OOM, "prediction fields");
    ABS_CHECK(launch_filter_fft_real(ctx, *s, d_C, d_mask, P));
    ABS_CHECK(launch_filter_fft_real(ctx, *s, nullptr, d_mask, I));
    return launch_bana_sums(ctx, *s, P, I, n_trip, d_ijk, d_count, f_over_sigma, d_out);
}

abs_status abs_simulate_vis(abs_ctx *ctx, int32_t m, double dtheta, const float *d_sky, int32_t beam,
                            double beam_param, int64_t n_vis, const float *d_uv, float *d_vis) {
    if (!ctx) return ABS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (m < 1 || m > 8192) return fail(ctx, ABS_ERR_INVALID_ARG, "m must be in [1, 8192]");
    if (!(dtheta > 0.0) || !std::isfinite(dtheta)) return fail(ctx, ABS_ERR_INVALID_ARG, "dtheta must be finite and > 0");
    if (beam != ABS_BEAM_NONE && beam != ABS_BEAM_MWA_TILE && beam != ABS_BEAM_GAUSS)
        return fail(ctx, ABS_ERR_INVALID_ARG, "unknown beam");
    if (beam != ABS_BEAM_NONE && (!(beam_param > 0.0) || !std::isfinite(beam_param)))
        return fail(ctx, ABS_ERR_INVALID_ARG, "beam_param must be finite and > 0");
    if (n_vis < 0) return fail(ctx, ABS_ERR_INVALID_ARG, "n_vis < 0");
    if (!d_sky || (n_vis > 0 && (!d_uv || !d_vis))) return fail(ctx, ABS_ERR_INVALID_ARG, "NULL buffer");
    return launch_simulate_vis(ctx, m, dtheta, d_sky, beam, beam_param, n_vis, d_uv, d_vis);
}

namespace absk {
// A bounded wait on a flag nothing sets: gives up after max_polls and latches a timeout.
__global__ void k_wait_probe(const volatile int *flag, int max_polls, int32_t *err) {
    if (threadIdx.x != 0) return;
    for (int i = 0; i < max_polls; ++i) {
        if (*flag) return;
        __nanosleep(1000);
    }
    atomicCAS(err, 0, DERR_TIMEOUT);
}
}  // namespace absk

abs_status abs_inject_alloc_failures(abs_ctx *ctx, int32_t count) {
    if (!ctx || count < 0) return ABS_ERR_INVALID_ARG;
    ctx->fail_allocs = count;
    return ABS_OK;
}

abs_status abs_probe_timeout(abs_ctx *ctx, int32_t max_polls) {
    if (!ctx) return ABS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (max_polls < 1 || max_polls > (1 << 20)) return fail(ctx, ABS_ERR_INVALID_ARG, "max_polls must be in [1, 2^20]");
    int *flag = (int *)workspace_zeroed(ctx, "probe.flag", sizeof(int));
    if (!flag) return fail(ctx, ABS_ERR_OOM, "probe flag");
    k_wait_probe<<<1, 32, 0, ctx->stream>>>(flag, max_polls, ctx->d_err);
    return check_launch(ctx, "timeout probe");
}

abs_status abs_autotune(abs_ctx *ctx, int32_t enable) {
    if (!ctx) return ABS_ERR_INVALID_ARG;
    ctx->autotune = enable != 0;
    return ABS_OK;
}

abs_status abs_tuned_shape(abs_ctx *ctx, const abs_config *cfg, int32_t *set_cols, int32_t *waves,
                           int32_t *measured) {
    if (!ctx || !cfg || !cfg->ell_edges || cfg->n_bins < 1 || cfg->n_bins > ABS_MAX_BINS)
        return ABS_ERR_INVALID_ARG;
    auto it = ctx->tc_shapes.find(setup_key(cfg));
    const bool have = it != ctx->tc_shapes.end();
    if (set_cols) *set_cols = have ? it->second.budget : 0;
    if (waves) *waves = have ? it->second.waves : 0;
    if (measured) *measured = have && it->second.measured ? 1 : 0;
    return ABS_OK;
}

abs_status abs_profile_read(abs_ctx *ctx, int32_t cap, int32_t *n, abs_stage_time *out) {
    if (!ctx || !n || cap < 0) return ABS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    profile_drain(ctx);
    int32_t k = 0;
    for (auto &kv : ctx->stage_totals) {
        if (out && k < cap) {
            std::memset(out[k].name, 0, sizeof out[k].name);
            std::strncpy(out[k].name, kv.first.c_str(), sizeof out[k].name - 1);
            out[k].ms = kv.second.first;
            out[k].launches = kv.second.second;
        }
        ++k;
    }
    *n = k;
    return ABS_OK;
}

abs_status abs_ring_q(const abs_config *cfg, int64_t *q) {
    if (!q) return ABS_ERR_INVALID_ARG;
    Setup s;
    std::string err;
    ABS_CHECK(make_setup(cfg, s, err));
    for (int m = 0; m <= s.nb; ++m) q[m] = s.q[m];
    return ABS_OK;
}

abs_status abs_fft_size(const abs_config *cfg, int32_t *n_fft) {
    if (!n_fft) return ABS_ERR_INVALID_ARG;
    Setup s;
    std::string err;
    ABS_CHECK(make_setup(cfg, s, err));
    *n_fft = s.N;
    return ABS_OK;
}

abs_status abs_triplets(const abs_config *cfg, int32_t cap, int32_t *n_trip, int32_t *ijk) {
    if (!n_trip || cap < 0) return ABS_ERR_INVALID_ARG;
    Setup s;
    std::string err;
    ABS_CHECK(make_setup(cfg, s, err));
    const int32_t n = (int32_t)(s.ijk.size() / 3);
    *n_trip = n;
    if (ijk) std::memcpy(ijk, s.ijk.data(), sizeof(int32_t) * 3 * std::min(n, cap));
    return ABS_OK;
}

abs_status abs_triplets_3d(const abs_config3d *cfg, int32_t cap, int32_t *n_trip, int32_t *uvw) {
    if (!cfg || !n_trip || cap < 0) return ABS_ERR_INVALID_ARG;
    if (cfg->n_dbins < 1 || !cfg->delay_edges) return ABS_ERR_INVALID_ARG;
    Setup s;
    std::string err;
    ABS_CHECK(make_setup(&cfg->base, s, err));
    int t_max = 0, Nz = 0;
    std::vector<int64_t> T1;
    std::vector<int32_t> list;
    const char *msg = "";
    ABS_CHECK(derive_cube(cfg, s, t_max, Nz, T1, list, &msg));
    const int32_t n = (int32_t)(list.size() / 3);
    *n_trip = n;
    if (uvw) std::memcpy(uvw, list.data(), sizeof(int32_t) * 3 * std::min(n, cap));
    return ABS_OK;
}

abs_status abs_grid(abs_ctx *ctx, const abs_config *cfg, int64_t n_vis, const float *d_uv,
                    const float *d_vis, float *d_grid, float *d_wsum, uint8_t *d_mask) {
    if (!ctx) return ABS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    abs_status st;
    const Setup *s = get_setup(ctx, cfg, st);
    if (!s) return st;
    if (n_vis < 0 || n_vis > 0x7fffffffLL) return fail(ctx, ABS_ERR_INVALID_ARG, "n_vis must be in [0, 2^31)");
    if ((n_vis > 0 && (!d_uv || !d_vis)) || !d_grid || !d_wsum || !d_mask)
        return fail(ctx, ABS_ERR_INVALID_ARG, "NULL buffer");
    ABS_CHECK(launch_grid_plan(ctx, *s, n_vis, d_uv));
    return launch_grid_accumulate(ctx, *s, n_vis, d_vis, d_grid, d_wsum, d_mask);
}

abs_status abs_filter_fft(abs_ctx *ctx, const abs_config *cfg, const float *d_grid, const float *d_wsum,
                          const uint8_t *d_mask, float *d_fields) {
    if (!ctx) return ABS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    abs_status st;
    const Setup *s = get_setup(ctx, cfg, st);
    if (!s) return st;
    if (!d_grid || !d_wsum || !d_mask || !d_fields) return fail(ctx, ABS_ERR_INVALID_ARG, "NULL buffer");
    return launch_filter_fft(ctx, *s, d_grid, d_wsum, d_mask, d_fields);
}

abs_status abs_triple(abs_ctx *ctx, const abs_config *cfg, const float *d_fields, const uint8_t *d_mask,
                      int32_t n_trip, const int32_t *d_ijk, double *d_sum, int64_t *d_count) {
    if (!ctx) return ABS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    abs_status st;
    const Setup *s = get_setup(ctx, cfg, st);
    if (!s) return st;
    if (n_trip < 0) return fail(ctx, ABS_ERR_INVALID_ARG, "n_trip < 0");
    if (n_trip > 0 && !d_ijk) return fail(ctx, ABS_ERR_INVALID_ARG, "d_ijk is NULL");
    if (d_sum && !d_fields) return fail(ctx, ABS_ERR_INVALID_ARG, "d_fields is NULL");
    if (d_count && !d_mask) return fail(ctx, ABS_ERR_INVALID_ARG, "d_mask is NULL");
    ABS_CHECK(launch_check_triplets(ctx, *s, n_trip, d_ijk));
    if (d_sum) ABS_CHECK(launch_triple_sums(ctx, *s, d_fields, n_trip, d_ijk, d_sum));
    if (d_count) ABS_CHECK(launch_counts(ctx, *s, d_mask, n_trip, d_ijk, d_count, nullptr));
    return ABS_OK;
}

abs_status abs_normalise(abs_ctx *ctx, const abs_config *cfg, int32_t n_trip, const double *d_sum,
                         const int64_t *d_count, double *d_B, const uint8_t *d_mask, double *d_ellbar) {
    if (!ctx) return ABS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    abs_status st;
    const Setup *s = get_setup(ctx, cfg, st);
    if (!s) return st;
    if (n_trip < 0 || (n_trip > 0 && (!d_sum || !d_count || !d_B)))
        return fail(ctx, ABS_ERR_INVALID_ARG, "NULL buffer or n_trip < 0");
    if (d_ellbar && !d_mask) return fail(ctx, ABS_ERR_INVALID_ARG, "d_mask is NULL");
    ABS_CHECK(launch_normalise(ctx, *s, n_trip, d_sum, d_count, d_B));
    if (d_ellbar) ABS_CHECK(launch_ellbar(ctx, *s, d_mask, d_ellbar));
    return ABS_OK;
}

// With h_uv / h_vis (page-locked host buffers) the inputs are first copied into
// d_uv / d_vis: the positions on the main stream ahead of the gridding plan, the
// visibilities on the side stream beside it (the plan needs only the positions).
// (The plan's first kernel reading the positions from the host buffer through
// its device-mapped address was slower than the copy engine.)
static abs_status estimate_many(abs_ctx *ctx, const Setup &s, int64_t n_vis, const float *d_uv,
                                int32_t n_real, const float *d_vis, int32_t n_trip,
                                const int32_t *d_ijk, double *d_B, int64_t *d_count, double *d_ellbar,
                                const float *h_uv = nullptr, const float *h_vis = nullptr) {
    const int64_t cells = (int64_t)s.n * s.n;
    const int64_t P = (int64_t)s.N * s.N;
    // the weighted forms (literal, noise) divide by the sums S_W of their I fields
    const bool literal = s.weight_mode != ABS_W_MEAN_UNITMASK;
    // split-BF16 sums over the canonical list: the transform writes the kernel's split
    // planes directly, and no FP32 fields are kept
    const bool to_planes = s.precision == ABS_SPLIT_BF16 && d_ijk == s.d_ijk && !literal && n_trip > 0;
    SplitOut planes{};
    if (to_planes) ABS_CHECK(tc_split_target(ctx, s, planes));
    float *fields = to_planes ? nullptr : (float *)workspace(ctx, "est.fields", sizeof(float) * (size_t)s.nb * P);
    double *sum = (double *)workspace(ctx, "est.sum", sizeof(double) * std::max(n_trip, 1));
    float *ifields = literal ? (float *)workspace(ctx, "est.ifields", sizeof(float) * (size_t)s.nb * P) : nullptr;
    double *sumw = literal ? (double *)workspace(ctx, "est.sumw", sizeof(double) * std::max(n_trip, 1)) : nullptr;
    if (literal && (!ifields || !sumw)) return fail(ctx, ABS_ERR_OOM, "estimate workspace");
    int64_t *count = d_count ? d_count : (int64_t *)workspace(ctx, "est.count", sizeof(int64_t) * std::max(n_trip, 1));
    if ((!fields && !to_planes) || !sum || !count) return fail(ctx, ABS_ERR_OOM, "estimate workspace");
    // the canonical list (d_ijk == NULL at the ABI) was built and checked with the setup
    if (d_ijk != s.d_ijk) ABS_CHECK(launch_check_triplets(ctx, s, n_trip, d_ijk));
    // the first realisation's accumulators are cleared on the side stream while
    // the plan runs (not while profiling stages)
    double *acc0 = nullptr;
    grid_acc_buffers(ctx, s, &acc0);
    if (!acc0) return fail(ctx, ABS_ERR_OOM, "grid accumulation workspace");
    const bool pre_zero = !ctx->profiling && ctx->side;
    const size_t uvb = sizeof(float) * 2 * (size_t)n_vis;
    const bool copy_in = h_uv && h_vis && n_vis > 0;
    if (pre_zero) {
        cudaEventRecord(ctx->ev_fork, ctx->stream);
        cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0);
        cudaMemsetAsync(acc0, 0, sizeof(double) * grid_acc_planes(s) * (size_t)cells, ctx->side);
        if (copy_in)
            cudaMemcpyAsync((void *)d_vis, h_vis, uvb * (size_t)n_real, cudaMemcpyHostToDevice, ctx->side);
        cudaEventRecord(ctx->ev_join, ctx->side);
    } else if (copy_in) {
        cudaMemcpyAsync((void *)d_vis, h_vis, uvb * (size_t)n_real, cudaMemcpyHostToDevice, ctx->stream);
    }
    if (copy_in) cudaMemcpyAsync((void *)d_uv, h_uv, uvb, cudaMemcpyHostToDevice, ctx->stream);
    const abs_status sp = launch_grid_plan(ctx, s, n_vis, d_uv, true);
    if (pre_zero) cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0);
    if (sp != ABS_OK) return sp;
    for (int32_t r = 0; r < n_real; ++r) {
        // the transform and the counts read the FP64 accumulators directly
        ABS_CHECK(launch_grid_accumulate(ctx, s, n_vis, d_vis + (size_t)r * 2 * n_vis, nullptr, nullptr, nullptr,
                                         r == 0 && pre_zero));
        cudaEvent_t join = nullptr;
        if (r == 0) {
            // the filled mask depends on the baselines only: counts and mean l once,
            // on the side stream beside the transforms (not while profiling stages)
            if (!ctx->profiling && ctx->side) {
                cudaEventRecord(ctx->ev_fork, ctx->stream);
                cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0);
                cudaStream_t main = ctx->stream;
                ctx->stream = ctx->side;
                const abs_status st = launch_counts(ctx, s, nullptr, n_trip, d_ijk, count, d_ellbar,
                                                    acc0 + 2 * cells);
                cudaEventRecord(ctx->ev_join, ctx->side);
                ctx->stream = main;
                join = ctx->ev_join;
                if (st != ABS_OK) {
                    cudaStreamWaitEvent(ctx->stream, join, 0);
                    return st;
                }
            } else {
                ABS_CHECK(launch_counts(ctx, s, nullptr, n_trip, d_ijk, count, d_ellbar, acc0 + 2 * cells));
            }
        }
        double *acc;
        grid_acc_buffers(ctx, s, &acc);
        const abs_status sf = launch_filter_fft_acc(ctx, s, acc, fields, to_planes ? &planes : nullptr);
        if (sf != ABS_OK) {
            if (join) cudaStreamWaitEvent(ctx->stream, join, 0);
            return sf;
        }
        if (!literal) {
            ABS_CHECK(launch_triple_sums(ctx, s, fields, n_trip, d_ijk, sum, count,
                                         d_B ? d_B + (size_t)r * n_trip : nullptr, join));
            continue;
        }
        // the weighted forms: S, then (once: the weights are the baselines') the sums
        // S_W of the I fields (W_g = 1 / N_g, or N_eff), then B = Re S / (A S_W)
        abs_status sl = launch_triple_sums(ctx, s, fields, n_trip, d_ijk, sum);
        if (sl == ABS_OK && r == 0) sl = launch_filter_fft_w(ctx, s, acc, ifields);
        if (sl == ABS_OK && r == 0) sl = launch_triple_sums(ctx, s, ifields, n_trip, d_ijk, sumw);
        if (join) cudaStreamWaitEvent(ctx->stream, join, 0);   // the counts are done before the call ends
        if (sl != ABS_OK) return sl;
        ABS_CHECK(launch_normalise_w(ctx, s, n_trip, sum, sumw, d_B ? d_B + (size_t)r * n_trip : nullptr));
    }
    return ABS_OK;
}

// estimate_many through the context's graph cache (see abs_ctx::graphs).  Not
// used while the stage profiler runs or on the legacy default stream.
// Runs `eager` through the context's graph cache (see abs_ctx::graphs) under
// `key`: eagerly the first time, captured and launched the second, replayed
// after that.  Not used while the stage profiler runs or on the legacy
// default stream.  The cache entry is looked up again after every eager run,
// since a workspace regrowth inside it drops the whole cache.
extern "C++" {
template <class F>
static abs_status graphed(abs_ctx *ctx, const std::string &key, const F &eager) {
    if (ctx->profiling || ctx->stream == nullptr) return eager();
    {
        abs_ctx::Graph &g = ctx->graphs[key];
        if (g.exec) {
            if (cudaGraphLaunch(g.exec, ctx->stream) == cudaSuccess) return ABS_OK;
            cudaGetLastError();
            cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
            g.failed = true;
            return eager();
        }
        if (g.failed || g.seen++ == 0) return eager();
    }
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        ctx->graphs[key].failed = true;
        return eager();
    }
    const abs_status st = eager();
    const cudaError_t ce = cudaStreamEndCapture(ctx->stream, &graph);
    cudaGraphExec_t exec = nullptr;
    if (st != ABS_OK || ce != cudaSuccess || !graph || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
        // nothing captured ran: run it eagerly (and never capture this key again)
        cudaGetLastError();
        if (graph) cudaGraphDestroy(graph);
        ctx->graphs[key].failed = true;
        ctx->last_error.clear();
        return eager();
    }
    cudaGraphDestroy(graph);
    abs_ctx::Graph &g = ctx->graphs[key];
    g.exec = exec;
    if (cudaGraphLaunch(g.exec, ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
        g.failed = true;
        return eager();
    }
    return ABS_OK;
}
}  // extern "C++"

static abs_status estimate_graphed(abs_ctx *ctx, const Setup &s, int64_t n_vis, const float *d_uv,
                                   int32_t n_real, const float *d_vis, int32_t n_trip, const int32_t *d_ijk,
                                   double *d_B, int64_t *d_count, double *d_ellbar,
                                   const float *h_uv = nullptr, const float *h_vis = nullptr) {
    char key[320];
    snprintf(key, sizeof key, "%p|%p|%lld|%p|%d|%p|%d|%p|%p|%p|%p|%p|%p", (const void *)&s,
             (const void *)ctx->stream, (long long)n_vis, (const void *)d_uv, n_real, (const void *)d_vis, n_trip,
             (const void *)d_ijk, (void *)d_B, (void *)d_count, (void *)d_ellbar, (const void *)h_uv,
             (const void *)h_vis);
    return graphed(ctx, key, [&]() {
        return estimate_many(ctx, s, n_vis, d_uv, n_real, d_vis, n_trip, d_ijk, d_B, d_count, d_ellbar, h_uv,
                             h_vis);
    });
}

// Page-locked (pinned or registered) host memory: its copies can be captured into a graph.
static bool page_locked(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

static abs_status estimate_args(abs_ctx *ctx, const Setup &s, int64_t n_vis, const void *uv,
                                int32_t n_real, const void *vis, int32_t n_trip, const int32_t *&ijk) {
    if (n_vis < 0 || n_vis > 0x7fffffffLL) return fail(ctx, ABS_ERR_INVALID_ARG, "n_vis must be in [0, 2^31)");
    if (n_real < 1) return fail(ctx, ABS_ERR_INVALID_ARG, "n_real must be >= 1");
    if (n_vis > 0 && (!uv || !vis)) return fail(ctx, ABS_ERR_INVALID_ARG, "NULL visibility buffer");
    if (n_trip < 0) return fail(ctx, ABS_ERR_INVALID_ARG, "n_trip < 0");
    if (!ijk) {
        if (n_trip != (int32_t)(s.ijk.size() / 3))
            return fail(ctx, ABS_ERR_INVALID_ARG, "n_trip must equal the canonical triplet count when d_ijk is NULL");
        ijk = s.d_ijk;
    }
    return ABS_OK;
}

abs_status abs_estimate_many(abs_ctx *ctx, const abs_config *cfg, int64_t n_vis, const float *d_uv,
                             int32_t n_real, const float *d_vis, int32_t n_trip, const int32_t *d_ijk,
                             double *d_B, int64_t *d_count, double *d_ellbar) {
    if (!ctx) return ABS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    abs_status st;
    const Setup *s = get_setup(ctx, cfg, st);
    if (!s) return st;
    ABS_CHECK(estimate_args(ctx, *s, n_vis, d_uv, n_real, d_vis, n_trip, d_ijk));
    return estimate_graphed(ctx, *s, n_vis, d_uv, n_real, d_vis, n_trip, d_ijk, d_B, d_count, d_ellbar);
}

abs_status abs_estimate(abs_ctx *ctx, const abs_config *cfg, int64_t n_vis, const float *d_uv,
                        const float *d_vis, int32_t n_trip, const int32_t *d_ijk, double *d_B,
                        int64_t *d_count, double *d_ellbar) {
    return abs_estimate_many(ctx, cfg, n_vis, d_uv, 1, d_vis, n_trip, d_ijk, d_B, d_count, d_ellbar);
}

abs_status abs_estimate_3d(abs_ctx *ctx, const abs_config3d *cfg, int64_t n_vis, const float *d_uv,
                           const float *d_vis, int32_t n_trip, const int32_t *d_uvw, double *d_B,
                           int64_t *d_count, double *d_ellbar) {
    if (!ctx) return ABS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    abs_status st;
    const CubeSetup *c = get_cube_setup(ctx, cfg, st);
    if (!c) return st;
    if (n_vis < 0 || n_vis > 0x7fffffffLL) return fail(ctx, ABS_ERR_INVALID_ARG, "n_vis must be in [0, 2^31)");
    if (n_vis > 0 && (!d_uv || !d_vis)) return fail(ctx, ABS_ERR_INVALID_ARG, "NULL visibility buffer");
    if (n_trip < 0) return fail(ctx, ABS_ERR_INVALID_ARG, "n_trip < 0");
    if (!d_uvw) {
        if (n_trip != (int32_t)(c->st.ijk.size() / 3))
            return fail(ctx, ABS_ERR_INVALID_ARG, "n_trip must equal the canonical triplet count when d_uvw is NULL");
        d_uvw = c->st.d_ijk;
    }
    char key[320];
    snprintf(key, sizeof key, "cube|%p|%p|%lld|%p|%p|%d|%p|%p|%p|%p", (const void *)c, (const void *)ctx->stream,
             (long long)n_vis, (const void *)d_uv, (const void *)d_vis, n_trip, (const void *)d_uvw, (void *)d_B,
             (void *)d_count, (void *)d_ellbar);
    return graphed(ctx, key, [&]() {
        return launch_cube_estimate(ctx, *c, n_vis, d_uv, d_vis, n_trip, d_uvw, d_B, d_count, d_ellbar);
    });
}

// A lane of ctx: its own non-blocking streams and events, the parent's device error word.
static abs_ctx *make_lane(abs_ctx *ctx) {
    abs_ctx *l = new abs_ctx;
    l->device = ctx->device;
    l->sm_count = ctx->sm_count;
    l->parent = ctx;
    l->d_err = ctx->d_err;
    l->owns_stream = true;
    if (cudaStreamCreateWithFlags(&l->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&l->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&l->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&l->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&l->ev_lane, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        release_ctx(l);
        return nullptr;
    }
    return l;
}

extern "C++" {
namespace absk {
abs_status ensure_lanes(abs_ctx *ctx, int K) {
    while ((int)ctx->lanes.size() < K) {
        abs_ctx *l = make_lane(ctx);
        if (!l) return fail(ctx, ABS_ERR_OOM, "lanes");
        ctx->lanes.push_back(l);
    }
    return ABS_OK;
}
}  // namespace absk
}  // extern "C++"

// The batch driver of abs_estimate_batched and abs_estimate_batched_host.  With
// host = true the items' uv / vis are host inputs and B / count / ellbar host
// outputs: each item is staged through its lane's own device buffers (copies in,
// estimate, copies out, all on the lane's streams, so one item's copies overlap the
// other lanes' work), and the call waits for the batch.
static abs_status batched(abs_ctx *ctx, int32_t n_items, const abs_item *items, bool host) {
    if (!ctx) return ABS_ERR_INVALID_ARG;
    if (n_items < 0 || (n_items > 0 && !items)) return fail(ctx, ABS_ERR_INVALID_ARG, "n_items < 0 or items NULL");
    DeviceGuard g(ctx->device);
    // items run round-robin over lanes (concurrent streams with their own workspaces),
    // except while the stage profiler runs, on the legacy default stream, for one item,
    // or while a split-BF16 configuration still waits for its launch shape to be
    // measured (the autotuner times candidates on an otherwise idle device, once)
    bool untuned = false;
    if (ctx->autotune)
        for (int32_t i = 0; i < n_items && !untuned; ++i) {
            const abs_config *c = items[i].cfg;
            if (!c || !c->ell_edges || c->n_bins < 1 || c->n_bins > ABS_MAX_BINS) continue;
            const std::string k = setup_key(c);
            if (!ctx->fft_shapes.count(k + "|fft|f64") ||
                (c->precision == ABS_SPLIT_BF16 && !items[i].d_ijk && items[i].n_trip > 0 && !ctx->tc_shapes.count(k)))
                untuned = true;
        }
    const int K = (ctx->profiling || !ctx->stream || n_items < 2 || untuned)
                      ? 1 : std::min<int>(ABS_BATCH_LANES, n_items);
    while ((int)ctx->lanes.size() < K && K > 1) {
        abs_ctx *l = make_lane(ctx);
        if (!l) return fail(ctx, ABS_ERR_OOM, "batch lanes");
        ctx->lanes.push_back(l);
    }
    auto where = [&](int32_t i) { return K > 1 ? ctx->lanes[i % K] : ctx; };
    // validate every item and resolve its setup and triplet list before queuing anything
    std::vector<const Setup *> setups(n_items);
    std::vector<const int32_t *> ijks(n_items);
    std::string key = host ? "batch-host" : "batch";
    bool locked = true;
    for (int32_t i = 0; i < n_items; ++i) {
        abs_status st;
        const abs_item &it = items[i];
        abs_ctx *c = where(i);
        setups[i] = get_setup(c, it.cfg, st);
        if (!setups[i]) return fail(ctx, st, "item " + std::to_string(i) + ": " + c->last_error);
        ijks[i] = it.d_ijk;
        if (estimate_args(c, *setups[i], it.n_vis, it.d_uv, 1, it.d_vis, it.n_trip, ijks[i]) != ABS_OK)
            return fail(ctx, ABS_ERR_INVALID_ARG, "item " + std::to_string(i) + ": " + c->last_error);
        if (host) {
            for (const void *p : {(const void *)it.d_uv, (const void *)it.d_vis, (const void *)it.d_B,
                                  (const void *)it.d_count, (const void *)it.d_ellbar})
                if (p && !page_locked(p)) locked = false;
        }
        char k[256];
        snprintf(k, sizeof k, "|%p|%lld|%p|%p|%d|%p|%p|%p|%p", (const void *)setups[i], (long long)it.n_vis,
                 (const void *)it.d_uv, (const void *)it.d_vis, it.n_trip, (const void *)ijks[i], (void *)it.d_B,
                 (void *)it.d_count, (void *)it.d_ellbar);
        key += k;
    }
    char ks[48];
    snprintf(ks, sizeof ks, "|%p|%d", (const void *)ctx->stream, K);
    key += ks;
    // one item on context c: its estimate, staged through c's buffers for host items
    auto run_item = [&](int32_t i) -> abs_status {
        const abs_item &it = items[i];
        abs_ctx *c = where(i);
        const Setup &s = *setups[i];
        if (!host)
            return estimate_many(c, s, it.n_vis, it.d_uv, 1, it.d_vis, it.n_trip, ijks[i], it.d_B, it.d_count,
                                 it.d_ellbar);
        const size_t uvb = sizeof(float) * 2 * (size_t)it.n_vis;
        float *d_uv = (float *)workspace(c, "host.uv", uvb);
        float *d_vis = (float *)workspace(c, "host.vis", uvb);
        double *d_B = (double *)workspace(c, "host.B", sizeof(double) * (size_t)std::max(it.n_trip, 1));
        int64_t *d_count = (int64_t *)workspace(c, "host.count", sizeof(int64_t) * std::max(it.n_trip, 1));
        double *d_ellbar = (double *)workspace(c, "host.ellbar", sizeof(double) * s.nb);
        if (!d_uv || !d_vis || !d_B || !d_count || !d_ellbar) return fail(c, ABS_ERR_OOM, "host staging");
        abs_status st;
        if (locked) {   // the copies in go inside the estimate (the visibilities beside the plan)
            st = estimate_many(c, s, it.n_vis, d_uv, 1, d_vis, it.n_trip, ijks[i], d_B, d_count, d_ellbar, it.d_uv,
                               it.d_vis);
        } else {
            if (it.n_vis > 0) {
                cudaMemcpyAsync(d_uv, it.d_uv, uvb, cudaMemcpyHostToDevice, c->stream);
                cudaMemcpyAsync(d_vis, it.d_vis, uvb, cudaMemcpyHostToDevice, c->stream);
            }
            st = estimate_many(c, s, it.n_vis, d_uv, 1, d_vis, it.n_trip, ijks[i], d_B, d_count, d_ellbar);
        }
        if (st != ABS_OK) return st;
        if (it.d_B && it.n_trip > 0)
            cudaMemcpyAsync(it.d_B, d_B, sizeof(double) * it.n_trip, cudaMemcpyDeviceToHost, c->stream);
        if (it.d_count && it.n_trip > 0)
            cudaMemcpyAsync(it.d_count, d_count, sizeof(int64_t) * it.n_trip, cudaMemcpyDeviceToHost, c->stream);
        if (it.d_ellbar) cudaMemcpyAsync(it.d_ellbar, d_ellbar, sizeof(double) * s.nb, cudaMemcpyDeviceToHost, c->stream);
        return check_launch(c, "device to host copies");
    };
    auto eager = [&]() {
        if (K > 1) {   // fork: every lane starts after the work queued so far on ctx->stream
            cudaEventRecord(ctx->ev_fork, ctx->stream);
            for (int l = 0; l < K; ++l) cudaStreamWaitEvent(ctx->lanes[l]->stream, ctx->ev_fork, 0);
        }
        abs_status st = ABS_OK;
        for (int32_t i = 0; i < n_items && st == ABS_OK; ++i) {
            abs_ctx *c = where(i);
            st = run_item(i);
            if (st != ABS_OK && c != ctx) ctx->last_error = "item " + std::to_string(i) + ": " + c->last_error;
        }
        if (K > 1) {   // join: ctx->stream waits for every lane
            for (int l = 0; l < K; ++l) {
                cudaEventRecord(ctx->lanes[l]->ev_lane, ctx->lanes[l]->stream);
                cudaStreamWaitEvent(ctx->stream, ctx->lanes[l]->ev_lane, 0);
            }
        }
        return st;
    };
    if (!host) return graphed(ctx, key, eager);
    // pageable host buffers cannot be copied inside a captured graph
    ABS_CHECK(locked ? graphed(ctx, key, eager) : eager());
    return abs_sync(ctx);
}

abs_status abs_estimate_batched(abs_ctx *ctx, int32_t n_items, const abs_item *items) {
    return batched(ctx, n_items, items, false);
}

abs_status abs_estimate_batched_host(abs_ctx *ctx, int32_t n_items, const abs_item *items) {
    return batched(ctx, n_items, items, true);
}

abs_status abs_estimate_host(abs_ctx *ctx, const abs_config *cfg, int64_t n_vis, const float *h_uv,
                             int32_t n_real, const float *h_vis, int32_t n_trip, const int32_t *h_ijk,
                             double *h_B, int64_t *h_count, double *h_ellbar) {
    if (!ctx) return ABS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    abs_status st;
    const Setup *s = get_setup(ctx, cfg, st);
    if (!s) return st;
    const int32_t *probe = h_ijk;
    ABS_CHECK(estimate_args(ctx, *s, n_vis, h_uv, n_real, h_vis, n_trip, probe));
    const size_t uvb = sizeof(float) * 2 * (size_t)n_vis, visb = uvb * (size_t)n_real;
    float *d_uv = (float *)workspace(ctx, "host.uv", uvb);
    float *d_vis = (float *)workspace(ctx, "host.vis", visb);
    double *d_B = (double *)workspace(ctx, "host.B", sizeof(double) * (size_t)std::max(n_trip, 1) * n_real);
    int64_t *d_count = (int64_t *)workspace(ctx, "host.count", sizeof(int64_t) * std::max(n_trip, 1));
    double *d_ellbar = (double *)workspace(ctx, "host.ellbar", sizeof(double) * s->nb);
    const int32_t *d_ijk = s->d_ijk;
    if (h_ijk) {
        int32_t *p = (int32_t *)workspace(ctx, "host.ijk", sizeof(int32_t) * 3 * std::max(n_trip, 1));
        if (!p) return fail(ctx, ABS_ERR_OOM, "host staging");
        if (n_trip > 0) cudaMemcpyAsync(p, h_ijk, sizeof(int32_t) * 3 * n_trip, cudaMemcpyHostToDevice, ctx->stream);
        d_ijk = p;
    }
    if (!d_uv || !d_vis || !d_B || !d_count || !d_ellbar) return fail(ctx, ABS_ERR_OOM, "host staging");
    if (n_vis > 0 && page_locked(h_uv) && page_locked(h_vis)) {
        // the copies go inside the estimate (and its graph): the visibilities' copy runs
        // beside the gridding plan
        ABS_CHECK(estimate_graphed(ctx, *s, n_vis, d_uv, n_real, d_vis, n_trip, d_ijk, d_B, d_count, d_ellbar,
                                   h_uv, h_vis));
    } else {
        if (n_vis > 0) {
            cudaMemcpyAsync(d_uv, h_uv, uvb, cudaMemcpyHostToDevice, ctx->stream);
            cudaMemcpyAsync(d_vis, h_vis, visb, cudaMemcpyHostToDevice, ctx->stream);
        }
        ABS_CHECK(check_launch(ctx, "host to device copies"));
        ABS_CHECK(estimate_graphed(ctx, *s, n_vis, d_uv, n_real, d_vis, n_trip, d_ijk, d_B, d_count, d_ellbar));
    }
    if (h_B && n_trip > 0)
        cudaMemcpyAsync(h_B, d_B, sizeof(double) * (size_t)n_trip * n_real, cudaMemcpyDeviceToHost, ctx->stream);
    if (h_count && n_trip > 0)
        cudaMemcpyAsync(h_count, d_count, sizeof(int64_t) * n_trip, cudaMemcpyDeviceToHost, ctx->stream);
    if (h_ellbar) cudaMemcpyAsync(h_ellbar, d_ellbar, sizeof(double) * s->nb, cudaMemcpyDeviceToHost, ctx->stream);
    ABS_CHECK(check_launch(ctx, "device to host copies"));
    return abs_sync(ctx);
}

}  // extern "C"
