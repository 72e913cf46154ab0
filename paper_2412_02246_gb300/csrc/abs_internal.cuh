// Internal declarations shared by the CUDA translation units of libabs.
// Nothing here is part of the C ABI (include/abs.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/abs.h"

namespace absk {

// --------------------------------------------------------------------------- setup
// Everything derived on the host from an abs_config (validated), cached per
// context.  Integer ring thresholds, sky-grid size and its radix plan, ring
// list offsets, the canonical triplet list.
struct Setup {
    int n = 0, half = 0;          // uv grid side, largest |g| component on the grid
    float du = 0.f;               // binary32 grid spacing
    int kernel = 1, r = 3;        // gridding kernel, footprint half-width
    float s_hi = 0.5f, s_lo = 0.f;  // 1/(2 sigma^2) as a float pair
    int nb = 0;                   // rings
    std::vector<int64_t> q;       // nb+1 thresholds in |g|^2
    std::vector<int> Rm;          // per ring: largest |g_x| of its cells on the grid (-1 empty)
    int R = 0;                    // max over rings
    int N = 0;                    // sky-grid side
    int64_t P = 0;                // points the triple sums run over: N^2 pixels, or the N_z N^2
                                  // voxels of the multi-frequency form's triple stage
    std::vector<int> radices;     // N = prod(radices)
    std::vector<int64_t> lat;     // lattice cells per ring (full annulus, on the grid)
    std::vector<int64_t> lat_off; // nb+1 prefix offsets of lat
    std::vector<int64_t> up_off;  // nb+1 prefix offsets of lat/2 (upper half plane of each ring)
    std::vector<int32_t> ijk;     // canonical closing triplets [t][3]
    int precision = ABS_FP32;
    double norm_A = 1.0;
    int weight_mode = ABS_W_MEAN_UNITMASK;
    // device copies (owned by the context)
    int64_t *d_q = nullptr;
    int64_t *d_lat_off = nullptr;
    int64_t *d_ring_off = nullptr;  // [3][nb+1] family f, ring m: f * up_off[nb] + up_off[m]
    int32_t *d_ijk = nullptr;
    float4 *d_tw = nullptr;       // exp(-2 pi i t / N) = c + i s, t < N, as packed double-float pairs:
                                  // [2t] = (c.hi, c.hi, c.lo, c.lo), [2t+1] = (-s.hi, s.hi, -s.lo, s.lo),
                                  // then in FP32: [2N + t] = (c, c, -s, s)
    int32_t *d_Rm = nullptr;
    // ordered closed-triangle counts of the full annuli [nb][nb][nb] (halved),
    // a property of the ring geometry, computed on first use
    unsigned long long *d_full_counts = nullptr;
    bool full_counts_ready = false;
    // the split-BF16 kernel's tiling of the canonical list, made on first use (type
    // known to triple_tc.cu; its deleter frees the device copies)
    std::shared_ptr<void> tc_plan;
    std::string key;              // the configuration's key (setups, tuned shapes)
};

// The multi-frequency form's setup: the per-channel setup, the triple stage over bins
// u = m n_dbins + a (ring m, delay bin a) and N_z N^2 points with the canonical bin-triplet
// list, and its tables (made on the host from an abs_config3d, cached per context).
struct CubeSetup {
    const Setup *s2 = nullptr;    // per-channel setup (owned by the context's setups)
    Setup st;                     // triple stage: nb = n_bins n_dbins, P = N_z N^2, ijk = bin triplets
    int n_chan = 0, na = 0, t_max = 0, Nz = 0;
    std::vector<int32_t> tau;     // n_dbins + 1 delay-bin edges in |t|
    std::vector<int64_t> T1;      // delay counts [na][na][na]
    int32_t *d_idx2d = nullptr;   // [nb][nb][nb]: index of the sorted ring triple in s2's list, or -1
    int32_t *d_rm2 = nullptr;     // [2 nb (t_max + 1)]: the ring extent of each delay-transform pair, twice
    int32_t *d_tau = nullptr;
    int64_t *d_T1 = nullptr;
    float4 *d_los_tw = nullptr;   // [n_chan] exp(-2 pi i e / n_chan), double-float (re.hi, im.hi, re.lo, im.lo)
    float2 *d_ztw = nullptr;      // [t_max + 1][N_z] c_t (cos, sin)(2 pi (t z mod N_z) / N_z), c_0 = 1, else 2
    ~CubeSetup();
};

// Host-side validation + derivation.  Returns ABS_OK or an error with text in err.
abs_status make_setup(const abs_config *cfg, Setup &s, std::string &err);
// The allocation-free core of make_setup: validation, ring thresholds q[0..nb],
// per-ring largest |g_x| Rm[0..nb-1], R and the sky-grid side N, written to
// caller storage; *err is a static message on failure.
abs_status derive_grid(const abs_config *cfg, int64_t *q, int *Rm, int *R, int *N, const char **err);
// Canonical closing triplets for thresholds q (shared by abs_triplets and Setup).
void closing_triplets(const std::vector<int64_t> &q, std::vector<int32_t> &ijk);
int64_t ring_threshold(double ell, float du);

// --------------------------------------------------------------------------- context
struct Workspace {
    void *p = nullptr;
    size_t bytes = 0;
};

}  // namespace absk

struct abs_ctx {
    // stage profiler: pending (name, start, stop) event triples, totals by name
    struct Pending { std::string name; cudaEvent_t a, b; };
    bool profiling = false;
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> event_pool;
    std::map<std::string, std::pair<double, int64_t>> stage_totals;
    int device = 0;
    cudaStream_t stream = nullptr;
    // a second stream for the exact counts, which abs_estimate runs beside the
    // transforms and triple sums (fork and join by events; both join a graph capture)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int sm_count = 0;
    std::string last_error;
    int32_t *d_err = nullptr;  // latched device error word: 0 ok, else a code below
    std::map<std::string, absk::Workspace> ws;
    std::map<std::string, std::unique_ptr<absk::Setup>> setups;
    // CUDA graphs of abs_estimate(_many) calls, keyed by their arguments: the
    // first call with a key runs eagerly (sizing workspaces, caching per-config
    // tables), the second is captured and replayed from then on.  Dropped
    // whenever a workspace is reallocated (the graphs hold its old address).
    struct Graph { cudaGraphExec_t exec = nullptr; int seen = 0; bool failed = false; };
    std::map<std::string, Graph> graphs;
    // lanes: child contexts, each with its own streams and workspaces (sharing
    // this context's device error word), over which abs_estimate_batched runs
    // its items concurrently; created on first use.  A lane's parent is the
    // context whose graphs may hold the lane's buffers.
    abs_ctx *parent = nullptr;
    // autotuner: launch shapes of the split-BF16 kernel measured on a configuration's
    // first eager call, by configuration key; kept by the root context (lanes share it)
    bool autotune = true;
    int32_t fail_allocs = 0;         // test hook: this many workspace allocations fail next
    // split-BF16 launch shape. budget: accumulator columns per set; waves: work items
    // per CTA (pixel ranges x sets / SMs)
    struct TcShape { bool measured = false; int budget = 0; int waves = 0; };
    std::map<std::string, TcShape> tc_shapes;
    std::map<std::string, std::pair<int, int>> fft_shapes;   // lines per CTA: column pass, row pass
    std::vector<abs_ctx *> lanes;
    // multi-frequency setups by configuration key (they point at entries of setups)
    std::map<std::string, std::unique_ptr<absk::CubeSetup>> cubes;
    bool owns_stream = false;
    cudaEvent_t ev_lane = nullptr;   // a lane's end, joined by the parent
};

namespace absk {

// Concurrent lanes of abs_estimate_batched (items round-robin over them).
constexpr int ABS_BATCH_LANES = 4;
// Creates lanes of ctx (child contexts with their own streams and workspaces, sharing its
// device error word) until it has K.
abs_status ensure_lanes(abs_ctx *ctx, int K);

// Device error codes latched into ctx->d_err (first one wins).
enum : int32_t {
    DERR_NONE = 0,
    DERR_TRIPLET_ORDER = 1,   // triplet list not canonical / bin out of range
    DERR_TRIPLET_BIN = 2,
    DERR_TIMEOUT = 3,
    DERR_CAPACITY = 4,        // an internal work list was too small for the problem
};

// Grow-only named workspace.  Returns nullptr on allocation failure.
void *workspace(abs_ctx *ctx, const char *name, size_t bytes);
// The same, zero-filled (on the context's stream) whenever it is (re)allocated;
// for counters that kernels re-arm themselves after use.
void *workspace_zeroed(abs_ctx *ctx, const char *name, size_t bytes);
abs_status fail(abs_ctx *ctx, abs_status st, const std::string &msg);
abs_status check_launch(abs_ctx *ctx, const char *what);
const Setup *get_setup(abs_ctx *ctx, const abs_config *cfg, abs_status &st);

// --------------------------------------------------------------------------- stage launchers
// Each enqueues on ctx->stream and returns ABS_OK / an error status.
// Gridding is split in a per-baseline-set plan (sort by uv tile and cell) and a
// per-realisation accumulation that reuses it.
// rings_only: the estimate's plan, over the visibilities whose footprint can reach a ring
// cell only (launch_grid_accumulate's estimate form reads it).
abs_status launch_grid_plan(abs_ctx *ctx, const Setup &s, int64_t n_vis, const float *d_uv,
                            bool rings_only = false);
// With d_grid == d_wsum == nullptr only the FP64 accumulators (and, if d_mask,
// the filled mask) are produced.  acc_zeroed: the caller has already cleared
// the accumulators (grid_acc_buffers) on this stream's timeline.
abs_status launch_grid_accumulate(abs_ctx *ctx, const Setup &s, int64_t n_vis, const float *d_vis,
                                  float *d_grid, float *d_wsum, uint8_t *d_mask, bool acc_zeroed = false);
abs_status launch_filter_fft(abs_ctx *ctx, const Setup &s, const float *d_grid,
                             const float *d_wsum, const uint8_t *d_mask, float *d_fields);
// The split-BF16 kernel's operands: the fields as three chunk-blocked planes
// [P_pad / 64][nbp][64] (BF16 hi, BF16 lo, FP32), every 64-pixel row of a ring
// in the 128-byte swizzle of the tensor-core operand (16-byte units XOR-permuted
// by ring & 7), zeros past the last pixel and the last ring.
struct SplitOut {
    void *hi, *lo;   // __nv_bfloat16
    float *f32;
    int nbp;
    int64_t P_pad;
};
// The planes of the canonical triplet list's tiling (workspace of ctx), for the
// transform to write directly; launch_triple_tc with d_fields == NULL then
// reads them as they are (clearing only the padding).
abs_status tc_split_target(abs_ctx *ctx, const Setup &s, SplitOut &out);
// The same transform fed directly from the FP64 gridding accumulators (mirror
// applied on the fly), as abs_estimate uses it; with split given (split-BF16
// precision) the fields go straight into those planes instead of d_fields.
abs_status launch_filter_fft_acc(abs_ctx *ctx, const Setup &s, const double *acc,
                                 float *d_fields, const SplitOut *split = nullptr);
// The I fields of Eq. iFT_I as printed (ABS_W_PAPER_LITERAL): W_g = 1 / (the
// cell's mirrored weight sum) on filled cells, from the FP64 accumulators.
abs_status launch_filter_fft_w(abs_ctx *ctx, const Setup &s, const double *acc, float *d_fields);
// Multi-frequency form: the ring transforms of the delay modes Xt [t_max + 1][(2R + 1)^2]
// (packed double-float complex, cells |gx|, |gy| <= R of the setup), one pair p = m (t_max + 1)
// + t per ring m and delay t >= 0: real fields F [2 p] = FFT of the Hermitian part H1 and
// F [2 p + 1] = FFT of H2 (Xt(., t) = H1 + i H2), each N x N.  d_rm2 [2 nb (t_max + 1)]:
// the largest |g_x| of the pair's ring, twice per pair.
abs_status launch_filter_fft_delay(abs_ctx *ctx, const Setup &s, int t_max, const float4 *d_xt, const int32_t *d_rm2,
                                   float *d_F);
// FP64 accumulators [planes][n*n] (re, im, w before the mirror; see grid_acc_planes) of the last
// launch_grid_accumulate on this context.  A cell received a contribution
// exactly when its weight sum is > 0 (every footprint weight is a normal,
// positive FP32 number, which the sigma_cells bound guarantees).
void grid_acc_buffers(abs_ctx *ctx, const Setup &s, double **acc);
// Accumulator planes the estimate path grids into: re, im and the weight sum (the
// count N_g in the literal form), and the squared-weight sum in the noise form.
int grid_acc_planes(const Setup &s);
// With d_count and d_B also given, B = S / (A T) is written as well (fused
// into the final reduction on the FP32 path).
// wait_before_b, if given, is waited for (on ctx->stream) before B is formed.
abs_status launch_triple_sums(abs_ctx *ctx, const Setup &s, const float *d_fields,
                              int32_t n_trip, const int32_t *d_ijk, double *d_sum,
                              const int64_t *d_count = nullptr, double *d_B = nullptr,
                              cudaEvent_t wait_before_b = nullptr);
// Split-BF16 tcgen05 form of the same sums (precision == ABS_SPLIT_BF16).
// d_fields == NULL (canonical list only): the planes of tc_split_target hold
// the fields already.
abs_status launch_triple_tc(abs_ctx *ctx, const Setup &s, const float *d_fields,
                            int32_t n_trip, const int32_t *d_ijk, double *d_sum);
// Ring tables (cell lists, byte map) from d_mask, or, with d_accw given, from
// the FP64 weight sums before the mirror (a cell is filled when it or its
// mirror has a nonzero sum), then exact counts (d_count may be NULL) and, if
// d_ellbar is not NULL, the mean l of every ring.
abs_status launch_counts(abs_ctx *ctx, const Setup &s, const uint8_t *d_mask, int32_t n_trip,
                         const int32_t *d_ijk, int64_t *d_count, double *d_ellbar,
                         const double *d_accw = nullptr);
// Exclusive scan of len uint32 values on the context's stream (2 kernels);
// bsum holds cdiv(len, 4096) + 1 entries.  False if its counter cannot be allocated.
bool scan_u32(abs_ctx *ctx, const uint32_t *in, int64_t len, uint32_t *out, uint32_t *bsum);
abs_status launch_normalise(abs_ctx *ctx, const Setup &s, int32_t n_trip, const double *d_sum,
                            const int64_t *d_count, double *d_B);
// B = Re S / (A S_W) (NaN where S_W = 0), the literal denominator of Eq. estimator_t.
abs_status launch_normalise_w(abs_ctx *ctx, const Setup &s, int32_t n_trip, const double *d_sum,
                              const double *d_sumw, double *d_B);
abs_status launch_ellbar(abs_ctx *ctx, const Setup &s, const uint8_t *d_mask, double *d_ellbar);
// Fields of a real value per filled cell (d_c [n][n], C(l_g) = C(l_-g); nullptr: the unit mask).
abs_status launch_filter_fft_real(abs_ctx *ctx, const Setup &s, const double *d_c, const uint8_t *d_mask,
                                  float *d_fields);
// out[t] = 2 fs sum_p (P_i P_j I_k + P_j P_k I_i + P_k P_i I_j) / (N^2 T_t): the discretely
// sampled prediction from C fields P and unit-mask fields I (NaN where T = 0).
abs_status launch_bana_sums(abs_ctx *ctx, const Setup &s, const float *d_P, const float *d_I, int32_t n_trip,
                            const int32_t *d_ijk, const int64_t *d_count, double fs, double *d_out);
// Beam-weighted flat sky and its direct DFT at every baseline (visibility simulator).
abs_status launch_simulate_vis(abs_ctx *ctx, int32_t m, double dtheta, const float *d_sky, int32_t beam,
                               double beam_param, int64_t n_vis, const float *d_uv, float *d_vis);
// Count-weighted (l1, mu, t) cells of B and their ensemble mean and spread (results layer).
abs_status launch_rebin(abs_ctx *ctx, const Setup &s, int32_t n_real, int32_t n_trip, const double *d_B,
                        const int64_t *d_count, const double *d_ellbar, const int32_t *d_ijk, int32_t n_mu,
                        int32_t n_t, double *d_mean, double *d_sigma, double *d_weight);
abs_status launch_check_triplets(abs_ctx *ctx, const Setup &s, int32_t n_trip,
                                 const int32_t *d_ijk);

// Multi-frequency form: validation of cfg against the per-channel setup s2, the largest delay
// t_max, the line-of-sight length N_z, the delay counts T1 and the canonical bin triplets
// (rings closing in s2's list, delay count > 0), u <= v <= w lexicographic; *err is a static
// message on failure.
abs_status derive_cube(const abs_config3d *cfg, const Setup &s2, int &t_max, int &Nz, std::vector<int64_t> &T1,
                       std::vector<int32_t> &uvw, const char **err);
const CubeSetup *get_cube_setup(abs_ctx *ctx, const abs_config3d *cfg, abs_status &st);
// The whole multi-frequency estimate on ctx->stream (d_uv, d_vis: [n_chan][n_vis][2]).
abs_status launch_cube_estimate(abs_ctx *ctx, const CubeSetup &c, int64_t n_vis, const float *d_uv,
                                const float *d_vis, int32_t n_trip, const int32_t *d_uvw, double *d_B,
                                int64_t *d_count, double *d_ellbar);

// Brackets the kernel launches of its scope with events when profiling is on.
struct StageTimer {
    abs_ctx *ctx;
    const char *name;
    cudaEvent_t a = nullptr, b = nullptr;
    StageTimer(abs_ctx *c, const char *n);
    ~StageTimer();
};

// --------------------------------------------------------------------------- helpers
__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

#define ABS_CHECK(x)                      \
    do {                                  \
        const abs_status _st = (x);       \
        if (_st != ABS_OK) return _st;    \
    } while (0)

// Lets `kernel` take dynamic shared memory up to the current device's opt-in
// limit less its static shared memory; false when `bytes` is above that or the
// attribute is refused.  The
// attribute belongs to the function, not to a launch: set per call to that
// call's own size, it would go down again for a later configuration while a
// graph captured earlier still holds launches of the larger size, and any
// replay that checks a node against the function (a profiler relaunching the
// nodes one by one does) would refuse them.  It is therefore only ever raised,
// to the limit.
template <class K>
inline bool allow_smem(K kernel, size_t bytes) {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const int limit = optin - (int)fa.sharedSizeBytes;
    if (limit < 0 || bytes > (size_t)limit) return false;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, limit) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

}  // namespace absk
