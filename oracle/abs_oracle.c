/*
 * FP64 CPU oracle for the visibility-based binned angular bispectrum (ABS)
 * estimator of Sec. 2 (Eqs. vg, iFT, iFT_I, estimator_t).
 *
 * TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the
 * CPU-baseline leg of the benchmark are the only callers.  This file shares
 * no code, header, table or helper with the CUDA library; it is a plain,
 * slow, direct restatement of the definitions:
 *
 *   gridding      V_g = sum_i w(U_g - U_i) V(U_i) over the visibilities
 *                 assigned around their nearest grid point (Eq. vg), every
 *                 visibility also entered at -U_i with V* (the sky is real);
 *   mean          X_g = V_g / sum_i w(U_g - U_i) on filled cells, 0 elsewhere
 *                 (the weighting W_g of Eq. iFT);
 *   rings         a_m = { g : Q_m <= |g|^2 < Q_{m+1} },
 *                 Q_m = ceil((l_m / (2 pi dU))^2)  (l = 2 pi |U|, Eq. iFT);
 *   triple sum    S_ijk = sum over ordered (g1,g2,g3), g1 in a_i, g2 in a_j,
 *                 g3 in a_k, all filled, g1+g2+g3 = 0, of X(g1) X(g2) X(g3);
 *   count         T_ijk = number of such closed grid triangles;
 *   estimate      B_ijk = Re S_ijk / (A T_ijk)   (Eq. estimator_t read as the
 *                 average over closed triangles stated after it, Sec. 2).
 *
 * Multi-frequency (3-D) form, a reading of the generalisation that Sec. 1
 * and Sec. 5 name as future work (the paper gives no formula for it):
 *
 *   channels      every channel c = 0 .. n_chan-1 is gridded on the same uv
 *                 grid as above (Eq. vg), giving X_c(g) and its filled mask;
 *   common cells  a cell is used only if it is filled in every channel;
 *   delay modes   Xt(g, t) = sum_c X_c(g) exp(-2 pi i c t / n_chan) on those
 *                 cells (the line-of-sight transform along frequency), for
 *                 integer t with |t| <= t_max, 2 t_max < n_chan;
 *   bins          voxel (g, t) lies in bin u = m n_dbins + a when g is in
 *                 ring a_m and tau_a <= |t| < tau_{a+1};
 *   triple sum    S_uvw = sum over ordered voxel triples, one in each of the
 *                 bins u, v, w, with g1+g2+g3 = 0 and t1+t2+t3 = 0, of
 *                 Xt(g1,t1) Xt(g2,t2) Xt(g3,t3); T_uvw = their number;
 *   estimate      B_uvw = Re S_uvw / (A T_uvw), as in the 2-D form.
 *
 * The triple sum is done by brute force over pairs of ring cells (the O(N^4)
 * "direct" route that Sec. 2 contrasts with the FFT route); no transform is
 * involved, so the FFT identity the CUDA path relies on is checked, not
 * assumed.
 *
 * Floating point: FP64 throughout, except the nearest-cell index, which is
 * defined in IEEE binary32 so that masks (and therefore counts) are
 * reproducible bit for bit: c(u) = floor( fl32( fl32(u / dU) + 0.5 ) ).
 * The grid spacing dU is an IEEE binary32 value everywhere.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared (no fast-math).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* Nearest grid point of a baseline coordinate (Eq. vg: "the grid point U_g
 * nearest to U_i"); binary32 round-to-nearest, ties go up. */
int32_t orc_cell(float u, float du)
{
    volatile float q = u / du;
    volatile float s = q + 0.5f;
    return (int32_t)floorf(s);
}

/* Ring thresholds in integer |g|^2 (half-open [l_m, l_{m+1}) in l = 2 pi |U_g|,
 * U_g = g dU).  q has n_bins + 1 entries. */
void orc_ring_q(int32_t n_bins, const double *ell_edges, float du, int64_t *q)
{
    for (int32_t m = 0; m <= n_bins; ++m) {
        double t = ell_edges[m] / (2.0 * M_PI * (double)du);
        q[m] = (int64_t)ceil(t * t);
    }
}

/* Closing bin triplets i <= j <= k (every combination of three rings that
 * can hold a closed triangle, Sec. 3).  A ring-m cell has
 * Q_m <= |g|^2 <= Q_{m+1} - 1, so g1 + g2 + g3 = 0 needs
 * sqrt(Q_k) <= sqrt(Q_{i+1} - 1) + sqrt(Q_{j+1} - 1); tested in integers.
 * Writes up to `cap` triplets (ijk may be NULL) and returns how many exist. */
int32_t orc_triplets(int32_t n_bins, const int64_t *q, int32_t cap, int32_t *ijk)
{
    int32_t n = 0;
    for (int32_t i = 0; i < n_bins; ++i)
        for (int32_t j = i; j < n_bins; ++j)
            for (int32_t k = j; k < n_bins; ++k) {
                int64_t a = q[i + 1] - 1, b = q[j + 1] - 1;
                int64_t l = q[k] - a - b;
                int closes = (a >= 0 && b >= 0) && (l <= 0 || l * l <= 4 * a * b);
                if (!closes) continue;
                if (ijk && n < cap) {
                    ijk[3 * n + 0] = i;
                    ijk[3 * n + 1] = j;
                    ijk[3 * n + 2] = k;
                }
                ++n;
            }
    return n;
}

static int32_t bin_of(int64_t r2, int32_t n_bins, const int64_t *q)
{
    if (r2 < q[0] || r2 >= q[n_bins]) return -1;
    for (int32_t m = 0; m < n_bins; ++m)
        if (r2 < q[m + 1]) return m;
    return -1;
}

/* Grid cell g = (gx, gy), |gx|,|gy| <= n/2 - 1, stored in FFT order. */
static int64_t cell_at(int32_t n, int32_t gx, int32_t gy)
{
    int32_t ix = gx < 0 ? gx + n : gx;
    int32_t iy = gy < 0 ? gy + n : gy;
    return (int64_t)iy * n + ix;
}

/* Gridding, Eq. vg.  kernel 0: nearest grid point, w = 1.  kernel 1:
 * Gaussian of width sigma (cells) over the (2r+1)^2 cells around the nearest
 * grid point, w = exp(-|U_g - U_i|^2 / (2 sigma^2 dU^2)).  Cells with
 * |gx| or |gy| > n/2 - 1 are dropped (so g and -g are both on the grid).
 * Each visibility is also entered at -U_i with V* and the same weight.
 * Outputs (all n*n, FFT order, zeroed here): grid (re,im), wsum, the sum of
 * the squared weights wsum2 (the noise variance of V_g in units of one
 * visibility's, for equal uncorrelated visibility noise, Sec. 2), and
 * ncontrib, the number N_g of visibilities entered at the cell (Eq. vg). */
int orc_grid(int32_t n, float du, int32_t kernel, double sigma, int32_t radius,
             int64_t n_vis, const float *uv, const float *vis,
             double *grid, double *wsum, double *wsum2, int64_t *ncontrib)
{
    if (n < 4 || (n & 1)) return 1;
    const int64_t cells = (int64_t)n * n;
    memset(grid, 0, sizeof(double) * 2 * cells);
    memset(wsum, 0, sizeof(double) * cells);
    memset(wsum2, 0, sizeof(double) * cells);
    memset(ncontrib, 0, sizeof(int64_t) * cells);
    const int32_t half = n / 2 - 1;
    const double d = (double)du;
    const int32_t r = kernel == 0 ? 0 : radius;
    for (int64_t i = 0; i < n_vis; ++i) {
        const double u = uv[2 * i], v = uv[2 * i + 1];
        const double vre = vis[2 * i], vim = vis[2 * i + 1];
        const int32_t cx = orc_cell(uv[2 * i], du), cy = orc_cell(uv[2 * i + 1], du);
        for (int32_t dy = -r; dy <= r; ++dy)
            for (int32_t dx = -r; dx <= r; ++dx) {
                const int32_t gx = cx + dx, gy = cy + dy;
                if (gx < -half || gx > half || gy < -half || gy > half) continue;
                double w = 1.0;
                if (kernel != 0) {
                    const double ex = gx * d - u, ey = gy * d - v;
                    w = exp(-(ex * ex + ey * ey) / (2.0 * sigma * sigma * d * d));
                }
                const int64_t p = cell_at(n, gx, gy), pm = cell_at(n, -gx, -gy);
                grid[2 * p] += w * vre;
                grid[2 * p + 1] += w * vim;
                wsum[p] += w;
                wsum2[p] += w * w;
                ncontrib[p] += 1;
                grid[2 * pm] += w * vre;      /* mirror: V* at -U */
                grid[2 * pm + 1] -= w * vim;
                wsum[pm] += w;
                wsum2[pm] += w * w;
                ncontrib[pm] += 1;
            }
    }
    return 0;
}

/* Weighted mean on filled cells: X_g = V_g / sum w, filled <=> ncontrib > 0. */
void orc_mean_grid(int32_t n, const double *grid, const double *wsum, const int64_t *ncontrib,
                   double *X, uint8_t *filled)
{
    const int64_t cells = (int64_t)n * n;
    for (int64_t p = 0; p < cells; ++p) {
        if (ncontrib[p] > 0) {
            X[2 * p] = grid[2 * p] / wsum[p];
            X[2 * p + 1] = grid[2 * p + 1] / wsum[p];
            filled[p] = 1;
        } else {
            X[2 * p] = X[2 * p + 1] = 0.0;
            filled[p] = 0;
        }
    }
}

typedef struct { int32_t gx, gy, m; int64_t p; } ring_cell;

static int32_t collect_ring_cells(int32_t n, const uint8_t *filled, int32_t n_bins,
                                  const int64_t *q, ring_cell **out)
{
    const int32_t half = n / 2 - 1;
    int32_t cnt = 0, cap = 1024;
    ring_cell *c = (ring_cell *)malloc(sizeof(ring_cell) * cap);
    for (int32_t gy = -half; gy <= half; ++gy)
        for (int32_t gx = -half; gx <= half; ++gx) {
            const int64_t p = cell_at(n, gx, gy);
            if (!filled[p]) continue;
            const int32_t m = bin_of((int64_t)gx * gx + (int64_t)gy * gy, n_bins, q);
            if (m < 0) continue;
            if (cnt == cap) {
                cap *= 2;
                c = (ring_cell *)realloc(c, sizeof(ring_cell) * cap);
            }
            c[cnt].gx = gx; c[cnt].gy = gy; c[cnt].m = m; c[cnt].p = p;
            ++cnt;
        }
    *out = c;
    return cnt;
}

static int32_t bin_of_cell(int32_t n, const uint8_t *filled, int32_t n_bins, const int64_t *q,
                           int32_t gx, int32_t gy, int64_t *p_out)
{
    const int32_t half = n / 2 - 1;
    if (gx < -half || gx > half || gy < -half || gy > half) return -1;
    const int64_t p = cell_at(n, gx, gy);
    if (!filled[p]) return -1;
    *p_out = p;
    return bin_of((int64_t)gx * gx + (int64_t)gy * gy, n_bins, q);
}

/* Brute-force triple sums and counts for a list of triplets (i,j,k), each
 * over all ordered closed triangles g1 in a_i, g2 in a_j, g3 = -(g1+g2) in
 * a_k.  X: complex [n*n][2]; S: complex [n_trip][2]; absum: sum of |product|
 * per triplet (may be NULL); T: int64 [n_trip].  Visits every pair of ring
 * cells once and files the product under the rings of (g1, g2, g3). */
int orc_triple_bruteforce(int32_t n, const double *X, const uint8_t *filled, int32_t n_bins,
                          const int64_t *q, int32_t n_trip, const int32_t *ijk,
                          double *S, double *absum, int64_t *T)
{
    ring_cell *c = NULL;
    const int32_t nc = collect_ring_cells(n, filled, n_bins, q, &c);
    const int64_t nb = n_bins, nb3 = nb * nb * nb;
    double *sd = (double *)calloc((size_t)(2 * nb3), sizeof(double));
    double *ad = (double *)calloc((size_t)nb3, sizeof(double));
    int64_t *td = (int64_t *)calloc((size_t)nb3, sizeof(int64_t));
    if (!sd || !ad || !td) { free(c); free(sd); free(ad); free(td); return 2; }
    for (int32_t a = 0; a < nc; ++a) {
        const double x1r = X[2 * c[a].p], x1i = X[2 * c[a].p + 1];
        for (int32_t b = 0; b < nc; ++b) {
            int64_t p3 = 0;
            const int32_t k = bin_of_cell(n, filled, n_bins, q, -(c[a].gx + c[b].gx),
                                          -(c[a].gy + c[b].gy), &p3);
            if (k < 0) continue;
            const double x2r = X[2 * c[b].p], x2i = X[2 * c[b].p + 1];
            const double x3r = X[2 * p3], x3i = X[2 * p3 + 1];
            const double pr = x1r * x2r - x1i * x2i, pi = x1r * x2i + x1i * x2r;
            const double tr = pr * x3r - pi * x3i, ti = pr * x3i + pi * x3r;
            const int64_t idx = ((int64_t)c[a].m * nb + c[b].m) * nb + k;
            sd[2 * idx] += tr;
            sd[2 * idx + 1] += ti;
            ad[idx] += sqrt(tr * tr + ti * ti);
            td[idx] += 1;
        }
    }
    for (int32_t t = 0; t < n_trip; ++t) {
        const int64_t idx = ((int64_t)ijk[3 * t] * nb + ijk[3 * t + 1]) * nb + ijk[3 * t + 2];
        S[2 * t] = sd[2 * idx];
        S[2 * t + 1] = sd[2 * idx + 1];
        if (absum) absum[t] = ad[idx];
        T[t] = td[idx];
    }
    free(c); free(sd); free(ad); free(td);
    return 0;
}

/* The discretely sampled analytic bispectrum of the quadratic sky (Sec. 4,
 * Fig. 2): for every ordered closed triangle (g1 in a_i, g2 in a_j, g3 in a_k,
 * all filled) the sum of C(g1) C(g2) + C(g2) C(g3) + C(g3) C(g1), with C a
 * real value per cell ([n][n], FFT order), and the triangle count. */
int orc_bana_bruteforce(int32_t n, const double *C, const uint8_t *filled, int32_t n_bins,
                        const int64_t *q, int32_t n_trip, const int32_t *ijk, double *S, int64_t *T)
{
    ring_cell *c = NULL;
    const int32_t nc = collect_ring_cells(n, filled, n_bins, q, &c);
    const int64_t nb = n_bins, nb3 = nb * nb * nb;
    double *sd = (double *)calloc((size_t)nb3, sizeof(double));
    int64_t *td = (int64_t *)calloc((size_t)nb3, sizeof(int64_t));
    if (!sd || !td) { free(c); free(sd); free(td); return 2; }
    for (int32_t a = 0; a < nc; ++a) {
        const double c1 = C[c[a].p];
        for (int32_t b = 0; b < nc; ++b) {
            int64_t p3 = 0;
            const int32_t k = bin_of_cell(n, filled, n_bins, q, -(c[a].gx + c[b].gx),
                                          -(c[a].gy + c[b].gy), &p3);
            if (k < 0) continue;
            const double c2 = C[c[b].p], c3 = C[p3];
            const int64_t idx = ((int64_t)c[a].m * nb + c[b].m) * nb + k;
            sd[idx] += c1 * c2 + c2 * c3 + c3 * c1;
            td[idx] += 1;
        }
    }
    for (int32_t t = 0; t < n_trip; ++t) {
        const int64_t idx = ((int64_t)ijk[3 * t] * nb + ijk[3 * t + 1]) * nb + ijk[3 * t + 2];
        S[t] = sd[idx];
        T[t] = td[idx];
    }
    free(c); free(sd); free(td);
    return 0;
}

/* The same sums for one triplet only (cost |a_i| |a_j|): used to check
 * sampled outputs of full-size runs. */
int orc_triple_one(int32_t n, const double *X, const uint8_t *filled, int32_t n_bins,
                   const int64_t *q, int32_t i, int32_t j, int32_t k,
                   double *S, double *absum, int64_t *T)
{
    ring_cell *c = NULL;
    const int32_t nc = collect_ring_cells(n, filled, n_bins, q, &c);
    double sr = 0.0, si = 0.0, ab = 0.0;
    int64_t cnt = 0;
    for (int32_t a = 0; a < nc; ++a) {
        if (c[a].m != i) continue;
        const double x1r = X[2 * c[a].p], x1i = X[2 * c[a].p + 1];
        for (int32_t b = 0; b < nc; ++b) {
            if (c[b].m != j) continue;
            int64_t p3 = 0;
            const int32_t m3 = bin_of_cell(n, filled, n_bins, q, -(c[a].gx + c[b].gx),
                                           -(c[a].gy + c[b].gy), &p3);
            if (m3 != k) continue;
            const double x2r = X[2 * c[b].p], x2i = X[2 * c[b].p + 1];
            const double x3r = X[2 * p3], x3i = X[2 * p3 + 1];
            const double pr = x1r * x2r - x1i * x2i, pi = x1r * x2i + x1i * x2r;
            const double tr = pr * x3r - pi * x3i, ti = pr * x3i + pi * x3r;
            sr += tr; si += ti; ab += sqrt(tr * tr + ti * ti);
            ++cnt;
        }
    }
    S[0] = sr; S[1] = si;
    if (absum) *absum = ab;
    *T = cnt;
    free(c);
    return 0;
}

/* Mean multipole of each ring over its filled cells, l_g = 2 pi |g| dU
 * (the ring's "mean radius", Sec. 2).  NaN for a ring with no filled cell. */
void orc_ellbar(int32_t n, float du, const uint8_t *filled, int32_t n_bins, const int64_t *q,
                double *ellbar)
{
    ring_cell *c = NULL;
    const int32_t nc = collect_ring_cells(n, filled, n_bins, q, &c);
    for (int32_t m = 0; m < n_bins; ++m) {
        double s = 0.0;
        int64_t k = 0;
        for (int32_t a = 0; a < nc; ++a)
            if (c[a].m == m) {
                s += 2.0 * M_PI * (double)du * sqrt((double)c[a].gx * c[a].gx + (double)c[a].gy * c[a].gy);
                ++k;
            }
        ellbar[m] = k ? s / (double)k : NAN;
    }
    free(c);
}

/* Binned estimate, Eq. estimator_t: B = Re S / (A T); NaN where T = 0. */
void orc_normalise(int32_t n_trip, const double *S, const int64_t *T, double norm_A, double *B)
{
    for (int32_t t = 0; t < n_trip; ++t)
        B[t] = T[t] > 0 ? S[2 * t] / (norm_A * (double)T[t]) : NAN;
}

/* ------------------------------------------------------------------------
 * Multi-frequency (3-D) form.  See the file header for the definitions.
 * ------------------------------------------------------------------------ */

/* Delay modes of the channel cube.  X: complex [n_chan][n*n][2] (the
 * per-channel means of orc_mean_grid), filled: [n_chan][n*n].  Outputs:
 * common[n*n] = 1 where every channel is filled; Xt: complex
 * [2 t_max + 1][n*n][2], Xt[t + t_max] = sum_c X_c exp(-2 pi i c t / n_chan)
 * on common cells and 0 elsewhere.  Returns 1 unless 0 <= 2 t_max < n_chan. */
int orc_delay_modes(int32_t n, int32_t n_chan, const double *X, const uint8_t *filled, int32_t t_max,
                    double *Xt, uint8_t *common)
{
    if (n_chan < 1 || t_max < 0 || 2 * t_max >= n_chan) return 1;
    const int64_t cells = (int64_t)n * n;
    const int32_t nt = 2 * t_max + 1;
    for (int64_t p = 0; p < cells; ++p) {
        uint8_t all = 1;
        for (int32_t c = 0; c < n_chan; ++c)
            if (!filled[(int64_t)c * cells + p]) all = 0;
        common[p] = all;
        for (int32_t ti = 0; ti < nt; ++ti) {
            const int32_t t = ti - t_max;
            double sr = 0.0, si = 0.0;
            if (all)
                for (int32_t c = 0; c < n_chan; ++c) {
                    /* exp(-2 pi i c t / n_chan), the exponent reduced to [0, n_chan) */
                    const int64_t e = (((int64_t)c * t) % n_chan + n_chan) % n_chan;
                    const double ang = -2.0 * M_PI * (double)e / (double)n_chan;
                    const double wr = cos(ang), wi = sin(ang);
                    const double xr = X[2 * ((int64_t)c * cells + p)], xi = X[2 * ((int64_t)c * cells + p) + 1];
                    sr += xr * wr - xi * wi;
                    si += xr * wi + xi * wr;
                }
            Xt[2 * ((int64_t)ti * cells + p)] = sr;
            Xt[2 * ((int64_t)ti * cells + p) + 1] = si;
        }
    }
    return 0;
}

/* Delay bin of a delay index t: a with tau_a <= |t| < tau_{a+1}, or -1. */
static int32_t dbin_of(int32_t t, int32_t n_dbins, const int32_t *tau)
{
    const int32_t at = t < 0 ? -t : t;
    for (int32_t a = 0; a < n_dbins; ++a)
        if (at >= tau[a] && at < tau[a + 1]) return a;
    return -1;
}

typedef struct { int32_t gx, gy, t, u; int64_t p; } voxel;

/* Brute-force 3-D triple sums and counts for a list of bin triplets (u, v, w):
 * every ordered pair of voxels in the bins is visited once, the third voxel
 * is (-(g1+g2), -(t1+t2)), and the product is filed under the bins of the
 * three.  Xt, common as from orc_delay_modes; S: complex [n_trip][2]; absum
 * (may be NULL): sum of |product|; T: int64 [n_trip]. */
int orc_triple3d_bruteforce(int32_t n, int32_t t_max, const double *Xt, const uint8_t *common, int32_t n_bins,
                            const int64_t *q, int32_t n_dbins, const int32_t *tau, int32_t n_trip,
                            const int32_t *uvw, double *S, double *absum, int64_t *T)
{
    const int64_t cells = (int64_t)n * n;
    ring_cell *c = NULL;
    const int32_t nc = collect_ring_cells(n, common, n_bins, q, &c);
    const int32_t nt = 2 * t_max + 1;
    voxel *vx = (voxel *)malloc(sizeof(voxel) * ((size_t)nc * nt + 1));
    const int64_t nb3 = (int64_t)n_bins * n_dbins, nb33 = nb3 * nb3 * nb3;
    double *sd = (double *)calloc((size_t)(2 * nb33), sizeof(double));
    double *ad = (double *)calloc((size_t)nb33, sizeof(double));
    int64_t *td = (int64_t *)calloc((size_t)nb33, sizeof(int64_t));
    if (!vx || !sd || !ad || !td) { free(c); free(vx); free(sd); free(ad); free(td); return 2; }
    int64_t nv = 0;
    for (int32_t a = 0; a < nc; ++a)
        for (int32_t t = -t_max; t <= t_max; ++t) {
            const int32_t d = dbin_of(t, n_dbins, tau);
            if (d < 0) continue;
            vx[nv].gx = c[a].gx; vx[nv].gy = c[a].gy; vx[nv].t = t;
            vx[nv].u = c[a].m * n_dbins + d;
            vx[nv].p = c[a].p;
            ++nv;
        }
    for (int64_t a = 0; a < nv; ++a) {
        const int64_t o1 = (int64_t)(vx[a].t + t_max) * cells + vx[a].p;
        const double x1r = Xt[2 * o1], x1i = Xt[2 * o1 + 1];
        for (int64_t b = 0; b < nv; ++b) {
            const int32_t t3 = -(vx[a].t + vx[b].t);
            if (t3 < -t_max || t3 > t_max) continue;
            const int32_t d3 = dbin_of(t3, n_dbins, tau);
            if (d3 < 0) continue;
            int64_t p3 = 0;
            const int32_t m3 = bin_of_cell(n, common, n_bins, q, -(vx[a].gx + vx[b].gx),
                                           -(vx[a].gy + vx[b].gy), &p3);
            if (m3 < 0) continue;
            const int64_t o2 = (int64_t)(vx[b].t + t_max) * cells + vx[b].p;
            const int64_t o3 = (int64_t)(t3 + t_max) * cells + p3;
            const double x2r = Xt[2 * o2], x2i = Xt[2 * o2 + 1];
            const double x3r = Xt[2 * o3], x3i = Xt[2 * o3 + 1];
            const double pr = x1r * x2r - x1i * x2i, pi = x1r * x2i + x1i * x2r;
            const double tr = pr * x3r - pi * x3i, ti = pr * x3i + pi * x3r;
            const int64_t w = (int64_t)m3 * n_dbins + d3;
            const int64_t idx = ((int64_t)vx[a].u * nb3 + vx[b].u) * nb3 + w;
            sd[2 * idx] += tr;
            sd[2 * idx + 1] += ti;
            ad[idx] += sqrt(tr * tr + ti * ti);
            td[idx] += 1;
        }
    }
    for (int32_t t = 0; t < n_trip; ++t) {
        const int64_t u = uvw[3 * t], v = uvw[3 * t + 1], w = uvw[3 * t + 2];
        if (u < 0 || v < 0 || w < 0 || u >= nb3 || v >= nb3 || w >= nb3) {
            S[2 * t] = S[2 * t + 1] = 0.0;
            if (absum) absum[t] = 0.0;
            T[t] = 0;
            continue;
        }
        const int64_t idx = (u * nb3 + v) * nb3 + w;
        S[2 * t] = sd[2 * idx];
        S[2 * t + 1] = sd[2 * idx + 1];
        if (absum) absum[t] = ad[idx];
        T[t] = td[idx];
    }
    free(c); free(vx); free(sd); free(ad); free(td);
    return 0;
}
