// Stage 2: ring-restricted transforms, Eqs. iFT and iFT_I (Sec. 2).
//
// For ring m, X_m(g) = V_g / sum w on the filled cells of a_m, zero elsewhere,
// and D_m(p) = sum_g X_m(g) exp(-2 pi i g.p / N) on the N x N sky grid.
// Because X_m is Hermitian, D_m is real, so two rings a, b are transformed at
// once as Z = X_a + i X_b, giving D_a = Re FFT(Z) and D_b = Im FFT(Z).
//
// The 2D transform is a column pass then a row pass.  Only the columns
// |g_x| <= R_b of a ring pair are nonzero, so the column pass transforms
// just those columns (along y) into a compact intermediate [2R+1][N]; the
// row pass reads RB adjacent sky rows of it, expands each to length N with
// the zero columns, transforms along x and writes RB whole rows of both
// fields, so the dominant write (the fields) is contiguous.
//
// Arithmetic.  Rounding inside an FP32 FFT leaves an error of order
// eps log N ||X|| on every output, independent of the output's size, and
// the triple sums amplify it by their cancellation; rounding the exact
// field to FP32 once costs far less.  The butterflies therefore run in
// double-float: every real is an unevaluated sum hi + lo of two FP32 values
// (Dekker/Knuth two-sum and FMA two-product), twiddles and radix constants
// carry their own low parts, and only the output is rounded to FP32.  That
// is the FP32 path.  The split-BF16 path rounds its triplet operands to
// about 2^-17 relative anyway, far above the plain FP32 transform's error,
// so its butterflies run in plain packed FP32 (float2 complex values, half
// the intermediate's bytes) with each cell's value rounded once on entry.
//
// Both passes are radix-2/3/4/5 Stockham transforms in shared memory (pass
// with span p and radix R reads x[i + q N/R], applies the twiddle
// exp(-2 pi i q (i mod p) / (p R)), and writes the R outputs at
// (i div p) p R + (i mod p) + s p); divisions by runtime constants use
// precomputed multiply-high magic numbers.
#include "abs_internal.cuh"

namespace absk {
namespace {

constexpr int MAXRAD = 16;
constexpr int FFT_NT = 128;     // threads per transform CTA
constexpr int FFT_FIXED = 2;    // a CTA's fixed cost (barriers, first loads) in lines of work

struct FftPass {
    int R, p, T, tstep;
    uint32_t mag_p, mag_T;   // floor(x / p) = umulhi(x, mag_p) for x < 2^16
};

struct FftPlan {
    int N, nrad;
    FftPass pass[MAXRAD];
};

struct RingGeom {
    int n, half, nb, N, Rmax;
};

// ------------------------------------------------------------------ double-float
// A complex double-float value is held as two float2 registers, hi = (re.hi,
// im.hi) and lo = (re.lo, im.lo), so that the real and imaginary parts go
// through the same packed FP32x2 instruction (FADD2 / FMUL2 / FFMA2): every
// complex addition or real scaling costs what one real double-float operation
// costs in scalar code.  Stored as float4 (re.hi, im.hi, re.lo, im.lo).

struct pdf {
    float2 hi, lo;
};

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.f, -1.f), a); }  // a - b

// TwoSum of the high parts, low parts added, then Fast2Sum renormalisation.
__device__ __forceinline__ pdf p_add(pdf a, pdf b) {
    const float2 s = __fadd2_rn(a.hi, b.hi);
    const float2 bb = f2sub(s, a.hi);
    float2 e = __fadd2_rn(f2sub(a.hi, f2sub(s, bb)), f2sub(b.hi, bb));
    e = __fadd2_rn(e, __fadd2_rn(a.lo, b.lo));
    const float2 hi = __fadd2_rn(s, e);
    return {hi, f2sub(e, f2sub(hi, s))};
}
__device__ __forceinline__ pdf p_neg(pdf a) { return {f2(-a.hi.x, -a.hi.y), f2(-a.lo.x, -a.lo.y)}; }
__device__ __forceinline__ pdf p_sub(pdf a, pdf b) { return p_add(a, p_neg(b)); }
// TwoProduct of the high parts (FMA), cross terms added, renormalised.
__device__ __forceinline__ pdf p_mul(pdf a, pdf b) {
    const float2 p = __fmul2_rn(a.hi, b.hi);
    float2 e = __ffma2_rn(a.hi, b.hi, f2(-p.x, -p.y));
    e = __ffma2_rn(a.hi, b.lo, e);
    e = __ffma2_rn(a.lo, b.hi, e);
    const float2 hi = __fadd2_rn(p, e);
    return {hi, f2sub(e, f2sub(hi, p))};
}
__device__ __forceinline__ pdf p_half(pdf a) { return {__fmul2_rn(a.hi, f2(0.5f, 0.5f)), __fmul2_rn(a.lo, f2(0.5f, 0.5f))}; }
__device__ __forceinline__ pdf ld(const float4 v) { return {f2(v.x, v.y), f2(v.z, v.w)}; }
__device__ __forceinline__ float4 st(pdf a) { return make_float4(a.hi.x, a.hi.y, a.lo.x, a.lo.y); }
// a * (-i) = (im, -re)
__device__ __forceinline__ pdf c_mi(pdf a) { return {f2(a.hi.y, -a.hi.x), f2(a.lo.y, -a.lo.x)}; }
// a * w with w = c + i s given as wr = (c, c), wi = (-s, s): a wr + swap(a) wi
__device__ __forceinline__ pdf c_mul_tw(pdf a, pdf wr, pdf wi) {
    const pdf sw = {f2(a.hi.y, a.hi.x), f2(a.lo.y, a.lo.x)};
    return p_add(p_mul(a, wr), p_mul(sw, wi));
}

// radix constants as double-float pairs, broadcast to (re, im)
constexpr double kS3 = 0.86602540378443864676372317075294;   // sin(2 pi / 3)
constexpr double kC1 = 0.30901699437494742410229341718282;   // cos(2 pi / 5)
constexpr double kC2 = -0.80901699437494742410229341718282;  // cos(4 pi / 5)
constexpr double kS1 = 0.95105651629515357211643933337938;   // sin(2 pi / 5)
constexpr double kS2 = 0.58778525229247312916870595463907;   // sin(4 pi / 5)
__device__ __forceinline__ pdf pconst(double v) {
    const float h = (float)v, l = (float)(v - (double)h);
    return {f2(h, h), f2(l, l)};
}

// The two arithmetics of the butterflies.  DF: double-float complex values
// stored as float4, twiddles as two float4 per index (the packed layout of
// Setup::d_tw).  F32: plain FP32 complex values stored as float2 (re, im),
// twiddles as one float4 (c, c, -s, s) per index (the table after it).  The
// twiddles are read through the L1 cache, shared by every CTA on the SM.
struct ArithDF {
    using E = float4;
    using C = pdf;
    __host__ __device__ static const float4 *table(const float4 *tw, int N) { return tw; }
    __device__ static C ld(E v) { return ::absk::ld(v); }
    __device__ static E st(C a) { return ::absk::st(a); }
    __device__ static C add(C a, C b) { return p_add(a, b); }
    __device__ static C sub(C a, C b) { return p_sub(a, b); }
    __device__ static C mi(C a) { return c_mi(a); }
    __device__ static C half(C a) { return p_half(a); }
    __device__ static C cst(double v) { return pconst(v); }
    __device__ static C mul(C a, C c) { return p_mul(a, c); }
    __device__ static C twiddle(C v, const float4 *__restrict__ tw, int t) {
        return c_mul_tw(v, ::absk::ld(__ldg(tw + 2 * t)), ::absk::ld(__ldg(tw + 2 * t + 1)));
    }
    // a cell value (re.hi, im.hi, re.lo, im.lo) as stored, and i times it
    __device__ static E from_cell(float4 v) { return v; }
    __device__ static E times_i(float4 v) { return make_float4(-v.y, v.x, -v.w, v.z); }
    __device__ static E zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    __device__ static float re(E v) { return __fadd_rn(v.x, v.z); }
    __device__ static float im(E v) { return __fadd_rn(v.y, v.w); }
};

struct ArithF32 {
    using E = float2;
    using C = float2;
    __host__ __device__ static const float4 *table(const float4 *tw, int N) { return tw + 2 * (size_t)N; }
    __device__ static C ld(E v) { return v; }
    __device__ static E st(C a) { return a; }
    __device__ static C add(C a, C b) { return __fadd2_rn(a, b); }
    __device__ static C sub(C a, C b) { return f2sub(a, b); }
    __device__ static C mi(C a) { return f2(a.y, -a.x); }
    __device__ static C half(C a) { return __fmul2_rn(a, f2(0.5f, 0.5f)); }
    __device__ static C cst(double v) { return f2((float)v, (float)v); }
    __device__ static C mul(C a, C c) { return __fmul2_rn(a, c); }
    // v w = v (c, c) + (v.im, v.re) (-s, s)
    __device__ static C twiddle(C v, const float4 *__restrict__ tw, int t) {
        const float4 w = __ldg(tw + t);
        return __ffma2_rn(f2(v.y, v.x), f2(w.z, w.w), __fmul2_rn(v, f2(w.x, w.y)));
    }
    // the cell value rounded once to FP32
    __device__ static E from_cell(float4 v) { return f2(__fadd_rn(v.x, v.z), __fadd_rn(v.y, v.w)); }
    __device__ static E times_i(float4 v) { return f2(-__fadd_rn(v.y, v.w), __fadd_rn(v.x, v.z)); }
    __device__ static E zero() { return f2(0.f, 0.f); }
    __device__ static float re(E v) { return v.x; }
    __device__ static float im(E v) { return v.y; }
};

// One Stockham pass over `lines` transforms of length N stored line-major.
template <class A>
__device__ __forceinline__ void stockham_pass(const typename A::E *__restrict__ in, typename A::E *__restrict__ out,
                                              int N, const FftPass &P, int lines,
                                              const float4 *__restrict__ tw) {
    using C = typename A::C;
    const int R = P.R, p = P.p, T = P.T;
    const int nbf = lines * T;
    for (int b = threadIdx.x; b < nbf; b += blockDim.x) {
        const int l = (int)__umulhi((uint32_t)b, P.mag_T);
        const int i = b - l * T;
        const int ip = p == 1 ? i : (int)__umulhi((uint32_t)i, P.mag_p);
        const int k = i - ip * p;
        const typename A::E *src = in + (size_t)l * N + i;
        typename A::E *dst = out + (size_t)l * N + ip * p * R + k;
        C x[5];
        x[0] = A::ld(src[0]);
#pragma unroll
        for (int q = 1; q < 5; ++q) {
            if (q < R) {
                const C v = A::ld(src[q * T]);
                x[q] = k ? A::twiddle(v, tw, q * k * P.tstep) : v;
            }
        }
        if (R == 4) {
            const C a0 = A::add(x[0], x[2]), a1 = A::sub(x[0], x[2]);
            const C b0 = A::add(x[1], x[3]), b1 = A::mi(A::sub(x[1], x[3]));
            dst[0] = A::st(A::add(a0, b0));
            dst[p] = A::st(A::add(a1, b1));
            dst[2 * p] = A::st(A::sub(a0, b0));
            dst[3 * p] = A::st(A::sub(a1, b1));
        } else if (R == 2) {
            dst[0] = A::st(A::add(x[0], x[1]));
            dst[p] = A::st(A::sub(x[0], x[1]));
        } else if (R == 3) {
            const C t = A::add(x[1], x[2]);
            const C m = A::sub(x[0], A::half(t));
            const C d = A::mul(A::mi(A::sub(x[1], x[2])), A::cst(kS3));
            dst[0] = A::st(A::add(x[0], t));
            dst[p] = A::st(A::add(m, d));
            dst[2 * p] = A::st(A::sub(m, d));
        } else {  // R == 5
            const C c1 = A::cst(kC1), c2 = A::cst(kC2), s1 = A::cst(kS1), s2 = A::cst(kS2);
            const C t1 = A::add(x[1], x[4]), t2 = A::add(x[2], x[3]);
            const C t3 = A::sub(x[1], x[4]), t4 = A::sub(x[2], x[3]);
            const C a1 = A::add(x[0], A::add(A::mul(t1, c1), A::mul(t2, c2)));
            const C a2 = A::add(x[0], A::add(A::mul(t1, c2), A::mul(t2, c1)));
            const C b1 = A::mi(A::add(A::mul(t3, s1), A::mul(t4, s2)));
            const C b2 = A::mi(A::sub(A::mul(t3, s2), A::mul(t4, s1)));
            dst[0] = A::st(A::add(x[0], A::add(t1, t2)));
            dst[p] = A::st(A::add(a1, b1));
            dst[4 * p] = A::st(A::sub(a1, b1));
            dst[2 * p] = A::st(A::add(a2, b2));
            dst[3 * p] = A::st(A::sub(a2, b2));
        }
    }
}

// Transforms `lines` lines in buffer a (scratch b); returns the buffer holding the result.
template <class A>
__device__ typename A::E *fft_lines(typename A::E *a, typename A::E *b, int lines, const FftPlan &P,
                                    const float4 *__restrict__ tw) {
    for (int s = 0; s < P.nrad; ++s) {
        __syncthreads();
        stockham_pass<A>(a, b, P.N, P.pass[s], lines, tw);
        typename A::E *t = a;
        a = b;
        b = t;
    }
    __syncthreads();
    return a;
}

// Double-float a / b (hi, lo pairs, b > 0): q1 = a_hi / b_hi, the exact
// remainder a - q1 b by TwoProduct, one correction q2 = r / b_hi, renormalised.
// Relative error about 2^-44, in FP32 arithmetic only.
__device__ __forceinline__ void df_div(float a_hi, float a_lo, float b_hi, float b_lo, float &q_hi, float &q_lo) {
    const float q1 = __fdiv_rn(a_hi, b_hi);
    const float p_hi = __fmul_rn(q1, b_hi);
    const float p_lo = fmaf(q1, b_hi, -p_hi);
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(__fsub_rn(a_hi, p_hi), p_lo), __fmul_rn(q1, b_lo)), a_lo);
    const float q2 = __fdiv_rn(r, b_hi);
    q_hi = __fadd_rn(q1, q2);
    q_lo = __fsub_rn(q2, __fsub_rn(q_hi, q1));
}

// A double as a double-float pair (two roundings to FP32).
__device__ __forceinline__ void df_of(double v, float &hi, float &lo) {
    hi = __double2float_rn(v);
    lo = __double2float_rn(v - (double)hi);
}

// Gridded data as the transform reads it: the weighted mean X on a filled
// cell, as a packed double-float complex (re.hi, im.hi, re.lo, im.lo).
struct GridF32 {   // abs_grid outputs (FP32)
    static constexpr const char *tag = "f32";
    const float2 *grid;
    const float *wsum;
    const uint8_t *mask;
    __device__ bool value(int64_t cell, int64_t mcell, float4 &x) const {
        if (!mask[cell]) return false;
        const float2 g = grid[cell];
        const float w = wsum[cell];
        float rh, rl, ih, il;
        df_div(g.x, 0.f, w, 0.f, rh, rl);
        df_div(g.y, 0.f, w, 0.f, ih, il);
        x = make_float4(rh, ih, rl, il);
        return true;
    }
};
struct GridF64 {   // FP64 accumulators before the mirror (inside abs_estimate)
    static constexpr const char *tag = "f64";
    const double *re, *im, *w;
    __device__ bool value(int64_t cell, int64_t mcell, float4 &x) const {
        // the mirrored sums in FP64, then the division in double-float (GB300's
        // FP64 pipe is narrow; the sums need FP64, the quotient does not)
        const double ww = w[cell] + w[mcell];   // > 0 exactly on filled cells
        if (!(ww > 0.0)) return false;
        float wh, wl, ah, al, bh, bl, rh, rl, ih, il;
        df_of(ww, wh, wl);
        df_of(re[cell] + re[mcell], ah, al);
        df_of(im[cell] - im[mcell], bh, bl);
        df_div(ah, al, wh, wl, rh, rl);
        df_div(bh, bl, wh, wl, ih, il);
        x = make_float4(rh, ih, rl, il);
        return true;
    }
};

// Weights of the I fields of Eq. iFT_I as printed: W_g = 1 / N_g on a filled
// cell, N_g its mirrored weight sum in FP64 (real: N_g = N_-g), the quotient
// in double-float.
struct GridW64 {
    static constexpr const char *tag = "w64";
    const double *w;
    __device__ bool value(int64_t cell, int64_t mcell, float4 &x) const {
        const double ww = w[cell] + w[mcell];
        if (!(ww > 0.0)) return false;
        float wh, wl, rh, rl;
        df_of(ww, wh, wl);
        df_div(1.f, 0.f, wh, wl, rh, rl);
        x = make_float4(rh, 0.f, rl, 0.f);
        return true;
    }
};

// A real value per cell on the filled cells (the caller's C(l_g), which must
// equal C(l_-g); with C == nullptr the unit mask): the fields of the
// discretely sampled prediction.
struct GridReal {
    static constexpr const char *tag = "real";
    const double *c;
    const uint8_t *mask;
    __device__ bool value(int64_t cell, int64_t mcell, float4 &x) const {
        if (!mask[cell]) return false;
        float h = 1.f, l = 0.f;
        if (c) df_of(c[cell], h, l);
        x = make_float4(h, 0.f, l, 0.f);
        return true;
    }
};

// Column pass: one CTA per (block of CB columns x, ring pair), transforming
// along y the 2R+1 columns |x| <= R that hold ring cells.  W[pair][x + Rmax][N].
template <class Src, class A>
__global__ void __launch_bounds__(FFT_NT) k_fft_cols(RingGeom G, FftPlan P, int CB, const int64_t *__restrict__ q,
                                                  const int32_t *__restrict__ Rm, Src src,
                                                  const float4 *__restrict__ tw,
                                                  typename A::E *__restrict__ W) {
    using E = typename A::E;
    extern __shared__ float4 sbuf[];
    const int pair = blockIdx.y;
    const int a = 2 * pair, b = a + 1 < G.nb ? a + 1 : -1;
    const int Rp = max(Rm[a], b >= 0 ? Rm[b] : -1);
    const int x0 = (int)blockIdx.x * CB - G.Rmax;
    if (Rp < 0 || x0 > Rp || x0 + CB - 1 < -Rp) return;
    E *l0 = (E *)sbuf, *l1 = l0 + (size_t)CB * G.N;
    for (int i = threadIdx.x; i < CB * G.N; i += blockDim.x) l0[i] = A::zero();
    __syncthreads();
    const int span = 2 * Rp + 1;
    const int64_t qa0 = q[a], qa1 = q[a + 1], qb0 = b >= 0 ? q[b] : 0, qb1 = b >= 0 ? q[b + 1] : 0;
    // consecutive threads take consecutive x of one row (adjacent cells)
    for (int e = threadIdx.x; e < CB * span; e += blockDim.x) {
        const int yy = e / CB, c = e - yy * CB, x = x0 + c, y = yy - Rp;
        if (x < -Rp || x > Rp || y < -G.half || y > G.half || x < -G.half || x > G.half) continue;
        const int64_t r2 = (int64_t)x * x + (int64_t)y * y;
        const bool in_a = r2 >= qa0 && r2 < qa1, in_b = b >= 0 && r2 >= qb0 && r2 < qb1;
        if (!in_a && !in_b) continue;
        const int64_t cell = (int64_t)(y < 0 ? y + G.n : y) * G.n + (x < 0 ? x + G.n : x);
        const int64_t mcell = (int64_t)(y > 0 ? G.n - y : -y) * G.n + (x > 0 ? G.n - x : -x);
        float4 v;
        if (!src.value(cell, mcell, v)) continue;
        // Z = X_a + i X_b
        l0[(size_t)c * G.N + (y < 0 ? y + G.N : y)] = in_a ? A::from_cell(v) : A::times_i(v);
    }
    E *res = fft_lines<A>(l0, l1, CB, P, tw);
    for (int e = threadIdx.x; e < CB * G.N; e += blockDim.x) {
        const int c = e / G.N, x = x0 + c;
        if (x < -Rp || x > Rp) continue;
        W[((size_t)pair * (2 * G.Rmax + 1) + (x + G.Rmax)) * G.N + (e - c * G.N)] = res[e];
    }
}

// Row pass: one CTA per (block of RB sky rows py, ring pair), transforming
// along x; each output row of both fields is written whole (contiguous).
template <class A>
__global__ void __launch_bounds__(FFT_NT) k_fft_rows(RingGeom G, FftPlan P, int RB,
                                                  const int32_t *__restrict__ Rm,
                                                  const typename A::E *__restrict__ W,
                                                  const float4 *__restrict__ tw,
                                                  float *__restrict__ fields) {
    using E = typename A::E;
    extern __shared__ float4 sbuf[];
    const int pair = blockIdx.y;
    const int a = 2 * pair, b = a + 1 < G.nb ? a + 1 : -1;
    const int Rp = max(Rm[a], b >= 0 ? Rm[b] : -1);
    const int py0 = blockIdx.x * RB;
    const int rb = min(RB, G.N - py0);
    const size_t P2 = (size_t)G.N * G.N;
    float *fa = fields + (size_t)a * P2 + (size_t)py0 * G.N;
    float *fb = b >= 0 ? fields + (size_t)b * P2 + (size_t)py0 * G.N : nullptr;
    if (Rp < 0) {  // both rings empty: zero fields
        for (int i = threadIdx.x; i < rb * G.N; i += blockDim.x) {
            fa[i] = 0.f;
            if (fb) fb[i] = 0.f;
        }
        return;
    }
    E *l0 = (E *)sbuf, *l1 = l0 + (size_t)RB * G.N;
    for (int i = threadIdx.x; i < RB * G.N; i += blockDim.x) l0[i] = A::zero();
    __syncthreads();
    const int cols = 2 * Rp + 1;
    const E *src = W + (size_t)pair * (2 * G.Rmax + 1) * G.N;
    for (int i = threadIdx.x; i < cols * rb; i += blockDim.x) {
        const int col = i / rb, r = i - col * rb;
        const int x = col - Rp;
        l0[(size_t)r * G.N + (x < 0 ? x + G.N : x)] = src[(size_t)(x + G.Rmax) * G.N + py0 + r];
    }
    E *res = fft_lines<A>(l0, l1, RB, P, tw);
    for (int i = threadIdx.x; i < rb * G.N; i += blockDim.x) {
        const E v = res[i];
        fa[i] = A::re(v);
        if (fb) fb[i] = A::im(v);
    }
}

uint32_t magic(int d) {  // floor(x / d) == umulhi(x, magic(d)) for 0 <= x < 2^16, 2 <= d < 2^16
    return d < 2 ? 0u : (uint32_t)(((uint64_t)1 << 32) / (uint64_t)d + 1);
}

FftPlan make_plan(const Setup &s) {
    FftPlan P;
    P.N = s.N;
    P.nrad = (int)s.radices.size();
    int p = 1;
    for (int i = 0; i < P.nrad && i < MAXRAD; ++i) {
        FftPass &q = P.pass[i];
        q.R = s.radices[i];
        q.p = p;
        q.T = s.N / q.R;
        q.tstep = s.N / (p * q.R);
        q.mag_p = magic(p);
        q.mag_T = magic(q.T);
        p *= q.R;
    }
    return P;
}

struct FftLaunch {
    int CB, RB;   // columns per CTA of the column pass, rows per CTA of the row pass
    size_t col_smem, row_smem;
};

// Lines per CTA for a pass over `lines` lines of each of `npairs` ring pairs:
// the count that minimises (CTA waves) x (lines per CTA + FFT_FIXED), a CTA
// holding two line buffers in shared memory and at most max_per_sm CTAs
// sharing an SM (threads and registers); both passes are latency-bound at
// moderate N, so a last, part-filled wave costs a whole one.
static int lines_per_cta(size_t line, int lines, int npairs, int sm_count, int max_per_sm) {
    int best = 1;
    int64_t best_cost = INT64_MAX;
    for (int w = 1; w <= 16; ++w) {
        const size_t smem = line * 2 * w;
        if (smem > 200 * 1024) break;
        const int per_sm = (int)std::min<size_t>(max_per_sm, (228 * 1024) / (smem + 1024));
        if (per_sm < 1) break;
        const int64_t ctas = cdiv(lines, w) * (int64_t)npairs;
        const int64_t cost = cdiv(ctas, (int64_t)sm_count * per_sm) * (w + FFT_FIXED);
        if (cost < best_cost) {
            best_cost = cost;
            best = w;
        }
    }
    return best;
}

// The transforms run in double-float on the FP32 path and in plain FP32 on the
// split-BF16 path, whose triplet products carry a larger error of their own.
static bool plain_fp32(const Setup &s) { return s.precision == ABS_SPLIT_BF16; }

FftLaunch fft_launch(const Setup &s, int sm_count) {
    FftLaunch L;
    const bool f32 = plain_fp32(s);
    const size_t line = (f32 ? sizeof(float2) : sizeof(float4)) * (size_t)s.N;
    const int npairs = (s.nb + 1) / 2;
    // resident CTAs per SM: 2048 threads, and 65,536 registers at about 32 (FP32) or 64
    // (double-float) a thread
    const int per_sm = std::min(2048 / FFT_NT, 65536 / (FFT_NT * (f32 ? 32 : 64)));
    L.CB = lines_per_cta(line, 2 * s.R + 1, npairs, sm_count, per_sm);
    L.RB = lines_per_cta(line, s.N, npairs, sm_count, per_sm);
    L.col_smem = line * 2 * L.CB;   // two line buffers
    L.row_smem = line * 2 * L.RB;
    return L;
}

template <class Src, class A>
abs_status run_fft_as(abs_ctx *ctx, const Setup &s, const Src &src, float *d_fields) {
    using E = typename A::E;
    RingGeom G{s.n, s.half, s.nb, s.N, s.R};
    const FftPlan P = make_plan(s);
    FftLaunch L = fft_launch(s, ctx->sm_count);
    const int npairs = (s.nb + 1) / 2;
    const size_t wbytes = sizeof(E) * (size_t)npairs * (2 * s.R + 1) * s.N;
    E *W = (E *)workspace(ctx, "fft.rows", wbytes);
    if (!W) return fail(ctx, ABS_ERR_OOM, "FFT row workspace");
    const size_t line = sizeof(E) * (size_t)s.N;
    cudaStream_t st = ctx->stream;
    const float4 *tw = A::table(s.d_tw, s.N);
    auto cols = [&](int cb) {
        const size_t sm = line * 2 * cb;
        allow_smem(k_fft_cols<Src, A>, sm);
        k_fft_cols<Src, A><<<dim3((unsigned)cdiv(2 * s.R + 1, cb), npairs), FFT_NT, sm, st>>>(G, P, cb, s.d_q,
                                                                                             s.d_Rm, src, tw, W);
    };
    auto rows = [&](int rb) {
        const size_t sm = line * 2 * rb;
        allow_smem(k_fft_rows<A>, sm);
        k_fft_rows<A><<<dim3((unsigned)cdiv(s.N, rb), npairs), FFT_NT, sm, st>>>(G, P, rb, s.d_Rm, W, tw, d_fields);
    };
    // Autotuner: lines per CTA of each pass, measured on the configuration's first eager
    // call (the model's count and 1, 2, 4, 8 lines, each timed twice) and kept by the
    // root context per configuration and source; else the model above.
    abs_ctx *root = ctx->parent ? ctx->parent : ctx;
    const std::string key = s.key + "|fft|" + Src::tag;
    auto hit = root->fft_shapes.find(key);
    if (hit != root->fft_shapes.end()) {
        L.CB = hit->second.first;
        L.RB = hit->second.second;
    } else {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (st) cudaStreamIsCapturing(st, &cs);
        if (root->autotune && !ctx->profiling && st && cs == cudaStreamCaptureStatusNone && !s.key.empty()) {
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
                auto best_of = [&](int model, const auto &run) {
                    int best = model;
                    float tbest = 1e30f;
                    for (int w : {model, 1, 2, 4, 8}) {
                        if (line * 2 * w > 200 * 1024 || (w != model && w == best && tbest < 1e30f)) continue;
                        float tmin = 1e30f;
                        for (int rep = 0; rep < 2; ++rep) {
                            cudaEventRecord(e0, st);
                            run(w);
                            cudaEventRecord(e1, st);
                            float t = 1e30f;
                            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
                                cudaGetLastError();
                                t = 1e30f;
                            }
                            tmin = std::min(tmin, t);
                        }
                        if (tmin < tbest) {
                            tbest = tmin;
                            best = w;
                        }
                    }
                    return best;
                };
                L.CB = best_of(L.CB, cols);     // leaves W transformed (any count gives the same W)
                L.RB = best_of(L.RB, rows);
                root->fft_shapes[key] = {L.CB, L.RB};
            }
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
            cudaGetLastError();
        }
    }
    if (line * 2 * L.RB > 227 * 1024 || line * 2 * L.CB > 227 * 1024)
        return fail(ctx, ABS_ERR_UNSUPPORTED, "FFT lines do not fit shared memory");
    {
        StageTimer timer(ctx, "fft_cols");
        cols(L.CB);
    }
    {
        StageTimer timer(ctx, "fft_rows");
        rows(L.RB);
    }
    return check_launch(ctx, "filter+FFT");
}

template <class Src>
abs_status run_fft(abs_ctx *ctx, const Setup &s, const Src &src, float *d_fields) {
    if ((int)s.radices.size() > MAXRAD) return fail(ctx, ABS_ERR_UNSUPPORTED, "FFT radix plan too long");
    return plain_fp32(s) ? run_fft_as<Src, ArithF32>(ctx, s, src, d_fields)
                         : run_fft_as<Src, ArithDF>(ctx, s, src, d_fields);
}

}  // namespace

abs_status launch_filter_fft(abs_ctx *ctx, const Setup &s, const float *d_grid, const float *d_wsum,
                             const uint8_t *d_mask, float *d_fields) {
    GridF32 src{(const float2 *)d_grid, d_wsum, d_mask};
    return run_fft(ctx, s, src, d_fields);
}

abs_status launch_filter_fft_acc(abs_ctx *ctx, const Setup &s, const double *acc, float *d_fields) {
    const int64_t cells = (int64_t)s.n * s.n;
    GridF64 src{acc, acc + cells, acc + 2 * cells};
    return run_fft(ctx, s, src, d_fields);
}

abs_status launch_filter_fft_w(abs_ctx *ctx, const Setup &s, const double *acc, float *d_fields) {
    const int64_t cells = (int64_t)s.n * s.n;
    GridW64 src{acc + 2 * cells};
    return run_fft(ctx, s, src, d_fields);
}

abs_status launch_filter_fft_real(abs_ctx *ctx, const Setup &s, const double *d_c, const uint8_t *d_mask,
                                  float *d_fields) {
    GridReal src{d_c, d_mask};
    return run_fft(ctx, s, src, d_fields);
}

}  // namespace absk
