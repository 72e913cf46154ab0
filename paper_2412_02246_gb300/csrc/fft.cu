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
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "abs_internal.cuh"

namespace absk {
namespace {

constexpr int MAXRAD = 16;
constexpr int MAX_RADIX = 16;   // largest radix of a pass (composite radices up to it, see Dft)
__host__ __device__ constexpr int itw_off(int R) { return R * (R - 1) / 2; }
constexpr int ITW_N = itw_off(MAX_RADIX + 1);
constexpr int FFT_NT = 128;     // threads per transform CTA
constexpr int FFT_FIXED = 2;    // a CTA's fixed cost (barriers, first loads) in lines of work

struct FftPass {
    int R, p, T, tstep;
    uint32_t mag_p, mag_T;   // floor(x / p) = umulhi(x, mag_p) for x < 2^16
};

struct FftPlan {
    int N, nrad;
    FftPass pass[MAXRAD];
    float4 itw[2 * ITW_N];   // the composite radices' twiddles (see Dft)
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
    // w = exp(-2 pi i t / N) as a complex value (re, im) from the table, and v w
    __device__ static C tw_load(const float4 *__restrict__ tw, int t) {
        const float4 c = __ldg(tw + 2 * t), s = __ldg(tw + 2 * t + 1);
        return {f2(c.x, s.y), f2(c.z, s.w)};
    }
    // the same from a table in the kernel's parameters (plain loads)
    __device__ static C tw_param(const float4 *tw, int t) {
        const float4 c = tw[2 * t], s = tw[2 * t + 1];
        return {f2(c.x, s.y), f2(c.z, s.w)};
    }
    __device__ static C cmul(C v, C w) {
        return c_mul_tw(v, {f2(w.hi.x, w.hi.x), f2(w.lo.x, w.lo.x)}, {f2(-w.hi.y, w.hi.y), f2(-w.lo.y, w.lo.y)});
    }
    __device__ static C neg(C a) { return p_neg(a); }
    __device__ static C pi(C a) { return {f2(-a.hi.y, a.hi.x), f2(-a.lo.y, a.lo.x)}; }   // a * i
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
    __device__ static C tw_load(const float4 *__restrict__ tw, int t) {
        const float4 w = __ldg(tw + t);
        return f2(w.x, w.w);
    }
    // from the double-float layout of a parameter table: the high parts
    __device__ static C tw_param(const float4 *tw, int t) { return f2(tw[2 * t].x, tw[2 * t + 1].y); }
    __device__ static C cmul(C v, C w) { return __ffma2_rn(f2(v.y, v.x), f2(-w.y, w.y), __fmul2_rn(v, f2(w.x, w.x))); }
    __device__ static C neg(C a) { return f2(-a.x, -a.y); }
    __device__ static C pi(C a) { return f2(-a.y, a.x); }   // a * i
    // the cell value rounded once to FP32
    __device__ static E from_cell(float4 v) { return f2(__fadd_rn(v.x, v.z), __fadd_rn(v.y, v.w)); }
    __device__ static E times_i(float4 v) { return f2(-__fadd_rn(v.y, v.w), __fadd_rn(v.x, v.z)); }
    __device__ static E zero() { return f2(0.f, 0.f); }
    __device__ static float re(E v) { return v.x; }
    __device__ static float im(E v) { return v.y; }
};

// ------------------------------------------------------------------ in-register DFTs
// Dft<A, R>::run(x, itw) replaces x[0..R) by its R-point DFT, x[k] = sum_n
// x[n] exp(-2 pi i n k / R), in registers.  R = 2, 3, 4, 5 are written out;
// the composite radices up to 16 are one Cooley-Tukey step R = R1 R2 (n = R2 n1
// + n2, k = k1 + R1 k2: R2 DFTs of R1 points, the twiddles exp(-2 pi i n2 k1 /
// R), R1 DFTs of R2 points).  Their twiddles come from itw, exp(-2 pi i m / R)
// at itw_off(R) + m in the double-float layout of the N-point table (two
// float4 an entry); a twiddle that is a power of -i is a swap of parts.
template <class A, int R>
__device__ __forceinline__ typename A::C rot(typename A::C v, int m, const float4 *itw) {
    if (m == 0) return v;
    if ((4 * m) % R == 0) {
        const int qd = (4 * m / R) & 3;
        return qd == 1 ? A::mi(v) : qd == 2 ? A::neg(v) : A::pi(v);
    }
    return A::cmul(v, A::tw_param(itw, itw_off(R) + m));
}

template <class A, int R>
struct Dft;

template <class A>
struct Dft<A, 2> {
    using C = typename A::C;
    __device__ static __forceinline__ void run(C *x, const float4 *) {
        const C t = x[0];
        x[0] = A::add(t, x[1]);
        x[1] = A::sub(t, x[1]);
    }
};

template <class A>
struct Dft<A, 3> {
    using C = typename A::C;
    __device__ static __forceinline__ void run(C *x, const float4 *) {
        const C t = A::add(x[1], x[2]);
        const C m = A::sub(x[0], A::half(t));
        const C d = A::mul(A::mi(A::sub(x[1], x[2])), A::cst(kS3));
        x[0] = A::add(x[0], t);
        x[1] = A::add(m, d);
        x[2] = A::sub(m, d);
    }
};

template <class A>
struct Dft<A, 4> {
    using C = typename A::C;
    __device__ static __forceinline__ void run(C *x, const float4 *) {
        const C a0 = A::add(x[0], x[2]), a1 = A::sub(x[0], x[2]);
        const C b0 = A::add(x[1], x[3]), b1 = A::mi(A::sub(x[1], x[3]));
        x[0] = A::add(a0, b0);
        x[1] = A::add(a1, b1);
        x[2] = A::sub(a0, b0);
        x[3] = A::sub(a1, b1);
    }
};

template <class A>
struct Dft<A, 5> {
    using C = typename A::C;
    __device__ static __forceinline__ void run(C *x, const float4 *) {
        const C c1 = A::cst(kC1), c2 = A::cst(kC2), s1 = A::cst(kS1), s2 = A::cst(kS2);
        const C t1 = A::add(x[1], x[4]), t2 = A::add(x[2], x[3]);
        const C t3 = A::sub(x[1], x[4]), t4 = A::sub(x[2], x[3]);
        const C a1 = A::add(x[0], A::add(A::mul(t1, c1), A::mul(t2, c2)));
        const C a2 = A::add(x[0], A::add(A::mul(t1, c2), A::mul(t2, c1)));
        const C b1 = A::mi(A::add(A::mul(t3, s1), A::mul(t4, s2)));
        const C b2 = A::mi(A::sub(A::mul(t3, s2), A::mul(t4, s1)));
        x[0] = A::add(x[0], A::add(t1, t2));
        x[1] = A::add(a1, b1);
        x[4] = A::sub(a1, b1);
        x[2] = A::add(a2, b2);
        x[3] = A::sub(a2, b2);
    }
};

template <class A, int R1, int R2>
struct DftCT {
    using C = typename A::C;
    __device__ static __forceinline__ void run(C *x, const float4 *itw) {
        constexpr int R = R1 * R2;
        C y[R];
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) {
            C t[R1];
#pragma unroll
            for (int n1 = 0; n1 < R1; ++n1) t[n1] = x[R2 * n1 + n2];
            Dft<A, R1>::run(t, itw);
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1) y[n2 * R1 + k1] = rot<A, R>(t[k1], n2 * k1, itw);
        }
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) {
            C u[R2];
#pragma unroll
            for (int n2 = 0; n2 < R2; ++n2) u[n2] = y[n2 * R1 + k1];
            Dft<A, R2>::run(u, itw);
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) x[k1 + R1 * k2] = u[k2];
        }
    }
};
template <class A> struct Dft<A, 6> : DftCT<A, 2, 3> {};
template <class A> struct Dft<A, 8> : DftCT<A, 2, 4> {};
template <class A> struct Dft<A, 9> : DftCT<A, 3, 3> {};
template <class A> struct Dft<A, 10> : DftCT<A, 2, 5> {};
template <class A> struct Dft<A, 12> : DftCT<A, 3, 4> {};
template <class A> struct Dft<A, 15> : DftCT<A, 3, 5> {};
template <class A> struct Dft<A, 16> : DftCT<A, 4, 4> {};

// x[q] *= w^q for q = 1 .. R-1, the powers of w by repeated halving of the exponent
// (w^q = w^(q/2) w^(q - q/2)): one table load a butterfly, at most log2(R) products
// deep.
template <class A, int R>
__device__ __forceinline__ void apply_powers(typename A::C *x, typename A::C w) {
    using C = typename A::C;
    C pw[R];
    pw[1] = w;
#pragma unroll
    for (int q = 2; q < R; ++q) pw[q] = A::cmul(pw[q / 2], pw[q - q / 2]);
#pragma unroll
    for (int q = 1; q < R; ++q) x[q] = A::cmul(x[q], pw[q]);
}

// The butterfly of one Stockham pass (span p = P.p, radix R): inputs x[i + q T],
// twiddles exp(-2 pi i q (i mod p) / (p R)), outputs at (i div p) p R + (i mod p) + s p.
template <class A, int R>
__device__ __forceinline__ void stockham_bfly(const typename A::E *__restrict__ in, typename A::E *__restrict__ out,
                                              const FftPass &P, int i, const float4 *__restrict__ tw,
                                              const float4 *itw) {
    using C = typename A::C;
    const int p = P.p, T = P.T;
    const int ip = p == 1 ? i : (int)__umulhi((uint32_t)i, P.mag_p);
    const int k = i - ip * p;
    C x[R];
#pragma unroll
    for (int q = 0; q < R; ++q) x[q] = A::ld(in[i + q * T]);
    if (k) apply_powers<A, R>(x, A::tw_load(tw, k * P.tstep));
    Dft<A, R>::run(x, itw);
    typename A::E *dst = out + ip * p * R + k;
#pragma unroll
    for (int s = 0; s < R; ++s) dst[s * p] = A::st(x[s]);
}

template <class A, int R>
__device__ __forceinline__ void stockham_lines(const typename A::E *__restrict__ in, typename A::E *__restrict__ out,
                                               int N, const FftPass &P, int lines, const float4 *__restrict__ tw,
                                               const float4 *itw) {
    const int T = P.T, nbf = lines * T;
    for (int b = threadIdx.x; b < nbf; b += blockDim.x) {
        const int l = (int)__umulhi((uint32_t)b, P.mag_T);
        stockham_bfly<A, R>(in + (size_t)l * N, out + (size_t)l * N, P, b - l * T, tw, itw);
    }
}

// One Stockham pass over `lines` transforms of length N stored line-major.
template <class A>
__device__ __forceinline__ void stockham_pass(const typename A::E *__restrict__ in, typename A::E *__restrict__ out,
                                              int N, const FftPass &P, int lines,
                                              const float4 *__restrict__ tw, const float4 *itw) {
    switch (P.R) {
        case 2: stockham_lines<A, 2>(in, out, N, P, lines, tw, itw); break;
        case 3: stockham_lines<A, 3>(in, out, N, P, lines, tw, itw); break;
        case 4: stockham_lines<A, 4>(in, out, N, P, lines, tw, itw); break;
        case 5: stockham_lines<A, 5>(in, out, N, P, lines, tw, itw); break;
        case 6: stockham_lines<A, 6>(in, out, N, P, lines, tw, itw); break;
        case 8: stockham_lines<A, 8>(in, out, N, P, lines, tw, itw); break;
        case 9: stockham_lines<A, 9>(in, out, N, P, lines, tw, itw); break;
        case 10: stockham_lines<A, 10>(in, out, N, P, lines, tw, itw); break;
        case 12: stockham_lines<A, 12>(in, out, N, P, lines, tw, itw); break;
        case 15: stockham_lines<A, 15>(in, out, N, P, lines, tw, itw); break;
        default: stockham_lines<A, 16>(in, out, N, P, lines, tw, itw); break;
    }
}

// Transforms `lines` lines in buffer a (scratch b); returns the buffer holding the result.
template <class A>
__device__ typename A::E *fft_lines(typename A::E *a, typename A::E *b, int lines, const FftPlan &P,
                                    const float4 *__restrict__ tw) {
    for (int s = 0; s < P.nrad; ++s) {
        __syncthreads();
        stockham_pass<A>(a, b, P.N, P.pass[s], lines, tw, P.itw);
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
// cell, N_g from the third accumulator plane mirrored in FP64 (real: N_g =
// N_-g; the estimate's literal form accumulates the count of visibilities
// there), the quotient in double-float.
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

// The noise-optimised weighting: N_eff = (sum w)^2 / sum w^2 from the mirrored
// FP64 sums (the weight sums w and squared-weight sums w2 before the mirror).
// D fields: N_eff X_g = V_g (sum w) / (sum w^2); I fields: N_eff.
struct GridNoise64 {
    static constexpr const char *tag = "noise";
    const double *re, *im, *w, *w2;
    __device__ bool value(int64_t cell, int64_t mcell, float4 &x) const {
        const double ww = w[cell] + w[mcell];
        if (!(ww > 0.0)) return false;
        const double f = ww / (w2[cell] + w2[mcell]);
        float rh, rl, ih, il;
        df_of((re[cell] + re[mcell]) * f, rh, rl);
        df_of((im[cell] - im[mcell]) * f, ih, il);
        x = make_float4(rh, ih, rl, il);
        return true;
    }
};
struct GridNeff64 {
    static constexpr const char *tag = "neff";
    const double *w, *w2;
    __device__ bool value(int64_t cell, int64_t mcell, float4 &x) const {
        const double ww = w[cell] + w[mcell];
        if (!(ww > 0.0)) return false;
        float h, l;
        df_of(ww * ww / (w2[cell] + w2[mcell]), h, l);
        x = make_float4(h, 0.f, l, 0.f);
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
__global__ void __launch_bounds__(FFT_NT) k_fft_cols(RingGeom G, const __grid_constant__ FftPlan P, int CB, const int64_t *__restrict__ q,
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
// along x.  The first Stockham pass reads its inputs straight from the column
// pass's output (zero outside |x| <= R of the pair; consecutive threads take
// consecutive rows of one column, which are adjacent there), the middle passes
// go between two shared-memory line buffers (line pitch LS), and the last pass
// writes each output row of both fields to global memory, consecutive threads
// consecutive pixels.  Rounding aside, the same transform as fft_lines.
// Where the row pass puts the fields of a ring pair (a, b; b = -1 for none).
// FieldsOut: the fields [nb][N][N] FP32, written by the last pass itself.
// PlanesOut: the split-BF16 kernel's three chunk-blocked planes (see SplitOut),
// each value split once into hi = bf16(v) and lo = bf16(v - hi) beside its FP32
// copy; the last pass leaves its rows in shared memory (staged) and the CTA then
// stores whole 16-byte units: 8 pixels of hi, of lo, two units of FP32.
struct FieldsOut {
    static constexpr bool staged = false;
    float *fields;
    __device__ void put(const RingGeom &G, int a, int b, size_t pix, float re, float im) const {
        const size_t P2 = (size_t)G.N * G.N;
        fields[(size_t)a * P2 + pix] = re;
        if (b >= 0) fields[(size_t)b * P2 + pix] = im;
    }
};

struct PlanesOut {
    static constexpr bool staged = true;
    SplitOut o;
    __device__ void put1(int m, size_t pix, float v) const {
        const int u = (int)(pix & 63), key = m & 7;
        const size_t row = ((pix >> 6) * (size_t)o.nbp + m) * 64;
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        const __nv_bfloat16 l = __float2bfloat16_rn(__fsub_rn(v, __bfloat162float(h)));   // exact in FP32
        const size_t ob = row + (size_t)((((u >> 3) ^ key) << 3) | (u & 7));   // 8 BF16 a 16-byte unit
        const size_t of = row + (size_t)((((u >> 2) ^ key) << 2) | (u & 3));   // 4 FP32 a 16-byte unit
        ((__nv_bfloat16 *)o.hi)[ob] = h;
        ((__nv_bfloat16 *)o.lo)[ob] = l;
        o.f32[of] = v;
    }
    __device__ void put(const RingGeom &, int a, int b, size_t pix, float re, float im) const {
        put1(a, pix, re);
        if (b >= 0) put1(b, pix, im);
    }
    // 8 pixels from pix0 (a multiple of 8, inside one 64-pixel chunk) of ring m
    __device__ void put8(int m, size_t pix0, const float *v) const {
        const int unit = (int)((pix0 & 63) >> 3), key = m & 7;
        const size_t row = ((pix0 >> 6) * (size_t)o.nbp + m) * 64;
        uint32_t h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const __nv_bfloat162 hh = __float22bfloat162_rn(make_float2(v[2 * e], v[2 * e + 1]));
            const float2 hf = __bfloat1622float2(hh);
            const __nv_bfloat162 ll =
                __float22bfloat162_rn(make_float2(__fsub_rn(v[2 * e], hf.x), __fsub_rn(v[2 * e + 1], hf.y)));
            h[e] = *(const uint32_t *)&hh;
            l[e] = *(const uint32_t *)&ll;
        }
        const size_t ob = row + (size_t)((unit ^ key) << 3);
        *(uint4 *)((__nv_bfloat16 *)o.hi + ob) = make_uint4(h[0], h[1], h[2], h[3]);
        *(uint4 *)((__nv_bfloat16 *)o.lo + ob) = make_uint4(l[0], l[1], l[2], l[3]);
        *(float4 *)(o.f32 + row + (size_t)(((2 * unit) ^ key) << 2)) = make_float4(v[0], v[1], v[2], v[3]);
        *(float4 *)(o.f32 + row + (size_t)(((2 * unit + 1) ^ key) << 2)) = make_float4(v[4], v[5], v[6], v[7]);
    }
    // The CTA's rows py0 .. py0 + rb - 1 (res: line r at r LS, complex (D_a, D_b)):
    // the whole 8-pixel groups inside the block vectorised, the ragged ends one by one.
    template <class A>
    __device__ void store_block(const RingGeom &G, int a, int b, const typename A::E *res, int LS, int py0,
                                int rb) const {
        const size_t P0 = (size_t)py0 * G.N, P1 = P0 + (size_t)rb * G.N;
        const size_t g0 = (P0 + 7) / 8, g1 = P1 / 8;
        for (size_t gi = g0 + threadIdx.x; gi < g1; gi += blockDim.x) {
            const size_t pix0 = gi * 8;
            int local = (int)(pix0 - P0);
            int r = local / G.N, n = local - r * G.N;
            float va[8], vb[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const typename A::E v = res[(size_t)r * LS + n];
                va[e] = A::re(v);
                vb[e] = A::im(v);
                if (++n == G.N) {
                    n = 0;
                    ++r;
                }
            }
            put8(a, pix0, va);
            if (b >= 0) put8(b, pix0, vb);
        }
        // pixels of a group shared with the neighbouring block
        const size_t e0 = g0 * 8 > P1 ? P1 : g0 * 8, e1 = g1 * 8 < e0 ? e0 : g1 * 8;
        for (size_t pix = P0 + threadIdx.x; pix < e0; pix += blockDim.x) {
            const int local = (int)(pix - P0), r = local / G.N;
            const typename A::E v = res[(size_t)r * LS + (local - r * G.N)];
            put(G, a, b, pix, A::re(v), A::im(v));
        }
        for (size_t pix = e1 + threadIdx.x; pix < P1; pix += blockDim.x) {
            const int local = (int)(pix - P0), r = local / G.N;
            const typename A::E v = res[(size_t)r * LS + (local - r * G.N)];
            put(G, a, b, pix, A::re(v), A::im(v));
        }
    }
};

template <class A>
struct RowNT {
    static constexpr int value = sizeof(typename A::E) == 8 ? 256 : 128;
    static constexpr int min_blocks = sizeof(typename A::E) == 8 ? 3 : 1;   // resident CTAs an SM
};

template <class A, int R, class Out>
__device__ __forceinline__ void row_pass(const RingGeom &G, const FftPlan &P, const FftPass &ps, bool first, bool last,
                                         int RB, int rb, uint32_t mag_rb, int LS, int Rp, int py0,
                                         const typename A::E *__restrict__ src, const typename A::E *in,
                                         typename A::E *out, const float4 *__restrict__ tw, const Out &dst_out,
                                         int ring_a, int ring_b) {
    using C = typename A::C;
    using E = typename A::E;
    const int N = G.N, T = ps.T, p = ps.p, nbf = (first ? RB : rb) * T;
    for (int b = threadIdx.x; b < nbf; b += blockDim.x) {
        int r, i;
        C x[R];
        if (first) {   // p = 1: no twiddles; RB rows a column, the tail block's missing ones idle
            i = RB == 1 ? b : (int)__umulhi((uint32_t)b, mag_rb);
            r = b - i * RB;
            if (r >= rb) continue;
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int n = i + q * T;
                const int xc = n <= N / 2 ? n : n - N;
                x[q] = (xc >= -Rp && xc <= Rp) ? A::ld(src[(size_t)(xc + G.Rmax) * N + py0 + r]) : A::ld(A::zero());
            }
        } else {
            r = (int)__umulhi((uint32_t)b, ps.mag_T);
            i = b - r * T;
            const E *l = in + (size_t)r * LS;
#pragma unroll
            for (int q = 0; q < R; ++q) x[q] = A::ld(l[i + q * T]);
            const int ip = p == 1 ? i : (int)__umulhi((uint32_t)i, ps.mag_p);
            const int k = i - ip * p;
            if (k) apply_powers<A, R>(x, A::tw_load(tw, k * ps.tstep));
        }
        Dft<A, R>::run(x, P.itw);
        if (last) {   // p R = N: the outputs are pixels i + s p of row py0 + r
            const size_t row = (size_t)(py0 + r) * N;
#pragma unroll
            for (int s = 0; s < R; ++s) {
                const E e = A::st(x[s]);
                dst_out.put(G, ring_a, ring_b, row + i + s * p, A::re(e), A::im(e));
            }
        } else {
            const int ip = p == 1 ? i : (int)__umulhi((uint32_t)i, ps.mag_p);
            E *dst = out + (size_t)r * LS + ip * p * R + (i - ip * p);
#pragma unroll
            for (int s = 0; s < R; ++s) dst[s * p] = A::st(x[s]);
        }
    }
}

template <class A, class Out>
__global__ void __launch_bounds__(RowNT<A>::value, RowNT<A>::min_blocks)
    k_fft_rows(RingGeom G, const __grid_constant__ FftPlan P, int RB, uint32_t mag_rb, int LS,
               const int32_t *__restrict__ Rm, const typename A::E *__restrict__ W, const float4 *__restrict__ tw,
               const Out dst_out) {
    using E = typename A::E;
    extern __shared__ float4 sbuf[];
    const int pair = blockIdx.y;
    const int a = 2 * pair, b = a + 1 < G.nb ? a + 1 : -1;
    const int Rp = max(Rm[a], b >= 0 ? Rm[b] : -1);
    const int py0 = blockIdx.x * RB;
    const int rb = min(RB, G.N - py0);
    if (Rp < 0) {  // both rings empty: zero fields
        const size_t o = (size_t)py0 * G.N;
        for (int i = threadIdx.x; i < rb * G.N; i += blockDim.x) dst_out.put(G, a, b, o + i, 0.f, 0.f);
        return;
    }
    E *const buf0 = (E *)sbuf;
    const size_t bstride = (size_t)RB * LS;
    const E *src = W + (size_t)pair * (2 * G.Rmax + 1) * G.N;
    for (int s = 0; s < P.nrad; ++s) {
        if (s) __syncthreads();
        const FftPass &ps = P.pass[s];
        const bool first = s == 0, last = s == P.nrad - 1 && !Out::staged;
        const E *in = buf0 + ((s + 1) & 1) * bstride;   // what pass s - 1 wrote
        E *out = buf0 + (s & 1) * bstride;
        switch (ps.R) {
#define ABS_ROW_CASE(RR) \
    case RR: row_pass<A, RR>(G, P, ps, first, last, RB, rb, mag_rb, LS, Rp, py0, src, in, out, tw, dst_out, a, b); break;
            ABS_ROW_CASE(2) ABS_ROW_CASE(3) ABS_ROW_CASE(4) ABS_ROW_CASE(5) ABS_ROW_CASE(6) ABS_ROW_CASE(8)
            ABS_ROW_CASE(9) ABS_ROW_CASE(10) ABS_ROW_CASE(12) ABS_ROW_CASE(15)
            default: row_pass<A, 16>(G, P, ps, first, last, RB, rb, mag_rb, LS, Rp, py0, src, in, out, tw, dst_out, a, b);
                break;
#undef ABS_ROW_CASE
        }
    }
    if constexpr (Out::staged) {
        __syncthreads();
        dst_out.template store_block<A>(G, a, b, buf0 + ((P.nrad - 1) & 1) * bstride, LS, py0, rb);
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
    // exp(-2 pi i m / R) for the composite radices, in the double-float layout of Setup::d_tw
    std::memset(P.itw, 0, sizeof P.itw);
    for (int R = 6; R <= MAX_RADIX; ++R)
        for (int m = 1; m < R; ++m) {
            const double a = 2.0 * M_PI * (double)m / (double)R;
            const double c = std::cos(a), sn = -std::sin(a);
            const float ch = (float)c, sh = (float)sn;
            const float cl = (float)(c - (double)ch), sl = (float)(sn - (double)sh);
            P.itw[2 * (itw_off(R) + m)] = make_float4(ch, ch, cl, cl);
            P.itw[2 * (itw_off(R) + m) + 1] = make_float4(-sh, sh, -sl, sl);
        }
    return P;
}

struct FftLaunch {
    int CB, RB;   // columns per CTA of the column pass, rows per CTA of the row pass
    size_t col_smem;
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

// Line pitch of the row pass's buffers: N plus the pad (0 to 15 elements) that
// spreads the first pass's stores (consecutive threads in consecutive lines, at
// i R0 in line i mod RB) over the most shared-memory banks: per 128-byte phase
// of a warp's store, the largest count of distinct words one bank must serve.
static int row_pitch(int N, int R0, int RB, size_t esize) {
    const int words = (int)(esize / 4), per_phase = 32 / words;
    int best = N, best_cost = INT32_MAX;
    for (int pad = 0; pad < 16; ++pad) {
        const int LS = N + pad;
        int cost = 0;
        for (int ph = 0; ph < 32; ph += per_phase) {
            std::vector<std::vector<int>> bank(32);
            for (int t = ph; t < ph + per_phase; ++t) {
                const int i = t / RB, r = t - i * RB;
                const int w0 = (r * LS + i * R0) * words;
                for (int w = 0; w < words; ++w) {
                    auto &v = bank[(w0 + w) & 31];
                    if (std::find(v.begin(), v.end(), w0 + w) == v.end()) v.push_back(w0 + w);
                }
            }
            size_t worst = 0;
            for (const auto &v : bank) worst = std::max(worst, v.size());
            cost += (int)worst;
        }
        if (cost < best_cost) {
            best_cost = cost;
            best = LS;
        }
    }
    return best;
}

// Shared memory of a row-pass CTA: line buffers of RB lines at pitch LS, one a
// pass that writes to shared memory (all but the last, which writes there too
// when its output is staged), two at most.
static size_t row_smem(const Setup &s, int RB, int LS, size_t esize, bool staged) {
    const int to_smem = (int)s.radices.size() - (staged ? 0 : 1);
    return (size_t)std::min(std::max(to_smem, 0), 2) * RB * LS * esize;
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
    L.RB = 2;   // the row pass: two rows a CTA (the autotuner tries 1 to 8)
    L.col_smem = line * 2 * L.CB;   // two line buffers
    return L;
}

template <class Src, class A>
abs_status run_fft_as(abs_ctx *ctx, const Setup &s, const Src &src, float *d_fields, const SplitOut *split) {
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
    auto rows_to = [&](int rb, const auto &out) {
        using Out = std::decay_t<decltype(out)>;
        const int LS = row_pitch(s.N, s.radices.empty() ? 1 : s.radices[0], rb, sizeof(E));
        const size_t sm = row_smem(s, rb, LS, sizeof(E), Out::staged);
        allow_smem(k_fft_rows<A, Out>, sm);
        k_fft_rows<A, Out><<<dim3((unsigned)cdiv(s.N, rb), npairs), RowNT<A>::value, sm, st>>>(
            G, P, rb, magic(rb), LS, s.d_Rm, W, tw, out);
    };
    auto rows = [&](int rb) {
        if constexpr (std::is_same<A, ArithF32>::value) {
            if (split) {
                rows_to(rb, PlanesOut{*split});
                return;
            }
        }
        rows_to(rb, FieldsOut{d_fields});
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
                        if (line * 2 * w > 200 * 1024 || w > s.N || (w != model && w == best && tbest < 1e30f))
                            continue;
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
    const size_t rsm = row_smem(s, L.RB, row_pitch(s.N, s.radices.empty() ? 1 : s.radices[0], L.RB, sizeof(E)),
                                sizeof(E), split != nullptr);
    if (rsm > 227 * 1024 || line * 2 * L.CB > 227 * 1024)
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

// Multi-frequency form: the ring transforms of the delay modes.  Pair p = m (t_max + 1) + t
// (ring m, delay t >= 0) transforms Z(g) = Xt(g, t) on the cells of ring m (Xt is zero on
// cells not filled in every channel), read from the region [t][(2 Rr + 1)^2] of cells
// |gx|, |gy| <= Rr as packed double-float complex values.  The channel maps are real, so
// Xt(-g, -t) = conj Xt(g, t): H1 = (Xt(., t) + Xt(., -t)) / 2 and H2 = (Xt(., t) -
// Xt(., -t)) / 2i are Hermitian on the ring and Z = H1 + i H2.  The row pass therefore
// gives the real fields F1 = FFT(H1) and F2 = FFT(H2) of the pair in its slots 2p and
// 2p + 1, and the transforms of Xt(., +-t) are F1 +- i F2.  Same W layout as k_fft_cols.
template <class A>
__global__ void __launch_bounds__(FFT_NT) k_fft_cols_delay(RingGeom G, const __grid_constant__ FftPlan P, int CB,
                                                        const int64_t *__restrict__ q, const int32_t *__restrict__ Rm,
                                                        int t1, int Rr, const float4 *__restrict__ Xt,
                                                        const float4 *__restrict__ tw, typename A::E *__restrict__ W) {
    using E = typename A::E;
    extern __shared__ float4 sbuf[];
    const int pair = blockIdx.y;
    const int m = pair / t1, t = pair - m * t1;
    const int Rp = Rm[m];
    const int x0 = (int)blockIdx.x * CB - G.Rmax;
    if (Rp < 0 || x0 > Rp || x0 + CB - 1 < -Rp) return;
    E *l0 = (E *)sbuf, *l1 = l0 + (size_t)CB * G.N;
    for (int i = threadIdx.x; i < CB * G.N; i += blockDim.x) l0[i] = A::zero();
    __syncthreads();
    const int span = 2 * Rp + 1, side = 2 * Rr + 1;
    const int64_t q0 = q[m], q1 = q[m + 1];
    const float4 *src = Xt + (size_t)t * side * side;
    for (int e = threadIdx.x; e < CB * span; e += blockDim.x) {
        const int yy = e / CB, c = e - yy * CB, x = x0 + c, y = yy - Rp;
        if (x < -Rp || x > Rp) continue;
        const int64_t r2 = (int64_t)x * x + (int64_t)y * y;
        if (r2 < q0 || r2 >= q1) continue;
        l0[(size_t)c * G.N + (y < 0 ? y + G.N : y)] = A::from_cell(src[(size_t)(y + Rr) * side + (x + Rr)]);
    }
    E *res = fft_lines<A>(l0, l1, CB, P, tw);
    for (int e = threadIdx.x; e < CB * G.N; e += blockDim.x) {
        const int c = e / G.N, x = x0 + c;
        if (x < -Rp || x > Rp) continue;
        W[((size_t)pair * (2 * G.Rmax + 1) + (x + G.Rmax)) * G.N + (e - c * G.N)] = res[e];
    }
}

template <class A>
abs_status run_fft_delay(abs_ctx *ctx, const Setup &s, int t_max, const float4 *d_xt, const int32_t *d_rm2,
                         float *d_F) {
    using E = typename A::E;
    const int t1 = t_max + 1;
    const int npairs = s.nb * t1;
    if (npairs > 65535) return fail(ctx, ABS_ERR_UNSUPPORTED, "delay transforms: rings x delays above 65535");
    RingGeom G{s.n, s.half, 2 * npairs, s.N, s.R};
    const FftPlan P = make_plan(s);
    const size_t line = sizeof(E) * (size_t)s.N;
    // lines per CTA of the column pass: the model of fft_launch for this many pairs
    const int per_sm = std::min(2048 / FFT_NT, 65536 / (FFT_NT * (sizeof(E) == 8 ? 32 : 64)));
    const int CB = lines_per_cta(line, 2 * s.R + 1, npairs, ctx->sm_count, per_sm);
    const int RB = 2;
    const int LS = row_pitch(s.N, s.radices.empty() ? 1 : s.radices[0], RB, sizeof(E));
    const size_t csm = line * 2 * CB, rsm = row_smem(s, RB, LS, sizeof(E), false);
    if (csm > 227 * 1024 || rsm > 227 * 1024) return fail(ctx, ABS_ERR_UNSUPPORTED, "FFT lines do not fit shared memory");
    E *W = (E *)workspace(ctx, "fft.delay", sizeof(E) * (size_t)npairs * (2 * s.R + 1) * s.N);
    if (!W) return fail(ctx, ABS_ERR_OOM, "delay transform workspace");
    cudaStream_t st = ctx->stream;
    const float4 *tw = A::table(s.d_tw, s.N);
    {
        StageTimer timer(ctx, "fft_cols_delay");
        allow_smem(k_fft_cols_delay<A>, csm);
        k_fft_cols_delay<A><<<dim3((unsigned)cdiv(2 * s.R + 1, CB), npairs), FFT_NT, csm, st>>>(
            G, P, CB, s.d_q, s.d_Rm, t1, s.R, d_xt, tw, W);
    }
    {
        StageTimer timer(ctx, "fft_rows_delay");
        allow_smem(k_fft_rows<A, FieldsOut>, rsm);
        k_fft_rows<A, FieldsOut><<<dim3((unsigned)cdiv(s.N, RB), npairs), RowNT<A>::value, rsm, st>>>(
            G, P, RB, magic(RB), LS, d_rm2, W, tw, FieldsOut{d_F});
    }
    return check_launch(ctx, "delay transforms");
}

template <class Src>
abs_status run_fft(abs_ctx *ctx, const Setup &s, const Src &src, float *d_fields, const SplitOut *split = nullptr) {
    if ((int)s.radices.size() > MAXRAD) return fail(ctx, ABS_ERR_UNSUPPORTED, "FFT radix plan too long");
    if (split && !plain_fp32(s)) return fail(ctx, ABS_ERR_INVALID_ARG, "split planes need the split-BF16 precision");
    return plain_fp32(s) ? run_fft_as<Src, ArithF32>(ctx, s, src, d_fields, split)
                         : run_fft_as<Src, ArithDF>(ctx, s, src, d_fields, split);
}

}  // namespace

abs_status launch_filter_fft(abs_ctx *ctx, const Setup &s, const float *d_grid, const float *d_wsum,
                             const uint8_t *d_mask, float *d_fields) {
    GridF32 src{(const float2 *)d_grid, d_wsum, d_mask};
    return run_fft(ctx, s, src, d_fields);
}

abs_status launch_filter_fft_acc(abs_ctx *ctx, const Setup &s, const double *acc, float *d_fields,
                                 const SplitOut *split) {
    const int64_t cells = (int64_t)s.n * s.n;
    if (s.weight_mode == ABS_W_NOISE) {
        GridNoise64 src{acc, acc + cells, acc + 2 * cells, acc + 3 * cells};
        return run_fft(ctx, s, src, d_fields, split);
    }
    GridF64 src{acc, acc + cells, acc + 2 * cells};   // the literal form holds N_g in plane 2
    return run_fft(ctx, s, src, d_fields, split);
}

abs_status launch_filter_fft_w(abs_ctx *ctx, const Setup &s, const double *acc, float *d_fields) {
    const int64_t cells = (int64_t)s.n * s.n;
    if (s.weight_mode == ABS_W_NOISE) {
        GridNeff64 src{acc + 2 * cells, acc + 3 * cells};
        return run_fft(ctx, s, src, d_fields);
    }
    GridW64 src{acc + 2 * cells};
    return run_fft(ctx, s, src, d_fields);
}

abs_status launch_filter_fft_real(abs_ctx *ctx, const Setup &s, const double *d_c, const uint8_t *d_mask,
                                  float *d_fields) {
    GridReal src{d_c, d_mask};
    return run_fft(ctx, s, src, d_fields);
}

abs_status launch_filter_fft_delay(abs_ctx *ctx, const Setup &s, int t_max, const float4 *d_xt, const int32_t *d_rm2,
                                   float *d_F) {
    if ((int)s.radices.size() > MAXRAD) return fail(ctx, ABS_ERR_UNSUPPORTED, "FFT radix plan too long");
    return plain_fp32(s) ? run_fft_delay<ArithF32>(ctx, s, t_max, d_xt, d_rm2, d_F)
                         : run_fft_delay<ArithDF>(ctx, s, t_max, d_xt, d_rm2, d_F);
}

}  // namespace absk
