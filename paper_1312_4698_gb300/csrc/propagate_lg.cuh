// Lane-group propagation kernel (Sec. III.A / III.B of arXiv:1312.4698).
//
// A group of G lanes (G = 8, 16 or 32, 2F <= G) owns one trajectory; a warp
// holds T = 32/G trajectories.  Steps are processed in chunks of C (C = G, or
// 16 / 8 steps for the one-trajectory-per-warp groups at F = 9 / F > 9), and
// work is split by what parallelises:
//
//   phase 1 (per step, group-parallel, arithmetic type Real):
//     lane g < 2F owns column g of the monodromy matrix M (its p- and q-rows
//     in registers); lane a < F owns mode a: p_a, q_a (FP64) and the
//     separable diagonal of the potential.  The Hessian's packed coupling
//     entries e(a,b) are spread over the group, reading the coupling tensors
//     staged in shared memory.  det M is Gaussian elimination of M^T across the
//     group (pivot column by warp reduction, pivot entries by shuffle).  The
//     Herman-Kluk matrix A of the step goes to shared memory.
//   phase 2 (once per chunk, job-parallel): lane j < T*C takes job j =
//     (trajectory j / C, step j % C) and computes det A and its argument by an
//     LU in place in shared memory (FP64 path in FP64; mixed path in FP32, the
//     entries being FP32 already).
//   phase 3: the continuous phase, a segmented prefix sum over each group.
//   phase 4 (job-parallel): overlap <chi|p q>, action, phase and the amplitude;
//     each group writes C consecutive samples of its row.
//
// Real = float is the mixed-precision path: monodromy, potential, det M, A,
// the elimination that gives det A, the overlap and each step's action
// increment in FP32; positions, momenta, the accumulated action and the
// continuous phase in FP64; the amplitude's phase is reduced modulo 2 pi in FP64
// and its sine, cosine and magnitude are evaluated in FP32.  Real = double is the
// same schedule in FP64 throughout.
//
// On GB300 a warp-wide FP64 instruction holds a sub-partition's FP64 pipe for
// about 64 cycles, so in the mixed path phase 1 keeps FP64 to the state updates
// (one FMA per drift and per kick in the mode lanes) and one FP64 add per step.
#pragma once

#include <math_constants.h>
#include <cstddef>
#include <algorithm>
#include <utility>
#include <type_traits>

#include "scivr_internal.cuh"

namespace scivr {
namespace lg {

constexpr unsigned FULL = 0xffffffffu;

template <int F>
__host__ __device__ constexpr int pidx(int a, int b)
{
    return a * F - a * (a - 1) / 2 + (b - a);
}

template <typename Real> __device__ __forceinline__ Real rexp(Real x);
template <> __device__ __forceinline__ float rexp<float>(float x) { return expf(x); }
template <> __device__ __forceinline__ double rexp<double>(double x) { return exp(x); }

// 1/x in FP64 from the FP32 reciprocal refined by two Newton steps
// (e_{k+1} = e_k^2: 2^-23 -> 2^-46 -> below FP64 rounding); FP64 division
// outside the FP32 exponent range.
__device__ __forceinline__ double recip64(double x)
{
    const double ax = fabs(x);
    if (!(ax > 1e-30 && ax < 1e30)) return 1.0 / x;
    double r = (double)__frcp_rn((float)x);
    r = r * fma(-x, r, 2.0);
    r = r * fma(-x, r, 2.0);
    return r;
}


// Compile-time loop: f(std::integral_constant<int, k>) for k = 0..N-1, every index a
// constant (the unroller would leave long loops rolled, indexing register arrays).
template <typename Fn, int... Ks>
__device__ __forceinline__ void static_for_impl(Fn &&f, std::integer_sequence<int, Ks...>)
{
    (f(std::integral_constant<int, Ks>{}), ...);
}
template <int N, typename Fn>
__device__ __forceinline__ void static_for(Fn &&f)
{
    static_for_impl(f, std::make_integer_sequence<int, N>{});
}

template <typename Real> struct Vec2;
template <> struct Vec2<float> { using T = float2; };
template <> struct Vec2<double> { using T = double2; };

// Storage of one entry of the Herman-Kluk matrix A during its elimination: FP64
// path a double2 (re, im); mixed path a double-FP32 complex (re.hi, im.hi, re.lo,
// im.lo) -- the entries are formed in FP32 and eliminated to FP64-class accuracy, the
// real and imaginary words side by side for packed FP32 arithmetic.
template <typename Real> struct AEntry;
template <> struct AEntry<float> { using T = float4; };
template <> struct AEntry<double> { using T = double2; };

// ---- double-FP32 arithmetic (hi + lo, |lo| <= ulp(hi)/2): error-free sum and
// product of two floats (Knuth's TwoSum, the FMA form of Dekker's TwoProduct) and
// the compositions the elimination needs.  Accuracy about 2^-46 relative per
// operation, on the FP32 pipe.
struct ff { float hi, lo; };

__device__ __forceinline__ void ff_two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ ff ff_norm(float hi, float lo)    // |lo| well below |hi| or hi == 0
{
    ff r;
    r.hi = hi + lo;
    r.lo = lo - (r.hi - hi);
    return r;
}

__device__ __forceinline__ ff ff_mul(ff x, ff y)
{
    const float p = x.hi * y.hi;
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    return ff_norm(p, e);
}

__device__ __forceinline__ ff ff_add(ff x, ff y)
{
    float s, e;
    ff_two_sum(x.hi, y.hi, s, e);
    return ff_norm(s, e + (x.lo + y.lo));
}

// a - x u + y v for double-FP32 a, x, u, y, v (one real part of a complex
// multiply-subtract): both products exact to their double-FP32 width, both sums
// error-free in their leading words.
__device__ __forceinline__ ff ff_sub_mul_add_mul(ff a, ff x, ff u, ff y, ff v)
{
    const float p1 = x.hi * u.hi;
    float e1 = fmaf(x.hi, u.hi, -p1);
    e1 = fmaf(x.hi, u.lo, e1);
    e1 = fmaf(x.lo, u.hi, e1);
    const float p2 = y.hi * v.hi;
    float e2 = fmaf(y.hi, v.hi, -p2);
    e2 = fmaf(y.hi, v.lo, e2);
    e2 = fmaf(y.lo, v.hi, e2);
    float s1, t1, s2, t2;
    ff_two_sum(a.hi, -p1, s1, t1);
    ff_two_sum(s1, p2, s2, t2);
    return ff_norm(s2, ((a.lo - e1) + e2) + (t1 + t2));
}

// 1 / m for double-FP32 m > 0: the FP32 reciprocal refined by one Newton step on
// the exact FMA residual.
__device__ __forceinline__ ff ff_recip(ff m)
{
    const float y0 = 1.0f / m.hi;
    float r = fmaf(-m.hi, y0, 1.0f);   // 1 - m.hi y0, exact
    r = fmaf(-m.lo, y0, r);
    return ff_norm(y0, y0 * r);
}

// Positions, momenta and the action: FP64 in the FP64 path, double-FP32 pairs in the
// mixed path (FP64-class accuracy, about 2^-46 relative per operation, on the FP32 pipe:
// on this GPU an FP64 instruction or conversion costs the FP64 pipe ~70 times the issue
// of an FP32 one).  coord_axpy: c + t x; coord_kick: c - t g for an FP32 force g; t is
// given as FP64 (td) and as FP32 leading and trailing words (th, tl).
__device__ __forceinline__ void coord_set(double &c, double x) { c = x; }
__device__ __forceinline__ void coord_set(ff &c, double x)
{
    c.hi = (float)x;
    c.lo = (float)(x - (double)c.hi);
}
__device__ __forceinline__ double coord_get(double c) { return c; }
__device__ __forceinline__ double coord_get(ff c) { return (double)c.hi + (double)c.lo; }
__device__ __forceinline__ double coord_f(double c) { return c; }
__device__ __forceinline__ float coord_f(ff c) { return c.hi; }
__device__ __forceinline__ bool coord_finite(double c) { return isfinite(c); }
__device__ __forceinline__ bool coord_finite(ff c) { return isfinite(c.hi) && isfinite(c.lo); }
__device__ __forceinline__ double coord_axpy(double c, double td, float, float, double x) { return fma(td, x, c); }
__device__ __forceinline__ ff coord_axpy(ff c, double, float th, float tl, ff x)
{
    const float p = th * x.hi;
    float e = fmaf(th, x.hi, -p);   // th x.hi - p, exact
    e = fmaf(th, x.lo, e);
    e = fmaf(tl, x.hi, e);
    float s, e2;
    ff_two_sum(c.hi, p, s, e2);
    return ff_norm(s, e2 + (c.lo + e));
}
__device__ __forceinline__ double coord_kick(double c, double td, float, float, double g) { return fma(-td, g, c); }
__device__ __forceinline__ ff coord_kick(ff c, double, float th, float tl, float g)
{
    const float p = -th * g;
    float e = fmaf(-th, g, -p);
    e = fmaf(-tl, g, e);
    float s, e2;
    ff_two_sum(c.hi, p, s, e2);
    return ff_norm(s, e2 + (c.lo + e));
}
// the action increment (FP32 partial sums) joins the running action
__device__ __forceinline__ double coord_add(double c, double d) { return c + d; }
__device__ __forceinline__ ff coord_add(ff c, float d)
{
    float s, e;
    ff_two_sum(c.hi, d, s, e);
    return ff_norm(s, e + c.lo);
}

// Complex double-FP32 numbers as packed pairs: hi = (re.hi, im.hi), lo = (re.lo, im.lo).
// ff2_sub_mul_add_mul(a, x, u, y, v) = a - x u + y v for real double-FP32 x, y: per part
// the same operations in the same order as ff_sub_mul_add_mul, each instruction doing the
// real and the imaginary part at once.
struct ff2 { float2 hi, lo; };

__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }

__device__ __forceinline__ void ff2_two_sum(float2 a, float2 b, float2 &s, float2 &e)
{
    s = add2(a, b);
    const float2 bb = sub2(s, a);
    e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}

__device__ __forceinline__ ff2 ff2_sub_mul_add_mul(ff2 a, ff x, ff2 u, ff y, ff2 v)
{
    const float2 xh = make_float2(x.hi, x.hi), xl = make_float2(x.lo, x.lo);
    const float2 yh = make_float2(y.hi, y.hi), yl = make_float2(y.lo, y.lo);
    const float2 p1 = __fmul2_rn(xh, u.hi);
    float2 e1 = __ffma2_rn(xh, u.hi, neg2(p1));
    e1 = __ffma2_rn(xh, u.lo, e1);
    e1 = __ffma2_rn(xl, u.hi, e1);
    const float2 p2 = __fmul2_rn(yh, v.hi);
    float2 e2 = __ffma2_rn(yh, v.hi, neg2(p2));
    e2 = __ffma2_rn(yh, v.lo, e2);
    e2 = __ffma2_rn(yl, v.hi, e2);
    float2 s1, t1, s2, t2;
    ff2_two_sum(a.hi, neg2(p1), s1, t1);
    ff2_two_sum(s1, p2, s2, t2);
    const float2 lo = add2(add2(sub2(a.lo, e1), e2), add2(t1, t2));
    ff2 r;
    r.hi = add2(s2, lo);
    r.lo = sub2(lo, sub2(r.hi, s2));
    return r;
}

// Per-mode and per-reference-state constants, staged in shared memory so that
// lane- or chi-dependent indexing never touches the kernel-parameter space.
template <int F>
struct CtaConst {
    double qw[F], pw[F];
    double p_eq[SCIVR_MAX_CHI][F], q_eq[SCIVR_MAX_CHI][F];
    float Df[F], af[F], w2f[F];            // diagonal parameters in FP32
    double Dd[F], ad[F], w2d[F];           // and in FP64
    float qwf[F], pwf[F];                  // overlap constants in FP32 (mixed path's overlap)
    float p_eqf[SCIVR_MAX_CHI][F], q_eqf[SCIVR_MAX_CHI][F];
};

// Real-typed views of the staged constants.
template <typename Real, int F> __device__ __forceinline__ Real c_D(const CtaConst<F> &c, int i) { if constexpr (sizeof(Real) == 4) return c.Df[i]; else return c.Dd[i]; }
template <typename Real, int F> __device__ __forceinline__ Real c_a(const CtaConst<F> &c, int i) { if constexpr (sizeof(Real) == 4) return c.af[i]; else return c.ad[i]; }
template <typename Real, int F> __device__ __forceinline__ Real c_w2(const CtaConst<F> &c, int i) { if constexpr (sizeof(Real) == 4) return c.w2f[i]; else return c.w2d[i]; }

// Column of job j in row r of the per-job arrays: the F mode lanes of a group
// store one job into F different rows, which a plain [row][job] layout puts
// into a single shared-memory bank; XOR-ing the job with the row spreads them
// over banks, and every row is still a permutation of the chunk's jobs.
template <int JOBS>
__device__ __forceinline__ int jswz(int r, int j) { return j ^ (r & (JOBS >= 16 ? 15 : JOBS - 1)); }

// Steps per chunk of a lane group.  Phases 2-4 work on T * C jobs (trajectory, step)
// per warp.  FP64 path: one lane per job; groups of 8 and 16 lanes fill all 32 lanes,
// the one-trajectory-per-warp groups take 16 jobs (F = 9) or 8 (F > 9).  Mixed path:
// the double-FP32 elimination keeps two FP32 words per real entry, so chunks are
// shorter (8 steps; 4 above F = 12) and 32 / (T * C) lanes share a job's elimination
// by rows; the per-job prefactor matrices then take the same shared memory as one
// FP32 word per entry at the FP64 path's chunk length.
// Mixed path: steps between stability tests (a multiple of every mixed chunk length).
// The flag is sticky and a bad trajectory is dropped whole, so a coarser test differs
// from the per-step one only for a deviation that crosses the threshold and falls back
// below it between two tests (on the recipe surfaces, none: the good sets at 8- and
// 16-step cadences equal the per-step ones).
constexpr int kDetMEvery = 16;

template <int F, int G, typename Real> __host__ __device__ constexpr int lg_chunk()
{
    if constexpr (sizeof(Real) == 4) return G == 32 && F > 16 ? 2 : ((G == 32 && F > 12) || (G == 16 && F > 8) ? 4 : 8);
    else return G < 32 ? G : (F > 9 ? 8 : 16);
}

// Warps per CTA and the launch-bounds CTA count: the wide groups (F > 9) run one CTA per
// SM on one copy of the coupling tensors, 8 warps up to F = 12 and 4 above (measured:
// at F = 15 the 8-warp CTA's 216 KB of shared memory leaves too little L1 and runs 16 %
// slower; at F = 12 8 warps are 5 % faster).
template <int F, int G> __host__ __device__ constexpr int lg_warps() { return G < 32 ? 4 : (F <= 9 ? 2 : (F <= 12 ? 8 : 4)); }
// (F > 16: 4 warps, one CTA per SM: 18 KB of per-job prefactor matrices and 9 KB of det M
// workspace per warp at F = 24)
// Two-trajectory mixed warps (F = 6..9) hold the coupling tensors in registers (no
// shared-memory reads of them, more registers: lg_min_ctas) or read them from shared
// memory in the same half-split layout (TensorLayout::split).  Measured on the recipe
// surfaces: registers win at F = 7 (7 %) and F = 8 (10 %: the shared-memory schedule there
// is held to 128 registers by its four CTAs per SM); shared memory wins at F = 6 (6 %, four
// CTAs per SM against three) and at F = 9 (12 %, three against two).
template <int F> __host__ __device__ constexpr bool lg_tensor_regs() { return F == 7 || F == 8; }

template <int F, int G, typename Real> __host__ __device__ constexpr int lg_min_ctas()
{
    // register-held tensors: two CTAs per SM at F = 8, 9 (up to 255 registers), three at F = 6, 7
    if constexpr (sizeof(Real) == 4 && G == 16 && F >= 6 && lg_tensor_regs<F>()) return F >= 8 ? 2 : 3;
    return F > 9 ? 1 : (sizeof(Real) == 4 && 2 * F > G ? 3 : 4);
}

// 16-byte vectors of Real for shared-memory loads.
template <typename Real> struct V16;
template <> struct V16<float> { using T = float4; static constexpr int N = 4; };
template <> struct V16<double> { using T = double2; static constexpr int N = 2; };

template <typename Real>
__device__ __forceinline__ Real vcomp(const typename V16<Real>::T &v, int j)
{
    if constexpr (V16<Real>::N == 4) return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
    else return j == 0 ? v.x : v.y;
}

// Length of a row padded to whole 16-byte vectors.
template <typename Real>
__host__ __device__ constexpr int vec_len(int n)
{
    return (n + V16<Real>::N - 1) / V16<Real>::N * V16<Real>::N;
}

// Row stride for rows that different lanes read with 16-byte loads at the same
// time: whole vectors, an odd number of them, so that the 8 lanes served by one
// shared-memory wavefront start in 8 different groups of 4 banks.
template <typename Real>
__host__ __device__ constexpr int row_stride(int n)
{
    return (vec_len<Real>(n) / V16<Real>::N) % 2 == 0 ? vec_len<Real>(n) + V16<Real>::N : vec_len<Real>(n);
}

// Packed FP32 multiply-add on register pairs (one instruction, two lanes of work).
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 lo2(const float4 &v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4 &v) { return make_float2(v.z, v.w); }

// sum_{i < S} a[i] b[i] over 16-byte aligned shared rows (S a multiple of the
// vector length) with one partial sum per vector lane (FP32: packed pairs).
template <typename Real, int S>
__device__ __forceinline__ Real dot16(const Real *a, const Real *b)
{
    using VT = typename V16<Real>::T;
    constexpr int N = V16<Real>::N;
    static_assert(S % N == 0, "padded length");
    if constexpr (sizeof(Real) == 4) {
        float2 a0 = make_float2(0.0f, 0.0f), a1 = a0;
#pragma unroll
        for (int i = 0; i < S; i += 4) {
            const float4 x = *reinterpret_cast<const float4 *>(a + i);
            const float4 y = *reinterpret_cast<const float4 *>(b + i);
            a0 = ffma2(lo2(x), lo2(y), a0);
            a1 = ffma2(hi2(x), hi2(y), a1);
        }
        return (a0.x + a1.x) + (a0.y + a1.y);
    }
    Real acc[N];
#pragma unroll
    for (int j = 0; j < N; ++j) acc[j] = Real(0);
#pragma unroll
    for (int i = 0; i < S; i += N) {
        const VT x = *reinterpret_cast<const VT *>(a + i);
        const VT y = *reinterpret_cast<const VT *>(b + i);
#pragma unroll
        for (int j = 0; j < N; ++j) acc[j] = fma(vcomp<Real>(x, j), vcomp<Real>(y, j), acc[j]);
    }
    Real r = acc[0];
#pragma unroll
    for (int j = 1; j < N; ++j) r += acc[j];
    return r;
}

// Coupling tensors staged per CTA, transposed so that one potential entry e
// reads one contiguous row: sT3[e][k] (k < F, stride S3), sT4[e][kl] (kl < P,
// stride S4), zero-padded.
template <int F, typename Real, bool STAGED = (F <= 16)>
struct TensorLayout {
    static constexpr int P = F * (F + 1) / 2;
    static constexpr int S3 = vec_len<Real>(F);   // short rows: fewer loads outweigh a 2-way conflict
    static constexpr int S4 = row_stride<Real>(P);
    // Above F = 16 the quartic tensor (P^2 entries, 360 KB at F = 24) does not fit shared
    // memory: both tensors are read from global memory (L2) and only the coefficients are staged.
    static constexpr bool staged = STAGED;
    // Two-trajectory mixed warps (F = 6..9) cut x = (q, zero pad to an even length F3E, the
    // pair products, zero pad) into two halves of KH elements; those that do not hold the
    // tensors in registers read them from shared memory cut the same way ("split"):
    // sTh[h][e][KHS] = the tensor row of entry e over half h of x, KHS an odd number of
    // 16-byte vectors so that 8 lanes reading 8 consecutive entries hit disjoint banks.
    static constexpr int F3E = (F + 1) & ~1;
    static constexpr int KH = (((F3E + P + 1) / 2) + 3) & ~3;
    static constexpr int KHS = (KH / 4) % 2 ? KH : KH + 4;
    static constexpr bool split = sizeof(Real) == 4 && STAGED && F >= 6 && F <= 9 && !lg_tensor_regs<F>();
    static constexpr size_t tensor_elems = !staged ? 0 : (split ? (size_t)2 * P * KHS : (size_t)P * S3 + (size_t)P * S4);
    // after the tensors: the Herman-Kluk matrix coefficients acoef[a][b][4] =
    // (1/2) {rg_a/rg_b, rg_b/rg_a, -rg_a rg_b, 1/(rg_a rg_b)}, rg = sqrt(gamma)
    static constexpr size_t bytes = ((sizeof(Real) * (tensor_elems + (size_t)4 * F * F)) + 15) & ~(size_t)15;
};

template <int F, int G, typename Real>
struct WarpShared {
    static constexpr int P = F * (F + 1) / 2;
    static constexpr int T = 32 / G;
    static constexpr int JOBS = T * lg_chunk<F, G, Real>();   // jobs per chunk (phases 2-4)
    static constexpr int S3 = TensorLayout<F, Real>::S3;   // q, zero-padded (also the Gc row stride)
    static constexpr int S4 = TensorLayout<F, Real>::S4;   // pair products q_k q_l, zero-padded
    static constexpr int SH = vec_len<Real>(F);            // row stride of H (rows read by the whole group)
    alignas(16) Real qr[T][S3];
    alignas(16) Real qq[T][S4];
    // x = (q, zero pad to an even length, pair products, zero pad) in two halves of KH for the
    // half-split Hessian of two-trajectory warps (see TensorLayout and lg_body)
    static constexpr int F3E = TensorLayout<F, Real>::F3E;
    static constexpr int KH = TensorLayout<F, Real>::KH;
    // only two-trajectory mixed warps use it: elsewhere a stub, so that the shared memory
    // left to L1 (the wide groups read their tensors through it) does not shrink
    static constexpr bool kHalves = (T == 2) && (sizeof(Real) == 4) && F >= 6 && F <= 9;
    alignas(16) Real xs[T][kHalves ? 2 * KH : 4];
    alignas(16) Real Gc[T][F][S3];          // gradient coefficients, full symmetric matrix (row a read by mode lane a)
    alignas(16) Real H[T][F][SH];
    // prefactor matrix per job, job-major rows of AS entries (AS odd): a lane that walks one
    // row of its job's matrix advances its address by one entry, and lanes of different jobs
    // at the same entry start in different banks
    static constexpr int AS = ((F * F) % 2) ? F * F : F * F + 1;
    typename AEntry<Real>::T A[JOBS][AS];
    __device__ __forceinline__ typename AEntry<Real>::T &a_at(int job, int e) { return A[job][e]; }
    Real pj[F][JOBS], qj[F][JOBS];         // state per job, for the overlap (job column swizzled); FP32
                                           // in the mixed path, where the overlap is evaluated in FP32
    double Sj[JOBS];                        // action per job
    double lnA[JOBS];                       // log |det A|^{1/2} per job (Herman-Kluk summand only)
    double argj[JOBS];                      // arg det A per job (mixed path: from the elimination's lanes)
    double2 detAj[JOBS];                    // det A per job (mixed path)
    double2 ov0[SCIVR_MAX_CHI][T];          // log of the Herman-Kluk summand's divisor per trajectory
};

// One CTA's share of a propagation: trajectories (cta * WARPS + warp) * T + t.
// Called by the per-molecule kernel (cta = blockIdx.x) and by the batched
// persistent kernel (cta = the work item's tile).  Stages the molecule's
// constants itself and leaves shared memory free for the next call.
template <int F, int G, typename Real, int WARPS, bool STAGED = (F <= 16)>
__device__ __forceinline__ void lg_body(const PropLaunch &L, int64_t cta, unsigned char *smem_raw)
{
    constexpr int N2 = 2 * F;
    constexpr int P = F * (F + 1) / 2;
    constexpr int T = 32 / G;
    constexpr int C = lg_chunk<F, G, Real>();  // steps per chunk
    constexpr int JOBS = T * C;                // jobs per chunk: job t * C + c is trajectory t's step c
    constexpr int EPL = (P + G - 1) / G;       // packed Hessian entries per lane
    constexpr int NCOL = (N2 + G - 1) / G;     // monodromy columns per lane: column c sits in lane c % G, slot c / G
    static_assert(F <= G && NCOL <= 2, "a group holds every mode and at most two columns per lane");
    using Sh = WarpShared<F, G, Real>;
    using R2 = typename Vec2<Real>::T;

    using TL = TensorLayout<F, Real, STAGED>;
    constexpr int S3 = TL::S3, S4 = TL::S4;
    Real *sT3 = reinterpret_cast<Real *>(smem_raw);
    Real *sT4 = sT3 + ((TL::staged && !TL::split) ? P * S3 : 0);
    Real *sTh = sT3;                                  // the half-split layout (TL::split)
    Real *sAc = sT3 + TL::tensor_elems;   // Herman-Kluk matrix coefficients [a][b][4] (16-byte aligned: the tensor block is a vector multiple)
    size_t off = TL::bytes;
    CtaConst<F> &cc = *reinterpret_cast<CtaConst<F> *>(smem_raw + off);
    off += (sizeof(CtaConst<F>) + 15) & ~(size_t)15;
    Sh *wsh_all = reinterpret_cast<Sh *>(smem_raw + off);

    const PesDev &pes = L.pes;
    const PropArgs &A = L.args;
    const bool use3 = pes.has3, use4 = pes.has4;
    // stage the coupling tensors once per CTA
    if constexpr (TL::staged) {
        const Real *g3 = nullptr, *g4 = nullptr;
        if constexpr (sizeof(Real) == 4) { g3 = reinterpret_cast<const Real *>(pes.T3f); g4 = reinterpret_cast<const Real *>(pes.T4f); }
        else { g3 = reinterpret_cast<const Real *>(pes.T3); g4 = reinterpret_cast<const Real *>(pes.T4); }
        if constexpr (TL::split) {
            constexpr int KH = TL::KH, KHS = TL::KHS, F3E = TL::F3E;
            for (int i = threadIdx.x; i < 2 * P * KHS; i += blockDim.x) {
                const int h = i / (P * KHS), e = (i / KHS) % P, kk = i % KHS, gk = h * KH + kk;
                Real v = Real(0);
                if (kk < KH) {
                    if (gk < F) v = use3 ? g3[gk * P + e] : Real(0);
                    else if (gk >= F3E && gk - F3E < P) v = use4 ? g4[(gk - F3E) * P + e] : Real(0);
                }
                sTh[i] = v;
            }
        } else {
            for (int i = threadIdx.x; i < P * S3; i += blockDim.x) {
                const int e = i / S3, k = i % S3;
                sT3[i] = (use3 && k < F) ? g3[k * P + e] : Real(0);
            }
            for (int i = threadIdx.x; i < P * S4; i += blockDim.x) {
                const int e = i / S4, kl = i % S4;
                sT4[i] = (use4 && kl < P) ? g4[kl * P + e] : Real(0);
            }
        }
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int a = 0; a < F; ++a) {
            cc.qw[a] = A.qw[a];
            cc.pw[a] = A.pw[a];
            cc.qwf[a] = (float)A.qw[a];
            cc.pwf[a] = (float)A.pw[a];
            cc.Dd[a] = pes.D[a];
            cc.ad[a] = pes.a[a];
            cc.w2d[a] = pes.omega[a] * pes.omega[a];
            cc.Df[a] = pes.D_f[a];
            cc.af[a] = pes.a_f[a];
            cc.w2f[a] = pes.omega_f[a] * pes.omega_f[a];
        }
        // (rolled: thread 0 alone, and unrolling F^2 iterations starves the step loop of registers)
        for (int a = 0; a < F; ++a)
            for (int b = 0; b < F; ++b) {
                const Real rga = (Real)A.rg[a], irga = (Real)A.irg[a], rgb = (Real)A.rg[b], irgb = (Real)A.irg[b];
                Real *k = sAc + 4 * (a * F + b);
                k[0] = Real(0.5) * (rga * irgb);
                k[1] = Real(0.5) * (rgb * irga);
                k[2] = Real(-0.5) * (rga * rgb);
                k[3] = Real(0.5) * (irga * irgb);
            }
#pragma unroll
        for (int x = 0; x < SCIVR_MAX_CHI; ++x)
#pragma unroll
            for (int a = 0; a < F; ++a) {
                cc.p_eq[x][a] = x < A.n_chi ? A.p_eq[x * F + a] : 0.0;
                cc.q_eq[x][a] = x < A.n_chi ? A.q_eq[x * F + a] : 0.0;
                cc.p_eqf[x][a] = (float)cc.p_eq[x][a];
                cc.q_eqf[x][a] = (float)cc.q_eq[x][a];
            }
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, ln = threadIdx.x & 31;
    const int t = ln / G, g = ln % G, base = t * G;
    Sh &sh = wsh_all[warp];
    {
        // padding entries of the vector rows are read (multiplied by zero or skipped) but never
        // written by the step loop: clear the warp's rows once
        Real *z = &sh.qr[0][0];
        constexpr int nz = (int)((offsetof(Sh, H) + sizeof(Sh::H) - offsetof(Sh, qr)) / sizeof(Real));
        for (int i = ln; i < nz; i += 32) z[i] = Real(0);
        __syncwarp();
    }
    const int64_t n = L.n_traj;
    const int64_t j_traj = (cta * WARPS + warp) * T + t;
    const bool active = j_traj < n;
    const int64_t jl = active ? j_traj : n - 1;

    // packed entries handled by this lane
    int ea[EPL], eb[EPL];
#pragma unroll
    for (int i = 0; i < EPL; ++i) {
        int e = g + i * G, a = 0;
        if (e >= P) e = 0;
        while (e >= F - a) { e -= F - a; ++a; }
        ea[i] = a;
        eb[i] = a + e;
    }
    // two trajectories per warp (16-lane groups, mixed path, P <= 64): the coupling tensors
    // live in registers.  x = (q, qq) is cut into two halves of KH elements; lane ln holds,
    // for its half hx = ln / 16, the matching parts of the tensor rows of the entries
    // jx + 16 i (jx = ln % 16, i < EPH), and multiplies them by both trajectories' halves of
    // x (read as warp-broadcast 16-byte loads).  Lanes ln and ln ^ 16 then exchange partial
    // sums so that each ends with whole entries of its own trajectory.
    constexpr bool kPair = (T == 2) && (sizeof(Real) == 4) && TL::staged && (P <= 64) && (P > 16);
    constexpr bool kTreg = kPair && lg_tensor_regs<F>();
    // or the same cut with the tensor rows read from shared memory (TL::split)
    constexpr bool kSplit = kPair && !kTreg && TL::split;
    static_assert(kPair == (kTreg || kSplit), "two-trajectory warps take one of the two half-split schedules");
    static_assert(!kPair || Sh::kHalves, "the half-split schedules need the halves of x");
    // packed FP32 pairs in the monodromy drift and kick
    constexpr bool kPacked = sizeof(Real) == 4;
    constexpr int F3E = Sh::F3E, KH = Sh::KH, KHS = TL::KHS;
    constexpr int EPH = (kTreg || kSplit) ? (P + 15) / 16 : 1;
    const int hx = ln >> 4, jx = ln & 15;
    int ebA[EPH], ebB[EPH];
    float2 Tr[EPH][kTreg ? KH / 2 : 1];
    if constexpr (kSplit) {
#pragma unroll
        for (int i = 0; i < EPH; ++i) {
            const int e0 = jx + 16 * i;
            int e = e0 < P ? e0 : 0, a = 0;
            while (e >= F - a) { e -= F - a; ++a; }
            ebA[i] = a;
            ebB[i] = a + e;
        }
    }
    if constexpr (kTreg) {
#pragma unroll
        for (int i = 0; i < EPH; ++i) {
            const int e0 = jx + 16 * i;
            int e = e0 < P ? e0 : 0, a = 0;
            while (e >= F - a) { e -= F - a; ++a; }
            ebA[i] = a;
            ebB[i] = a + e;
#pragma unroll
            for (int k2 = 0; k2 < KH / 2; ++k2) {
                float v[2];
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int gk = hx * KH + 2 * k2 + c;   // position in x
                    v[c] = 0.0f;
                    if (e0 < P) {
                        if (gk < F) v[c] = sT3[e0 * S3 + gk];
                        else if (gk >= F3E && gk - F3E < P) v[c] = sT4[e0 * S4 + gk - F3E];
                    }
                }
                Tr[i][k2] = make_float2(v[0], v[1]);
            }
        }
    }
    // above F = 16: four consecutive entries 4 (g + i G) .. + 3 per load, (a, b) packed as a | b << 8
    constexpr int P4 = (P + 3) & ~3;
    constexpr int NQ = TL::staged ? 1 : (P4 / 4 + G - 1) / G;
    int eq[TL::staged ? 1 : 4 * NQ];
    if constexpr (!TL::staged) {
#pragma unroll
        for (int i = 0; i < 4 * NQ; ++i) {
            int e = 4 * (g + (i / 4) * G) + i % 4, a = 0;
            if (e >= P) e = 0;
            while (e >= F - a) { e -= F - a; ++a; }
            eq[i] = a | ((a + e) << 8);
        }
    }

    // mode state (lane g < F)
    const int mode = g < F ? g : 0;
    using Coord = std::conditional_t<sizeof(Real) == 4, ff, double>;
    Coord p, q;
    coord_set(p, L.p0[mode * n + jl]);
    coord_set(q, L.q0[mode * n + jl]);
    Real pr = (Real)coord_get(p);   // the momentum as seen by the Real-precision bulk
    Coord S;                        // accumulated action (lane 0 of the group holds the total)
    coord_set(S, 0.0);
    // per-job action in the job table: FP64, or the double-FP32 pair in the same 8 bytes
    auto sj_put = [&](int j, Coord v) {
        if constexpr (sizeof(Real) == 4) reinterpret_cast<float2 *>(sh.Sj)[j] = make_float2(v.hi, v.lo);
        else sh.Sj[j] = v;
    };
    auto sj_get = [&](int j) -> double {
        if constexpr (sizeof(Real) == 4) {
            const float2 v = reinterpret_cast<const float2 *>(sh.Sj)[j];
            return (double)v.x + (double)v.y;
        } else {
            return sh.Sj[j];
        }
    };
    // column state: slot s of lane g holds column c = g + s G of M = d(p,q)/d(p0,q0) (c < 2F;
    // a slot past 2F holds a zero column)
    Real Mp[NCOL][F], Mq[NCOL][F];
#pragma unroll
    for (int s = 0; s < NCOL; ++s) {
        const int col = g + s * G;
#pragma unroll
        for (int a = 0; a < F; ++a) {
            Mp[s][a] = (col < F && a == col) ? Real(1) : Real(0);
            Mq[s][a] = (col >= F && col < N2 && a == col - F) ? Real(1) : Real(0);
        }
    }
    bool good = true;
    Real stab = Real(0);
    double detM_last = 1.0;
    double theta_last = 0.0, arg_last = 0.0;
    double2 detA_last = make_double2(1.0, 0.0);   // det A of the last step

    // amplitude at c = 0 (M = I, S = 0, theta = 0): lane 0 of each group
    if (g == 0 && active) {
        double re00 = 0.0;   // Re log <chi_0|p0 q0>
        for (int x = 0; x < A.n_chi; ++x) {
            double re = 0.0, im = 0.0;
            for (int a = 0; a < F; ++a) {
                const double pa = L.p0[a * n + jl], qa = L.q0[a * n + jl];
                const double dq = cc.q_eq[x][a] - qa, dp = cc.p_eq[x][a] - pa;
                re = fma(-cc.qw[a] * dq, dq, re);
                re = fma(-cc.pw[a] * dp, dp, re);
                im = fma(0.5 * (cc.p_eq[x][a] + pa), dq, im);
            }
            if (x == 0) re00 = re;
            // what the Herman-Kluk summand divides by: <chi_x|p0 q0> |<p0 q0|chi_0>|^2 / |<p0 q0|chi_x>|^2,
            // i.e. the initial overlap times the importance weight of the sampling density (the first
            // reference state's); its real logarithm 2 re00 - re equals re for x = 0
            const double rdiv = x == 0 ? re : 2.0 * re00 - re;
            sh.ov0[x][t] = make_double2(rdiv, im);
            double sn, cs;
            sincos(im, &sn, &cs);
            const double mag = exp(re);
            // the Herman-Kluk summand at t = 0 (C = 1, S = 0) is |<chi_x|p0 q0>|^2 / |<chi_0|p0 q0>|^2,
            // exactly 1 for x = 0
            if (A.amplitude == SCIVR_AMP_HK) amp_store(L, x * L.chi_stride + jl * L.amp_ld, x == 0 ? 1.0 : exp(re - rdiv), 0.0);
            else amp_store(L, x * L.chi_stride + jl * L.amp_ld, mag * cs, mag * sn);
        }
    }

    for (int step0 = 0; step0 < A.n_steps; step0 += C) {
        const int cnt = min(C, A.n_steps - step0);
        // ---------------- phase 1: cnt steps, group-parallel ----------------
        for (int c = 0; c < cnt; ++c) {
            Real dS = Real(0);   // this lane's share of the step's action increment
#pragma unroll 1
            for (int sub = 0; sub < 4; ++sub) {
                // drift: q += tau p, S += tau p.p/2, M_q += tau M_p
                {
                    Real rt;
                    if constexpr (sizeof(Real) == 4) rt = A.tdrift_f[sub]; else rt = A.tdrift[sub];
                    if (g < F) {
                        q = coord_axpy(q, A.tdrift[sub], A.tdrift_f[sub], A.tdrift_lo[sub], p);
                        dS = fma(rt * Real(0.5) * pr, pr, dS);
                    }
                    if constexpr (kPacked) {
                        const float2 rt2 = make_float2(rt, rt);
#pragma unroll
                        for (int s = 0; s < NCOL; ++s) {
#pragma unroll
                            for (int a = 0; a + 1 < F; a += 2) {
                                const float2 r = ffma2(rt2, make_float2(Mp[s][a], Mp[s][a + 1]), make_float2(Mq[s][a], Mq[s][a + 1]));
                                Mq[s][a] = r.x;
                                Mq[s][a + 1] = r.y;
                            }
                            if constexpr (F % 2) Mq[s][F - 1] = fmaf(rt, Mp[s][F - 1], Mq[s][F - 1]);
                        }
                    } else {
#pragma unroll
                        for (int s = 0; s < NCOL; ++s)
#pragma unroll
                            for (int a = 0; a < F; ++a) Mq[s][a] = fma(rt, Mp[s][a], Mq[s][a]);
                    }
                }
                if (sub == 3) break;
                // kick: potential at q
                const double tk = A.tkick[sub];
                Real rtk;
                if constexpr (sizeof(Real) == 4) rtk = A.tkick_f[sub]; else rtk = tk;
                __syncwarp();   // previous kick's readers of qr/H are done
                if (g < F) {
                    sh.qr[t][g] = (Real)coord_f(q);
                    if constexpr (kTreg || kSplit) sh.xs[t][g] = (Real)coord_f(q);
                }
                __syncwarp();
#pragma unroll
                for (int i = 0; i < EPL; ++i) {
                    const int e = g + i * G;
                    if (e < P) {
                        const Real v = sh.qr[t][ea[i]] * sh.qr[t][eb[i]];
                        sh.qq[t][e] = v;
                        if constexpr (kTreg || kSplit) sh.xs[t][F3E + e] = v;
                    }
                }
                __syncwarp();
                Real vpart = Real(0);
                if constexpr (!TL::staged) {
                    // entry quads against the tensors in global memory (L2-resident; [k][e] and
                    // [kl][e] rows padded to P4): one 16-byte load feeds four entries
                    static_assert(sizeof(Real) == 4, "the global-tensor schedule is the mixed path's");
                    const float4 *T3v = reinterpret_cast<const float4 *>(pes.T3p);
                    const float4 *T4v = reinterpret_cast<const float4 *>(pes.T4p);
#pragma unroll
                    for (int i = 0; i < NQ; ++i) {
                        const int q4 = g + i * G;
                        if (4 * q4 < P) {
                            float4 h3 = make_float4(0.f, 0.f, 0.f, 0.f), h4 = h3;
                            if (use3) {
#pragma unroll 8
                                for (int k = 0; k < F; ++k) {
                                    const float4 tv = __ldg(T3v + k * (P4 / 4) + q4);
                                    const float x = sh.qr[t][k];
                                    h3.x = fmaf(tv.x, x, h3.x); h3.y = fmaf(tv.y, x, h3.y);
                                    h3.z = fmaf(tv.z, x, h3.z); h3.w = fmaf(tv.w, x, h3.w);
                                }
                            }
                            if (use4) {
#pragma unroll 4
                                for (int kl = 0; kl < P; ++kl) {
                                    const float4 tv = __ldg(T4v + kl * (P4 / 4) + q4);
                                    const float x = sh.qq[t][kl];
                                    h4.x = fmaf(tv.x, x, h4.x); h4.y = fmaf(tv.y, x, h4.y);
                                    h4.z = fmaf(tv.z, x, h4.z); h4.w = fmaf(tv.w, x, h4.w);
                                }
                            }
                            const float h3j[4] = {h3.x, h3.y, h3.z, h3.w}, h4j[4] = {h4.x, h4.y, h4.z, h4.w};
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const int e = 4 * q4 + j;
                                if (e < P) {
                                    const int a = eq[4 * i + j] & 255, b = eq[4 * i + j] >> 8;
                                    const Real h = h3j[j] + h4j[j];
                                    sh.H[t][a][b] = h;
                                    sh.H[t][b][a] = h;
                                    const Real gce = fma(Real(0.5), h3j[j], h4j[j] * Real(1.0 / 3.0));
                                    sh.Gc[t][a][b] = gce;
                                    sh.Gc[t][b][a] = gce;
                                    const Real vc = fma(Real(1.0 / 6.0), h3j[j], h4j[j] * Real(1.0 / 12.0));
                                    vpart = fma(a == b ? vc : Real(2) * vc, sh.qq[t][e], vpart);
                                }
                            }
                        }
                    }
                } else if constexpr (kTreg || kSplit) {
                    float2 aF[EPH][2], a4[EPH][2];   // packed partial sums per entry and trajectory
                    float sF[EPH][2];                // the first F3E elements of x (q in half 0)
#pragma unroll
                    for (int i = 0; i < EPH; ++i)
#pragma unroll
                        for (int tt = 0; tt < 2; ++tt) {
                            aF[i][tt] = a4[i][tt] = make_float2(0.0f, 0.0f);
                            sF[i][tt] = 0.0f;
                        }
                    const float *x0 = &sh.xs[0][hx * KH], *x1 = &sh.xs[1][hx * KH];
                    const float *trow[EPH];          // kSplit: this lane's rows (entries past P read row 0)
#pragma unroll
                    for (int i = 0; i < EPH; ++i) {
                        const int e = jx + 16 * i;
                        trow[i] = sTh + (hx * P + (e < P ? e : 0)) * KHS;
                    }
                    // a surface without couplings (uniform over the CTA) leaves every sum zero
                    if (use3 || use4)
#pragma unroll
                    for (int c = 0; c < KH; c += 4) {
                        const float4 u = *reinterpret_cast<const float4 *>(x0 + c);
                        const float4 w = *reinterpret_cast<const float4 *>(x1 + c);
                        float4 tv[EPH];
                        if constexpr (kSplit) {
#pragma unroll
                            for (int i = 0; i < EPH; ++i) tv[i] = *reinterpret_cast<const float4 *>(trow[i] + c);
                        }
#pragma unroll
                        for (int hp = 0; hp < 2; ++hp) {
                            const int kk = c + 2 * hp;
                            const float2 xu = hp ? hi2(u) : lo2(u), xw = hp ? hi2(w) : lo2(w);
#pragma unroll
                            for (int i = 0; i < EPH; ++i) {
                                float2 t2;
                                if constexpr (kSplit) t2 = hp ? hi2(tv[i]) : lo2(tv[i]);
                                else t2 = Tr[i][kk / 2];
                                if (kk < F3E) {
                                    aF[i][0] = ffma2(t2, xu, aF[i][0]);
                                    aF[i][1] = ffma2(t2, xw, aF[i][1]);
                                } else {
                                    a4[i][0] = ffma2(t2, xu, a4[i][0]);
                                    a4[i][1] = ffma2(t2, xw, a4[i][1]);
                                }
                            }
                            if (kk + 2 == F3E) {
#pragma unroll
                                for (int i = 0; i < EPH; ++i)
#pragma unroll
                                    for (int tt = 0; tt < 2; ++tt) sF[i][tt] = aF[i][tt].x + aF[i][tt].y;
                            }
                        }
                    }
                    // half 0 holds the cubic rows (h3) and the first pair products; half 1 only
                    // pair products.  Keep trajectory hx, pass the partner its trajectory's sums.
                    float vp = 0.0f;
#pragma unroll
                    for (int i = 0; i < EPH; ++i) {
                        float s3[2], s4[2];
#pragma unroll
                        for (int tt = 0; tt < 2; ++tt) {
                            const float r = a4[i][tt].x + a4[i][tt].y;
                            s3[tt] = hx == 0 ? sF[i][tt] : 0.0f;
                            s4[tt] = hx == 0 ? r : sF[i][tt] + r;
                        }
                        const float o3 = __shfl_xor_sync(FULL, hx ? s3[0] : s3[1], 16);
                        const float o4 = __shfl_xor_sync(FULL, hx ? s4[0] : s4[1], 16);
                        const float h3 = (hx ? s3[1] : s3[0]) + o3, h4 = (hx ? s4[1] : s4[0]) + o4;
                        const int e = jx + 16 * i;
                        if (e < P) {
                            const int a = ebA[i], b = ebB[i];
                            const float h = h3 + h4;
                            sh.H[hx][a][b] = h;
                            sh.H[hx][b][a] = h;
                            const float gce = fmaf(0.5f, h3, h4 * (1.0f / 3.0f));
                            sh.Gc[hx][a][b] = gce;
                            sh.Gc[hx][b][a] = gce;
                            const float vc = fmaf(1.0f / 6.0f, h3, h4 * (1.0f / 12.0f));
                            vp = fmaf(a == b ? vc : 2.0f * vc, sh.qq[hx][e], vp);
                        }
                    }
                    vpart = vp;   // lane ln belongs to group hx = t
                } else
#pragma unroll
                for (int i = 0; i < EPL; ++i) {
                    const int e = g + i * G;
                    if (e < P) {
                        const Real h3 = use3 ? dot16<Real, S3>(sT3 + e * S3, sh.qr[t]) : Real(0);
                        const Real h4 = use4 ? dot16<Real, S4>(sT4 + e * S4, sh.qq[t]) : Real(0);
                        const int a = ea[i], b = eb[i];
                        // coupling part only: the mode lanes add the diagonal term below
                        const Real h = h3 + h4;
                        sh.H[t][a][b] = h;
                        sh.H[t][b][a] = h;
                        const Real gce = fma(Real(0.5), h3, h4 * Real(1.0 / 3.0));
                        sh.Gc[t][a][b] = gce;
                        sh.Gc[t][b][a] = gce;
                        const Real vc = fma(Real(1.0 / 6.0), h3, h4 * Real(1.0 / 12.0));
                        vpart = fma(a == b ? vc : Real(2) * vc, sh.qq[t][e], vpart);
                    }
                }
                __syncwarp();
                // gradient, p and action (mode lanes)
                Real vlane = vpart;
                if (g < F) {
                    const Real gr = dot16<Real, S3>(sh.Gc[t][g], sh.qr[t]);
                    Real Vd, gd, hd;   // the separable diagonal: value, gradient, Hessian
                    if (pes.diag_kind == SCIVR_DIAG_MORSE) {
                        const Real Dm = c_D<Real>(cc, g), am = c_a<Real>(cc, g);
                        const Real u = rexp<Real>(-am * sh.qr[t][g]);
                        const Real omu = Real(1) - u;
                        Vd = Dm * omu * omu;
                        gd = Real(2) * Dm * am * u * omu;
                        hd = Real(2) * Dm * am * am * u * (Real(2) * u - Real(1));
                    } else {
                        const Real w2 = c_w2<Real>(cc, g);
                        Vd = Real(0.5) * w2 * sh.qr[t][g] * sh.qr[t][g];
                        gd = w2 * sh.qr[t][g];
                        hd = w2;
                    }
                    sh.H[t][g][g] += hd;
                    p = coord_kick(p, tk, A.tkick_f[sub], A.tkick_lo[sub], gr + gd);
                    pr = (Real)coord_f(p);
                    vlane += Vd;
                }
                __syncwarp();   // H complete before the monodromy kick reads it
                dS = fma(-rtk, vlane, dS);
                // monodromy kick: M_p -= tau H M_q (column lanes; rows of H by 16-byte broadcast loads)
                if constexpr (kPacked) {
                    // packed pairs of H's row entries against pairs of the column's entries
                    constexpr int SH = Sh::SH;
#pragma unroll
                    for (int a = 0; a < F; ++a) {
                        float2 acc[NCOL];
#pragma unroll
                        for (int s = 0; s < NCOL; ++s) acc[s] = make_float2(0.0f, 0.0f);
#pragma unroll
                        for (int b0 = 0; b0 < SH; b0 += 4) {
                            const float4 v = *reinterpret_cast<const float4 *>(&sh.H[t][a][b0]);
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const int b = b0 + 2 * h;
                                const float2 hv = h ? hi2(v) : lo2(v);
#pragma unroll
                                for (int s = 0; s < NCOL; ++s) {
                                    if (b + 1 < F) acc[s] = ffma2(hv, make_float2(Mq[s][b], Mq[s][b + 1]), acc[s]);
                                    else if (b < F) acc[s].x = fmaf(hv.x, Mq[s][b], acc[s].x);
                                }
                            }
                        }
#pragma unroll
                        for (int s = 0; s < NCOL; ++s) Mp[s][a] = fmaf(-rtk, acc[s].x + acc[s].y, Mp[s][a]);
                    }
                } else {
                    using VT = typename V16<Real>::T;
                    constexpr int NV = V16<Real>::N, SH = Sh::SH;
#pragma unroll
                    for (int a = 0; a < F; ++a) {
                        Real acc[NCOL];
#pragma unroll
                        for (int s = 0; s < NCOL; ++s) acc[s] = Real(0);
#pragma unroll
                        for (int b0 = 0; b0 < SH; b0 += NV) {
                            const VT v = *reinterpret_cast<const VT *>(&sh.H[t][a][b0]);
#pragma unroll
                            for (int j = 0; j < NV; ++j)
                                if (b0 + j < F) {
#pragma unroll
                                    for (int s = 0; s < NCOL; ++s) acc[s] = fma(vcomp<Real>(v, j), Mq[s][b0 + j], acc[s]);
                                }
                        }
#pragma unroll
                        for (int s = 0; s < NCOL; ++s) Mp[s][a] = fma(-rtk, acc[s], Mp[s][a]);
                    }
                }
            }
            // ---- stability: det M = det M^T by Gaussian elimination of M^T with partial pivoting ----
            // Column c of M (lane c % G, slot c / G) is row c of M^T.  Stage k picks, among the rows
            // not used yet, the one with the largest |M[k][c]| (an arg-max over the group by warp
            // reduction, ties to the higher row), and every other unused row subtracts its multiple
            // of the pivot row's entries below k.  Rows are marked used instead of being moved; the
            // sign of det is the parity of the order in which they were picked, counted as
            // inversions on the bitmask of unused rows.
            // Cadence: the FP64 path tests every step (flags equal to the oracle's bit for bit);
            // the mixed path tests every kDetMEvery steps, after phase 2 (below).  The FP32
            // threshold (537) sits far above the rounding noise, where a deviation that has
            // grown past it keeps growing (Sec. III.A: chaotic trajectories are the ones removed).
            if constexpr (sizeof(Real) == 8) {
                Real W[NCOL][N2];
#pragma unroll
                for (int s = 0; s < NCOL; ++s)
#pragma unroll
                    for (int a = 0; a < F; ++a) { W[s][a] = Mp[s][a]; W[s][F + a] = Mq[s][a]; }
                Real det = Real(1);
                unsigned long long unused = N2 == 64 ? ~0ull : (1ull << N2) - 1ull;
                unsigned parity = 0u;
                static_for<N2>([&](auto kc) {
                    constexpr int k = decltype(kc)::value;
                    // non-negative floats order like their bit patterns; the low 6 bits carry row + 1
                    // (so a used or idle slot's key 0 never wins), at the cost of 6 mantissa bits of
                    // the comparison
                    unsigned key = 0u;
#pragma unroll
                    for (int s = 0; s < NCOL; ++s) {
                        const int col = g + s * G;
                        if (col < N2 && ((unused >> col) & 1ull)) {
                            float mag;
                            if constexpr (sizeof(Real) == 4) mag = fabsf(W[s][k]); else mag = (float)fabs(W[s][k]);
                            const unsigned kk = (__float_as_uint(mag) & ~63u) | (unsigned)(col + 1);
                            key = kk > key ? kk : key;
                        }
                    }
                    // one full-warp integer max per group (the other groups' lanes contribute 0)
                    unsigned kmax = 0u;
#pragma unroll
                    for (int tt = 0; tt < T; ++tt) {
                        const unsigned r = __reduce_max_sync(FULL, t == tt ? key : 0u);
                        kmax = (t == tt) ? r : kmax;
                    }
                    const int pc = (int)(kmax & 63u) - 1;          // pivot row of M^T
                    const int pl = base + pc % G, ps = pc / G;     // its lane and slot
                    auto sel = [&](int i) -> Real { if constexpr (NCOL == 1) return W[0][i]; else return ps ? W[1][i] : W[0][i]; };
                    const Real pk = __shfl_sync(FULL, sel(k), pl);
                    // FP32: the hardware reciprocal (det M only feeds the stability test, whose FP32
                    // tolerance is far above its ulp-level error); FP64: exact division
                    Real inv;
                    if constexpr (sizeof(Real) == 4) inv = __fdividef(1.0f, pk); else inv = Real(1) / pk;
                    parity ^= (unsigned)__popcll(unused & ((1ull << pc) - 1ull)) & 1u;
                    unused &= ~(1ull << pc);
                    det *= pk;
                    Real l[NCOL];
                    bool elim[NCOL];
#pragma unroll
                    for (int s = 0; s < NCOL; ++s) {
                        const int col = g + s * G;
                        elim[s] = col < N2 && ((unused >> col) & 1ull);
                        l[s] = W[s][k] * inv;
                    }
#pragma unroll
                    for (int i = k + 1; i < N2; ++i) {
                        const Real wp = __shfl_sync(FULL, sel(i), pl);
#pragma unroll
                        for (int s = 0; s < NCOL; ++s)
                            if (elim[s]) W[s][i] = fma(-l[s], wp, W[s][i]);
                    }
                });
                if (parity) det = -det;
                const Real dev = isfinite(det) ? fabs(fma(det, det, Real(-1))) : Real(CUDART_INF);
                stab = dev > stab ? dev : stab;
                Real tolr;
                if constexpr (sizeof(Real) == 4) tolr = A.stab_tol_f; else tolr = A.stab_tol;
                if (dev > tolr) good = false;
                if (c == cnt - 1) detM_last = (double)det;
            }
            // ---- Herman-Kluk matrix column b = g (needs column F + b) ----
            {
                // column F + g sits in lane (F + g) % G; a lane h sends column h (h >= F, slot 0)
                // or column h + G (h < F, slot 1) -- the only one any mode lane asks it for
                const int src = base + (F + (g < F ? g : 0)) % G;
                const int job = t * C + c;
#pragma unroll
                for (int a = 0; a < F; ++a) {
                    Real sp, sq;
                    if constexpr (NCOL == 1) { sp = Mp[0][a]; sq = Mq[0][a]; }
                    else { sp = g >= F ? Mp[0][a] : Mp[1][a]; sq = g >= F ? Mq[0][a] : Mq[1][a]; }
                    const Real mpq = __shfl_sync(FULL, sp, src);
                    const Real mqq = __shfl_sync(FULL, sq, src);
                    if (g < F) {
                        using VT = typename V16<Real>::T;
                        constexpr int NV = V16<Real>::N;
                        Real k4[4];
#pragma unroll
                        for (int j0 = 0; j0 < 4; j0 += NV) {
                            const VT kv = *reinterpret_cast<const VT *>(sAc + 4 * (a * F + g) + j0);
#pragma unroll
                            for (int j = 0; j < NV; ++j) k4[j0 + j] = vcomp<Real>(kv, j);
                        }
                        R2 v;
                        v.x = fma(k4[0], mqq, k4[1] * Mp[0][a]);
                        v.y = fma(k4[2], Mq[0][a], k4[3] * mpq);
                        if constexpr (sizeof(Real) == 4)
                            sh.a_at(job, a * F + g) = make_float4(v.x, v.y, 0.0f, 0.0f);
                        else
                            sh.a_at(job, a * F + g) = v;
                    }
                }
                if (g < F) {
                    sh.pj[g][jswz<JOBS>(g, job)] = pr;   // p did not change since the last kick set pr
                    sh.qj[g][jswz<JOBS>(g, job)] = (Real)coord_f(q);
                }
                // the step's action increment, summed over the group, joins the FP64 action
#pragma unroll
                for (int o = G / 2; o > 0; o >>= 1) dS += __shfl_xor_sync(FULL, dS, o, G);
                if (g == 0) {
                    S = coord_add(S, dS);
                    sj_put(job, S);
                }
            }
        }
        {
            // non-finite state persists, so testing once per chunk marks the same trajectories
            const unsigned bad_bits = __ballot_sync(FULL, (g < F) && !(coord_finite(p) && coord_finite(q)));
            const unsigned gmask = (G == 32 ? FULL : (((1u << G) - 1u) << base));
            if (bad_bits & gmask) good = false;
        }
        __syncwarp();
        // ---------------- phase 2: det A per job ----------------
        const int jc = g;                 // phases 3-4: this lane's step of its trajectory (job t * C + jc)
        const int jb = t * C + jc;
        const bool jvalid = jc < cnt;
        double argA = 0.0;                // arg det A of this lane's job (principal value)
        double2 detA = make_double2(1.0, 0.0);
        if constexpr (sizeof(Real) == 4) {
            // Mixed path: the entries of A are FP32 (formed from the FP32 monodromy) and the
            // elimination runs in double-FP32 on the FP32 pipe, so det A carries FP64-class
            // accuracy for those entries.  LPJ lanes share a job: the rows still to be
            // eliminated are dealt out over them through a permutation (a 4-bit field per row
            // up to F = 16, 5 bits above, in two 64-bit words; positions k.. are the active
            // rows), the pivot is an arg-max of
            // |a_ik|^2 over the job's lanes, and det A is the product of the pivots in FP64,
            // its sign flipped per exchange of the permutation.
            constexpr int LPJ = 32 / JOBS;
            static_assert(LPJ * JOBS == 32, "jobs must tile the warp");
            const int job = ln / LPJ, r = ln % LPJ;
            auto at = [&](int e) -> float4 & { return sh.a_at(job, e); };
            constexpr int PB = F > 16 ? 5 : 4, PPW = 64 / PB;   // bits per field, fields per word
            constexpr unsigned long long PMASK = (1ull << PB) - 1ull;
            unsigned long long perm0 = 0ull, perm1 = 0ull;
#pragma unroll
            for (int i = 0; i < F; ++i) {
                if (i < PPW) perm0 |= (unsigned long long)i << (PB * i);
                else perm1 |= (unsigned long long)i << (PB * (i - PPW));
            }
            auto prow = [&](int pos) -> int {
                return pos < PPW ? (int)((perm0 >> (PB * pos)) & PMASK) : (int)((perm1 >> (PB * (pos - PPW))) & PMASK);
            };
            auto pset = [&](int pos, unsigned long long v) {
                if (pos < PPW) perm0 = (perm0 & ~(PMASK << (PB * pos))) | (v << (PB * pos));
                else perm1 = (perm1 & ~(PMASK << (PB * (pos - PPW)))) | (v << (PB * (pos - PPW)));
            };
            // det A, the product of the pivots: double-FP32 (re, im) times 2^dexp, renormalised by
            // an exact power of two after every factor (the FP32 exponent range alone could overflow)
            ff dr = {1.0f, 0.0f}, di = {0.0f, 0.0f};
            int dexp = 0;
#pragma unroll 1
            for (int k = 0; k < F; ++k) {
                // pivot: the largest |a_ik|^2 (leading words) over the active rows
                float best = -1.0f;
                int bpos = k;
                for (int s0 = k; s0 < F; s0 += LPJ) {
                    const int pos = s0 + r;
                    if (pos < F) {
                        const float4 v = at(prow(pos) * F + k);
                        const float m = fmaf(v.x, v.x, v.y * v.y);
                        if (m > best) { best = m; bpos = pos; }
                    }
                }
#pragma unroll
                for (int o = 1; o < LPJ; o <<= 1) {
                    const float ob = __shfl_xor_sync(FULL, best, o);
                    const int op = __shfl_xor_sync(FULL, bpos, o);
                    if (ob > best || (ob == best && op < bpos)) { best = ob; bpos = op; }
                }
                if (bpos != k) {
                    const unsigned long long a = (unsigned long long)prow(k), b = (unsigned long long)prow(bpos);
                    pset(k, b);
                    pset(bpos, a);
                    dr = {-dr.hi, -dr.lo};
                    di = {-di.hi, -di.lo};
                }
                const int pr = prow(k);
                const float4 pk4 = at(pr * F + k);
                const ff pre = {pk4.x, pk4.z}, pim = {pk4.y, pk4.w};
                {
                    const ff a1 = ff_mul(dr, pre), a2 = ff_mul(di, pim), b1 = ff_mul(dr, pim), b2 = ff_mul(di, pre);
                    dr = ff_add(a1, {-a2.hi, -a2.lo});
                    di = ff_add(b1, b2);
                    const float m = fmaxf(fabsf(dr.hi), fabsf(di.hi));
                    const int eb = (__float_as_int(m) >> 23) & 255;   // biased exponent of the larger part
                    if (eb > 0 && eb < 255) {
                        const float sc = __int_as_float((254 - eb) << 23);   // 2^(127 - eb): the larger part to [1, 2)
                        dr.hi *= sc; dr.lo *= sc; di.hi *= sc; di.lo *= sc;
                        dexp += eb - 127;
                    }
                }
                // 1 / pivot = conj(pivot) / |pivot|^2
                const ff m2 = ff_add(ff_mul(pre, pre), ff_mul(pim, pim));
                const ff rm = ff_recip(m2);
                const ff ir = ff_mul(pre, rm);
                const ff nii = ff_mul(pim, rm);
                const ff ii = {-nii.hi, -nii.lo};
                for (int s0 = k + 1; s0 < F; s0 += LPJ) {
                    const int pos = s0 + r;
                    if (pos < F) {
                        const int row = prow(pos);
                        const float4 aik = at(row * F + k);
                        const ff ar = {aik.x, aik.z}, ai = {aik.y, aik.w};
                        // l = a_ik / pivot
                        const ff zero = {0.0f, 0.0f};
                        const ff lr = ff_sub_mul_add_mul(zero, ai, ii, ar, ir);                       // ar ir - ai ii
                        const ff li = ff_sub_mul_add_mul(zero, {-ar.hi, -ar.lo}, ii, ai, ir);         // ar ii + ai ir
#pragma unroll 2
                        for (int cc = k + 1; cc < F; ++cc) {
                            const float4 pv = at(pr * F + cc);
                            float4 &dst = at(row * F + cc);
                            const float4 av = dst;
                            // a -= l p: re = a.re - lr pr + li pi, im = a.im - lr pi - li pr, i.e.
                            // a - lr u + li v with u = p and v = (pi, -pr), both parts packed
                            const ff2 u = {lo2(pv), hi2(pv)};
                            const ff2 v = {make_float2(pv.y, -pv.x), make_float2(pv.w, -pv.z)};
                            const ff2 n = ff2_sub_mul_add_mul({lo2(av), hi2(av)}, lr, u, li, v);
                            dst = make_float4(n.hi.x, n.hi.y, n.lo.x, n.lo.y);
                        }
                    }
                }
                if (LPJ > 1) __syncwarp();   // rows updated by the job's other lanes feed the next pivot
            }
            if (r == 0) {
                const double mr = (double)dr.hi + (double)dr.lo, mi = (double)di.hi + (double)di.lo;
                sh.argj[job] = atan2(mi, mr);   // the power of two does not change the argument
                sh.detAj[job] = make_double2(ldexp(mr, dexp), ldexp(mi, dexp));
                if (A.amplitude == SCIVR_AMP_HK) sh.lnA[job] = 0.5 * (log(hypot(mr, mi)) + dexp * 0.69314718055994530942);
            }
            __syncwarp();
            if (jvalid) {
                argA = sh.argj[jb];
                detA = sh.detAj[jb];
            }
        } else if (ln >= JOBS) {
            // no job for this lane (wide groups): the in-place elimination must not touch a job's storage
        } else {
            // FP64 path: in-place elimination in FP64, one lane per job, det A as the product of
            // the pivots (no range concern in FP64)
            auto at = [&](int e) -> R2 & { return sh.a_at(ln, e); };
            double dr = 1.0, di = 0.0;
#pragma unroll
            for (int k = 0; k < F; ++k) {
                int piv = k;
                double best;
                {
                    const R2 v = at(k * F + k);
                    best = v.x * v.x + v.y * v.y;
                }
#pragma unroll
                for (int i = k + 1; i < F; ++i) {
                    const R2 v = at(i * F + k);
                    const double m = v.x * v.x + v.y * v.y;
                    if (m > best) { best = m; piv = i; }
                }
                R2 prow[F];
#pragma unroll
                for (int cc = k; cc < F; ++cc) prow[cc] = at(piv * F + cc);
                if (piv != k) {
#pragma unroll
                    for (int cc = k; cc < F; ++cc) at(piv * F + cc) = at(k * F + cc);
                    dr = -dr;
                    di = -di;
                }
                const double kr = prow[k].x, ki = prow[k].y;
                const double nr = fma(dr, kr, -di * ki), ni = fma(dr, ki, di * kr);
                dr = nr;
                di = ni;
                const double rr = recip64(fma(kr, kr, ki * ki));
                const double ir = kr * rr, ii = -ki * rr;
#pragma unroll
                for (int i = k + 1; i < F; ++i) {
                    const R2 aik = at(i * F + k);
                    const double lr = fma(aik.x, ir, -aik.y * ii);
                    const double li = fma(aik.x, ii, aik.y * ir);
#pragma unroll
                    for (int cc = k + 1; cc < F; ++cc) {
                        R2 a = at(i * F + cc);
                        a.x = fma(-lr, prow[cc].x, fma(li, prow[cc].y, a.x));
                        a.y = fma(-lr, prow[cc].y, fma(-li, prow[cc].x, a.y));
                        at(i * F + cc) = a;
                    }
                }
            }
            detA = make_double2(dr, di);
            argA = atan2(di, dr);
            if (A.amplitude == SCIVR_AMP_HK) sh.lnA[ln] = 0.5 * log(hypot(dr, di));
        }
        if constexpr (sizeof(Real) == 4) {
            // det M every kDetMEvery steps and at the last step (at a chunk end: M is unchanged
            // since): rows of M^T in the job matrices' storage, free once det A is done
            // (2F (2F + 1) words per trajectory fit in its 4 F^2 C words), row stride 2F + 1 so
            // that lanes reading one column of different rows hit different banks; a rolled
            // loop keeps the code and registers small
            static_assert(kDetMEvery % C == 0, "det M cadence falls on chunk ends");
            if ((step0 + cnt) % kDetMEvery == 0 || step0 + cnt == A.n_steps) {
                float (*Wm)[N2 + 1] = reinterpret_cast<float (*)[N2 + 1]>(&sh.A[0][0]) + t * N2;
                static_assert(sizeof(float) * T * N2 * (N2 + 1) <= sizeof(sh.A), "det M workspace");
#pragma unroll
                    for (int s = 0; s < NCOL; ++s) {
                        const int col = g + s * G;
                        if (col < N2) {
#pragma unroll
                            for (int a = 0; a < F; ++a) { Wm[col][a] = Mp[s][a]; Wm[col][F + a] = Mq[s][a]; }
                        }
                    }
                    __syncwarp();
                    float det = 1.0f;
                    unsigned long long unused = N2 == 64 ? ~0ull : (1ull << N2) - 1ull;
                    unsigned parity = 0u;
#pragma unroll 1
                    for (int k = 0; k < N2; ++k) {
                        unsigned key = 0u;
#pragma unroll
                        for (int s = 0; s < NCOL; ++s) {
                            const int col = g + s * G;
                            if (col < N2 && ((unused >> col) & 1ull)) {
                                const unsigned kk = (__float_as_uint(fabsf(Wm[col][k])) & ~63u) | (unsigned)(col + 1);
                                key = kk > key ? kk : key;
                            }
                        }
                        // one full-warp integer max per group (the other groups' lanes contribute 0)
                        unsigned kmax = 0u;
#pragma unroll
                        for (int tt = 0; tt < T; ++tt) {
                            const unsigned r = __reduce_max_sync(FULL, t == tt ? key : 0u);
                            kmax = (t == tt) ? r : kmax;
                        }
                        const int pc = (int)(kmax & 63u) - 1;
                        const float pk = Wm[pc][k];
                        const float inv = __fdividef(1.0f, pk);
                        parity ^= (unsigned)__popcll(unused & ((1ull << pc) - 1ull)) & 1u;
                        unused &= ~(1ull << pc);
                        det *= pk;
#pragma unroll
                        for (int s = 0; s < NCOL; ++s) {
                            const int col = g + s * G;
                            if (col < N2 && ((unused >> col) & 1ull)) {
                                const float l = Wm[col][k] * inv;
                                for (int i = k + 1; i < N2; ++i) Wm[col][i] = fmaf(-l, Wm[pc][i], Wm[col][i]);
                            }
                        }
                        __syncwarp();
                    }
                    if (parity) det = -det;
                    const float dev = isfinite(det) ? fabsf(fmaf(det, det, -1.0f)) : CUDART_INF_F;
                    stab = dev > stab ? dev : stab;
                    if (dev > A.stab_tol_f) good = false;
                    detM_last = (double)det;
            }
            __syncwarp();   // the next chunk's phase 1 refills the job matrices
        }
        // ---------------- phase 3: continuous phase (segmented scan) ----------------
        const double arg = argA;
        double arg_prev = __shfl_up_sync(FULL, arg, 1, G);
        if (g == 0) arg_prev = arg_last;
        double d = arg - arg_prev + A.ref_step;
        d = fma(-kTwoPi, rint(d * kInvTwoPi), d);
        double inc = jvalid ? d - A.ref_step : 0.0;
#pragma unroll
        for (int o = 1; o < G; o <<= 1) {
            const double v = __shfl_up_sync(FULL, inc, o, G);
            if (g >= o) inc += v;
        }
        const double theta = theta_last + inc;
        const int lastlane = base + cnt - 1;     // lane of the chunk's last step of this trajectory
        theta_last = __shfl_sync(FULL, theta, lastlane);
        arg_last = __shfl_sync(FULL, arg, lastlane);
        detA_last.x = __shfl_sync(FULL, detA.x, lastlane);
        detA_last.y = __shfl_sync(FULL, detA.y, lastlane);
        if (!isfinite(theta_last)) good = false;
        // ---------------- phase 4: amplitudes (job-parallel) ----------------
        if (jvalid && active) {
            const double S = sj_get(jb);
            for (int x = 0; x < A.n_chi; ++x) {
                if constexpr (sizeof(Real) == 4) {
                    // the overlap's exponent and phase are O(1)-O(10) in size: FP32 from the FP32
                    // state copies; the action and the continuous phase join in FP64, and the
                    // total phase is reduced modulo 2 pi in FP64 before FP32 sine and cosine
                    float rf = 0.0f, imf = 0.0f;
#pragma unroll
                    for (int a = 0; a < F; ++a) {
                        const float pa = sh.pj[a][jswz<JOBS>(a, jb)], qa = sh.qj[a][jswz<JOBS>(a, jb)];
                        const float dq = cc.q_eqf[x][a] - qa, dp = cc.p_eqf[x][a] - pa;
                        rf = fmaf(-cc.qwf[a] * dq, dq, rf);
                        rf = fmaf(-cc.pwf[a] * dp, dp, rf);
                        imf = fmaf(0.5f * (cc.p_eqf[x][a] + pa), dq, imf);
                    }
                    double ph = fma(0.5, theta, (double)imf + S);
                    if (A.amplitude == SCIVR_AMP_HK) {
                        // Herman-Kluk summand: |det A|^{1/2} and the division by the initial
                        // overlap times the sampling weight
                        const double2 o = sh.ov0[x][t];
                        rf = (float)((double)rf - o.x + sh.lnA[jb]);
                        ph -= o.y;
                    }
                    const double red = fma(-kTwoPi, rint(ph * kInvTwoPi), ph);   // FP64 reduction to [-pi, pi]
                    float sf, cf;
                    sincosf((float)red, &sf, &cf);
                    const float mag = expf(rf);
                    const int64_t ia = x * L.chi_stride + jl * L.amp_ld + step0 + jc + 1;
                    if (L.amp_f32) reinterpret_cast<float2 *>(L.amp)[ia] = make_float2(mag * cf, mag * sf);
                    else L.amp[ia] = make_double2((double)(mag * cf), (double)(mag * sf));
                } else {
                    double re = 0.0, im = 0.0;
#pragma unroll
                    for (int a = 0; a < F; ++a) {
                        const double pa = sh.pj[a][jswz<JOBS>(a, jb)], qa = sh.qj[a][jswz<JOBS>(a, jb)];
                        const double dq = cc.q_eq[x][a] - qa, dp = cc.p_eq[x][a] - pa;
                        re = fma(-cc.qw[a] * dq, dq, re);
                        re = fma(-cc.pw[a] * dp, dp, re);
                        im = fma(0.5 * (cc.p_eq[x][a] + pa), dq, im);
                    }
                    double ph = im + S + 0.5 * theta;
                    if (A.amplitude == SCIVR_AMP_HK) {
                        const double2 o = sh.ov0[x][t];
                        re = re - o.x + sh.lnA[jb];
                        ph -= o.y;
                    }
                    double sn, cs;
                    sincos(ph, &sn, &cs);
                    const double mag = exp(re);
                    amp_store(L, x * L.chi_stride + jl * L.amp_ld + step0 + jc + 1, mag * cs, mag * sn);
                }
            }
        }
        if (!isfinite(sj_get(t * C + cnt - 1))) good = false;
        __syncwarp();
    }

    if (active) {
    if (g == 0) L.good[jl] = good ? 1 : 0;
    const FinalDev &fo = L.fin;
    if (g < F) {
        if (fo.p) fo.p[g * n + jl] = coord_get(p);
        if (fo.q) fo.q[g * n + jl] = coord_get(q);
    }
    if (g == 0) {
        if (fo.S) fo.S[jl] = sj_get(t * C + ((A.n_steps - 1) % C));
        if (fo.theta) fo.theta[jl] = theta_last;
        if (fo.detM) fo.detM[jl] = detM_last;
        if (fo.stab) fo.stab[jl] = (double)stab;
        if (fo.detA) { fo.detA[2 * jl] = detA_last.x; fo.detA[2 * jl + 1] = detA_last.y; }
    }
    if (fo.M) {
#pragma unroll
        for (int s = 0; s < NCOL; ++s) {
            const int col = g + s * G;
            if (col < N2) {
#pragma unroll
                for (int a = 0; a < F; ++a) {
                    fo.M[jl * N2 * N2 + a * N2 + col] = (double)Mp[s][a];
                    fo.M[jl * N2 * N2 + (F + a) * N2 + col] = (double)Mq[s][a];
                }
            }
        }
    }
    }
    __syncthreads();   // the caller may restage shared memory next
}

template <int F, int G, typename Real, int WARPS>
__global__ void __launch_bounds__(32 * WARPS, lg_min_ctas<F, G, Real>()) k_propagate_lg(const PropLaunch L)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    lg_body<F, G, Real, WARPS>(L, blockIdx.x, smem_raw);
}

// Batched persistent kernel: CTAs pull (molecule, tile) work items from a
// list sorted by decreasing cost until it is exhausted.  items: device array
// of per-molecule launches (all of this F); work: (item, tile) pairs.
template <int F, int G, typename Real, int WARPS>
__global__ void __launch_bounds__(32 * WARPS, lg_min_ctas<F, G, Real>()) k_propagate_lg_batch(const PropLaunch *__restrict__ items,
                                                                       const int2 *__restrict__ work,
                                                                       int n_work, int *__restrict__ counter)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int next;
    for (;;) {
        if (threadIdx.x == 0) next = atomicAdd(counter, 1);
        __syncthreads();
        const int w = next;
        __syncthreads();
        if (w >= n_work) break;
        const int2 it = work[w];
        lg_body<F, G, Real, WARPS>(items[it.x], it.y, smem_raw);
    }
}

// One persistent launch for molecules of several F: CTAs of four warps pull (molecule,
// tile) work items from one list (all molecules, sorted by decreasing cost) and run the
// body specialised for each item's F.  Above F = 9 the coupling tensors are read from L2
// here, so that no class's shared memory sets the whole launch's occupancy.
template <int... Fs>
__global__ void __launch_bounds__(128, 1) k_propagate_lg_multi(const PropLaunch *__restrict__ items,
                                                               const int2 *__restrict__ work, int n_work,
                                                               int *__restrict__ counter)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int next;
    for (;;) {
        if (threadIdx.x == 0) next = atomicAdd(counter, 1);
        __syncthreads();
        const int w = next;
        __syncthreads();
        if (w >= n_work) break;
        const int2 it = work[w];
        const int F = items[it.x].args.F;
        const bool ran = ((F == Fs ? (lg_body<Fs, mixed_group_lanes(Fs), float, 4, (Fs <= 9)>(items[it.x], it.y, smem_raw),
                                      true)
                                   : false) ||
                          ...);
        (void)ran;
    }
}

}  // namespace lg

template <int F, int G, typename Real, int WARPS, bool STAGED = (F <= 16)>
size_t lg_smem_bytes()
{
    using namespace lg;
    const size_t tensors = TensorLayout<F, Real, STAGED>::bytes;
    const size_t consts = (sizeof(CtaConst<F>) + 15) & ~(size_t)15;
    return tensors + consts + WARPS * sizeof(WarpShared<F, G, Real>);
}

template <int F, int G, typename Real, int WARPS>
cudaError_t launch_lg_batch(const PropLaunch *items, const int2 *work, int n_work, int *counter, int n_sm,
                            cudaStream_t s)
{
    using namespace lg;
    const size_t bytes = lg_smem_bytes<F, G, Real, WARPS>();
    auto kern = k_propagate_lg_batch<F, G, Real, WARPS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    // the largest shared-memory carveout, so that as many CTAs fit as the registers allow
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * WARPS, bytes);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int grid = n_sm * per_sm;
    if (grid > n_work) grid = n_work;
    if (grid < 1) return cudaSuccess;
    kern<<<grid, 32 * WARPS, bytes, s>>>(items, work, n_work, counter);
    return cudaGetLastError();
}

template <int F, int G, typename Real, int WARPS>
cudaError_t launch_lg(const PropLaunch &L, cudaStream_t s)
{
    using namespace lg;
    constexpr int T = 32 / G;
    const size_t bytes = lg_smem_bytes<F, G, Real, WARPS>();
    auto kern = k_propagate_lg<F, G, Real, WARPS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    // the largest shared-memory carveout, so that as many CTAs fit as the registers allow
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    const int64_t per_cta = (int64_t)WARPS * T;
    const int64_t blocks = (L.n_traj + per_cta - 1) / per_cta;
    kern<<<(unsigned)blocks, 32 * WARPS, bytes, s>>>(L);
    return cudaGetLastError();
}

// Launchers instantiated by the prop_lg_*.cu units: lanes per trajectory by F
// (2F columns must fit), warps per CTA, and the batch variants the tuner may pick.
template <int F> constexpr int group_lanes() { return 2 * F <= 8 ? 8 : (2 * F <= 16 ? 16 : 32); }

template <int F> cudaError_t launch_group_mixed(const PropLaunch &L, cudaStream_t s)
{
    constexpr int G = mixed_group_lanes(F);
    return launch_lg<F, G, float, lg::lg_warps<F, G>()>(L, s);
}

template <int F>
cudaError_t launch_group_batch_mixed_F(int warps, const PropLaunch *items, const int2 *work, int n_work,
                                      int *counter, int n_sm, cudaStream_t s)
{
    constexpr int G = mixed_group_lanes(F);
    if constexpr (G == 32 && F > 9) {
        constexpr int W = lg::lg_warps<F, G>();
        if (warps == W) return launch_lg_batch<F, G, float, W>(items, work, n_work, counter, n_sm, s);
    } else if constexpr (G == 32) {
        if (warps == 1) return launch_lg_batch<F, G, float, 1>(items, work, n_work, counter, n_sm, s);
        if (warps == 2) return launch_lg_batch<F, G, float, 2>(items, work, n_work, counter, n_sm, s);
    } else {
        if (warps == 2) return launch_lg_batch<F, G, float, 2>(items, work, n_work, counter, n_sm, s);
        if (warps == 4) return launch_lg_batch<F, G, float, 4>(items, work, n_work, counter, n_sm, s);
    }
    return cudaErrorInvalidValue;
}

// The classes one persistent launch can hold, and the trajectories per work tile of each.
template <int... Fs>
struct MultiLaunch {
    static constexpr bool holds(int F) { return ((F == Fs) || ...); }
    static size_t smem_bytes()
    {
        size_t m = 0;
        ((m = std::max(m, lg_smem_bytes<Fs, mixed_group_lanes(Fs), float, 4, (Fs <= 9)>())), ...);
        return m;
    }
    static cudaError_t launch(const PropLaunch *items, const int2 *work, int n_work, int *counter, int n_sm,
                              cudaStream_t s)
    {
        const size_t bytes = smem_bytes();
        auto kern = lg::k_propagate_lg_multi<Fs...>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, bytes);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        int grid = n_sm * per_sm;
        if (grid > n_work) grid = n_work;
        if (grid < 1) return cudaSuccess;
        kern<<<grid, 128, bytes, s>>>(items, work, n_work, counter);
        return cudaGetLastError();
    }
};

template <int F> cudaError_t launch_group_fp64(const PropLaunch &L, cudaStream_t s)
{
    return launch_lg<F, group_lanes<F>(), double, group_lanes<F>() == 32 ? 2 : 4>(L, s);
}


}  // namespace scivr
