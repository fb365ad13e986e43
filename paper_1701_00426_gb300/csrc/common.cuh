// common.cuh -- geometry, double-float arithmetic and small device helpers
// shared by the sm_103a kernels of liblqcd.
//
// Geometry follows the paper's half-lattice index (Sec. 4.1, Eq.
// lexicographic_eo): idxh = (x0 + N0 (x1 + N1 (x2 + N2 x3))) / 2 over the
// sites of one parity, all sides even.  Staggered phases and the
// antiperiodic time boundary are computed from coordinates (no phase array).
//
// Double-float ("df64") arithmetic: an FP64 quantity is carried as an
// unevaluated sum hi + lo of two binary32 numbers (48 significant bits).
// GB300 issues FP64 FMA/ADD at ~1/70 of its FP32 rate, so every per-element
// FP64 product and sum of the hot path is done with error-free transforms on
// the FP32 pipes instead:
//   two_prod  (Dekker 1971, with FMA): a*b = p + e exactly;
//   two_sum   (Knuth, TAOCP vol. 2):   a+b = s + e exactly;
//   dot accumulation in the style of Ogita, Rump and Oishi's Dot2 (2005):
//   the rounded products are summed with two_sum, every rounding error is
//   collected in a second float and added back at the end.
// All operations use the _rn intrinsics so that nvcc never contracts them
// into FMAs (contraction would break the error-free transforms).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_fp16.h>

namespace lqcd {

constexpr int kTile = 256;          // sites per tile (= threads per block of tiled kernels)
constexpr int kMaxShifts = 32;
constexpr int kMaxJobs = 64;        // lattices / requests per packed launch

// ------------------------------------------------------------------ fast division
// Division by a runtime-invariant divisor (Granlund & Montgomery 1994,
// round-up multiplier form), exact for 0 <= n < 2^31.
struct FastDiv {
    uint32_t d, m, s;
};

inline FastDiv make_fastdiv(uint32_t d)
{
    FastDiv f;
    f.d = d;
    uint32_t l = 0;
    while ((1ull << l) < d) ++l;
    f.s = l;
    f.m = (uint32_t)((((1ull << 32) * ((1ull << l) - d)) / d) + 1);
    return f;
}

__host__ __device__ __forceinline__ uint32_t umulhi32(uint32_t a, uint32_t b)
{
#ifdef __CUDA_ARCH__
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

__host__ __device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv &f)
{
    return (umulhi32(n, f.m) + n) >> f.s;
}

// ------------------------------------------------------------------ geometry
struct Geom {
    int N[4];        // sides
    int N0h;         // N0 / 2
    int Vh;          // sites per parity
    int s1, s2, s3;  // half-index strides of directions 1..3 (s0 handled apart)
    FastDiv d0h, d1, d2;
};

inline Geom make_geom(const int dims[4])
{
    Geom g;
    for (int i = 0; i < 4; ++i) g.N[i] = dims[i];
    g.N0h = dims[0] / 2;
    g.Vh = g.N0h * dims[1] * dims[2] * dims[3];
    g.s1 = g.N0h;
    g.s2 = g.N0h * dims[1];
    g.s3 = g.N0h * dims[1] * dims[2];
    g.d0h = make_fastdiv(g.N0h);
    g.d1 = make_fastdiv(dims[1]);
    g.d2 = make_fastdiv(dims[2]);
    return g;
}

// Coordinates of one output site (half index i, parity P), kept in registers.
struct Stencil {
    int i, x0, x1, x2, x3, rest;  // rest = i - x0h (half index of x0 = 0, 1)
};

__host__ __device__ __forceinline__ void make_stencil(const Geom &g, int i, int P, Stencil &S)
{
    const uint32_t q0 = fdiv((uint32_t)i, g.d0h);
    const int x0h = i - (int)q0 * g.N0h;
    const uint32_t q1 = fdiv(q0, g.d1);
    S.x1 = (int)q0 - (int)q1 * g.N[1];
    const uint32_t q2 = fdiv(q1, g.d2);
    S.x2 = (int)q1 - (int)q2 * g.N[2];
    S.x3 = (int)q2;
    S.x0 = 2 * x0h + ((S.x1 + S.x2 + S.x3 + P) & 1);
    S.rest = i - x0h;
    S.i = i;
}

// ------------------------------------------------------------------ bounds-checked builds
// Built with -DLQCD_CHECK_BOUNDS, every neighbour index a kernel computes
// (hop, the gauge kernels' site_of, the staged link stream's tile offsets)
// is compared with its array extent before it is used.  An index out of
// range is replaced by 0, an element in range, and bit 0 of the
// translation unit's error word is set; lqcd_bounds_errors() reads and
// clears the words.  Nothing traps, so the kernel runs to completion and
// the context stays usable.  In the default build the check compiles to
// nothing.
#ifdef LQCD_CHECK_BOUNDS
static __device__ unsigned int g_lqcd_bounds_err;
#endif

__host__ __device__ __forceinline__ int bound_index(int idx, int n)
{
#if defined(LQCD_CHECK_BOUNDS) && defined(__CUDA_ARCH__)
    if ((unsigned)idx < (unsigned)n) return idx;
    atomicOr(&g_lqcd_bounds_err, 1u);
    return 0;
#else
    (void)n;
    return idx;
#endif
}

#ifdef LQCD_CHECK_BOUNDS
// Host side: each translation unit registers a reader of its own word.
using BoundsReader = unsigned (*)();
void register_bounds_reader(BoundsReader f);  // api.cu
static unsigned read_bounds_word()
{
    unsigned v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, g_lqcd_bounds_err, sizeof v) != cudaSuccess ||
        cudaMemcpyToSymbol(g_lqcd_bounds_err, &z, sizeof z) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return v;
}
static const int g_lqcd_bounds_registered = (register_bounds_reader(read_bounds_word), 0);
#endif

// Hop mu of site S: half indices of n+mu (fwd) and n-mu (bwd) and the sign
// masks (0 or 0x80000000) of their contributions.  The forward hop adds
// +s_mu(n) U_mu(n) psi(n+mu), the backward hop -s_mu(n-mu) U_mu(n-mu)^dag
// psi(n-mu); eta_mu(n-mu) = eta_mu(n) because eta_mu depends on x_nu, nu < mu
// only: eta_0 = 1, eta_1 = (-1)^x0, eta_2 = (-1)^(x0+x1), eta_3 =
// (-1)^(x0+x1+x2); the time links at x3 = N3-1 carry the antiperiodic -1.
__host__ __device__ __forceinline__ void hop(const Geom &g, const Stencil &S, int mu, int &fwd, int &bwd,
                                             uint32_t &neg_f, uint32_t &neg_b)
{
    if (mu == 0) {
        const int xf = (S.x0 + 1 == g.N[0]) ? 0 : S.x0 + 1;
        const int xb = (S.x0 == 0) ? g.N[0] - 1 : S.x0 - 1;
        fwd = bound_index(S.rest + (xf >> 1), g.Vh);
        bwd = bound_index(S.rest + (xb >> 1), g.Vh);
        neg_f = 0u;
        neg_b = 1u << 31;
        return;
    }
    const int x = mu == 1 ? S.x1 : (mu == 2 ? S.x2 : S.x3);
    const int n = g.N[mu];
    const int st = mu == 1 ? g.s1 : (mu == 2 ? g.s2 : g.s3);
    fwd = bound_index((x == n - 1) ? S.i - (n - 1) * st : S.i + st, g.Vh);
    bwd = bound_index((x == 0) ? S.i + (n - 1) * st : S.i - st, g.Vh);
    const int esum = mu == 1 ? S.x0 : (mu == 2 ? S.x0 + S.x1 : S.x0 + S.x1 + S.x2);
    uint32_t e = (uint32_t)(esum & 1);
    const uint32_t tf = (mu == 3 && x == n - 1) ? 1u : 0u;
    const uint32_t tb = (mu == 3 && x == 0) ? 1u : 0u;
    neg_f = (e ^ tf) << 31;
    neg_b = (1u ^ e ^ tb) << 31;
}

// ------------------------------------------------------------------ df64 primitives
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e)
{
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// Dot2-style accumulator: value = s + c.
struct Acc2 {
    float s, c;
};

__device__ __forceinline__ void acc_zero(Acc2 &A) { A.s = 0.f; A.c = 0.f; }

// A += (ah + al) * (bh + bl); the al*bl term (relative 2^-48) is dropped.
// The rounding errors of the product and of the sum and the two cross terms
// (all ~2^-24 of the product) are first added together, then once into c.
__device__ __forceinline__ void acc_prod(Acc2 &A, float ah, float al, float bh, float bl)
{
    float p, e, s, t;
    two_prod(ah, bh, p, e);
    two_sum(A.s, p, s, t);
    A.s = s;
    float tmp = __fadd_rn(t, e);
    tmp = __fmaf_rn(ah, bl, tmp);
    tmp = __fmaf_rn(al, bh, tmp);
    A.c = __fadd_rn(A.c, tmp);
}

// Same, with the small terms collected in a separate per-hop accumulator
// ch (added into A.c once per hop by acc_flush): fewer roundings at the
// magnitude of the running error sum.
__device__ __forceinline__ void acc_prod_h(Acc2 &A, float &ch, float ah, float al, float bh, float bl)
{
    float p, e, s, t;
    two_prod(ah, bh, p, e);
    two_sum(A.s, p, s, t);
    A.s = s;
    float tmp = __fadd_rn(t, e);
    tmp = __fmaf_rn(ah, bl, tmp);
    tmp = __fmaf_rn(al, bh, tmp);
    ch = __fadd_rn(ch, tmp);
}

__device__ __forceinline__ void acc_flush(Acc2 &A, float &ch)
{
    A.c = __fadd_rn(A.c, ch);
    ch = 0.f;
}

// A += (bh + bl) (plain df64 value, no product)
__device__ __forceinline__ void acc_add(Acc2 &A, float bh, float bl)
{
    float s, t;
    two_sum(A.s, bh, s, t);
    A.s = s;
    A.c = __fadd_rn(A.c, __fadd_rn(t, bl));
}

// Normalise s + c into (hi, lo) with |lo| <= ulp(hi)/2.
__device__ __forceinline__ float2 acc_result(const Acc2 &A)
{
    float h, l;
    two_sum(A.s, A.c, h, l);
    return make_float2(h, l);
}

// Merge two accumulators (used by warp reductions).
__device__ __forceinline__ void acc_merge(Acc2 &A, float s2, float c2)
{
    float s, t;
    two_sum(A.s, s2, s, t);
    A.s = s;
    A.c = __fadd_rn(__fadd_rn(A.c, c2), t);
}

// df64 value helpers on float2 = (hi, lo)
__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }

// a*b (both df64), normalised
__device__ __forceinline__ float2 df_mul(float2 a, float2 b)
{
    float p, e;
    two_prod(a.x, b.x, p, e);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    float h, l;
    fast_two_sum(p, e, h, l);
    return make_float2(h, l);
}

// a + b (both df64), normalised ("sloppy" add: relative error ~2^-47 of |a|+|b|)
__device__ __forceinline__ float2 df_add(float2 a, float2 b)
{
    float s, e;
    two_sum(a.x, b.x, s, e);
    e = __fadd_rn(e, __fadd_rn(a.y, b.y));
    float h, l;
    fast_two_sum(s, e, h, l);
    return make_float2(h, l);
}

// c + a*b (all df64), normalised
__device__ __forceinline__ float2 df_fma(float2 a, float2 b, float2 c)
{
    float p, e;
    two_prod(a.x, b.x, p, e);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    float s, t;
    two_sum(c.x, p, s, t);
    t = __fadd_rn(t, __fadd_rn(c.y, e));
    float h, l;
    fast_two_sum(s, t, h, l);
    return make_float2(h, l);
}

// a*b + c*d (all df64), normalised
__device__ __forceinline__ float2 df_mul2(float2 a, float2 b, float2 c, float2 d)
{
    float p1, e1, p2, e2;
    two_prod(a.x, b.x, p1, e1);
    e1 = __fmaf_rn(a.x, b.y, e1);
    e1 = __fmaf_rn(a.y, b.x, e1);
    two_prod(c.x, d.x, p2, e2);
    e2 = __fmaf_rn(c.x, d.y, e2);
    e2 = __fmaf_rn(c.y, d.x, e2);
    float s, t;
    two_sum(p1, p2, s, t);
    t = __fadd_rn(t, __fadd_rn(e1, e2));
    float h, l;
    fast_two_sum(s, t, h, l);
    return make_float2(h, l);
}

// ------------------------------------------------------------------ FP64 <-> df64
// Split an IEEE double into hi + lo floats with integer operations only (no
// FP64 instruction).  hi = d rounded to 24 significant bits, lo = the signed
// remainder rounded to 24 bits; |d - hi - lo| <= 2^-48 |d|.  Exact zero and
// FP64 subnormals give 0.  Magnitudes outside [2^-60, 2^64) set *bad (the
// caller then recomputes that site in native FP64).
__device__ __forceinline__ float2 split_f64(double d, bool &bad)
{
    const uint32_t hi = (uint32_t)__double2hiint(d);
    const uint32_t lo = (uint32_t)__double2loint(d);
    const uint32_t e = (hi >> 20) & 0x7FFu;
    const bool zero = (e == 0u);
    bad |= (!zero) && ((e - 963u) > (1086u - 963u));
    const uint32_t rb = (lo >> 28) & 1u;  // first dropped significand bit
    // |hi|: exponent rebased 1023 -> 127, 23 fraction bits, rounded to nearest
    const uint32_t hmag = (__funnelshift_l(lo, hi - (896u << 20), 3) & 0x7FFFFFFFu) + rb;
    const uint32_t hb = hmag | (hi & 0x80000000u);
    // remainder in units of 2^(e-1075): the 29 dropped bits, or 2^29 minus them
    // (opposite sign) when hi was rounded up; |rem| <= 2^28.
    const uint32_t m = lo & 0x1FFFFFFFu;
    const uint32_t mag = rb ? (0x20000000u - m) : m;
    // lo = Y + round(mag / 32) ulp(Y) - Y with Y = 2^(e-1047), ulp(Y) = 2^(e-1070):
    // the integer add builds the float exactly, the subtraction is exact.
    const uint32_t yb = ((hi & 0x80000000u) ^ (rb << 31)) | ((e - 920u) << 23);
    const uint32_t xb = yb + ((mag + 16u) >> 5);
    const float h = __uint_as_float(hb);
    const float l = __fsub_rn(__uint_as_float(xb), __uint_as_float(yb));
    return zero ? make_float2(0.f, 0.f) : make_float2(h, l);
}

// df64 -> nearest-ish IEEE double (two conversions and one FP64 add).
__device__ __forceinline__ double df_to_f64(float2 a)
{
    return (double)a.x + (double)a.y;
}

__device__ __forceinline__ float2 f64_to_df_slow(double d)
{
    const float h = __double2float_rn(d);
    const float l = __double2float_rn(d - (double)h);
    return make_float2(h, l);
}

__device__ __forceinline__ float2 xor_sign(float2 a, uint32_t m)
{
    return make_float2(__uint_as_float(__float_as_uint(a.x) ^ m), __uint_as_float(__float_as_uint(a.y) ^ m));
}

__device__ __forceinline__ float4 xor_sign4(float4 a, uint32_t m)
{
    return make_float4(__uint_as_float(__float_as_uint(a.x) ^ m), __uint_as_float(__float_as_uint(a.y) ^ m),
                       __uint_as_float(__float_as_uint(a.z) ^ m), __uint_as_float(__float_as_uint(a.w) ^ m));
}

// ------------------------------------------------------------------ reductions
// Warp-level sum of a df64 accumulator; the result is valid in lane 0.
__device__ __forceinline__ void warp_reduce_acc(Acc2 &A)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_down_sync(0xFFFFFFFFu, A.s, o);
        const float c2 = __shfl_down_sync(0xFFFFFFFFu, A.c, o);
        acc_merge(A, s2, c2);
    }
}

// Block-level deterministic reduction of per-thread df64 values into a
// double written by thread 0 (fixed order: lane tree, then warps in order).
template <int NT>
__device__ __forceinline__ double block_reduce_acc(Acc2 A, double *smem /* NT/32 doubles */)
{
    warp_reduce_acc(A);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) smem[w] = (double)A.s + (double)A.c;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NT / 32; ++k) r += smem[k];
    }
    return r;
}

// ------------------------------------------------------------------ load helpers
__device__ __forceinline__ float4 ldg4(const float4 *p) { return __ldg(p); }

// Loads of data streamed once per kernel (links): read-only path with an L2
// evict-first policy, so that the neighbour spinors and Krylov vectors that
// are re-read stay in L2.  Compiled out with -DLQCD_NO_L2_HINTS.
__device__ __forceinline__ uint64_t l2_evict_first_policy()
{
#ifdef LQCD_NO_L2_HINTS
    return 0;
#else
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
#endif
}

__device__ __forceinline__ float4 ldg4_stream(const float4 *p, uint64_t pol)
{
#ifdef LQCD_NO_L2_HINTS
    (void)pol;
    return __ldg(p);
#else
    float4 v;
    asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p), "l"(pol));
    return v;
#endif
}
__device__ __forceinline__ float2 ldg2(const float2 *p) { return __ldg(p); }

// 8- and 16-byte streamed loads with the evict-first policy (FP32 / FP16 links)
__device__ __forceinline__ float2 ldg2_stream(const float2 *p, uint64_t pol)
{
#ifdef LQCD_NO_L2_HINTS
    (void)pol;
    return __ldg(p);
#else
    float2 v;
    asm volatile("ld.global.nc.L2::cache_hint.v2.f32 {%0,%1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(p), "l"(pol));
    return v;
#endif
}

__device__ __forceinline__ uint4 ldg4u_stream(const uint4 *p, uint64_t pol)
{
#ifdef LQCD_NO_L2_HINTS
    (void)pol;
    return __ldg(p);
#else
    uint4 v;
    asm volatile("ld.global.nc.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p), "l"(pol));
    return v;
#endif
}

__device__ __forceinline__ uint2 ldg2u_stream(const uint2 *p, uint64_t pol)
{
#ifdef LQCD_NO_L2_HINTS
    (void)pol;
    return __ldg(p);
#else
    uint2 v;
    asm volatile("ld.global.nc.L2::cache_hint.v2.u32 {%0,%1}, [%2], %3;" : "=r"(v.x), "=r"(v.y) : "l"(p), "l"(pol));
    return v;
#endif
}
__device__ __forceinline__ double2 ldg2d(const double2 *p) { return __ldg(p); }

// Streaming loads/stores for data touched once per kernel (Krylov vectors).
__device__ __forceinline__ float4 ld_stream4(const float4 *p) { return __ldcs(p); }
__device__ __forceinline__ void st_stream4(float4 *p, float4 v) { __stcs(p, v); }

}  // namespace lqcd
