// deo_core.cuh -- the staggered hopping term D_eo / D_oe (Sec. 2.2,
// Eq. diracblock) as sm_103a device code, in four arithmetics:
//
//   DF   links stored as df64 pairs (hi, lo floats; 18 reals -> 9 float4 per
//        link), spinors df64 (float4 per complex) or IEEE complex128; every
//        product and sum done with error-free FP32 transforms (common.cuh);
//   F32  FP32 links (18 reals as 9 float2, or 12 reals as 3 float4 with the
//        third row rebuilt, Sec. 2.3) and FP32 spinors (float2 per complex);
//   F16  FP16 links, 12 reals (uint4 + uint2 per link), FP32 spinors/math;
//   NAT  IEEE links and spinors with native FP64 FMA (reference variant).
//
// One thread computes one output site n of parity P:
//   out(n) = 1/2 sum_mu [ s_mu(n) U_mu(n) in(n+mu) - s_mu(n-mu) U_mu(n-mu)^dag in(n-mu) ]
// Links of direction mu are stored per parity of their base site, indexed by
// the base site's half index: the forward link of n sits in (mu, P) at n's
// own index and the backward link U_mu(n-mu) in (mu, 1-P) at the neighbour's
// index, so each link is read exactly once per application.
// All link arrays are structure-of-arrays over the half lattice
// (component-major, site fastest): every load of a warp is one contiguous
// 128-bit-per-thread stream.
#pragma once

#include "common.cuh"

namespace lqcd {

// Link storage formats
enum LinkFmt { LF_DF18 = 0, LF_F32_18 = 1, LF_F32_12 = 2, LF_F16_12 = 3, LF_NAT18 = 4 };
// Spinor formats
enum SpinFmt { SF_DF = 0, SF_IEEE = 1, SF_F32 = 2 };

// Offsets: the link array of (mu, parity) starts at (mu*2 + par) * comps * Vh.
__device__ __forceinline__ size_t link_base(int mu, int par, int comps, int Vh)
{
    return (size_t)((mu * 2 + par) * comps) * (size_t)Vh;
}

// ------------------------------------------------------------------ DF hops
// U component c = (re_h, re_l, im_h, im_l); v component likewise.
__device__ __forceinline__ void hop_fwd_df(Acc2 (&acc)[6], float (&ch)[6], const float4 (&U)[9], const float4 (&v)[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const float4 u = U[a * 3 + b], w = v[b];
            acc_prod_h(acc[2 * a], ch[2 * a], u.x, u.y, w.x, w.y);          // + ur vr
            acc_prod_h(acc[2 * a], ch[2 * a], -u.z, -u.w, w.z, w.w);        // - ui vi
            acc_prod_h(acc[2 * a + 1], ch[2 * a + 1], u.x, u.y, w.z, w.w);  // + ur vi
            acc_prod_h(acc[2 * a + 1], ch[2 * a + 1], u.z, u.w, w.x, w.y);  // + ui vr
        }
}

// (U^dag v)_a = sum_b conj(U_ba) v_b
__device__ __forceinline__ void hop_bwd_df(Acc2 (&acc)[6], float (&ch)[6], const float4 (&U)[9], const float4 (&v)[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const float4 u = U[b * 3 + a], w = v[b];
            acc_prod_h(acc[2 * a], ch[2 * a], u.x, u.y, w.x, w.y);          // + ur vr
            acc_prod_h(acc[2 * a], ch[2 * a], u.z, u.w, w.z, w.w);          // + ui vi
            acc_prod_h(acc[2 * a + 1], ch[2 * a + 1], u.x, u.y, w.z, w.w);  // + ur vi
            acc_prod_h(acc[2 * a + 1], ch[2 * a + 1], -u.z, -u.w, w.x, w.y); // - ui vr
        }
}

template <int SF>
__device__ __forceinline__ void load_spinor_df(const void *in, int idx, int Vh, uint32_t neg, float4 (&v)[3], bool &bad)
{
    if (SF == SF_DF) {
        const float4 *p = (const float4 *)in;
#pragma unroll
        for (int c = 0; c < 3; ++c) v[c] = xor_sign4(ldg4(p + (size_t)c * Vh + idx), neg);
    } else {  // IEEE complex128: split on the fly with integer operations
        const double2 *p = (const double2 *)in;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double2 d = ldg2d(p + (size_t)c * Vh + idx);
            const float2 re = split_f64(d.x, bad), im = split_f64(d.y, bad);
            v[c] = xor_sign4(make_float4(re.x, re.y, im.x, im.y), neg);
        }
    }
}

// a0 b0 + a1 b1 + a2 b2 + a3 b3 for df64 factors (hi, lo), returned as a
// normalised df64 pair.  The products of the high parts are split exactly
// (two_prod) and their rounded values summed with two_sum; the product
// errors, the sum errors and the mixed high-low products (relative 2^-24 of
// a product) are added together in FP32 and once to the sum at the end.
// Low-low products (relative 2^-48) are dropped.
__device__ __forceinline__ float2 df_dot4(float2 a0, float2 b0, float2 a1, float2 b1, float2 a2, float2 b2,
                                          float2 a3, float2 b3)
{
    float p0, e0, p1, e1, p2, e2, p3, e3;
    two_prod(a0.x, b0.x, p0, e0);
    two_prod(a1.x, b1.x, p1, e1);
    two_prod(a2.x, b2.x, p2, e2);
    two_prod(a3.x, b3.x, p3, e3);
    e0 = __fmaf_rn(a0.x, b0.y, __fmaf_rn(a0.y, b0.x, e0));
    e1 = __fmaf_rn(a1.x, b1.y, __fmaf_rn(a1.y, b1.x, e1));
    e2 = __fmaf_rn(a2.x, b2.y, __fmaf_rn(a2.y, b2.x, e2));
    e3 = __fmaf_rn(a3.x, b3.y, __fmaf_rn(a3.y, b3.x, e3));
    float s, t0, t1, t2;
    two_sum(p0, p1, s, t0);
    two_sum(s, p2, s, t1);
    two_sum(s, p3, s, t2);
    const float err = __fadd_rn(__fadd_rn(__fadd_rn(t0, t1), t2), __fadd_rn(__fadd_rn(e0, e1), __fadd_rn(e2, e3)));
    float h, l;
    two_sum(s, err, h, l);
    return make_float2(h, l);
}

// Third row of an SU(3) link from its first two (Sec. 2.3, 12 reals per
// link): r2 = conj(r0 x r1), component k = conj(a_i b_j - a_j b_i) with
// (i, j) = (k+1, k+2) mod 3, a = r0, b = r1, in df64 (components are
// (re_h, re_l, im_h, im_l)).  Exact for an SU(3) matrix up to the df64
// rounding of each component (a few 2^-48 of the largest entry).
__device__ __forceinline__ void reconstruct_row2_df(float4 (&U)[9])
{
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int i = (k + 1) % 3, j = (k + 2) % 3;
        const float4 a_i = U[i], a_j = U[j], b_i = U[3 + i], b_j = U[3 + j];
        const float2 air = make_float2(a_i.x, a_i.y), aii = make_float2(a_i.z, a_i.w);
        const float2 ajr = make_float2(a_j.x, a_j.y), aji = make_float2(a_j.z, a_j.w);
        const float2 bir = make_float2(b_i.x, b_i.y), bii = make_float2(b_i.z, b_i.w);
        const float2 bjr = make_float2(b_j.x, b_j.y), bji = make_float2(b_j.z, b_j.w);
        // re(a_i b_j - a_j b_i) = air bjr - aii bji - ajr bir + aji bii
        const float2 re = df_dot4(air, bjr, df_neg(aii), bji, df_neg(ajr), bir, aji, bii);
        // im(a_i b_j - a_j b_i) = air bji + aii bjr - ajr bii - aji bir
        const float2 im = df_dot4(air, bji, aii, bjr, df_neg(ajr), bii, df_neg(aji), bir);
        U[6 + k] = make_float4(re.x, re.y, -im.x, -im.y);
    }
}

// RECON 18: all nine components streamed; RECON 12: the first two rows
// (components 0..5 of the same arrays, 96 of the 144 bytes) streamed and
// the third row rebuilt.
template <int RECON = 18>
__device__ __forceinline__ void load_link_df(const float4 *L, int mu, int par, int idx, int Vh, float4 (&U)[9])
{
    const float4 *p = L + link_base(mu, par, 9, Vh) + idx;
    const uint64_t pol = l2_evict_first_policy();
#pragma unroll
    for (int c = 0; c < (RECON == 12 ? 6 : 9); ++c) U[c] = ldg4_stream(p + (size_t)c * Vh, pol);
    if (RECON == 12) reconstruct_row2_df(U);
}

// D applied at one site in df64.  Returns the six (re, im) x colour results
// as normalised df64 pairs, already multiplied by 1/2.
template <int SF, int RECON = 18>
__device__ __forceinline__ void deo_site_df(const Geom &g, const float4 *L, const void *in, const Stencil &S, int i,
                                            int P, int Vh, float2 (&res)[6], bool &bad)
{
    Acc2 acc[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) acc_zero(acc[k]);
#pragma unroll 1
    for (int mu = 0; mu < 4; ++mu) {
        int f, b;
        uint32_t nf, nb;
        hop(g, S, mu, f, b, nf, nb);
        float4 U[9], v[3];
        float ch[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        load_link_df<RECON>(L, mu, P, i, Vh, U);
        load_spinor_df<SF>(in, f, Vh, nf, v, bad);
        hop_fwd_df(acc, ch, U, v);
        load_link_df<RECON>(L, mu, 1 - P, b, Vh, U);
        load_spinor_df<SF>(in, b, Vh, nb, v, bad);
        hop_bwd_df(acc, ch, U, v);
#pragma unroll
        for (int k = 0; k < 6; ++k) acc_flush(acc[k], ch[k]);
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const float2 r = acc_result(acc[k]);
        res[k] = make_float2(0.5f * r.x, 0.5f * r.y);
    }
}

// Native FP64 evaluation of one site from df64 links and IEEE spinors: the
// fallback for sites whose inputs fall outside the df64 exponent window.
static __device__ __noinline__ void deo_site_native_from_df(const Geom &g, const float4 *L, const double2 *in,
                                                            const Stencil &S, int i, int P, int Vh, double2 (&res)[3])
{
    double2 acc[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int mu = 0; mu < 4; ++mu) {
        int f, b;
        uint32_t nf, nb;
        hop(g, S, mu, f, b, nf, nb);
        for (int dir = 0; dir < 2; ++dir) {
            const int idx = dir == 0 ? f : b;
            const int par = dir == 0 ? P : 1 - P;
            const int lidx = dir == 0 ? i : b;
            const double sg = ((dir == 0 ? nf : nb) != 0u) ? -1.0 : 1.0;
            const float4 *lp = L + link_base(mu, par, 9, Vh) + lidx;
            double2 v[3];
            for (int c = 0; c < 3; ++c) v[c] = in[(size_t)c * Vh + idx];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    const float4 u4 = lp[(size_t)(dir == 0 ? a * 3 + b : b * 3 + a) * Vh];
                    const double ur = (double)u4.x + (double)u4.y;
                    double ui = (double)u4.z + (double)u4.w;
                    if (dir == 1) ui = -ui;
                    acc[a].x += sg * (ur * v[b].x - ui * v[b].y);
                    acc[a].y += sg * (ur * v[b].y + ui * v[b].x);
                }
        }
    }
    for (int a = 0; a < 3; ++a) res[a] = make_double2(0.5 * acc[a].x, 0.5 * acc[a].y);
}

// ------------------------------------------------------------------ native FP64 (reference)
__device__ __forceinline__ void deo_site_nat(const Geom &g, const double2 *L, const double2 *in, const Stencil &S,
                                             int i, int P, int Vh, double2 (&res)[3])
{
    double2 acc[3] = {{0, 0}, {0, 0}, {0, 0}};
#pragma unroll 1
    for (int mu = 0; mu < 4; ++mu) {
        int f, b;
        uint32_t nf, nb;
        hop(g, S, mu, f, b, nf, nb);
#pragma unroll
        for (int dir = 0; dir < 2; ++dir) {
            const int idx = dir == 0 ? f : b;
            const int par = dir == 0 ? P : 1 - P;
            const int lidx = dir == 0 ? i : b;
            const double sg = ((dir == 0 ? nf : nb) != 0u) ? -1.0 : 1.0;
            const double2 *lp = L + link_base(mu, par, 9, Vh) + lidx;
            double2 v[3], U[9];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double2 t = ldg2d(in + (size_t)c * Vh + idx);
                v[c] = make_double2(sg * t.x, sg * t.y);
            }
#pragma unroll
            for (int c = 0; c < 9; ++c) U[c] = ldg2d(lp + (size_t)c * Vh);
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    if (dir == 0) {
                        const double2 u = U[a * 3 + b];
                        acc[a].x = fma(u.x, v[b].x, fma(-u.y, v[b].y, acc[a].x));
                        acc[a].y = fma(u.x, v[b].y, fma(u.y, v[b].x, acc[a].y));
                    } else {
                        const double2 u = U[b * 3 + a];
                        acc[a].x = fma(u.x, v[b].x, fma(u.y, v[b].y, acc[a].x));
                        acc[a].y = fma(u.x, v[b].y, fma(-u.y, v[b].x, acc[a].y));
                    }
                }
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) res[a] = make_double2(0.5 * acc[a].x, 0.5 * acc[a].y);
}

// ------------------------------------------------------------------ FP32 / FP16 hops
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(__fmaf_rn(a.x, b.x, -a.y * b.y), __fmaf_rn(a.x, b.y, a.y * b.x));
}

// third row of an SU(3) matrix from the first two: r2 = conj(r0 x r1) (Sec. 2.3)
__device__ __forceinline__ void reconstruct_row2(float2 (&U)[9])
{
    const float2 a0 = U[0], a1 = U[1], a2 = U[2], b0 = U[3], b1 = U[4], b2 = U[5];
    float2 c;
    c = make_float2(a1.x * b2.x - a1.y * b2.y - (a2.x * b1.x - a2.y * b1.y),
                    a1.x * b2.y + a1.y * b2.x - (a2.x * b1.y + a2.y * b1.x));
    U[6] = make_float2(c.x, -c.y);
    c = make_float2(a2.x * b0.x - a2.y * b0.y - (a0.x * b2.x - a0.y * b2.y),
                    a2.x * b0.y + a2.y * b0.x - (a0.x * b2.y + a0.y * b2.x));
    U[7] = make_float2(c.x, -c.y);
    c = make_float2(a0.x * b1.x - a0.y * b1.y - (a1.x * b0.x - a1.y * b0.y),
                    a0.x * b1.y + a0.y * b1.x - (a1.x * b0.y + a1.y * b0.x));
    U[8] = make_float2(c.x, -c.y);
}

__device__ __forceinline__ float2 h2f(uint32_t w)
{
    const __half2 h = *reinterpret_cast<const __half2 *>(&w);
    return __half22float2(h);
}

// Links are streamed once per application: loads carry the L2 evict-first
// policy so that the re-read spinors keep their place in L2.
template <int LF>
__device__ __forceinline__ void load_link_f32(const void *L, int mu, int par, int idx, int Vh, float2 (&U)[9])
{
    const uint64_t pol = l2_evict_first_policy();
    if (LF == LF_F32_18) {
        const float2 *p = (const float2 *)L + link_base(mu, par, 9, Vh) + idx;
#pragma unroll
        for (int c = 0; c < 9; ++c) U[c] = ldg2_stream(p + (size_t)c * Vh, pol);
    } else if (LF == LF_F32_12) {
        const float4 *p = (const float4 *)L + link_base(mu, par, 3, Vh) + idx;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float4 t = ldg4_stream(p + (size_t)k * Vh, pol);
            U[2 * k] = make_float2(t.x, t.y);
            U[2 * k + 1] = make_float2(t.z, t.w);
        }
        reconstruct_row2(U);
    } else {  // LF_F16_12: [8 Vh] uint4 (c00 c01 c02 c10) then [8 Vh] uint2 (c11 c12)
        const uint4 *pa = (const uint4 *)L;
        const uint2 *pb = (const uint2 *)(pa + (size_t)8 * Vh);
        const uint4 a = ldg4u_stream(pa + (size_t)(mu * 2 + par) * Vh + idx, pol);
        const uint2 b = ldg2u_stream(pb + (size_t)(mu * 2 + par) * Vh + idx, pol);
        U[0] = h2f(a.x); U[1] = h2f(a.y); U[2] = h2f(a.z); U[3] = h2f(a.w);
        U[4] = h2f(b.x); U[5] = h2f(b.y);
        reconstruct_row2(U);
    }
}

// UNROLL 4 unrolls the direction loop, so that the compiler may issue the
// link and spinor loads of later hops before the FMAs of earlier ones (more
// bytes in flight per thread, at the cost of registers); the FMAs and their
// order are the same, so are the bits.
template <int LF, int UNROLL = 1>
__device__ __forceinline__ void deo_site_f32(const Geom &g, const void *L, const float2 *in, const Stencil &S, int i,
                                             int P, int Vh, float2 (&res)[3])
{
    float2 acc[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
#pragma unroll UNROLL
    for (int mu = 0; mu < 4; ++mu) {
        int f, b;
        uint32_t nf, nb;
        hop(g, S, mu, f, b, nf, nb);
        float2 U[9], v[3];
        load_link_f32<LF>(L, mu, P, i, Vh, U);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float2 t = ldg2(in + (size_t)c * Vh + f);
            v[c] = make_float2(__uint_as_float(__float_as_uint(t.x) ^ nf),
                               __uint_as_float(__float_as_uint(t.y) ^ nf));
        }
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const float2 u = U[a * 3 + b];
                acc[a].x = __fmaf_rn(u.x, v[b].x, __fmaf_rn(-u.y, v[b].y, acc[a].x));
                acc[a].y = __fmaf_rn(u.x, v[b].y, __fmaf_rn(u.y, v[b].x, acc[a].y));
            }
        load_link_f32<LF>(L, mu, 1 - P, b, Vh, U);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float2 t = ldg2(in + (size_t)c * Vh + b);
            v[c] = make_float2(__uint_as_float(__float_as_uint(t.x) ^ nb),
                               __uint_as_float(__float_as_uint(t.y) ^ nb));
        }
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const float2 u = U[b * 3 + a];
                acc[a].x = __fmaf_rn(u.x, v[b].x, __fmaf_rn(u.y, v[b].y, acc[a].x));
                acc[a].y = __fmaf_rn(u.x, v[b].y, __fmaf_rn(-u.y, v[b].x, acc[a].y));
            }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) res[a] = make_float2(0.5f * acc[a].x, 0.5f * acc[a].y);
}

}  // namespace lqcd
