// gauge.cu -- the gauge part of the molecular dynamics step (Sec. 2.1, the
// tree-level Symanzik improved action; Sec. 4.2 and Algorithm 2, the gauge
// cycle; Listing lst:rect_staples, the staples; Table md-norm, its cost per
// site) in FP64 and in FP32 (Algorithm 1, step 5: "possibly in single
// precision").
//
//   S_g = -(beta/3) sum_x [ c0 sum_{mu<nu} Re Tr P_{mu nu}(x) + c1 sum_{mu!=nu} Re Tr R_{mu nu}(x) ]
//   c0 = 5/3, c1 = -1/12;  P: 1x1 plaquette, R: 2 links along mu, 1 along nu
//   force:  F_mu(x) = traceless part of -(i beta/6)(M - M^dag), M = U_mu(x) A_mu(x)
//   momenta: H <- H - eps F          links: U <- exp(i eps H) U
// where A_mu(x) is the sum of the staples of U_mu(x): c0 times the 3-link
// paths and c1 times the 5-link paths that close the plaquettes and
// rectangles through U_mu(x), for nu != mu and both signs of nu.
//
// Storage: links in the context's SoA formats, [4 mu][2 parity][9 comp][V/2]
// (double2 for FP64 -- the master copy -- and float2 for FP32); momenta as 8
// reals per link (traceless Hermitian: h00, h11, re/im of h01, h02, h12),
// [4][2][8][V/2].  One thread per link.  Neighbour links are gathered through
// L1/L2 (every link is read by ~80 threads of nearby sites).
#include <cmath>
#include <mutex>

#include "deo_core.cuh"
#include "internal.h"

namespace lqcd {

constexpr double kSymC0 = 5.0 / 3.0;
constexpr double kSymC1 = -1.0 / 12.0;
constexpr int kGaugeThreads = 128;

template <class T> struct Cplx { T re, im; };
template <class T> struct Mat3 { Cplx<T> e[9]; };
template <class T> struct Vec2T;
template <> struct Vec2T<double> { using t = double2; };
template <> struct Vec2T<float> { using t = float2; };

template <class T>
__device__ __forceinline__ void mat_mul(const Mat3<T> &a, const Mat3<T> &b, Mat3<T> &c)
{
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            T re = 0, im = 0;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const Cplx<T> x = a.e[i * 3 + k], y = b.e[k * 3 + j];
                re = fma(x.re, y.re, fma(-x.im, y.im, re));
                im = fma(x.re, y.im, fma(x.im, y.re, im));
            }
            c.e[i * 3 + j] = {re, im};
        }
}

// c = a b^dag
template <class T>
__device__ __forceinline__ void mat_mul_dag(const Mat3<T> &a, const Mat3<T> &b, Mat3<T> &c)
{
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            T re = 0, im = 0;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const Cplx<T> x = a.e[i * 3 + k], y = b.e[j * 3 + k];  // conj(b_jk)
                re = fma(x.re, y.re, fma(x.im, y.im, re));
                im = fma(-x.re, y.im, fma(x.im, y.re, im));
            }
            c.e[i * 3 + j] = {re, im};
        }
}

template <class T>
__device__ __forceinline__ void mat_dag(Mat3<T> &a)
{
    Mat3<T> t = a;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) a.e[i * 3 + j] = {t.e[j * 3 + i].re, -t.e[j * 3 + i].im};
}

template <class T>
__device__ __forceinline__ void mat_axpy(T s, const Mat3<T> &x, Mat3<T> &y)
{
#pragma unroll
    for (int i = 0; i < 9; ++i) y.e[i] = {fma(s, x.e[i].re, y.e[i].re), fma(s, x.e[i].im, y.e[i].im)};
}

// ------------------------------------------------------------------ geometry of links
struct LinkGeo {
    int N[4];
    int Vh;
};

__device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// (parity, half index) of x + d, |d_m| <= 2 <= N_m
__device__ __forceinline__ void site_of(const LinkGeo &g, const int (&x)[4], int d0, int d1, int d2, int d3, int &par,
                                        int &idx)
{
    const int y0 = wrap(x[0] + d0, g.N[0]), y1 = wrap(x[1] + d1, g.N[1]);
    const int y2 = wrap(x[2] + d2, g.N[2]), y3 = wrap(x[3] + d3, g.N[3]);
    par = (y0 + y1 + y2 + y3) & 1;
    idx = bound_index((y0 + g.N[0] * (y1 + g.N[1] * (y2 + g.N[2] * y3))) >> 1, g.Vh);
}

template <class T>
__device__ __forceinline__ void load_link_soa(const typename Vec2T<T>::t *__restrict__ L, int mu, int par, int idx,
                                              int Vh, Mat3<T> &U)
{
    const typename Vec2T<T>::t *p = L + (size_t)((mu * 2 + par) * 9) * Vh + idx;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        const typename Vec2T<T>::t v = __ldg(p + (size_t)c * Vh);
        U.e[c] = {v.x, v.y};
    }
}

// Link of the step from x + d in direction s * nu (s = +-1):
// U_nu(x + d) for s = +1, U_nu(x + d - nu)^dag for s = -1.
template <class T>
__device__ __forceinline__ void step_link(const LinkGeo &g, const typename Vec2T<T>::t *L, const int (&x)[4],
                                          const int (&d)[4], int nu, int s, Mat3<T> &U)
{
    int e[4] = {d[0], d[1], d[2], d[3]};
    if (s < 0) e[nu] -= 1;
    int par, idx;
    site_of(g, x, e[0], e[1], e[2], e[3], par, idx);
    load_link_soa<T>(L, nu, par, idx, g.Vh, U);
    if (s < 0) mat_dag(U);
}

// U_mu(x + d)^dag (a step -mu from x + d + mu)
template <class T>
__device__ __forceinline__ void back_mu(const LinkGeo &g, const typename Vec2T<T>::t *L, const int (&x)[4],
                                        const int (&d)[4], int mu, Mat3<T> &U)
{
    int par, idx;
    site_of(g, x, d[0], d[1], d[2], d[3], par, idx);
    load_link_soa<T>(L, mu, par, idx, g.Vh, U);
    mat_dag(U);
}

__device__ __forceinline__ void coords_of(const LinkGeo &g, int P, int i, int (&x)[4])
{
    const int n0h = g.N[0] >> 1;
    int r = i / n0h;
    const int x0h = i - r * n0h;
    x[1] = r % g.N[1];
    r /= g.N[1];
    x[2] = r % g.N[2];
    x[3] = r / g.N[2];
    x[0] = 2 * x0h + ((x[1] + x[2] + x[3] + P) & 1);
}

// Staple sum A of the link U_mu(x) (see the file header).  Prefix sharing
// per (nu, s): P1 = step +s nu from x+mu, Q = P1 U_mu(x+s nu)^dag,
// E = step from x+s nu back to x; plaquette = Q E, rectangle (b) =
// Q U_mu(x-mu+s nu)^dag (step -s nu) U_mu(x-mu), rectangles (a) and (c)
// end in E, so c0 Q + c1 (a' + c') is multiplied by E once.
template <class T>
__device__ void staple_sum_dev(const LinkGeo &g, const typename Vec2T<T>::t *L, const int (&x)[4], int mu,
                               Mat3<T> &A)
{
#pragma unroll
    for (int k = 0; k < 9; ++k) A.e[k] = {T(0), T(0)};
    const T c0 = T(kSymC0), c1 = T(kSymC1);
#pragma unroll 1
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
#pragma unroll 1
        for (int s = -1; s <= 1; s += 2) {
            int d[4] = {0, 0, 0, 0};
            Mat3<T> P1, Q, W, t1, t2;
            // P1 = step(x+mu, s nu)
            d[mu] = 1;
            step_link<T>(g, L, x, d, nu, s, P1);
            // Q = P1 U_mu(x + s nu)^dag
            d[mu] = 0;
            d[nu] = s;
            back_mu<T>(g, L, x, d, mu, t1);
            mat_mul(P1, t1, Q);
            // rectangle (b): Q U_mu(x - mu + s nu)^dag step(x-mu+s nu, -s nu) U_mu(x - mu)
            d[mu] = -1;
            back_mu<T>(g, L, x, d, mu, t1);
            mat_mul(Q, t1, t2);
            step_link<T>(g, L, x, d, nu, -s, t1);
            mat_mul(t2, t1, W);
            d[nu] = 0;
            {
                int par, idx;
                site_of(g, x, d[0], d[1], d[2], d[3], par, idx);
                load_link_soa<T>(L, mu, par, idx, g.Vh, t1);
            }
            mat_mul(W, t1, t2);
            mat_axpy(c1, t2, A);
            // W = c0 Q + c1 (a' + c'), multiplied by E below
#pragma unroll
            for (int k = 0; k < 9; ++k) W.e[k] = {c0 * Q.e[k].re, c0 * Q.e[k].im};
            // c' = P1 step(x+mu+s nu, s nu) U_mu(x + 2 s nu)^dag step(x + 2 s nu, -s nu)
            d[mu] = 1;
            d[nu] = s;
            step_link<T>(g, L, x, d, nu, s, t1);
            mat_mul(P1, t1, t2);
            d[mu] = 0;
            d[nu] = 2 * s;
            back_mu<T>(g, L, x, d, mu, t1);
            mat_mul(t2, t1, Q);
            step_link<T>(g, L, x, d, nu, -s, t1);
            mat_mul(Q, t1, t2);
            mat_axpy(c1, t2, W);
            // a' = U_mu(x + mu) step(x + 2 mu, s nu) U_mu(x + mu + s nu)^dag U_mu(x + s nu)^dag
            d[nu] = 0;
            d[mu] = 1;
            {
                int par, idx;
                site_of(g, x, d[0], d[1], d[2], d[3], par, idx);
                load_link_soa<T>(L, mu, par, idx, g.Vh, P1);
            }
            d[mu] = 2;
            step_link<T>(g, L, x, d, nu, s, t1);
            mat_mul(P1, t1, t2);
            d[mu] = 1;
            d[nu] = s;
            back_mu<T>(g, L, x, d, mu, t1);
            mat_mul(t2, t1, Q);
            d[mu] = 0;
            back_mu<T>(g, L, x, d, mu, t1);
            mat_mul(Q, t1, t2);
            mat_axpy(c1, t2, W);
            // E = step(x + s nu, -s nu);  A += W E
            step_link<T>(g, L, x, d, nu, -s, t1);
            mat_mul(W, t1, t2);
            mat_axpy(T(1), t2, A);
        }
    }
}

// ------------------------------------------------------------------ double-float (FP64 on FP32 pipes)
// The FP64 MD step in double-float arithmetic: an SU(3) element is 9
// complex numbers of (hi, lo) float pairs (the context's df64 link copy, one
// float4 per complex), products summed Dot2-style (common.cuh), so the
// result carries ~48 significant bits on the FP32 pipes, which GB300 issues
// 64 times faster than FP64.
struct DC {
    float2 re, im;
};
struct DM3 {
    DC e[9];
};

__device__ __forceinline__ void dm_load(const float4 *__restrict__ L, int mu, int par, int idx, int Vh, DM3 &U)
{
    const float4 *p = L + (size_t)((mu * 2 + par) * 9) * Vh + idx;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        const float4 v = __ldg(p + (size_t)c * Vh);
        U.e[c].re = make_float2(v.x, v.y);
        U.e[c].im = make_float2(v.z, v.w);
    }
}

// c = a b (dg = false) or a b^dag (dg = true)
template <bool dg>
__device__ __forceinline__ void dm_mul(const DM3 &a, const DM3 &b, DM3 &c)
{
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            Acc2 re, im;
            acc_zero(re);
            acc_zero(im);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const DC x = a.e[i * 3 + k];
                const DC y = dg ? b.e[j * 3 + k] : b.e[k * 3 + j];
                const float2 yi = dg ? df_neg(y.im) : y.im;  // conj for the dagger
                acc_prod(re, x.re.x, x.re.y, y.re.x, y.re.y);
                acc_prod(re, -x.im.x, -x.im.y, yi.x, yi.y);
                acc_prod(im, x.re.x, x.re.y, yi.x, yi.y);
                acc_prod(im, x.im.x, x.im.y, y.re.x, y.re.y);
            }
            c.e[i * 3 + j].re = acc_result(re);
            c.e[i * 3 + j].im = acc_result(im);
        }
}

// A += s t (s a df64 scalar)
__device__ __forceinline__ void dm_axpy(float2 s, const DM3 &t, DM3 &A)
{
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        A.e[q].re = df_fma(s, t.e[q].re, A.e[q].re);
        A.e[q].im = df_fma(s, t.e[q].im, A.e[q].im);
    }
}

__device__ __forceinline__ void dm_at(const LinkGeo &g, const float4 *L, const int (&x)[4], const int (&d)[4], int dir,
                                      DM3 &U)
{
    int par, idx;
    site_of(g, x, d[0], d[1], d[2], d[3], par, idx);
    dm_load(L, dir, par, idx, g.Vh, U);
}

// Staple paths as step tables, all starting at x + mu and ending at x
// (direction 0 = mu, 1 = nu; the sign of a nu step is multiplied by s):
//   plaquette      nu, -mu, -nu                   (coefficient c0)
//   rectangle (a)  mu, nu, -mu, -mu, -nu          (c1)
//   rectangle (b)  nu, -mu, -mu, -nu, mu          (c1)
//   rectangle (c)  nu, nu, -mu, -nu, -nu          (c1)
// One loop with a single product site keeps the double-float code small
// enough for the instruction cache: with the staple chains unrolled (78
// products of ~1400 instructions) the kernel stalled on instruction fetch
// (46 ns/site at 32^4, 25.6 with the loop, 84 products).  In FP32 and native
// FP64 a product is ~110 instructions and the shared-prefix form of
// staple_sum_dev (67 products) is faster (2.7 against 3.2 ns/site in FP32).
__device__ __forceinline__ int path_len(int p) { return p == 0 ? 3 : 5; }
__device__ __forceinline__ int path_dir(int p, int k)
{
    // bit k of the mask: 1 = nu step
    const unsigned m = p == 0 ? 0x5u : (p == 1 ? 0x12u : (p == 2 ? 0x9u : 0x1Bu));
    return (int)((m >> k) & 1u);
}
__device__ __forceinline__ int path_sgn(int p, int k)
{
    // bit k of the mask: 1 = positive step
    const unsigned m = p == 0 ? 0x1u : (p == 1 ? 0x3u : (p == 2 ? 0x11u : 0x3u));
    return ((m >> k) & 1u) ? 1 : -1;
}

__device__ void staple_sum_df_paths(const LinkGeo &g, const float4 *L, const int (&x)[4], int mu, DM3 &A)
{
#pragma unroll
    for (int q = 0; q < 9; ++q) A.e[q].re = A.e[q].im = make_float2(0.f, 0.f);
    const float2 c0 = make_float2((float)kSymC0, (float)(kSymC0 - (double)(float)kSymC0));
    const float2 c1 = make_float2((float)kSymC1, (float)(kSymC1 - (double)(float)kSymC1));
#pragma unroll 1
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
#pragma unroll 1
        for (int s = -1; s <= 1; s += 2) {
#pragma unroll 1
            for (int p = 0; p < 4; ++p) {
                int d[4] = {0, 0, 0, 0};
                d[mu] = 1;
                DM3 M, u, T;
                const int len = path_len(p);
#pragma unroll 1
                for (int k = 0; k < len; ++k) {
                    const int isnu = path_dir(p, k);
                    const int D = isnu ? nu : mu;
                    const int sg = path_sgn(p, k) * (isnu ? s : 1);
                    if (sg < 0) d[D] -= 1;
                    dm_at(g, L, x, d, D, u);
                    if (sg > 0) d[D] += 1;
                    if (sg < 0) {
#pragma unroll
                        for (int i = 0; i < 3; ++i)
#pragma unroll
                            for (int j = 0; j < 3; ++j) {
                                if (j <= i) continue;
                                const DC a = u.e[i * 3 + j], b = u.e[j * 3 + i];
                                u.e[i * 3 + j] = {b.re, df_neg(b.im)};
                                u.e[j * 3 + i] = {a.re, df_neg(a.im)};
                            }
#pragma unroll
                        for (int i = 0; i < 3; ++i) u.e[i * 4].im = df_neg(u.e[i * 4].im);
                    }
                    if (k == 0) {
                        M = u;
                    } else {
                        dm_mul<false>(M, u, T);
                        M = T;
                    }
                }
                dm_axpy(p == 0 ? c0 : c1, M, A);
            }
        }
    }
}

// H_mu(x) -= eps F_mu(x) with the staple sum and U A in double-float; F
// and the update itself in native FP64 (about 20 operations per link).
__global__ void __launch_bounds__(kGaugeThreads)
    k_gauge_mom_update_df(LinkGeo g, const float4 *__restrict__ L, double *__restrict__ mom, double beta6, double eps)
{
    const int Vh = g.Vh;
    const long t = blockIdx.x * (long)kGaugeThreads + threadIdx.x;
    if (t >= 8L * Vh) return;
    const int i = (int)(t % Vh);
    const int mp = (int)(t / Vh);
    const int mu = mp >> 1, P = mp & 1;
    int x[4];
    coords_of(g, P, i, x);
    DM3 A, U, M;
    staple_sum_df_paths(g, L, x, mu, A);
    dm_load(L, mu, P, i, Vh, U);
    dm_mul<false>(U, A, M);
    double mre[9], mim[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        mre[q] = df_to_f64(M.e[q].re);
        mim[q] = df_to_f64(M.e[q].im);
    }
    double f[8];
    const double d0 = 2.0 * beta6 * mim[0], d1 = 2.0 * beta6 * mim[4], d2 = 2.0 * beta6 * mim[8];
    const double tr = (d0 + d1 + d2) / 3.0;
    f[0] = d0 - tr;
    f[1] = d1 - tr;
    f[2] = beta6 * (mim[1] + mim[3]);
    f[3] = beta6 * (mre[3] - mre[1]);
    f[4] = beta6 * (mim[2] + mim[6]);
    f[5] = beta6 * (mre[6] - mre[2]);
    f[6] = beta6 * (mim[5] + mim[7]);
    f[7] = beta6 * (mre[7] - mre[5]);
    double *h = mom + (size_t)(mp * 8) * Vh + i;
#pragma unroll
    for (int k = 0; k < 8; ++k) h[(size_t)k * Vh] = fma(-eps, f[k], h[(size_t)k * Vh]);
}

// U <- exp(i eps H) U in double-float: Z = i eps H scaled by 2^-k to
// 1-norm <= 1/4 (scaling in FP64), Taylor series of degree 14 by Horner,
// squared k times; the product is written to the IEEE master and to the
// df64 copy.
__global__ void __launch_bounds__(kGaugeThreads)
    k_gauge_link_update_df(int Vh, double2 *__restrict__ nat, float4 *__restrict__ Ldf,
                           const double *__restrict__ mom, double eps)
{
    const long t = blockIdx.x * (long)kGaugeThreads + threadIdx.x;
    if (t >= 8L * Vh) return;
    const int i = (int)(t % Vh);
    const int mp = (int)(t / Vh);
    double h[8];
    const double *hp = mom + (size_t)(mp * 8) * Vh + i;
#pragma unroll
    for (int k = 0; k < 8; ++k) h[k] = hp[(size_t)k * Vh];
    // 1-norm of H (columns), in FP64
    const double h22 = -h[0] - h[1];
    const double a01 = sqrt(h[2] * h[2] + h[3] * h[3]), a02 = sqrt(h[4] * h[4] + h[5] * h[5]),
                 a12 = sqrt(h[6] * h[6] + h[7] * h[7]);
    double nrm = fmax(fabs(h[0]) + a01 + a02, fmax(a01 + fabs(h[1]) + a12, a02 + a12 + fabs(h22)));
    nrm *= fabs(eps);
    int k = 0;
    double sc = eps;
    while (nrm > 0.25 && k < 60) {
        nrm *= 0.5;
        sc *= 0.5;
        ++k;
    }
    // Z = i sc H: Z_ab = i sc H_ab -> re = -sc Im H_ab, im = sc Re H_ab
    DM3 Z;
    {
        const double hr[9] = {h[0], h[2], h[4], h[2], h[1], h[6], h[4], h[6], h22};
        const double hi[9] = {0.0, h[3], h[5], -h[3], 0.0, h[7], -h[5], -h[7], 0.0};
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            Z.e[q].re = f64_to_df_slow(-sc * hi[q]);
            Z.e[q].im = f64_to_df_slow(sc * hr[q]);
        }
    }
    DM3 R, ZR;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        R.e[q].re = make_float2(q % 4 == 0 ? 1.f : 0.f, 0.f);
        R.e[q].im = make_float2(0.f, 0.f);
    }
#pragma unroll 1
    for (int n = 14; n >= 1; --n) {
        dm_mul<false>(Z, R, ZR);
        const float2 inv = f64_to_df_slow(1.0 / n);
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            R.e[q].re = df_mul(inv, ZR.e[q].re);
            R.e[q].im = df_mul(inv, ZR.e[q].im);
            if (q % 4 == 0) R.e[q].re = df_add(R.e[q].re, make_float2(1.f, 0.f));
        }
    }
#pragma unroll 1
    for (int q = 0; q < k; ++q) {
        dm_mul<false>(R, R, ZR);
        R = ZR;
    }
    DM3 U;
    dm_load(Ldf, mp >> 1, mp & 1, i, Vh, U);
    dm_mul<false>(R, U, ZR);
    double2 *pn = nat + (size_t)(mp * 9) * Vh + i;
    float4 *pd = Ldf + (size_t)(mp * 9) * Vh + i;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        const float2 re = ZR.e[c].re, im = ZR.e[c].im;
        pn[(size_t)c * Vh] = make_double2(df_to_f64(re), df_to_f64(im));
        pd[(size_t)c * Vh] = make_float4(re.x, re.y, im.x, im.y);
    }
}

// IEEE master -> df64 copy (the form k_convert_links writes)
__global__ void k_links_nat_to_df(const double2 *__restrict__ nat, float4 *Ldf, long n)
{
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const double2 d = nat[t];
    const float2 re = f64_to_df_slow(d.x), im = f64_to_df_slow(d.y);
    Ldf[t] = make_float4(re.x, re.y, im.x, im.y);
}

// 8 reals <-> traceless Hermitian matrix
template <class T>
__device__ __forceinline__ void herm_unpack(const T (&h)[8], Mat3<T> &H)
{
    H.e[0] = {h[0], T(0)};
    H.e[4] = {h[1], T(0)};
    H.e[8] = {-h[0] - h[1], T(0)};
    H.e[1] = {h[2], h[3]};
    H.e[3] = {h[2], -h[3]};
    H.e[2] = {h[4], h[5]};
    H.e[6] = {h[4], -h[5]};
    H.e[5] = {h[6], h[7]};
    H.e[7] = {h[6], -h[7]};
}

template <class T>
__device__ __forceinline__ const T *mom_ptr(const T *m, int mu, int P, int Vh)
{
    return m + (size_t)((mu * 2 + P) * 8) * Vh;
}

// H_mu(x) -= eps F_mu(x) for every link.  Thread = (mu, parity, site).
template <class T>
__global__ void __launch_bounds__(kGaugeThreads)
    k_gauge_mom_update(LinkGeo g, const typename Vec2T<T>::t *__restrict__ L, T *__restrict__ mom, T beta6, T eps)
{
    const int Vh = g.Vh;
    const long t = blockIdx.x * (long)kGaugeThreads + threadIdx.x;
    if (t >= 8L * Vh) return;
    const int i = (int)(t % Vh);
    const int mp = (int)(t / Vh);  // mu * 2 + P
    const int mu = mp >> 1, P = mp & 1;
    int x[4];
    coords_of(g, P, i, x);
    Mat3<T> A, U, M;
    staple_sum_dev<T>(g, L, x, mu, A);
    load_link_soa<T>(L, mu, P, i, Vh, U);
    mat_mul(U, A, M);
    // F = -(i beta/6)(M - M^dag): F_ij = (beta/6) * (i (conj(M_ji) - M_ij))
    //   re F_ij = (beta/6) (M_ij.im + M_ji.im),  im F_ij = (beta/6) (M_ji.re - M_ij.re)
    T f[8];
    const T d0 = beta6 * (M.e[0].im + M.e[0].im), d1 = beta6 * (M.e[4].im + M.e[4].im),
            d2 = beta6 * (M.e[8].im + M.e[8].im);
    const T tr = (d0 + d1 + d2) / T(3);
    f[0] = d0 - tr;
    f[1] = d1 - tr;
    f[2] = beta6 * (M.e[1].im + M.e[3].im);
    f[3] = beta6 * (M.e[3].re - M.e[1].re);
    f[4] = beta6 * (M.e[2].im + M.e[6].im);
    f[5] = beta6 * (M.e[6].re - M.e[2].re);
    f[6] = beta6 * (M.e[5].im + M.e[7].im);
    f[7] = beta6 * (M.e[7].re - M.e[5].re);
    T *h = mom + (size_t)(mp * 8) * Vh + i;
#pragma unroll
    for (int k = 0; k < 8; ++k) h[(size_t)k * Vh] = fma(-eps, f[k], h[(size_t)k * Vh]);
}

// E = exp(i t H): Z = i t H scaled by 2^-k to 1-norm <= 1/4, Taylor series of
// degree 16 (FP64) or 9 (FP32), squared k times.
template <class T>
__device__ __forceinline__ void exp_iH_dev(const Mat3<T> &H, T t, Mat3<T> &E)
{
    T nrm = 0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        T c = 0;
#pragma unroll
        for (int i = 0; i < 3; ++i) c += sqrt(H.e[i * 3 + j].re * H.e[i * 3 + j].re + H.e[i * 3 + j].im * H.e[i * 3 + j].im);
        nrm = c > nrm ? c : nrm;
    }
    nrm *= fabs(t);
    int k = 0;
    while (nrm > T(0.25) && k < 60) {
        nrm *= T(0.5);
        ++k;
    }
    T sc = t;
    for (int q = 0; q < k; ++q) sc *= T(0.5);
    Mat3<T> Z;
#pragma unroll
    for (int q = 0; q < 9; ++q) Z.e[q] = {-sc * H.e[q].im, sc * H.e[q].re};
    // Horner: E = I + Z (I + Z/2 (I + Z/3 (... (I + Z/n))))
    constexpr int deg = sizeof(T) == 8 ? 16 : 9;
    Mat3<T> R;
#pragma unroll
    for (int q = 0; q < 9; ++q) R.e[q] = {(q % 4 == 0) ? T(1) : T(0), T(0)};
#pragma unroll 1
    for (int n = deg; n >= 1; --n) {
        Mat3<T> ZR;
        mat_mul(Z, R, ZR);
        const T inv = T(1) / T(n);
#pragma unroll
        for (int q = 0; q < 9; ++q) R.e[q] = {((q % 4 == 0) ? T(1) : T(0)) + inv * ZR.e[q].re, inv * ZR.e[q].im};
    }
#pragma unroll 1
    for (int q = 0; q < k; ++q) {
        Mat3<T> S2;
        mat_mul(R, R, S2);
        R = S2;
    }
    E = R;
}

// U_mu(x) <- exp(i eps H_mu(x)) U_mu(x) for every link.
template <class T>
__global__ void __launch_bounds__(kGaugeThreads)
    k_gauge_link_update(int Vh, typename Vec2T<T>::t *__restrict__ L, const T *__restrict__ mom, T eps)
{
    const long t = blockIdx.x * (long)kGaugeThreads + threadIdx.x;
    if (t >= 8L * Vh) return;
    const int i = (int)(t % Vh);
    const int mp = (int)(t / Vh);
    T h[8];
    const T *hp = mom + (size_t)(mp * 8) * Vh + i;
#pragma unroll
    for (int k = 0; k < 8; ++k) h[k] = hp[(size_t)k * Vh];
    Mat3<T> H, E, U, R;
    herm_unpack(h, H);
    exp_iH_dev(H, eps, E);
    typename Vec2T<T>::t *p = L + (size_t)(mp * 9) * Vh + i;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        const typename Vec2T<T>::t v = p[(size_t)c * Vh];
        U.e[c] = {v.x, v.y};
    }
    mat_mul(E, U, R);
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        typename Vec2T<T>::t v;
        v.x = R.e[c].re;
        v.y = R.e[c].im;
        p[(size_t)c * Vh] = v;
    }
}

// U_dir(x + d)
template <class T>
__device__ __forceinline__ void link_at(const LinkGeo &g, const typename Vec2T<T>::t *L, const int (&x)[4], int d0,
                                        int d1, int d2, int d3, int dir, Mat3<T> &U)
{
    int par, idx;
    site_of(g, x, d0, d1, d2, d3, par, idx);
    load_link_soa<T>(L, dir, par, idx, g.Vh, U);
}

// Per-block partial of sum_x [c0 sum_{mu<nu} Re Tr P + c1 sum_{mu!=nu} Re Tr R]
// (FP64 accumulation); thread = site (parity, half index):
//   P = U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
//   R = U_mu(x) U_mu(x+mu) U_nu(x+2mu) U_mu(x+mu+nu)^dag U_mu(x+nu)^dag U_nu(x)^dag
template <class T>
__global__ void __launch_bounds__(kGaugeThreads)
    k_gauge_action_part(LinkGeo g, const typename Vec2T<T>::t *__restrict__ L, double *part)
{
    __shared__ double s_red[kGaugeThreads / 32];
    const long t = blockIdx.x * (long)kGaugeThreads + threadIdx.x;
    double acc = 0.0;
    if (t < 2L * g.Vh) {
        const int P = (int)(t / g.Vh), i = (int)(t % g.Vh);
        int x[4];
        coords_of(g, P, i, x);
        double sp = 0.0, sr = 0.0;
#pragma unroll 1
        for (int mu = 0; mu < 4; ++mu)
#pragma unroll 1
            for (int nu = 0; nu < 4; ++nu) {
                if (nu == mu) continue;
                int em[4] = {0, 0, 0, 0}, en[4] = {0, 0, 0, 0};
                em[mu] = 1;
                en[nu] = 1;
                Mat3<T> u, b, c, d;
                link_at<T>(g, L, x, 0, 0, 0, 0, mu, u);
                if (mu < nu) {
                    link_at<T>(g, L, x, em[0], em[1], em[2], em[3], nu, b);
                    mat_mul(u, b, c);
                    link_at<T>(g, L, x, en[0], en[1], en[2], en[3], mu, b);
                    mat_mul_dag(c, b, d);
                    link_at<T>(g, L, x, 0, 0, 0, 0, nu, b);
                    mat_mul_dag(d, b, c);
                    sp += (double)c.e[0].re + (double)c.e[4].re + (double)c.e[8].re;
                }
                link_at<T>(g, L, x, em[0], em[1], em[2], em[3], mu, b);
                mat_mul(u, b, c);
                link_at<T>(g, L, x, 2 * em[0], 2 * em[1], 2 * em[2], 2 * em[3], nu, b);
                mat_mul(c, b, d);
                link_at<T>(g, L, x, em[0] + en[0], em[1] + en[1], em[2] + en[2], em[3] + en[3], mu, b);
                mat_mul_dag(d, b, c);
                link_at<T>(g, L, x, en[0], en[1], en[2], en[3], mu, b);
                mat_mul_dag(c, b, d);
                link_at<T>(g, L, x, 0, 0, 0, 0, nu, b);
                mat_mul_dag(d, b, c);
                sr += (double)c.e[0].re + (double)c.e[4].re + (double)c.e[8].re;
            }
        acc = kSymC0 * sp + kSymC1 * sr;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < kGaugeThreads / 32; ++k) s += s_red[k];
        part[blockIdx.x] = s;
    }
}

// Per-block partial of (1/2) sum Tr H^2.
template <class T>
__global__ void __launch_bounds__(kGaugeThreads) k_mom_energy_part(int Vh, const T *__restrict__ mom, double *part)
{
    __shared__ double s_red[kGaugeThreads / 32];
    const long t = blockIdx.x * (long)kGaugeThreads + threadIdx.x;
    double acc = 0.0;
    if (t < 8L * Vh) {
        const int i = (int)(t % Vh), mp = (int)(t / Vh);
        const T *hp = mom + (size_t)(mp * 8) * Vh + i;
        double h[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) h[k] = (double)hp[(size_t)k * Vh];
        const double d2 = -h[0] - h[1];
        acc = 0.5 * (h[0] * h[0] + h[1] * h[1] + d2 * d2 +
                     2.0 * (h[2] * h[2] + h[3] * h[3] + h[4] * h[4] + h[5] * h[5] + h[6] * h[6] + h[7] * h[7]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < kGaugeThreads / 32; ++k) s += s_red[k];
        part[blockIdx.x] = s;
    }
}

// One block: sum of part[0..n) in a fixed order.
__global__ void __launch_bounds__(256) k_gauge_sum_ordered(const double *__restrict__ part, int n, double *out)
{
    __shared__ double s_red[8];
    double s = 0.0;
    for (int k = threadIdx.x; k < n; k += 256) s += part[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int k = 0; k < 8; ++k) tot += s_red[k];
        *out = tot;
    }
}

// ------------------------------------------------------------------ format conversions
// canonical host momenta [4][V][3][3] complex128 (staged on the device) -> 8 reals SoA (FP64 and FP32)
__global__ void k_mom_from_canonical(LinkGeo g, const double2 *__restrict__ src, double *m64, float *m32, int *bad,
                                     long V)
{
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= 4 * V) return;
    const int mu = (int)(t / V);
    const long lex = t - (long)mu * V;
    int x[4];
    long r = lex;
    for (int m = 0; m < 4; ++m) {
        x[m] = (int)(r % g.N[m]);
        r /= g.N[m];
    }
    const int P = (x[0] + x[1] + x[2] + x[3]) & 1;
    const int idx = (int)(lex >> 1);
    const double2 *h = src + t * 9;
    // Hermitian and traceless to 1e-12 relative, else rejected
    double scale = 0.0;
    for (int c = 0; c < 9; ++c) scale = fmax(scale, fmax(fabs(h[c].x), fabs(h[c].y)));
    const double tol = 1e-12 * fmax(scale, 1e-300);
    bool ok = isfinite(scale) && fabs(h[0].y) <= tol && fabs(h[4].y) <= tol && fabs(h[8].y) <= tol &&
              fabs(h[0].x + h[4].x + h[8].x) <= 3 * tol;
    const int off[3][2] = {{1, 3}, {2, 6}, {5, 7}};
    for (int q = 0; q < 3; ++q)
        ok = ok && fabs(h[off[q][0]].x - h[off[q][1]].x) <= tol && fabs(h[off[q][0]].y + h[off[q][1]].y) <= tol;
    if (!ok) atomicOr(bad, 1);
    const double v[8] = {h[0].x, h[4].x, h[1].x, h[1].y, h[2].x, h[2].y, h[5].x, h[5].y};
    for (int k = 0; k < 8; ++k) {
        const size_t o = (size_t)((mu * 2 + P) * 8 + k) * g.Vh + idx;
        m64[o] = v[k];
        if (m32) m32[o] = (float)v[k];
    }
}

template <class T>
__global__ void k_mom_to_canonical(LinkGeo g, const T *__restrict__ m, double2 *dst, long V)
{
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= 4 * V) return;
    const int mu = (int)(t / V);
    const long lex = t - (long)mu * V;
    int x[4];
    long r = lex;
    for (int q = 0; q < 4; ++q) {
        x[q] = (int)(r % g.N[q]);
        r /= g.N[q];
    }
    const int P = (x[0] + x[1] + x[2] + x[3]) & 1;
    const int idx = (int)(lex >> 1);
    double h[8];
    for (int k = 0; k < 8; ++k) h[k] = (double)m[(size_t)((mu * 2 + P) * 8 + k) * g.Vh + idx];
    double2 *o = dst + t * 9;
    o[0] = make_double2(h[0], 0.0);
    o[4] = make_double2(h[1], 0.0);
    o[8] = make_double2(-h[0] - h[1], 0.0);
    o[1] = make_double2(h[2], h[3]);
    o[3] = make_double2(h[2], -h[3]);
    o[2] = make_double2(h[4], h[5]);
    o[6] = make_double2(h[4], -h[5]);
    o[5] = make_double2(h[6], h[7]);
    o[7] = make_double2(h[6], -h[7]);
}

// FP64 <-> FP32 copies of links (SoA, same layout) and momenta
__global__ void k_links_f64_to_f32(const double2 *__restrict__ a, float2 *b, long n)
{
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t < n) b[t] = make_float2((float)a[t].x, (float)a[t].y);
}
__global__ void k_links_f32_to_f64(const float2 *__restrict__ a, double2 *b, long n)
{
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t < n) b[t] = make_double2((double)a[t].x, (double)a[t].y);
}
__global__ void k_mom_f64_to_f32(const double *__restrict__ a, float *b, long n)
{
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t < n) b[t] = (float)a[t];
}
__global__ void k_mom_f32_to_f64(const float *__restrict__ a, double *b, long n)
{
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t < n) b[t] = (double)a[t];
}

// ------------------------------------------------------------------ fermion force
// Force of the rational pseudofermion action S_f = phi^dag r(A) phi
// (Sec. 2.2, Eqs. rooting, shlineq), from x_i = (A + sigma_i)^{-1} phi (even
// sites) and y_i = D_oe x_i (odd sites):
//   F_mu(n) = traceless part of (i s_mu(n) / 2) c sum_i a_i (W_i - W_i^dag),
//   n even: W_i = U_mu(n) y_i(n+mu) x_i(n)^dag (c = +1); n odd: W_i = U_mu(n) x_i(n+mu) y_i(n)^dag (c = -1);
// and H -= eps F.  One thread per link, native FP64 (about 36 n + 110 FMAs).
struct FFCoef {
    double a[kMaxShifts];
    int n;
};

__global__ void __launch_bounds__(kGaugeThreads)
    k_fermion_force_update(Geom g, const double2 *__restrict__ L, const double2 *__restrict__ x,
                           const double2 *__restrict__ y, const __grid_constant__ FFCoef C, double *__restrict__ mom,
                           double eps)
{
    const int Vh = g.Vh;
    const long t = blockIdx.x * (long)kGaugeThreads + threadIdx.x;
    if (t >= 8L * Vh) return;
    const int i = (int)(t % Vh);
    const int mp = (int)(t / Vh);
    const int mu = mp >> 1, P = mp & 1;
    Stencil S;
    make_stencil(g, i, P, S);
    int f, b;
    uint32_t nf, nb;
    hop(g, S, mu, f, b, nf, nb);
    const double sgn = nf ? -1.0 : 1.0;            // s_mu(n): staggered phase and time boundary
    const double2 *left = P == 0 ? y : x;          // field at n + mu
    const double2 *right = P == 0 ? x : y;         // field at n
    const size_t n3 = 3 * (size_t)Vh;
    double2 O[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) O[q] = make_double2(0.0, 0.0);
#pragma unroll 1
    for (int k = 0; k < C.n; ++k) {
        double2 l[3], r[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            l[c] = __ldg(left + k * n3 + (size_t)c * Vh + f);
            r[c] = __ldg(right + k * n3 + (size_t)c * Vh + i);
        }
        const double ak = C.a[k];
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                // a_k l_p conj(r_q)
                const double re = l[p].x * r[q].x + l[p].y * r[q].y;
                const double im = l[p].y * r[q].x - l[p].x * r[q].y;
                O[p * 3 + q].x = fma(ak, re, O[p * 3 + q].x);
                O[p * 3 + q].y = fma(ak, im, O[p * 3 + q].y);
            }
    }
    double2 U[9];
    const double2 *lp = L + link_base(mu, P, 9, Vh) + i;
#pragma unroll
    for (int c = 0; c < 9; ++c) U[c] = __ldg(lp + (size_t)c * Vh);
    double2 W[9];
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            double re = 0.0, im = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const double2 u = U[p * 3 + k], o = O[k * 3 + q];
                re = fma(u.x, o.x, fma(-u.y, o.y, re));
                im = fma(u.x, o.y, fma(u.y, o.x, im));
            }
            W[p * 3 + q] = make_double2(re, im);
        }
    // F = (i h)(W - W^dag), h = s c / 2:  re F_pq = -h (Im W_pq + Im W_qp),  im F_pq = h (Re W_pq - Re W_qp)
    const double hsc = 0.5 * sgn * (P == 0 ? 1.0 : -1.0);
    const double d0 = -2.0 * hsc * W[0].y, d1 = -2.0 * hsc * W[4].y, d2 = -2.0 * hsc * W[8].y;
    const double tr = (d0 + d1 + d2) / 3.0;
    double fv[8];
    fv[0] = d0 - tr;
    fv[1] = d1 - tr;
    fv[2] = -hsc * (W[1].y + W[3].y);
    fv[3] = hsc * (W[1].x - W[3].x);
    fv[4] = -hsc * (W[2].y + W[6].y);
    fv[5] = hsc * (W[2].x - W[6].x);
    fv[6] = -hsc * (W[5].y + W[7].y);
    fv[7] = hsc * (W[5].x - W[7].x);
    double *h = mom + (size_t)(mp * 8) * Vh + i;
#pragma unroll
    for (int k = 0; k < 8; ++k) h[(size_t)k * Vh] = fma(-eps, fv[k], h[(size_t)k * Vh]);
}

// ------------------------------------------------------------------ stout smearing
// Stout smearing of the links (Sec. 2.1, stout-improved staggered action,
// after Morningstar and Peardon), isotropic weight rho per level:
//   C_mu(x) = rho sum_{nu != mu} [ U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag
//                                 + U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) ],
//   Omega = C U^dag, Q = (i/2)(Omega^dag - Omega) - (i/6) Tr(Omega^dag - Omega),
//   U' = exp(iQ) U.
// Native FP64, one thread per link, the SoA layout of the IEEE links.

__device__ __forceinline__ void stout_C(const LinkGeo &g, const double2 *L, const int (&x)[4], int mu, double rho,
                                        Mat3<double> &C)
{
#pragma unroll
    for (int q = 0; q < 9; ++q) C.e[q] = {0.0, 0.0};
#pragma unroll 1
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        int dn[4] = {0, 0, 0, 0}, dm[4] = {0, 0, 0, 0}, dmn[4] = {0, 0, 0, 0};
        dn[nu] = 1;
        dm[mu] = 1;
        dmn[mu] = 1;
        dmn[nu] = -1;
        Mat3<double> a, b, t, u;
        // upper: U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag
        link_at<double>(g, L, x, 0, 0, 0, 0, nu, a);
        link_at<double>(g, L, x, dn[0], dn[1], dn[2], dn[3], mu, b);
        mat_mul(a, b, t);
        link_at<double>(g, L, x, dm[0], dm[1], dm[2], dm[3], nu, a);
        mat_mul_dag(t, a, u);
        mat_axpy(rho, u, C);
        // lower: U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu)
        link_at<double>(g, L, x, -dn[0], -dn[1], -dn[2], -dn[3], nu, a);
        mat_dag(a);
        link_at<double>(g, L, x, -dn[0], -dn[1], -dn[2], -dn[3], mu, b);
        mat_mul(a, b, t);
        link_at<double>(g, L, x, dmn[0], dmn[1], dmn[2], dmn[3], nu, a);
        mat_mul(t, a, u);
        mat_axpy(rho, u, C);
    }
}

// Q from C and U (Hermitian, traceless)
__device__ __forceinline__ void stout_Q(const Mat3<double> &C, const Mat3<double> &U, Mat3<double> &Q)
{
    Mat3<double> Om;
    mat_mul_dag(C, U, Om);
    // Q_ij = (i/2)(conj(Om_ji) - Om_ij):  re = (Om_ij.im + Om_ji.im)/2, im = (Om_ji.re - Om_ij.re)/2
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            Q.e[i * 3 + j] = {0.5 * (Om.e[i * 3 + j].im + Om.e[j * 3 + i].im),
                              0.5 * (Om.e[j * 3 + i].re - Om.e[i * 3 + j].re)};
    const double tr = (Q.e[0].re + Q.e[4].re + Q.e[8].re) / 3.0;
    Q.e[0].re -= tr;
    Q.e[4].re -= tr;
    Q.e[8].re -= tr;
}

// E = exp(X) and D = d/dt exp(X + t A) at t = 0, from the block matrix
// B = [[X, A], [0, X]], exp(B) = [[E, D], [0, E]]: B scaled by 2^-k to
// 1-norm <= 1/4 (the norm of X bounds the scaling; A scales with it),
// Horner on the block form (P <- 1 + X P / n, R <- (X R + A P) / n, degree
// 18), then k block squarings (P, R) <- (P P, P R + R P).
__device__ void exp_frechet_dev(const Mat3<double> &X, const Mat3<double> &A, Mat3<double> &E, Mat3<double> &D)
{
    // D is linear in A: run with A / ||A||_1 and scale D back
    double nx = 0.0, na = 0.0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        double c = 0.0, ca = 0.0;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            c += hypot(X.e[i * 3 + j].re, X.e[i * 3 + j].im);
            ca += hypot(A.e[i * 3 + j].re, A.e[i * 3 + j].im);
        }
        nx = fmax(nx, c);
        na = fmax(na, ca);
    }
    const double an = na > 0.0 ? 1.0 / na : 0.0;
    double nrm = nx + (na > 0.0 ? 1.0 : 0.0);
    int k = 0;
    while (nrm > 0.25 && k < 60) {
        nrm *= 0.5;
        ++k;
    }
    const double sc = ldexp(1.0, -k);
    Mat3<double> Xs, As, P, R;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        Xs.e[q] = {sc * X.e[q].re, sc * X.e[q].im};
        As.e[q] = {sc * an * A.e[q].re, sc * an * A.e[q].im};
        P.e[q] = {(q % 4 == 0) ? 1.0 : 0.0, 0.0};
        R.e[q] = {0.0, 0.0};
    }
#pragma unroll 1
    for (int n = 18; n >= 1; --n) {
        Mat3<double> XP, XR, AP;
        mat_mul(Xs, P, XP);
        mat_mul(Xs, R, XR);
        mat_mul(As, P, AP);
        const double inv = 1.0 / n;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            P.e[q] = {((q % 4 == 0) ? 1.0 : 0.0) + inv * XP.e[q].re, inv * XP.e[q].im};
            R.e[q] = {inv * (XR.e[q].re + AP.e[q].re), inv * (XR.e[q].im + AP.e[q].im)};
        }
    }
#pragma unroll 1
    for (int q = 0; q < k; ++q) {
        Mat3<double> PP, PR, RP;
        mat_mul(P, P, PP);
        mat_mul(P, R, PR);
        mat_mul(R, P, RP);
        P = PP;
#pragma unroll
        for (int c = 0; c < 9; ++c) R.e[c] = {PR.e[c].re + RP.e[c].re, PR.e[c].im + RP.e[c].im};
    }
    E = P;
#pragma unroll
    for (int c = 0; c < 9; ++c) D.e[c] = {na * R.e[c].re, na * R.e[c].im};
}

__device__ __forceinline__ void store_link_soa(double2 *L, int mu, int P, int i, int Vh, const Mat3<double> &U)
{
    double2 *p = L + (size_t)((mu * 2 + P) * 9) * Vh + i;
#pragma unroll
    for (int c = 0; c < 9; ++c) p[(size_t)c * Vh] = make_double2(U.e[c].re, U.e[c].im);
}

// Lout = one stout level of Lin.  Thread = (mu, parity, site).
__global__ void __launch_bounds__(kGaugeThreads)
    k_stout_level(LinkGeo g, const double2 *__restrict__ Lin, double2 *__restrict__ Lout, double rho)
{
    const int Vh = g.Vh;
    const long t = blockIdx.x * (long)kGaugeThreads + threadIdx.x;
    if (t >= 8L * Vh) return;
    const int i = (int)(t % Vh);
    const int mp = (int)(t / Vh);
    const int mu = mp >> 1, P = mp & 1;
    int x[4];
    coords_of(g, P, i, x);
    Mat3<double> C, U, Q, E, R;
    stout_C(g, Lin, x, mu, rho, C);
    load_link_soa<double>(Lin, mu, P, i, Vh, U);
    stout_Q(C, U, Q);
    exp_iH_dev(Q, 1.0, E);
    mat_mul(E, U, R);
    store_link_soa(Lout, mu, P, i, Vh, R);
}

// First pass of the force chain of one level (the force on U' = smear(U),
// Fp as 8 reals per link, to the force on U): per link
//   Sigma' = -i U'^dag Fp,  Gamma = Dexp_{iQ}[U Sigma'],  L = traceless
//   anti-Hermitian part of Gamma,
//   Gl = Sigma' exp(iQ) - C^dag L  (the link's own terms of the gradient),
//   M = U^dag L                    (what the staples of C carry to their links).
__global__ void __launch_bounds__(kGaugeThreads)
    k_stout_local(LinkGeo g, const double2 *__restrict__ L, const double *__restrict__ Fp, double rho,
                  double2 *__restrict__ Mout, double2 *__restrict__ Gl)
{
    const int Vh = g.Vh;
    const long t = blockIdx.x * (long)kGaugeThreads + threadIdx.x;
    if (t >= 8L * Vh) return;
    const int i = (int)(t % Vh);
    const int mp = (int)(t / Vh);
    const int mu = mp >> 1, P = mp & 1;
    int x[4];
    coords_of(g, P, i, x);
    Mat3<double> C, U, Q, E, D, W, S, iQ, F;
    stout_C(g, L, x, mu, rho, C);
    load_link_soa<double>(L, mu, P, i, Vh, U);
    stout_Q(C, U, Q);
    double h[8];
    const double *hp = Fp + (size_t)(mp * 8) * Vh + i;
#pragma unroll
    for (int k = 0; k < 8; ++k) h[k] = hp[(size_t)k * Vh];
    herm_unpack(h, F);
#pragma unroll
    for (int q = 0; q < 9; ++q) iQ.e[q] = {-Q.e[q].im, Q.e[q].re};
    exp_iH_dev(Q, 1.0, E);
    mat_mul(E, U, W);  // U'
    // S = -i U'^dag F
    Mat3<double> Wd = W;
    mat_dag(Wd);
    mat_mul(Wd, F, S);
#pragma unroll
    for (int q = 0; q < 9; ++q) S.e[q] = {S.e[q].im, -S.e[q].re};
    Mat3<double> US, E2;
    mat_mul(U, S, US);
    exp_frechet_dev(iQ, US, E2, D);
    // L = (D - D^dag)/2 - Tr(D - D^dag)/6
    Mat3<double> Lm;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            Lm.e[a * 3 + b] = {0.5 * (D.e[a * 3 + b].re - D.e[b * 3 + a].re),
                               0.5 * (D.e[a * 3 + b].im + D.e[b * 3 + a].im)};
    const double tri = (Lm.e[0].im + Lm.e[4].im + Lm.e[8].im) / 3.0;
    Lm.e[0].im -= tri;
    Lm.e[4].im -= tri;
    Lm.e[8].im -= tri;
    // Gl = S E - C^dag L
    Mat3<double> SE, CdL, Cd = C;
    mat_mul(S, E, SE);
    mat_dag(Cd);
    mat_mul(Cd, Lm, CdL);
#pragma unroll
    for (int q = 0; q < 9; ++q) SE.e[q] = {SE.e[q].re - CdL.e[q].re, SE.e[q].im - CdL.e[q].im};
    store_link_soa(Gl, mu, P, i, Vh, SE);
    // M = U^dag L
    Mat3<double> Ud = U, M;
    mat_dag(Ud);
    mat_mul(Ud, Lm, M);
    store_link_soa(Mout, mu, P, i, Vh, M);
}

// Second pass: each link (y, l) gathers the staple terms that carry M of the
// links whose C contains it (rho times, for every mu != l and nu != l):
//   U_mu(y+l) U_l(y+mu)^dag M_mu(y)            U_mu(y-mu+l)^dag U_l(y-mu)^dag M_mu(y-mu)^dag
//   M_mu(y+l)^dag U_l(y+mu)^dag U_mu(y)^dag    M_mu(y+l-mu) U_l(y-mu)^dag U_mu(y-mu)
//   U_nu(y-nu+l)^dag M_l(y-nu) U_nu(y-nu)      U_nu(y+l) M_l(y+nu) U_nu(y)^dag
// adds the link's own terms Gl and writes the force on the link,
//   F = traceless part of (i/2)(U G - G^dag U^dag), as 8 reals.
__global__ void __launch_bounds__(kGaugeThreads)
    k_stout_gather(LinkGeo g, const double2 *__restrict__ L, const double2 *__restrict__ M,
                   const double2 *__restrict__ Gl, double rho, double *__restrict__ Fout)
{
    const int Vh = g.Vh;
    const long t = blockIdx.x * (long)kGaugeThreads + threadIdx.x;
    if (t >= 8L * Vh) return;
    const int i = (int)(t % Vh);
    const int mp = (int)(t / Vh);
    const int l = mp >> 1, P = mp & 1;
    int y[4];
    coords_of(g, P, i, y);
    Mat3<double> G, acc;
    load_link_soa<double>(Gl, l, P, i, Vh, G);
#pragma unroll
    for (int q = 0; q < 9; ++q) acc.e[q] = {0.0, 0.0};
    int el[4] = {0, 0, 0, 0};
    el[l] = 1;
#pragma unroll 1
    for (int m = 0; m < 4; ++m) {
        if (m == l) continue;
        int em[4] = {0, 0, 0, 0};
        em[m] = 1;
        Mat3<double> a, b, c, t1, t2;
        // U_m(y+l) U_l(y+m)^dag M_m(y)
        link_at<double>(g, L, y, el[0], el[1], el[2], el[3], m, a);
        link_at<double>(g, L, y, em[0], em[1], em[2], em[3], l, b);
        mat_mul_dag(a, b, t1);
        link_at<double>(g, M, y, 0, 0, 0, 0, m, c);
        mat_mul(t1, c, t2);
        mat_axpy(1.0, t2, acc);
        // U_m(y-m+l)^dag U_l(y-m)^dag M_m(y-m)^dag = (M_m(y-m) U_l(y-m) U_m(y-m+l))^dag
        link_at<double>(g, M, y, -em[0], -em[1], -em[2], -em[3], m, c);
        link_at<double>(g, L, y, -em[0], -em[1], -em[2], -em[3], l, b);
        mat_mul(c, b, t1);
        link_at<double>(g, L, y, el[0] - em[0], el[1] - em[1], el[2] - em[2], el[3] - em[3], m, a);
        mat_mul(t1, a, t2);
        mat_dag(t2);
        mat_axpy(1.0, t2, acc);
        // M_m(y+l)^dag U_l(y+m)^dag U_m(y)^dag = (U_m(y) U_l(y+m) M_m(y+l))^dag
        link_at<double>(g, L, y, 0, 0, 0, 0, m, a);
        link_at<double>(g, L, y, em[0], em[1], em[2], em[3], l, b);
        mat_mul(a, b, t1);
        link_at<double>(g, M, y, el[0], el[1], el[2], el[3], m, c);
        mat_mul(t1, c, t2);
        mat_dag(t2);
        mat_axpy(1.0, t2, acc);
        // M_m(y+l-m) U_l(y-m)^dag U_m(y-m)
        link_at<double>(g, M, y, el[0] - em[0], el[1] - em[1], el[2] - em[2], el[3] - em[3], m, c);
        link_at<double>(g, L, y, -em[0], -em[1], -em[2], -em[3], l, b);
        mat_mul_dag(c, b, t1);
        link_at<double>(g, L, y, -em[0], -em[1], -em[2], -em[3], m, a);
        mat_mul(t1, a, t2);
        mat_axpy(1.0, t2, acc);
        // (m plays nu) U_m(y-m+l)^dag M_l(y-m) U_m(y-m)
        link_at<double>(g, L, y, el[0] - em[0], el[1] - em[1], el[2] - em[2], el[3] - em[3], m, a);
        mat_dag(a);
        link_at<double>(g, M, y, -em[0], -em[1], -em[2], -em[3], l, c);
        mat_mul(a, c, t1);
        link_at<double>(g, L, y, -em[0], -em[1], -em[2], -em[3], m, b);
        mat_mul(t1, b, t2);
        mat_axpy(1.0, t2, acc);
        // U_m(y+l) M_l(y+m) U_m(y)^dag
        link_at<double>(g, L, y, el[0], el[1], el[2], el[3], m, a);
        link_at<double>(g, M, y, em[0], em[1], em[2], em[3], l, c);
        mat_mul(a, c, t1);
        link_at<double>(g, L, y, 0, 0, 0, 0, m, b);
        mat_mul_dag(t1, b, t2);
        mat_axpy(1.0, t2, acc);
    }
    mat_axpy(rho, acc, G);
    Mat3<double> U, W;
    load_link_soa<double>(L, l, P, i, Vh, U);
    mat_mul(U, G, W);
    // F = (i/2)(W - W^dag): re F_pq = -(Im W_pq + Im W_qp)/2, im F_pq = (Re W_pq - Re W_qp)/2
    const double d0 = -W.e[0].im, d1 = -W.e[4].im, d2 = -W.e[8].im;
    const double tr = (d0 + d1 + d2) / 3.0;
    double f[8];
    f[0] = d0 - tr;
    f[1] = d1 - tr;
    f[2] = -0.5 * (W.e[1].im + W.e[3].im);
    f[3] = 0.5 * (W.e[1].re - W.e[3].re);
    f[4] = -0.5 * (W.e[2].im + W.e[6].im);
    f[5] = 0.5 * (W.e[2].re - W.e[6].re);
    f[6] = -0.5 * (W.e[5].im + W.e[7].im);
    f[7] = 0.5 * (W.e[5].re - W.e[7].re);
    double *fo = Fout + (size_t)(mp * 8) * Vh + i;
#pragma unroll
    for (int k = 0; k < 8; ++k) fo[(size_t)k * Vh] = f[k];
}

// y += a x over n doubles
__global__ void k_daxpy(long n, double a, const double *__restrict__ x, double *__restrict__ y)
{
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t < n) y[t] = fma(a, x[t], y[t]);
}

static LinkGeo link_geo(const lqcd_ctx *c)
{
    LinkGeo g;
    for (int m = 0; m < 4; ++m) g.N[m] = c->dims[m];
    g.Vh = (int)c->Vh;
    return g;
}

static inline unsigned nblocks(long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// ------------------------------------------------------------------ copies and staleness
// links: the FP64 SoA (lnk_nat) is the master; an FP32 MD step works on lnk_f18
// and makes it the newest copy; FP64 MD steps update lnk_nat and leave every
// derived format stale until links_ready rebuilds them.
static int links_to_prec(lqcd_ctx *c, int prec)
{
    const long n = 72L * (long)c->Vh;
    if (prec == LQCD_PREC_FP32) {
        if (c->md_links_newest == LQCD_PREC_FP64 && c->links_derived_stale) {
            k_links_f64_to_f32<<<nblocks(n, 256), 256, 0, c->stream>>>(c->lnk_nat.as<double2>(), c->lnk_f18.as<float2>(), n);
            LQCD_CUDA(cudaGetLastError());
            c->launches += 1;
        }
        return LQCD_OK;
    }
    if (c->md_links_newest == LQCD_PREC_FP32) {
        k_links_f32_to_f64<<<nblocks(n, 256), 256, 0, c->stream>>>(c->lnk_f18.as<float2>(), c->lnk_nat.as<double2>(), n);
        LQCD_CUDA(cudaGetLastError());
        c->launches += 1;
        c->md_links_newest = LQCD_PREC_FP64;
        c->links_derived_stale = true;
        c->df_stale = true;
    }
    if (prec == LQCD_PREC_FP64 && c->df_stale) {  // double-float steps work on the df64 copy
        k_links_nat_to_df<<<nblocks(n, 256), 256, 0, c->stream>>>(c->lnk_nat.as<double2>(), c->lnk_df.as<float4>(), n);
        LQCD_CUDA(cudaGetLastError());
        c->launches += 1;
        c->df_stale = false;
    }
    return LQCD_OK;
}

// FP64 and native FP64 share the FP64 momenta
static inline int mom_prec(int prec) { return prec == LQCD_PREC_FP32 ? LQCD_PREC_FP32 : LQCD_PREC_FP64; }

static int mom_to_prec(lqcd_ctx *c, int prec)
{
    prec = mom_prec(prec);
    if (c->mom_newest == prec) return LQCD_OK;
    const long n = 64L * (long)c->Vh;
    if (prec == LQCD_PREC_FP32)
        k_mom_f64_to_f32<<<nblocks(n, 256), 256, 0, c->stream>>>(c->mom64.as<double>(), c->mom32.as<float>(), n);
    else
        k_mom_f32_to_f64<<<nblocks(n, 256), 256, 0, c->stream>>>(c->mom32.as<float>(), c->mom64.as<double>(), n);
    LQCD_CUDA(cudaGetLastError());
    c->launches += 1;
    c->mom_newest = prec;
    return LQCD_OK;
}

static int check_md(lqcd_ctx *c, int prec)
{
    if (!c) return fail(LQCD_EINVAL, "NULL context");
    LQCD_ON_DEVICE(c->device);
    if (!c->links_ok) return fail(LQCD_ESTATE, "no links uploaded");
    if (!c->mom64.ptr) return fail(LQCD_ESTATE, "no momenta uploaded");
    if (prec != LQCD_PREC_FP64 && prec != LQCD_PREC_FP32 && prec != LQCD_PREC_FP64_NATIVE)
        return fail(LQCD_EINVAL, "MD precision must be FP64, FP64_NATIVE or FP32");
    return LQCD_OK;
}

static void launch_mom_update(lqcd_ctx *c, int prec, double beta, double eps)
{
    const LinkGeo g = link_geo(c);
    const unsigned nb = nblocks(8L * (long)c->Vh, kGaugeThreads);
    if (prec == LQCD_PREC_FP64)
        k_gauge_mom_update_df<<<nb, kGaugeThreads, 0, c->stream>>>(g, c->lnk_df.as<float4>(), c->mom64.as<double>(),
                                                                   beta / 6.0, eps);
    else if (prec == LQCD_PREC_FP64_NATIVE)
        k_gauge_mom_update<double><<<nb, kGaugeThreads, 0, c->stream>>>(g, c->lnk_nat.as<double2>(), c->mom64.as<double>(),
                                                                        beta / 6.0, eps);
    else
        k_gauge_mom_update<float><<<nb, kGaugeThreads, 0, c->stream>>>(g, c->lnk_f18.as<float2>(), c->mom32.as<float>(),
                                                                       (float)(beta / 6.0), (float)eps);
    c->launches += 1;
}

static void launch_link_update(lqcd_ctx *c, int prec, double eps)
{
    const unsigned nb = nblocks(8L * (long)c->Vh, kGaugeThreads);
    if (prec == LQCD_PREC_FP64) {
        k_gauge_link_update_df<<<nb, kGaugeThreads, 0, c->stream>>>((int)c->Vh, c->lnk_nat.as<double2>(),
                                                                    c->lnk_df.as<float4>(), c->mom64.as<double>(), eps);
        c->md_links_newest = LQCD_PREC_FP64;
    } else if (prec == LQCD_PREC_FP64_NATIVE) {
        k_gauge_link_update<double><<<nb, kGaugeThreads, 0, c->stream>>>((int)c->Vh, c->lnk_nat.as<double2>(),
                                                                         c->mom64.as<double>(), eps);
        c->md_links_newest = LQCD_PREC_FP64;
        c->df_stale = true;
    } else {
        k_gauge_link_update<float><<<nb, kGaugeThreads, 0, c->stream>>>((int)c->Vh, c->lnk_f18.as<float2>(),
                                                                        c->mom32.as<float>(), (float)eps);
        c->md_links_newest = LQCD_PREC_FP32;
        c->df_stale = true;
    }
    c->links_derived_stale = true;
    c->launches += 1;
}

static int prepare(lqcd_ctx *c, int prec)
{
    int st;
    if ((st = links_to_prec(c, prec))) return st;
    return mom_to_prec(c, prec);
}

// MD updates move the uploaded (thin) links; they are refused while the
// links in use are stout-smeared.
static int check_thin(const lqcd_ctx *c)
{
    if (c->stout_n) return fail(LQCD_ESTATE, "links are stout-smeared: call lqcd_stout_restore first");
    return LQCD_OK;
}

// Force on the stout levels' thin links from the force F (8 reals per link,
// mom layout) on the smeared links, in place: one local and one gather
// pass per level, from level n-1 down to 0.
static int stout_chain(lqcd_ctx *c, double *F, cudaStream_t s)
{
    const LinkGeo g = link_geo(c);
    const size_t nl = 72 * c->Vh, nf = 64 * c->Vh;
    int st;
    if ((st = c->stout_M.ensure(nl * sizeof(double2))) || (st = c->stout_G.ensure(nl * sizeof(double2))) ||
        (st = c->stout_F.ensure(2 * nf * sizeof(double))))
        return st;
    double *tmp = F == c->stout_F.as<double>() ? c->stout_F.as<double>() + nf : c->stout_F.as<double>();
    double *fa = F, *fb = tmp;
    const unsigned nb = nblocks(8L * (long)c->Vh, kGaugeThreads);
    for (int k = c->stout_n - 1; k >= 0; --k) {
        const double2 *Lk = c->stout_lv.as<double2>() + (size_t)k * nl;
        k_stout_local<<<nb, kGaugeThreads, 0, s>>>(g, Lk, fa, c->stout_rho, c->stout_M.as<double2>(),
                                                    c->stout_G.as<double2>());
        k_stout_gather<<<nb, kGaugeThreads, 0, s>>>(g, Lk, c->stout_M.as<double2>(), c->stout_G.as<double2>(),
                                                     c->stout_rho, fb);
        c->launches += 2;
        std::swap(fa, fb);
    }
    LQCD_CUDA(cudaGetLastError());
    if (fa != F) LQCD_CUDA(cudaMemcpyAsync(F, fa, nf * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return LQCD_OK;
}

}  // namespace lqcd

using namespace lqcd;

extern "C" {

int lqcd_mom_upload(lqcd_ctx *c, const double *H, size_t n)
{
    if (!c) return fail(LQCD_EINVAL, "NULL context");
    LQCD_ON_DEVICE(c->device);
    const size_t want = 4 * c->V * 18;
    if (!H || n != want) return fail(LQCD_EINVAL, "momenta: expected 4*V*18 doubles");
    int st;
    if ((st = c->mom64.ensure(64 * c->Vh * sizeof(double))) || (st = c->mom32.ensure(64 * c->Vh * sizeof(float))))
        return st;
    DevBuf stage;
    if ((st = stage.ensure(want * sizeof(double) + 16))) return st;
    int *bad = (int *)((char *)stage.ptr + want * sizeof(double));
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(stage.ptr, H, want * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) {
        k_mom_from_canonical<<<nblocks(4L * (long)c->V, 256), 256, 0, c->stream>>>(
            link_geo(c), stage.as<double2>(), c->mom64.as<double>(), c->mom32.as<float>(), bad, (long)c->V);
        e = cudaGetLastError();
    }
    int hbad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    stage.release();
    if (e != cudaSuccess) return cuda_fail(e, "momenta upload");
    c->launches += 1;
    c->mom_newest = LQCD_PREC_FP64;  // both copies written; FP64 is the exact one
    if (hbad) {
        c->mom64.release();
        c->mom32.release();
        return fail(LQCD_EINVAL, "momenta must be finite, Hermitian and traceless");
    }
    return LQCD_OK;
}

int lqcd_mom_download(lqcd_ctx *c, double *H, size_t n)
{
    if (!c) return fail(LQCD_EINVAL, "NULL context");
    LQCD_ON_DEVICE(c->device);
    const size_t want = 4 * c->V * 18;
    if (!H || n != want) return fail(LQCD_EINVAL, "momenta: expected 4*V*18 doubles");
    if (!c->mom64.ptr) return fail(LQCD_ESTATE, "no momenta uploaded");
    DevBuf stage;
    int st;
    if ((st = stage.ensure(want * sizeof(double)))) return st;
    const unsigned nb = nblocks(4L * (long)c->V, 256);
    if (c->mom_newest == LQCD_PREC_FP32)
        k_mom_to_canonical<float><<<nb, 256, 0, c->stream>>>(link_geo(c), c->mom32.as<float>(), stage.as<double2>(), (long)c->V);
    else
        k_mom_to_canonical<double><<<nb, 256, 0, c->stream>>>(link_geo(c), c->mom64.as<double>(), stage.as<double2>(), (long)c->V);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(H, stage.ptr, want * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    stage.release();
    if (e != cudaSuccess) return cuda_fail(e, "momenta download");
    c->launches += 1;
    return LQCD_OK;
}

int lqcd_gauge_mom_update(lqcd_ctx *c, int prec, double beta, double eps)
{
    NvtxRange nvtx_("lqcd_gauge_mom_update");
    if (!c) return fail(LQCD_EINVAL, "NULL context");
    LQCD_ON_DEVICE(c->device);
    int st;
    if ((st = check_md(c, prec)) || (st = check_thin(c)) || (st = prepare(c, prec))) return st;
    launch_mom_update(c, prec, beta, eps);
    LQCD_CUDA(cudaGetLastError());
    LQCD_CUDA(cudaStreamSynchronize(c->stream));
    return LQCD_OK;
}

int lqcd_gauge_link_update(lqcd_ctx *c, int prec, double eps)
{
    NvtxRange nvtx_("lqcd_gauge_link_update");
    if (!c) return fail(LQCD_EINVAL, "NULL context");
    LQCD_ON_DEVICE(c->device);
    int st;
    if ((st = check_md(c, prec)) || (st = check_thin(c)) || (st = prepare(c, prec))) return st;
    launch_link_update(c, prec, eps);
    LQCD_CUDA(cudaGetLastError());
    LQCD_CUDA(cudaStreamSynchronize(c->stream));
    return LQCD_OK;
}

int lqcd_gauge_md_steps(lqcd_ctx *c, int prec, double beta, double eps, int n_steps)
{
    NvtxRange nvtx_("lqcd_gauge_md_steps");
    if (!c) return fail(LQCD_EINVAL, "NULL context");
    LQCD_ON_DEVICE(c->device);
    int st;
    if ((st = check_md(c, prec)) || (st = check_thin(c)) || (st = prepare(c, prec))) return st;
    if (n_steps < 0) return fail(LQCD_EINVAL, "n_steps must be >= 0");
    for (int k = 0; k < n_steps; ++k) {
        launch_mom_update(c, prec, beta, eps);
        launch_link_update(c, prec, eps);
    }
    LQCD_CUDA(cudaGetLastError());
    LQCD_CUDA(cudaStreamSynchronize(c->stream));
    return LQCD_OK;
}

int lqcd_fermion_force_update(lqcd_ctx *c, double mass, double a0, const double *a, const double *shifts, int n_shift,
                              double tol, const double *phi, double eps, double *action, lqcd_solve_info *info)
{
    NvtxRange nvtx_("lqcd_fermion_force_update");
    if (!c) return fail(LQCD_EINVAL, "NULL context");
    LQCD_ON_DEVICE(c->device);
    int st;
    if ((st = check_md(c, LQCD_PREC_FP64))) return st;
    if (!phi || !a || !shifts) return fail(LQCD_EINVAL, "NULL argument");
    if (n_shift < 1 || n_shift > kMaxShifts) return fail(LQCD_EINVAL, "n_shift must be in 1..32");
    if (!std::isfinite(eps)) return fail(LQCD_EINVAL, "eps is not finite");
    if ((st = links_to_prec(c, LQCD_PREC_FP64_NATIVE)) || (st = mom_to_prec(c, LQCD_PREC_FP64))) return st;
    const size_t n3 = 3 * c->Vh;
    DevBuf dphi, dr;
    if ((st = dphi.ensure(n3 * sizeof(double2))) || (st = dr.ensure(n3 * sizeof(double2)))) return st;
    cudaStream_t s = c->stream;
    if ((st = host_to_soa(c, phi, dphi.as<double2>(), 1, s))) return st;
    // x_i in the context's scratch (rat_x), S_f = Re <phi, r(A) phi>
    double act = 0.0;
    const int rs = rational_apply_dev(c, mass, a0, a, shifts, n_shift, tol, dphi.as<double2>(), dr.as<double2>(), &act,
                                      info, s);
    if (rs != LQCD_OK && rs != LQCD_ENOCONV) return rs;
    if ((st = c->ff_y.ensure((size_t)n_shift * n3 * sizeof(double2)))) return st;
    const double2 *x = c->rat_x.as<double2>();
    double2 *y = c->ff_y.as<double2>();
    for (int k = 0; k < n_shift; ++k)
        if ((st = deo_launch(c, 1, LQCD_PREC_FP64, 18, x + (size_t)k * n3, y + (size_t)k * n3, s))) return st;
    FFCoef C;
    C.n = n_shift;
    for (int k = 0; k < kMaxShifts; ++k) C.a[k] = k < n_shift ? a[k] : 0.0;
    const unsigned nb = nblocks(8L * (long)c->Vh, kGaugeThreads);
    if (c->stout_n) {
        // force on the smeared links (into a zeroed buffer: 0 - (-1) F), chained
        // back to the thin links, then H -= eps F
        const size_t nf = 64 * c->Vh;
        if ((st = c->stout_F.ensure(2 * nf * sizeof(double)))) return st;
        double *F = c->stout_F.as<double>();
        LQCD_CUDA(cudaMemsetAsync(F, 0, nf * sizeof(double), s));
        k_fermion_force_update<<<nb, kGaugeThreads, 0, s>>>(c->g, c->lnk_nat.as<double2>(), x, y, C, F, -1.0);
        LQCD_CUDA(cudaGetLastError());
        c->launches += 1;
        if ((st = stout_chain(c, F, s))) return st;
        k_daxpy<<<nblocks((long)nf, 256), 256, 0, s>>>((long)nf, -eps, F, c->mom64.as<double>());
    } else {
        k_fermion_force_update<<<nb, kGaugeThreads, 0, s>>>(c->g, c->lnk_nat.as<double2>(), x, y, C,
                                                             c->mom64.as<double>(), eps);
    }
    LQCD_CUDA(cudaGetLastError());
    c->launches += 1;
    c->mom_newest = LQCD_PREC_FP64;
    LQCD_CUDA(cudaStreamSynchronize(s));
    if (action) *action = act;
    if (rs == LQCD_ENOCONV) set_error("solver did not reach tol within max_iter");
    return rs;
}

int lqcd_stout_smear(lqcd_ctx *c, double rho, int n_levels)
{
    NvtxRange nvtx_("lqcd_stout_smear");
    if (!c) return fail(LQCD_EINVAL, "NULL context");
    LQCD_ON_DEVICE(c->device);
    if (!c->links_ok) return fail(LQCD_ESTATE, "no links uploaded");
    if (c->stout_n) return fail(LQCD_ESTATE, "links are already stout-smeared: call lqcd_stout_restore first");
    if (!(rho >= 0.0) || !std::isfinite(rho)) return fail(LQCD_EINVAL, "rho must be finite and >= 0");
    if (n_levels < 1 || n_levels > 8) return fail(LQCD_EINVAL, "n_levels must be in 1..8");
    int st;
    if ((st = links_to_prec(c, LQCD_PREC_FP64_NATIVE))) return st;
    const size_t nl = 72 * c->Vh;
    if ((st = c->stout_lv.ensure((size_t)n_levels * nl * sizeof(double2)))) return st;
    cudaStream_t s = c->stream;
    const unsigned nb = nblocks(8L * (long)c->Vh, kGaugeThreads);
    for (int k = 0; k < n_levels; ++k) {
        double2 *lv = c->stout_lv.as<double2>() + (size_t)k * nl;
        LQCD_CUDA(cudaMemcpyAsync(lv, c->lnk_nat.ptr, nl * sizeof(double2), cudaMemcpyDeviceToDevice, s));
        k_stout_level<<<nb, kGaugeThreads, 0, s>>>(link_geo(c), lv, c->lnk_nat.as<double2>(), rho);
        c->launches += 1;
    }
    LQCD_CUDA(cudaGetLastError());
    c->stout_n = n_levels;
    c->stout_rho = rho;
    c->md_links_newest = LQCD_PREC_FP64;
    c->links_derived_stale = true;
    c->df_stale = true;
    LQCD_CUDA(cudaStreamSynchronize(s));
    return LQCD_OK;
}

int lqcd_stout_restore(lqcd_ctx *c)
{
    if (!c) return fail(LQCD_EINVAL, "NULL context");
    LQCD_ON_DEVICE(c->device);
    if (!c->stout_n) return LQCD_OK;
    const size_t nl = 72 * c->Vh;
    LQCD_CUDA(cudaMemcpyAsync(c->lnk_nat.ptr, c->stout_lv.ptr, nl * sizeof(double2), cudaMemcpyDeviceToDevice,
                              c->stream));
    c->stout_n = 0;
    c->md_links_newest = LQCD_PREC_FP64;
    c->links_derived_stale = true;
    c->df_stale = true;
    LQCD_CUDA(cudaStreamSynchronize(c->stream));
    return LQCD_OK;
}

int lqcd_stout_force(lqcd_ctx *c, const double *F_smeared, double *F_thin, size_t n)
{
    NvtxRange nvtx_("lqcd_stout_force");
    if (!c) return fail(LQCD_EINVAL, "NULL context");
    LQCD_ON_DEVICE(c->device);
    if (!c->stout_n) return fail(LQCD_ESTATE, "links are not stout-smeared");
    const size_t want = 4 * c->V * 18;
    if (!F_smeared || !F_thin || n != want) return fail(LQCD_EINVAL, "forces: expected 4*V*18 doubles");
    const size_t nf = 64 * c->Vh;
    int st;
    if ((st = c->stout_F.ensure(2 * nf * sizeof(double)))) return st;
    DevBuf stage;
    if ((st = stage.ensure(want * sizeof(double) + 16))) return st;
    int *bad = (int *)((char *)stage.ptr + want * sizeof(double));
    cudaStream_t s = c->stream;
    double *F = c->stout_F.as<double>();
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(stage.ptr, F_smeared, want * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "force upload");
    k_mom_from_canonical<<<nblocks(4L * (long)c->V, 256), 256, 0, s>>>(link_geo(c), stage.as<double2>(), F, nullptr,
                                                                        bad, (long)c->V);
    c->launches += 1;
    int hbad = 0;
    LQCD_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    LQCD_CUDA(cudaStreamSynchronize(s));
    if (hbad) return fail(LQCD_EINVAL, "forces must be finite, Hermitian and traceless");
    if ((st = stout_chain(c, F, s))) return st;
    k_mom_to_canonical<double><<<nblocks(4L * (long)c->V, 256), 256, 0, s>>>(link_geo(c), F, stage.as<double2>(),
                                                                            (long)c->V);
    c->launches += 1;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(F_thin, stage.ptr, want * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "force download");
    return LQCD_OK;
}

int lqcd_gauge_action(lqcd_ctx *c, int prec, double beta, double *S)
{
    NvtxRange nvtx_("lqcd_gauge_action");
    if (!c || !S) return fail(LQCD_EINVAL, "NULL argument");
    LQCD_ON_DEVICE(c->device);
    if (!c->links_ok) return fail(LQCD_ESTATE, "no links uploaded");
    if (prec != LQCD_PREC_FP64 && prec != LQCD_PREC_FP32 && prec != LQCD_PREC_FP64_NATIVE)
        return fail(LQCD_EINVAL, "precision must be FP64, FP64_NATIVE or FP32");
    if (prec == LQCD_PREC_FP64_NATIVE) prec = LQCD_PREC_FP64;  // the action is computed from the IEEE master
    int st;
    if ((st = links_to_prec(c, prec == LQCD_PREC_FP64 ? LQCD_PREC_FP64_NATIVE : prec))) return st;
    const unsigned nb = nblocks(2L * (long)c->Vh, kGaugeThreads);
    if ((st = c->md_part.ensure(((size_t)nb + 1) * sizeof(double)))) return st;
    double *part = c->md_part.as<double>();
    if (prec == LQCD_PREC_FP64)
        k_gauge_action_part<double><<<nb, kGaugeThreads, 0, c->stream>>>(link_geo(c), c->lnk_nat.as<double2>(), part);
    else
        k_gauge_action_part<float><<<nb, kGaugeThreads, 0, c->stream>>>(link_geo(c), c->lnk_f18.as<float2>(), part);
    k_gauge_sum_ordered<<<1, 256, 0, c->stream>>>(part, (int)nb, part + nb);
    LQCD_CUDA(cudaGetLastError());
    c->launches += 2;
    LQCD_CUDA(cudaMemcpyAsync(c->h_pinned_d, part + nb, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LQCD_CUDA(cudaStreamSynchronize(c->stream));
    *S = -(beta / 3.0) * c->h_pinned_d[0];
    return LQCD_OK;
}

int lqcd_mom_energy(lqcd_ctx *c, int prec, double *K)
{
    int st;
    if (!K) return fail(LQCD_EINVAL, "NULL argument");
    if (!c) return fail(LQCD_EINVAL, "NULL context");
    LQCD_ON_DEVICE(c->device);
    if ((st = check_md(c, prec)) || (st = mom_to_prec(c, prec))) return st;
    const unsigned nb = nblocks(8L * (long)c->Vh, kGaugeThreads);
    if ((st = c->md_part.ensure(((size_t)nb + 1) * sizeof(double)))) return st;
    double *part = c->md_part.as<double>();
    if (mom_prec(prec) == LQCD_PREC_FP64)
        k_mom_energy_part<double><<<nb, kGaugeThreads, 0, c->stream>>>((int)c->Vh, c->mom64.as<double>(), part);
    else
        k_mom_energy_part<float><<<nb, kGaugeThreads, 0, c->stream>>>((int)c->Vh, c->mom32.as<float>(), part);
    k_gauge_sum_ordered<<<1, 256, 0, c->stream>>>(part, (int)nb, part + nb);
    LQCD_CUDA(cudaGetLastError());
    c->launches += 2;
    LQCD_CUDA(cudaMemcpyAsync(c->h_pinned_d, part + nb, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LQCD_CUDA(cudaStreamSynchronize(c->stream));
    *K = c->h_pinned_d[0];
    return LQCD_OK;
}

}  // extern "C"
