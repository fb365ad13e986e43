// deo.cu -- link upload / storage conversion, host <-> device spinor
// layouts, and the stand-alone D_eo / D_oe launches of the C ABI.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "deo_core.cuh"
#include "internal.h"
#include "stencil_staged.cuh"

namespace lqcd {

// ------------------------------------------------------------------ link conversion
// One thread per (mu, site): canonical [4][V][3][3] complex128 (staged on the
// device) -> every device storage format.  Entries of magnitude >= 2^60 set
// *bad (the df64 pairs must stay inside the FP32 exponent range).
__global__ void k_convert_links(Geom g, const double2 *__restrict__ src, double2 *nat, float4 *df, float2 *f18,
                                float2 *f12, uint32_t *h12, int *bad, long V)
{
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= 4 * V) return;
    const int mu = (int)(t / V);
    const long lex = t - (long)mu * V;
    const int N0 = g.N[0], N1 = g.N[1], N2 = g.N[2];
    const int x0 = (int)(lex % N0);
    const long r1 = lex / N0;
    const int x1 = (int)(r1 % N1);
    const long r2 = r1 / N1;
    const int x2 = (int)(r2 % N2);
    const int x3 = (int)(r2 / N2);
    const int par = (x0 + x1 + x2 + x3) & 1;
    const int idx = (int)(lex >> 1);
    const int Vh = g.Vh;
    for (int c = 0; c < 9; ++c) {
        const double2 d = src[t * 9 + c];
        if (!(fabs(d.x) < 0x1p60) || !(fabs(d.y) < 0x1p60)) atomicOr(bad, 1);
        nat[link_base(mu, par, 9, Vh) + (size_t)c * Vh + idx] = d;
        const float2 re = f64_to_df_slow(d.x), im = f64_to_df_slow(d.y);
        df[link_base(mu, par, 9, Vh) + (size_t)c * Vh + idx] = make_float4(re.x, re.y, im.x, im.y);
        const float2 f = make_float2((float)d.x, (float)d.y);
        f18[link_base(mu, par, 9, Vh) + (size_t)c * Vh + idx] = f;
        if (c < 6) {
            f12[(link_base(mu, par, 3, Vh) + (size_t)(c >> 1) * Vh + idx) * 2 + (c & 1)] = f;
            const __half2 h = __floats2half2_rn(f.x, f.y);
            const uint32_t w = *reinterpret_cast<const uint32_t *>(&h);
            if (c < 4)
                h12[((size_t)(mu * 2 + par) * Vh + idx) * 4 + c] = w;
            else
                h12[(size_t)8 * Vh * 4 + ((size_t)(mu * 2 + par) * Vh + idx) * 2 + (c - 4)] = w;
        }
    }
}

__global__ void k_links_to_canonical(Geom g, const double2 *__restrict__ nat, double2 *dst, long V)
{
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= 4 * V) return;
    const int mu = (int)(t / V);
    const long lex = t - (long)mu * V;
    const int N0 = g.N[0], N1 = g.N[1], N2 = g.N[2];
    const int x0 = (int)(lex % N0);
    const long r1 = lex / N0;
    const int x1 = (int)(r1 % N1);
    const long r2 = r1 / N1;
    const int x2 = (int)(r2 % N2);
    const int x3 = (int)(r2 / N2);
    const int par = (x0 + x1 + x2 + x3) & 1;
    const int idx = (int)(lex >> 1);
    for (int c = 0; c < 9; ++c) dst[t * 9 + c] = nat[link_base(mu, par, 9, g.Vh) + (size_t)c * g.Vh + idx];
}

// Tile-ordered FP64 link stream of the staged kernels (stencil_staged.cuh),
// gathered from the SoA df64 links: element (P, tile, h, c, s) is component
// c of the forward (h even) or backward (h odd) link of direction h/2 seen
// from output site tile*256 + s of parity P; zero beyond V/2.
__global__ void k_build_staged_df(Geom g, const float4 *__restrict__ L, float4 *__restrict__ st, int ntiles)
{
    const size_t n = staged_df_elems(ntiles);
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int s = (int)(t % kTile);
    size_t r = t / kTile;
    const int c = (int)(r % kDFComps);
    r /= kDFComps;
    const int h = (int)(r % 8);
    r /= 8;
    const int tile = (int)(r % (size_t)ntiles);
    const int P = (int)(r / (size_t)ntiles);
    const int i = tile * kTile + s;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < g.Vh) {
        Stencil S;
        make_stencil(g, i, P, S);
        int f, b;
        uint32_t nf, nb;
        const int mu = h >> 1;
        hop(g, S, mu, f, b, nf, nb);
        if ((h & 1) == 0)
            v = L[link_base(mu, P, 9, g.Vh) + (size_t)c * g.Vh + i];
        else
            v = L[link_base(mu, 1 - P, 9, g.Vh) + (size_t)c * g.Vh + b];
    }
    st[t] = v;
}

// Every derived link format from the FP64 SoA master (after molecular
// dynamics moved the links): one thread per (mu, parity, site), the same
// conversions as k_convert_links.
__global__ void k_derive_links(int Vh, const double2 *__restrict__ nat, float4 *df, float2 *f18, float2 *f12,
                               uint32_t *h12)
{
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= 8L * Vh) return;
    const int idx = (int)(t % Vh), mp = (int)(t / Vh);
    const int mu = mp >> 1, par = mp & 1;
    for (int c = 0; c < 9; ++c) {
        const size_t o = link_base(mu, par, 9, Vh) + (size_t)c * Vh + idx;
        const double2 d = nat[o];
        const float2 re = f64_to_df_slow(d.x), im = f64_to_df_slow(d.y);
        df[o] = make_float4(re.x, re.y, im.x, im.y);
        const float2 f = make_float2((float)d.x, (float)d.y);
        f18[o] = f;
        if (c < 6) {
            f12[(link_base(mu, par, 3, Vh) + (size_t)(c >> 1) * Vh + idx) * 2 + (c & 1)] = f;
            const __half2 h = __floats2half2_rn(f.x, f.y);
            const uint32_t w = *reinterpret_cast<const uint32_t *>(&h);
            if (c < 4)
                h12[((size_t)(mu * 2 + par) * Vh + idx) * 4 + c] = w;
            else
                h12[(size_t)8 * Vh * 4 + ((size_t)(mu * 2 + par) * Vh + idx) * 2 + (c - 4)] = w;
        }
    }
}

__global__ void k_promote_f32_links(const float2 *__restrict__ a, double2 *b, long n)
{
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t < n) b[t] = make_double2((double)a[t].x, (double)a[t].y);
}

int links_ready(lqcd_ctx *c)
{
    if (!c->links_ok) return fail(LQCD_ESTATE, "no links uploaded");
    if (!c->links_derived_stale) return LQCD_OK;
    const long Vh = (long)c->Vh;
    if (c->md_links_newest == LQCD_PREC_FP32) {
        const long n = 72 * Vh;
        k_promote_f32_links<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(c->lnk_f18.as<float2>(),
                                                                           c->lnk_nat.as<double2>(), n);
        c->launches += 1;
        c->md_links_newest = LQCD_PREC_FP64;
    }
    k_derive_links<<<(unsigned)((8 * Vh + 255) / 256), 256, 0, c->stream>>>(
        (int)Vh, c->lnk_nat.as<double2>(), c->lnk_df.as<float4>(), c->lnk_f18.as<float2>(), c->lnk_f12.as<float2>(),
        c->lnk_h12.as<uint32_t>());
    c->launches += 1;
    if (c->lnk_dfs.ptr) {
        const int ntiles = (int)((Vh + kTile - 1) / kTile);
        const size_t ne = staged_df_elems(ntiles);
        k_build_staged_df<<<(unsigned)((ne + 255) / 256), 256, 0, c->stream>>>(c->g, c->lnk_df.as<float4>(),
                                                                          c->lnk_dfs.as<float4>(), ntiles);
        c->launches += 1;
    }
    LQCD_CUDA(cudaGetLastError());
    c->links_derived_stale = false;
    c->df_stale = false;
    return LQCD_OK;
}

int upload_links(lqcd_ctx *c, const double *host, size_t n)
{
    const size_t want = 4 * c->V * 18;
    if (!host) return fail(LQCD_EINVAL, "links pointer is NULL");
    if (n != want) return fail(LQCD_EINVAL, "links: expected 4*V*18 = " + std::to_string(want) + " doubles, got " + std::to_string(n));
    const size_t Vh = c->Vh;
    int st;
    // until this upload completes the context has no usable links: a failure
    // below (allocation, copy, invalid entries) leaves it in that state
    c->links_ok = false;
    if ((st = c->lnk_nat.ensure(72 * Vh * sizeof(double2)))) return st;
    if ((st = c->lnk_df.ensure(72 * Vh * sizeof(float4)))) return st;
    if ((st = c->lnk_f18.ensure(72 * Vh * sizeof(float2)))) return st;
    if ((st = c->lnk_f12.ensure(24 * Vh * sizeof(float4)))) return st;
    if ((st = c->lnk_h12.ensure(8 * Vh * (sizeof(uint4) + sizeof(uint2))))) return st;
    const int ntiles = (int)((Vh + kTile - 1) / kTile);
    c->stout_n = 0;  // new links: no stout levels
    (void)persist_blocks();  // occupancy query now, never first inside a graph capture
    const bool staged = c->opts.staged && staged_deo_ready() && staged_solver_ready();
    if (staged) {
        if ((st = c->lnk_dfs.ensure(staged_df_elems(ntiles) * sizeof(float4)))) return st;
        if ((st = c->err_word.ensure(4 * sizeof(int)))) return st;
    } else {
        c->lnk_dfs.release();
    }
    DevBuf stage;
    if ((st = stage.ensure(want * sizeof(double) + 16))) return st;
    int *bad = (int *)((char *)stage.ptr + want * sizeof(double));
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(stage.ptr, host, want * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) {
        const long V = (long)c->V;
        const int bs = 256;
        const long nb = (4 * V + bs - 1) / bs;
        k_convert_links<<<(unsigned)nb, bs, 0, c->stream>>>(c->g, stage.as<double2>(), c->lnk_nat.as<double2>(),
                                                            c->lnk_df.as<float4>(), c->lnk_f18.as<float2>(),
                                                            c->lnk_f12.as<float2>(), c->lnk_h12.as<uint32_t>(), bad, V);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && staged) {
        const size_t ne = staged_df_elems(ntiles);
        k_build_staged_df<<<(unsigned)((ne + 255) / 256), 256, 0, c->stream>>>(c->g, c->lnk_df.as<float4>(),
                                                                          c->lnk_dfs.as<float4>(), ntiles);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemsetAsync(c->err_word.ptr, 0, 4 * sizeof(int), c->stream);
    }
    int hbad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    stage.release();
    if (e != cudaSuccess) return cuda_fail(e, "links upload");
    if (hbad) {
        c->links_ok = false;
        return fail(LQCD_EINVAL, "links: an entry is NaN/Inf or has magnitude >= 2^60");
    }
    c->links_ok = true;
    c->md_links_newest = LQCD_PREC_FP64;
    c->links_derived_stale = false;
    c->df_stale = false;
    return LQCD_OK;
}

int download_links(lqcd_ctx *c, double *host, size_t n)
{
    const size_t want = 4 * c->V * 18;
    if (!host || n != want) return fail(LQCD_EINVAL, "links download: expected 4*V*18 doubles");
    if (int lr = links_ready(c)) return lr;
    DevBuf stage;
    int st;
    if ((st = stage.ensure(want * sizeof(double)))) return st;
    const long V = (long)c->V;
    k_links_to_canonical<<<(unsigned)((4 * V + 255) / 256), 256, 0, c->stream>>>(c->g, c->lnk_nat.as<double2>(),
                                                                              stage.as<double2>(), V);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, stage.ptr, want * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    stage.release();
    if (e != cudaSuccess) return cuda_fail(e, "links download");
    return LQCD_OK;
}

// ------------------------------------------------------------------ spinor layouts
// host canonical [nf][Vh][3] complex128 <-> device [nf][3][Vh] double2
__global__ void k_aos_to_soa(const double2 *__restrict__ a, double2 *__restrict__ s, long Vh, int nf)
{
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= Vh * nf) return;
    const long f = t / Vh, i = t - f * Vh;
    for (int cc = 0; cc < 3; ++cc) s[(f * 3 + cc) * Vh + i] = a[t * 3 + cc];
}

__global__ void k_soa_to_aos(const double2 *__restrict__ s, double2 *__restrict__ a, long Vh, int nf)
{
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= Vh * nf) return;
    const long f = t / Vh, i = t - f * Vh;
    for (int cc = 0; cc < 3; ++cc) a[t * 3 + cc] = s[(f * 3 + cc) * Vh + i];
}

int host_to_soa(lqcd_ctx *c, const double *host, double2 *dev_soa, int nf, cudaStream_t s)
{
    const size_t bytes = (size_t)nf * c->Vh * 3 * sizeof(double2);
    int st;
    if ((st = c->io_a.ensure(bytes))) return st;
    LQCD_CUDA(cudaMemcpyAsync(c->io_a.ptr, host, bytes, cudaMemcpyHostToDevice, s));
    const long n = (long)c->Vh * nf;
    k_aos_to_soa<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(c->io_a.as<double2>(), dev_soa, (long)c->Vh, nf);
    LQCD_CUDA(cudaGetLastError());
    return LQCD_OK;
}

int soa_to_host(lqcd_ctx *c, const double2 *dev_soa, double *host, int nf, cudaStream_t s)
{
    const size_t bytes = (size_t)nf * c->Vh * 3 * sizeof(double2);
    int st;
    if ((st = c->io_b.ensure(bytes))) return st;
    const long n = (long)c->Vh * nf;
    k_soa_to_aos<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(dev_soa, c->io_b.as<double2>(), (long)c->Vh, nf);
    LQCD_CUDA(cudaGetLastError());
    LQCD_CUDA(cudaMemcpyAsync(host, c->io_b.ptr, bytes, cudaMemcpyDeviceToHost, s));
    return LQCD_OK;
}

// ------------------------------------------------------------------ stand-alone D_eo
// FP64 result from df64 arithmetic; IEEE complex128 spinors in and out.
// RECON 12 streams the first two rows of every link and rebuilds the third.
template <int RECON>
__device__ __forceinline__ void deo_df_ieee_site(const Geom &g, const float4 *__restrict__ L,
                                                 const double2 *__restrict__ in, double2 *__restrict__ out, int P)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.Vh) return;
    Stencil S;
    make_stencil(g, i, P, S);
    float2 res[6];
    bool bad = false;
    deo_site_df<SF_IEEE, RECON>(g, L, in, S, i, P, g.Vh, res, bad);
    double2 o[3];
    if (bad) {
        deo_site_native_from_df(g, L, in, S, i, P, g.Vh, o);
    } else {
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) o[cc] = make_double2(df_to_f64(res[2 * cc]), df_to_f64(res[2 * cc + 1]));
    }
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) out[(size_t)cc * g.Vh + i] = o[cc];
}

__global__ void __launch_bounds__(kTile, 2)
    k_deo_df_ieee(Geom g, const float4 *__restrict__ L, const double2 *__restrict__ in, double2 *__restrict__ out, int P)
{
    deo_df_ieee_site<18>(g, L, in, out, P);
}

__global__ void __launch_bounds__(kTile, 2)
    k_deo_df12_ieee(Geom g, const float4 *__restrict__ L, const double2 *__restrict__ in, double2 *__restrict__ out,
                    int P)
{
    deo_df_ieee_site<12>(g, L, in, out, P);
}

// Same operator with SPLIT threads per site (adjacent lanes): thread `part`
// takes directions mu in [part*4/SPLIT, (part+1)*4/SPLIT) (SPLIT 8: one
// half-hop, direction part/2, forward for even part), the partial
// double-float sums are merged across the lanes by a fixed xor butterfly
// (two_sum is exact and symmetric, so every lane ends with the same value)
// and the first lane writes.  Shortens the per-thread chain of dependent
// loads on small lattices, where one wave of threads cannot fill the GPU.
template <int SPLIT>
__global__ void __launch_bounds__(kTile)
    k_deo_df_ieee_split(Geom g, const float4 *__restrict__ L, const double2 *__restrict__ in,
                        double2 *__restrict__ out, int P)
{
    const long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
    const int i = (int)(tid / SPLIT);
    const int part = (int)(tid - (long)i * SPLIT);
    if (i >= g.Vh) return;  // all SPLIT lanes of a site leave together
    const unsigned lane = threadIdx.x & 31u;
    const unsigned gmask = ((1u << SPLIT) - 1u) << (lane & ~(unsigned)(SPLIT - 1));
    Stencil S;
    make_stencil(g, i, P, S);
    Acc2 acc[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) acc_zero(acc[k]);
    bool bad = false;
    const int Vh = g.Vh;
    if (SPLIT == 8) {
        // one half-hop per lane: lane part takes direction part / 2, forward
        // (even part) or backward (odd part); all its loads are independent
        const int mu = part >> 1;
        int f, b;
        uint32_t nf, nb;
        hop(g, S, mu, f, b, nf, nb);
        float4 U[9], v[3];
        float ch[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if ((part & 1) == 0) {
            load_link_df(L, mu, P, i, Vh, U);
            load_spinor_df<SF_IEEE>(in, f, Vh, nf, v, bad);
            hop_fwd_df(acc, ch, U, v);
        } else {
            load_link_df(L, mu, 1 - P, b, Vh, U);
            load_spinor_df<SF_IEEE>(in, b, Vh, nb, v, bad);
            hop_bwd_df(acc, ch, U, v);
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) acc_flush(acc[k], ch[k]);
    } else {
#pragma unroll 1
        for (int mu = part * (4 / SPLIT); mu < (part + 1) * (4 / SPLIT); ++mu) {
            int f, b;
            uint32_t nf, nb;
            hop(g, S, mu, f, b, nf, nb);
            float4 U[9], v[3];
            float ch[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            load_link_df(L, mu, P, i, Vh, U);
            load_spinor_df<SF_IEEE>(in, f, Vh, nf, v, bad);
            hop_fwd_df(acc, ch, U, v);
            load_link_df(L, mu, 1 - P, b, Vh, U);
            load_spinor_df<SF_IEEE>(in, b, Vh, nb, v, bad);
            hop_bwd_df(acc, ch, U, v);
#pragma unroll
            for (int k = 0; k < 6; ++k) acc_flush(acc[k], ch[k]);
        }
    }
#pragma unroll
    for (int o = 1; o < SPLIT; o <<= 1)
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float s2 = __shfl_xor_sync(gmask, acc[k].s, o);
            const float c2 = __shfl_xor_sync(gmask, acc[k].c, o);
            acc_merge(acc[k], s2, c2);
        }
    bad = __any_sync(gmask, bad);
    if (part != 0) return;
    double2 o[3];
    if (bad) {
        deo_site_native_from_df(g, L, in, S, i, P, Vh, o);
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float2 re = acc_result(acc[2 * c]), im = acc_result(acc[2 * c + 1]);
            o[c] = make_double2(df_to_f64(make_float2(0.5f * re.x, 0.5f * re.y)),
                                df_to_f64(make_float2(0.5f * im.x, 0.5f * im.y)));
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) out[(size_t)c * Vh + i] = o[c];
}

__global__ void __launch_bounds__(kTile, 2)
    k_deo_nat(Geom g, const double2 *__restrict__ L, const double2 *__restrict__ in, double2 *__restrict__ out, int P)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.Vh) return;
    Stencil S;
    make_stencil(g, i, P, S);
    double2 o[3];
    deo_site_nat(g, L, in, S, i, P, g.Vh, o);
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) out[(size_t)cc * g.Vh + i] = o[cc];
}

template <int LF, int UNROLL = 1>
__global__ void __launch_bounds__(kTile)
    k_deo_f32(Geom g, const void *__restrict__ L, const float2 *__restrict__ in, float2 *__restrict__ out, int P)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.Vh) return;
    Stencil S;
    make_stencil(g, i, P, S);
    float2 o[3];
    deo_site_f32<LF, UNROLL>(g, L, in, S, i, P, g.Vh, o);
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) out[(size_t)cc * g.Vh + i] = o[cc];
}

// FP16 links (12 reals) and FP16 spinors with a per-site FP32 norm: the
// value of colour c at half index k is norm[k] * in[c][k] (half2 re, im).
// Products and sums in FP32, as deo_site_f32 with FP16 links, the direction
// loop unrolled (the FP16 kernels are latency-bound rolled).  The output
// site's norm is the largest |re|, |im| of its three colours, and the halves
// are the result over that norm, rounded to nearest (0 for a zero result).
__global__ void __launch_bounds__(kTile)
    k_deo_h16(Geom g, const void *__restrict__ L, const __half2 *__restrict__ in, const float *__restrict__ in_norm,
              __half2 *__restrict__ out, float *__restrict__ out_norm, int P)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int Vh = g.Vh;
    if (i >= Vh) return;
    Stencil S;
    make_stencil(g, i, P, S);
    float2 acc[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        int f, b;
        uint32_t nf, nb;
        hop(g, S, mu, f, b, nf, nb);
#pragma unroll
        for (int dir = 0; dir < 2; ++dir) {
            const int idx = dir == 0 ? f : b;
            const uint32_t ng = dir == 0 ? nf : nb;
            float2 U[9], v[3];
            load_link_f32<LF_F16_12>(L, mu, dir == 0 ? P : 1 - P, dir == 0 ? i : b, Vh, U);
            const float nrm = __uint_as_float(__float_as_uint(__ldg(in_norm + idx)) ^ ng);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float2 t = __half22float2(in[(size_t)c * Vh + idx]);
                v[c] = make_float2(nrm * t.x, nrm * t.y);
            }
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int bb = 0; bb < 3; ++bb) {
                    if (dir == 0) {
                        const float2 u = U[a * 3 + bb];
                        acc[a].x = __fmaf_rn(u.x, v[bb].x, __fmaf_rn(-u.y, v[bb].y, acc[a].x));
                        acc[a].y = __fmaf_rn(u.x, v[bb].y, __fmaf_rn(u.y, v[bb].x, acc[a].y));
                    } else {
                        const float2 u = U[bb * 3 + a];
                        acc[a].x = __fmaf_rn(u.x, v[bb].x, __fmaf_rn(u.y, v[bb].y, acc[a].x));
                        acc[a].y = __fmaf_rn(u.x, v[bb].y, __fmaf_rn(-u.y, v[bb].x, acc[a].y));
                    }
                }
        }
    }
    float m = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        acc[c] = make_float2(0.5f * acc[c].x, 0.5f * acc[c].y);
        m = fmaxf(m, fmaxf(fabsf(acc[c].x), fabsf(acc[c].y)));
    }
    const float inv = m > 0.f ? 1.f / m : 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) out[(size_t)c * Vh + i] = __floats2half2_rn(acc[c].x * inv, acc[c].y * inv);
    out_norm[i] = m;
}

// Stand-alone D_eo, consumers.
template <int RECON>
__device__ __forceinline__ void deo_staged_consume(const Geom &g, RingDF &R, const float4 *__restrict__ L,
                                                   const double2 *__restrict__ in, double2 *__restrict__ out, int P,
                                                   int ntiles, int *err)
{
    const int Vh = g.Vh;
    uint32_t q = 0;
    bool dead = false;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int i = tile * kTile + threadIdx.x;
        const bool live = i < Vh;
        Stencil S;
        make_stencil(g, live ? i : 0, P, S);
        float2 res[6];
        bool bad = false;
        deo_site_df_staged<SF_IEEE, RECON>(R, q, dead, g, in, S, Vh, res, bad);
        if (!live) continue;
        double2 o[3];
        if (bad) {
            deo_site_native_from_df(g, L, in, S, i, P, Vh, o);
        } else {
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) o[cc] = make_double2(df_to_f64(res[2 * cc]), df_to_f64(res[2 * cc + 1]));
        }
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) out[(size_t)cc * Vh + i] = o[cc];
    }
    if (dead) atomicOr(err, 1);
}

// Stand-alone FP64 D_eo with the link stream staged through shared memory
// (stencil_staged.cuh): IEEE complex128 spinors in and out, double-float
// arithmetic, the native FP64 fallback for inputs outside the df64 window.
// Persistent: gridDim.x <= resident blocks; err bit 0/1 records a stall.
// RECON 12 copies the first two rows of every hop's stage and rebuilds the
// third row in the consumers.
template <int RECON>
__global__ void __launch_bounds__(kStagedThreads, kStagedMinBlocks)
    k_deo_df_ieee_staged(Geom g, const float4 *__restrict__ Lst, const float4 *__restrict__ L,
                         const double2 *__restrict__ in, double2 *__restrict__ out, int P, int ntiles, int *err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    RingDF &R = *reinterpret_cast<RingDF *>(smem_raw);
    ring_init(R);
    if (threadIdx.x >= kStagedConsumers) {
        if (threadIdx.x == kStagedConsumers) {
            int tile = blockIdx.x;
            const bool ok = ring_produce<RECON>(R, [&](const float4 *&base) -> bool {
                if (tile >= ntiles) return false;
                base = staged_tile_base(Lst, P, ntiles, tile);
                tile += gridDim.x;
                return true;
            });
            if (!ok) atomicOr(err, 2);
        }
    } else {
        deo_staged_consume<RECON>(g, R, L, in, out, P, ntiles, err);
    }
    ring_finish(R);
}


// Self-test of the bounded stage wait.  One block of the staged layout whose
// producer issues nothing: every consumer waits for stage 0, which no copy
// ever fills, gives up after limit_ns (the wait the staged kernels use, with
// a short limit), records the stall, and the block leaves through
// ring_finish like a staged kernel.  *status = 1 when the waits gave up.
__global__ void __launch_bounds__(kStagedThreads) k_stage_wait_selftest(uint64_t limit_ns, int *status)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    RingDF &R = *reinterpret_cast<RingDF *>(smem_raw);
    ring_init(R);
    if (threadIdx.x < kStagedConsumers && !mbar_wait(&R.full[0], 0u, limit_ns)) R.stalled = 1;
    __syncthreads();
    if (threadIdx.x == 0) *status = R.stalled;
    ring_finish(R);
}

int stage_wait_selftest(lqcd_ctx *c, double limit_s)
{
    if (!(limit_s > 0.0 && limit_s <= 10.0)) return fail(LQCD_EINVAL, "limit must be in (0, 10] seconds");
    LQCD_CUDA(cudaFuncSetAttribute(k_stage_wait_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)kRingDFBytes));
    DevBuf st;
    int rc;
    if ((rc = st.ensure(sizeof(int)))) return rc;
    LQCD_CUDA(cudaMemsetAsync(st.ptr, 0, sizeof(int), c->stream));
    k_stage_wait_selftest<<<1, kStagedThreads, kRingDFBytes, c->stream>>>((uint64_t)(limit_s * 1e9), st.as<int>());
    LQCD_CUDA(cudaGetLastError());
    c->launches += 1;
    int h = 0;
    LQCD_CUDA(cudaMemcpyAsync(&h, st.ptr, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    LQCD_CUDA(cudaStreamSynchronize(c->stream));
    if (h) return fail(LQCD_ETIMEOUT, "self-test: the bounded wait for an unfilled stage ran out");
    return LQCD_OK;
}

// Residency of the staged stand-alone kernel per device (0: cannot run).
static std::mutex g_staged_mu;
static int g_staged_blocks[64];
static bool g_staged_done[64];

bool staged_deo_ready()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
    std::lock_guard<std::mutex> lk(g_staged_mu);
    if (!g_staged_done[dev]) {
        g_staged_done[dev] = true;
        int occ = 0, nsm = 0;
        int occ12 = 0;
        if (cudaFuncSetAttribute(k_deo_df_ieee_staged<18>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kRingDFBytes) == cudaSuccess &&
            cudaFuncSetAttribute(k_deo_df_ieee_staged<12>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kRingDFBytes) == cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_deo_df_ieee_staged<18>, kStagedThreads,
                                                          kRingDFBytes) == cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ12, k_deo_df_ieee_staged<12>, kStagedThreads,
                                                          kRingDFBytes) == cudaSuccess &&
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
            g_staged_blocks[dev] = std::min(occ, occ12) * nsm;
        cudaGetLastError();  // a refusal above only disables the staged path
    }
    return g_staged_blocks[dev] > 0;
}

static int staged_deo_blocks(int dev)
{
    std::lock_guard<std::mutex> lk(g_staged_mu);
    return dev >= 0 && dev < 64 ? g_staged_blocks[dev] : 0;
}

bool staged_active(const lqcd_ctx *c) { return c->opts.staged && c->lnk_dfs.ptr != nullptr; }

int deo_check_stall(lqcd_ctx *c)
{
    if (!c->err_word.ptr) return LQCD_OK;
    int w = 0;
    LQCD_CUDA(cudaMemcpyAsync(&w, c->err_word.ptr, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    LQCD_CUDA(cudaStreamSynchronize(c->stream));
    if (!w) return LQCD_OK;
    LQCD_CUDA(cudaMemsetAsync(c->err_word.ptr, 0, sizeof(int), c->stream));
    LQCD_CUDA(cudaStreamSynchronize(c->stream));
    return fail(LQCD_ETIMEOUT, "a staged D_eo wait for shared-memory link data ran out");
}

// ------------------------------------------------------------------ autotuner
// Threads per block of the stand-alone D_eo kernels, chosen per (variant,
// lattice) by timing 64, 128 and 256 on the first call (CUDA events on the
// call's stream, L2 emptied before each timed launch; D_eo does not depend
// on the block size, so the tuning runs produce the right output).  Cached for the process and, when the
// environment variable LQCD_TUNE_CACHE names a file, across processes.
// During stream capture the default (256) is used without tuning.
static std::mutex g_tune_mu;
static std::map<std::string, int> g_tune;
static bool g_tune_loaded = false;

static std::string tune_key(const lqcd_ctx *c, int variant)
{
    char buf[128];
    snprintf(buf, sizeof buf, "deo2 v%d %dx%dx%dx%d", variant, c->dims[0], c->dims[1], c->dims[2], c->dims[3]);
    return buf;
}

static void tune_load()
{
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *f = getenv("LQCD_TUNE_CACHE");
    if (!f) return;
    FILE *fp = fopen(f, "r");
    if (!fp) return;
    char line[256];
    while (fgets(line, sizeof line, fp)) {
        char k1[16];
        int v, d0, d1, d2, d3, bs;
        if (sscanf(line, "%15s v%d %dx%dx%dx%d %d", k1, &v, &d0, &d1, &d2, &d3, &bs) == 7) {
            char buf[128];
            snprintf(buf, sizeof buf, "%s v%d %dx%dx%dx%d", k1, v, d0, d1, d2, d3);
            g_tune[buf] = bs;
        }
    }
    fclose(fp);
}

static void tune_save(const std::string &key, int bs)
{
    const char *f = getenv("LQCD_TUNE_CACHE");
    if (!f) return;
    FILE *fp = fopen(f, "a");
    if (!fp) return;
    fprintf(fp, "%s %d\n", key.c_str(), bs);
    fclose(fp);
}

// Reads n float4 of buf (grid-stride) and keeps nothing: run between two
// timed launches of the tuner it replaces every line of L2 with clean lines
// of buf, so the next launch starts with cold links and spinors, as a
// stand-alone application does.  (The store is never taken: the XOR of the
// buffer's zero bytes is zero.)
__global__ void k_l2_evict_read(const float4 *__restrict__ buf, size_t n, unsigned *sink)
{
    unsigned x = 0;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const float4 v = __ldcg(buf + k);
        x ^= __float_as_uint(v.x) ^ __float_as_uint(v.y) ^ __float_as_uint(v.z) ^ __float_as_uint(v.w);
    }
    if (x == 0x9E3779B9u) *sink = x;
}

// Scratch of the tuner's L2 eviction: twice the L2 size, zero-filled.
constexpr size_t kEvictBytes = 256ull << 20;

// Candidates are encoded as kind * 1024 + threads per block; kind selects a
// kernel variant (0: one thread per site, 1/2/4: 2/4/8 threads per site,
// 3: the staged persistent kernel, 5: FP32/FP16 with the direction loop
// unrolled).
template <class Launch>
static int tuned_launch(lqcd_ctx *c, int variant, cudaStream_t s, Launch launch, int ncand = 3,
                        const int *cands = nullptr)
{
    const std::string key = tune_key(c, variant);
    int bs = 0;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_load();
        auto it = g_tune.find(key);
        if (it != g_tune.end()) bs = it->second;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cap);
    if (bs == 0 && cap != cudaStreamCaptureStatusNone) bs = kTile;
    if (bs == 0) {
        const int def[3] = {64, 128, 256};
        const int *cand = cands ? cands : def;
        float best = 1e30f;
        cudaEvent_t e0, e1;
        LQCD_CUDA(cudaEventCreate(&e0));
        LQCD_CUDA(cudaEventCreate(&e1));
        // each timed launch starts with L2 emptied of the operator's data (a
        // stand-alone application streams cold links); without the scratch
        // buffer (allocation refused) the launches run back to back
        DevBuf evict;
        unsigned *sink = nullptr;
        if (evict.ensure(kEvictBytes + 16) == LQCD_OK &&
            cudaMemsetAsync(evict.ptr, 0, kEvictBytes + 16, s) == cudaSuccess)
            sink = (unsigned *)((char *)evict.ptr + kEvictBytes);
        else
            set_error("");
        cudaGetLastError();
        for (int k = 0; k < ncand; ++k) {
            launch(cand[k]);  // warm
            float t = 0.f;
            for (int r = 0; r < 3; ++r) {
                if (sink) {
                    k_l2_evict_read<<<1216, 256, 0, s>>>((const float4 *)evict.ptr, kEvictBytes / sizeof(float4),
                                                         sink);
                    c->launches += 1;
                }
                float tr = 0.f;
                cudaEventRecord(e0, s);
                launch(cand[k]);
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                cudaEventElapsedTime(&tr, e0, e1);
                t += tr;
            }
            c->launches += 4;
            if (t < best) {
                best = t;
                bs = cand[k];
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        evict.release();
        LQCD_CUDA(cudaGetLastError());
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[key] = bs;
        tune_save(key, bs);
    }
    launch(bs);
    c->launches += 1;
    return LQCD_OK;
}

int deo_tuned_block(const lqcd_ctx *c, int variant)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(tune_key(c, variant));
    return it == g_tune.end() ? 0 : it->second;
}

// Tuner variant of a (prec, recon) pair of the stand-alone D_eo (-1: none).
static int deo_variant(int prec, int recon)
{
    if (prec == LQCD_PREC_FP64) return recon == 12 ? 5 : (recon == 18 ? 0 : -1);
    if (prec == LQCD_PREC_FP64_NATIVE) return recon == 18 ? 1 : -1;
    if (prec == LQCD_PREC_FP32) return recon == 18 ? 2 : (recon == 12 ? 3 : -1);
    if (prec == LQCD_PREC_FP16) return recon == 12 ? 4 : -1;
    return -1;
}

int deo_launch(lqcd_ctx *c, int P, int prec, int recon, const void *in, void *out, cudaStream_t s)
{
    if (int lr = links_ready(c)) return lr;
    if (P != 0 && P != 1) return fail(LQCD_EINVAL, "out_parity must be 0 or 1");
    if (!in || !out) return fail(LQCD_EINVAL, "NULL spinor pointer");
    if (in == out) return fail(LQCD_EINVAL, "in and out must not overlap");
    const Geom g = c->g;
    auto nb = [&](int bs) { return (unsigned)((c->Vh + bs - 1) / bs); };
    int st = LQCD_OK;
    switch (prec) {
    case LQCD_PREC_FP64: {
        if (recon != 18 && recon != 12) return fail(LQCD_EINVAL, "recon must be 18 or 12");
        const float4 *L = c->lnk_df.as<float4>();
        const bool staged = staged_active(c);
        const int ntiles = (int)((c->Vh + kTile - 1) / kTile);
        const int sgrid = std::min(ntiles, staged_deo_blocks(c->device));
        if (recon == 12) {
            // 12-real links: the first two rows of the df64 arrays (96 of 144
            // bytes per link) and the third row rebuilt, per thread or staged
            static const int cand12[4] = {64, 128, 256, 3072 + kStagedThreads};
            st = tuned_launch(c, 5, s, [&](int code) {
                int kind = code >> 10, bs = code & 1023;
                if (kind == 3 && (!staged || sgrid < 1)) kind = 0, bs = kTile;
                if (kind == 3)
                    k_deo_df_ieee_staged<12><<<(unsigned)sgrid, kStagedThreads, kRingDFBytes, s>>>(
                        g, c->lnk_dfs.as<float4>(), L, (const double2 *)in, (double2 *)out, P, ntiles,
                        c->err_word.as<int>());
                else
                    k_deo_df12_ieee<<<nb(bs), bs, 0, s>>>(g, L, (const double2 *)in, (double2 *)out, P);
            }, staged ? 4 : 3, cand12);
            break;
        }
        static const int cand[10] = {64, 128, 256, 1024 + 128, 1024 + 256, 2048 + 128, 2048 + 256,
                                     4096 + 128, 4096 + 256, 3072 + kStagedThreads};
        st = tuned_launch(c, 0, s, [&](int code) {
            int kind = code >> 10, bs = code & 1023;
            if (kind == 3 && (!staged || sgrid < 1)) kind = 0, bs = kTile;  // staged stream not built
            if (kind == 3)
                k_deo_df_ieee_staged<18><<<(unsigned)sgrid, kStagedThreads, kRingDFBytes, s>>>(
                    g, c->lnk_dfs.as<float4>(), L, (const double2 *)in, (double2 *)out, P, ntiles,
                    c->err_word.as<int>());
            else if (kind == 0)
                k_deo_df_ieee<<<nb(bs), bs, 0, s>>>(g, L, (const double2 *)in, (double2 *)out, P);
            else if (kind == 1)
                k_deo_df_ieee_split<2><<<(unsigned)((2 * c->Vh + bs - 1) / bs), bs, 0, s>>>(
                    g, L, (const double2 *)in, (double2 *)out, P);
            else if (kind == 2)
                k_deo_df_ieee_split<4><<<(unsigned)((4 * c->Vh + bs - 1) / bs), bs, 0, s>>>(
                    g, L, (const double2 *)in, (double2 *)out, P);
            else
                k_deo_df_ieee_split<8><<<(unsigned)((8 * c->Vh + bs - 1) / bs), bs, 0, s>>>(
                    g, L, (const double2 *)in, (double2 *)out, P);
        }, staged ? 10 : 9, cand);
        break;
    }
    case LQCD_PREC_FP64_NATIVE:
        if (recon != 18) return fail(LQCD_EINVAL, "native FP64 D_eo uses 18-real links");
        st = tuned_launch(c, 1, s, [&](int bs) {
            k_deo_nat<<<nb(bs), bs, 0, s>>>(g, c->lnk_nat.as<double2>(), (const double2 *)in, (double2 *)out, P);
        });
        break;
    case LQCD_PREC_FP32:
    case LQCD_PREC_FP16: {
        // kind 0: the direction loop rolled; kind 5: unrolled (loads of
        // later hops issued early)
        static const int cand_f[6] = {64, 128, 256, 5120 + 64, 5120 + 128, 5120 + 256};
        if (prec == LQCD_PREC_FP16 && recon != 12) return fail(LQCD_EINVAL, "FP16 links use 12-real storage");
        if (recon != 18 && recon != 12) return fail(LQCD_EINVAL, "recon must be 18 or 12");
        const int lf = prec == LQCD_PREC_FP16 ? LF_F16_12 : (recon == 18 ? LF_F32_18 : LF_F32_12);
        const void *Lp = lf == LF_F16_12 ? c->lnk_h12.ptr : (lf == LF_F32_18 ? c->lnk_f18.ptr : c->lnk_f12.ptr);
        const int variant = lf == LF_F16_12 ? 4 : (lf == LF_F32_18 ? 2 : 3);
        st = tuned_launch(c, variant, s, [&](int code) {
            const bool unr = (code >> 10) == 5;
            const int bs = code & 1023;
            const float2 *xi = (const float2 *)in;
            float2 *xo = (float2 *)out;
            if (lf == LF_F32_18)
                unr ? k_deo_f32<LF_F32_18, 4><<<nb(bs), bs, 0, s>>>(g, Lp, xi, xo, P)
                    : k_deo_f32<LF_F32_18, 1><<<nb(bs), bs, 0, s>>>(g, Lp, xi, xo, P);
            else if (lf == LF_F32_12)
                unr ? k_deo_f32<LF_F32_12, 4><<<nb(bs), bs, 0, s>>>(g, Lp, xi, xo, P)
                    : k_deo_f32<LF_F32_12, 1><<<nb(bs), bs, 0, s>>>(g, Lp, xi, xo, P);
            else
                unr ? k_deo_f32<LF_F16_12, 4><<<nb(bs), bs, 0, s>>>(g, Lp, xi, xo, P)
                    : k_deo_f32<LF_F16_12, 1><<<nb(bs), bs, 0, s>>>(g, Lp, xi, xo, P);
        }, 6, cand_f);
        break;
    }
    default:
        return fail(LQCD_EINVAL, "unknown precision");
    }
    if (st) return st;
    LQCD_CUDA(cudaGetLastError());
    return LQCD_OK;
}

}  // namespace lqcd

extern "C" int lqcd_deo_tuned_config(const lqcd_ctx *c, int prec, int recon, int *code)
{
    if (!c || !code) return lqcd::fail(LQCD_EINVAL, "NULL argument");
    const int v = lqcd::deo_variant(prec, recon);
    if (v < 0) return lqcd::fail(LQCD_EINVAL, "no such D_eo variant");
    *code = lqcd::deo_tuned_block(c, v);
    return LQCD_OK;
}

extern "C" int lqcd_deo_apply_h16(lqcd_ctx *c, int out_parity, const void *in, const float *in_norm, void *out,
                                  float *out_norm, void *stream)
{
    using namespace lqcd;
    NvtxRange nvtx_("lqcd_deo_apply_h16");
    if (!c) return fail(LQCD_EINVAL, "NULL context");
    LQCD_ON_DEVICE(c->device);
    if (int lr = links_ready(c)) return lr;
    if (out_parity != 0 && out_parity != 1) return fail(LQCD_EINVAL, "out_parity must be 0 or 1");
    if (!in || !in_norm || !out || !out_norm) return fail(LQCD_EINVAL, "NULL spinor pointer");
    if (in == out || (const void *)in_norm == (const void *)out_norm) return fail(LQCD_EINVAL, "in and out must not overlap");
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    const unsigned nb = (unsigned)((c->Vh + 127) / 128);
    k_deo_h16<<<nb, 128, 0, s>>>(c->g, c->lnk_h12.ptr, (const __half2 *)in, in_norm, (__half2 *)out, out_norm,
                                 out_parity);
    LQCD_CUDA(cudaGetLastError());
    c->launches += 1;
    return LQCD_OK;
}
