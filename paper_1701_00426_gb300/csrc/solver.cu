// solver.cu -- host driver of the multi-shift CG (Sec. 2.2, Eqs. lineqeo,
// shlineq) and its helper kernels.
//
// FP64 solve (opts.prec = FP64): the Krylov iteration runs with df64
// vectors and df64 D_eo (48-bit significands, FP32 pipes).  Afterwards each
// shift's solution is converted to IEEE FP64, its true residual
// ||(A + sigma_i) x_i - b|| is recomputed from the IEEE solution, and a shift
// whose true residual exceeds tol is corrected by solving for the residual
// (defect correction) until it meets tol.
//
// Mixed solve (opts.prec = FP32 / FP16): the multi-shift iteration runs with
// FP32 vectors and FP32 (or FP16-stored) links; then every shift is finished
// by a single-shift CG with FP32 iterations and FP64 reliable updates: when
// the FP32 residual has fallen below delta times the residual of the last
// update, the FP32 solution is added to the FP64 one, the FP64 true residual
// replaces the FP32 residual and the search direction is kept.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "solver_kernels.cuh"
#include "solver_persist.cuh"

namespace lqcd {

// ------------------------------------------------------------------ helper kernels
__global__ void k_norm2_ieee(const double2 *__restrict__ v, int Vh, int nvec, double *part, unsigned *ticket,
                             int ntiles, double *out)
{
    __shared__ double s_red[kTile / 32];
    const int tile = blockIdx.x;
    const int i = tile * kTile + threadIdx.x;
    double a = 0.0;
    if (i < Vh)
        for (int c = 0; c < 3 * nvec; ++c) {
            const double2 d = v[(size_t)c * Vh + i];
            a = fma(d.x, d.x, fma(d.y, d.y, a));
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xFFFFFFFFu, a, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = a;
    __syncthreads();
    double v0 = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < kTile / 32; ++k) v0 += s_red[k];
    reduce_finish(part, ticket, ntiles, tile, v0, [&](double tot) { *out = tot; });
}

// dst (engine format) = scale * src (IEEE)
template <int VP>
__global__ void k_ieee_to_vec(const double2 *__restrict__ src, void *dst, long n, double scale)
{
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const double2 d = src[t];
    if constexpr (VP == VP_DF) {
        const float2 re = f64_to_df_slow(d.x * scale), im = f64_to_df_slow(d.y * scale);
        ((float4 *)dst)[t] = make_float4(re.x, re.y, im.x, im.y);
    } else {
        ((float2 *)dst)[t] = make_float2((float)(d.x * scale), (float)(d.y * scale));
    }
}

// dst (IEEE) (+)= scale * src (engine format)
template <int VP>
__global__ void k_vec_to_ieee(const void *src, double2 *dst, long n, double scale, int accumulate)
{
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= n) return;
    double re, im;
    if constexpr (VP == VP_DF) {
        const float4 v = ((const float4 *)src)[t];
        re = df_to_f64(make_float2(v.x, v.y));
        im = df_to_f64(make_float2(v.z, v.w));
    } else {
        const float2 v = ((const float2 *)src)[t];
        re = (double)v.x;
        im = (double)v.y;
    }
    re *= scale;
    im *= scale;
    if (accumulate) {
        const double2 o = dst[t];
        re += o.x;
        im += o.y;
    }
    dst[t] = make_double2(re, im);
}

// r = ps[s] = src for every shift, x[s] = 0 (engine format; one field = n3 complex)
template <int VP>
__global__ void k_init_vectors(const void *src, void *r, void *x, void *ps, long n3, int n_shift)
{
    using T = typename VecT<VP>::T;
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= n3) return;
    const T v = ((const T *)src)[t];
    if (r != src) ((T *)r)[t] = v;
    T z;
    memset(&z, 0, sizeof(T));
    for (int s = 0; s < n_shift; ++s) {
        ((T *)ps)[(long)s * n3 + t] = v;
        ((T *)x)[(long)s * n3 + t] = z;
    }
}

// dst (FP32) = scale * src (double-float), rounded to nearest
__global__ void k_df_to_f32(const float4 *__restrict__ src, float2 *__restrict__ dst, long n, double scale)
{
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float4 v = src[t];
    dst[t] = make_float2((float)(df_to_f64(make_float2(v.x, v.y)) * scale),
                         (float)(df_to_f64(make_float2(v.z, v.w)) * scale));
}

template <int VP>
__global__ void k_scale_vec(void *v, long n3, float f)
{
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= n3) return;
    if constexpr (VP == VP_DF) {
        float4 a = ((float4 *)v)[t];
        ((float4 *)v)[t] = make_float4(a.x * f, a.y * f, a.z * f, a.w * f);
    } else {
        float2 a = ((float2 *)v)[t];
        ((float2 *)v)[t] = make_float2(a.x * f, a.y * f);
    }
}

template <int VP>
__global__ void k_zero_vec(void *v, long n3)
{
    using T = typename VecT<VP>::T;
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= n3) return;
    T z;
    memset(&z, 0, sizeof(T));
    ((T *)v)[t] = z;
}

// True residual in native IEEE FP64 (FP64 FMA on the FP64 pipe): it runs a
// few times per solve, and it must not share the df64 rounding of the
// iteration it checks.
// Part 1: t = D_oe x.
__global__ void __launch_bounds__(kTile)
    k_res_nat1(Geom g, const double2 *__restrict__ L, const double2 *__restrict__ x, double2 *__restrict__ t)
{
    const int i = blockIdx.x * kTile + threadIdx.x;
    if (i >= g.Vh) return;
    Stencil S;
    make_stencil(g, i, 1, S);
    double2 o[3];
    deo_site_nat(g, L, x, S, i, 1, g.Vh, o);
#pragma unroll
    for (int c = 0; c < 3; ++c) t[(size_t)c * g.Vh + i] = o[c];
}

// Part 2: r = b - ((m^2 + sigma) x - D_eo t).  Writes r_hi (IEEE, optional),
// r_lo = lo_scale * r in the engine format (optional) and ||r||^2 to *out.
template <int VP>
__global__ void __launch_bounds__(kTile)
    k_res_nat2(Geom g, const double2 *__restrict__ L, const double2 *__restrict__ t, const double2 *__restrict__ x,
               const double2 *__restrict__ b, double a, double2 *r_hi, void *r_lo, double lo_scale, double *part,
               unsigned *ticket, double *out)
{
    __shared__ double s_red[kTile / 32];
    const int tile = blockIdx.x;
    const int i = tile * kTile + threadIdx.x;
    double nrm = 0.0;
    if (i < g.Vh) {
        Stencil S;
        make_stencil(g, i, 0, S);
        double2 o[3];
        deo_site_nat(g, L, t, S, i, 0, g.Vh, o);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double2 xv = x[(size_t)c * g.Vh + i], bv = b[(size_t)c * g.Vh + i];
            const double2 r = make_double2(bv.x - fma(a, xv.x, -o[c].x), bv.y - fma(a, xv.y, -o[c].y));
            nrm = fma(r.x, r.x, fma(r.y, r.y, nrm));
            if (r_hi) r_hi[(size_t)c * g.Vh + i] = r;
            if (r_lo) {
                if constexpr (VP == VP_DF) {
                    const float2 a0 = f64_to_df_slow(r.x * lo_scale), a1 = f64_to_df_slow(r.y * lo_scale);
                    ((float4 *)r_lo)[(size_t)c * g.Vh + i] = make_float4(a0.x, a0.y, a1.x, a1.y);
                } else {
                    ((float2 *)r_lo)[(size_t)c * g.Vh + i] = make_float2((float)(r.x * lo_scale), (float)(r.y * lo_scale));
                }
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nrm += __shfl_down_sync(0xFFFFFFFFu, nrm, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = nrm;
    __syncthreads();
    double v = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < kTile / 32; ++k) v += s_red[k];
    const int ntiles = (g.Vh + kTile - 1) / kTile;
    reduce_finish(part, ticket, ntiles, tile, v, [&](double tot) { *out = tot; });
}

// Residual of the reliable updates in double-float (about 2^-47 relative to
// the terms; 2.5x cheaper than native FP64): r = b - ((m^2+sigma) x - D_eo t)
// with t = D_oe x from the stand-alone double-float kernel.  The acceptance
// test of a solve always uses the native FP64 residual above.
__global__ void __launch_bounds__(kTile, 2)
    k_res_df2(Geom g, const float4 *__restrict__ L, const double2 *__restrict__ t, const double2 *__restrict__ x,
              const double2 *__restrict__ b, double a, double2 *r_hi, double *part, unsigned *ticket, double *out)
{
    __shared__ double s_red[kTile / 32];
    const int tile = blockIdx.x;
    const int i = tile * kTile + threadIdx.x;
    Acc2 nrm;
    acc_zero(nrm);
    bool bad = false;
    if (i < g.Vh) {
        Stencil S;
        make_stencil(g, i, 0, S);
        float2 res[6];
        deo_site_df<SF_IEEE>(g, L, t, S, i, 0, g.Vh, res, bad);
        const float2 adf = f64_to_df_slow(a);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double2 xv = x[(size_t)c * g.Vh + i], bv = b[(size_t)c * g.Vh + i];
            const float2 xr = split_f64(xv.x, bad), xi = split_f64(xv.y, bad);
            const float2 br = split_f64(bv.x, bad), bi = split_f64(bv.y, bad);
            const float2 o0 = df_add(df_fma(df_neg(adf), xr, br), res[2 * c]);
            const float2 o1 = df_add(df_fma(df_neg(adf), xi, bi), res[2 * c + 1]);
            acc_prod(nrm, o0.x, o0.y, o0.x, o0.y);
            acc_prod(nrm, o1.x, o1.y, o1.x, o1.y);
            if (r_hi) r_hi[(size_t)c * g.Vh + i] = make_double2(df_to_f64(o0), df_to_f64(o1));
        }
    }
    // a site outside the double-float window poisons the sum: the caller
    // then falls back to the native residual
    if (bad) nrm.s = __int_as_float(0x7fc00000);
    const double v = block_reduce_acc<kTile>(nrm, s_red);
    const int ntiles = (g.Vh + kTile - 1) / kTile;
    reduce_finish(part, ticket, ntiles, tile, v, [&](double tot) { *out = tot; });
}

// Host wrappers used by the batched solver (mrhs.cu).
void k_res_nat1_ext(const Geom &g, const double2 *L, const double2 *x, double2 *t, int ntiles, cudaStream_t s)
{
    k_res_nat1<<<ntiles, kTile, 0, s>>>(g, L, x, t);
}

void k_res_nat2_ext(const Geom &g, const double2 *L, const double2 *t, const double2 *x, const double2 *b, double a,
                    double2 *r_hi, double *part, unsigned *ticket, double *out, int ntiles, cudaStream_t s)
{
    k_res_nat2<VP_F32><<<ntiles, kTile, 0, s>>>(g, L, t, x, b, a, r_hi, nullptr, 1.0, part, ticket, out);
}

// ------------------------------------------------------------------ workspace


int ensure_workspace_in(lqcd_ctx *c, Workspace &W, int vp, int n_shift, WsPtrs &P)
{
    const size_t Vh = c->Vh, n3 = 3 * Vh;
    const size_t E = vp == VP_DF ? sizeof(float4) : sizeof(float2);
    const size_t vec_bytes = (3 + 2 * (size_t)n_shift) * n3 * E;
    const size_t ieee_bytes = 2 * n3 * sizeof(double2);
    const int ntiles = (int)((Vh + kSites - 1) / kSites);
    const int ntiles256 = (int)((Vh + kTile - 1) / kTile);
    int st;
    if (vec_bytes > W.vec.bytes || ieee_bytes > W.ieee.bytes) W.gen++;
    if ((st = W.vec.ensure(std::max(vec_bytes, W.vec.bytes)))) return st;
    if ((st = W.ieee.ensure(std::max(ieee_bytes, W.ieee.bytes)))) return st;
    if ((st = W.part.ensure((size_t)ntiles * sizeof(double) + 64 * sizeof(double)))) return st;
    if (!W.tickets.ptr) {
        if ((st = W.tickets.ensure(64))) return st;
        LQCD_CUDA(cudaMemset(W.tickets.ptr, 0, 64));
        W.gen++;
    }
    if (!W.state.ptr) {
        if ((st = W.state.ensure(sizeof(SolverState)))) return st;
        W.gen++;
    }
    char *v = (char *)W.vec.ptr;
    P.r = v;
    P.q = v + n3 * E;
    P.t = v + 2 * n3 * E;
    P.x = v + 3 * n3 * E;
    P.ps = v + (3 + (size_t)n_shift) * n3 * E;
    P.r_hi = (double2 *)W.ieee.ptr;
    P.t_nat = (double2 *)W.ieee.ptr + n3;
    P.part = (double *)W.part.ptr;
    P.scal = P.part + ntiles;
    P.ticket = (unsigned *)W.tickets.ptr;
    P.st = (SolverState *)W.state.ptr;
    P.ntiles = ntiles;
    P.ntiles256 = ntiles256;
    W.prec = vp;
    W.n_shift = n_shift;
    return LQCD_OK;
}

static int ensure_workspace(lqcd_ctx *c, int vp, int n_shift, WsPtrs &P)
{
    return ensure_workspace_in(c, c->ws, vp, n_shift, P);
}

static inline unsigned nblk(long n, int bs = 256) { return (unsigned)((n + bs - 1) / bs); }

static int norm2_ieee(lqcd_ctx *c, const WsPtrs &P, const double2 *v, int nvec, cudaStream_t s, double &out)
{
    k_norm2_ieee<<<P.ntiles256, kTile, 0, s>>>(v, (int)c->Vh, nvec, P.part, P.ticket + 1, P.ntiles256, P.scal);
    LQCD_CUDA(cudaGetLastError());
    c->launches += 1;
    LQCD_CUDA(cudaMemcpyAsync(c->h_pinned_d, P.scal, sizeof(double), cudaMemcpyDeviceToHost, s));
    LQCD_CUDA(cudaStreamSynchronize(s));
    out = c->h_pinned_d[0];
    return LQCD_OK;
}

// r = b - (A + sigma) x with IEEE x, b; optional r_hi / r_lo; returns ||r||^2.
static int true_residual(lqcd_ctx *c, const WsPtrs &P, int vp, double a, const double2 *x, const double2 *b,
                         double2 *r_hi, void *r_lo, double lo_scale, cudaStream_t s, double &rr)
{
    const double2 *L = c->lnk_nat.as<double2>();
    k_res_nat1<<<P.ntiles256, kTile, 0, s>>>(c->g, L, x, P.t_nat);
    LQCD_CUDA(cudaGetLastError());
    c->launches += 2;
    if (vp == VP_DF)
        k_res_nat2<VP_DF><<<P.ntiles256, kTile, 0, s>>>(c->g, L, P.t_nat, x, b, a, r_hi, r_lo, lo_scale, P.part,
                                                      P.ticket + 1, P.scal);
    else
        k_res_nat2<VP_F32><<<P.ntiles256, kTile, 0, s>>>(c->g, L, P.t_nat, x, b, a, r_hi, r_lo, lo_scale, P.part,
                                                       P.ticket + 1, P.scal);
    LQCD_CUDA(cudaGetLastError());
    LQCD_CUDA(cudaMemcpyAsync(c->h_pinned_d, P.scal, sizeof(double), cudaMemcpyDeviceToHost, s));
    LQCD_CUDA(cudaStreamSynchronize(s));
    rr = c->h_pinned_d[0];
    return LQCD_OK;
}

// Reliable-update residual: double-float, with the native FP64 residual as
// fallback when an input leaves the double-float exponent window.
static int refresh_residual(lqcd_ctx *c, const WsPtrs &P, int vp, double a, const double2 *x, const double2 *b,
                            double2 *r_hi, cudaStream_t s, double &rr)
{
    const float4 *L = c->lnk_df.as<float4>();
    k_deo_df_ieee<<<P.ntiles256, kTile, 0, s>>>(c->g, L, x, P.t_nat, 1);
    k_res_df2<<<P.ntiles256, kTile, 0, s>>>(c->g, L, P.t_nat, x, b, a, r_hi, P.part, P.ticket + 1, P.scal);
    LQCD_CUDA(cudaGetLastError());
    c->launches += 2;
    LQCD_CUDA(cudaMemcpyAsync(c->h_pinned_d, P.scal, sizeof(double), cudaMemcpyDeviceToHost, s));
    LQCD_CUDA(cudaStreamSynchronize(s));
    rr = c->h_pinned_d[0];
    if (std::isfinite(rr)) return LQCD_OK;
    return true_residual(c, P, vp, a, x, b, r_hi, nullptr, 1.0, s, rr);
}

// power of two bringing a field of squared norm n2 over n reals to O(1) entries
double unit_scale_pub(double n2, double n);
static double unit_scale(double n2, double n) { return unit_scale_pub(n2, n); }
double unit_scale_pub(double n2, double n)
{
    if (!(n2 > 0.0) || !std::isfinite(n2)) return 1.0;
    const double rms = std::sqrt(n2 / n);
    return std::ldexp(1.0, -(int)std::lround(std::log2(rms)));
}

// ------------------------------------------------------------------ staged kernels
// Shared-memory attribute and resident blocks of the staged K1 / K2, once per
// device (called outside stream capture: at link upload).  0 blocks = the
// staged path is unavailable and the per-thread kernels run.
static std::mutex g_st_mu;
static int g_st_blocks[64];
static bool g_st_done[64];

template <class K>
static int staged_kernel_blocks(K kern, int nsm)
{
    int occ = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStagedIterSmem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kStagedThreads, kStagedIterSmem) != cudaSuccess)
        occ = 0;
    cudaGetLastError();
    return occ * nsm;
}

bool staged_solver_ready()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
    std::lock_guard<std::mutex> lk(g_st_mu);
    if (!g_st_done[dev]) {
        g_st_done[dev] = true;
        int nsm = 0;
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) nsm = 0;
        int b = staged_kernel_blocks(k_it_deo1_st<1>, nsm);
        b = std::min(b, staged_kernel_blocks(k_it_deo2_st<1>, nsm));
        b = std::min(b, staged_kernel_blocks(k_it_deo1_st<kMaxJobs>, nsm));
        b = std::min(b, staged_kernel_blocks(k_it_deo2_st<kMaxJobs>, nsm));
        g_st_blocks[dev] = b;
    }
    return g_st_blocks[dev] > 0;
}

static int staged_solver_blocks()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    std::lock_guard<std::mutex> lk(g_st_mu);
    return g_st_blocks[dev];
}

// Grid of the persistent reduction kernels (FP32 / FP16 K2, K3 of every
// precision): the resident blocks of the FP32 K2 (all link formats and batch
// sizes), once per device; 0 = the one-block-per-tile k_it_deo2 /
// k_it_upd_r run.
static int g_f32p_blocks[64];
static bool g_f32p_done[64];

template <class K>
static int kernel_resident_blocks(K kern, int nsm)
{
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kIterThreads, 0) != cudaSuccess) occ = 0;
    cudaGetLastError();
    return occ * nsm;
}

int persist_blocks()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    std::lock_guard<std::mutex> lk(g_st_mu);
    if (!g_f32p_done[dev]) {
        g_f32p_done[dev] = true;
        const char *env = getenv("LQCD_PERSIST_REDUCTIONS");
        if (env && env[0] == '0' && env[1] == '\0') {
            g_f32p_blocks[dev] = 0;  // one block per tile (k_it_deo2, k_it_upd_r)
            return 0;
        }
        int nsm = 0;
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) nsm = 0;
        int b = kernel_resident_blocks(k_it_deo2_f32p<1, LF_F32_18>, nsm);
        b = std::min(b, kernel_resident_blocks(k_it_deo2_f32p<1, LF_F32_12>, nsm));
        b = std::min(b, kernel_resident_blocks(k_it_deo2_f32p<1, LF_F16_12>, nsm));
        b = std::min(b, kernel_resident_blocks(k_it_deo2_f32p<kMaxJobs, LF_F32_18>, nsm));
        b = std::min(b, kernel_resident_blocks(k_it_deo2_f32p<kMaxJobs, LF_F32_12>, nsm));
        b = std::min(b, kernel_resident_blocks(k_it_deo2_f32p<kMaxJobs, LF_F16_12>, nsm));
        g_f32p_blocks[dev] = b;
    }
    return g_f32p_blocks[dev];
}

// All jobs of the batch carry the staged link stream.
template <int NJ>
static bool batch_staged(const IterBatch<NJ> &B)
{
    if (kSites != kTile) return false;  // the staged stream is laid out in 256-site tiles
    for (int j = 0; j < B.njobs; ++j)
        if (!B.job[j].links_st) return false;
    return B.njobs > 0;
}

// ------------------------------------------------------------------ iteration chunks
// Launch with programmatic stream serialisation when dep is set: the kernel
// may start while the previous kernel of the stream drains (its prologue
// overlaps that kernel's tail; see dep_wait in solver_kernels.cuh).  Only
// for a kernel whose predecessor in the stream is the previous kernel of the
// same iteration sequence.
template <class... P, class... A>
static void launch_dep(void (*kern)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool dep, A... args)
{
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = dep ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kern, args...);
}

// Kernel k (0: K1 .. 3: K4) of one iteration; dep: launch it dependent on
// the kernel before it (K1: on the previous iteration's K4).
template <int NJ>
static void launch_kernel_k(const IterBatch<NJ> &B, int k, int ntot, int vp, int lf, cudaStream_t s, bool dep)
{
    const dim3 g1((unsigned)ntot), tb(kIterThreads);
    if (vp == VP_DF) {
        const int sb = (k < 2 && batch_staged(B)) ? std::min(ntot, staged_solver_blocks()) : 0;
        const dim3 gs((unsigned)sb), ts(kStagedThreads);
        if (k == 0 && sb > 0) launch_dep(k_it_deo1_st<NJ>, gs, ts, kStagedIterSmem, s, dep, B, ntot);
        if (k == 1 && sb > 0) launch_dep(k_it_deo2_st<NJ>, gs, ts, kStagedIterSmem, s, dep, B, ntot);
        if (k == 0 && sb == 0) launch_dep(k_it_deo1<NJ, VP_DF, LF_DF18>, g1, tb, 0, s, dep, B);
        if (k == 1 && sb == 0) launch_dep(k_it_deo2<NJ, VP_DF, LF_DF18>, g1, tb, 0, s, dep, B);
        if (k == 2) {
            const int pb = std::min(ntot, persist_blocks());
            if (pb > 0) launch_dep(k_it_upd_r_p<NJ, VP_DF>, dim3((unsigned)pb), tb, 0, s, dep, B, ntot);
            else launch_dep(k_it_upd_r<NJ, VP_DF>, g1, tb, 0, s, dep, B);
        }
        if (k == 3) launch_dep(k_it_upd_shifts<NJ, VP_DF>, g1, tb, 0, s, dep, B);
        return;
    }
    if (k == 0) {
        if (lf == LF_F32_18) launch_dep(k_it_deo1<NJ, VP_F32, LF_F32_18>, g1, tb, 0, s, dep, B);
        else if (lf == LF_F32_12) launch_dep(k_it_deo1<NJ, VP_F32, LF_F32_12>, g1, tb, 0, s, dep, B);
        else launch_dep(k_it_deo1<NJ, VP_F32, LF_F16_12>, g1, tb, 0, s, dep, B);
    }
    if (k == 1) {
        const int pb = std::min(ntot, persist_blocks());
        const dim3 gp((unsigned)pb);
        if (pb > 0) {
            if (lf == LF_F32_18) launch_dep(k_it_deo2_f32p<NJ, LF_F32_18>, gp, tb, 0, s, dep, B, ntot);
            else if (lf == LF_F32_12) launch_dep(k_it_deo2_f32p<NJ, LF_F32_12>, gp, tb, 0, s, dep, B, ntot);
            else launch_dep(k_it_deo2_f32p<NJ, LF_F16_12>, gp, tb, 0, s, dep, B, ntot);
        } else if (lf == LF_F32_18) {
            launch_dep(k_it_deo2<NJ, VP_F32, LF_F32_18>, g1, tb, 0, s, dep, B);
        } else if (lf == LF_F32_12) {
            launch_dep(k_it_deo2<NJ, VP_F32, LF_F32_12>, g1, tb, 0, s, dep, B);
        } else {
            launch_dep(k_it_deo2<NJ, VP_F32, LF_F16_12>, g1, tb, 0, s, dep, B);
        }
    }
    if (k == 2) {
        const int pb = std::min(ntot, persist_blocks());
        if (pb > 0) launch_dep(k_it_upd_r_p<NJ, VP_F32>, dim3((unsigned)pb), tb, 0, s, dep, B, ntot);
        else launch_dep(k_it_upd_r<NJ, VP_F32>, g1, tb, 0, s, dep, B);
    }
    if (k == 3) launch_dep(k_it_upd_shifts<NJ, VP_F32>, g1, tb, 0, s, dep, B);
}

// One iteration.  K2..K4 always follow their predecessor kernel; K1 does
// only when `chained` (the previous iteration's K4 is the last launch).
template <int NJ>
static void launch_iteration(const IterBatch<NJ> &B, int ntot, int vp, int lf, cudaStream_t s, bool pdl, bool chained)
{
    for (int k = 0; k < 4; ++k) launch_kernel_k<NJ>(B, k, ntot, vp, lf, s, pdl && (k > 0 || chained));
}

void GraphCache::reset()
{
    for (int k = 0; k < kEntries; ++k) {
        if (exec[k]) cudaGraphExecDestroy(exec[k]);
        exec[k] = nullptr;
        key[k] = ~0ull;
        used[k] = 0;
    }
}

cudaGraphExec_t GraphCache::find(uint64_t k)
{
    for (int e = 0; e < kEntries; ++e)
        if (exec[e] && key[e] == k) {
            used[e] = ++tick;
            return exec[e];
        }
    return nullptr;
}

void GraphCache::put(uint64_t k, cudaGraphExec_t g)
{
    int v = 0;
    for (int e = 1; e < kEntries; ++e)
        if (used[e] < used[v]) v = e;
    if (exec[v]) cudaGraphExecDestroy(exec[v]);
    exec[v] = g;
    key[v] = k;
    used[v] = ++tick;
}

static uint64_t fnv1a(const void *p, size_t n, uint64_t h = 1469598103934665603ull)
{
    const unsigned char *b = (const unsigned char *)p;
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

// Run iteration chunks (graph of `chunk` iterations) until every job halts.
// Pipelined: chunk k+1 is queued before chunk k's halt words are read.
// The cached graph of `chunk` iterations of batch B (captured on first use).
template <int NJ>
static int chunk_graph(lqcd_ctx *c, const IterBatch<NJ> &B, int vp, int lf, int chunk, cudaStream_t s,
                       cudaGraphExec_t &out)
{
    // blocks of the launch: interleaved jobs share one tile count
    const int ntot = B.interleave ? B.job[0].ntiles * B.njobs : B.tile_start[B.njobs];
    if (ntot <= 0) return fail(LQCD_EINVAL, "empty iteration batch");
    uint64_t key = fnv1a(&B, sizeof(B));
    key = fnv1a(&vp, sizeof vp, key);
    key = fnv1a(&lf, sizeof lf, key);
    key = fnv1a(&chunk, sizeof chunk, key);
    const int pdl = c->opts.pdl;
    key = fnv1a(&pdl, sizeof pdl, key);
    key ^= (uint64_t)NJ * 0x9E3779B97F4A7C15ull;
    out = c->graph.find(key);
    if (out) return LQCD_OK;
    cudaGraph_t g;
    LQCD_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < chunk; ++k) launch_iteration<NJ>(B, ntot, vp, lf, s, pdl != 0, k > 0);
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (e != cudaSuccess) return cuda_fail(e, "graph capture");
    e = cudaGraphInstantiate(&out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    c->graph.put(key, out);
    return LQCD_OK;
}

template <int NJ>
static int run_until_halt(lqcd_ctx *c, const IterBatch<NJ> &B, int vp, int lf, int chunk, int max_iter,
                          cudaStream_t s, std::vector<int> &halts)
{
    cudaGraphExec_t exec = nullptr;
    if (int st = chunk_graph<NJ>(c, B, vp, lf, chunk, s, exec)) return st;
    const int nj = B.njobs;
    // pinned status words: [2][nj] halts
    int *hs = c->h_pinned;
    const int max_chunks = max_iter / chunk + 4;
    int slot = 0;
    cudaEvent_t ev[2];
    LQCD_CUDA(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
    LQCD_CUDA(cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
    auto enqueue = [&](int sl) -> cudaError_t {
        cudaError_t e = cudaGraphLaunch(exec, s);
        c->launches += 4 * (uint64_t)chunk;
        for (int j = 0; j < nj && e == cudaSuccess; ++j)
            e = cudaMemcpyAsync(hs + sl * kMaxJobs + j, &B.job[j].st->halt, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaEventRecord(ev[sl], s);
        return e;
    };
    cudaError_t e = enqueue(0);
    int rc = LQCD_OK;
    for (int k = 0; k < max_chunks && e == cudaSuccess; ++k) {
        const int nxt = slot ^ 1;
        e = enqueue(nxt);
        if (e != cudaSuccess) break;
        e = cudaEventSynchronize(ev[slot]);
        if (e != cudaSuccess) break;
        bool all = true;
        for (int j = 0; j < nj; ++j) all &= hs[slot * kMaxJobs + j] != HALT_NONE;
        if (all) break;
        slot = nxt;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (e != cudaSuccess) return cuda_fail(e, "iteration chunks");
    halts.assign(nj, 0);
    for (int j = 0; j < nj; ++j) {
        LQCD_CUDA(cudaMemcpy(&halts[j], &B.job[j].st->halt, sizeof(int), cudaMemcpyDeviceToHost));
    }
    return rc;
}

static int link_fmt_for(const lqcd_ctx *c, int prec, const void **links)
{
    if (prec == LQCD_PREC_FP64) {
        *links = c->lnk_df.ptr;
        return LF_DF18;
    }
    if (prec == LQCD_PREC_FP16) {
        *links = c->lnk_h12.ptr;
        return LF_F16_12;
    }
    if (c->opts.recon == 12) {
        *links = c->lnk_f12.ptr;
        return LF_F32_12;
    }
    *links = c->lnk_f18.ptr;
    return LF_F32_18;
}

static void fill_job(lqcd_ctx *c, const WsPtrs &P, const void *links, IterJob &J)
{
    J.g = c->g;
    J.links = links;
    // the staged stream holds the df64 links: only the FP64 engine uses it
    J.links_st = (links == c->lnk_df.ptr && staged_active(c)) ? c->lnk_dfs.as<float4>() : nullptr;
    J.r = P.r;
    J.q = P.q;
    J.t = P.t;
    J.x = P.x;
    J.ps = P.ps;
    J.st = P.st;
    J.part = P.part;
    J.ticket = P.ticket;
    J.tile0 = 0;
    J.ntiles = P.ntiles;
}

// Host-side initial state of a solve of (A + shifts) with source norm^2 b2.
void init_state_pub(SolverState &S, double mass, const double *shifts, int n_shift, double tol_iter, double b2,
                    int max_iter);
static void init_state(SolverState &S, double mass, const double *shifts, int n_shift, double tol_iter, double b2,
                       int max_iter)
{
    init_state_pub(S, mass, shifts, n_shift, tol_iter, b2, max_iter);
}
void init_state_pub(SolverState &S, double mass, const double *shifts, int n_shift, double tol_iter, double b2,
                       int max_iter)
{
    memset(&S, 0, sizeof S);
    int base = 0;
    for (int i = 1; i < n_shift; ++i)
        if (shifts[i] < shifts[base]) base = i;
    S.n_shift = n_shift;
    S.base = base;
    S.max_iter = max_iter;
    S.a0 = mass * mass + shifts[base];
    const float a0h = (float)S.a0;
    S.a0_df = make_float2(a0h, (float)(S.a0 - (double)a0h));
    S.tol2_b2 = tol_iter * tol_iter * b2;
    S.rho = b2;
    S.alpha = 1.0;
    S.beta = 0.0;
    for (int i = 0; i < n_shift; ++i) {
        S.shift_rel[i] = shifts[i] - shifts[base];
        S.zeta[i] = S.zeta_prev[i] = S.zeta_new[i] = 1.0;
        S.active_next[i] = 1;
    }
}

// Algorithmic device bytes of one iteration (per even site) given the
// engine, without the per-shift part.
static double iter_bytes_base(int vp, int lf)
{
    const double spin = vp == VP_DF ? 48.0 : 24.0;
    double link = 144.0;
    if (lf == LF_F32_18) link = 72.0;
    if (lf == LF_F32_12) link = 48.0;
    if (lf == LF_F16_12) link = 24.0;
    const double deo = 8 * link + 2 * spin;
    // K1, K2 (+ p read), K3 (r, q read, r write), K4 (r read)
    return 2 * deo + spin + 3 * spin + spin;
}

// ------------------------------------------------------------------ one engine run
// Solve (A + shifts) y = src (engine-format source already in P.r) from
// y = 0 to the iterated tolerance tol_iter; solutions stay in P.x.
static int engine_mscg(lqcd_ctx *c, const WsPtrs &P, int vp, int lf, const void *links, double mass,
                       const double *shifts, int n_shift, double tol_iter, double b2, cudaStream_t s,
                       SolverState &out_state, double &bytes)
{
    SolverState S;
    init_state(S, mass, shifts, n_shift, tol_iter, b2, c->opts.max_iter);
    LQCD_CUDA(cudaMemcpyAsync(P.st, &S, sizeof S, cudaMemcpyHostToDevice, s));
    const long n3 = 3 * (long)c->Vh;
    if (vp == VP_DF)
        k_init_vectors<VP_DF><<<nblk(n3), 256, 0, s>>>(P.r, P.r, P.x, P.ps, n3, n_shift);
    else
        k_init_vectors<VP_F32><<<nblk(n3), 256, 0, s>>>(P.r, P.r, P.x, P.ps, n3, n_shift);
    LQCD_CUDA(cudaGetLastError());
    c->launches += 1;
    IterBatch<1> B;
    memset(&B, 0, sizeof B);
    B.njobs = 1;
    B.max_shift = n_shift;
    B.tile_start[0] = 0;
    B.tile_start[1] = P.ntiles;
    fill_job(c, P, links, B.job[0]);
    std::vector<int> halts;
    int st = run_until_halt<1>(c, B, vp, lf, c->opts.check_every, c->opts.max_iter, s, halts);
    if (st) return st;
    LQCD_CUDA(cudaMemcpy(&out_state, P.st, sizeof out_state, cudaMemcpyDeviceToHost));
    double shift_it = 0;
    for (int i = 0; i < n_shift; ++i) shift_it += out_state.shift_iters[i] ? out_state.shift_iters[i] : out_state.iters;
    const double spin = vp == VP_DF ? 48.0 : 24.0;
    bytes += (double)c->Vh * (out_state.iters * iter_bytes_base(vp, lf) + shift_it * 4 * spin);
    return LQCD_OK;
}

// Finish one shift to the FP64 true-residual tolerance.
// FP64 engine: defect correction; mixed engine: CG with reliable updates.
static int refine_shift(lqcd_ctx *c, const WsPtrs &P, int vp, int lf, const void *links, double mass, double sigma,
                        const double2 *b, double b2, double2 *x_hi, double tol, bool allow_iter, cudaStream_t s,
                        double &resid_out, int &iters, int &reliable, double &bytes)
{
    const double a = mass * mass + sigma;
    const long n3 = 3 * (long)c->Vh;
    const double target2 = tol * tol * b2;
    double rr;
    int st = true_residual(c, P, vp, a, x_hi, b, P.r_hi, nullptr, 1.0, s, rr);
    if (st) return st;
    const double delta = c->opts.delta_reliable;
    bool hit_max = false;
    for (int round = 0; allow_iter && !hit_max && round < 40 && rr > target2; ++round) {
        // new low-precision residual, scaled to O(1) entries
        double scale = unit_scale(rr, 6.0 * c->Vh);
        if (vp == VP_DF)
            k_ieee_to_vec<VP_DF><<<nblk(n3), 256, 0, s>>>(P.r_hi, P.r, n3, scale);
        else
            k_ieee_to_vec<VP_F32><<<nblk(n3), 256, 0, s>>>(P.r_hi, P.r, n3, scale);
        LQCD_CUDA(cudaGetLastError());
        c->launches += 1;
        SolverState S;
        const double rho = rr * scale * scale;
        // iterate a little below the target so that rounding drift stays inside tol
        const double tol_rel = std::min(0.5, 0.5 * std::sqrt(target2 / rr));
        init_state(S, mass, &sigma, 1, tol_rel, rho, c->opts.max_iter);
        if (vp == VP_F32) S.rel_stop2 = delta * delta * rho;
        LQCD_CUDA(cudaMemcpyAsync(P.st, &S, sizeof S, cudaMemcpyHostToDevice, s));
        if (vp == VP_DF)
            k_init_vectors<VP_DF><<<nblk(n3), 256, 0, s>>>(P.r, P.r, P.x, P.ps, n3, 1);
        else
            k_init_vectors<VP_F32><<<nblk(n3), 256, 0, s>>>(P.r, P.r, P.x, P.ps, n3, 1);
        LQCD_CUDA(cudaGetLastError());
        c->launches += 1;
        IterBatch<1> B;
        memset(&B, 0, sizeof B);
        B.njobs = 1;
        B.max_shift = 1;
        B.tile_start[1] = P.ntiles;
        fill_job(c, P, links, B.job[0]);
        for (int inner = 0; inner < 100000; ++inner) {
            std::vector<int> halts;
            if ((st = run_until_halt<1>(c, B, vp, lf, c->opts.check_every, c->opts.max_iter, s, halts))) return st;
            SolverState O;
            LQCD_CUDA(cudaMemcpy(&O, P.st, sizeof O, cudaMemcpyDeviceToHost));
            const double spin = vp == VP_DF ? 48.0 : 24.0;
            bytes += (double)c->Vh * ((O.iters - S.iters) * (iter_bytes_base(vp, lf) + 4 * spin));
            iters += O.iters - S.iters;
            S = O;
            // x_hi += x_lo / scale
            if (vp == VP_DF)
                k_vec_to_ieee<VP_DF><<<nblk(n3), 256, 0, s>>>(P.x, x_hi, n3, 1.0 / scale, 1);
            else
                k_vec_to_ieee<VP_F32><<<nblk(n3), 256, 0, s>>>(P.x, x_hi, n3, 1.0 / scale, 1);
            LQCD_CUDA(cudaGetLastError());            LQCD_CUDA(cudaGetLastError());
            c->launches += 1;
            if (O.halt == HALT_NAN) return fail(LQCD_ENAN, "NaN/Inf or breakdown in refinement");
            if (O.halt == HALT_MAXITER) hit_max = true;
            if (O.halt != HALT_RELIABLE) break;
            // reliable update: FP64 true residual replaces the FP32 one
            ++reliable;
            const double old_scale = scale;
            if ((st = true_residual(c, P, vp, a, x_hi, b, P.r_hi, nullptr, 1.0, s, rr))) return st;
            if (rr <= target2) break;
            scale = unit_scale(rr, 6.0 * c->Vh);
            k_ieee_to_vec<VP_F32><<<nblk(n3), 256, 0, s>>>(P.r_hi, P.r, n3, scale);
            k_zero_vec<VP_F32><<<nblk(n3), 256, 0, s>>>(P.x, n3);
            k_scale_vec<VP_F32><<<nblk(n3), 256, 0, s>>>(P.ps, n3, (float)(scale / old_scale));
            LQCD_CUDA(cudaGetLastError());            LQCD_CUDA(cudaGetLastError());
            c->launches += 1;
            // continue the same CG: new rho, new reliable threshold, halt cleared
            SolverState U = O;
            U.rho = rr * scale * scale;
            U.rel_stop2 = delta * delta * U.rho;
            U.tol2_b2 = target2 * scale * scale * 0.25;
            U.halt = HALT_NONE;
            U.do_k4 = 0;
            LQCD_CUDA(cudaMemcpyAsync(P.st, &U, sizeof U, cudaMemcpyHostToDevice, s));
            S = U;
        }
        if ((st = true_residual(c, P, vp, a, x_hi, b, P.r_hi, nullptr, 1.0, s, rr))) return st;
    }
    resid_out = std::sqrt(rr / b2);
    return LQCD_OK;
}

// ------------------------------------------------------------------ jobs
int validate_solve(const lqcd_ctx *c, double mass, const double *shifts, int n_shift, double tol)
{
    if (!c->links_ok) return fail(LQCD_ESTATE, "no links uploaded");
    if (!shifts) return fail(LQCD_EINVAL, "NULL shifts");
    if (n_shift < 1 || n_shift > LQCD_MAX_SHIFTS) return fail(LQCD_EINVAL, "n_shift must be in 1..32");
    if (!(tol > 0.0) || !std::isfinite(mass)) return fail(LQCD_EINVAL, "tol must be > 0 and mass finite");
    double mn = shifts[0];
    for (int i = 0; i < n_shift; ++i) {
        if (!(shifts[i] >= 0.0) || !std::isfinite(shifts[i])) return fail(LQCD_EINVAL, "shifts must be finite and >= 0");
        mn = std::min(mn, shifts[i]);
    }
    if (!(mass * mass + mn > 0.0)) return fail(LQCD_EINVAL, "m^2 + min(shift) must be > 0 (A would be singular)");
    return LQCD_OK;
}

// Prepare one multi-shift solve: ||b||, power-of-two scaling, engine-format
// source, zero solutions, device scalars.  No iteration is launched.
int job_setup(JobRun &J, cudaStream_t s)
{
    lqcd_ctx *c = J.c;
    const long n3 = 3 * (long)c->Vh;
    memset(&J.I, 0, sizeof J.I);
    J.I.n_shift = J.n_shift;
    J.bytes = 0;
    J.launches0 = c->launches;
    int st;
    if ((st = norm2_ieee(c, J.P, J.b, 1, s, J.b2))) return st;
    if (!std::isfinite(J.b2)) return fail(LQCD_ENAN, "source contains NaN/Inf");
    J.zero = J.b2 == 0.0;
    SolverState S;
    if (J.zero) {
        memset(&S, 0, sizeof S);
        S.halt = HALT_CONVERGED;
        LQCD_CUDA(cudaMemcpyAsync(J.P.st, &S, sizeof S, cudaMemcpyHostToDevice, s));
        LQCD_CUDA(cudaMemsetAsync(J.x, 0, (size_t)J.n_shift * n3 * sizeof(double2), s));
        return LQCD_OK;
    }
    double rho0 = J.b2;
    const double2 *src = J.b;
    if (J.warm) {
        // start from the guess in x: iterate on its FP64 true residual
        const double a0 = J.mass * J.mass + J.shifts[0];
        if ((st = refresh_residual(c, J.P, J.vp, a0, J.x, J.b, J.P.r_hi, s, rho0))) return st;
        if (rho0 <= 0.25 * J.tol * J.tol * J.b2) {
            memset(&S, 0, sizeof S);
            S.halt = HALT_CONVERGED;
            S.n_shift = 1;
            LQCD_CUDA(cudaMemcpyAsync(J.P.st, &S, sizeof S, cudaMemcpyHostToDevice, s));
            J.scale = 1.0;
            if (J.vp == VP_F32)
                k_zero_vec<VP_F32><<<nblk(n3), 256, 0, s>>>(J.P.x, n3);
            return LQCD_OK;
        }
        src = J.P.r_hi;
    }
    J.scale = unit_scale(rho0, 6.0 * c->Vh);
    if (J.vp == VP_DF)
        k_ieee_to_vec<VP_DF><<<nblk(n3), 256, 0, s>>>(src, J.P.r, n3, J.scale);
    else
        k_ieee_to_vec<VP_F32><<<nblk(n3), 256, 0, s>>>(src, J.P.r, n3, J.scale);
    LQCD_CUDA(cudaGetLastError());
    // FP64: iterate to half the tolerance; mixed: FP32 reaches ~1e-6 at best
    // both engines iterate to tol/2; the FP32 engine refreshes its residual
    // in FP64 (reliable update) whenever it has fallen by delta
    // FP16 links differ from the operator by ~1e-3 relative; with the
    // condition numbers of the small shifts that error times kappa exceeds
    // one, so FP16 iterations stop at a moderate residual (no reliable
    // updates) and the FP32 batched refinement finishes every shift.
    const bool f16 = J.lf == LF_F16_12;
    const double tol_iter = f16 ? std::max(0.5 * J.tol, 3e-4) : 0.5 * J.tol;
    init_state(S, J.mass, J.shifts, J.n_shift, tol_iter, J.b2 * J.scale * J.scale, c->opts.max_iter);
    S.rho = rho0 * J.scale * J.scale;  // the iterated residual starts at b (or at the guess's residual)
    if (J.vp == VP_DF && J.switch_rel > 0.0) S.rel_stop2 = J.switch_rel * J.switch_rel * J.b2 * J.scale * J.scale;
    if (J.vp == VP_F32) {
        if (!f16) S.rel_stop2 = c->opts.delta_reliable * c->opts.delta_reliable * S.rho;
        if (J.x && !J.warm) LQCD_CUDA(cudaMemsetAsync(J.x, 0, (size_t)J.n_shift * n3 * sizeof(double2), s));
    }
    LQCD_CUDA(cudaMemcpyAsync(J.P.st, &S, sizeof S, cudaMemcpyHostToDevice, s));
    if (J.vp == VP_DF)
        k_init_vectors<VP_DF><<<nblk(n3), 256, 0, s>>>(J.P.r, J.P.r, J.P.x, J.P.ps, n3, J.n_shift);
    else
        k_init_vectors<VP_F32><<<nblk(n3), 256, 0, s>>>(J.P.r, J.P.r, J.P.x, J.P.ps, n3, J.n_shift);
    LQCD_CUDA(cudaGetLastError());
    c->launches += 2;
    return LQCD_OK;
}

void job_fill(const JobRun &J, IterJob &out) { fill_job(J.c, J.P, J.links, out); }

// Reliable update of the FP32 multi-shift iteration: every shift's FP32
// solution is added to its FP64 solution and cleared, the base residual is
// replaced by the FP64 true residual of the base system (rescaled to O(1)
// entries), and the search directions are kept (rescaled with it).  The
// shifted residuals stay zeta_i times the base residual.
int job_reliable_update(JobRun &J, cudaStream_t s)
{
    lqcd_ctx *c = J.c;
    const long n3 = 3 * (long)c->Vh;
    SolverState O;
    LQCD_CUDA(cudaMemcpyAsync(&O, J.P.st, sizeof O, cudaMemcpyDeviceToHost, s));
    LQCD_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < J.n_shift; ++i) {
        const size_t off = (size_t)i * n3;
        k_vec_to_ieee<VP_F32><<<nblk(n3), 256, 0, s>>>((const float2 *)J.P.x + off, J.x + off, n3, 1.0 / J.scale, 1);
    }
    k_zero_vec<VP_F32><<<nblk(n3 * J.n_shift), 256, 0, s>>>(J.P.x, n3 * J.n_shift);
    LQCD_CUDA(cudaGetLastError());
    c->launches += J.n_shift + 1;
    double rr;
    const double a0 = J.mass * J.mass + J.shifts[O.base];
    int st = refresh_residual(c, J.P, VP_F32, a0, J.x + (size_t)O.base * n3, J.b, J.P.r_hi, s, rr);
    if (st) return st;
    if (!std::isfinite(rr)) return fail(LQCD_ENAN, "NaN/Inf in a reliable update");
    const double old = J.scale;
    J.scale = unit_scale(rr, 6.0 * c->Vh);
    k_ieee_to_vec<VP_F32><<<nblk(n3), 256, 0, s>>>(J.P.r_hi, J.P.r, n3, J.scale);
    k_scale_vec<VP_F32><<<nblk(n3 * J.n_shift), 256, 0, s>>>(J.P.ps, n3 * J.n_shift, (float)(J.scale / old));
    LQCD_CUDA(cudaGetLastError());
    c->launches += 2;
    SolverState U = O;
    U.rho = rr * J.scale * J.scale;
    U.rel_stop2 = c->opts.delta_reliable * c->opts.delta_reliable * U.rho;
    U.tol2_b2 = 0.25 * J.tol * J.tol * J.b2 * J.scale * J.scale;
    U.halt = HALT_NONE;
    U.do_k4 = 0;
    LQCD_CUDA(cudaMemcpyAsync(J.P.st, &U, sizeof U, cudaMemcpyHostToDevice, s));
    ++J.I.reliable_updates;
    // the iterated residual may already meet the target after the refresh
    if (rr <= 0.25 * J.tol * J.tol * J.b2) {
        U.halt = HALT_CONVERGED;
        U.n_act = 0;
        LQCD_CUDA(cudaMemcpyAsync(J.P.st, &U, sizeof U, cudaMemcpyHostToDevice, s));
    }
    return LQCD_OK;
}

// Finish every shift of a mixed-precision multi-shift job: warm-started
// single-shift FP32 CG with FP64 reliable updates, one job per shift, all in
// one interleaved packed launch.  Fills J.I.true_resid; returns the largest
// iteration count and the number of reliable updates.
static int refine_shifts_packed(JobRun &J, int lf, cudaStream_t s, int &iters, int &reliable)
{
    lqcd_ctx *c = J.c;
    const long n3 = 3 * (long)c->Vh;
    const void *links = lf == LF_F32_12 ? c->lnk_f12.ptr : c->lnk_f18.ptr;
    std::vector<JobRun> R(J.n_shift);
    std::vector<Workspace> &W = c->ref_ws;
    if ((int)W.size() < J.n_shift) W.resize(J.n_shift);
    std::vector<int> idx;
    int st;
    for (int i = 0; i < J.n_shift; ++i) {
        JobRun &K = R[i];
        K.c = c;
        K.vp = VP_F32;
        K.lf = lf;
        K.links = links;
        K.mass = J.mass;
        K.n_shift = 1;
        K.shifts[0] = J.shifts[i];
        K.tol = J.tol;
        K.b = J.b;
        K.x = J.x + (size_t)i * n3;
        K.warm = true;
        if ((st = ensure_workspace_in(c, W[i], VP_F32, 1, K.P))) return st;
        if ((st = job_setup(K, s))) return st;
        SolverState O;
        LQCD_CUDA(cudaMemcpyAsync(&O, K.P.st, sizeof O, cudaMemcpyDeviceToHost, s));
        LQCD_CUDA(cudaStreamSynchronize(s));
        if (O.halt == HALT_NONE) idx.push_back(i);
    }
    iters = 0;
    reliable = 0;
    if (!idx.empty()) {
        IterBatch<kMaxJobs> B;
        memset(&B, 0, sizeof B);
        B.njobs = (int)idx.size();
        B.max_shift = 1;
        B.interleave = 1;
        for (int k = 0; k < B.njobs; ++k) job_fill(R[idx[k]], B.job[k]);
        const int chunk = c->opts.check_every;
        cudaGraphExec_t exec = nullptr;
        if ((st = chunk_graph<kMaxJobs>(c, B, VP_F32, lf, chunk, s, exec))) return st;
        int *hs = c->h_pinned;
        const int max_chunks = 4 * (c->opts.max_iter / chunk + 4);
        int rc = LQCD_OK;
        for (int k = 0; k < max_chunks && rc == LQCD_OK; ++k) {
            cudaError_t e = cudaGraphLaunch(exec, s);
            c->launches += 4 * (uint64_t)chunk;
            for (int q = 0; q < B.njobs && e == cudaSuccess; ++q)
                e = cudaMemcpyAsync(hs + q, &B.job[q].st->halt, sizeof(int), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) { rc = cuda_fail(e, "refinement chunk"); break; }
            bool all = true;
            for (int q = 0; q < B.njobs && rc == LQCD_OK; ++q) {
                if (hs[q] == HALT_RELIABLE) rc = job_reliable_update(R[idx[q]], s), all = false;
                else if (hs[q] == HALT_NAN) rc = fail(LQCD_ENAN, "NaN/Inf or breakdown in refinement");
                else if (hs[q] == HALT_NONE) all = false;
            }
            if (all) break;
        }
        if (rc) return rc;
    }
    for (int i = 0; i < J.n_shift; ++i) {
        JobRun &K = R[i];
        k_vec_to_ieee<VP_F32><<<nblk(n3), 256, 0, s>>>(K.P.x, K.x, n3, 1.0 / K.scale, 1);
        LQCD_CUDA(cudaGetLastError());
        SolverState O;
        LQCD_CUDA(cudaMemcpyAsync(&O, K.P.st, sizeof O, cudaMemcpyDeviceToHost, s));
        double rr;
        if ((st = true_residual(c, K.P, VP_F32, J.mass * J.mass + J.shifts[i], K.x, J.b, nullptr, nullptr, 1.0, s,
                                rr)))
            return st;
        J.I.true_resid[i] = std::sqrt(rr / J.b2);
        iters = std::max(iters, O.iters);
        reliable += K.I.reliable_updates;
        const double spin = 24.0;
        J.bytes += (double)c->Vh * O.iters * (iter_bytes_base(VP_F32, lf) + 4 * spin);
    }
    return LQCD_OK;
}

// Algorithmic bytes of the iterations a job ran since iteration J.iters0.
static double phase_bytes(const JobRun &J, const SolverState &O)
{
    double shift_it = 0;
    for (int i = 0; i < J.n_shift; ++i)
        shift_it += std::max(0, (O.shift_iters[i] ? O.shift_iters[i] : O.iters) - J.iters0);
    const double spin = J.vp == VP_DF ? 48.0 : 24.0;
    return (double)J.c->Vh * (std::max(0, O.iters - J.iters0) * iter_bytes_base(J.vp, J.lf) + shift_it * 4 * spin);
}

// After the iterations: IEEE solutions, FP64 true residuals, refinement.
int job_finish(JobRun &J, cudaStream_t s)
{
    lqcd_ctx *c = J.c;
    const long n3 = 3 * (long)c->Vh;
    int st;
    if (J.zero) {
        J.I.status = LQCD_OK;
        return LQCD_OK;
    }
    SolverState O;
    LQCD_CUDA(cudaMemcpyAsync(&O, J.P.st, sizeof O, cudaMemcpyDeviceToHost, s));
    LQCD_CUDA(cudaStreamSynchronize(s));
    if (O.halt == HALT_NAN) return fail(LQCD_ENAN, "NaN/Inf or breakdown in the multi-shift iteration");
    if (O.halt == HALT_STALL) return fail(LQCD_ETIMEOUT, "a staged stencil wait for shared-memory link data ran out");
    J.I.iters = O.iters;
    for (int i = 0; i < J.n_shift; ++i) J.I.shift_iters[i] = O.shift_iters[i];
    J.bytes += phase_bytes(J, O);
    const bool maxed = O.halt == HALT_MAXITER;
    for (int i = 0; i < J.n_shift; ++i) {
        const size_t off = (size_t)i * n3;
        if (J.vp == VP_DF)
            k_vec_to_ieee<VP_DF><<<nblk(n3), 256, 0, s>>>((const float4 *)J.P.x + off, J.x + off, n3, 1.0 / J.scale, 0);
        else
            k_vec_to_ieee<VP_F32><<<nblk(n3), 256, 0, s>>>((const float2 *)J.P.x + off, J.x + off, n3, 1.0 / J.scale, 1);
        LQCD_CUDA(cudaGetLastError());
        c->launches += 1;
    }
    int status = maxed ? LQCD_ENOCONV : LQCD_OK;
    if (J.vp == VP_DF || maxed) {
        // FP64: the df64 iteration already ran to tol/2; check each shift in
        // native FP64 and correct the rare one above tol
        for (int i = 0; i < J.n_shift; ++i) {
            double res = 0;
            int it = 0, rel = 0;
            if ((st = refine_shift(c, J.P, J.vp, J.lf, J.links, J.mass, J.shifts[i], J.b, J.b2, J.x + (size_t)i * n3,
                                   J.tol, !maxed, s, res, it, rel, J.bytes)))
                return st;
            J.I.true_resid[i] = res;
            J.I.refine_iters += it;
            J.I.reliable_updates += rel;
            if (!(res <= J.tol)) status = LQCD_ENOCONV;
        }
    } else {
        // mixed: every shift above tol is finished by its own single-shift
        // CG (FP32 iterations, FP64 reliable updates) started from its
        // multi-shift solution; all of them run as one packed launch whose
        // blocks interleave the shifts, so the blocks of different shifts
        // that read the same links run together and share them in L2.  The
        // FP16 variant uses FP32 links here (FP16 rounding times the
        // condition number of the smallest shifts exceeds one).
        const int lf2 = c->opts.recon == 12 || J.lf == LF_F16_12 ? LF_F32_12 : LF_F32_18;
        int it = 0, rel = 0;
        if ((st = refine_shifts_packed(J, lf2, s, it, rel))) return st;
        J.I.refine_iters += it;
        J.I.reliable_updates += rel;
        for (int i = 0; i < J.n_shift; ++i)
            if (!(J.I.true_resid[i] <= J.tol)) status = LQCD_ENOCONV;
    }
    LQCD_CUDA(cudaStreamSynchronize(s));
    J.I.bytes_moved = J.bytes;
    J.I.kernel_launches = (int)(c->launches - J.launches0);
    J.I.status = status;
    return status;
}

int job_init_prec(JobRun &J, lqcd_ctx *c, Workspace *W, int prec, double mass, const double *shifts, int n_shift,
                  double tol, const double2 *b, double2 *x)
{
    int st = validate_solve(c, mass, shifts, n_shift, tol);
    if (st || (st = links_ready(c))) return st;
    J.c = c;
    J.vp = prec == LQCD_PREC_FP64 || prec == LQCD_PREC_FP64_NATIVE ? VP_DF : VP_F32;
    J.lf = link_fmt_for(c, J.vp == VP_DF ? LQCD_PREC_FP64 : prec, &J.links);
    J.mass = mass;
    J.n_shift = n_shift;
    for (int i = 0; i < n_shift; ++i) J.shifts[i] = shifts[i];
    J.tol = tol;
    J.b = b;
    J.x = x;
    return ensure_workspace_in(c, W ? *W : c->ws, J.vp, n_shift, J.P);
}

int job_init(JobRun &J, lqcd_ctx *c, Workspace *W, double mass, const double *shifts, int n_shift, double tol,
             const double2 *b, double2 *x)
{
    return job_init_prec(J, c, W, c->opts.prec, mass, shifts, n_shift, tol, b, x);
}

// Hybrid mixed precision, switch from the double-float phase D (halted at
// ||r|| <= fp64_until ||b||) to the FP32 phase F: the double-float solutions
// go to the IEEE accumulators, the base residual is recomputed against the
// FP64 operator, the directions are rounded to FP32 at the new scale, and the
// recurrence scalars carry over unchanged (the same Krylov iteration goes on).
int job_switch_to_f32(JobRun &D, JobRun &F, cudaStream_t s)
{
    lqcd_ctx *c = D.c;
    const long n3 = 3 * (long)c->Vh;
    SolverState O;
    LQCD_CUDA(cudaMemcpyAsync(&O, D.P.st, sizeof O, cudaMemcpyDeviceToHost, s));
    LQCD_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < D.n_shift; ++i) {
        const size_t off = (size_t)i * n3;
        k_vec_to_ieee<VP_DF><<<nblk(n3), 256, 0, s>>>((const float4 *)D.P.x + off, D.x + off, n3, 1.0 / D.scale, 0);
    }
    LQCD_CUDA(cudaGetLastError());
    c->launches += D.n_shift;
    double rr;
    const double a0 = D.mass * D.mass + D.shifts[O.base];
    int st = refresh_residual(c, F.P, VP_F32, a0, D.x + (size_t)O.base * n3, D.b, F.P.r_hi, s, rr);
    if (st) return st;
    if (!std::isfinite(rr)) return fail(LQCD_ENAN, "NaN/Inf at the switch to FP32");
    F.scale = unit_scale(rr, 6.0 * c->Vh);
    k_ieee_to_vec<VP_F32><<<nblk(n3), 256, 0, s>>>(F.P.r_hi, F.P.r, n3, F.scale);
    k_df_to_f32<<<nblk(n3 * D.n_shift), 256, 0, s>>>((const float4 *)D.P.ps, (float2 *)F.P.ps, n3 * D.n_shift,
                                                     F.scale / D.scale);
    k_zero_vec<VP_F32><<<nblk(n3 * D.n_shift), 256, 0, s>>>(F.P.x, n3 * D.n_shift);
    LQCD_CUDA(cudaGetLastError());
    c->launches += 3;
    SolverState U = O;
    U.rho = rr * F.scale * F.scale;
    U.rel_stop2 = c->opts.delta_reliable * c->opts.delta_reliable * U.rho;
    U.tol2_b2 = 0.25 * F.tol * F.tol * F.b2 * F.scale * F.scale;
    U.halt = rr <= 0.25 * F.tol * F.tol * F.b2 ? HALT_CONVERGED : HALT_NONE;
    U.do_k4 = 0;
    if (U.halt) U.n_act = 0;
    LQCD_CUDA(cudaMemcpyAsync(F.P.st, &U, sizeof U, cudaMemcpyHostToDevice, s));
    F.iters0 = O.iters;
    F.bytes = D.bytes + phase_bytes(D, O);
    F.I = D.I;
    F.launches0 = D.launches0;
    return LQCD_OK;
}

// One packed iteration launch over several jobs (serving ticks).
void launch_iteration_packed(const IterBatch<kMaxJobs> &B, int vp, int lf, cudaStream_t s, bool pdl, bool chained)
{
    launch_iteration<kMaxJobs>(B, B.tile_start[B.njobs], vp, lf, s, pdl, chained);
}

int run_packed_until_halt(lqcd_ctx *c, const IterBatch<kMaxJobs> &B, int vp, int lf, cudaStream_t s)
{
    std::vector<int> halts;
    return run_until_halt<kMaxJobs>(c, B, vp, lf, c->opts.check_every, c->opts.max_iter, s, halts);
}

// ------------------------------------------------------------------ public drivers
int mscg_solve_dev(lqcd_ctx *c, double mass, const double *shifts, int n_shift, double tol, const double2 *b,
                   double2 *x, lqcd_solve_info *info, cudaStream_t s_user)
{
    const auto t0 = std::chrono::steady_clock::now();
    if (!b || !x) return fail(LQCD_EINVAL, "NULL argument");
    // FP32 links: double-float iterations down to fp64_until, then FP32
    const bool hybrid = c->opts.prec == LQCD_PREC_FP32 && c->opts.fp64_until > 0.0;
    JobRun J;
    int st = job_init_prec(J, c, nullptr, hybrid ? LQCD_PREC_FP64 : c->opts.prec, mass, shifts, n_shift, tol, b, x);
    if (st) return st;
    if (hybrid) J.switch_rel = c->opts.fp64_until;
    cudaStream_t s = c->stream;
    if (s_user && s_user != s) LQCD_CUDA(cudaStreamSynchronize(s_user));
    if ((st = job_setup(J, s))) return st;
    auto iterate = [&](JobRun &R, bool stop_on_reliable, int &halt) -> int {
        IterBatch<1> B;
        memset(&B, 0, sizeof B);
        B.njobs = 1;
        B.max_shift = R.n_shift;
        B.tile_start[1] = R.P.ntiles;
        job_fill(R, B.job[0]);
        for (;;) {
            std::vector<int> halts;
            int rc = run_until_halt<1>(c, B, R.vp, R.lf, c->opts.check_every, c->opts.max_iter, s, halts);
            if (rc) return rc;
            halt = halts[0];
            if (halt != HALT_RELIABLE || stop_on_reliable) return LQCD_OK;
            if ((rc = job_reliable_update(R, s))) return rc;
        }
    };
    JobRun F;
    JobRun *fin = &J;
    if (!J.zero) {
        int halt = HALT_NONE;
        if ((st = iterate(J, hybrid, halt))) return st;
        if (hybrid && halt == HALT_RELIABLE) {
            if ((st = job_init_prec(F, c, &c->ws32, LQCD_PREC_FP32, mass, shifts, n_shift, tol, b, x))) return st;
            F.b2 = J.b2;
            if ((st = job_switch_to_f32(J, F, s))) return st;
            if ((st = iterate(F, false, halt))) return st;
            fin = &F;
        }
    }
    JobRun &R = *fin;
    st = job_finish(R, s);
    J.I = R.I;
    J.I.secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = J.I;
    if (st == LQCD_ENOCONV) set_error("solver did not reach tol within max_iter");
    return st;
}

int profile_iteration(lqcd_ctx *c, double mass, const double *shifts, int n_shift, double tol, const double2 *b,
                      int iters, double ms[4], double *n_act_avg)
{
    if (!b || iters < 1 || iters > 100000) return fail(LQCD_EINVAL, "bad profile arguments");
    JobRun J;
    int st = job_init(J, c, nullptr, mass, shifts, n_shift, tol, b, nullptr);
    if (st) return st;
    cudaStream_t s = c->stream;
    if ((st = job_setup(J, s))) return st;
    if (J.zero) return fail(LQCD_EINVAL, "zero source");
    // iterate as the solve does (same stopping rule), past its end if asked
    SolverState S;
    LQCD_CUDA(cudaMemcpy(&S, J.P.st, sizeof S, cudaMemcpyDeviceToHost));
    S.max_iter = iters + 1;
    LQCD_CUDA(cudaMemcpy(J.P.st, &S, sizeof S, cudaMemcpyHostToDevice));
    IterBatch<1> B;
    memset(&B, 0, sizeof B);
    B.njobs = 1;
    B.max_shift = n_shift;
    B.tile_start[1] = J.P.ntiles;
    job_fill(J, B.job[0]);
    std::vector<cudaEvent_t> ev(5 * (size_t)iters);
    for (auto &e : ev) LQCD_CUDA(cudaEventCreate(&e));
    int *hn = nullptr;
    LQCD_CUDA(cudaHostAlloc((void **)&hn, (size_t)iters * sizeof(int), cudaHostAllocDefault));
    const int ntot = J.P.ntiles;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < iters && e == cudaSuccess; ++k) {
        cudaEvent_t *E = &ev[5 * (size_t)k];
        cudaEventRecord(E[0], s);
        for (int q = 0; q < 4; ++q) {
            launch_kernel_k<1>(B, q, ntot, J.vp, J.lf, s, false);
            cudaEventRecord(E[q + 1], s);
        }
        c->launches += 4;
        e = cudaMemcpyAsync(hn + k, &J.P.st->n_act, sizeof(int), cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    double acc[4] = {0, 0, 0, 0}, na = 0;
    int counted = 0;
    if (e == cudaSuccess) {
        SolverState O;
        e = cudaMemcpy(&O, J.P.st, sizeof O, cudaMemcpyDeviceToHost);
        // only iterations that ran (the solve may converge before `iters`)
        counted = std::min(iters, O.iters);
        for (int k = 0; k < counted; ++k) {
            for (int q = 0; q < 4; ++q) {
                float t = 0.f;
                cudaEventElapsedTime(&t, ev[5 * (size_t)k + q], ev[5 * (size_t)k + q + 1]);
                acc[q] += t;
            }
            na += hn[k];
        }
    }
    for (auto &ee : ev) cudaEventDestroy(ee);
    cudaFreeHost(hn);
    if (e != cudaSuccess) return cuda_fail(e, "profile iteration");
    if (counted == 0) return fail(LQCD_EINVAL, "no iteration ran");
    for (int q = 0; q < 4; ++q) ms[q] = acc[q] / counted;
    *n_act_avg = na / counted;
    return LQCD_OK;
}

int mscg_solve_packed(lqcd_ctx *const *ctxs, int n, const double *mass, const double *const *shifts,
                      const int *n_shift, const double *tol, const double *const *b, double *const *x,
                      lqcd_solve_info *info)
{
    const auto t0 = std::chrono::steady_clock::now();
    lqcd_ctx *c0 = ctxs[0];
    cudaStream_t s = c0->stream;
    std::vector<JobRun> J(n);
    std::vector<DevBuf> bd(n), xd(n);
    int st;
    for (int i = 0; i < n; ++i) {
        lqcd_ctx *c = ctxs[i];
        if (!c || !b[i] || !x[i]) return fail(LQCD_EINVAL, "NULL context or buffer in packed solve");
        if (c->device != c0->device) return fail(LQCD_EINVAL, "packed contexts must share a device");
        for (int k = 0; k < i; ++k)
            if (ctxs[k] == c) return fail(LQCD_EINVAL, "a context appears twice in a packed solve");
        const size_t n3 = 3 * c->Vh;
        if ((st = bd[i].ensure(n3 * sizeof(double2))) || (st = xd[i].ensure((size_t)n_shift[i] * n3 * sizeof(double2))))
            return st;
        if ((st = job_init(J[i], c, nullptr, mass[i], shifts[i], n_shift[i], tol[i], bd[i].as<double2>(),
                           xd[i].as<double2>())))
            return st;
        if (i > 0 && J[i].vp != J[0].vp) return fail(LQCD_EINVAL, "packed contexts must use the same precision");
        if (i > 0 && J[i].lf != J[0].lf) return fail(LQCD_EINVAL, "packed contexts must use the same link storage");
        LQCD_CUDA(cudaStreamSynchronize(c->stream));
        if ((st = host_to_soa(c, b[i], bd[i].as<double2>(), 1, s))) return st;
        if ((st = job_setup(J[i], s))) return st;
    }
    IterBatch<kMaxJobs> B;
    memset(&B, 0, sizeof B);
    int nj = 0, tiles = 0;
    for (int i = 0; i < n; ++i) {
        if (J[i].zero) continue;
        B.max_shift = std::max(B.max_shift, J[i].n_shift);
        B.tile_start[nj] = tiles;
        job_fill(J[i], B.job[nj]);
        tiles += J[i].P.ntiles;
        ++nj;
    }
    B.njobs = nj;
    B.tile_start[nj] = tiles;
    if (nj > 0 && (st = run_packed_until_halt(c0, B, J[0].vp, J[0].lf, s))) return st;
    int status = LQCD_OK;
    const double secs_iter = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int i = 0; i < n; ++i) {
        st = job_finish(J[i], s);
        if (st != LQCD_OK && st != LQCD_ENOCONV) return st;
        if (st == LQCD_ENOCONV) status = st;
        if ((st = soa_to_host(ctxs[i], xd[i].as<double2>(), x[i], n_shift[i], s))) return st;
        LQCD_CUDA(cudaStreamSynchronize(s));
        J[i].I.secs = secs_iter;
        if (info) info[i] = J[i].I;
    }
    if (status == LQCD_ENOCONV) set_error("a packed solve did not reach tol within max_iter");
    return status;
}

}  // namespace lqcd
