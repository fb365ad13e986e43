// shard.cu -- domain decomposition of D_eo / D_oe and of CG into slabs of
// time slices (the distribution of the lattice over GPUs that the paper's
// concluding remarks leave for future work, Sec. 6), one context per rank.
//
// Layout (half index of Eq. lexicographic_eo, t = x3 the slowest
// coordinate): the sites of either parity in t-slices [ta, tb) are the half
// indices [ta S/2, tb S/2), S = N0 N1 N2, in the same order in every slice.
// Rank r of W owns global slices [t0, t0 + nt), t0 = r nt, nt = Lt / W (even,
// >= 2).  Its context holds an extended slab of nt + 2 G slices, G = 2:
// local slice k is global slice (t0 - G + k) mod Lt.  Because t0 - G is
// even, a site keeps its global parity and every slice keeps the global
// half-index order, so:
//   - a field of the rank is [3][Vh_ext] complex128 over the extended slab;
//   - the owned sites are the half-index range [G h, (G + nt) h), h = S/2;
//   - the hops of the owned sites reach one slice beyond each side, the
//     "ghost faces" [(G-1) h, G h) and [(G+nt) h, (G+nt+1) h), filled by
//     one plain copy each from the neighbouring ranks' owned boundary slices
//     (lqcd_shard_exchange: one cudaMemcpy2DAsync per face, all three colour
//     arrays at once, into the receiving rank's own memory before use).
// Links are static during a solve: each rank uploads the links of its whole
// extended slab once.  The global antiperiodic sign sits on the time links
// of global slice Lt - 1; the kernels apply the sign of the LOCAL last slice
// (which no owned site's hop reaches), so the upload multiplies the time
// links of every local slice that is global slice Lt - 1 by -1.
//
// The sharded CG adds each rank's FP64 partial sums (fixed block order) and
// then the ranks' sums in rank order, so every rank uses the same bits for
// alpha and beta whatever the number of ranks in flight.
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "deo_core.cuh"
#include "internal.h"

namespace lqcd {

constexpr int kShardGhost = 2;
constexpr int kShardThreads = 256;

// Sharded D: out = D_eo in (P = 0) or D_oe in (P = 1) at the sites [lo, hi)
// of the extended slab, in the double-float arithmetic of the unsharded
// operator (same hop order, same bits per site).
__global__ void __launch_bounds__(kShardThreads, 2)
    k_shard_deo(Geom g, const float4 *__restrict__ L, const double2 *__restrict__ in, double2 *__restrict__ out,
                int P, int lo, int hi)
{
    const int i = lo + blockIdx.x * kShardThreads + threadIdx.x;
    if (i >= hi) return;
    Stencil S;
    make_stencil(g, i, P, S);
    float2 res[6];
    bool bad = false;
    deo_site_df<SF_IEEE>(g, L, in, S, i, P, g.Vh, res, bad);
    double2 o[3];
    if (bad) {
        deo_site_native_from_df(g, L, in, S, i, P, g.Vh, o);
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) o[c] = make_double2(df_to_f64(res[2 * c]), df_to_f64(res[2 * c + 1]));
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) out[(size_t)c * g.Vh + i] = o[c];
}

// Fixed-order block sum of one double per thread; thread 0 writes part[blockIdx.x].
__device__ __forceinline__ void shard_block_sum(double v, double *part)
{
    __shared__ double s_red[kShardThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < kShardThreads / 32; ++k) s += s_red[k];
        part[blockIdx.x] = s;
    }
}

// q = a p - D_eo t at the owned even sites [lo, hi); part[block] = Re <p, q>.
__global__ void __launch_bounds__(kShardThreads, 2)
    k_shard_normal(Geom g, const float4 *__restrict__ L, const double2 *__restrict__ t,
                   const double2 *__restrict__ p, double2 *__restrict__ q, double a, int lo, int hi, double *part)
{
    const int i = lo + blockIdx.x * kShardThreads + threadIdx.x;
    double acc = 0.0;
    if (i < hi) {
        Stencil S;
        make_stencil(g, i, 0, S);
        float2 res[6];
        bool bad = false;
        deo_site_df<SF_IEEE>(g, L, t, S, i, 0, g.Vh, res, bad);
        double2 o[3];
        if (bad) {
            deo_site_native_from_df(g, L, t, S, i, 0, g.Vh, o);
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) o[c] = make_double2(df_to_f64(res[2 * c]), df_to_f64(res[2 * c + 1]));
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t k = (size_t)c * g.Vh + i;
            const double2 pv = p[k];
            const double2 qv = make_double2(fma(a, pv.x, -o[c].x), fma(a, pv.y, -o[c].y));
            q[k] = qv;
            acc = fma(pv.x, qv.x, fma(pv.y, qv.y, acc));
        }
    }
    shard_block_sum(acc, part);
}

// x += alpha p, r -= alpha q at [lo, hi); part[block] = ||r||^2.
__global__ void __launch_bounds__(kShardThreads)
    k_shard_update_xr(int Vh, double2 *__restrict__ x, double2 *__restrict__ r, const double2 *__restrict__ p,
                      const double2 *__restrict__ q, double alpha, int lo, int hi, double *part)
{
    const int i = lo + blockIdx.x * kShardThreads + threadIdx.x;
    double acc = 0.0;
    if (i < hi) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t k = (size_t)c * Vh + i;
            const double2 pv = p[k], qv = q[k];
            double2 xv = x[k], rv = r[k];
            xv.x = fma(alpha, pv.x, xv.x);
            xv.y = fma(alpha, pv.y, xv.y);
            rv.x = fma(-alpha, qv.x, rv.x);
            rv.y = fma(-alpha, qv.y, rv.y);
            x[k] = xv;
            r[k] = rv;
            acc = fma(rv.x, rv.x, fma(rv.y, rv.y, acc));
        }
    }
    shard_block_sum(acc, part);
}

// p = r + beta p at [lo, hi).
__global__ void __launch_bounds__(kShardThreads)
    k_shard_xpay(int Vh, double2 *__restrict__ p, const double2 *__restrict__ r, double beta, int lo, int hi)
{
    const int i = lo + blockIdx.x * kShardThreads + threadIdx.x;
    if (i >= hi) return;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const size_t k = (size_t)c * Vh + i;
        const double2 rv = r[k], pv = p[k];
        p[k] = make_double2(fma(beta, pv.x, rv.x), fma(beta, pv.y, rv.y));
    }
}

// r = b - q (q = A x) at [lo, hi); part[block] = ||r||^2.  Also used with
// q = 0 to start from r = b.
__global__ void __launch_bounds__(kShardThreads)
    k_shard_residual(int Vh, double2 *__restrict__ r, const double2 *__restrict__ b, const double2 *__restrict__ q,
                     int lo, int hi, double *part)
{
    const int i = lo + blockIdx.x * kShardThreads + threadIdx.x;
    double acc = 0.0;
    if (i < hi) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t k = (size_t)c * Vh + i;
            const double2 bv = b[k];
            const double2 qv = q ? q[k] : make_double2(0.0, 0.0);
            const double2 rv = make_double2(bv.x - qv.x, bv.y - qv.y);
            r[k] = rv;
            acc = fma(rv.x, rv.x, fma(rv.y, rv.y, acc));
        }
    }
    shard_block_sum(acc, part);
}

// out[0] = sum of part[0 .. n) in a fixed order (one block).
__global__ void __launch_bounds__(kShardThreads) k_shard_sum(const double *__restrict__ part, int n, double *out)
{
    __shared__ double s_red[kShardThreads / 32];
    double v = 0.0;
    for (int k = threadIdx.x; k < n; k += kShardThreads) v += part[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < kShardThreads / 32; ++k) s += s_red[k];
        *out = s;
    }
}

// ------------------------------------------------------------------ host side
struct ShardGeom {
    long h;       // sites per parity and slice (S / 2)
    long lo, hi;  // owned half-index range of the extended slab
    long vh;      // half sites of the extended slab
};

static ShardGeom shard_geom(const lqcd_ctx *c)
{
    ShardGeom s;
    s.h = (long)c->dims[0] * c->dims[1] * c->dims[2] / 2;
    s.lo = kShardGhost * s.h;
    s.hi = (kShardGhost + c->shard_nt) * s.h;
    s.vh = (long)c->Vh;
    return s;
}

static int check_shard(const lqcd_ctx *c)
{
    if (!c) return fail(LQCD_EINVAL, "NULL context");
    if (c->shard_world < 1) return fail(LQCD_EINVAL, "not a shard context (use lqcd_shard_create)");
    return LQCD_OK;
}

// The contexts of one decomposition, in rank order: same global lattice and
// world size, ranks 0 .. n-1, all of them present (n == world).
static int check_world(lqcd_ctx *const *ctxs, int n)
{
    if (!ctxs || n < 1) return fail(LQCD_EINVAL, "no shard contexts");
    for (int r = 0; r < n; ++r) {
        if (int st = check_shard(ctxs[r])) return st;
        const lqcd_ctx *c = ctxs[r];
        if (c->shard_world != n || c->shard_rank != r)
            return fail(LQCD_EINVAL, "shard contexts must be the ranks 0..world-1 of one decomposition, in order");
        for (int d = 0; d < 4; ++d)
            if (c->gdims[d] != ctxs[0]->gdims[d]) return fail(LQCD_EINVAL, "shard contexts of different lattices");
    }
    return LQCD_OK;
}

// Every rank's stream waits for the work queued so far on every other
// rank's stream (events; the ranks may live on different devices).
static int join_streams(lqcd_ctx *const *ctxs, int n)
{
    std::vector<cudaEvent_t> ev(n, nullptr);
    int st = LQCD_OK;
    for (int r = 0; r < n && !st; ++r) {
        DeviceGuard dg(ctxs[r]->device);
        cudaError_t e = cudaEventCreateWithFlags(&ev[r], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ev[r], ctxs[r]->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "shard stream join (record)");
    }
    for (int r = 0; r < n && !st; ++r) {
        DeviceGuard dg(ctxs[r]->device);
        for (int k = 0; k < n && !st; ++k) {
            if (k == r) continue;
            const cudaError_t e = cudaStreamWaitEvent(ctxs[r]->stream, ev[k], 0);
            if (e != cudaSuccess) st = cuda_fail(e, "shard stream join (wait)");
        }
    }
    for (int r = 0; r < n; ++r)
        if (ev[r]) {
            DeviceGuard dg(ctxs[r]->device);
            cudaEventDestroy(ev[r]);
        }
    return st;
}

// Fill the ghost faces of every rank's field (device complex128 [3][Vh_ext]):
// the lower ghost slice of rank r is the top owned slice of rank r-1, the
// upper ghost slice the bottom owned slice of rank r+1 (periodic in rank).
// Each face is one 2-D copy (three colour rows of h sites) on the receiving
// rank's stream, between two joins of all ranks' streams.
static int exchange_faces(lqcd_ctx *const *ctxs, int n, void *const *fields)
{
    for (int r = 0; r < n; ++r)
        if (!fields[r]) return fail(LQCD_EINVAL, "NULL shard field");
    if (int st = join_streams(ctxs, n)) return st;
    const ShardGeom G = shard_geom(ctxs[0]);
    const size_t pitch = (size_t)G.vh * sizeof(double2), width = (size_t)G.h * sizeof(double2);
    for (int r = 0; r < n; ++r) {
        DeviceGuard dg(ctxs[r]->device);
        const int below = (r + n - 1) % n, above = (r + 1) % n;
        double2 *dst = (double2 *)fields[r];
        const double2 *top_below = (const double2 *)fields[below] + (G.hi - G.h);
        const double2 *bottom_above = (const double2 *)fields[above] + G.lo;
        LQCD_CUDA(cudaMemcpy2DAsync(dst + (G.lo - G.h), pitch, top_below, pitch, width, 3, cudaMemcpyDefault,
                                    ctxs[r]->stream));
        LQCD_CUDA(cudaMemcpy2DAsync(dst + G.hi, pitch, bottom_above, pitch, width, 3, cudaMemcpyDefault,
                                    ctxs[r]->stream));
    }
    return join_streams(ctxs, n);
}

static unsigned shard_blocks(const ShardGeom &G) { return (unsigned)((G.hi - G.lo + kShardThreads - 1) / kShardThreads); }

}  // namespace lqcd

using namespace lqcd;

extern "C" {

int lqcd_shard_create(const int dims[4], int world, int rank, const lqcd_opts *opts, lqcd_ctx **out)
{
    if (!dims || !out) return fail(LQCD_EINVAL, "NULL argument");
    *out = nullptr;
    for (int d = 0; d < 4; ++d)
        if (dims[d] < 2 || (dims[d] & 1)) return fail(LQCD_EINVAL, "lattice sides must be even and >= 2");
    if (world < 1 || rank < 0 || rank >= world) return fail(LQCD_EINVAL, "rank must be in 0..world-1");
    if (dims[3] % world) return fail(LQCD_EINVAL, "the time extent must be divisible by the number of ranks");
    const int nt = dims[3] / world;
    if (nt < 2 || (nt & 1)) return fail(LQCD_EINVAL, "the slab extent N3/world must be even and >= 2");
    const int ext[4] = {dims[0], dims[1], dims[2], nt + 2 * kShardGhost};
    lqcd_opts o;
    lqcd_default_opts(&o);
    if (opts) o = *opts;
    o.staged = 0;  // the sharded kernels read the structure-of-arrays links only
    lqcd_ctx *c = nullptr;
    int st = lqcd_create(ext, &o, &c);
    if (st) return st;
    c->shard_world = world;
    c->shard_rank = rank;
    c->shard_nt = nt;
    c->shard_t0 = rank * nt;
    for (int d = 0; d < 4; ++d) c->gdims[d] = dims[d];
    *out = c;
    return LQCD_OK;
}

int lqcd_shard_geometry(const lqcd_ctx *c, long info[6])
{
    if (int st = check_shard(c)) return st;
    if (!info) return fail(LQCD_EINVAL, "NULL argument");
    const ShardGeom G = shard_geom(c);
    info[0] = c->shard_t0;
    info[1] = c->shard_nt;
    info[2] = G.vh;
    info[3] = G.h;
    info[4] = G.lo;
    info[5] = G.hi;
    return LQCD_OK;
}

int lqcd_shard_links_upload(lqcd_ctx *c, const double *links, size_t n_doubles)
{
    NvtxRange nvtx_("lqcd_shard_links_upload");
    if (int st = check_shard(c)) return st;
    LQCD_ON_DEVICE(c->device);
    const long S = (long)c->gdims[0] * c->gdims[1] * c->gdims[2];
    const long Lt = c->gdims[3], V = S * Lt;
    if (!links || n_doubles != (size_t)(4 * V * 18))
        return fail(LQCD_EINVAL, "shard links: expected the global field, 4*V*18 doubles");
    const long next = c->dims[3];
    std::vector<double> ext((size_t)4 * next * S * 18);
    for (int mu = 0; mu < 4; ++mu)
        for (long k = 0; k < next; ++k) {
            const long tg = ((c->shard_t0 - kShardGhost + k) % Lt + Lt) % Lt;
            const double *src = links + ((size_t)mu * V + (size_t)tg * S) * 18;
            double *dst = ext.data() + ((size_t)mu * next * S + (size_t)k * S) * 18;
            const double sg = (mu == 3 && tg == Lt - 1) ? -1.0 : 1.0;  // global antiperiodic time links
            if (sg > 0)
                memcpy(dst, src, (size_t)S * 18 * sizeof(double));
            else
                for (long j = 0; j < S * 18; ++j) dst[j] = -src[j];
        }
    c->graph.reset();
    return upload_links(c, ext.data(), ext.size());
}

int lqcd_shard_deo_apply(lqcd_ctx *c, int out_parity, const void *in, void *out, void *stream)
{
    NvtxRange nvtx_("lqcd_shard_deo_apply");
    if (int st = check_shard(c)) return st;
    LQCD_ON_DEVICE(c->device);
    if (int lr = links_ready(c)) return lr;
    if (out_parity != 0 && out_parity != 1) return fail(LQCD_EINVAL, "out_parity must be 0 or 1");
    if (!in || !out) return fail(LQCD_EINVAL, "NULL spinor pointer");
    if (in == out) return fail(LQCD_EINVAL, "in and out must not overlap");
    const ShardGeom G = shard_geom(c);
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    k_shard_deo<<<shard_blocks(G), kShardThreads, 0, s>>>(c->g, c->lnk_df.as<float4>(), (const double2 *)in,
                                                          (double2 *)out, out_parity, (int)G.lo, (int)G.hi);
    LQCD_CUDA(cudaGetLastError());
    c->launches += 1;
    return LQCD_OK;
}

int lqcd_shard_exchange(lqcd_ctx *const *ctxs, int n, void *const *fields)
{
    NvtxRange nvtx_("lqcd_shard_exchange");
    if (int st = check_world(ctxs, n)) return st;
    if (!fields) return fail(LQCD_EINVAL, "NULL field array");
    LQCD_ON_DEVICE(ctxs[0]->device);
    return exchange_faces(ctxs, n, fields);
}

}  // extern "C"

namespace lqcd {

// Device vectors of one rank's sharded CG, each a [3][Vh_ext] complex128 field.
struct ShardVecs {
    double2 *b, *x, *r, *p, *q, *t;
    double *part;  // per-block partials, then the rank's total at [nblocks]
    unsigned nb;
};

static int shard_vecs(lqcd_ctx *c, ShardVecs &V)
{
    const ShardGeom G = shard_geom(c);
    const size_t f = 3 * (size_t)G.vh;
    V.nb = shard_blocks(G);
    int st;
    if ((st = c->shard_ws.ensure(6 * f * sizeof(double2) + ((size_t)V.nb + 1) * sizeof(double)))) return st;
    double2 *base = c->shard_ws.as<double2>();
    V.b = base;
    V.x = base + f;
    V.r = base + 2 * f;
    V.p = base + 3 * f;
    V.q = base + 4 * f;
    V.t = base + 5 * f;
    V.part = (double *)(base + 6 * f);
    return LQCD_OK;
}

// Sum over ranks, in rank order, of each rank's total at V[r].part[nb]
// (copied to the host once every rank's stream has reached it).
static int ordered_total(lqcd_ctx *const *ctxs, int n, const std::vector<ShardVecs> &V, double &out)
{
    for (int r = 0; r < n; ++r) {
        DeviceGuard dg(ctxs[r]->device);
        LQCD_CUDA(cudaMemcpyAsync(ctxs[r]->h_pinned_d, V[r].part + V[r].nb, sizeof(double), cudaMemcpyDeviceToHost,
                                  ctxs[r]->stream));
    }
    double s = 0.0;
    for (int r = 0; r < n; ++r) {
        DeviceGuard dg(ctxs[r]->device);
        LQCD_CUDA(cudaStreamSynchronize(ctxs[r]->stream));
        s += ctxs[r]->h_pinned_d[0];
    }
    out = s;
    return LQCD_OK;
}

static void rank_sum(lqcd_ctx *c, const ShardVecs &V)
{
    k_shard_sum<<<1, kShardThreads, 0, c->stream>>>(V.part, (int)V.nb, V.part + V.nb);
    c->launches += 1;
}

// q = (m^2 + sigma) v - D_eo D_oe v on every rank (two face exchanges), with
// each rank's Re <v, q> total at part[nb].
static int shard_apply_A(lqcd_ctx *const *ctxs, int n, std::vector<ShardVecs> &V, double2 *ShardVecs::*v,
                         double a)
{
    std::vector<void *> f(n);
    for (int r = 0; r < n; ++r) f[r] = V[r].*v;
    if (int st = exchange_faces(ctxs, n, f.data())) return st;
    for (int r = 0; r < n; ++r) {
        lqcd_ctx *c = ctxs[r];
        DeviceGuard dg(c->device);
        const ShardGeom G = shard_geom(c);
        k_shard_deo<<<V[r].nb, kShardThreads, 0, c->stream>>>(c->g, c->lnk_df.as<float4>(), V[r].*v, V[r].t, 1,
                                                               (int)G.lo, (int)G.hi);
        c->launches += 1;
        LQCD_CUDA(cudaGetLastError());
    }
    for (int r = 0; r < n; ++r) f[r] = V[r].t;
    if (int st = exchange_faces(ctxs, n, f.data())) return st;
    for (int r = 0; r < n; ++r) {
        lqcd_ctx *c = ctxs[r];
        DeviceGuard dg(c->device);
        const ShardGeom G = shard_geom(c);
        k_shard_normal<<<V[r].nb, kShardThreads, 0, c->stream>>>(c->g, c->lnk_df.as<float4>(), V[r].t, V[r].*v,
                                                                 V[r].q, a, (int)G.lo, (int)G.hi, V[r].part);
        c->launches += 1;
        rank_sum(c, V[r]);
        LQCD_CUDA(cudaGetLastError());
    }
    return LQCD_OK;
}

// r = b - q on every rank, returning the rank-ordered ||r||^2.
static int shard_residual(lqcd_ctx *const *ctxs, int n, std::vector<ShardVecs> &V, bool with_q, double &rr)
{
    for (int r = 0; r < n; ++r) {
        lqcd_ctx *c = ctxs[r];
        DeviceGuard dg(c->device);
        const ShardGeom G = shard_geom(c);
        k_shard_residual<<<V[r].nb, kShardThreads, 0, c->stream>>>((int)G.vh, V[r].r, V[r].b,
                                                                   with_q ? V[r].q : nullptr, (int)G.lo,
                                                                   (int)G.hi, V[r].part);
        c->launches += 1;
        rank_sum(c, V[r]);
        LQCD_CUDA(cudaGetLastError());
    }
    return ordered_total(ctxs, n, V, rr);
}

static int shard_cg(lqcd_ctx *const *ctxs, int n, double mass, double sigma, double tol, const double *b,
                    double *x, lqcd_solve_info *info)
{
    const long S = (long)ctxs[0]->gdims[0] * ctxs[0]->gdims[1] * ctxs[0]->gdims[2];
    const long h = S / 2;
    const double a = mass * mass + sigma;
    const int max_iter = ctxs[0]->opts.max_iter;
    std::vector<ShardVecs> V(n);
    std::vector<double> host;
    uint64_t launches0 = 0;
    for (int r = 0; r < n; ++r) launches0 += ctxs[r]->launches;
    // scatter: each rank's owned slices of b into its extended slab
    for (int r = 0; r < n; ++r) {
        lqcd_ctx *c = ctxs[r];
        DeviceGuard dg(c->device);
        if (int lr = links_ready(c)) return lr;
        if (int st = shard_vecs(c, V[r])) return st;
        const ShardGeom G = shard_geom(c);
        LQCD_CUDA(cudaMemsetAsync(c->shard_ws.ptr, 0, 6 * 3 * (size_t)G.vh * sizeof(double2), c->stream));
        host.assign((size_t)G.vh * 6, 0.0);
        memcpy(host.data() + (size_t)G.lo * 6, b + (size_t)c->shard_t0 * h * 6,
               (size_t)(G.hi - G.lo) * 6 * sizeof(double));
        if (int st = host_to_soa(c, host.data(), V[r].b, 1, c->stream)) return st;
        LQCD_CUDA(cudaStreamSynchronize(c->stream));
    }
    double rr = 0.0;
    if (int st = shard_residual(ctxs, n, V, false, rr)) return st;  // r = b
    const double bb = rr;
    int it = 0, status = LQCD_OK, restarts = 0;
    double true_res = 0.0;
    if (bb == 0.0) {
        status = LQCD_OK;
    } else {
        const double stop = 0.25 * tol * tol * bb;  // iterate to tol / 2, then check the true residual
        for (;;) {
            // p = r (a start or a restart)
            for (int r = 0; r < n; ++r) {
                lqcd_ctx *c = ctxs[r];
                DeviceGuard dg(c->device);
                const ShardGeom G = shard_geom(c);
                k_shard_xpay<<<V[r].nb, kShardThreads, 0, c->stream>>>((int)G.vh, V[r].p, V[r].r, 0.0, (int)G.lo,
                                                                       (int)G.hi);
                c->launches += 1;
            }
            while (rr > stop) {
                if (it >= max_iter) break;
                double pq = 0.0;
                if (int st = shard_apply_A(ctxs, n, V, &ShardVecs::p, a)) return st;
                if (int st = ordered_total(ctxs, n, V, pq)) return st;
                if (!(pq > 0.0) || !std::isfinite(pq)) return fail(LQCD_ENAN, "sharded CG: <p, A p> is not positive");
                const double alpha = rr / pq;
                for (int r = 0; r < n; ++r) {
                    lqcd_ctx *c = ctxs[r];
                    DeviceGuard dg(c->device);
                    const ShardGeom G = shard_geom(c);
                    k_shard_update_xr<<<V[r].nb, kShardThreads, 0, c->stream>>>(
                        (int)G.vh, V[r].x, V[r].r, V[r].p, V[r].q, alpha, (int)G.lo, (int)G.hi, V[r].part);
                    c->launches += 1;
                    rank_sum(c, V[r]);
                }
                double rr_new = 0.0;
                if (int st = ordered_total(ctxs, n, V, rr_new)) return st;
                const double beta = rr_new / rr;
                rr = rr_new;
                ++it;
                if (rr <= stop) break;
                for (int r = 0; r < n; ++r) {
                    lqcd_ctx *c = ctxs[r];
                    DeviceGuard dg(c->device);
                    const ShardGeom G = shard_geom(c);
                    k_shard_xpay<<<V[r].nb, kShardThreads, 0, c->stream>>>((int)G.vh, V[r].p, V[r].r, beta,
                                                                           (int)G.lo, (int)G.hi);
                    c->launches += 1;
                }
            }
            // FP64 true residual r = b - A x (the sharded operator, rank-ordered sums)
            if (int st = shard_apply_A(ctxs, n, V, &ShardVecs::x, a)) return st;
            if (int st = shard_residual(ctxs, n, V, true, rr)) return st;
            true_res = std::sqrt(rr / bb);
            if (true_res <= tol) break;
            if (it >= max_iter || ++restarts > 3) {
                status = LQCD_ENOCONV;
                break;
            }
        }
    }
    // gather: each rank's owned slices of x into the global array
    for (int r = 0; r < n; ++r) {
        lqcd_ctx *c = ctxs[r];
        DeviceGuard dg(c->device);
        const ShardGeom G = shard_geom(c);
        host.assign((size_t)G.vh * 6, 0.0);
        if (int st = soa_to_host(c, V[r].x, host.data(), 1, c->stream)) return st;
        LQCD_CUDA(cudaStreamSynchronize(c->stream));
        memcpy(x + (size_t)c->shard_t0 * h * 6, host.data() + (size_t)G.lo * 6,
               (size_t)(G.hi - G.lo) * 6 * sizeof(double));
    }
    if (info) {
        uint64_t launches = 0;
        for (int r = 0; r < n; ++r) launches += ctxs[r]->launches;
        info->iters = it;
        info->n_shift = 1;
        info->shift_iters[0] = it;
        info->true_resid[0] = true_res;
        info->status = status;
        info->kernel_launches = (int)(launches - launches0);
    }
    if (status == LQCD_ENOCONV) set_error("sharded CG did not reach tol within max_iter");
    return status;
}

}  // namespace lqcd

extern "C" int lqcd_shard_cg_solve(lqcd_ctx *const *ctxs, int n, double mass, double sigma, double tol,
                                   const double *b, double *x, lqcd_solve_info *info)
{
    NvtxRange nvtx_("lqcd_shard_cg_solve");
    if (int st = check_world(ctxs, n)) return st;
    if (!b || !x) return fail(LQCD_EINVAL, "NULL argument");
    if (!(tol > 0.0) || !std::isfinite(mass) || !(sigma >= 0.0)) return fail(LQCD_EINVAL, "bad mass, sigma or tol");
    LQCD_ON_DEVICE(ctxs[0]->device);
    if (info) memset(info, 0, sizeof *info);
    const auto t0 = std::chrono::steady_clock::now();
    const int st = shard_cg(ctxs, n, mass, sigma, tol, b, x, info);
    if (info) info->secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return st;
}
