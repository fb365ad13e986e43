// mrhs.cu -- multi-right-hand-side D_eo / D_oe in FP32 and the batched CG
// built on it (n_rhs independent single-shift solves of Eq. lineqeo sharing
// one gauge field).
//
// Layout of a batch of n half-lattice fields: complex64 [3][Vh][n] (colour,
// site, right-hand side fastest).  A thread owns one site and R = 4, 2 or 1
// consecutive right-hand sides (G = n / R threads per site, adjacent in the
// warp): the G threads of a site read the same link addresses, which the
// load unit serves once, and every link read from memory is applied to all n
// fields -- the link traffic per site-field falls as 1/n.  12-real links
// rebuild the third row once per thread (shared by its R fields).
//
// Batched CG: FP32 iterations with FP64 reliable updates per right-hand side
// (the FP64 solution, the FP64 true residual and its norm live in IEEE
// complex128 on the device); each field has its own device scalars and stops
// on its own.  The iteration kernels carry per-field reductions with the same
// deterministic tile-ordered scheme as the multi-shift solver.
#include <algorithm>
#include <cstdio>
#include <string>
#include <mutex>
#include <map>
#include <chrono>
#include <cmath>
#include <cstring>
#include <cstdlib>
#include <vector>

#include "solver_kernels.cuh"

namespace lqcd {

constexpr int kMaxRhs = 16;

struct MrhsArgs {
    Geom g;
    const void *links;
    int n, G;             // fields, threads per site
    int P;                // output parity
    const float2 *in;     // [3][Vh][n]
    float2 *out;          // [3][Vh][n]
    // solver epilogue / reductions
    const float2 *p;      // output-parity p for q = a p - D t
    SolverState *st;      // [n]
    double *part;         // [n][ntiles]
    unsigned *ticket;
    int ntiles;
};

// Field (c, site, j) of a batch: site-major [3][Vh][n] (FM = false: the
// fields of a site are contiguous) or field-major [3][n][Vh] (FM = true:
// the sites of a field are contiguous, so consecutive threads read
// consecutive sites).
template <bool FM>
__device__ __forceinline__ size_t mrhs_at(int c, int site, int j, int Vh, int n)
{
    return FM ? ((size_t)c * n + j) * Vh + site : ((size_t)c * Vh + site) * n + j;
}

template <int LF, int R, bool FM = false>
__device__ __forceinline__ void mrhs_site(const MrhsArgs &A, const Stencil &S, int i, int j0, float2 (&acc)[R][3])
{
    const int Vh = A.g.Vh, n = A.n;
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[r][c] = make_float2(0.f, 0.f);
#pragma unroll 1
    for (int mu = 0; mu < 4; ++mu) {
        int f, b;
        uint32_t nf, nb;
        hop(A.g, S, mu, f, b, nf, nb);
#pragma unroll
        for (int dir = 0; dir < 2; ++dir) {
            float2 U[9];
            const int idx = dir == 0 ? f : b;
            const uint32_t ng = dir == 0 ? nf : nb;
            load_link_f32<LF>(A.links, mu, dir == 0 ? A.P : 1 - A.P, dir == 0 ? i : b, Vh, U);
            // fields two at a time in one 16-byte load when R is even (the
            // fields of a site are contiguous, so the G threads of a site
            // read one contiguous run); per field the arithmetic is the same
            constexpr int W = (R % 2 == 0 && !FM) ? 2 : 1;
#pragma unroll
            for (int r = 0; r < R; r += W) {
                float2 v[W][3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float2 *src = A.in + mrhs_at<FM>(c, idx, j0 + r, Vh, n);
                    if constexpr (W == 2) {
                        const float4 t = __ldg(reinterpret_cast<const float4 *>(src));
                        v[0][c] = make_float2(__uint_as_float(__float_as_uint(t.x) ^ ng),
                                              __uint_as_float(__float_as_uint(t.y) ^ ng));
                        v[1][c] = make_float2(__uint_as_float(__float_as_uint(t.z) ^ ng),
                                              __uint_as_float(__float_as_uint(t.w) ^ ng));
                    } else {
                        const float2 t = __ldg(src);
                        v[0][c] = make_float2(__uint_as_float(__float_as_uint(t.x) ^ ng),
                                              __uint_as_float(__float_as_uint(t.y) ^ ng));
                    }
                }
#pragma unroll
                for (int q = 0; q < W; ++q)
#pragma unroll
                    for (int a = 0; a < 3; ++a)
#pragma unroll
                        for (int bb = 0; bb < 3; ++bb) {
                            if (dir == 0) {
                                const float2 u = U[a * 3 + bb];
                                acc[r + q][a].x = __fmaf_rn(u.x, v[q][bb].x, __fmaf_rn(-u.y, v[q][bb].y, acc[r + q][a].x));
                                acc[r + q][a].y = __fmaf_rn(u.x, v[q][bb].y, __fmaf_rn(u.y, v[q][bb].x, acc[r + q][a].y));
                            } else {
                                const float2 u = U[bb * 3 + a];
                                acc[r + q][a].x = __fmaf_rn(u.x, v[q][bb].x, __fmaf_rn(u.y, v[q][bb].y, acc[r + q][a].x));
                                acc[r + q][a].y = __fmaf_rn(u.x, v[q][bb].y, __fmaf_rn(-u.y, v[q][bb].x, acc[r + q][a].y));
                            }
                        }
            }
        }
    }
}

// Plain multi-RHS D (API call and solver K1).
template <int LF, int R>
__global__ void __launch_bounds__(kTile) k_deo_mrhs(const MrhsArgs A)
{
    const long tid = blockIdx.x * (long)kTile + threadIdx.x;
    const int site = (int)(tid / A.G);
    const int grp = (int)(tid - (long)site * A.G);
    if (site >= A.g.Vh) return;
    if (A.st && blockIdx.x == 0 && threadIdx.x < A.n) A.st[threadIdx.x].do_k4 = 0;
    const int j0 = grp * R;
    if (A.st) {  // solver use: fields that have stopped are not recomputed
        bool all = true;
#pragma unroll
        for (int r = 0; r < R; ++r) all &= A.st[j0 + r].halt != HALT_NONE;
        if (all) return;
    }
    Stencil S;
    make_stencil(A.g, site, A.P, S);
    float2 acc[R][3];
    mrhs_site<LF, R>(A, S, site, j0, acc);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float2 *dst = A.out + ((size_t)c * A.g.Vh + site) * A.n + j0;
        if constexpr (R % 2 == 0) {
#pragma unroll
            for (int r = 0; r < R; r += 2)
                *reinterpret_cast<float4 *>(dst + r) = make_float4(0.5f * acc[r][c].x, 0.5f * acc[r][c].y,
                                                                   0.5f * acc[r + 1][c].x, 0.5f * acc[r + 1][c].y);
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) dst[r] = make_float2(0.5f * acc[r][c].x, 0.5f * acc[r][c].y);
        }
    }
}

// Sites per block of the field-major kernel for G (1..16) field groups: the
// block holds every group of its sites, G * sites <= 256 threads.
__host__ __device__ constexpr int mrhs_fm_sites(int G) { return 256 / G; }

// Plain multi-RHS D on field-major batches.  A block takes mrhs_fm_sites(G)
// consecutive sites and all G = n / R groups of R fields: thread t works on
// site t % sites, fields (t / sites) * R ... + R - 1.  The G threads of a
// site are in different warps of the same block, so the link they share is
// read from memory once and served to the other warps from L1; each warp's
// spinor accesses are consecutive sites of one field.  The hop sign is
// applied to the link (18 sign flips per hop, whatever R) instead of to each
// field's spinor; products of a sign-flipped link and a spinor equal those of
// the link and the sign-flipped spinor bit for bit, so every field keeps the
// bits of the single-field operator.
template <int LF, int R>
__global__ void __launch_bounds__(256, R >= 16 ? 1 : 2) k_deo_mrhs_fm(const MrhsArgs A)
{
    const int sites = mrhs_fm_sites(A.G);
    const int grp = threadIdx.x / sites;
    const int site = blockIdx.x * sites + (threadIdx.x - grp * sites);
    if (site >= A.g.Vh) return;
    const int j0 = grp * R, Vh = A.g.Vh, n = A.n;
    Stencil S;
    make_stencil(A.g, site, A.P, S);
    float2 acc[R][3];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[r][c] = make_float2(0.f, 0.f);
#pragma unroll 1
    for (int mu = 0; mu < 4; ++mu) {
        int f, b;
        uint32_t nf, nb;
        hop(A.g, S, mu, f, b, nf, nb);
#pragma unroll
        for (int dir = 0; dir < 2; ++dir) {
            float2 U[9];
            const int idx = dir == 0 ? f : b;
            const uint32_t ng = dir == 0 ? nf : nb;
            load_link_f32<LF>(A.links, mu, dir == 0 ? A.P : 1 - A.P, dir == 0 ? site : b, Vh, U);
#pragma unroll
            for (int k = 0; k < 9; ++k)
                U[k] = make_float2(__uint_as_float(__float_as_uint(U[k].x) ^ ng),
                                   __uint_as_float(__float_as_uint(U[k].y) ^ ng));
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float2 v[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) v[c] = __ldg(A.in + mrhs_at<true>(c, idx, j0 + r, Vh, n));
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int bb = 0; bb < 3; ++bb) {
                        if (dir == 0) {
                            const float2 u = U[a * 3 + bb];
                            acc[r][a].x = __fmaf_rn(u.x, v[bb].x, __fmaf_rn(-u.y, v[bb].y, acc[r][a].x));
                            acc[r][a].y = __fmaf_rn(u.x, v[bb].y, __fmaf_rn(u.y, v[bb].x, acc[r][a].y));
                        } else {
                            const float2 u = U[bb * 3 + a];
                            acc[r][a].x = __fmaf_rn(u.x, v[bb].x, __fmaf_rn(u.y, v[bb].y, acc[r][a].x));
                            acc[r][a].y = __fmaf_rn(u.x, v[bb].y, __fmaf_rn(-u.y, v[bb].x, acc[r][a].y));
                        }
                    }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            A.out[mrhs_at<true>(c, site, j0 + r, Vh, n)] = make_float2(0.5f * acc[r][c].x, 0.5f * acc[r][c].y);
}

// Per-field deterministic block + tile reduction: vals[r] belongs to field
// j0 + r of this thread.  fn(j, total) runs once per field in the last block.
template <int R, class Fn>
__device__ __forceinline__ void mrhs_reduce(const MrhsArgs &A, const double (&vals)[R], int j0, Fn fn)
{
    __shared__ double s_v[kTile * R];
    __shared__ int s_last;
#pragma unroll
    for (int r = 0; r < R; ++r) s_v[threadIdx.x * R + r] = vals[r];
    __syncthreads();
    // field j of this block: threads t with t % G == j / R, slot j % R, in thread order
    if (threadIdx.x < A.n) {
        const int j = threadIdx.x, g = j / R, r = j % R;
        double s = 0.0;
        for (int t = g; t < kTile; t += A.G) s += s_v[t * R + r];
        A.part[(size_t)j * A.ntiles + blockIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(A.ticket, 1u) == (unsigned)(A.ntiles - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // one warp per field, lanes strided over tiles, then a fixed shuffle tree
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = w; j < A.n; j += kTile / 32) {
        double s = 0.0;
        for (int k = lane; k < A.ntiles; k += 32) s += __ldcg(A.part + (size_t)j * A.ntiles + k);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
        if (lane == 0) fn(j, s);
    }
    __syncthreads();
    if (threadIdx.x == 0) *A.ticket = 0u;
}

// K2: q = a p - D_eo t, <p_j, q_j> per field.
template <int LF, int R>
__global__ void __launch_bounds__(kTile) k_mrhs_deo2(const MrhsArgs A)
{
    const long tid = blockIdx.x * (long)kTile + threadIdx.x;
    const int site = (int)(tid / A.G);
    const int grp = (int)(tid - (long)site * A.G);
    const int j0 = grp * R;
    double dots[R];
#pragma unroll
    for (int r = 0; r < R; ++r) dots[r] = 0.0;
    bool live = false;
#pragma unroll
    for (int r = 0; r < R; ++r) live |= A.st[j0 + r].halt == HALT_NONE;
    if (site < A.g.Vh && live) {
        Stencil S;
        make_stencil(A.g, site, 0, S);
        float2 acc[R][3];
        mrhs_site<LF, R>(A, S, site, j0, acc);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const SolverState *st = A.st + j0 + r;
            const float a = st->a0_df.x;
            float d = 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const size_t o = ((size_t)c * A.g.Vh + site) * A.n + j0 + r;
                const float2 pv = A.p[o];
                const float2 qv = make_float2(__fmaf_rn(a, pv.x, -0.5f * acc[r][c].x), __fmaf_rn(a, pv.y, -0.5f * acc[r][c].y));
                A.out[o] = qv;
                d = __fmaf_rn(pv.x, qv.x, __fmaf_rn(pv.y, qv.y, d));
            }
            dots[r] = (double)d;
        }
    }
    mrhs_reduce<R>(A, dots, j0, [&](int j, double tot) {
        if (!A.st[j].halt) finalize_pq(A.st + j, tot);
    });
}

// K3: r -= alpha_j q, ||r_j||^2 (in = q, out = r)
template <int R>
__global__ void __launch_bounds__(kTile) k_mrhs_upd_r(const MrhsArgs A)
{
    const long tid = blockIdx.x * (long)kTile + threadIdx.x;
    const int site = (int)(tid / A.G);
    const int grp = (int)(tid - (long)site * A.G);
    const int j0 = grp * R;
    double nr[R];
#pragma unroll
    for (int r = 0; r < R; ++r) nr[r] = 0.0;
    if (site < A.g.Vh) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const SolverState *st = A.st + j0 + r;
            if (st->halt) continue;
            const float na = -st->alpha_df.x;
            float d = 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const size_t o = ((size_t)c * A.g.Vh + site) * A.n + j0 + r;
                const float2 qv = A.in[o], rv = A.out[o];
                const float2 w = make_float2(__fmaf_rn(na, qv.x, rv.x), __fmaf_rn(na, qv.y, rv.y));
                A.out[o] = w;
                d = __fmaf_rn(w.x, w.x, __fmaf_rn(w.y, w.y, d));
            }
            nr[r] = (double)d;
        }
    }
    mrhs_reduce<R>(A, nr, j0, [&](int j, double tot) {
        if (!A.st[j].halt) finalize_rr(A.st + j, tot);
    });
}

// K4: x_j += alpha_j p_j; p_j = r_j + beta_j p_j (in = r, out = x, p = p)
template <int R>
__global__ void __launch_bounds__(kTile) k_mrhs_upd_xp(const MrhsArgs A, float2 *pvec)
{
    const long tid = blockIdx.x * (long)kTile + threadIdx.x;
    const int site = (int)(tid / A.G);
    const int grp = (int)(tid - (long)site * A.G);
    if (site >= A.g.Vh) return;
    const int j0 = grp * R;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const SolverState *st = A.st + j0 + r;
        if (!st->do_k4) continue;
        const float as = st->alpha_s_df[0].x, bs = st->beta_s_df[0].x;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t o = ((size_t)c * A.g.Vh + site) * A.n + j0 + r;
            const float2 pv = pvec[o], xv = A.out[o], rv = A.in[o];
            A.out[o] = make_float2(__fmaf_rn(as, pv.x, xv.x), __fmaf_rn(as, pv.y, xv.y));
            pvec[o] = make_float2(__fmaf_rn(bs, pv.x, rv.x), __fmaf_rn(bs, pv.y, rv.y));
        }
    }
}

// IEEE [3][Vh] field <-> column j of an interleaved FP32 batch
__global__ void k_col_from_ieee(const double2 *__restrict__ src, float2 *dst, long n3, int n, int j, double scale)
{
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= n3) return;
    const double2 d = src[t];
    dst[t * n + j] = make_float2((float)(d.x * scale), (float)(d.y * scale));
}

__global__ void k_col_to_ieee_add(const float2 *__restrict__ src, double2 *dst, long n3, int n, int j, double scale)
{
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= n3) return;
    const float2 v = src[t * n + j];
    double2 o = dst[t];
    o.x += (double)v.x * scale;
    o.y += (double)v.y * scale;
    dst[t] = o;
}

__global__ void k_col_scale(float2 *v, long n3, int n, int j, float f)
{
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= n3) return;
    float2 a = v[t * n + j];
    v[t * n + j] = make_float2(a.x * f, a.y * f);
}

__global__ void k_col_set(float2 *v, const float2 *src, long n3, int n, int j, int zero)
{
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= n3) return;
    v[t * n + j] = zero ? make_float2(0.f, 0.f) : src[t * n + j];
}

// ------------------------------------------------------------------ launch helpers
static int pick_R(int n) { return (n % 4 == 0) ? 4 : (n % 2 == 0 ? 2 : 1); }

template <int LF>
static void launch_deo_mrhs_R(const MrhsArgs &A, int R, unsigned nb, cudaStream_t s)
{
    if (R == 16) k_deo_mrhs<LF, 16><<<nb, kTile, 0, s>>>(A);
    else if (R == 8) k_deo_mrhs<LF, 8><<<nb, kTile, 0, s>>>(A);
    else if (R == 4) k_deo_mrhs<LF, 4><<<nb, kTile, 0, s>>>(A);
    else if (R == 2) k_deo_mrhs<LF, 2><<<nb, kTile, 0, s>>>(A);
    else k_deo_mrhs<LF, 1><<<nb, kTile, 0, s>>>(A);
}

template <int LF>
static void launch_deo_mrhs_fm_R(const MrhsArgs &A, int R, cudaStream_t s)
{
    // A.G = n / R groups; a block holds all groups of its sites
    const int sites = mrhs_fm_sites(A.G);
    const unsigned grid = (unsigned)((A.g.Vh + sites - 1) / sites), block = (unsigned)(sites * A.G);
    if (R == 16) k_deo_mrhs_fm<LF, 16><<<grid, block, 0, s>>>(A);
    else if (R == 8) k_deo_mrhs_fm<LF, 8><<<grid, block, 0, s>>>(A);
    else if (R == 4) k_deo_mrhs_fm<LF, 4><<<grid, block, 0, s>>>(A);
    else if (R == 2) k_deo_mrhs_fm<LF, 2><<<grid, block, 0, s>>>(A);
    else k_deo_mrhs_fm<LF, 1><<<grid, block, 0, s>>>(A);
}

// layout: 0 site-major, 1 field-major
static void launch_deo_mrhs(const MrhsArgs &A, int lf, int R, unsigned nb, cudaStream_t s, int layout = 0)
{
    if (layout == 1) {
        if (lf == LF_F32_18) launch_deo_mrhs_fm_R<LF_F32_18>(A, R, s);
        else if (lf == LF_F32_12) launch_deo_mrhs_fm_R<LF_F32_12>(A, R, s);
        else launch_deo_mrhs_fm_R<LF_F16_12>(A, R, s);
        return;
    }
    if (lf == LF_F32_18) launch_deo_mrhs_R<LF_F32_18>(A, R, nb, s);
    else if (lf == LF_F32_12) launch_deo_mrhs_R<LF_F32_12>(A, R, nb, s);
    else launch_deo_mrhs_R<LF_F16_12>(A, R, nb, s);
}

template <int LF>
static void launch_deo2_R(const MrhsArgs &A, int R, unsigned nb, cudaStream_t s)
{
    if (R == 4) k_mrhs_deo2<LF, 4><<<nb, kTile, 0, s>>>(A);
    else if (R == 2) k_mrhs_deo2<LF, 2><<<nb, kTile, 0, s>>>(A);
    else k_mrhs_deo2<LF, 1><<<nb, kTile, 0, s>>>(A);
}

// Fields per thread of the stand-alone multi-RHS D_eo, picked per (n, recon,
// lattice) on the first call by timing every R that divides n (1..16) with
// CUDA events on the call's stream; cached for the process.  Each field's
// sum does not depend on R, so every choice gives the same bits.  During
// stream capture the default (4, 2 or 1) is used without tuning.
static std::mutex g_mr_mu;
static std::map<std::string, int> g_mr_tune;

static int mrhs_pick_R(lqcd_ctx *c, MrhsArgs A, int lf, cudaStream_t s, int layout)
{
    // LQCD_MRHS_R=<R> fixes the fields per thread (when R divides n), for
    // tests of every variant and for tuning studies
    if (const char *e = getenv("LQCD_MRHS_R")) {
        const int R = atoi(e);
        if (R >= 1 && R <= 16 && (R & (R - 1)) == 0 && A.n % R == 0) return R;
    }
    char key[96];
    snprintf(key, sizeof key, "n%d lf%d L%d %dx%dx%dx%d", A.n, lf, layout, c->dims[0], c->dims[1], c->dims[2],
             c->dims[3]);
    {
        std::lock_guard<std::mutex> lk(g_mr_mu);
        auto it = g_mr_tune.find(key);
        if (it != g_mr_tune.end()) return it->second;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cap);
    if (cap != cudaStreamCaptureStatusNone) return pick_R(A.n);
    int best_R = pick_R(A.n);
    float best = 1e30f;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return best_R;
    for (int R = 1; R <= 16; R <<= 1) {
        if (A.n % R) continue;
        A.G = A.n / R;
        const unsigned nb = (unsigned)(((long)c->Vh * A.G + kTile - 1) / kTile);
        launch_deo_mrhs(A, lf, R, nb, s, layout);  // warm
        cudaEventRecord(e0, s);
        for (int r = 0; r < 3; ++r) launch_deo_mrhs(A, lf, R, nb, s, layout);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        c->launches += 4;
        if (t < best) {
            best = t;
            best_R = R;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> lk(g_mr_mu);
    g_mr_tune[key] = best_R;
    return best_R;
}

int deo_mrhs_launch(lqcd_ctx *c, int P, int n, int recon, const void *in, void *out, cudaStream_t s, int layout)
{
    if (layout != 0 && layout != 1) return fail(LQCD_EINVAL, "layout must be 0 (site-major) or 1 (field-major)");
    if (int lr = links_ready(c)) return lr;
    if (P != 0 && P != 1) return fail(LQCD_EINVAL, "out_parity must be 0 or 1");
    if (n < 1 || n > kMaxRhs) return fail(LQCD_EINVAL, "n_rhs must be in 1..16");
    if (!in || !out || in == out) return fail(LQCD_EINVAL, "bad spinor pointers");
    if (recon != 18 && recon != 12) return fail(LQCD_EINVAL, "recon must be 18 or 12");
    MrhsArgs A;
    memset(&A, 0, sizeof A);
    A.g = c->g;
    A.links = recon == 18 ? c->lnk_f18.ptr : c->lnk_f12.ptr;
    A.n = n;
    A.P = P;
    A.in = (const float2 *)in;
    A.out = (float2 *)out;
    const int lf = recon == 18 ? LF_F32_18 : LF_F32_12;
    // an even R reads and writes two fields per 16-byte access
    const bool al16 = ((uintptr_t)in % 16 == 0) && ((uintptr_t)out % 16 == 0);
    const int R = (al16 || layout == 1) ? mrhs_pick_R(c, A, lf, s, layout) : 1;
    A.G = n / R;
    const unsigned nb = (unsigned)(((long)c->Vh * A.G + kTile - 1) / kTile);
    launch_deo_mrhs(A, lf, R, nb, s, layout);
    LQCD_CUDA(cudaGetLastError());
    c->launches += 1;
    return LQCD_OK;
}

// ------------------------------------------------------------------ batched CG
// Batched CG core on the device.  n fields (1..16, padded internally to a
// power of two so that the fields of a site never straddle a block), field j
// solves (A + sigma[j]) x_j = b_j with b_j = b + j * b_stride * 3 Vh (stride 0:
// one shared source), starting from the IEEE guess in xh[j] and leaving the
// FP64 solution there.  lf: link storage of the FP32 iterations.
// infos[j] (may be NULL) receive iterations, reliable updates and the FP64
// true residual; bytes accumulates the algorithmic traffic.
int mrhs_cg_core(lqcd_ctx *c, double mass, const double *sigma, int n, double tol, const double2 *b,
                 int b_stride, double2 *xh, int lf, lqcd_solve_info *infos, double &bytes)
{
    const uint64_t l0 = c->launches;
    cudaStream_t s = c->stream;
    const long Vh = (long)c->Vh, n3 = 3 * Vh;
    int np = 1;
    while (np < n) np <<= 1;
    const int R = np >= 4 ? 4 : np, G = np / R;
    const int ntiles = (int)((Vh * G + kTile - 1) / kTile);
    const void *links = lf == LF_F16_12 ? c->lnk_h12.ptr : (lf == LF_F32_12 ? c->lnk_f12.ptr : c->lnk_f18.ptr);
    DevBuf vec, ieee, part, tick, stb;
    int st;
    if ((st = vec.ensure(5 * (size_t)n3 * np * sizeof(float2)))) return st;
    if ((st = ieee.ensure(2 * (size_t)n3 * sizeof(double2)))) return st;
    if ((st = part.ensure(((size_t)np * ntiles + 64) * sizeof(double)))) return st;
    if ((st = tick.ensure(64))) return st;
    if ((st = stb.ensure((size_t)np * sizeof(SolverState)))) return st;
    LQCD_CUDA(cudaMemsetAsync(tick.ptr, 0, 64, s));
    LQCD_CUDA(cudaMemsetAsync(vec.ptr, 0, 5 * (size_t)n3 * np * sizeof(float2), s));
    float2 *r = vec.as<float2>(), *p = r + n3 * np, *x = p + n3 * np, *q = x + n3 * np, *t = q + n3 * np;
    double2 *rh = ieee.as<double2>(), *tn = rh + n3;
    SolverState *sts = stb.as<SolverState>();
    double *partd = part.as<double>(), *res = partd + (size_t)np * ntiles;
    unsigned *tk = tick.as<unsigned>();
    const double2 *Lnat = c->lnk_nat.as<double2>();
    const int nt1 = (int)((Vh + kTile - 1) / kTile);
    const unsigned nb3 = (unsigned)((n3 + 255) / 256);
    auto bj = [&](int j) { return b + (size_t)j * b_stride * n3; };
    auto true_res = [&](int j, double &rr) -> int {
        const double a = mass * mass + sigma[j];
        k_res_nat1_ext(c->g, Lnat, xh + (size_t)j * n3, tn, nt1, s);
        k_res_nat2_ext(c->g, Lnat, tn, xh + (size_t)j * n3, bj(j), a, rh, partd, tk + 1, res, nt1, s);
        LQCD_CUDA(cudaGetLastError());
        c->launches += 2;
        LQCD_CUDA(cudaMemcpyAsync(c->h_pinned_d, res, sizeof(double), cudaMemcpyDeviceToHost, s));
        LQCD_CUDA(cudaStreamSynchronize(s));
        rr = c->h_pinned_d[0];
        return LQCD_OK;
    };
    std::vector<double> b2(np, 0.0), scale(np, 1.0), target2(np, 0.0);
    std::vector<int> done(np, 1), rel(np, 0);
    const double delta = c->opts.delta_reliable;
    // (re)start field j from the IEEE residual in rh: FP32 residual scaled to
    // O(1) entries, x_lo = 0, p kept (rescaled) or set to r
    auto restart = [&](int j, double rr, const SolverState *prev) -> int {
        const double old = scale[j];
        scale[j] = unit_scale_pub(rr, 6.0 * Vh);
        k_col_from_ieee<<<nb3, 256, 0, s>>>(rh, r, n3, np, j, scale[j]);
        k_col_set<<<nb3, 256, 0, s>>>(x, nullptr, n3, np, j, 1);
        if (prev)
            k_col_scale<<<nb3, 256, 0, s>>>(p, n3, np, j, (float)(scale[j] / old));
        else
            k_col_set<<<nb3, 256, 0, s>>>(p, r, n3, np, j, 0);
        LQCD_CUDA(cudaGetLastError());
        c->launches += 3;
        const double rho = rr * scale[j] * scale[j];
        SolverState T;
        if (prev) {
            T = *prev;
            T.halt = HALT_NONE;
            T.do_k4 = 0;
            T.rho = rho;
        } else {
            init_state_pub(T, mass, sigma + j, 1, 1.0, rho, c->opts.max_iter);
        }
        T.tol2_b2 = 0.25 * target2[j] * scale[j] * scale[j];
        T.rel_stop2 = delta * delta * rho;
        LQCD_CUDA(cudaMemcpyAsync(sts + j, &T, sizeof T, cudaMemcpyHostToDevice, s));
        return LQCD_OK;
    };
    SolverState idle;
    memset(&idle, 0, sizeof idle);
    idle.halt = HALT_CONVERGED;
    for (int j = 0; j < np; ++j) LQCD_CUDA(cudaMemcpyAsync(sts + j, &idle, sizeof idle, cudaMemcpyHostToDevice, s));
    for (int j = 0; j < n; ++j) {
        LQCD_CUDA(cudaMemsetAsync(tn, 0, n3 * sizeof(double2), s));
        // ||b_j||^2 from the residual of x = 0 (A applied to zero)
        double2 *xj = xh + (size_t)j * n3;
        {
            const double a = mass * mass + sigma[j];
            k_res_nat2_ext(c->g, Lnat, tn, tn, bj(j), a, nullptr, partd, tk + 1, res, nt1, s);
            LQCD_CUDA(cudaGetLastError());
            LQCD_CUDA(cudaMemcpyAsync(c->h_pinned_d, res, sizeof(double), cudaMemcpyDeviceToHost, s));
            LQCD_CUDA(cudaStreamSynchronize(s));
            b2[j] = c->h_pinned_d[0];
        }
        if (!std::isfinite(b2[j])) return fail(LQCD_ENAN, "source contains NaN/Inf");
        target2[j] = tol * tol * b2[j];
        if (b2[j] == 0.0) {
            LQCD_CUDA(cudaMemsetAsync(xj, 0, n3 * sizeof(double2), s));
            continue;
        }
        double rr;
        if ((st = true_res(j, rr))) return st;
        if (rr <= target2[j]) continue;
        done[j] = 0;
        if ((st = restart(j, rr, nullptr))) return st;
    }
    MrhsArgs A;
    memset(&A, 0, sizeof A);
    A.g = c->g;
    A.links = links;
    A.n = np;
    A.G = G;
    A.st = sts;
    A.part = partd;
    A.ticket = tk;
    A.ntiles = ntiles;
    const unsigned nb = (unsigned)ntiles;
    MrhsArgs A1 = A, A2 = A, A3 = A, A4 = A;
    A1.P = 1; A1.in = p; A1.out = t;
    A2.P = 0; A2.in = t; A2.out = q; A2.p = p;
    A3.in = q; A3.out = r;
    A4.in = r; A4.out = x;
    const int chunk = c->opts.check_every;
    cudaGraphExec_t exec = nullptr;
    {
        cudaGraph_t g;
        LQCD_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        for (int k = 0; k < chunk; ++k) {
            launch_deo_mrhs(A1, lf, R, nb, s);
            if (lf == LF_F32_18) launch_deo2_R<LF_F32_18>(A2, R, nb, s);
            else if (lf == LF_F32_12) launch_deo2_R<LF_F32_12>(A2, R, nb, s);
            else launch_deo2_R<LF_F16_12>(A2, R, nb, s);
            if (R == 4) { k_mrhs_upd_r<4><<<nb, kTile, 0, s>>>(A3); k_mrhs_upd_xp<4><<<nb, kTile, 0, s>>>(A4, p); }
            else if (R == 2) { k_mrhs_upd_r<2><<<nb, kTile, 0, s>>>(A3); k_mrhs_upd_xp<2><<<nb, kTile, 0, s>>>(A4, p); }
            else { k_mrhs_upd_r<1><<<nb, kTile, 0, s>>>(A3); k_mrhs_upd_xp<1><<<nb, kTile, 0, s>>>(A4, p); }
        }
        cudaError_t e = cudaStreamEndCapture(s, &g);
        if (e != cudaSuccess) return cuda_fail(e, "batched CG graph capture");
        e = cudaGraphInstantiate(&exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(e, "batched CG graph instantiate");
    }
    int *hs = c->h_pinned;
    std::vector<SolverState> O(np);
    std::vector<int> iters(np, 0);
    const double link = lf == LF_F16_12 ? 24.0 : (lf == LF_F32_12 ? 48.0 : 72.0);
    int rc = LQCD_OK;
    for (int guard = 0; guard < 1000000 && rc == LQCD_OK; ++guard) {
        bool all = true;
        for (int j = 0; j < n; ++j) all &= done[j] != 0;
        if (all) break;
        const int max_chunks = c->opts.max_iter / chunk + 4;
        int k = 0;
        for (; k < max_chunks; ++k) {
            cudaError_t e = cudaGraphLaunch(exec, s);
            c->launches += 4 * (uint64_t)chunk;
            for (int j = 0; j < n && e == cudaSuccess; ++j)
                e = cudaMemcpyAsync(hs + j, &sts[j].halt, sizeof(int), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "batched CG iteration");
                break;
            }
            bytes += (double)Vh * chunk * (2 * 8 * link + 2 * 2 * 24.0 * np + 24.0 * 8 * np);
            bool any_new = false;
            for (int j = 0; j < n; ++j) any_new |= (!done[j] && hs[j] != HALT_NONE);
            if (any_new) break;
        }
        if (rc) break;
        cudaError_t e = cudaMemcpy(O.data(), sts, (size_t)np * sizeof(SolverState), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) { rc = cuda_fail(e, "batched CG state"); break; }
        bool progressed = false;
        for (int j = 0; j < n && rc == LQCD_OK; ++j) {
            if (done[j] || O[j].halt == HALT_NONE) continue;
            progressed = true;
            iters[j] = O[j].iters;
            if (O[j].halt == HALT_NAN) { rc = fail(LQCD_ENAN, "NaN/Inf or breakdown in the batched CG"); break; }
            k_col_to_ieee_add<<<nb3, 256, 0, s>>>(x, xh + (size_t)j * n3, n3, np, j, 1.0 / scale[j]);
            c->launches += 1;
            double rr;
            if ((rc = true_res(j, rr))) break;
            if (O[j].halt == HALT_MAXITER) { done[j] = 2; continue; }
            if (O[j].halt == HALT_RELIABLE) ++rel[j];
            if (rr <= target2[j]) {
                done[j] = 1;
                SolverState T = O[j];
                T.halt = HALT_CONVERGED;
                e = cudaMemcpyAsync(sts + j, &T, sizeof T, cudaMemcpyHostToDevice, s);
                if (e != cudaSuccess) rc = cuda_fail(e, "batched CG state");
                continue;
            }
            rc = restart(j, rr, &O[j]);
        }
        if (!progressed && rc == LQCD_OK)
            for (int j = 0; j < n; ++j)
                if (!done[j]) done[j] = 2;
    }
    cudaGraphExecDestroy(exec);
    if (rc) return rc;
    int status = LQCD_OK;
    for (int j = 0; j < n; ++j) {
        double rr = 0;
        if (b2[j] > 0 && (st = true_res(j, rr))) return st;
        const double res_j = b2[j] > 0 ? std::sqrt(rr / b2[j]) : 0.0;
        if (!(res_j <= tol)) status = LQCD_ENOCONV;
        if (infos) {
            lqcd_solve_info &I = infos[j];
            I.n_shift = 1;
            I.iters = iters[j];
            I.shift_iters[0] = iters[j];
            I.true_resid[0] = res_j;
            I.reliable_updates = rel[j];
            I.status = res_j <= tol ? LQCD_OK : LQCD_ENOCONV;
            I.kernel_launches = (int)(c->launches - l0);
        }
    }
    return status;
}

int cg_solve_mrhs(lqcd_ctx *c, double mass, double sigma, int n, double tol, const double *b_host, double *x_host,
                  lqcd_solve_info *info)
{
    const auto t0 = std::chrono::steady_clock::now();
    if (int lr = links_ready(c)) return lr;
    if (n < 1 || n > kMaxRhs) return fail(LQCD_EINVAL, "n_rhs must be in 1..16");
    if (!b_host || !x_host) return fail(LQCD_EINVAL, "NULL argument");
    if (!(tol > 0) || !(sigma >= 0) || !std::isfinite(sigma) || !std::isfinite(mass) || !(mass * mass + sigma > 0))
        return fail(LQCD_EINVAL, "need tol > 0, sigma >= 0 and m^2 + sigma > 0");
    cudaStream_t s = c->stream;
    const size_t n3 = 3 * c->Vh;
    DevBuf bd, xd;
    int st;
    if ((st = bd.ensure((size_t)n * n3 * sizeof(double2))) || (st = xd.ensure((size_t)n * n3 * sizeof(double2))))
        return st;
    if ((st = host_to_soa(c, b_host, bd.as<double2>(), n, s))) return st;
    LQCD_CUDA(cudaMemsetAsync(xd.ptr, 0, (size_t)n * n3 * sizeof(double2), s));
    std::vector<double> sig(n, sigma);
    std::vector<lqcd_solve_info> I(n);
    memset(I.data(), 0, n * sizeof(lqcd_solve_info));
    double bytes = 0;
    const int lf = c->opts.prec == LQCD_PREC_FP16 ? LF_F16_12 : (c->opts.recon == 12 ? LF_F32_12 : LF_F32_18);
    const int rc = mrhs_cg_core(c, mass, sig.data(), n, tol, bd.as<double2>(), 1, xd.as<double2>(), lf, I.data(), bytes);
    if (rc != LQCD_OK && rc != LQCD_ENOCONV) return rc;
    if ((st = soa_to_host(c, xd.as<double2>(), x_host, n, s))) return st;
    LQCD_CUDA(cudaStreamSynchronize(s));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info)
        for (int j = 0; j < n; ++j) {
            info[j] = I[j];
            info[j].secs = secs;
            info[j].bytes_moved = bytes / n;
        }
    if (rc == LQCD_ENOCONV) set_error("batched CG did not reach tol within max_iter");
    return rc;
}

}  // namespace lqcd
