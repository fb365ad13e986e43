// solver_kernels.cuh -- iteration kernels of the multi-shift CG (Sec. 2.2,
// Eqs. lineqeo and shlineq) for df64 ("FP64") and FP32 Krylov vectors.
//
// One iteration = four launches, each tiled over every job of the batch
// (a job = one lattice / one request with its own device scalars):
//   K1  t = D_oe p                                   (deo, odd output)
//   K2  q = (m^2 + sigma_b) p - D_eo t, <p, q>      (deo + fused epilogue);
//       the last tile to finish computes alpha and the shifted zeta_i,
//       alpha_i (one thread, FP64)
//   K3  r -= alpha q, ||r||^2; last tile: beta, beta_i, convergence per shift
//   K4  for every active shift: x_i += alpha_i p_i; p_i = zeta_i r + beta_i p_i
// The base direction p is the direction of the smallest shift (its zeta is 1).
// Reductions are deterministic: per-thread df64 partials, fixed-order warp
// and block trees, per-tile doubles summed in tile order by the last block
// (ticket counter), so a job's result does not depend on what else is in the
// batch.
#pragma once

#include "deo_core.cuh"
#include "internal.h"
#include "stencil_staged.cuh"

namespace lqcd {

// Block -> job.  Contiguous batches give each job a range of blocks;
// interleaved batches (jobs on one lattice) give block b to job b % njobs,
// so that the jobs' blocks reading the same links run next to each other
// and share them through L2.
template <int NJ>
__device__ __forceinline__ int find_job(const IterBatch<NJ> &B)
{
    int j = 0;
    if (NJ > 1) {
        if (B.interleave) return (int)(blockIdx.x % (unsigned)B.njobs);
#pragma unroll 1
        while (j + 1 < B.njobs && (int)blockIdx.x >= B.tile_start[j + 1]) ++j;
    }
    return j;
}

template <int NJ>
__device__ __forceinline__ int job_tile(const IterBatch<NJ> &B, int j)
{
    if (NJ > 1 && B.interleave) return (int)(blockIdx.x / (unsigned)B.njobs);
    return (int)blockIdx.x - B.tile_start[j];
}

// s = (((0 + part[k0]) + part[k0 + d]) + part[k0 + 2d]) ..., k < n: the loads
// go out eight at a time, so the sum waits on one round trip per eight
// partials instead of one per partial; the order of the additions, and so
// the result, is that of the plain strided loop.
__device__ __forceinline__ double sum_strided(const double *part, int n, int k0, int d)
{
    double s = 0.0;
    int k = k0;
    for (; k + 7 * d < n; k += 8 * d) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldcg(part + k + u * d);
#pragma unroll
        for (int u = 0; u < 8; ++u) s += v[u];
    }
    for (; k < n; k += d) s += __ldcg(part + k);
    return s;
}

// Sum per-tile partials in tile order and hand the total to fn (thread 0 of
// the last block to finish).  Every block of the reduction must call this.
template <class Fn>
__device__ __forceinline__ void reduce_finish(double *part, unsigned *ticket, int ntiles, int tile, double v, Fn fn)
{
    // blockDim.x is a multiple of 32 and at most 1024
    __shared__ int s_last;
    __shared__ double s_red[32];
    if (threadIdx.x == 0) {
        part[tile] = v;
        __threadfence();
        const unsigned prev = atomicAdd(ticket, 1u);
        s_last = (prev == (unsigned)(ntiles - 1));
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double s = sum_strided(part, ntiles, (int)threadIdx.x, (int)blockDim.x);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        const int nw = blockDim.x >> 5;
        for (int k = 0; k < nw; ++k) tot += s_red[k];
        fn(tot);
        *ticket = 0u;
        __threadfence();
    }
}

template <class Fn>
__device__ __forceinline__ void tile_finish(const IterJob &J, int tile, double v, Fn fn)
{
    reduce_finish(J.part, J.ticket, J.ntiles, tile, v, fn);
}

// As reduce_finish, but every thread of the last block calls fn(total), so
// that the finaliser can spread per-shift work over the block.
template <class Fn>
__device__ __forceinline__ void reduce_finish_block(double *part, unsigned *ticket, int n, int idx, double v, Fn fn)
{
    __shared__ int s_last;
    __shared__ double s_red[32];
    __shared__ double s_tot;
    if (threadIdx.x == 0) {
        part[idx] = v;
        __threadfence();
        const unsigned prev = atomicAdd(ticket, 1u);
        s_last = (prev == (unsigned)(n - 1));
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double s = sum_strided(part, n, (int)threadIdx.x, (int)blockDim.x);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        const int nw = blockDim.x >> 5;
        for (int k = 0; k < nw; ++k) tot += s_red[k];
        s_tot = tot;
        *ticket = 0u;
    }
    __syncthreads();
    fn(s_tot);
    __threadfence();
}

template <class Fn>
__device__ __forceinline__ void tile_finish_block(const IterJob &J, int tile, double v, Fn fn)
{
    reduce_finish_block(J.part, J.ticket, J.ntiles, tile, v, fn);
}

__device__ __forceinline__ float2 split_scalar(double d)
{
    const float h = __double2float_rn(d);
    return make_float2(h, __double2float_rn(d - (double)h));
}

// alpha and the shifted coefficients (FP64, one thread).
__device__ inline void finalize_pq(SolverState *st, double pq)
{
    st->last_sum = pq;
    st->alpha_prev = st->alpha;
    st->beta_prev = st->beta;
    int n_act = 0;
    for (int s = 0; s < st->n_shift; ++s) {
        if (!st->active_next[s]) continue;
        st->zeta_prev[s] = st->zeta[s];
        st->zeta[s] = st->zeta_new[s];
        st->act_list[n_act++] = s;
    }
    st->n_act = n_act;
    const double alpha = st->rho / pq;
    if (!(pq > 0.0) || !isfinite(alpha)) {
        st->halt = HALT_NAN;
        st->nan_flag = 1;
        return;
    }
    st->alpha = alpha;
    st->alpha_df = split_scalar(alpha);
    for (int k = 0; k < n_act; ++k) {
        const int s = st->act_list[k];
        const double z = st->zeta[s], zp = st->zeta_prev[s];
        const double den = alpha * st->beta_prev * (zp - z) + zp * st->alpha_prev * (1.0 + st->shift_rel[s] * alpha);
        const double zn = z * zp * st->alpha_prev / den;
        st->zeta_new[s] = zn;
        st->zeta_new_df[s] = split_scalar(zn);
        st->alpha_s_df[s] = split_scalar(alpha * zn / z);
    }
}

// finalize_pq on one warp, lane s = shift s (kMaxShifts == 32): every lane
// loads its shift's scalars at once, the active list is compacted with a
// ballot, and the recurrences of all shifts are updated in parallel.  Called
// by warp 0 of the last block.
static_assert(kMaxShifts == 32, "one lane per shift");
__device__ inline void finalize_pq_warp(SolverState *st, double pq)
{
    const int lane = threadIdx.x & 31;
    const int ns = st->n_shift;
    const double rho = st->rho, alpha_old = st->alpha, beta_old = st->beta;
    // every lane loads its shift's slots (kMaxShifts == 32) in one round trip
    const int act = (lane < ns) ? st->active_next[lane] : 0;
    const double zo = st->zeta[lane], zc = st->zeta_new[lane], srel = st->shift_rel[lane];
    const unsigned m = __ballot_sync(0xFFFFFFFFu, act);
    const double alpha = rho / pq;
    const bool ok = (pq > 0.0) && isfinite(alpha);
    if (lane == 0) {
        st->last_sum = pq;
        st->alpha_prev = alpha_old;
        st->beta_prev = beta_old;
        st->n_act = __popc(m);
        if (ok) {
            st->alpha = alpha;
            st->alpha_df = split_scalar(alpha);
        } else {
            st->halt = HALT_NAN;
            st->nan_flag = 1;
        }
    }
    if (!act) return;
    // rotate: zeta_prev <- zeta, zeta <- zeta_new
    st->zeta_prev[lane] = zo;
    st->zeta[lane] = zc;
    st->act_list[__popc(m & ((1u << lane) - 1u))] = lane;
    if (!ok) return;
    const double den = alpha * beta_old * (zo - zc) + zo * alpha_old * (1.0 + srel * alpha);
    const double zn = zc * zo * alpha_old / den;
    st->zeta_new[lane] = zn;
    st->zeta_new_df[lane] = split_scalar(zn);
    st->alpha_s_df[lane] = split_scalar(alpha * zn / zc);
}

// finalize_rr on one warp: lane k handles the k-th active shift (beta_i and
// the convergence test); lane 0 the base scalars and the halt decision.
// Called by warp 0 of the last block.
__device__ inline void finalize_rr_warp(SolverState *st, double rr)
{
    const int lane = threadIdx.x & 31;
    const bool ok = isfinite(rr);
    const double beta = rr / st->rho;
    const int iters = st->iters + 1;
    const int n_act = st->n_act;
    const double tol2_b2 = st->tol2_b2;
    // loaded up front so that lane 0's decisions wait on no further round trip
    const int base = st->base, max_iter = st->max_iter;
    const double rel_stop2 = st->rel_stop2;
    // lane l loads slot l of every per-shift array; lane k of the active list
    // takes shift s = act_list[k]'s values by shuffle (one round trip)
    const int s = st->act_list[lane] & (kMaxShifts - 1);
    const double zc_l = st->zeta[lane], zn_l = st->zeta_new[lane];
    const int it_l = st->shift_iters[lane];
    const double zc = __shfl_sync(0xFFFFFFFFu, zc_l, s);
    const double zn = __shfl_sync(0xFFFFFFFFu, zn_l, s);
    const int its = __shfl_sync(0xFFFFFFFFu, it_l, s);
    int open = 0;
    if (ok && lane < n_act) {
        const double ratio = zn / zc;
        st->beta_s_df[s] = split_scalar(beta * ratio * ratio);
        const bool conv = zn * zn * rr <= tol2_b2;
        if (conv && its == 0) st->shift_iters[s] = iters;
        st->active_next[s] = conv ? 0 : 1;
        open = !conv;
    }
    const int any = __any_sync(0xFFFFFFFFu, open);
    __syncwarp();
    if (lane != 0) return;
    st->last_sum = rr;
    if (st->stall) {  // a staged stencil of this iteration gave up waiting
        st->halt = HALT_STALL;
        return;
    }
    if (!ok) {
        st->halt = HALT_NAN;
        st->nan_flag = 1;
        return;
    }
    st->beta = beta;
    st->rho = rr;
    st->iters = iters;
    // the base direction must keep moving while any shift still iterates
    if (any) st->active_next[base] = 1;
    st->do_k4 = 1;
    if (!any)
        st->halt = HALT_CONVERGED;
    else if (rel_stop2 > 0.0 && rr < rel_stop2)
        st->halt = HALT_RELIABLE;
    else if (iters >= max_iter)
        st->halt = HALT_MAXITER;
}

// beta, beta_i and the stopping decisions (FP64, one thread).
__device__ inline void finalize_rr(SolverState *st, double rr)
{
    st->last_sum = rr;
    if (st->stall) {
        st->halt = HALT_STALL;
        return;
    }
    if (!isfinite(rr)) {
        st->halt = HALT_NAN;
        st->nan_flag = 1;
        return;
    }
    const double beta = rr / st->rho;
    st->beta = beta;
    st->rho = rr;
    st->iters += 1;
    int any = 0;
    for (int k = 0; k < st->n_act; ++k) {
        const int s = st->act_list[k];
        const double ratio = st->zeta_new[s] / st->zeta[s];
        st->beta_s_df[s] = split_scalar(beta * ratio * ratio);
        const double zn = st->zeta_new[s];
        const bool conv = zn * zn * rr <= st->tol2_b2;
        if (conv && st->shift_iters[s] == 0) st->shift_iters[s] = st->iters;
        st->active_next[s] = conv ? 0 : 1;
        any |= !conv;
    }
    // the base direction must keep moving while any shift still iterates
    if (any) st->active_next[st->base] = 1;
    st->do_k4 = 1;
    if (!any)
        st->halt = HALT_CONVERGED;
    else if (st->rel_stop2 > 0.0 && rr < st->rel_stop2)
        st->halt = HALT_RELIABLE;
    else if (st->iters >= st->max_iter)
        st->halt = HALT_MAXITER;
}

// ------------------------------------------------------------------ vector element helpers
template <int VP> struct VecT;
template <> struct VecT<VP_DF> { using T = float4; };
template <> struct VecT<VP_F32> { using T = float2; };

// ------------------------------------------------------------------ launch shape
// One thread per even site; a tile is kSites consecutive half-lattice sites
// and one block of kIterThreads = kSites threads.  Reductions produce one
// partial per tile, which fixes their order for a given lattice.  Measured
// on the 32^4 15-shift solve: 256-site tiles with 2 blocks per SM beat 128
// (4 or 5 blocks) and 64-site tiles; a thread per (site, colour) was slower
// still (the colour threads re-load the neighbour spinors).
#ifndef LQCD_TILE_SITES
#define LQCD_TILE_SITES 256
#endif
#ifndef LQCD_ITER_MINB
#define LQCD_ITER_MINB 2
#endif
constexpr int kSites = LQCD_TILE_SITES;
constexpr int kIterThreads = kSites;

template <int NT>
__device__ __forceinline__ double block_reduce_acc_n(Acc2 A, double *smem)
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

// Programmatic dependent launch.  The iteration kernels may be launched with
// programmatic stream serialisation: the next kernel of the stream then
// starts while this one drains.  dep_wait() returns once the previous kernel
// has completed and its writes are visible; dep_launch() lets the next
// kernel start.  Every iteration kernel calls dep_launch() only after
// dep_wait(), so the code of a kernel before its dep_wait() (its prologue)
// may read what the kernel two launches back, or any earlier one, wrote, but
// nothing the previous kernel writes; it writes nothing.  Prologue loads
// bypass L1 (ld.global.cg).  Without the launch attribute both are no-ops.
__device__ __forceinline__ void dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ------------------------------------------------------------------ K1
template <int NJ, int VP, int LF>
__global__ void __launch_bounds__(kIterThreads, LQCD_ITER_MINB) k_it_deo1(const __grid_constant__ IterBatch<NJ> B)
{
    using T = typename VecT<VP>::T;
    dep_wait();
    dep_launch();
    const int j = find_job(B);
    const IterJob &J = B.job[j];
    SolverState *st = J.st;
    const int tile = job_tile(B, j);
    if (tile == 0 && threadIdx.x == 0) st->do_k4 = 0;
    if (st->halt) return;
    const int Vh = J.g.Vh;
    const int i = tile * kSites + threadIdx.x;
    if (i >= Vh) return;
    const T *p = (const T *)J.ps + (size_t)st->base * 3 * Vh;
    T *t = (T *)J.t;
    Stencil S;
    make_stencil(J.g, i, 1, S);
    if constexpr (VP == VP_DF) {
        float2 res[6];
        bool bad = false;
        deo_site_df<SF_DF>(J.g, (const float4 *)J.links, p, S, i, 1, Vh, res, bad);
#pragma unroll
        for (int c = 0; c < 3; ++c)
            t[(size_t)c * Vh + i] = make_float4(res[2 * c].x, res[2 * c].y, res[2 * c + 1].x, res[2 * c + 1].y);
    } else {
        float2 o[3];
        deo_site_f32<LF>(J.g, J.links, p, S, i, 1, Vh, o);
#pragma unroll
        for (int c = 0; c < 3; ++c) t[(size_t)c * Vh + i] = o[c];
    }
}

// ------------------------------------------------------------------ K2
template <int NJ, int VP, int LF>
__global__ void __launch_bounds__(kIterThreads, LQCD_ITER_MINB) k_it_deo2(const __grid_constant__ IterBatch<NJ> B)
{
    using T = typename VecT<VP>::T;
    __shared__ double s_red[kIterThreads / 32];
    dep_wait();
    dep_launch();
    const int j = find_job(B);
    const IterJob &J = B.job[j];
    SolverState *st = J.st;
    if (st->halt) return;
    const int Vh = J.g.Vh;
    const int tile = job_tile(B, j);
    const int i = tile * kSites + threadIdx.x;
    Acc2 dot;
    acc_zero(dot);
    if (i < Vh) {
        const T *p = (const T *)J.ps + (size_t)st->base * 3 * Vh;
        T *q = (T *)J.q;
        Stencil S;
        make_stencil(J.g, i, 0, S);
        // p of the epilogue, loaded before the stencil (its latency is spent
        // under the hops)
        T pp[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) pp[c] = p[(size_t)c * Vh + i];
        if constexpr (VP == VP_DF) {
            float2 res[6];
            bool bad = false;
            deo_site_df<SF_DF>(J.g, (const float4 *)J.links, J.t, S, i, 0, Vh, res, bad);
            const float2 a = st->a0_df;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float4 pv = pp[c];
                const float2 qr = df_fma(a, make_float2(pv.x, pv.y), df_neg(res[2 * c]));
                const float2 qi = df_fma(a, make_float2(pv.z, pv.w), df_neg(res[2 * c + 1]));
                q[(size_t)c * Vh + i] = make_float4(qr.x, qr.y, qi.x, qi.y);
                acc_prod(dot, pv.x, pv.y, qr.x, qr.y);
                acc_prod(dot, pv.z, pv.w, qi.x, qi.y);
            }
        } else {
            float2 o[3];
            deo_site_f32<LF>(J.g, J.links, (const float2 *)J.t, S, i, 0, Vh, o);
            const float a = st->a0_df.x;
            float d = 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float2 pv = pp[c];
                const float2 qv = make_float2(__fmaf_rn(a, pv.x, -o[c].x), __fmaf_rn(a, pv.y, -o[c].y));
                q[(size_t)c * Vh + i] = qv;
                d = __fmaf_rn(pv.x, qv.x, __fmaf_rn(pv.y, qv.y, d));
            }
            dot.s = d;
        }
    }
    const double v = block_reduce_acc_n<kIterThreads>(dot, s_red);
    tile_finish_block(J, tile, v, [&](double tot) {
        if (threadIdx.x < 32) finalize_pq_warp(st, tot);
    });
}

// ------------------------------------------------------------------ staged K1 / K2 (double-float)
// The two stencil kernels of the FP64 iteration with the link stream staged
// through shared memory (stencil_staged.cuh).  Persistent: block b walks the
// batch's tiles b, b + gridDim.x, ...; the producer lane and the consumers
// walk the same sequence and skip the same halted jobs (a job's halt word
// does not change while its tiles are in flight).  Per-tile results, the
// per-tile partials of <p, q> and the last-tile finaliser are those of
// k_it_deo1 / k_it_deo2, so the iteration is bitwise the same.  No thread
// leaves early: every kernel ends in ring_finish.
template <int NJ>
__device__ __forceinline__ void tile_of(const IterBatch<NJ> &B, int gt, int &j, int &tile)
{
    if (NJ == 1) {
        j = 0;
        tile = gt;
        return;
    }
    if (B.interleave) {
        j = gt % B.njobs;
        tile = gt / B.njobs;
        return;
    }
    int k = 0;
#pragma unroll 1
    while (k + 1 < B.njobs && gt >= B.tile_start[k + 1]) ++k;
    j = k;
    tile = gt - B.tile_start[k];
}

// Producer lane of a staged iteration kernel: tiles of live jobs, in order.
template <int NJ>
__device__ __forceinline__ void staged_iter_produce(RingDF &R, const IterBatch<NJ> &B, int ntot, int P)
{
    int gt = (int)blockIdx.x;
    ring_produce(R, [&](const float4 *&base) -> bool {
        for (; gt < ntot; gt += gridDim.x) {
            int j, tile;
            tile_of(B, gt, j, tile);
            const IterJob &J = B.job[j];
            // prologue read (no dep_wait on this lane): the halt word is
            // written by finalisers at least two launches back
            if (__ldcg(&J.st->halt)) continue;
            base = staged_tile_base(J.links_st, P, J.ntiles, tile);
            gt += gridDim.x;
            return true;
        }
        return false;
    });
}

// Consumers of K1: t = D_oe p on the tiles of this block.
template <int NJ>
__device__ __forceinline__ void k1_staged_consume(RingDF &R, const IterBatch<NJ> &B, int ntot)
{
    dep_wait();
    dep_launch();
    uint32_t q = 0;
    bool dead = false;
    for (int gt = (int)blockIdx.x; gt < ntot; gt += gridDim.x) {
        int j, tile;
        tile_of(B, gt, j, tile);
        const IterJob &J = B.job[j];
        SolverState *st = J.st;
        if (tile == 0 && threadIdx.x == 0) st->do_k4 = 0;
        if (st->halt) continue;
        const int Vh = J.g.Vh;
        const int i = tile * kSites + threadIdx.x;
        const bool live = i < Vh;
        const float4 *p = (const float4 *)J.ps + (size_t)st->base * 3 * Vh;
        Stencil S;
        make_stencil(J.g, live ? i : 0, 1, S);
        float2 res[6];
        bool bad = false;
        deo_site_df_staged<SF_DF>(R, q, dead, J.g, p, S, Vh, res, bad);
        if (dead) st->stall = 1;
        if (!live) continue;
        float4 *t = (float4 *)J.t;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            t[(size_t)c * Vh + i] = make_float4(res[2 * c].x, res[2 * c].y, res[2 * c + 1].x, res[2 * c + 1].y);
    }
}

// Consumers of K2: q = a p - D_eo t and the tile partials of <p, q>; after
// its last tile, the block that completes a job's tile count forms the
// tile-ordered total and runs the alpha / zeta finaliser.  The tile partials
// are plain stores; one fence and one ticket per job and block, after the
// block's last tile, publish them, so no tile waits on a fence.
struct K2Shared {
    double red[2][kStagedConsumers / 32];
    double tot;
    unsigned cnt[kMaxJobs];
    unsigned long long last;
};

template <int NJ>
__device__ __forceinline__ void k2_staged_consume(RingDF &R, K2Shared &sh, const IterBatch<NJ> &B, int ntot)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    static_assert(kMaxJobs <= 64, "job mask is 64 bits");
    dep_wait();
    dep_launch();
    if (threadIdx.x < NJ) sh.cnt[threadIdx.x] = 0u;
    consumer_sync();
    uint32_t q = 0;
    bool dead = false;
    int nb = 0;
    for (int gt = (int)blockIdx.x; gt < ntot; gt += gridDim.x) {
        int j, tile;
        tile_of(B, gt, j, tile);
        const IterJob &J = B.job[j];
        SolverState *st = J.st;
        if (st->halt) continue;
        const int Vh = J.g.Vh;
        const int i = tile * kSites + threadIdx.x;
        const bool live = i < Vh;
        Stencil S;
        make_stencil(J.g, live ? i : 0, 0, S);
        // p of the epilogue, loaded before the stencil so that its latency
        // is spent under the eight hops
        float4 pp[3];
        if (live) {
            const float4 *p = (const float4 *)J.ps + (size_t)st->base * 3 * Vh;
#pragma unroll
            for (int c = 0; c < 3; ++c) pp[c] = p[(size_t)c * Vh + i];
        }
        float2 res[6];
        bool bad = false;
        deo_site_df_staged<SF_DF>(R, q, dead, J.g, J.t, S, Vh, res, bad);
        if (dead) st->stall = 1;
        Acc2 dot;
        acc_zero(dot);
        if (live) {
            float4 *qv = (float4 *)J.q;
            const float2 a = st->a0_df;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float4 pv = pp[c];
                const float2 qr = df_fma(a, make_float2(pv.x, pv.y), df_neg(res[2 * c]));
                const float2 qi = df_fma(a, make_float2(pv.z, pv.w), df_neg(res[2 * c + 1]));
                qv[(size_t)c * Vh + i] = make_float4(qr.x, qr.y, qi.x, qi.y);
                acc_prod(dot, pv.x, pv.y, qr.x, qr.y);
                acc_prod(dot, pv.z, pv.w, qi.x, qi.y);
            }
        }
        // tile partial: the order of block_reduce_acc_n<256>.  The warp sums
        // alternate between two buffers: thread 0 has read buffer b before it
        // reaches the barrier of the next tile, which every warp passes before
        // it writes b again.
        const int b = nb & 1;
        warp_reduce_acc(dot);
        if (lane == 0) sh.red[b][w] = (double)dot.s + (double)dot.c;
        consumer_sync();
        if (threadIdx.x == 0) {
            double v = 0.0;
#pragma unroll
            for (int k = 0; k < kStagedConsumers / 32; ++k) v += sh.red[b][k];
            J.part[tile] = v;
            sh.cnt[j] += 1u;
        }
        ++nb;
    }
    if (threadIdx.x == 0) {
        unsigned long long last = 0ull;
        __threadfence();
        for (int j = 0; j < B.njobs; ++j) {
            const unsigned n = sh.cnt[j];
            if (!n) continue;
            const unsigned prev = atomicAdd(B.job[j].ticket, n);
            if (prev + n == (unsigned)B.job[j].ntiles) last |= 1ull << j;
        }
        sh.last = last;
    }
    consumer_sync();
    unsigned long long last = sh.last;
    while (last) {
        const int j = __ffsll((long long)last) - 1;
        last &= last - 1ull;
        const IterJob &J = B.job[j];
        // partials in tile order (the order of tile_finish_block)
        __threadfence();
        double sum = sum_strided(J.part, J.ntiles, (int)threadIdx.x, kStagedConsumers);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xFFFFFFFFu, sum, o);
        if (lane == 0) sh.red[0][w] = sum;
        consumer_sync();
        if (threadIdx.x == 0) {
            double tot = 0.0;
            for (int k = 0; k < kStagedConsumers / 32; ++k) tot += sh.red[0][k];
            sh.tot = tot;
            *J.ticket = 0u;
        }
        consumer_sync();
        if (threadIdx.x < 32) finalize_pq_warp(J.st, sh.tot);
        __threadfence();
        consumer_sync();
    }
}

template <int NJ>
__global__ void __launch_bounds__(kStagedThreads, kStagedMinBlocks)
    k_it_deo1_st(const __grid_constant__ IterBatch<NJ> B, int ntot)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    RingDF &R = *reinterpret_cast<RingDF *>(smem_raw);
    ring_init(R);
    if (threadIdx.x >= kStagedConsumers) {
        if (threadIdx.x == kStagedConsumers) staged_iter_produce(R, B, ntot, 1);
    } else {
        k1_staged_consume(R, B, ntot);
    }
    ring_finish(R);
}

// The reduction scratch lives in the dynamic allocation after the ring, so
// both staged kernels place their barriers at the same offsets.
template <int NJ>
__global__ void __launch_bounds__(kStagedThreads, kStagedMinBlocks)
    k_it_deo2_st(const __grid_constant__ IterBatch<NJ> B, int ntot)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    RingDF &R = *reinterpret_cast<RingDF *>(smem_raw);
    K2Shared &sh = *reinterpret_cast<K2Shared *>(smem_raw + kRingDFBytes);
    ring_init(R);
    if (threadIdx.x >= kStagedConsumers) {
        if (threadIdx.x == kStagedConsumers) staged_iter_produce(R, B, ntot, 0);
    } else {
        k2_staged_consume(R, sh, B, ntot);
    }
    ring_finish(R);
}

// Dynamic shared memory of the staged iteration kernels.
constexpr size_t kStagedIterSmem = kRingDFBytes + sizeof(K2Shared);

// ------------------------------------------------------------------ K3
template <int NJ, int VP>
__global__ void __launch_bounds__(kIterThreads) k_it_upd_r(const __grid_constant__ IterBatch<NJ> B)
{
    using T = typename VecT<VP>::T;
    __shared__ double s_red[kIterThreads / 32];
    const int j = find_job(B);
    const IterJob &J = B.job[j];
    const int Vh = J.g.Vh;
    const int tile = job_tile(B, j);
    const int i = tile * kSites + threadIdx.x;
    T *r = (T *)J.r;
    // prologue: r was last written by the previous iteration's K3
    T rp[3];
    if (i < Vh) {
#pragma unroll
        for (int c = 0; c < 3; ++c) rp[c] = __ldcg(r + (size_t)c * Vh + i);
    }
    dep_wait();
    dep_launch();
    SolverState *st = J.st;
    if (st->halt) return;
    Acc2 nrm;
    acc_zero(nrm);
    if (i < Vh) {
        const T *q = (const T *)J.q;
        if constexpr (VP == VP_DF) {
            const float2 na = df_neg(st->alpha_df);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float4 rv = rp[c], qv = q[(size_t)c * Vh + i];
                const float2 x = df_fma(na, make_float2(qv.x, qv.y), make_float2(rv.x, rv.y));
                const float2 y = df_fma(na, make_float2(qv.z, qv.w), make_float2(rv.z, rv.w));
                r[(size_t)c * Vh + i] = make_float4(x.x, x.y, y.x, y.y);
                acc_prod(nrm, x.x, x.y, x.x, x.y);
                acc_prod(nrm, y.x, y.y, y.x, y.y);
            }
        } else {
            const float na = -st->alpha_df.x;
            float d = 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float2 rv = rp[c], qv = q[(size_t)c * Vh + i];
                const float2 w = make_float2(__fmaf_rn(na, qv.x, rv.x), __fmaf_rn(na, qv.y, rv.y));
                r[(size_t)c * Vh + i] = w;
                d = __fmaf_rn(w.x, w.x, __fmaf_rn(w.y, w.y, d));
            }
            nrm.s = d;
        }
    }
    const double v = block_reduce_acc_n<kIterThreads>(nrm, s_red);
    tile_finish_block(J, tile, v, [&](double tot) {
        if (threadIdx.x < 32) finalize_rr_warp(st, tot);
    });
}

// ------------------------------------------------------------------ K4
// x_s += alpha_s p_s, p_s = zeta_s r + beta_s p_s for every active shift s.
// One thread per site walks the active list: r is read once per site, the
// scalar chain (do_k4, the active list) is paid once per thread, and the
// next shift's x_s, p_s loads are issued before this shift's stores, so two
// shifts' streams are in flight per thread.  Per element the arithmetic is
// that of one thread per (site, shift).
template <int VP>
struct K4Slot {
    using T = typename VecT<VP>::T;
    T p[3], x[3];
};

template <int VP>
__device__ __forceinline__ void k4_load(K4Slot<VP> &L, const typename VecT<VP>::T *ps, const typename VecT<VP>::T *x,
                                        size_t off, int Vh)
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        L.p[c] = ps[off + (size_t)c * Vh];
        L.x[c] = x[off + (size_t)c * Vh];
    }
}

template <int NJ, int VP>
__global__ void __launch_bounds__(kIterThreads) k_it_upd_shifts(const __grid_constant__ IterBatch<NJ> B)
{
    using T = typename VecT<VP>::T;
    dep_wait();
    dep_launch();
    const int j = find_job(B);
    const IterJob &J = B.job[j];
    const SolverState *st = J.st;
    if (!st->do_k4) return;
    const int n_act = st->n_act;
    const int Vh = J.g.Vh;
    const int i = job_tile(B, j) * kSites + threadIdx.x;
    if (i >= Vh || n_act <= 0) return;
    T *x = (T *)J.x, *ps = (T *)J.ps;
    const T *r = (const T *)J.r;
    T rv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) rv[c] = r[(size_t)c * Vh + i];
    int s = st->act_list[0];
    K4Slot<VP> cur;
    k4_load<VP>(cur, ps, x, (size_t)s * 3 * Vh + i, Vh);
#pragma unroll 1
    for (int k = 0; k < n_act; ++k) {
        const size_t off = (size_t)s * 3 * Vh + i;
        K4Slot<VP> nxt;
        int sn = s;
        if (k + 1 < n_act) {
            sn = st->act_list[k + 1];
            k4_load<VP>(nxt, ps, x, (size_t)sn * 3 * Vh + i, Vh);
        }
        if constexpr (VP == VP_DF) {
            const float2 as = st->alpha_s_df[s], zn = st->zeta_new_df[s], bs = st->beta_s_df[s];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float4 pv = cur.p[c], xv = cur.x[c];
                const float2 xr = df_fma(as, make_float2(pv.x, pv.y), make_float2(xv.x, xv.y));
                const float2 xi = df_fma(as, make_float2(pv.z, pv.w), make_float2(xv.z, xv.w));
                const float2 pr = df_mul2(zn, make_float2(rv[c].x, rv[c].y), bs, make_float2(pv.x, pv.y));
                const float2 pi = df_mul2(zn, make_float2(rv[c].z, rv[c].w), bs, make_float2(pv.z, pv.w));
                x[off + (size_t)c * Vh] = make_float4(xr.x, xr.y, xi.x, xi.y);
                ps[off + (size_t)c * Vh] = make_float4(pr.x, pr.y, pi.x, pi.y);
            }
        } else {
            const float as = st->alpha_s_df[s].x, zn = st->zeta_new_df[s].x, bs = st->beta_s_df[s].x;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float2 pv = cur.p[c], xv = cur.x[c];
                x[off + (size_t)c * Vh] = make_float2(__fmaf_rn(as, pv.x, xv.x), __fmaf_rn(as, pv.y, xv.y));
                ps[off + (size_t)c * Vh] =
                    make_float2(__fmaf_rn(zn, rv[c].x, bs * pv.x), __fmaf_rn(zn, rv[c].y, bs * pv.y));
            }
        }
        cur = nxt;
        s = sn;
    }
}

}  // namespace lqcd
