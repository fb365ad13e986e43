// solver_persist.cuh -- persistent forms of the reduction kernels of the
// multi-shift CG iteration (Sec. 2.2, Eqs. lineqeo and shlineq):
//   K2  q = (m^2 + sigma_b) p - D_eo t and <p, q>, alpha / zeta finaliser
//       (FP32 and FP16 iterations; the double-float K2 is the staged kernel);
//   K3  r -= alpha q and ||r||^2, beta / convergence finaliser (every
//       precision).
//
// k_it_deo2 / k_it_upd_r launch one block per tile. Every block ends with a
// fence and an atomic ticket, and the last block forms the total. In the
// FP32 iteration that fixed cost is a large part of the kernels: K2 took
// 44.8 us against 30.1 us for K1 at 32^4 under ncu, with only 12.6 MB more
// to read. Here a grid of resident blocks walks the tiles gt = blockIdx.x,
// blockIdx.x + gridDim.x, ... .
// - Each tile's partial is a plain store.
// - After its last tile, a block takes one ticket per job it worked on.
// - The block that completes a job's tile count sums the partials in tile
//   order and runs the finaliser.
// Within a block, K2 loads p before the stencil and K3 loads the next
// tile's r and q before the current tile's reduction, so that the loads
// land under work instead of behind the tile's barrier.
// The per-site arithmetic and the in-tile reduction are those of the
// one-block-per-tile kernels, so the tile partials, their tile-ordered sum
// and the iteration are bitwise the same.
#pragma once

#include "solver_kernels.cuh"

namespace lqcd {

constexpr int kF32PersistMinBlocks = 4;  // resident blocks per SM asked of the compiler

// Tail of a persistent reduction kernel. Thread 0 takes one ticket per job
// the block worked on (sh.cnt), after one fence. For every job whose tile
// count this block completes, the block sums the tile partials in tile
// order (the order of tile_finish_block) and warp 0 runs fin(state, total).
template <int NJ, class Fin>
__device__ __forceinline__ void persist_finish(K2Shared &sh, const IterBatch<NJ> &B, Fin fin)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
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
    __syncthreads();
    unsigned long long last = sh.last;
    while (last) {
        const int j = __ffsll((long long)last) - 1;
        last &= last - 1ull;
        const IterJob &J = B.job[j];
        // partials in tile order (the order of tile_finish_block)
        __threadfence();
        double sum = sum_strided(J.part, J.ntiles, (int)threadIdx.x, kIterThreads);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xFFFFFFFFu, sum, o);
        if (lane == 0) sh.red[0][w] = sum;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tot = 0.0;
            for (int k = 0; k < kIterThreads / 32; ++k) tot += sh.red[0][k];
            sh.tot = tot;
            *J.ticket = 0u;
        }
        __syncthreads();
        if (threadIdx.x < 32) fin(J.st, sh.tot);
        __threadfence();
        __syncthreads();
    }
}

template <int NJ, int LF>
__global__ void __launch_bounds__(kIterThreads, kF32PersistMinBlocks)
    k_it_deo2_f32p(const __grid_constant__ IterBatch<NJ> B, int ntot)
{
    static_assert(kIterThreads == kStagedConsumers, "K2Shared holds one slot per warp of a 256-thread block");
    static_assert(kMaxJobs <= 64, "job mask is 64 bits");
    __shared__ K2Shared sh;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    dep_wait();
    dep_launch();
    if (threadIdx.x < NJ) sh.cnt[threadIdx.x] = 0u;
    __syncthreads();
    int nb = 0;
    for (int gt = (int)blockIdx.x; gt < ntot; gt += gridDim.x) {
        int j, tile;
        tile_of(B, gt, j, tile);
        const IterJob &J = B.job[j];
        SolverState *st = J.st;
        if (st->halt) continue;  // the same for every thread of the block
        const int Vh = J.g.Vh;
        const int i = tile * kSites + threadIdx.x;
        Acc2 dot;
        acc_zero(dot);
        if (i < Vh) {
            Stencil S;
            make_stencil(J.g, i, 0, S);
            // p of the epilogue, loaded before the stencil (its latency is
            // spent under the hops)
            const float2 *p = (const float2 *)J.ps + (size_t)st->base * 3 * Vh;
            float2 pp[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) pp[c] = p[(size_t)c * Vh + i];
            float2 o[3];
            deo_site_f32<LF>(J.g, J.links, (const float2 *)J.t, S, i, 0, Vh, o);
            float2 *q = (float2 *)J.q;
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
        // tile partial in the order of block_reduce_acc_n<256>.  The warp
        // sums alternate between two buffers: thread 0 has read buffer b
        // before it reaches the barrier of the next tile, which every warp
        // passes before it writes b again.
        const int b = nb & 1;
        warp_reduce_acc(dot);
        if (lane == 0) sh.red[b][w] = (double)dot.s + (double)dot.c;
        __syncthreads();
        if (threadIdx.x == 0) {
            double v = 0.0;
#pragma unroll
            for (int k = 0; k < kIterThreads / 32; ++k) v += sh.red[b][k];
            J.part[tile] = v;
            sh.cnt[j] += 1u;
        }
        ++nb;
    }
    persist_finish(sh, B, [](SolverState *st, double tot) { finalize_pq_warp(st, tot); });
}

// K3: r -= alpha q, ||r||^2 per tile, then beta and the convergence tests
// (finalize_rr_warp) in the block that completes the job.  The per-site
// arithmetic is that of k_it_upd_r.
template <int NJ, int VP>
__global__ void __launch_bounds__(kIterThreads, kF32PersistMinBlocks)
    k_it_upd_r_p(const __grid_constant__ IterBatch<NJ> B, int ntot)
{
    using T = typename VecT<VP>::T;
    __shared__ K2Shared sh;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    dep_wait();
    dep_launch();
    if (threadIdx.x < NJ) sh.cnt[threadIdx.x] = 0u;
    __syncthreads();
    // The block's tiles of live jobs; each tile's r and q are loaded while
    // the previous tile's norm is reduced.
    auto next_live = [&](int gt) -> int {
        for (; gt < ntot; gt += gridDim.x) {
            int j, tile;
            tile_of(B, gt, j, tile);
            if (!B.job[j].st->halt) return gt;
        }
        return -1;
    };
    T rc[3], qc[3];
    auto load_rq = [&](int gt) {
        int j, tile;
        tile_of(B, gt, j, tile);
        const IterJob &J = B.job[j];
        const int Vh = J.g.Vh;
        const int i = tile * kSites + threadIdx.x;
        if (i >= Vh) return;
        const T *r = (const T *)J.r, *q = (const T *)J.q;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            rc[c] = r[(size_t)c * Vh + i];
            qc[c] = q[(size_t)c * Vh + i];
        }
    };
    int nb = 0;
    int gt = next_live((int)blockIdx.x);
    if (gt >= 0) load_rq(gt);
    while (gt >= 0) {
        int j, tile;
        tile_of(B, gt, j, tile);
        const IterJob &J = B.job[j];
        SolverState *st = J.st;
        const int Vh = J.g.Vh;
        const int i = tile * kSites + threadIdx.x;
        Acc2 nrm;
        acc_zero(nrm);
        if (i < Vh) {
            T *r = (T *)J.r;
            if constexpr (VP == VP_DF) {
                const float2 na = df_neg(st->alpha_df);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float4 rv = rc[c], qv = qc[c];
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
                    const float2 rv = rc[c], qv = qc[c];
                    const float2 v = make_float2(__fmaf_rn(na, qv.x, rv.x), __fmaf_rn(na, qv.y, rv.y));
                    r[(size_t)c * Vh + i] = v;
                    d = __fmaf_rn(v.x, v.x, __fmaf_rn(v.y, v.y, d));
                }
                nrm.s = d;
            }
        }
        const int gn = next_live(gt + (int)gridDim.x);
        if (gn >= 0) load_rq(gn);
        const int b = nb & 1;  // double-buffered warp sums, as in k_it_deo2_f32p
        warp_reduce_acc(nrm);
        if (lane == 0) sh.red[b][w] = (double)nrm.s + (double)nrm.c;
        __syncthreads();
        if (threadIdx.x == 0) {
            double v = 0.0;
#pragma unroll
            for (int k = 0; k < kIterThreads / 32; ++k) v += sh.red[b][k];
            J.part[tile] = v;
            sh.cnt[j] += 1u;
        }
        ++nb;
        gt = gn;
    }
    persist_finish(sh, B, [](SolverState *st, double tot) { finalize_rr_warp(st, tot); });
}

}  // namespace lqcd
