// stencil_staged.cuh -- the FP64 (double-float) staggered hopping term with
// the link stream staged through shared memory by bulk asynchronous copies
// (Sec. 2.2, Eq. diracblock; the operator is that of deo_core.cuh).
//
// Why: one D_eo application reads 8 links x 144 B per output site and only
// 48 B of neighbour spinors that mostly hit L2.  With one thread per site and
// ~100 registers, the per-thread loads cannot keep enough link bytes in
// flight to cover HBM latency (16 warps per SM).  Here one producer lane per
// block streams whole tiles of links into a ring of shared-memory stages with
// cp.async.bulk while the 8 consumer warps compute, so the bytes in flight no
// longer depend on registers.
//
// Link layout of the staged stream (built once at upload from the SoA
// arrays): for output parity P, tile T of 256 consecutive half-lattice sites
// and hop h = 2 mu + dir (dir 0: forward link U_mu(n); dir 1: backward link
// U_mu(n - mu), stored at the OUTPUT site n), the 9 components of the 256
// sites form one contiguous stage of 9 x 256 float4 = 36 KB:
//     links_st[((P * ntiles + T) * 8 + h) * 9 * 256 + c * 256 + s]
// Every link appears twice (once as a forward, once as a backward link), so
// the stream is twice the SoA size, and every stage is one bulk copy.  Tail
// sites beyond V/2 are zero padding.
//
// Block: 256 consumer threads (one site each) + one producer warp (lane 0
// issues the copies).  Persistent: a block walks tiles blockIdx.x,
// blockIdx.x + gridDim.x, ... and the producer runs up to kStagedStages hops
// ahead, across tile boundaries.  The hop order and the arithmetic are those
// of deo_site_df, so results are bitwise identical to the per-thread kernels.
//
// Every wait is bounded (bulk.cuh).  A consumer whose wait runs out records
// the stall, stops waiting and still runs every barrier, so the block ends;
// the producer waits (bounded) for each copy it issued, and the block
// invalidates its barriers before it exits (ring_finish).
#pragma once

#include "bulk.cuh"
#include "deo_core.cuh"

namespace lqcd {

constexpr int kStagedConsumers = kTile;            // one consumer thread per site of a tile
constexpr int kStagedThreads = kTile + 32;         // + the producer warp
constexpr int kStagedStages = 3;                   // ring depth, in hops
constexpr int kStagedMinBlocks = 2;                // resident blocks per SM (shared memory bound)
constexpr int kDFComps = 9;
constexpr uint32_t kDFStageElems = kDFComps * kTile;
constexpr uint32_t kDFStageBytes = kDFStageElems * (uint32_t)sizeof(float4);  // 36864

struct RingDF {
    float4 U[kStagedStages][kDFComps][kTile];
    uint64_t full[kStagedStages];   // producer -> consumers: stage loaded (transaction bytes)
    uint64_t empty[kStagedStages];  // consumers -> producer: stage read (one arrival per consumer warp)
    int stalled;                    // a bounded wait ran out in this block
};
constexpr size_t kRingDFBytes = sizeof(RingDF);

// Elements of the staged stream of one context (both parities).
__host__ __device__ __forceinline__ size_t staged_df_elems(int ntiles)
{
    return (size_t)2 * (size_t)ntiles * 8 * kDFStageElems;
}

__device__ __forceinline__ const float4 *staged_tile_base(const float4 *links_st, int P, int ntiles, int tile)
{
    return links_st + (size_t)(bound_index(P, 2) * ntiles + bound_index(tile, ntiles)) * 8 * kDFStageElems;
}

// barrier of the 256 consumer threads only (named barrier 1)
__device__ __forceinline__ void consumer_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(kStagedConsumers) : "memory");
}

// Called by all threads of the block before the role split.
__device__ __forceinline__ void ring_init(RingDF &R)
{
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStagedStages; ++s) {
            mbar_init(&R.full[s], 1);
            mbar_init(&R.empty[s], kStagedConsumers / 32);
        }
        R.stalled = 0;
        mbar_fence_init();
    }
    __syncthreads();
}

// Called by all threads of the block after the roles end (no thread may
// leave a staged kernel early): every copy has landed (the producer drained
// them) and every arrival is done, so the barriers can be invalidated.  An
// mbarrier left valid in shared memory that the next block on the SM uses
// for data is undefined behaviour.
__device__ __forceinline__ void ring_finish(RingDF &R)
{
    __syncthreads();
    if (threadIdx.x == 0)
        for (int s = 0; s < kStagedStages; ++s) {
            mbar_inval(&R.full[s]);
            mbar_inval(&R.empty[s]);
        }
}

// Bytes of one hop's stage: all nine link components (RECON 18), or the
// first two rows, components 0..5, which lead each hop block of the stream
// (RECON 12: 24 KB, the third row is rebuilt by the consumers).
template <int RECON>
__host__ __device__ constexpr uint32_t staged_stage_bytes()
{
    return (RECON == 12 ? 6u : 9u) * (uint32_t)kTile * (uint32_t)sizeof(float4);
}

// Producer (one lane).  next(base) yields the tile bases of this block in
// the order the consumers walk them, and false at the end.  Returns false if
// a wait for a free stage ran out.
template <int RECON = 18, class Next>
__device__ __forceinline__ bool ring_produce(RingDF &R, Next next)
{
    const uint64_t pol = bulk_evict_first_policy();
    uint32_t q = 0;
    bool ok = true;
    const float4 *base;
    while (ok && next(base)) {
        for (int h = 0; h < 8; ++h, ++q) {
            const uint32_t s = q % kStagedStages;
            if (q >= (uint32_t)kStagedStages &&
                !mbar_wait(&R.empty[s], ((q / kStagedStages) + 1u) & 1u, kStageWaitNs)) {
                ok = false;
                break;
            }
            mbar_arrive_expect_tx(&R.full[s], staged_stage_bytes<RECON>());
            bulk_g2s(&R.U[s][0][0], base + (size_t)h * kDFStageElems, staged_stage_bytes<RECON>(), &R.full[s], pol);
        }
    }
    // every copy issued must have landed before the block may exit
    const uint32_t first = q > (uint32_t)kStagedStages ? q - kStagedStages : 0u;
    for (uint32_t k = first; k < q; ++k) mbar_wait(&R.full[k % kStagedStages], (k / kStagedStages) & 1u, kStageWaitNs);
    return ok;
}

// Consumer side: wait for stage q (all consumer threads, live or not).
__device__ __forceinline__ int ring_acquire(RingDF &R, uint32_t q, bool &dead)
{
    const int s = (int)(q % kStagedStages);
    if (!dead && !mbar_wait(&R.full[s], (q / kStagedStages) & 1u, kStageWaitNs)) {
        dead = true;
        R.stalled = 1;
    }
    return s;
}

// Consumer side: this warp is done with stage s.  Called only after the
// values read from the stage have been used by the arithmetic, and after a
// proxy fence: the next bulk copy rewrites the stage through the async
// proxy, and the warp's generic-proxy reads must be ordered before it.
// (Releasing straight after the shared-memory loads let a later copy land
// under reads still in flight: a few wrong link elements per thousand
// launches at 48^4, measured; with this order none were seen.)
__device__ __forceinline__ void ring_release(RingDF &R, int s)
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(&R.empty[s]);
}

// D at one site with links from the ring: same hop order and arithmetic as
// deo_site_df.  q is the block's running stage counter (8 stages per tile).
// Every consumer thread calls this once per tile (i is any valid site for
// threads beyond V/2; their result is discarded).
template <int SF, int RECON = 18>
__device__ __forceinline__ void deo_site_df_staged(RingDF &R, uint32_t &q, bool &dead, const Geom &g, const void *in,
                                                   const Stencil &S, int Vh, float2 (&res)[6], bool &bad)
{
    Acc2 acc[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) acc_zero(acc[k]);
    const int t = threadIdx.x;
    // The neighbour spinor of the next half-hop is loaded before the current
    // half-hop is computed, so its L2 latency overlaps the arithmetic (the
    // stage release, a memory barrier for the compiler, would otherwise keep
    // every gather behind the previous hop).
    int f, b;
    uint32_t nf, nb;
    hop(g, S, 0, f, b, nf, nb);
    float4 vf[3], vb[3];
    load_spinor_df<SF>(in, f, Vh, nf, vf, bad);
#pragma unroll 1
    for (int mu = 0; mu < 4; ++mu) {
        float4 U[9];
        float ch[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        load_spinor_df<SF>(in, b, Vh, nb, vb, bad);
        int s = ring_acquire(R, q++, dead);
#pragma unroll
        for (int c = 0; c < (RECON == 12 ? 6 : 9); ++c) U[c] = R.U[s][c][t];
        if (RECON == 12) reconstruct_row2_df(U);
        hop_fwd_df(acc, ch, U, vf);
        ring_release(R, s);
        if (mu < 3) {
            hop(g, S, mu + 1, f, b, nf, nb);
            load_spinor_df<SF>(in, f, Vh, nf, vf, bad);
        }
        s = ring_acquire(R, q++, dead);
#pragma unroll
        for (int c = 0; c < (RECON == 12 ? 6 : 9); ++c) U[c] = R.U[s][c][t];
        if (RECON == 12) reconstruct_row2_df(U);
        hop_bwd_df(acc, ch, U, vb);
        ring_release(R, s);
#pragma unroll
        for (int k = 0; k < 6; ++k) acc_flush(acc[k], ch[k]);
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const float2 r = acc_result(acc[k]);
        res[k] = make_float2(0.5f * r.x, 0.5f * r.y);
    }
}

}  // namespace lqcd
