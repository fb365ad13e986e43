// iteration.h -- device-visible structures of the multi-shift iteration
// (the scalars of one solve and the per-launch job table), shared by the
// iteration kernels and their host drivers.
#pragma once

#include <cstdint>

#include "common.cuh"

namespace lqcd {

// ------------------------------------------------------------------ solver state
// Device-resident scalars of one Krylov solve (one job).  Written by the
// host at set-up, then only by the one-thread finalisers of the iteration
// kernels, so an iteration needs no host round trip.
struct SolverState {
    // set-up (host)
    int n_shift, base, max_iter, halt;
    int iters, do_k4, n_act, nan_flag;
    double a0;                        // m^2 + sigma_base
    double tol2_b2;                   // (tol * ||b||)^2, iterated stopping rule
    double rel_stop2;                 // reliable update when rho < this (0 = off)
    double shift_rel[kMaxShifts];     // sigma_i - sigma_base
    // recurrences (device)
    double rho, alpha, alpha_prev, beta, beta_prev;
    double zeta[kMaxShifts], zeta_prev[kMaxShifts], zeta_new[kMaxShifts];
    int active_next[kMaxShifts];
    int act_list[kMaxShifts];
    int shift_iters[kMaxShifts];
    double last_sum;                  // last reduction result (diagnostics)
    int stall;                        // a staged stencil wait ran out (turned into HALT_STALL)
    // split copies for the vector kernels: df64 (hi, lo) and FP32 (hi only)
    float2 a0_df, alpha_df;
    float2 alpha_s_df[kMaxShifts], zeta_new_df[kMaxShifts], beta_s_df[kMaxShifts];
};

enum Halt { HALT_NONE = 0, HALT_CONVERGED = 1, HALT_RELIABLE = 2, HALT_MAXITER = 3, HALT_NAN = 4, HALT_STALL = 5 };

// Krylov vector precision of an engine
enum VecPrec { VP_DF = 0, VP_F32 = 1 };

// One job (one lattice / request) of a tiled iteration launch.
struct IterJob {
    Geom g;
    const void *links;   // link storage for the engine's deo variant
    const float4 *links_st;  // tile-ordered FP64 link stream of the staged kernels (NULL: per-thread loads)
    void *r, *q, *t;     // residual, A p, odd temporary
    void *x, *ps;        // n_shift solutions / directions, shift-major [n][3][Vh]
    SolverState *st;
    double *part;        // per-tile partial sums
    unsigned *ticket;    // last-block-done counter
    int tile0, ntiles;
};

template <int NJ>
struct IterBatch {
    int njobs;
    int max_shift;              // largest n_shift of the jobs
    int interleave;             // 1: jobs on one lattice, block b belongs to job b % njobs
    int tile_start[NJ + 1];
    IterJob job[NJ];
};

}  // namespace lqcd
