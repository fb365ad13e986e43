// internal.h -- host-side structures shared by the translation units of
// liblqcd (not part of the public C ABI, which is include/lqcd.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/lqcd.h"
#include "common.cuh"
#include "iteration.h"

namespace lqcd {

// NVTX range over a library call (header-only NVTX v3: a no-op unless a
// profiler is attached), so that ncu --nvtx filters and timelines can name
// the calls.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};


// Makes `dev` the calling thread's current device for the lifetime of the
// guard and restores the previous one afterwards, so that a context created on
// one device is driven on that device whichever device the calling thread has
// current.  ok is false when the switch failed.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        int cur = -1;
        if (cudaGetDevice(&cur) != cudaSuccess) {
            cudaGetLastError();
            cur = -1;
        }
        if (cur == dev) return;
        if (cudaSetDevice(dev) != cudaSuccess) {
            cudaGetLastError();
            ok = false;
            return;
        }
        prev = cur;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
    DeviceGuard(const DeviceGuard &) = delete;
    DeviceGuard &operator=(const DeviceGuard &) = delete;
};

// Every C entry point that receives a context (or a server) opens one of
// these right after its NULL check.
#define LQCD_ON_DEVICE(dev)                                                               \
    ::lqcd::DeviceGuard lqcd_device_guard_(dev);                                          \
    if (!lqcd_device_guard_.ok)                                                           \
        return ::lqcd::fail(LQCD_ECUDA, "cannot make the context's device current")

// ------------------------------------------------------------------ errors
void set_error(const std::string &msg);
int fail(int status, const std::string &msg);  // sets the message, returns status
int cuda_fail(cudaError_t e, const char *what);

#define LQCD_CUDA(call)                                                     \
    do {                                                                    \
        cudaError_t _e = (call);                                            \
        if (_e != cudaSuccess) return ::lqcd::cuda_fail(_e, #call);         \
    } while (0)

// ------------------------------------------------------------------ device buffer
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
    int ensure(size_t n);  // grow (contents dropped); LQCD_OK / LQCD_ENOMEM
    void release();
    template <class T> T *as() const { return (T *)ptr; }
};

// ------------------------------------------------------------------ context
struct Workspace {
    int prec = -1;          // VecPrec of the Krylov vectors
    int n_shift = 0;
    DevBuf vec;             // r, q, t, x[n], ps[n]
    DevBuf ieee;            // b, r_hi, x_hi[n] (complex128 SoA), tmp
    DevBuf part;            // partial sums
    DevBuf tickets;
    DevBuf state;           // SolverState
    DevBuf stage;           // host-format staging
    uint64_t gen = 0;       // bumped on every reallocation (graph cache key)
    void release()
    {
        vec.release(); ieee.release(); part.release(); tickets.release(); state.release(); stage.release();
    }
    size_t bytes() const { return vec.bytes + ieee.bytes + part.bytes + tickets.bytes + state.bytes + stage.bytes; }
};

struct WsPtrs {
    void *r, *q, *t, *x, *ps;
    double2 *r_hi;
    double2 *t_nat;
    double *part;
    unsigned *ticket;   // [0] iteration kernels, [1] helpers
    SolverState *st;
    double *scal;       // helper reduction outputs (device doubles)
    int ntiles;         // tiles of the iteration kernels
    int ntiles256;      // tiles (blocks) of the 256-thread helper kernels
};

// Instantiated iteration-chunk graphs of a context, keyed by a hash of the
// launch parameters (pointers included); least recently used is replaced.
struct GraphCache {
    static constexpr int kEntries = 4;
    uint64_t key[kEntries] = {~0ull, ~0ull, ~0ull, ~0ull};
    cudaGraphExec_t exec[kEntries] = {};
    uint64_t used[kEntries] = {};
    uint64_t tick = 0;
    cudaGraphExec_t find(uint64_t k);
    void put(uint64_t k, cudaGraphExec_t e);
    void reset();
};

}  // namespace lqcd

struct lqcd_ctx {
    int device = 0;
    int dims[4];
    lqcd::Geom g;
    size_t V = 0, Vh = 0;
    lqcd_opts opts;
    cudaStream_t stream = nullptr;
    bool links_ok = false;
    // link storage (see deo_core.cuh for the layouts)
    lqcd::DevBuf lnk_df;    // df64 pairs, 18 reals: [4][2][9][Vh] float4
    lqcd::DevBuf lnk_nat;   // IEEE, 18 reals:       [4][2][9][Vh] double2
    lqcd::DevBuf lnk_f18;   // FP32, 18 reals:       [4][2][9][Vh] float2
    lqcd::DevBuf lnk_f12;   // FP32, 12 reals:       [4][2][3][Vh] float4
    lqcd::DevBuf lnk_h12;   // FP16, 12 reals:       [8][Vh] uint4 + [8][Vh] uint2
    lqcd::DevBuf lnk_dfs;   // df64 pairs, tile-ordered stream of the staged kernels:
                            //   [2 parities][ntiles][8 hops][9][256] float4 (stencil_staged.cuh)
    lqcd::DevBuf err_word;  // device status word of the stand-alone staged D_eo (bit set = stall)
    lqcd::DevBuf io_a, io_b;  // device staging of host spinors for where = 0
    lqcd::DevBuf rat_x;       // shifted solutions of a rational application [n][3][Vh] double2
    lqcd::DevBuf rat_part;    // per-block partials of its action (+ the total)
    // gauge molecular dynamics (gauge.cu): momenta as 8 reals per link, SoA [4][2][8][Vh]
    lqcd::DevBuf mom64, mom32;
    lqcd::DevBuf md_part;     // partials of the action / kinetic energy (+ the total)
    lqcd::DevBuf stout_lv;    // stout levels 0 .. n-1 (level 0 = the thin links), IEEE SoA each; level n is lnk_nat
    lqcd::DevBuf stout_M, stout_G;  // force chain scratch: U^dag L and the link's own gradient terms, per link
    lqcd::DevBuf stout_F;     // two forces on the links, 8 reals each ([2][4][2][8][Vh] double)
    int stout_n = 0;          // active stout levels (0: the links in use are the uploaded ones)
    double stout_rho = 0.0;
    lqcd::DevBuf host_b, host_x;  // device copies of b and x of the host multi-shift call
    lqcd::DevBuf ff_y;        // D_oe x_i of the fermion force [n][3][Vh] double2
    int md_links_newest = 0;  // LQCD_PREC_FP64: lnk_nat holds the newest links; FP32: lnk_f18
    bool links_derived_stale = false;  // MD moved the links: derived formats need a rebuild
    bool df_stale = false;    // the df64 link copy lags the IEEE master (double-float MD reads it)
    int mom_newest = 0;       // which momentum copy is current
    lqcd::Workspace ws;
    lqcd::Workspace ws32;                  // FP32 phase of a hybrid mixed-precision solve
    std::vector<lqcd::Workspace> ref_ws;   // per-shift refinement jobs
    lqcd::GraphCache graph;
    int *h_pinned = nullptr;  // pinned host words for halt/iteration polling
    double *h_pinned_d = nullptr;
    uint64_t launches = 0;    // library kernels launched on behalf of this context
    // t-slab shard of a global lattice (shard.cu); shard_world = 0: not a shard
    int shard_world = 0, shard_rank = 0, shard_t0 = 0, shard_nt = 0;
    int gdims[4] = {0, 0, 0, 0};  // global lattice of a shard (dims is its extended slab)
    lqcd::DevBuf shard_ws;        // sharded CG vectors and partial sums
};

namespace lqcd {

size_t ctx_device_bytes(const lqcd_ctx *c);

// deo.cu
__global__ void k_aos_to_soa(const double2 *__restrict__ a, double2 *__restrict__ s, long Vh, int nf);
__global__ void k_soa_to_aos(const double2 *__restrict__ s, double2 *__restrict__ a, long Vh, int nf);
__global__ void k_deo_df_ieee(Geom g, const float4 *__restrict__ L, const double2 *__restrict__ in,
                              double2 *__restrict__ out, int P);
int deo_launch(lqcd_ctx *c, int out_parity, int prec, int recon, const void *in, void *out, cudaStream_t s);
int upload_links(lqcd_ctx *c, const double *host, size_t n);
// Staged kernels: shared-memory attribute and residency, once per device.
// Returns true when they can run on the current device.
bool staged_deo_ready();
int stage_wait_selftest(lqcd_ctx *c, double limit_s);
bool staged_solver_ready();
int persist_blocks();   // grid of the persistent K2 / K3 reduction kernels on this device (0: one block per tile)
bool staged_active(const lqcd_ctx *c);   // staged option on and the staged link stream built
// LQCD_ESTATE before an upload; otherwise makes every link format current
// after molecular-dynamics updates (FP32 copy promoted, formats rebuilt).
int links_ready(lqcd_ctx *c);
// LQCD_ETIMEOUT (and clears the word) if a stand-alone staged D_eo of this
// context recorded a stall; synchronises the context's stream.
int deo_check_stall(lqcd_ctx *c);
int download_links(lqcd_ctx *c, double *host, size_t n);
int host_to_soa(lqcd_ctx *c, const double *host, double2 *dev_soa, int nfields, cudaStream_t s);
int soa_to_host(lqcd_ctx *c, const double2 *dev_soa, double *host, int nfields, cudaStream_t s);

// solver.cu
int mscg_solve_dev(lqcd_ctx *c, double mass, const double *shifts, int n_shift, double tol, const double2 *b,
                   double2 *x, lqcd_solve_info *info, cudaStream_t s);
int profile_iteration(lqcd_ctx *c, double mass, const double *shifts, int n_shift, double tol, const double2 *b,
                      int iters, double ms[4], double *n_act_avg);
// One multi-shift solve in flight (single, packed or served).
struct JobRun {
    lqcd_ctx *c = nullptr;
    WsPtrs P;
    int vp = 0, lf = 0;
    const void *links = nullptr;
    double mass = 0, tol = 0;
    double shifts[kMaxShifts];
    int n_shift = 0;
    const double2 *b = nullptr;   // IEEE device source [3][Vh]
    double2 *x = nullptr;         // IEEE device solutions [n][3][Vh]
    double b2 = 0, scale = 1, bytes = 0;
    bool zero = false;
    bool warm = false;            // x holds an initial guess (single shift, FP32 engine)
    double switch_rel = 0;        // double-float phase of a hybrid solve: halt at ||r|| <= this * ||b||
    int iters0 = 0;               // iterations done by an earlier phase (byte accounting)
    uint64_t launches0 = 0;
    lqcd_solve_info I;
};
int validate_solve(const lqcd_ctx *c, double mass, const double *shifts, int n_shift, double tol);
int ensure_workspace_in(lqcd_ctx *c, Workspace &W, int vp, int n_shift, WsPtrs &P);
int job_init(JobRun &J, lqcd_ctx *c, Workspace *W, double mass, const double *shifts, int n_shift, double tol,
             const double2 *b, double2 *x);
int job_init_prec(JobRun &J, lqcd_ctx *c, Workspace *W, int prec, double mass, const double *shifts, int n_shift,
                  double tol, const double2 *b, double2 *x);
int job_setup(JobRun &J, cudaStream_t s);
int job_reliable_update(JobRun &J, cudaStream_t s);
int job_switch_to_f32(JobRun &D, JobRun &F, cudaStream_t s);
int validate_opts(const lqcd_opts *o);
void job_fill(const JobRun &J, IterJob &out);
int job_finish(JobRun &J, cudaStream_t s);
// One iteration of a packed batch; pdl: programmatic dependent launches,
// chained: the previous launch on s is the batch's previous iteration.
void launch_iteration_packed(const IterBatch<kMaxJobs> &B, int vp, int lf, cudaStream_t s, bool pdl, bool chained);
int run_packed_until_halt(lqcd_ctx *c, const IterBatch<kMaxJobs> &B, int vp, int lf, cudaStream_t s);
int mscg_solve_packed(lqcd_ctx *const *ctxs, int n, const double *mass, const double *const *shifts,
                      const int *n_shift, const double *tol, const double *const *b, double *const *x,
                      lqcd_solve_info *info);

// helpers shared by solver.cu and mrhs.cu
void k_res_nat1_ext(const Geom &g, const double2 *L, const double2 *x, double2 *t, int ntiles, cudaStream_t s);
void k_res_nat2_ext(const Geom &g, const double2 *L, const double2 *t, const double2 *x, const double2 *b, double a,
                    double2 *r_hi, double *part, unsigned *ticket, double *out, int ntiles, cudaStream_t s);
double unit_scale_pub(double n2, double n);
void init_state_pub(SolverState &S, double mass, const double *shifts, int n_shift, double tol_iter, double b2,
                    int max_iter);

// rational.cu: y = a0 b + sum_i a_i (A + sigma_i)^{-1} b on device buffers; the
// shifted solutions stay in c->rat_x.
int rational_apply_dev(lqcd_ctx *c, double mass, double a0, const double *a, const double *shifts, int n_shift,
                       double tol, const double2 *b, double2 *y, double *action, lqcd_solve_info *info,
                       cudaStream_t s_user);

// mrhs.cu
int deo_mrhs_launch(lqcd_ctx *c, int out_parity, int n_rhs, int recon, const void *in, void *out, cudaStream_t s,
                    int layout = 0);
int cg_solve_mrhs(lqcd_ctx *c, double mass, double sigma, int n_rhs, double tol, const double *b, double *x,
                  lqcd_solve_info *info);
int mrhs_cg_core(lqcd_ctx *c, double mass, const double *sigma, int n, double tol, const double2 *b, int b_stride,
                 double2 *xh, int lf, lqcd_solve_info *infos, double &bytes);

}  // namespace lqcd
