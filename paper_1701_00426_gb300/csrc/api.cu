// api.cu -- the extern "C" entry points declared in include/lqcd.h:
// argument validation, context life cycle, error reporting; the work is
// done by deo.cu, solver.cu, mrhs.cu and serve.cu.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <string>
#include <vector>

#include "internal.h"

namespace lqcd {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

int fail(int status, const std::string &msg)
{
    g_err = msg;
    return status;
}

int cuda_fail(cudaError_t e, const char *what)
{
    g_err = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return e == cudaErrorMemoryAllocation ? LQCD_ENOMEM : LQCD_ECUDA;
}

#ifdef LQCD_CHECK_BOUNDS
// Readers of the translation units' bounds error words (bounds-checked builds).
static std::vector<BoundsReader> &bounds_readers()
{
    static std::vector<BoundsReader> r;
    return r;
}

void register_bounds_reader(BoundsReader f) { bounds_readers().push_back(f); }
#endif

// Host-side fault injection (lqcd_inject_alloc_failure): the k-th device
// allocation from now fails as cudaMalloc would.
static std::atomic<long> g_fail_alloc{0};

int DevBuf::ensure(size_t n)
{
    if (n <= bytes && ptr) return LQCD_OK;
    release();
    if (n == 0) return LQCD_OK;
    if (g_fail_alloc.load() > 0 && g_fail_alloc.fetch_sub(1) == 1)
        return fail(LQCD_ENOMEM, "injected failure of a " + std::to_string(n) + "-byte device allocation");
    cudaError_t e = cudaMalloc(&ptr, n);
    if (e != cudaSuccess) {
        ptr = nullptr;
        bytes = 0;
        cudaGetLastError();
        return fail(LQCD_ENOMEM, "cudaMalloc of " + std::to_string(n) + " bytes failed");
    }
    bytes = n;
    return LQCD_OK;
}

void DevBuf::release()
{
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
}

size_t ctx_device_bytes(const lqcd_ctx *c)
{
    const DevBuf *b[] = {&c->lnk_df, &c->lnk_nat, &c->lnk_f18, &c->lnk_f12, &c->lnk_h12, &c->lnk_dfs,
                         &c->err_word, &c->io_a, &c->io_b, &c->rat_x, &c->rat_part, &c->mom64,
                         &c->mom32, &c->md_part, &c->ff_y, &c->stout_lv, &c->stout_M, &c->stout_G,
                         &c->stout_F, &c->host_b, &c->host_x, &c->ws.vec, &c->ws.ieee, &c->ws.part, &c->ws.tickets, &c->ws.state,
                         &c->ws.stage, &c->shard_ws};
    size_t s = 0;
    for (const DevBuf *p : b) s += p->bytes;
    s += c->ws32.bytes();
    for (const Workspace &w : c->ref_ws) s += w.bytes();
    return s;
}

int validate_opts(const lqcd_opts *o)
{
    if (o->prec < LQCD_PREC_FP64 || o->prec > LQCD_PREC_FP64_NATIVE) return fail(LQCD_EINVAL, "opts.prec out of range");
    if (o->recon != 18 && o->recon != 12) return fail(LQCD_EINVAL, "opts.recon must be 18 or 12");
    if (!(o->delta_reliable > 0.0 && o->delta_reliable < 1.0)) return fail(LQCD_EINVAL, "opts.delta_reliable must be in (0,1)");
    if (o->max_iter < 1) return fail(LQCD_EINVAL, "opts.max_iter must be >= 1");
    if (o->check_every < 1 || o->check_every > 4096) return fail(LQCD_EINVAL, "opts.check_every must be in 1..4096");
    if (!(o->fp64_until >= 0.0 && o->fp64_until < 1.0)) return fail(LQCD_EINVAL, "opts.fp64_until must be in [0,1)");
    if (o->staged != 0 && o->staged != 1) return fail(LQCD_EINVAL, "opts.staged must be 0 or 1");
    if (o->pdl != 0 && o->pdl != 1) return fail(LQCD_EINVAL, "opts.pdl must be 0 or 1");
    return LQCD_OK;
}

// Issue-rate probe: every thread runs 8 independent FMA chains of K steps,
// a = a * m + c, so the pipe never waits for a result; the sum is stored only
// when it takes a value it never takes (kept so the chains are not removed).
template <class T>
__global__ void __launch_bounds__(256) k_fma_rate(int K, T m, T c, T *sink)
{
    T a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
#pragma unroll 8
    for (int it = 0; it < K; ++it)
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fma(a[k], m, c);
    T s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == (T)-1.2345) *sink = s;
}

template <class T>
static int fma_rate(double *out)
{
    int dev = 0, nsm = 0;
    LQCD_CUDA(cudaGetDevice(&dev));
    LQCD_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    DevBuf sink;
    if (int st = sink.ensure(sizeof(double))) return st;
    const unsigned blocks = (unsigned)nsm * 8;
    const int K = 2048;
    cudaEvent_t e0, e1;
    LQCD_CUDA(cudaEventCreate(&e0));
    LQCD_CUDA(cudaEventCreate(&e1));
    k_fma_rate<T><<<blocks, 256>>>(K, (T)0.999, (T)1e-3, sink.as<T>());  // warm
    float best = 1e30f;
    for (int r = 0; r < 5; ++r) {
        cudaEventRecord(e0);
        k_fma_rate<T><<<blocks, 256>>>(K, (T)0.999, (T)1e-3, sink.as<T>());
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    LQCD_CUDA(cudaGetLastError());
    *out = (double)blocks * 256.0 * 8.0 * K / (best * 1e-3);
    return LQCD_OK;
}

}  // namespace lqcd

using namespace lqcd;

extern "C" {

int lqcd_measure_fma_rates(double *fp64_fma_per_s, double *fp32_fma_per_s)
{
    if (!fp64_fma_per_s || !fp32_fma_per_s) return fail(LQCD_EINVAL, "NULL argument");
    if (int st = fma_rate<double>(fp64_fma_per_s)) return st;
    return fma_rate<float>(fp32_fma_per_s);
}

void lqcd_default_opts(lqcd_opts *o)
{
    if (!o) return;
    o->prec = LQCD_PREC_FP64;
    o->recon = 18;
    o->delta_reliable = 0.1;
    o->max_iter = 20000;
    o->check_every = 32;
    o->fp64_until = 3e-4;
    o->staged = 1;
    o->pdl = 0;
}

const char *lqcd_last_error(void) { return g_err.c_str(); }

void lqcd_inject_alloc_failure(long k) { g_fail_alloc.store(k > 0 ? k : 0); }

int lqcd_bounds_errors(unsigned *word)
{
    if (!word) return fail(LQCD_EINVAL, "NULL argument");
#ifdef LQCD_CHECK_BOUNDS
    cudaDeviceSynchronize();
    unsigned w = 0;
    for (BoundsReader f : bounds_readers()) w |= f();
    *word = w;
    return LQCD_OK;
#else
    *word = 0;
    return fail(LQCD_ESTATE, "library built without LQCD_CHECK_BOUNDS");
#endif
}

int lqcd_version(void) { return 100; }

int lqcd_create(const int dims[4], const lqcd_opts *opts, lqcd_ctx **out)
{
    if (!dims || !out) return fail(LQCD_EINVAL, "NULL argument");
    *out = nullptr;
    long V = 1;
    for (int i = 0; i < 4; ++i) {
        if (dims[i] < 2 || (dims[i] & 1)) return fail(LQCD_EINVAL, "lattice sides must be even and >= 2");
        V *= dims[i];
    }
    if (V / 2 > (1l << 30)) return fail(LQCD_EINVAL, "lattice too large (V/2 must be < 2^30)");
    lqcd_opts o;
    lqcd_default_opts(&o);
    if (opts) o = *opts;
    int st = validate_opts(&o);
    if (st) return st;
    lqcd_ctx *c = new (std::nothrow) lqcd_ctx();
    if (!c) return fail(LQCD_ENOMEM, "host allocation failed");
    for (int i = 0; i < 4; ++i) c->dims[i] = dims[i];
    c->g = make_geom(dims);
    c->V = (size_t)V;
    c->Vh = (size_t)V / 2;
    c->opts = o;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaStreamCreate(&c->stream);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&c->h_pinned, 2 * kMaxJobs * sizeof(int), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&c->h_pinned_d, 64 * sizeof(double), cudaHostAllocDefault);
    if (e != cudaSuccess) {
        st = cuda_fail(e, "lqcd_create");
        lqcd_destroy(c);
        return st;
    }
    *out = c;
    return LQCD_OK;
}

void lqcd_destroy(lqcd_ctx *c)
{
    if (!c) return;
    DeviceGuard device_guard(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    c->graph.reset();
    DevBuf *b[] = {&c->lnk_df, &c->lnk_nat, &c->lnk_f18, &c->lnk_f12, &c->lnk_h12, &c->lnk_dfs, &c->err_word,
                   &c->io_a, &c->io_b, &c->rat_x, &c->rat_part, &c->mom64, &c->mom32, &c->md_part, &c->ff_y,
                   &c->stout_lv, &c->stout_M, &c->stout_G, &c->stout_F, &c->host_b, &c->host_x,
                   &c->ws.vec, &c->ws.ieee, &c->ws.part, &c->ws.tickets, &c->ws.state, &c->ws.stage,
                   &c->shard_ws};
    for (DevBuf *p : b) p->release();
    c->ws32.release();
    for (Workspace &w : c->ref_ws) w.release();
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    if (c->h_pinned_d) cudaFreeHost(c->h_pinned_d);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

int lqcd_set_opts(lqcd_ctx *c, const lqcd_opts *o)
{
    if (!c || !o) return fail(LQCD_EINVAL, "NULL argument");
    LQCD_ON_DEVICE(c->device);
    int st = validate_opts(o);
    if (st) return st;
    c->opts = *o;
    return LQCD_OK;
}

size_t lqcd_device_bytes(const lqcd_ctx *c) { return c ? ctx_device_bytes(c) : 0; }

int lqcd_links_upload(lqcd_ctx *c, const double *links, size_t n)
{
    NvtxRange nvtx_("lqcd_links_upload");
    if (!c) return fail(LQCD_EINVAL, "NULL context");
    LQCD_ON_DEVICE(c->device);
    c->graph.reset();
    return upload_links(c, links, n);
}

int lqcd_links_download(lqcd_ctx *c, double *links, size_t n)
{
    if (!c) return fail(LQCD_EINVAL, "NULL context");
    LQCD_ON_DEVICE(c->device);
    return download_links(c, links, n);
}

int lqcd_deo_apply(lqcd_ctx *c, int out_parity, const void *in, void *out, int where, void *stream)
{
    NvtxRange nvtx_("lqcd_deo_apply");
    if (!c) return fail(LQCD_EINVAL, "NULL context");
    LQCD_ON_DEVICE(c->device);
    if (where == 1) return deo_launch(c, out_parity, LQCD_PREC_FP64, 18, in, out, (cudaStream_t)stream ? (cudaStream_t)stream : c->stream);
    if (where != 0) return fail(LQCD_EINVAL, "where must be 0 (host) or 1 (device)");
    if (!in || !out) return fail(LQCD_EINVAL, "NULL spinor pointer");
    if (int lr = links_ready(c)) return lr;
    const size_t bytes = c->Vh * 3 * sizeof(double2);
    DevBuf din, dout;
    int st;
    if ((st = din.ensure(bytes)) || (st = dout.ensure(bytes))) return st;
    cudaStream_t s = c->stream;
    st = host_to_soa(c, (const double *)in, din.as<double2>(), 1, s);
    if (!st) st = deo_launch(c, out_parity, LQCD_PREC_FP64, 18, din.ptr, dout.ptr, s);
    if (!st) st = soa_to_host(c, dout.as<double2>(), (double *)out, 1, s);
    cudaError_t e = cudaStreamSynchronize(s);
    din.release();
    dout.release();
    if (st) return st;
    if (e != cudaSuccess) return cuda_fail(e, "lqcd_deo_apply");
    return deo_check_stall(c);
}

int lqcd_deo_apply_ex(lqcd_ctx *c, int out_parity, int prec, int recon, const void *in, void *out, void *stream)
{
    NvtxRange nvtx_("lqcd_deo_apply_ex");
    if (!c) return fail(LQCD_EINVAL, "NULL context");
    LQCD_ON_DEVICE(c->device);
    return deo_launch(c, out_parity, prec, recon, in, out, stream ? (cudaStream_t)stream : c->stream);
}

int lqcd_deo_apply_mrhs(lqcd_ctx *c, int out_parity, int n_rhs, int recon, const void *in, void *out, void *stream)
{
    NvtxRange nvtx_("lqcd_deo_apply_mrhs");
    if (!c) return fail(LQCD_EINVAL, "NULL context");
    LQCD_ON_DEVICE(c->device);
    return deo_mrhs_launch(c, out_parity, n_rhs, recon, in, out, stream ? (cudaStream_t)stream : c->stream);
}

int lqcd_selftest_stage_wait(lqcd_ctx *c, double limit_s)
{
    if (!c) return fail(LQCD_EINVAL, "NULL context");
    LQCD_ON_DEVICE(c->device);
    return stage_wait_selftest(c, limit_s);
}

int lqcd_deo_apply_mrhs_layout(lqcd_ctx *c, int out_parity, int n_rhs, int recon, int layout, const void *in,
                               void *out, void *stream)
{
    NvtxRange nvtx_("lqcd_deo_apply_mrhs_layout");
    if (!c) return fail(LQCD_EINVAL, "NULL context");
    LQCD_ON_DEVICE(c->device);
    return deo_mrhs_launch(c, out_parity, n_rhs, recon, in, out, stream ? (cudaStream_t)stream : c->stream, layout);
}

int lqcd_mscg_solve(lqcd_ctx *c, double mass, const double *shifts, int n_shift, double tol, const double *b,
                    double *x, lqcd_solve_info *info)
{
    NvtxRange nvtx_("lqcd_mscg_solve");
    const auto t0 = std::chrono::steady_clock::now();
    if (!c) return fail(LQCD_EINVAL, "NULL context");
    LQCD_ON_DEVICE(c->device);
    if (!b || !x || !shifts) return fail(LQCD_EINVAL, "NULL argument");
    if (n_shift < 1 || n_shift > LQCD_MAX_SHIFTS) return fail(LQCD_EINVAL, "n_shift must be in 1..32");
    const size_t n3 = 3 * c->Vh;
    // the device copies of b and x stay with the context (grown, never shrunk)
    // so that repeated host calls allocate nothing
    DevBuf &db = c->host_b, &dx = c->host_x;
    int st;
    if ((st = db.ensure(n3 * sizeof(double2))) || (st = dx.ensure((size_t)n_shift * n3 * sizeof(double2)))) return st;
    cudaStream_t s = c->stream;
    st = host_to_soa(c, b, db.as<double2>(), 1, s);
    if (!st) st = mscg_solve_dev(c, mass, shifts, n_shift, tol, db.as<double2>(), dx.as<double2>(), info, s);
    if (st == LQCD_OK || st == LQCD_ENOCONV) {
        const int st2 = soa_to_host(c, dx.as<double2>(), x, n_shift, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (st2) st = st2;
        else if (e != cudaSuccess) st = cuda_fail(e, "lqcd_mscg_solve");
    }
    if (info) info->secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return st;
}

int lqcd_mscg_solve_dev(lqcd_ctx *c, double mass, const double *shifts, int n_shift, double tol, const void *b,
                        void *x, lqcd_solve_info *info, void *stream)
{
    NvtxRange nvtx_("lqcd_mscg_solve_dev");
    if (!c) return fail(LQCD_EINVAL, "NULL context");
    LQCD_ON_DEVICE(c->device);
    return mscg_solve_dev(c, mass, shifts, n_shift, tol, (const double2 *)b, (double2 *)x, info, (cudaStream_t)stream);
}

int lqcd_profile_iteration(lqcd_ctx *c, double mass, const double *shifts, int n_shift, double tol, const void *b,
                           int iters, double ms_out[4], double *n_active_avg)
{
    if (!c || !ms_out || !n_active_avg) return fail(LQCD_EINVAL, "NULL argument");
    LQCD_ON_DEVICE(c->device);
    return profile_iteration(c, mass, shifts, n_shift, tol, (const double2 *)b, iters, ms_out, n_active_avg);
}

int lqcd_cg_solve_mrhs(lqcd_ctx *c, double mass, double sigma, int n_rhs, double tol, const double *b, double *x,
                       lqcd_solve_info *info)
{
    NvtxRange nvtx_("lqcd_cg_solve_mrhs");
    if (!c) return fail(LQCD_EINVAL, "NULL context");
    LQCD_ON_DEVICE(c->device);
    return cg_solve_mrhs(c, mass, sigma, n_rhs, tol, b, x, info);
}

int lqcd_mscg_solve_packed(lqcd_ctx *const *ctxs, int n, const double *mass, const double *const *shifts,
                           const int *n_shift, const double *tol, const double *const *b, double *const *x,
                           lqcd_solve_info *info)
{
    NvtxRange nvtx_("lqcd_mscg_solve_packed");
    if (!ctxs || n < 1 || n > kMaxJobs || !mass || !shifts || !n_shift || !tol || !b || !x)
        return fail(LQCD_EINVAL, "bad packed-solve arguments");
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) return fail(LQCD_EINVAL, "NULL context in a packed solve");
        if (ctxs[i]->device != ctxs[0]->device)
            return fail(LQCD_EINVAL, "the contexts of a packed solve must live on one device");
    }
    LQCD_ON_DEVICE(ctxs[0]->device);
    return mscg_solve_packed(ctxs, n, mass, shifts, n_shift, tol, b, x, info);
}

}  // extern "C"
