// serve.cu -- continuous-batching server for multi-shift solves.
//
// A scheduler thread owns every CUDA call of the server:
//   admit   queued requests move into free slots while the HBM budget (resident
//           fields + per-request workspaces) allows;
//   tick    one packed launch sequence advances every active request by a chunk
//           of iterations (the kernels are tiled over all requests' lattices,
//           each request with its own device scalars -- a request's arithmetic
//           does not depend on what else is in the batch);
//   retire  requests that halted get their FP64 true residuals (and, rarely,
//           a correction), their solutions are copied to host memory, their
//           slot and memory are freed, and their latency is recorded.
// Requests that arrive while others run are admitted at the next tick, so
// their work overlaps on the device with the requests already in flight.
// The packed iteration of the current batch is captured as a CUDA graph and
// replayed until the batch changes.
// Mixed precision (server options with prec = FP32): a request iterates in
// double-float down to fp64_until, switches to FP32 with reliable updates,
// and is refined per shift at retirement, exactly as a solo mixed solve.
// The requests of each engine are packed into their own launch each tick.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"

namespace lqcd {

struct Request {
    uint64_t ticket = 0;
    int field = -1;
    double mass = 0, tol = 0;
    std::vector<double> shifts;
    std::vector<double> b;        // host canonical source
    std::vector<double> x;        // host result
    lqcd_solve_info info;
    int status = LQCD_OK;
    std::chrono::steady_clock::time_point t_submit, t_done;
    // device side while active
    Workspace ws, ws32;
    DevBuf bd, xd;
    JobRun job;                   // first engine (double-float, or FP32 from the start)
    JobRun jobF;                  // FP32 phase after the switch
    bool mixed = false;           // FP32 links (server prec = FP32 at submit)
    double fp64_until = 0;
    int phase = 0;                // 1 after the switch to FP32
    size_t bytes = 0;
    JobRun &cur() { return phase ? jobF : job; }
};

struct Field {
    lqcd_ctx *ctx = nullptr;
    size_t bytes = 0;
};

static size_t request_bytes(const lqcd_ctx *c, int n_shift)
{
    const size_t n3 = 3 * c->Vh;
    const int ntiles = (int)((c->Vh + kTile - 1) / kTile);
    return (3 + 2 * (size_t)n_shift) * n3 * sizeof(float4)   // df64 Krylov vectors
           + 2 * n3 * sizeof(double2)                         // r_hi, t (true residual)
           + (1 + (size_t)n_shift) * n3 * sizeof(double2)     // IEEE b, x
           + (size_t)ntiles * sizeof(double) + 1024 + sizeof(SolverState);
}

// Extra device bytes of a mixed-precision request: the FP32 phase's Krylov
// vectors and IEEE temporaries, and the per-shift refinement workspaces
// (held by the field's context after first use; counted per request).
static size_t request_bytes_mixed(const lqcd_ctx *c, int n_shift)
{
    const size_t n3 = 3 * c->Vh;
    const int ntiles = (int)((c->Vh + kTile - 1) / kTile);
    const size_t phase = (3 + 2 * (size_t)n_shift) * n3 * sizeof(float2) + 2 * n3 * sizeof(double2) +
                         (size_t)ntiles * sizeof(double) + 1024 + sizeof(SolverState);
    const size_t refine = (size_t)n_shift * (5 * n3 * sizeof(float2) + 2 * n3 * sizeof(double2) +
                                             (size_t)ntiles * sizeof(double) + 1024 + sizeof(SolverState));
    return phase + refine;
}

}  // namespace lqcd

using namespace lqcd;

struct lqcd_server {
    int device = 0;
    size_t budget = 0;
    int max_slots = 0, max_queue = 0;
    cudaStream_t stream = nullptr;
    std::mutex mu;
    std::condition_variable cv, cv_done;
    std::thread th;
    bool stop = false;
    std::vector<Field> fields;
    size_t in_use = 0;
    uint64_t next_ticket = 1;
    std::deque<std::unique_ptr<Request>> queue;
    std::vector<std::unique_ptr<Request>> active;   // scheduler thread only
    std::map<uint64_t, std::unique_ptr<Request>> done;
    std::vector<double> latencies;
    uint64_t submitted = 0, completed = 0, rejected = 0, ticks = 0;
    std::chrono::steady_clock::time_point t_first, t_last;
    bool have_first = false;
    int n_active = 0;  // mirror for stats
    lqcd_opts opts;               // applied to fields and to requests submitted after
    // graphs of the current batches, one per engine (double-float, FP32)
    uint64_t batch_key[2] = {~0ull, ~0ull};
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    int chunk = 8;
    int error = LQCD_OK;
    std::string error_msg;

    void run();
    bool admit();
    int tick();
    void retire(std::unique_ptr<Request> &r, int st);
};

void lqcd_server::retire(std::unique_ptr<Request> &r, int st)
{
    Field &f = fields[r->field];
    lqcd_ctx *c = f.ctx;
    if (st == LQCD_OK || st == LQCD_ENOCONV) {
        st = job_finish(r->cur(), stream);
        if (st == LQCD_OK || st == LQCD_ENOCONV) {
            r->x.resize((size_t)r->shifts.size() * c->Vh * 6);
            const int st2 = soa_to_host(c, r->xd.as<double2>(), r->x.data(), (int)r->shifts.size(), stream);
            cudaStreamSynchronize(stream);
            if (st2) st = st2;
        }
    }
    r->status = st;
    r->info = r->cur().I;
    r->t_done = std::chrono::steady_clock::now();
    r->info.secs = std::chrono::duration<double>(r->t_done - r->t_submit).count();
    r->ws.release();
    r->ws32.release();
    r->bd.release();
    r->xd.release();
    std::lock_guard<std::mutex> lk(mu);
    in_use -= r->bytes;
    latencies.push_back(r->info.secs);
    t_last = r->t_done;
    ++completed;
    done[r->ticket] = std::move(r);
    cv_done.notify_all();
}

// Move queued requests into slots while slots and memory allow (FIFO).
bool lqcd_server::admit()
{
    bool changed = false;
    for (;;) {
        std::unique_ptr<Request> r;
        {
            std::lock_guard<std::mutex> lk(mu);
            if (queue.empty() || (int)active.size() >= max_slots) break;
            if (in_use + queue.front()->bytes > budget) break;
            r = std::move(queue.front());
            queue.pop_front();
            in_use += r->bytes;
        }
        lqcd_ctx *c = fields[r->field].ctx;
        const size_t n3 = 3 * c->Vh;
        int st = r->bd.ensure(n3 * sizeof(double2));
        if (!st) st = r->xd.ensure(r->shifts.size() * n3 * sizeof(double2));
        // a mixed request starts in double-float unless fp64_until is 0
        const int prec0 = r->mixed && r->fp64_until == 0.0 ? LQCD_PREC_FP32 : LQCD_PREC_FP64;
        if (!st) st = job_init_prec(r->job, c, &r->ws, prec0, r->mass, r->shifts.data(), (int)r->shifts.size(),
                                    r->tol, r->bd.as<double2>(), r->xd.as<double2>());
        if (r->mixed && prec0 == LQCD_PREC_FP64) r->job.switch_rel = r->fp64_until;
        if (!st) st = host_to_soa(c, r->b.data(), r->bd.as<double2>(), 1, stream);
        if (!st) st = job_setup(r->job, stream);
        if (st) {
            memset(&r->job.I, 0, sizeof r->job.I);
            retire(r, st);
            continue;
        }
        active.push_back(std::move(r));
        changed = true;
    }
    return changed;
}

// Advance every active request by one chunk of packed iterations; retire the
// ones that halted.  Returns a status on CUDA failure.
int lqcd_server::tick()
{
    // requests with a zero source finish without iterating
    for (size_t i = 0; i < active.size();) {
        if (active[i]->job.zero) {
            retire(active[i], LQCD_OK);
            active.erase(active.begin() + i);
        } else {
            ++i;
        }
    }
    if (active.empty()) return LQCD_OK;
    // one packed batch per engine: double-float (links df64) and FP32
    // (the server's link format); a batch holds at most kMaxJobs requests
    IterBatch<kMaxJobs> B[2];
    std::vector<int> idx[2];
    int lf[2] = {0, 0};
    for (int g = 0; g < 2; ++g) {
        memset(&B[g], 0, sizeof B[g]);
        int tiles = 0;
        for (size_t i = 0; i < active.size(); ++i) {
            JobRun &J = active[i]->cur();
            if (J.vp != g || B[g].njobs == kMaxJobs) continue;
            const int k = B[g].njobs++;
            B[g].tile_start[k] = tiles;
            job_fill(J, B[g].job[k]);
            tiles += J.P.ntiles;
            B[g].max_shift = std::max(B[g].max_shift, J.n_shift);
            lf[g] = J.lf;
            idx[g].push_back((int)i);
        }
        B[g].tile_start[B[g].njobs] = tiles;
    }
    cudaError_t e = cudaSuccess;
    for (int g = 0; g < 2 && e == cudaSuccess; ++g) {
        if (!B[g].njobs) continue;
        uint64_t key = 1469598103934665603ull;
        const unsigned char *p = (const unsigned char *)&B[g];
        for (size_t k = 0; k < sizeof B[g]; ++k) key = (key ^ p[k]) * 1099511628211ull;
        key = (key ^ (uint64_t)lf[g]) * 1099511628211ull;
        key = (key ^ (uint64_t)opts.pdl) * 1099511628211ull;
        if (key != batch_key[g] || !exec[g]) {
            if (exec[g]) cudaGraphExecDestroy(exec[g]);
            exec[g] = nullptr;
            cudaGraph_t gr;
            e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return cuda_fail(e, "serve capture");
            for (int k = 0; k < chunk; ++k) launch_iteration_packed(B[g], g, lf[g], stream, opts.pdl != 0, k > 0);
            e = cudaStreamEndCapture(stream, &gr);
            if (e != cudaSuccess) return cuda_fail(e, "serve capture");
            e = cudaGraphInstantiate(&exec[g], gr, 0);
            cudaGraphDestroy(gr);
            if (e != cudaSuccess) return cuda_fail(e, "serve instantiate");
            batch_key[g] = key;
        }
        e = cudaGraphLaunch(exec[g], stream);
    }
    std::vector<int> halts(active.size(), HALT_NONE);
    for (int g = 0; g < 2; ++g)
        for (int k = 0; k < B[g].njobs && e == cudaSuccess; ++k)
            e = cudaMemcpyAsync(&halts[idx[g][k]], &B[g].job[k].st->halt, sizeof(int), cudaMemcpyDeviceToHost,
                                stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "serve tick");
    {
        std::lock_guard<std::mutex> lk(mu);
        ++ticks;
    }
    for (int j = (int)active.size() - 1; j >= 0; --j) {
        Request &r = *active[j];
        const int h = halts[j];
        if (h == HALT_NONE) continue;
        int st = LQCD_OK;
        if (h == HALT_RELIABLE) {
            lqcd_ctx *c = fields[r.field].ctx;
            if (r.cur().vp == VP_DF) {
                // double-float phase reached fp64_until: switch to FP32
                st = job_init_prec(r.jobF, c, &r.ws32, LQCD_PREC_FP32, r.mass, r.shifts.data(),
                                   (int)r.shifts.size(), r.tol, r.bd.as<double2>(), r.xd.as<double2>());
                if (!st) {
                    r.jobF.b2 = r.job.b2;
                    st = job_switch_to_f32(r.job, r.jobF, stream);
                }
                if (!st) r.phase = 1;
            } else {
                st = job_reliable_update(r.cur(), stream);
            }
            if (!st) continue;
        } else if (h == HALT_NAN) {
            st = LQCD_ENAN;
        } else if (h == HALT_STALL) {
            st = LQCD_ETIMEOUT;
        }
        retire(active[j], st);
        active.erase(active.begin() + j);
    }
    return LQCD_OK;
}

void lqcd_server::run()
{
    cudaSetDevice(device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(mu);
            cv.wait(lk, [&] { return stop || !queue.empty() || !active.empty(); });
            if (stop) break;
        }
        admit();
        {
            std::lock_guard<std::mutex> lk(mu);
            n_active = (int)active.size();
        }
        const int st = tick();
        if (st) {
            std::lock_guard<std::mutex> lk(mu);
            error = st;
            error_msg = lqcd_last_error();
            // fail every in-flight request rather than spin
            for (auto &r : active) {
                r->status = st;
                r->t_done = std::chrono::steady_clock::now();
                in_use -= r->bytes;
                ++completed;
                done[r->ticket] = std::move(r);
            }
            active.clear();
            cv_done.notify_all();
        }
        std::lock_guard<std::mutex> lk(mu);
        n_active = (int)active.size();
        cv_done.notify_all();
    }
}

extern "C" {

int lqcd_serve_create(size_t hbm_budget_bytes, int max_slots, int max_queue, lqcd_server **out)
{
    if (!out) return fail(LQCD_EINVAL, "NULL argument");
    *out = nullptr;
    if (max_slots < 1 || max_slots > kMaxJobs) return fail(LQCD_EINVAL, "max_slots must be in 1..64");
    if (max_queue < 1) return fail(LQCD_EINVAL, "max_queue must be >= 1");
    if (hbm_budget_bytes == 0) return fail(LQCD_EINVAL, "hbm budget must be > 0");
    lqcd_server *s = new (std::nothrow) lqcd_server();
    if (!s) return fail(LQCD_ENOMEM, "host allocation failed");
    lqcd_default_opts(&s->opts);
    s->budget = hbm_budget_bytes;
    s->max_slots = max_slots;
    s->max_queue = max_queue;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaStreamCreate(&s->stream);
    if (e != cudaSuccess) {
        delete s;
        return cuda_fail(e, "lqcd_serve_create");
    }
    s->th = std::thread([s] { s->run(); });
    *out = s;
    return LQCD_OK;
}

int lqcd_serve_register_field(lqcd_server *s, const int dims[4], const double *links, size_t n_doubles,
                              int *field_id)
{
    if (!s || !dims || !links || !field_id) return fail(LQCD_EINVAL, "NULL argument");
    LQCD_ON_DEVICE(s->device);
    lqcd_ctx *c = nullptr;
    lqcd_opts o;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        o = s->opts;
    }
    int st = lqcd_create(dims, &o, &c);
    if (st) return st;
    // the field's links count against the budget (all storage formats)
    const size_t need = (size_t)c->Vh * (72 * 16 + 72 * 16 + 72 * 8 + 24 * 16 + 8 * 24);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->in_use + need > s->budget) {
            lqcd_destroy(c);
            return fail(LQCD_ENOMEM, "field does not fit the HBM budget");
        }
        s->in_use += need;
    }
    st = lqcd_links_upload(c, links, n_doubles);
    if (st) {
        lqcd_destroy(c);
        std::lock_guard<std::mutex> lk(s->mu);
        s->in_use -= need;
        return st;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->fields.push_back(Field{c, need});
    *field_id = (int)s->fields.size() - 1;
    return LQCD_OK;
}

int lqcd_serve_submit(lqcd_server *s, int field_id, double mass, const double *shifts, int n_shift, double tol,
                      const double *b, uint64_t *ticket)
{
    if (!s || !shifts || !b || !ticket) return fail(LQCD_EINVAL, "NULL argument");
    lqcd_ctx *c;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (field_id < 0 || field_id >= (int)s->fields.size()) return fail(LQCD_EINVAL, "unknown field id");
        c = s->fields[field_id].ctx;
    }
    int st = validate_solve(c, mass, shifts, n_shift, tol);
    if (st) return st;
    auto r = std::make_unique<Request>();
    r->field = field_id;
    r->mass = mass;
    r->tol = tol;
    r->shifts.assign(shifts, shifts + n_shift);
    r->b.assign(b, b + c->Vh * 6);
    r->t_submit = std::chrono::steady_clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    r->mixed = s->opts.prec == LQCD_PREC_FP32;
    r->fp64_until = s->opts.fp64_until;
    r->bytes = request_bytes(c, n_shift) + (r->mixed ? request_bytes_mixed(c, n_shift) : 0);
    if (r->bytes + s->fields[field_id].bytes > s->budget) {
        ++s->rejected;
        return fail(LQCD_ENOMEM, "request can never fit the HBM budget");
    }
    if ((int)s->queue.size() >= s->max_queue) {
        ++s->rejected;
        return fail(LQCD_EBUSY, "queue full");
    }
    r->ticket = s->next_ticket++;
    *ticket = r->ticket;
    if (!s->have_first) {
        s->t_first = r->t_submit;
        s->have_first = true;
    }
    ++s->submitted;
    s->queue.push_back(std::move(r));
    s->cv.notify_all();
    return LQCD_OK;
}

int lqcd_serve_set_opts(lqcd_server *s, const lqcd_opts *o)
{
    if (!s || !o) return fail(LQCD_EINVAL, "NULL argument");
    int st = validate_opts(o);
    if (st) return st;
    if (o->prec != LQCD_PREC_FP64 && o->prec != LQCD_PREC_FP32)
        return fail(LQCD_EINVAL, "the server runs FP64 or FP32 (mixed) requests");
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->completed < s->submitted) return fail(LQCD_EBUSY, "requests in flight");
    s->opts = *o;
    for (Field &f : s->fields) f.ctx->opts = *o;
    return LQCD_OK;
}

int lqcd_serve_poll(lqcd_server *s, uint64_t ticket, double *x, lqcd_solve_info *info)
{
    if (!s) return fail(LQCD_EINVAL, "NULL server");
    std::unique_ptr<Request> r;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->done.find(ticket);
        if (it == s->done.end()) {
            if (ticket == 0 || ticket >= s->next_ticket) return fail(LQCD_EINVAL, "unknown ticket");
            return LQCD_ENOTREADY;
        }
        r = std::move(it->second);
        s->done.erase(it);
    }
    if (x && !r->x.empty()) memcpy(x, r->x.data(), r->x.size() * sizeof(double));
    if (info) *info = r->info;
    if (r->status != LQCD_OK) {
        set_error("request finished with an error");
        return r->status;
    }
    return LQCD_OK;
}

int lqcd_serve_drain(lqcd_server *s, double timeout_s)
{
    if (!s) return fail(LQCD_EINVAL, "NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto idle = [&] { return s->completed >= s->submitted; };
    if (timeout_s > 0) {
        if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), idle))
            return fail(LQCD_ETIMEOUT, "drain timed out");
    } else {
        s->cv_done.wait(lk, idle);
    }
    return s->error;
}

int lqcd_serve_stats_get(lqcd_server *s, lqcd_serve_stats *o)
{
    if (!s || !o) return fail(LQCD_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    memset(o, 0, sizeof *o);
    o->submitted = s->submitted;
    o->completed = s->completed;
    o->rejected = s->rejected;
    o->active_slots = s->n_active;
    o->queued = (int)s->queue.size();
    o->hbm_in_use = s->in_use;
    o->hbm_budget = s->budget;
    o->ticks = s->ticks;
    if (!s->latencies.empty()) {
        std::vector<double> l = s->latencies;
        std::sort(l.begin(), l.end());
        auto q = [&](double f) { return l[std::min(l.size() - 1, (size_t)std::floor(f * (l.size() - 1) + 0.5))]; };
        o->p50_latency = q(0.50);
        o->p99_latency = q(0.99);
        double m = 0;
        for (double v : l) m += v;
        o->mean_latency = m / l.size();
        const double span = std::chrono::duration<double>(s->t_last - s->t_first).count();
        o->solves_per_sec = span > 0 ? s->completed / span : 0.0;
    }
    return LQCD_OK;
}

void lqcd_serve_destroy(lqcd_server *s)
{
    if (!s) return;
    DeviceGuard device_guard(s->device);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->th.joinable()) s->th.join();
    for (auto &r : s->active) {
        r->ws.release();
        r->ws32.release();
        r->bd.release();
        r->xd.release();
    }
    for (cudaGraphExec_t g : s->exec)
        if (g) cudaGraphExecDestroy(g);
    for (auto &f : s->fields) lqcd_destroy(f.ctx);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

}  // extern "C"
