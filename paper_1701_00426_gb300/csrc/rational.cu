// rational.cu -- a rational function of the even/odd operator applied to a
// source, and the pseudofermion action, as an epilogue of the multi-shift
// solve on the device (Sec. 2.2: the RHMC replaces the root of the fermion
// matrix in Eq. rooting by r(x) = a0 + sum_i a_i / (x + sigma_i) with real
// poles sigma_i, whose shifted systems are Eq. shlineq; Algorithm 1, steps
// 3, 4 and 6: heatbath and actions are such applications).
//
//   y = a0 b + sum_i a_i x_i,   (A + sigma_i) x_i = b,   A = m^2 - D_eo D_oe
//   S = Re <b, y>
//
// The x_i come from the multi-shift solve (each to its FP64 true residual
// <= tol) into a device scratch array of the context and never leave the
// GPU: one pass combines them (FP64, one thread per complex element) and
// writes per-block partials of S, which a one-block kernel sums in block
// order, so S does not depend on scheduling.
#include <cmath>

#include "internal.h"

namespace lqcd {

struct RatCoef {
    double a0;
    double a[kMaxShifts];
    int n;
};

constexpr int kRatThreads = 256;

__global__ void __launch_bounds__(kRatThreads)
    k_rational_combine(const __grid_constant__ RatCoef C, const double2 *__restrict__ b,
                       const double2 *__restrict__ x, double2 *__restrict__ y, long n3, double *part)
{
    __shared__ double s_red[kRatThreads / 32];
    const long t = blockIdx.x * (long)kRatThreads + threadIdx.x;
    double d = 0.0;
    if (t < n3) {
        const double2 bv = b[t];
        double2 v = make_double2(C.a0 * bv.x, C.a0 * bv.y);
        for (int i = 0; i < C.n; ++i) {
            const double2 xv = __ldcs(x + (size_t)i * n3 + t);
            v.x = fma(C.a[i], xv.x, v.x);
            v.y = fma(C.a[i], xv.y, v.y);
        }
        y[t] = v;
        d = fma(bv.x, v.x, bv.y * v.y);   // Re(conj(b) y)
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xFFFFFFFFu, d, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < kRatThreads / 32; ++k) s += s_red[k];
        part[blockIdx.x] = s;
    }
}

// One block: sum of part[0..n) in a fixed order.
__global__ void __launch_bounds__(kRatThreads) k_sum_ordered(const double *__restrict__ part, int n, double *out)
{
    __shared__ double s_red[kRatThreads / 32];
    double s = 0.0;
    for (int k = threadIdx.x; k < n; k += kRatThreads) s += part[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int k = 0; k < kRatThreads / 32; ++k) tot += s_red[k];
        *out = tot;
    }
}

int rational_apply_dev(lqcd_ctx *c, double mass, double a0, const double *a, const double *shifts, int n_shift,
                       double tol, const double2 *b, double2 *y, double *action, lqcd_solve_info *info,
                       cudaStream_t s_user)
{
    if (!b || !y || !a || !shifts) return fail(LQCD_EINVAL, "NULL argument");
    if (n_shift < 1 || n_shift > kMaxShifts) return fail(LQCD_EINVAL, "n_shift must be in 1..32");
    if (!std::isfinite(a0)) return fail(LQCD_EINVAL, "a0 is not finite");
    RatCoef C;
    C.a0 = a0;
    C.n = n_shift;
    for (int i = 0; i < n_shift; ++i) {
        if (!std::isfinite(a[i])) return fail(LQCD_EINVAL, "a coefficient is not finite");
        C.a[i] = a[i];
    }
    for (int i = n_shift; i < kMaxShifts; ++i) C.a[i] = 0.0;
    const long n3 = 3 * (long)c->Vh;
    const unsigned nb = (unsigned)((n3 + kRatThreads - 1) / kRatThreads);
    int st;
    if ((st = c->rat_x.ensure((size_t)n_shift * n3 * sizeof(double2)))) return st;
    if ((st = c->rat_part.ensure(((size_t)nb + 1) * sizeof(double)))) return st;
    const int rs = mscg_solve_dev(c, mass, shifts, n_shift, tol, b, c->rat_x.as<double2>(), info, s_user);
    if (rs != LQCD_OK && rs != LQCD_ENOCONV) return rs;
    cudaStream_t s = c->stream;
    double *part = c->rat_part.as<double>();
    k_rational_combine<<<nb, kRatThreads, 0, s>>>(C, b, c->rat_x.as<double2>(), y, n3, part);
    k_sum_ordered<<<1, kRatThreads, 0, s>>>(part, (int)nb, part + nb);
    LQCD_CUDA(cudaGetLastError());
    c->launches += 2;
    LQCD_CUDA(cudaMemcpyAsync(c->h_pinned_d, part + nb, sizeof(double), cudaMemcpyDeviceToHost, s));
    LQCD_CUDA(cudaStreamSynchronize(s));
    if (action) *action = c->h_pinned_d[0];
    if (info) info->kernel_launches += 2;
    if (rs == LQCD_ENOCONV) set_error("solver did not reach tol within max_iter");
    return rs;
}

}  // namespace lqcd

using namespace lqcd;

extern "C" {

int lqcd_rational_apply_dev(lqcd_ctx *c, double mass, double a0, const double *a, const double *shifts, int n_shift,
                            double tol, const void *b, void *y, double *action, lqcd_solve_info *info, void *stream)
{
    NvtxRange nvtx_("lqcd_rational_apply_dev");
    if (!c) return fail(LQCD_EINVAL, "NULL context");
    LQCD_ON_DEVICE(c->device);
    return rational_apply_dev(c, mass, a0, a, shifts, n_shift, tol, (const double2 *)b, (double2 *)y, action, info,
                              (cudaStream_t)stream);
}

int lqcd_rational_apply(lqcd_ctx *c, double mass, double a0, const double *a, const double *shifts, int n_shift,
                        double tol, const double *b, double *y, double *action, lqcd_solve_info *info)
{
    NvtxRange nvtx_("lqcd_rational_apply");
    if (!c) return fail(LQCD_EINVAL, "NULL context");
    LQCD_ON_DEVICE(c->device);
    if (!b || !y) return fail(LQCD_EINVAL, "NULL argument");
    const size_t bytes = 3 * c->Vh * sizeof(double2);
    DevBuf db, dy;
    int st;
    if ((st = db.ensure(bytes)) || (st = dy.ensure(bytes))) return st;
    cudaStream_t s = c->stream;
    st = host_to_soa(c, b, db.as<double2>(), 1, s);
    if (!st) st = rational_apply_dev(c, mass, a0, a, shifts, n_shift, tol, db.as<double2>(), dy.as<double2>(),
                                     action, info, s);
    if (st == LQCD_OK || st == LQCD_ENOCONV) {
        const int st2 = soa_to_host(c, dy.as<double2>(), y, 1, s);
        const cudaError_t e = cudaStreamSynchronize(s);
        if (st2) st = st2;
        else if (e != cudaSuccess) st = cuda_fail(e, "lqcd_rational_apply");
    }
    db.release();
    dy.release();
    return st;
}

}  // extern "C"
