// noalloc.cu -- host-buffer D_eo / D_oe that allocates no device memory.
//
// lqcd_deo_apply with host buffers stages its input and output through
// device buffers that it allocates.  Some callers cannot allow that: a
// process whose device memory is handed out by another framework's pool
// allocator, or a loop that cannot pay for the device-wide synchronisation
// of cudaMalloc / cudaFree.  This variant runs the same kernels through one
// fixed staging area that lives in the library itself: a file-scope device
// array, created when the library is loaded on a device and kept until the
// process exits.
//
// Host code cannot use the array's name as a device address: on the host it
// names a stand-in object, and a kernel handed it would fault or, where the
// GPU can reach host memory, use the wrong memory.  The device address is
// therefore looked up with cudaGetSymbolAddress, with the context's device
// current, on the first call made in a CUDA context of that device, and kept
// with that context's identifier.  A device reset replaces the context (and
// may move the array); the next call sees the new identifier and looks the
// address up again.
#include <mutex>

#include <cuda.h>  // driver API types only; the two functions are resolved at run time

#include "internal.h"

namespace lqcd {

// Largest half lattice served: V/2 <= 131072 sites (16^4 is 32768, 20^4 is
// 80000).  Layout: three regions of 3 * kNoAllocMaxVh complex128 each --
// host-format staging, structure-of-arrays input, structure-of-arrays output.
constexpr long kNoAllocMaxVh = 131072;
constexpr size_t kNoAllocRegion = 3 * (size_t)kNoAllocMaxVh;  // double2 elements per region

static __device__ __align__(256) double2 g_noalloc_stage[3 * kNoAllocRegion];

using PfnStreamGetCtx = CUresult (*)(CUstream, CUcontext *);
using PfnCtxGetId = CUresult (*)(CUcontext, unsigned long long *);

// Identifier of the CUDA context that owns stream s; 0 when the driver does
// not tell (then the address is looked up on every call).
static unsigned long long stream_context_id(cudaStream_t s)
{
    static PfnStreamGetCtx get_ctx = nullptr;
    static PfnCtxGetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuStreamGetCtx", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_ctx = (PfnStreamGetCtx)p;
        p = nullptr;
        q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (PfnCtxGetId)p;
        cudaGetLastError();
    });
    if (!get_ctx || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_ctx((CUstream)s, &ctx) != CUDA_SUCCESS || !ctx) return 0;
    if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

static std::mutex g_noalloc_mu;
struct NoAllocAddr {
    unsigned long long ctx_id = 0;
    double2 *ptr = nullptr;
};
static NoAllocAddr g_noalloc_addr[64];  // per device ordinal, set up on first use in a context

// Device address of the staging array for context c (its device is current).
static int noalloc_stage(const lqcd_ctx *c, double2 **out)
{
    const int dev = c->device;
    if (dev < 0 || dev >= 64) return fail(LQCD_EINVAL, "device ordinal out of range");
    const unsigned long long id = stream_context_id(c->stream);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    NoAllocAddr &a = g_noalloc_addr[dev];
    if (!a.ptr || id == 0 || a.ctx_id != id) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_stage);
        if (e != cudaSuccess) {
            a = NoAllocAddr{};
            return cuda_fail(e, "cudaGetSymbolAddress of the no-allocation staging array");
        }
        a.ptr = (double2 *)p;
        a.ctx_id = id;
    }
    *out = a.ptr;
    return LQCD_OK;
}

}  // namespace lqcd

using namespace lqcd;

extern "C" int lqcd_deo_apply_host_noalloc(lqcd_ctx *c, int out_parity, const double *in, double *out)
{
    if (!c) return fail(LQCD_EINVAL, "NULL context");
    LQCD_ON_DEVICE(c->device);
    if (!in || !out) return fail(LQCD_EINVAL, "NULL host buffer");
    if (out_parity != 0 && out_parity != 1) return fail(LQCD_EINVAL, "out_parity must be 0 or 1");
    if (int lr = links_ready(c)) return lr;
    if ((long)c->Vh > kNoAllocMaxVh)
        return fail(LQCD_EINVAL, "lattice too large for lqcd_deo_apply_host_noalloc: V/2 = " +
                                     std::to_string(c->Vh) + " exceeds its fixed staging of " +
                                     std::to_string(kNoAllocMaxVh) + " sites");
    double2 *stage = nullptr;
    int st = noalloc_stage(c, &stage);
    if (st) return st;
    // Every element read below is written earlier in the same call, so the
    // contents left by a previous call need no clearing.
    double2 *aos = stage, *soa_in = stage + kNoAllocRegion, *soa_out = stage + 2 * kNoAllocRegion;
    const size_t bytes = 3 * c->Vh * sizeof(double2);
    const long Vh = (long)c->Vh;
    const unsigned nb = (unsigned)((Vh + 255) / 256);
    cudaStream_t s = c->stream;
    LQCD_CUDA(cudaMemcpyAsync(aos, in, bytes, cudaMemcpyHostToDevice, s));
    k_aos_to_soa<<<nb, 256, 0, s>>>(aos, soa_in, Vh, 1);
    LQCD_CUDA(cudaGetLastError());
    k_deo_df_ieee<<<(unsigned)((Vh + kTile - 1) / kTile), kTile, 0, s>>>(c->g, c->lnk_df.as<float4>(), soa_in,
                                                                        soa_out, out_parity);
    LQCD_CUDA(cudaGetLastError());
    k_soa_to_aos<<<nb, 256, 0, s>>>(soa_out, aos, Vh, 1);
    LQCD_CUDA(cudaGetLastError());
    LQCD_CUDA(cudaMemcpyAsync(out, aos, bytes, cudaMemcpyDeviceToHost, s));
    LQCD_CUDA(cudaStreamSynchronize(s));
    c->launches += 3;
    return LQCD_OK;
}
