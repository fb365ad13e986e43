// mrhs.cu -- multi-right-hand-side D_eo and batched CG (placeholder).
#include "internal.h"

namespace lqcd {

int deo_mrhs_launch(lqcd_ctx *c, int out_parity, int n_rhs, int recon, const void *in, void *out, cudaStream_t s)
{
    (void)c; (void)out_parity; (void)n_rhs; (void)recon; (void)in; (void)out; (void)s;
    return fail(LQCD_EINVAL, "multi-RHS D_eo not built yet");
}

int cg_solve_mrhs(lqcd_ctx *c, double mass, double sigma, int n_rhs, double tol, const double *b, double *x,
                  lqcd_solve_info *info)
{
    (void)c; (void)mass; (void)sigma; (void)n_rhs; (void)tol; (void)b; (void)x; (void)info;
    return fail(LQCD_EINVAL, "multi-RHS CG not built yet");
}

}  // namespace lqcd
