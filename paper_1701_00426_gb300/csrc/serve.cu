// serve.cu -- continuous-batching solve server (placeholder).
#include "internal.h"

using namespace lqcd;

extern "C" {
int lqcd_serve_create(size_t, int, int, lqcd_server **srv) { if (srv) *srv = nullptr; return fail(LQCD_EINVAL, "server not built yet"); }
int lqcd_serve_register_field(lqcd_server *, const int *, const double *, size_t, int *) { return fail(LQCD_EINVAL, "server not built yet"); }
int lqcd_serve_submit(lqcd_server *, int, double, const double *, int, double, const double *, uint64_t *) { return fail(LQCD_EINVAL, "server not built yet"); }
int lqcd_serve_poll(lqcd_server *, uint64_t, double *, lqcd_solve_info *) { return fail(LQCD_EINVAL, "server not built yet"); }
int lqcd_serve_drain(lqcd_server *, double) { return fail(LQCD_EINVAL, "server not built yet"); }
int lqcd_serve_stats_get(lqcd_server *, lqcd_serve_stats *) { return fail(LQCD_EINVAL, "server not built yet"); }
void lqcd_serve_destroy(lqcd_server *) {}
}
