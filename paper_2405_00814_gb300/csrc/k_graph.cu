// Literal edge-list message passing (placeholder entry points until the graph kernels land).
#include "gem_internal.h"

namespace gem {
void graph_free(fdtd_ctx*) {}
}  // namespace gem

extern "C" {
int fdtd_step_edgelist(fdtd_ctx* c, int64_t) {
    if (!c) return FDTD_EINVAL;
    c->err = "edge-list path not available in this build";
    return FDTD_EINVAL;
}
int fdtd_export_graph(fdtd_ctx* c, int, int64_t*, int64_t*, int32_t*, int32_t*, float*) {
    if (!c) return FDTD_EINVAL;
    c->err = "edge-list path not available in this build";
    return FDTD_EINVAL;
}
}
