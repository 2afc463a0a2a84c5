// 3D Yee path (placeholder entry points until the 3D kernels land).
#include "gem_internal.h"

namespace gem {
static int no3(fdtd_ctx* c) {
    if (c) c->err = "3D grids are not available in this build";
    return FDTD_EINVAL;
}
int fdtd_create3(const fdtd_grid*, double, double, double, const uint8_t*, const fdtd_material*, int, void* stream,
                 fdtd_ctx** out) {
    *out = nullptr;
    (void)stream;
    return FDTD_EINVAL;
}
void fdtd_destroy3(fdtd_ctx*) {}
int fdtd_set_source3(fdtd_ctx* c, int, int, int, int, int, const double*, const float*, int64_t) { return no3(c); }
int fdtd_add_probe3(fdtd_ctx* c, int, int, int, int, int*) { return no3(c); }
int fdtd_add_dft_monitor3(fdtd_ctx* c, const int32_t*, int, const double*, int, int*) { return no3(c); }
int fdtd_add_dft_plane3(fdtd_ctx* c, int, int, const double*, int, int*) { return no3(c); }
int fdtd_step3(fdtd_ctx* c, int64_t) { return no3(c); }
int fdtd_read_probe3(fdtd_ctx* c, int, float*, int64_t) { return no3(c); }
int fdtd_read_dft3(fdtd_ctx* c, int, float*, float*) { return no3(c); }
int fdtd_get_field3(fdtd_ctx* c, int, float*, int) { return no3(c); }
int fdtd_set_field3(fdtd_ctx* c, int, const float*, int) { return no3(c); }
int fdtd_reset3(fdtd_ctx* c) { return no3(c); }
int fdtd_save_state3(fdtd_ctx* c, void*, size_t*) { return no3(c); }
int fdtd_load_state3(fdtd_ctx* c, const void*, size_t) { return no3(c); }
int fdtd_check_finite3(fdtd_ctx* c) { return no3(c); }
}  // namespace gem
