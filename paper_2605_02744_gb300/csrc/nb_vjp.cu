// Force vector-Jacobian product kernels (placeholder until the kernel lands).
#include "nb_internal.h"

namespace nb {
bool vjp_shape_compiled(const Shape &s) {
    return s.threads == 128 && (s.ipt == 1 || s.ipt == 2) && (s.tile_j == 64 || s.tile_j == 128);
}
int launch_vjp(const VjpJob &) { return fail(NB_ERR_UNSUPPORTED, "VJP kernel not built yet"); }
}  // namespace nb
