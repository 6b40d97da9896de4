// Batched persistent kernel (placeholder until the kernel lands).
#include "nb_internal.h"

namespace nb {
size_t batched_scratch_bytes(int32_t B) { return 64 * (size_t)(B + 1); }
int launch_batched(const BatchedJob &) {
    return fail(NB_ERR_UNSUPPORTED, "batched kernel not built yet");
}
}  // namespace nb
