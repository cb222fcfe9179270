// Mixed-precision tensor-core form (placeholder until the tcgen05 kernel lands).
#include "sse_internal.h"

namespace sse {
sse_status mixed_plan_init(Plan &p) {
    (void)p;
    set_error("mixed mode is not built into this library yet");
    return SSE_E_INVALID_ARG;
}
void mixed_plan_free(Plan &p) { (void)p; }
sse_status launch_mixed(Plan &p, const sse_io &io, cudaStream_t st) {
    (void)p; (void)io; (void)st;
    set_error("mixed mode is not built into this library yet");
    return SSE_E_INVALID_ARG;
}
}  // namespace sse
