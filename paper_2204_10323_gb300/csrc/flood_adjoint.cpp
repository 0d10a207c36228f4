// flood_adjoint.cpp -- reverse sweep driver (binomial checkpointing).
// Placeholder until the adjoint kernels land.
#include "flood_runtime.h"

using namespace flood;

namespace flood {
void destroy_adjoint(flood_handle *) {}
}  // namespace flood

extern "C" flood_status flood_adjoint(flood_handle *h, int64_t, const int64_t *, int32_t, const double *, int32_t,
                                      void *, void *, int32_t)
{
    return fail(h, FLOOD_ERR_UNSUPPORTED, "adjoint not built yet");
}

extern "C" int64_t flood_adjoint_forward_steps(const flood_handle *h) { return h ? h->adj_forward_steps : 0; }
