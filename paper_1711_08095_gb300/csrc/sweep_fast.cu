// Fast (lock-free) sweep: placeholder until the wave kernels land.
#include "common.cuh"

namespace snect {

int prep_fast_tiles(Ctx *c) { return fail(c, SNECT_EINVAL, "fast mode is not available yet"); }
int enqueue_fast_epoch(Ctx *c) { return fail(c, SNECT_EINVAL, "fast mode is not available yet"); }
void free_fast(Ctx *) {}

}  // namespace snect
