// particles32.cu -- FP32 cell+offset particle path (placeholder until the
// tiled kernel lands).
#include "pic_internal.h"

namespace pic {
void particles32(pic_ctx *c, double) { (void)c; }
void flux_from_acc(pic_ctx *c) { (void)c; }
int64_t sort32(pic_ctx *c) { return c->n_used; }
void charge32(pic_ctx *c, double *, double *) { (void)c; }
void reduce_particles32(pic_ctx *c) { (void)c; }
}  // namespace pic
