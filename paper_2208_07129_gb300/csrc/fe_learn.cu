// Learned cell-patch preconditioner (placeholder until the network kernels land).
#include "fe_internal.h"

namespace fe {
struct LearnedPrecond {};
bool learned_ready(const fe_ctx* c, int) { return c && c->learned != nullptr; }
fe_status learned_precond_apply(fe_ctx*, const void*, void*, int, bool, cudaStream_t) { return FE_EUNSUPPORTED; }
void free_learned(fe_ctx* c) {
  delete c->learned;
  c->learned = nullptr;
}
}  // namespace fe
