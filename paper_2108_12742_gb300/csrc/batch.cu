// Batched uneven 1D problems (placeholder until the persistent kernel lands).
#include "enoao.h"
#include "enoao_internal.h"

namespace enoao {
struct BatchState {};
void batch_destroy(BatchState* b) { delete b; }
enoao_status batch_create(enoao_ctx*, const enoao_config*, int, const int64_t*, const double*,
                          const double*) {
  return ENOAO_EINVAL;
}
enoao_status batch_advance(enoao_ctx*, int64_t, double, bool) { return ENOAO_EINVAL; }
enoao_status batch_init_state(enoao_ctx*, const double*, int) { return ENOAO_EINVAL; }
enoao_status batch_get_state(enoao_ctx*, double*, int) { return ENOAO_EINVAL; }
}  // namespace enoao
