// batch.cu — many independent instances in one launch sequence (placeholder until built).
#include "plan.h"

struct BatchState {};

void batch_release(BatchState *b) { delete b; }

extern "C" int dbscan_batch(dbscan_plan *plan, const dbscan_instance *inst, int32_t count, dbscan_stats *per_inst) {
    (void)plan; (void)inst; (void)count; (void)per_inst;
    return DBSCAN_ERR_UNSUPPORTED;
}
