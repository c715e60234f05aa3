// Batched persistent execution of many small circuits (qsim_batch_*).
#include "internal.h"
#include "plan.h"

using namespace qsim;
struct qsim_batch {};
extern "C" {
int qsim_batch_create(int, const qsim_circuit *const *, qsim_batch **) {
    return set_error(QSIM_EUNSUPPORTED, "batch not built yet");
}
int qsim_batch_destroy(qsim_batch *b) { delete b; return QSIM_OK; }
int qsim_batch_run(qsim_batch *, double *, void *) { return set_error(QSIM_EUNSUPPORTED, "batch not built yet"); }
int qsim_batch_set_config(qsim_batch *, int, int) { return set_error(QSIM_EUNSUPPORTED, "batch not built yet"); }
}
