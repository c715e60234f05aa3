// Cache-blocked multi-gate stages (QSIM_FUSE_STAGED).
#include "internal.h"
#include "plan.h"

namespace qsim {
struct StagedPlan {};
int build_staged(const qsim_circuit &, qsim_plan &) { return set_error(QSIM_EUNSUPPORTED, "staged fusion not built yet"); }
int run_staged(qsim_state *, qsim_plan &) { return set_error(QSIM_EUNSUPPORTED, "staged fusion not built yet"); }
int staged_nsweeps(const qsim_plan &) { return 0; }
}  // namespace qsim

void qsim_plan::release_staged() {
    delete staged;
    staged = nullptr;
}

int qsim_plan::nsweeps() const {
    if (mode == QSIM_FUSE_STAGED) return qsim::staged_nsweeps(*this);
    if (mode == QSIM_FUSE_TC) return qsim::tc_nsweeps(*this);
    return int(blocks.size());
}
