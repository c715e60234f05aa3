// Tensor-core fused k-qubit blocks (QSIM_FUSE_TC).
#include "internal.h"
#include "plan.h"

namespace qsim {
struct TcPlan {};
int build_tc(const qsim_circuit &, qsim_plan &) { return set_error(QSIM_EUNSUPPORTED, "tensor-core fusion not built yet"); }
int run_tc(qsim_state *, qsim_plan &) { return set_error(QSIM_EUNSUPPORTED, "tensor-core fusion not built yet"); }
int tc_nsweeps(const qsim_plan &) { return 0; }
void tc_describe(const qsim_plan &, std::string &) {}
}  // namespace qsim

void qsim_plan::release_tc() {
    delete tc;
    tc = nullptr;
}
