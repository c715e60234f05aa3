// Adjoint-method gradients (qsim_adjoint_grad).
#include "internal.h"
#include "plan.h"

using namespace qsim;
extern "C" int qsim_adjoint_grad(const qsim_circuit *, int, int, const double *, int, const uint64_t *,
                                 const uint64_t *, const double *, double *, double *, void *) {
    return set_error(QSIM_EUNSUPPORTED, "adjoint gradient not built yet");
}
