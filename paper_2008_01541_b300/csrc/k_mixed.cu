// Mixed-precision forms of the collision-region solve (placeholder until the
// low-precision factorisations are wired in).
#include "mixed.h"
#include "solver.h"

namespace pdm {
pd_status mixed_solve(pd_solver* s, const double*, const double*, double*) {
  s->err = "precision mode not available in this build";
  return PD_ERR_INVALID_ARG;
}
void mixed_free(pd_solver*) {}
}  // namespace pdm
