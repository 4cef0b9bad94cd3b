// Mixed-precision and PCG forms of the collision-region solve H u = g.
#pragma once
#include "pd.h"
struct pd_solver;
namespace pdm {
pd_status mixed_solve(pd_solver* s, const double* g, const double* u0, double* u);
// The two halves of mixed_solve: the refactorisation for the current contacts
// (on s->stream) and the refined solve with that factor.
pd_status mixed_factor(pd_solver* s);
pd_status mixed_iterate(pd_solver* s, const double* g, const double* u0, double* u);
void mixed_free(pd_solver* s);
// q = Sigma_0 p (3 right-hand sides) from Sigma_0's FP32 head + tail pair in
// double-float arithmetic (the residual product, FP64-accurate); false when
// the low-precision state does not exist (the FP64 form).
bool sigma_product(pd_solver* s, const double* p, double* q);
// the kept Sigma_0 u of the last solve no longer matches its buffer
void forget_sigma_product(pd_solver* s);
// z = M0^-1 r with the contact-free low-precision factor of Sigma_0.
pd_status apply_free(pd_solver* s, const double* r, double* z);
void mixed_invalidate(pd_solver* s);
// the contact nodes changed: the nested form's fixed part is rebuilt on next use
void mixed_nested_changed(pd_solver* s);
}  // namespace pdm
