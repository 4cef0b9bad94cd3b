// Numeric phase of the setup on the device (Section 3.1, Eq. 9): the partial
// Cholesky of the constant PD matrix with the collision-prone nodes x_2
// ordered last and never pivoted, yielding the interior factor L_1, L_21 and
// the dense Schur complement Sigma_0 = A_22 - L_21 L_21^T, in FP64.
#pragma once
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "host_setup.h"

namespace pdk {

// From the host's symbolic analysis s (ordering, supernodes, elimination
// tree, assembled matrix s.A and s.B22, built with Input::numeric = false):
// writes the supernodal factor into Lval (s.nnzL doubles on the device, the
// layout of pdh::Setup::Lval, per supernode an (nc + nr) x nc column-major
// panel, but with the off-diagonal rows multiplied by the inverse: the
// diagonal block holds L_ss^-1 (lower, zero above), the rows below
// L_rs L_ss^-1) and
// Sigma_0 into Sigma0 (m x m, column-major, both triangles).  Temporary
// device memory (the fronts) is allocated and freed here.  Returns 0, or
// a pd_status code with *err set (5: the interior matrix is not positive
// definite; 8: a CUDA call failed; 9: out of device memory).
int numeric_factor(const pdh::Setup& s, double* Lval, double* Sigma0, cudaStream_t st, std::string* err);

}  // namespace pdk
