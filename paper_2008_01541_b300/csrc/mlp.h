// Learned warm start for the PCG form of the collision-region solve: a per-node
// MLP 14 -> 256 -> 256 -> 256 -> 3 (ReLU) with BF16 weights and activations and
// FP32 accumulation, trained and evaluated with tcgen05 GEMMs.
#pragma once
#include <cstdint>
#include "pd.h"

struct pd_solver;

namespace pdn {

constexpr int IN = 14, IN_PAD = 128, HID = 256, OUT = 3, OUT_PAD = 128;
// logical parameter count: W1 [256][14] b1 [256] W2 [256][256] b2 W3 [256][256] b3 W4 [3][256] b4 [3]
constexpr int64_t NPARAMS = (int64_t)HID * IN + HID + 2 * ((int64_t)HID * HID + HID) + (int64_t)OUT * HID + OUT;

struct Net;

pd_status set_params(pd_solver* s, const float* params);
pd_status get_params(pd_solver* s, float* params);
pd_status record(pd_solver* s, int64_t max_solves);
pd_status train(pd_solver* s, int64_t steps, int64_t batch, double lr, uint64_t seed, double* loss);
pd_status eval(pd_solver* s, double* mse_net, double* mse_zero);
pd_status loss_grad(pd_solver* s, const float* X, const float* T, int64_t B, double* loss, float* grad);
// 0: mean squared error; 1: rows weighted by H_ii / mean diag(Sigma_0)
pd_status set_loss(pd_solver* s, int kind);
// Hooks around every collision-region solve.
pd_status before_solve(pd_solver* s, const double* g, double* u0 /* out, may be null */);
pd_status after_solve(pd_solver* s, const double* u);
void free_net(pd_solver* s);

}  // namespace pdn
