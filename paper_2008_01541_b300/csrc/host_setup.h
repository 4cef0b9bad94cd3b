// Host-side setup of the localized-collision PD solver: element rest data,
// the x_1 / x_2 split, assembly of the scalar PD matrix, nested-dissection
// ordering, supernodal symbolic analysis and the multifrontal partial
// Cholesky that yields L_1, L_21 and the dense Schur complement (Section 3.2).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace pdh {

struct Input {
  int64_t n = 0, E = 0;
  const double* X = nullptr;      // [n][3]
  const int32_t* tets = nullptr;  // [E][4]
  double mu = 0, mu_prime = 0, density = 0, dt = 0;   // mu_prime: bi-phasic term (Section 5)
  double kappa = 0;                                   // PD volume term (the lambda term of Eq. 1)
  const int32_t* region = nullptr;
  int64_t m = 0;
  const int32_t* dirichlet = nullptr;
  int64_t nd = 0;
  bool numeric = true;   // false: stop after the symbolic analysis (the device forms L and Sigma_0)
};

// Sparse symmetric matrix, lower triangle, compressed by column.
struct LowerCSC {
  int64_t n = 0;
  std::vector<int64_t> colptr;
  std::vector<int32_t> row;
  std::vector<double> val;
};

struct Setup {
  // --- element data (all elements, caller order) ---
  std::vector<double> Dminv;   // [E][9] row-major 3x3
  std::vector<double> vol;     // [E]
  std::vector<int32_t> alpha, beta;  // element ids of E_alpha and E_beta
  // --- node split ---
  int64_t n = 0, n1 = 0, m = 0, nfree = 0;
  std::vector<int32_t> pos;    // node -> factor position (x_1: 0..n1-1, x_2: n1 + region idx), -1 Dirichlet
  std::vector<int32_t> node_of_pos;  // factor position -> node
  std::vector<double> mass;    // [n] lumped mass (BE only), else empty
  // --- factor of the alpha matrix, supernodal ---
  int64_t nsn = 0;
  std::vector<int32_t> sn_col0;   // [nsn+1] first factor column of each supernode
  std::vector<int64_t> sn_rowptr; // [nsn+1] into rows
  std::vector<int32_t> rows;      // off-diagonal row positions (may be >= n1: x_2 rows)
  std::vector<int64_t> sn_valptr; // [nsn+1] into Lval; panel is (nc+nr) x nc column-major
  std::vector<double> Lval;       // diag block holds L_ss^-1 (lower), then L_rs (empty unless numeric)
  std::vector<int32_t> sn_parent; // parent supernode, -1 = the x_2 root
  std::vector<int32_t> sn_level;  // height above the leaves
  int64_t nlevels = 0;
  int64_t nnzL = 0;
  double factor_flops = 0;
  LowerCSC A;                     // the alpha matrix (lower, factor positions; kept unless numeric)
  // --- dense collision-region block ---
  std::vector<double> Sigma0;     // [m][m] = Sigma_alpha + A22^beta (+ M_2/dt^2) (empty unless numeric)
  LowerCSC B22;                   // A22^beta (+ M_2/dt^2), region indices, full symmetric pattern
  // --- gather maps: for each target, the element-vertex slots (e*4 + a) ---
  std::vector<int64_t> ga_ptr; std::vector<int32_t> ga_slot;  // alpha -> free positions [nfree]
  std::vector<int64_t> gb_ptr; std::vector<int32_t> gb_slot;  // beta  -> region idx [m]
  std::vector<int64_t> gall_ptr; std::vector<int32_t> gall_slot; // all -> nodes [n]
  double ms_total = 0;
  std::string log;
};

// Returns 0 on success; otherwise a pd_status code with *err filled.
int build(const Input& in, Setup& out, std::string* err);

}  // namespace pdh
