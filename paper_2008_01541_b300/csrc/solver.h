// Internal solver state behind the opaque pd_solver handle.
#pragma once
#include <cstdint>
#include <memory>
#include <string>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "host_setup.h"
#include "kernels.h"
#include "pd.h"

struct ElemSet {
  int64_t count = 0;
  int4* tets = nullptr;
  double* Dm = nullptr;   // SoA [9][count]
  double* w = nullptr;    // 2 mu Vol
  double* fe = nullptr;   // [count][4][3]
  int64_t nt = 0;
  int64_t* gptr = nullptr;
  int32_t* gslot = nullptr;
};

namespace pdm { struct MixedState; }
namespace pdn { struct Net; }

struct pd_solver {
  // configuration
  pd_options opt{};
  int precision = PD_FP64;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  double mu = 0, density = 0, dt = 0;
  double mu_prime = 0, kappa = 0;
  pdk::StrainLimit sl;   // bi-phasic and volume terms (frac = vfrac = 0: off)
  int64_t n = 0, E = 0, m = 0, nd = 0, n1 = 0, nfree = 0, mp = 0;
  std::vector<int32_t> tets_h, region_h, region_index;
  std::unique_ptr<pdh::Setup> hostdata;  // element data kept for pd_local_step
  std::string setup_log;
  double numeric_ms = 0;   // the numeric phase of the setup on the device
  // device state
  std::vector<void*> allocs;
  double *x = nullptr, *v = nullptr, *x_save = nullptr, *v_save = nullptr, *x_n = nullptr;
  double *dpos = nullptr, *mass_h2 = nullptr, *y_in = nullptr, *tmp3 = nullptr;
  int32_t *d_dirichlet = nullptr, *d_region = nullptr, *d_node_of_pos = nullptr;
  bool dirichlet_pending = false;
  ElemSet alpha, beta, all;
  // interior factor
  int32_t* sn_col0 = nullptr;
  int64_t* sn_rowptr = nullptr;
  int32_t* rows = nullptr;
  int64_t* sn_valptr = nullptr;
  double* Lval = nullptr;
  int4 *sf_ftasks = nullptr, *sf_btasks = nullptr;
  int64_t* sf_tptr = nullptr;
  int32_t* sf_tgt = nullptr;
  int *sf_cnt = nullptr, *sf_cnt_init = nullptr;
  pdk::SparseFactor sf;
  double *b = nullptr, *yv = nullptr, *u = nullptr, *z = nullptr;
  // collision-region block
  double* Sigma0 = nullptr;
  int64_t* b22_ptr = nullptr;
  int32_t* b22_row = nullptr;
  double* b22_val = nullptr;
  double *H = nullptr, *Linv = nullptr, *g = nullptr, *u0 = nullptr, *u2 = nullptr, *Sau = nullptr;
  double *U2 = nullptr, *work = nullptr, *x2_dev = nullptr;
  double* x2_host = nullptr;
  int* status = nullptr;      // [0] non-SPD column+1, [1] timeout code, [2] no convergence
  int* trsv_cnt = nullptr;    // task counters of the FP64 Schur solve
  int* status_h = nullptr;
  pdk::LookAhead la;             // side stream + events of the FP64 factorisation
  cudaStream_t fstream = nullptr;   // factor stream: 4.3 overlaps steps 1-3 of the outer iteration
  cudaEvent_t ev_in = nullptr, ev_fac = nullptr;
  bool prefactored = false;         // the factor for the current springs is issued (ev_fac)
  // nested Schur (FP64 form): region nodes that never carry springs come
  // first in the factor and their part of the factor is computed once; each
  // refactorisation covers only the trailing block from tile nk0 on
  bool nested = false;
  int nk0 = 0;
  int64_t n_fixed_rows = 0;                        // region nodes that never carry springs
  int32_t *d_perm = nullptr, *d_iperm = nullptr;   // region index <-> factor position
  double* Sp = nullptr;                            // saved trailing block (contact-free Schur complement)
  std::vector<char> contact_ok;                    // per region index: may carry springs
  pdm::MixedState* mixed = nullptr;
  pdn::Net* net = nullptr;       // learned warm start
  bool mlp_recording = false;
  int warm_source = 0;           // PD_PCG_WARM start: 0 zero, 1 previous solution, 2 network
  bool pcg_capacitance = true;   // PD_PCG_WARM: Woodbury correction of M0 for the active springs
  double* u_last = nullptr;      // [m][3] solution of the previous region solve
  std::vector<double> X_rest_h;  // rest positions (host)
  int last_refine = 0;
  int64_t starts_rejected = 0;   // PCG starts worse than zero, replaced by zero (counted)
  int64_t precision_fallbacks = 0;   // low-precision solves redone in FP64 (counted)
  bool precision_fallback = true;    // redo a failed low-precision solve in FP64
  bool mixed_escalate = false;       // set by the mixed solve: its failure may be escalated
  double last_residual = 0.0;
  // contacts (region indices)
  int64_t k = 0, kcap = 0;
  int32_t* c_idx = nullptr;
  double *c_w = nullptr, *c_t = nullptr, *c_s = nullptr;
  // device collision detection (0 = off, 1 = spheres, 2 = pairs, 3 = point-triangle)
  int detector = 0;
  int64_t det_n = 0, det_nb = 0;
  int nsph = 0;
  int32_t *det_a = nullptr, *det_b = nullptr;   // region indices
  double* det_sph = nullptr;                    // [nsph][4]
  double det_gap = 0.0, det_stiffness = 0.0;
  pdk::TriDetector tri;                         // point-triangle detector (device arrays owned here)
  int32_t *tri_prox = nullptr, *tri_idx = nullptr;
  double* tri_xr = nullptr;
  float4* tri_bnd = nullptr;
  // bookkeeping
  pd_stats stats{};
  std::string err;
  std::vector<cudaEvent_t> events;
  std::vector<std::pair<int, int>> marks;
  int ev_used = 0;

  pd_status upload(const pdh::Setup& h, const pdh::Input& in);
  pd_status step(int outer_iters, pd_contact_cb cb, void* user);
  pd_status region_solve(const double* g_dev, const double* u0_dev, double* u_dev);
  pd_status region_solve_core(const double* g_dev, const double* u0_dev, double* u_dev);
  pd_status refactor();
  pd_status check_status();
  pd_status ensure_all_elements();
  void tbegin(int phase);
  void tend();
  void tcollect(double* out);
};
