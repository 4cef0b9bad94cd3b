// The C ABI (include/pd.h): solver state on the device and the orchestration
// of Algorithm 1 (Section 3.4) over the kernels of k_local.cu, k_sparse.cu,
// k_dense.cu and k_mixed.cu.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <queue>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "host_setup.h"
#include "setup_dev.h"
#include "kernels.h"
#include "mixed.h"
#include "mlp.h"
#include "pd.h"
#include "solver.h"

using pdk::SparseFactor;

namespace {

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

// ----------------------------------------------------------------- helpers
#define CK(call)                                                           \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess) {                                               \
      s->err = std::string(#call) + ": " + cudaGetErrorString(e_);          \
      return e_ == cudaErrorMemoryAllocation ? PD_ERR_OOM : PD_ERR_CUDA;   \
    }                                                                      \
  } while (0)

template <class T>
static cudaError_t dalloc(pd_solver* s, T** p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
  if (e == cudaSuccess) s->allocs.push_back((void*)*p);
  return e;
}

template <class T>
static cudaError_t dupload(pd_solver* s, T** p, const T* h, size_t n) {
  cudaError_t e = dalloc(s, p, n);
  if (e != cudaSuccess) return e;
  if (n) e = cudaMemcpy(*p, h, n * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

// ---- claim order of the sparse substitution tasks
// The persistent substitution kernels claim tasks in list order and wait for
// a claimed task's inputs, so a task whose inputs are late holds its CTA.
// The list is therefore the start order of a list schedule simulated on the
// host: `nw` workers (the resident CTAs), each task's duration estimated from
// its nonzero entries, and among the ready tasks the one with the longest
// remaining path to the end first.  A task starts in the simulation only
// after its inputs have finished, so the order stays topological (a task
// waits only for tasks earlier in the list, which running CTAs hold).
// Dependencies go through group nodes of zero duration: group g waits for
// `pred` tasks and releases `succ` tasks.
struct TaskGraph {
  std::vector<double> dur;               // per task, microseconds (estimate)
  std::vector<std::vector<int>> out;     // node -> nodes it releases (tasks: 0 .. nt-1, groups after)
  std::vector<int> indeg;                // per node
  int nt = 0;
};

static std::vector<int> list_schedule(const TaskGraph& g, int nw) {
  const int nn = (int)g.indeg.size(), nt = g.nt;
  auto dur = [&](int v) { return v < nt ? g.dur[v] : 0.0; };
  // longest path from each node to a sink (reverse topological order by Kahn)
  std::vector<int> topo;
  topo.reserve(nn);
  {
    std::vector<int> deg(g.indeg);
    for (int v = 0; v < nn; ++v)
      if (deg[v] == 0) topo.push_back(v);
    for (size_t i = 0; i < topo.size(); ++i)
      for (int w : g.out[topo[i]])
        if (--deg[w] == 0) topo.push_back(w);
  }
  if ((int)topo.size() != nn) return {};   // not a DAG: keep the given order
  std::vector<double> blev(nn, 0.0);
  for (int i = nn - 1; i >= 0; --i) {
    const int v = topo[i];
    double b = 0.0;
    for (int w : g.out[v]) b = std::max(b, blev[w]);
    blev[v] = b + dur(v);
  }
  // event-driven list scheduling (groups complete the moment they are ready)
  std::vector<int> deg(g.indeg);
  std::priority_queue<std::pair<double, int>> ready;   // (remaining path, task)
  using Ev = std::pair<double, int>;                     // (finish time, task)
  std::priority_queue<Ev, std::vector<Ev>, std::greater<Ev>> run;
  std::vector<int> order, stack;
  order.reserve(nt);
  auto release = [&](int v) {   // v is done: release its successors
    stack.push_back(v);
    while (!stack.empty()) {
      const int u = stack.back();
      stack.pop_back();
      for (int w : g.out[u])
        if (--deg[w] == 0) {
          if (w >= nt) stack.push_back(w);
          else ready.push({blev[w], w});
        }
    }
  };
  for (int v = 0; v < nn; ++v)
    if (g.indeg[v] == 0) {
      if (v >= nt) release(v);
      else ready.push({blev[v], v});
    }
  double now = 0.0;
  int busy = 0;
  while (!ready.empty() || !run.empty()) {
    while (!ready.empty() && busy < nw) {
      const int v = ready.top().second;
      ready.pop();
      order.push_back(v);
      run.push({now + dur(v), v});
      ++busy;
    }
    if (run.empty()) break;
    const Ev e = run.top();
    run.pop();
    now = e.first;
    --busy;
    release(e.second);
  }
  if ((int)order.size() != nt) return {};
  return order;
}

static pd_status build_elemset(pd_solver* s, const pdh::Setup& h, const int32_t* tets,
                               const std::vector<int32_t>& elems, ElemSet& es) {
  const int64_t c = (int64_t)elems.size();
  es.count = c;
  std::vector<int4> t(c);
  std::vector<double> Dm(9 * c), w(c);
  for (int64_t i = 0; i < c; ++i) {
    int32_t e = elems[i];
    t[i] = make_int4(tets[4 * e], tets[4 * e + 1], tets[4 * e + 2], tets[4 * e + 3]);
    for (int q = 0; q < 9; ++q) Dm[q * c + i] = h.Dminv[9 * (int64_t)e + q];
    w[i] = 2.0 * (s->mu + s->mu_prime + s->kappa) * h.vol[e];
  }
  CK(dupload(s, &es.tets, t.data(), c));
  CK(dupload(s, &es.Dm, Dm.data(), 9 * c));
  CK(dupload(s, &es.w, w.data(), c));
  CK(dalloc(s, &es.fe, 12 * c));
  return PD_OK;
}

static pd_status upload_gather(pd_solver* s, ElemSet& es, int64_t nt, const std::vector<int64_t>& ptr,
                               const std::vector<int32_t>& slot) {
  es.nt = nt;
  CK(dupload(s, &es.gptr, ptr.data(), ptr.size()));
  CK(dupload(s, &es.gslot, slot.data(), slot.size()));
  return PD_OK;
}

// ----------------------------------------------------------------- timing
void pd_solver::tbegin(int phase) {
  if (!opt.timing) return;
  if (ev_used + 2 > (int)events.size()) {
    for (int i = 0; i < 64; ++i) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      events.push_back(e);
    }
  }
  cudaEventRecord(events[ev_used], stream);
  marks.push_back({phase, ev_used});
  ev_used += 2;
}

void pd_solver::tend() {
  if (!opt.timing || marks.empty()) return;
  cudaEventRecord(events[marks.back().second + 1], stream);
}

void pd_solver::tcollect(double* out /*[9]*/) {
  for (int i = 0; i < 9; ++i) out[i] = 0.0;
  // phase 7 (network inference) is reported inside phase 4; phase 8 (the
  // refactorisation) both inside phase 4 and on its own
  if (!opt.timing) return;
  cudaStreamSynchronize(stream);
  cudaStreamSynchronize(fstream);
  for (auto& mk : marks) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, events[mk.second], events[mk.second + 1]);
    out[mk.first == 7 || mk.first == 8 ? 4 : mk.first] += ms;
    if (mk.first == 8) out[8] += ms;
  }
  marks.clear();
  ev_used = 0;
}

// ----------------------------------------------------------------- the region solve
// H = Sigma_0 + C_22; factor; solve H u = g (Algorithm 1, 4.3 and 4.5).
pd_status pd_solver::region_solve(const double* g_dev, const double* u0_dev, double* u_dev) {
  pd_status r = region_solve_core(g_dev, u0_dev, u_dev);
  if (r != PD_OK) return r;
  if (net) {
    r = pdn::after_solve(this, u_dev);
    if (r != PD_OK) return r;
  }
  cudaMemcpyAsync(u_last, u_dev, sizeof(double) * 3 * m, cudaMemcpyDeviceToDevice, stream);
  return PD_OK;
}

pd_status pd_solver::region_solve_core(const double* g_dev, const double* u0_dev, double* u_dev) {
  pd_solver* s = this;
  // warm start of the PCG form (Section 3.3 solve with a learned or previous guess)
  if (precision == PD_PCG_WARM && !u0_dev && warm_source != 0) {
    if (warm_source == 2 && net) {
      tbegin(7);
      pd_status r = pdn::before_solve(this, g_dev, u0);
      tend();
      if (r != PD_OK) return r;
      u0_dev = u0;
    } else if (warm_source == 1) {
      cudaMemcpyAsync(u0, u_last, sizeof(double) * 3 * m, cudaMemcpyDeviceToDevice, stream);
      u0_dev = u0;
    } else if (warm_source == 3) {
      tbegin(7);
      pd_status r = pdm::apply_free(this, g_dev, u0);
      tend();
      if (r != PD_OK) return r;
      u0_dev = u0;
    }
  } else if (net && mlp_recording) {
    pd_status r = pdn::before_solve(this, g_dev, nullptr);
    if (r != PD_OK) return r;
  }
  if (!prefactored) {
    pd_status r = refactor();
    if (r != PD_OK) return r;
  }
  prefactored = false;
  CK(cudaStreamWaitEvent(stream, ev_fac, 0));
  if (precision == PD_FP64) {
    tbegin(4);
    pdk::chol_solve_fp64_tasks(H, mp, Linv, g_dev, u_dev, m, work, trsv_cnt, status, stream,
                               nested ? d_perm : nullptr);
    tend();
    last_refine = 0;
    last_residual = -1.0;   // the direct FP64 solve measures none
    return PD_OK;
  }
  mixed_escalate = false;
  pd_status r = pdm::mixed_iterate(this, g_dev, u0_dev, u_dev);
  if (r == PD_OK || !mixed_escalate || !precision_fallback || nested) return r;
  // Precision escalation: the low-precision factor lost a pivot or its
  // refinement did not reach tol; this system is factored and solved in FP64
  // (H from Sigma_0 and the same springs), and the next refactorisation is
  // low precision again.  A failing FP64 pivot is reported by the step's
  // status check, as in the FP64 form.
  const int low = precision;
  precision = PD_FP64;
  r = refactor();
  if (r == PD_OK) {
    CK(cudaStreamWaitEvent(stream, ev_fac, 0));
    tbegin(4);
    pdk::chol_solve_fp64_tasks(H, mp, Linv, g_dev, u_dev, m, work, trsv_cnt, status, stream, nullptr);
    tend();
    ++precision_fallbacks;
    last_residual = -1.0;
  }
  pdm::forget_sigma_product(this);   // u now comes from the FP64 solve
  precision = low;
  return r;
}

// Algorithm 1, 4.3: H = Sigma_0 + C_22 for the current springs, and its
// factorisation, issued on the factor stream once everything issued so far on
// the solver stream (springs, positions, the previous solve's use of the
// factor) is done.  The solve waits for ev_fac, so the factorisation of the
// first inner iteration can run during the alpha local step and the forward
// substitution, which it does not depend on.
pd_status pd_solver::refactor() {
  pd_solver* s = this;
  CK(cudaEventRecord(ev_in, stream));
  CK(cudaStreamWaitEvent(fstream, ev_in, 0));
  cudaStream_t main_stream = stream;
  stream = fstream;   // the factor kernels and their timing marks go to the factor stream
  pd_status r = PD_OK;
  if (precision == PD_FP64 && nested) {
    const int64_t off = 64 * (int64_t)nk0, ntr = mp - off;
    tbegin(2);
    pdk::block_copy(H, mp, off, Sp, ntr, true, stream);
    pdk::contact_scatter(k, c_idx, c_w, c_s, H, mp, stream, pdk::CSLOTS, d_perm);
    tend();
    tbegin(8);
    pdk::cholesky_fp64(H, mp, Linv, status, stream, &la, nk0, (int)(mp / 64));
    tend();
  } else if (precision == PD_FP64) {
    tbegin(2);
    pdk::copy_sigma(Sigma0, m, H, mp, stream);
    pdk::contact_scatter(k, c_idx, c_w, c_s, H, mp, stream);
    tend();
    tbegin(8);
    pdk::cholesky_fp64(H, mp, Linv, status, stream, &la);
    tend();
  } else {
    r = pdm::mixed_factor(this);
  }
  stream = main_stream;
  cudaError_t e = cudaEventRecord(ev_fac, fstream);
  if (r == PD_OK && e != cudaSuccess) {
    err = std::string("CUDA: ") + cudaGetErrorString(e);
    r = PD_ERR_CUDA;
  }
  return r;
}

// ----------------------------------------------------------------- C ABI
extern "C" {

static thread_local std::string g_setup_error;

pd_status pd_setup(const pd_mesh* mesh, const pd_material* mat, double dt, const int32_t* region, int64_t m,
                   const int32_t* dirichlet, int64_t nd, const pd_options* opts, pd_solver** out) {
  double t0 = now_ms();
  if (out) *out = nullptr;
  g_setup_error.clear();
  if (!mesh || !mat || !out || !mesh->rest_pos || !mesh->tets || (!region && m > 0) || (!dirichlet && nd > 0) ||
      nd < 0 || m < 0 || !(dt >= 0) || !std::isfinite(dt)) {
    g_setup_error = "invalid argument";
    return PD_ERR_INVALID_ARG;
  }
  pd_solver* s = nullptr;
  try {
    s = new pd_solver();
  } catch (...) {
    g_setup_error = "host allocation failed";
    return PD_ERR_OOM;
  }
  if (opts) s->opt = *opts;
  if (s->opt.tol <= 0) s->opt.tol = 1e-10;
  if (s->opt.max_refine <= 0) s->opt.max_refine = 50;
  if (s->opt.inner_iters <= 0) s->opt.inner_iters = 1;
  if (s->opt.precision < PD_FP64 || s->opt.precision > PD_PCG_WARM) {
    g_setup_error = "unknown precision";
    delete s;
    return PD_ERR_INVALID_ARG;
  }
  s->precision = s->opt.precision;
  s->mu = mat->mu; s->density = mat->density; s->dt = dt;
  if (!(mat->mu_prime >= 0) || !std::isfinite(mat->mu_prime) ||
      (mat->mu_prime > 0 && (!(mat->sigma_min >= 0) || !(mat->sigma_max >= mat->sigma_min) ||
                             !std::isfinite(mat->sigma_min)))) {
    g_setup_error = "strain limit needs mu_prime >= 0 and 0 <= sigma_min <= sigma_max";
    delete s;
    return PD_ERR_INVALID_ARG;
  }
  if (!(mat->kappa >= 0) || !std::isfinite(mat->kappa) ||
      (mat->kappa > 0 && (!(mat->det_min > 0) || !(mat->det_max >= mat->det_min) || !std::isfinite(mat->det_min)))) {
    g_setup_error = "volume term needs kappa >= 0 and 0 < det_min <= det_max";
    delete s;
    return PD_ERR_INVALID_ARG;
  }
  s->mu_prime = mat->mu_prime;
  s->kappa = mat->kappa;
  const double wsum = mat->mu + mat->mu_prime + mat->kappa;
  if (mat->mu_prime > 0) {
    s->sl.frac = mat->mu_prime / wsum;
    s->sl.lo = mat->sigma_min;
    s->sl.hi = mat->sigma_max;
  }
  if (mat->kappa > 0) {
    s->sl.vfrac = mat->kappa / wsum;
    s->sl.vlo = mat->det_min;
    s->sl.vhi = mat->det_max;
  }
  pdh::Input in;
  in.n = mesh->n_nodes; in.E = mesh->n_tets; in.X = mesh->rest_pos; in.tets = mesh->tets;
  in.mu = mat->mu; in.mu_prime = mat->mu_prime; in.kappa = mat->kappa; in.density = mat->density; in.dt = dt;
  in.region = region; in.m = m; in.dirichlet = dirichlet; in.nd = nd;
  in.numeric = false;   // L and Sigma_0 are formed on the device (upload)
  pdh::Setup h;
  std::string err;
  int st;
  try {
    st = pdh::build(in, h, &err);
  } catch (...) {
    st = PD_ERR_OOM;
    err = "host allocation failed during setup";
  }
  if (st) {
    g_setup_error = err;
    delete s;
    return (pd_status)st;
  }
  pd_status rs = s->upload(h, in);
  if (rs != PD_OK) {
    g_setup_error = s->err;
    pd_destroy(s);
    return rs;
  }
  s->stats.setup_ms = now_ms() - t0;
  char nb[64];
  std::snprintf(nb, sizeof nb, " | device numeric %.0f ms", s->numeric_ms);
  s->setup_log = h.log + nb;
  *out = s;
  return PD_OK;
}

pd_status pd_set_dirichlet(pd_solver* s, const double* pos) {
  if (!s) return PD_ERR_INVALID_ARG;
  if (!pos && s->nd > 0) { s->err = "pos is NULL"; return PD_ERR_INVALID_ARG; }
  for (int64_t i = 0; i < 3 * s->nd; ++i)
    if (!std::isfinite(pos[i])) { s->err = "non-finite Dirichlet position"; return PD_ERR_INVALID_ARG; }
  if (s->nd > 0) CK(cudaMemcpyAsync(s->dpos, pos, sizeof(double) * 3 * s->nd, cudaMemcpyHostToDevice, s->stream));
  s->dirichlet_pending = true;
  return PD_OK;
}

// Springs are stored with pdk::CSLOTS node slots; `ns` is the caller's slot count.
static pd_status set_contacts_slots(pd_solver* s, int64_t k, int ns, const int32_t* nodes, const double* w,
                                    const double* target, const double* stiffness) {
  if (!s) return PD_ERR_INVALID_ARG;
  if (k < 0 || (k > 0 && (!nodes || !w || !target || !stiffness))) { s->err = "invalid contact arrays"; return PD_ERR_INVALID_ARG; }
  constexpr int NS = pdk::CSLOTS;
  std::vector<int32_t> idx((size_t)NS * k, -1);
  std::vector<double> ww((size_t)NS * k, 0.0);
  for (int64_t j = 0; j < k; ++j) {
    if (!std::isfinite(stiffness[j])) { s->err = "non-finite stiffness"; return PD_ERR_INVALID_ARG; }
    for (int a = 0; a < 3; ++a)
      if (!std::isfinite(target[3 * j + a])) { s->err = "non-finite target"; return PD_ERR_INVALID_ARG; }
    for (int a = 0; a < ns; ++a) {
      int32_t v = nodes[(int64_t)ns * j + a];
      const double wa = w[(int64_t)ns * j + a];
      if (v < 0) {
        if (wa != 0.0) { s->err = "unused contact slot with nonzero weight"; return PD_ERR_INVALID_ARG; }
        continue;
      }
      if (v >= s->n || s->region_index[v] < 0) {
        s->err = "contact " + std::to_string(j) + " names node " + std::to_string(v) + " outside the region";
        return PD_ERR_CONTACT_OUTSIDE_REGION;
      }
      if (s->nested && wa != 0.0 && !s->contact_ok[s->region_index[v]]) {
        s->err = "contact " + std::to_string(j) + " names node " + std::to_string(v) +
                 ", which is not one of the contact nodes";
        return PD_ERR_CONTACT_OUTSIDE_REGION;
      }
      if (!std::isfinite(wa)) { s->err = "non-finite weight"; return PD_ERR_INVALID_ARG; }
      idx[(size_t)NS * j + a] = s->region_index[v];
      ww[(size_t)NS * j + a] = wa;
    }
  }
  if (k > s->kcap) {
    int64_t cap = std::max<int64_t>(k, 2 * s->kcap);
    int32_t* ni; double *nw, *nt, *nsf;
    CK(cudaMalloc(&ni, sizeof(int32_t) * NS * cap));
    CK(cudaMalloc(&nw, sizeof(double) * NS * cap));
    CK(cudaMalloc(&nt, sizeof(double) * 3 * cap));
    CK(cudaMalloc(&nsf, sizeof(double) * cap));
    cudaFree(s->c_idx); cudaFree(s->c_w); cudaFree(s->c_t); cudaFree(s->c_s);
    s->c_idx = ni; s->c_w = nw; s->c_t = nt; s->c_s = nsf;
    s->kcap = cap;
  }
  if (k > 0) {
    CK(cudaMemcpyAsync(s->c_idx, idx.data(), sizeof(int32_t) * NS * k, cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(s->c_w, ww.data(), sizeof(double) * NS * k, cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(s->c_t, target, sizeof(double) * 3 * k, cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(s->c_s, stiffness, sizeof(double) * k, cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));  // host arrays may be freed by the caller on return
  }
  s->k = k;
  return PD_OK;
}

pd_status pd_set_contacts(pd_solver* s, int64_t k, const int32_t* nodes, const double* w, const double* target,
                          const double* stiffness) {
  return set_contacts_slots(s, k, 4, nodes, w, target, stiffness);
}

pd_status pd_set_contact_pairs(pd_solver* s, int64_t k, const int32_t* nodes, const double* w, const double* target,
                               const double* stiffness) {
  return set_contacts_slots(s, k, 8, nodes, w, target, stiffness);
}

pd_status pd_step(pd_solver* s, int outer_iters, pd_contact_cb cb, void* user) {
  if (!s || outer_iters < 0) return PD_ERR_INVALID_ARG;
  return s->step(outer_iters, cb, user);
}

pd_status pd_get_positions(const pd_solver* cs, double* out) {
  pd_solver* s = const_cast<pd_solver*>(cs);
  if (!s || !out) return PD_ERR_INVALID_ARG;
  CK(cudaMemcpyAsync(out, s->x, sizeof(double) * 3 * s->n, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return PD_OK;
}

pd_status pd_get_positions_dev(const pd_solver* cs, double* out) {
  pd_solver* s = const_cast<pd_solver*>(cs);
  if (!s || !out) return PD_ERR_INVALID_ARG;
  CK(cudaMemcpyAsync(out, s->x, sizeof(double) * 3 * s->n, cudaMemcpyDeviceToDevice, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return PD_OK;
}

pd_status pd_get_state(const pd_solver* cs, double* x, double* v) {
  pd_solver* s = const_cast<pd_solver*>(cs);
  if (!s || !x) return PD_ERR_INVALID_ARG;
  CK(cudaMemcpyAsync(x, s->x, sizeof(double) * 3 * s->n, cudaMemcpyDeviceToHost, s->stream));
  if (v) CK(cudaMemcpyAsync(v, s->v, sizeof(double) * 3 * s->n, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return PD_OK;
}

pd_status pd_set_state(pd_solver* s, const double* x, const double* v) {
  if (!s || !x) return PD_ERR_INVALID_ARG;
  for (int64_t i = 0; i < 3 * s->n; ++i)
    if (!std::isfinite(x[i]) || (v && !std::isfinite(v[i]))) { s->err = "non-finite state"; return PD_ERR_INVALID_ARG; }
  CK(cudaMemcpyAsync(s->x, x, sizeof(double) * 3 * s->n, cudaMemcpyHostToDevice, s->stream));
  if (v) CK(cudaMemcpyAsync(s->v, v, sizeof(double) * 3 * s->n, cudaMemcpyHostToDevice, s->stream));
  else CK(cudaMemsetAsync(s->v, 0, sizeof(double) * 3 * s->n, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return PD_OK;
}

pd_status pd_get_stats(const pd_solver* s, pd_stats* out) {
  if (!s || !out) return PD_ERR_INVALID_ARG;
  *out = s->stats;
  out->starts_rejected = s->starts_rejected;
  out->precision_fallbacks = s->precision_fallbacks;
  return PD_OK;
}

const char* pd_last_error(const pd_solver* s) {
  if (!s) return g_setup_error.c_str();
  return s->err.c_str();
}

void pd_destroy(pd_solver* s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  if (s->fstream) cudaStreamSynchronize(s->fstream);
  if (s->la.side) cudaStreamSynchronize(s->la.side);
  for (void* p : s->allocs) cudaFree(p);
  cudaFree(s->c_idx); cudaFree(s->c_w); cudaFree(s->c_t); cudaFree(s->c_s);
  cudaFree(s->det_a); cudaFree(s->det_b); cudaFree(s->det_sph);
  cudaFree(s->tri_prox); cudaFree(s->tri_idx); cudaFree(s->tri_xr); cudaFree(s->tri_bnd);
  cudaFree(s->Sp);
  if (s->x2_host) cudaFreeHost(s->x2_host);
  if (s->status_h) cudaFreeHost(s->status_h);
  pdm::mixed_free(s);
  pdn::free_net(s);
  for (auto e : s->la.ev_panel) cudaEventDestroy(e);
  for (auto e : s->la.ev_rest) cudaEventDestroy(e);
  if (s->la.side) cudaStreamDestroy(s->la.side);
  if (s->fstream) cudaStreamDestroy(s->fstream);
  if (s->ev_in) cudaEventDestroy(s->ev_in);
  if (s->ev_fac) cudaEventDestroy(s->ev_fac);
  for (auto e : s->events) cudaEventDestroy(e);
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
  delete s;
}

pd_status pd_local_step(pd_solver* s, const double* x, double* R_out, double* f_out) {
  if (!s || !x) return PD_ERR_INVALID_ARG;
  pd_status r = s->ensure_all_elements();
  if (r != PD_OK) return r;
  double *xd = nullptr, *Rd = nullptr, *fd = nullptr;
  CK(cudaMalloc(&xd, sizeof(double) * 3 * s->n));
  CK(cudaMalloc(&fd, sizeof(double) * 3 * s->n));
  if (R_out) CK(cudaMalloc(&Rd, sizeof(double) * 9 * s->E));
  CK(cudaMemcpyAsync(xd, x, sizeof(double) * 3 * s->n, cudaMemcpyHostToDevice, s->stream));
  pdk::polar_forces(s->all.count, s->all.tets, s->all.Dm, s->all.w, xd, s->all.fe, Rd, s->stream, &s->sl);
  pdk::gather_forces(s->n, s->all.gptr, s->all.gslot, s->all.fe, fd, nullptr, nullptr, nullptr, nullptr,
                     nullptr, 0, s->stream);
  CK(cudaGetLastError());
  if (f_out) CK(cudaMemcpyAsync(f_out, fd, sizeof(double) * 3 * s->n, cudaMemcpyDeviceToHost, s->stream));
  if (R_out) CK(cudaMemcpyAsync(R_out, Rd, sizeof(double) * 9 * s->E, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  cudaFree(xd); cudaFree(fd); if (Rd) cudaFree(Rd);
  return PD_OK;
}

pd_status pd_get_schur(const pd_solver* cs, double* out) {
  pd_solver* s = const_cast<pd_solver*>(cs);
  if (!s || !out) return PD_ERR_INVALID_ARG;
  CK(cudaMemcpyAsync(out, s->Sigma0, sizeof(double) * s->m * s->m, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return PD_OK;
}

pd_status pd_schur_solve_dev(pd_solver* s, const double* g_dev, const double* u0_dev, double* u_dev) {
  if (!s || !g_dev || !u_dev) return PD_ERR_INVALID_ARG;
  CK(cudaMemsetAsync(s->status, 0, sizeof(int) * 4, s->stream));
  pd_status r = s->region_solve(g_dev, u0_dev, u_dev);
  s->stats.refine_iters = s->last_refine;
  s->stats.residual = s->last_residual;
  if (r != PD_OK) return r;
  CK(cudaGetLastError());
  return s->check_status();
}

pd_status pd_schur_solve(pd_solver* s, const double* g, const double* u0, double* u) {
  if (!s || !g || !u) return PD_ERR_INVALID_ARG;
  CK(cudaMemcpyAsync(s->g, g, sizeof(double) * 3 * s->m, cudaMemcpyHostToDevice, s->stream));
  if (u0) CK(cudaMemcpyAsync(s->u0, u0, sizeof(double) * 3 * s->m, cudaMemcpyHostToDevice, s->stream));
  pd_status r = pd_schur_solve_dev(s, s->g, u0 ? s->u0 : nullptr, s->u2);
  double ph[9];
  s->tcollect(ph);
  s->stats.ms_contact_update = ph[2];
  s->stats.ms_factor_solve = ph[4];
  s->stats.ms_refactor = ph[8];
  if (r != PD_OK) return r;
  CK(cudaMemcpyAsync(u, s->u2, sizeof(double) * 3 * s->m, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return PD_OK;
}

static pd_status detector_buffers(pd_solver* s, int64_t nslots) {
  if (nslots > s->kcap) {
    constexpr int NS = pdk::CSLOTS;
    int32_t* ni; double *nw, *nt, *nsf;
    CK(cudaMalloc(&ni, sizeof(int32_t) * NS * nslots));
    CK(cudaMalloc(&nw, sizeof(double) * NS * nslots));
    CK(cudaMalloc(&nt, sizeof(double) * 3 * nslots));
    CK(cudaMalloc(&nsf, sizeof(double) * nslots));
    cudaFree(s->c_idx); cudaFree(s->c_w); cudaFree(s->c_t); cudaFree(s->c_s);
    s->c_idx = ni; s->c_w = nw; s->c_t = nt; s->c_s = nsf;
    s->kcap = nslots;
  }
  return PD_OK;
}

static pd_status region_list(pd_solver* s, const int32_t* nodes, int64_t n, int32_t** dev) {
  std::vector<int32_t> r(n);
  for (int64_t i = 0; i < n; ++i) {
    if (nodes[i] < 0 || nodes[i] >= s->n || s->region_index[nodes[i]] < 0) {
      s->err = "detector node " + std::to_string(nodes[i]) + " is not in the region";
      return PD_ERR_CONTACT_OUTSIDE_REGION;
    }
    if (s->nested && !s->contact_ok[s->region_index[nodes[i]]]) {
      s->err = "detector node " + std::to_string(nodes[i]) + " is not one of the contact nodes";
      return PD_ERR_CONTACT_OUTSIDE_REGION;
    }
    r[i] = s->region_index[nodes[i]];
  }
  cudaFree(*dev);
  *dev = nullptr;
  CK(cudaMalloc(dev, sizeof(int32_t) * std::max<int64_t>(n, 1)));
  if (n) CK(cudaMemcpy(*dev, r.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice));
  return PD_OK;
}

pd_status pd_set_detector_spheres(pd_solver* s, const int32_t* proxies, int64_t np, int nsph, const double* spheres,
                                  double stiffness) {
  if (!s || np < 0 || nsph < 0 || (np > 0 && !proxies) || (nsph > 0 && !spheres) || !std::isfinite(stiffness))
    return PD_ERR_INVALID_ARG;
  for (int q = 0; q < 4 * nsph; ++q)
    if (!std::isfinite(spheres[q])) { s->err = "non-finite sphere"; return PD_ERR_INVALID_ARG; }
  pd_status r = region_list(s, proxies, np, &s->det_a);
  if (r != PD_OK) return r;
  r = detector_buffers(s, np);
  if (r != PD_OK) return r;
  cudaFree(s->det_sph);
  s->det_sph = nullptr;
  CK(cudaMalloc(&s->det_sph, sizeof(double) * 4 * std::max(nsph, 1)));
  if (nsph) CK(cudaMemcpy(s->det_sph, spheres, sizeof(double) * 4 * nsph, cudaMemcpyHostToDevice));
  s->nsph = nsph;
  s->det_n = np;
  s->det_stiffness = stiffness;
  s->detector = 1;
  return PD_OK;
}

pd_status pd_set_detector_pairs(pd_solver* s, const int32_t* side_a, int64_t na, const int32_t* side_b, int64_t nb,
                                double gap, double stiffness) {
  if (!s || na < 0 || nb < 0 || (na > 0 && !side_a) || (nb > 0 && !side_b) || !(gap > 0) || !std::isfinite(stiffness))
    return PD_ERR_INVALID_ARG;
  pd_status r = region_list(s, side_a, na, &s->det_a);
  if (r != PD_OK) return r;
  r = region_list(s, side_b, nb, &s->det_b);
  if (r != PD_OK) return r;
  r = detector_buffers(s, na);
  if (r != PD_OK) return r;
  s->det_n = na;
  s->det_nb = nb;
  s->det_gap = gap;
  s->det_stiffness = stiffness;
  s->detector = 2;
  return PD_OK;
}

pd_status pd_set_detector_triangles(pd_solver* s, const int32_t* prox_a, int64_t na, const int32_t* tris_a,
                                    int64_t nta, const int32_t* prox_b, int64_t nb, const int32_t* tris_b,
                                    int64_t ntb, double gap, double rest_min, double stiffness) {
  if (!s || na < 0 || nb < 0 || nta < 0 || ntb < 0 || (na > 0 && !prox_a) || (nb > 0 && !prox_b) ||
      (nta > 0 && !tris_a) || (ntb > 0 && !tris_b) || !(gap > 0) || !(rest_min >= 0) || !std::isfinite(rest_min) ||
      !std::isfinite(gap) || !std::isfinite(stiffness))
    return PD_ERR_INVALID_ARG;
  // every proxy and triangle node must be a region node (a contact node in the nested form)
  std::vector<int32_t> prox(na + nb), tris(3 * (nta + ntb));
  auto to_region = [&](int32_t node, int32_t* out) -> pd_status {
    if (node < 0 || node >= s->n || s->region_index[node] < 0) {
      s->err = "detector node " + std::to_string(node) + " is not in the region";
      return PD_ERR_CONTACT_OUTSIDE_REGION;
    }
    if (s->nested && !s->contact_ok[s->region_index[node]]) {
      s->err = "detector node " + std::to_string(node) + " is not one of the contact nodes";
      return PD_ERR_CONTACT_OUTSIDE_REGION;
    }
    *out = s->region_index[node];
    return PD_OK;
  };
  for (int64_t i = 0; i < na + nb; ++i) {
    pd_status r = to_region(i < na ? prox_a[i] : prox_b[i - na], &prox[i]);
    if (r != PD_OK) return r;
  }
  for (int64_t i = 0; i < 3 * (nta + ntb); ++i) {
    pd_status r = to_region(i < 3 * nta ? tris_a[i] : tris_b[i - 3 * nta], &tris[i]);
    if (r != PD_OK) return r;
  }
  pd_status r = detector_buffers(s, na + nb);
  if (r != PD_OK) return r;
  cudaFree(s->tri_prox); cudaFree(s->tri_idx); cudaFree(s->tri_bnd);
  s->tri_prox = s->tri_idx = nullptr;
  s->tri_bnd = nullptr;
  CK(cudaMalloc(&s->tri_prox, sizeof(int32_t) * std::max<int64_t>(1, na + nb)));
  CK(cudaMalloc(&s->tri_idx, sizeof(int32_t) * std::max<int64_t>(1, 3 * (nta + ntb))));
  CK(cudaMalloc(&s->tri_bnd, sizeof(float4) * std::max<int64_t>(1, nta + ntb)));
  if (na + nb) CK(cudaMemcpy(s->tri_prox, prox.data(), sizeof(int32_t) * (na + nb), cudaMemcpyHostToDevice));
  if (nta + ntb) CK(cudaMemcpy(s->tri_idx, tris.data(), sizeof(int32_t) * 3 * (nta + ntb), cudaMemcpyHostToDevice));
  if (!s->tri_xr) {   // rest positions of the region nodes, region order
    std::vector<double> xr(3 * s->m);
    for (int64_t i = 0; i < s->m; ++i)
      for (int c = 0; c < 3; ++c) xr[3 * i + c] = s->X_rest_h[3 * (int64_t)s->region_h[i] + c];
    CK(cudaMalloc(&s->tri_xr, sizeof(double) * 3 * s->m));
    CK(cudaMemcpy(s->tri_xr, xr.data(), sizeof(double) * 3 * s->m, cudaMemcpyHostToDevice));
  }
  s->tri.na = na; s->tri.nb = nb; s->tri.nta = nta; s->tri.ntb = ntb;
  s->tri.prox = s->tri_prox; s->tri.tris = s->tri_idx; s->tri.xr = s->tri_xr; s->tri.bnd = s->tri_bnd;
  s->tri.gap = gap; s->tri.rest_min = rest_min; s->tri.stiffness = stiffness;
  s->det_n = na + nb;
  s->detector = 3;
  return PD_OK;
}

pd_status pd_detect(pd_solver* s) {
  if (!s) return PD_ERR_INVALID_ARG;
  if (!s->detector) { s->err = "no detector is set"; return PD_ERR_INVALID_ARG; }
  if (s->detector == 1)
    pdk::detect_spheres(s->det_n, s->det_a, s->d_region, s->x, s->nsph, s->det_sph, s->det_stiffness, s->c_idx, s->c_w,
                        s->c_t, s->c_s, s->stream);
  else if (s->detector == 2)
    pdk::detect_pairs(s->det_n, s->det_a, s->det_nb, s->det_b, s->d_region, s->x, s->det_gap, s->det_stiffness,
                      s->c_idx, s->c_w, s->c_t, s->c_s, s->stream);
  else
    pdk::detect_tris(s->tri, s->d_region, s->x, s->c_idx, s->c_w, s->c_t, s->c_s, s->stream);
  s->k = s->det_n;
  CK(cudaStreamSynchronize(s->stream));
  return PD_OK;
}

pd_status pd_get_contacts(const pd_solver* s, int64_t cap, int64_t* k, int32_t* nodes, double* w, double* target,
                          double* stiffness) {
  if (!s || !k || cap < 0 || (cap > 0 && (!nodes || !w || !target || !stiffness))) return PD_ERR_INVALID_ARG;
  *k = s->k;
  const int64_t n = std::min(cap, s->k);
  if (n <= 0) return PD_OK;
  constexpr int NS = pdk::CSLOTS;
  if (cudaStreamSynchronize(s->stream) != cudaSuccess ||
      cudaMemcpy(nodes, s->c_idx, sizeof(int32_t) * NS * n, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(w, s->c_w, sizeof(double) * NS * n, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(target, s->c_t, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(stiffness, s->c_s, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess)
    return PD_ERR_CUDA;
  for (int64_t q = 0; q < NS * n; ++q)   // region index -> node id
    if (nodes[q] >= 0) nodes[q] = s->region_h[nodes[q]];
  return PD_OK;
}

pd_status pd_clear_detector(pd_solver* s) {
  if (!s) return PD_ERR_INVALID_ARG;
  s->detector = 0;
  s->k = 0;
  return PD_OK;
}

pd_status pd_set_contact_nodes(pd_solver* s, const int32_t* nodes, int64_t np) {
  if (!s || np < 0 || (np > 0 && !nodes)) return PD_ERR_INVALID_ARG;
  const int64_t m = s->m, mp = s->mp;
  if (np == 0) {
    s->nested = false;
    pdm::mixed_nested_changed(s);
    s->contact_ok.assign(m, 1);
    s->prefactored = false;
    return PD_OK;
  }
  std::vector<char> ok(m, 0);
  for (int64_t i = 0; i < np; ++i) {
    if (nodes[i] < 0 || nodes[i] >= s->n || s->region_index[nodes[i]] < 0) {
      s->err = "contact node " + std::to_string(nodes[i]) + " is not in the region";
      return PD_ERR_CONTACT_OUTSIDE_REGION;
    }
    ok[s->region_index[nodes[i]]] = 1;
  }
  // factor positions: the nodes that never carry springs first, in region
  // order; the leading whole 64-row tiles of them form the fixed part
  std::vector<int32_t> perm(m), iperm(m);
  int64_t pos = 0;
  for (int64_t r = 0; r < m; ++r)
    if (!ok[r]) iperm[pos++] = (int32_t)r;
  const int64_t nfree_rows = pos;
  for (int64_t r = 0; r < m; ++r)
    if (ok[r]) iperm[pos++] = (int32_t)r;
  for (int64_t q = 0; q < m; ++q) perm[iperm[q]] = (int32_t)q;
  const int nk0 = (int)(nfree_rows / 64);
  const int64_t ntr = mp - 64 * (int64_t)nk0;
  if (!s->d_perm) {
    CK(dalloc(s, &s->d_perm, m));
    CK(dalloc(s, &s->d_iperm, m));
  }
  CK(cudaMemcpy(s->d_perm, perm.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(s->d_iperm, iperm.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice));
  if (s->Sp) { cudaFree(s->Sp); s->Sp = nullptr; }
  CK(cudaMalloc(&s->Sp, sizeof(double) * ntr * ntr));
  // the fixed part: partial Cholesky of P Sigma_0 P^T over the first nk0
  // tiles; the trailing block is then the contact-free Schur complement
  pdk::permute_sym(s->Sigma0, m, s->d_iperm, s->H, mp, s->stream);
  pdk::cholesky_fp64(s->H, mp, s->Linv, s->status, s->stream, &s->la, 0, nk0);
  pdk::block_copy(s->H, mp, 64 * (int64_t)nk0, s->Sp, ntr, false, s->stream);
  CK(cudaStreamSynchronize(s->stream));
  pd_status st = s->check_status();
  if (st != PD_OK) return st;
  s->contact_ok = ok;
  s->nk0 = nk0;
  s->n_fixed_rows = nfree_rows;
  s->nested = true;
  pdm::mixed_nested_changed(s);
  s->prefactored = false;
  s->k = 0;           // springs set before are dropped: they may touch other nodes
  s->detector = 0;
  return PD_OK;
}

pd_status pd_set_warm_start(pd_solver* s, int source) {
  if (!s || source < 0 || source > 3) return PD_ERR_INVALID_ARG;
  s->warm_source = source;
  return PD_OK;
}

pd_status pd_set_precision_fallback(pd_solver* s, int on) {
  if (!s) return PD_ERR_INVALID_ARG;
  s->precision_fallback = on != 0;
  return PD_OK;
}

pd_status pd_set_pcg_capacitance(pd_solver* s, int on) {
  if (!s) return PD_ERR_INVALID_ARG;
  s->pcg_capacitance = on != 0;
  return PD_OK;
}

pd_status pd_mlp_set_params(pd_solver* s, const float* params, int64_t n) {
  if (!s || !params || n != pdn::NPARAMS) {
    if (s) s->err = "expected " + std::to_string(pdn::NPARAMS) + " parameters";
    return PD_ERR_INVALID_ARG;
  }
  return pdn::set_params(s, params);
}

pd_status pd_mlp_get_params(pd_solver* s, float* params, int64_t n) {
  if (!s || !params || n != pdn::NPARAMS) return PD_ERR_INVALID_ARG;
  return pdn::get_params(s, params);
}

pd_status pd_mlp_record(pd_solver* s, int64_t max_solves) {
  if (!s || max_solves < 0) return PD_ERR_INVALID_ARG;
  return pdn::record(s, max_solves);
}

pd_status pd_mlp_train(pd_solver* s, int64_t steps, int64_t batch, double lr, uint64_t seed, double* loss) {
  if (!s || steps < 0 || !(lr > 0)) return PD_ERR_INVALID_ARG;
  return pdn::train(s, steps, batch, lr, seed, loss);
}

pd_status pd_mlp_set_loss(pd_solver* s, int kind) {
  if (!s || kind < 0 || kind > 1) return PD_ERR_INVALID_ARG;
  return pdn::set_loss(s, kind);
}

pd_status pd_mlp_eval(pd_solver* s, double* mse_net, double* mse_zero) {
  if (!s) return PD_ERR_INVALID_ARG;
  return pdn::eval(s, mse_net, mse_zero);
}

pd_status pd_mlp_loss_grad(pd_solver* s, const float* X, const float* T, int64_t B, double* loss, float* grad) {
  if (!s || !X || !T || B < 1) return PD_ERR_INVALID_ARG;
  return pdn::loss_grad(s, X, T, B, loss, grad);
}

pd_status pd_set_inner_iters(pd_solver* s, int inner_iters) {
  if (!s || inner_iters < 1) return PD_ERR_INVALID_ARG;
  s->opt.inner_iters = inner_iters;
  return PD_OK;
}

pd_status pd_set_precision(pd_solver* s, int precision) {
  if (!s || precision < PD_FP64 || precision > PD_PCG_WARM) return PD_ERR_INVALID_ARG;
  s->precision = precision;
  return PD_OK;
}

}  // extern "C"

// ----------------------------------------------------------------- solver methods
pd_status pd_solver::check_status() {
  pd_solver* s = this;
  CK(cudaMemcpyAsync(status_h, status, sizeof(int) * 4, cudaMemcpyDeviceToHost, stream));
  CK(cudaStreamSynchronize(stream));
  if (status_h[0] != 0) {
    err = "Cholesky pivot " + std::to_string(status_h[0] - 1) + " of the collision-region matrix is not positive";
    return PD_ERR_NOT_SPD;
  }
  if (status_h[1] != 0) {
    err = "a bounded device wait gave up (code " + std::to_string(status_h[1]) + ")";
    return PD_ERR_TIMEOUT;
  }
  if (status_h[2] != 0) {
    err = "refinement did not reach tol within max_refine";
    return PD_ERR_NO_CONVERGENCE;
  }
  return PD_OK;
}

pd_status pd_solver::ensure_all_elements() {
  if (all.count > 0) return PD_OK;
  std::vector<int32_t> elems(E);
  for (int64_t e = 0; e < E; ++e) elems[e] = (int32_t)e;
  pd_status r = build_elemset(this, *hostdata, tets_h.data(), elems, all);
  if (r != PD_OK) return r;
  return upload_gather(this, all, n, hostdata->gall_ptr, hostdata->gall_slot);
}

pd_status pd_solver::upload(const pdh::Setup& h, const pdh::Input& in) {
  pd_solver* s = this;
  n = in.n; E = in.E; m = in.m; nd = in.nd; n1 = h.n1; nfree = h.nfree;
  mp = ((m + 63) / 64) * 64;
  CK(cudaGetDevice(&device));
  if (opt.cuda_stream) {
    stream = (cudaStream_t)opt.cuda_stream;
    own_stream = false;
  } else {
    CK(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
    own_stream = true;
  }
  tets_h.assign(in.tets, in.tets + 4 * E);
  region_h.assign(in.region, in.region + m);
  region_index.assign(n, -1);
  for (int64_t i = 0; i < m; ++i) region_index[in.region[i]] = (int32_t)i;
  contact_ok.assign(m, 1);
  hostdata.reset(new pdh::Setup());
  hostdata->Dminv = h.Dminv;
  hostdata->vol = h.vol;
  hostdata->gall_ptr = h.gall_ptr;
  hostdata->gall_slot = h.gall_slot;
  // state
  CK(dupload(s, &x, in.X, 3 * n));
  CK(dalloc(s, &v, 3 * n));
  CK(cudaMemset(v, 0, sizeof(double) * 3 * n));
  CK(dalloc(s, &x_save, 3 * n));
  CK(dalloc(s, &v_save, 3 * n));
  CK(dalloc(s, &x_n, 3 * n));
  CK(dalloc(s, &dpos, 3 * std::max<int64_t>(nd, 1)));
  CK(dupload(s, &d_dirichlet, in.dirichlet, nd));
  CK(dupload(s, &d_region, in.region, m));
  CK(dupload(s, &d_node_of_pos, h.node_of_pos.data(), nfree));
  if (nd > 0) {
    std::vector<double> dp(3 * nd);
    for (int64_t i = 0; i < nd; ++i)
      for (int a = 0; a < 3; ++a) dp[3 * i + a] = in.X[3 * in.dirichlet[i] + a];
    CK(cudaMemcpy(dpos, dp.data(), sizeof(double) * 3 * nd, cudaMemcpyHostToDevice));
  }
  if (dt > 0) {
    std::vector<double> mh(nfree);
    for (int64_t p = 0; p < nfree; ++p) mh[p] = h.mass[h.node_of_pos[p]] / (dt * dt);
    CK(dupload(s, &mass_h2, mh.data(), nfree));
    CK(dalloc(s, &y_in, 3 * nfree));
    CK(dalloc(s, &tmp3, 3 * nfree));
  }
  // elements
  pd_status r = build_elemset(s, h, in.tets, h.alpha, alpha);
  if (r != PD_OK) return r;
  r = upload_gather(s, alpha, nfree, h.ga_ptr, h.ga_slot);
  if (r != PD_OK) return r;
  r = build_elemset(s, h, in.tets, h.beta, beta);
  if (r != PD_OK) return r;
  r = upload_gather(s, beta, m, h.gb_ptr, h.gb_slot);
  if (r != PD_OK) return r;
  // sparse factor and per-level work lists
  CK(dupload(s, &sn_col0, h.sn_col0.data(), h.sn_col0.size()));
  CK(dupload(s, &sn_rowptr, h.sn_rowptr.data(), h.sn_rowptr.size()));
  CK(dupload(s, &rows, h.rows.data(), h.rows.size()));
  CK(dupload(s, &sn_valptr, h.sn_valptr.data(), h.sn_valptr.size()));
  CK(dalloc(s, &Lval, (size_t)h.nnzL));
  {
    int64_t nl = h.nlevels;
    std::vector<std::vector<int32_t>> bylevel(nl);
    for (int64_t k2 = 0; k2 < h.nsn; ++k2) bylevel[h.sn_level[k2]].push_back((int32_t)k2);
    // dependency-counter task lists (Section 3.2 substitutions without level
    // barriers): a supernode of at most 64 columns and 128 off-diagonal rows
    // is one fused task (its diagonal block and all its rows); larger ones
    // are split into 64 x 64 tile tasks that run in parallel.
    {
      const int64_t nsn = h.nsn;
      std::vector<int32_t> col2sn(n1, -1);
      for (int64_t k2 = 0; k2 < nsn; ++k2)
        for (int32_t c = h.sn_col0[k2]; c < h.sn_col0[k2 + 1]; ++c) col2sn[c] = (int32_t)k2;
      std::vector<int64_t> tptr(1, 0);
      std::vector<int32_t> tg;
      std::vector<int> init(4 * nsn + 2, 0);
      const int64_t FIN = 0, YD = nsn, NF = 2 * nsn, ZP = 2 * nsn + 1, UD = 3 * nsn + 1, NB2 = 4 * nsn + 1;
      auto ncol = [&](int32_t sn) { return h.sn_col0[sn + 1] - h.sn_col0[sn]; };
      auto nrow = [&](int32_t sn) { return (int32_t)(h.sn_rowptr[sn + 1] - h.sn_rowptr[sn]); };
      // distinct supernodes owning rows [r0, r1) of sn's off-diagonal block
      // (each of the `mult` tasks sharing the list signals every target once)
      auto targets = [&](int32_t sn, int32_t r0, int32_t r1, int mult) {
        int32_t last = -1;
        for (int32_t r = r0; r < r1; ++r) {
          const int32_t row = h.rows[h.sn_rowptr[sn] + r];
          if (row >= n1) break;                 // rows ascend; x_2 rows need no signal
          const int32_t a = col2sn[row];
          if (a != last) { tg.push_back(a); init[FIN + a] += mult; last = a; }
        }
        tptr.push_back((int64_t)tg.size());
        return (int)(tptr.size() - 2);
      };
      constexpr int KD = 0, KO = 1 << 29, KF = 2 << 29;
      // rows of the largest fused task: 256 measured the same, 512 and no
      // limit slower (serial row blocks on the tree's critical path)
      constexpr int kFusedRows = 128;
      std::vector<int4> fd, fo, ff;   // per level: diag tiles, off tiles, fused
      std::vector<int4> ft, bt;
      for (int64_t l = 0; l < nl; ++l) {
        fd.clear(); fo.clear(); ff.clear();
        for (int32_t sn : bylevel[l]) {
          const int32_t nc = ncol(sn), nr = nrow(sn);
          if (nc <= 64 && nr <= kFusedRows) {
            ff.push_back(make_int4(sn | KF, 0, 0, targets(sn, 0, nr, 1)));
            init[UD + sn] = 1;
            continue;
          }
          for (int32_t rb = 0; rb < nc; rb += 64)
            for (int32_t cb = 0; cb <= rb; cb += 64) {
              fd.push_back(make_int4(sn | KD, rb, cb, 0));
              init[YD + sn]++; init[UD + sn]++;
            }
          for (int32_t rb = 0; rb < nr; rb += 64) {
            const int ti = targets(sn, rb, std::min(nr, rb + 64), (nc + 63) / 64);
            for (int32_t cb = 0; cb < nc; cb += 64) {
              fo.push_back(make_int4(sn | KO, rb, cb, ti));
              init[ZP + sn]++; init[UD + sn]++;   // backward: every tile of sn adds into u_sn
            }
          }
        }
        ft.insert(ft.end(), fd.begin(), fd.end());
        ft.insert(ft.end(), ff.begin(), ff.end());
        ft.insert(ft.end(), fo.begin(), fo.end());
      }
      // backward: the same tasks, levels descending; off tiles, fused, diag tiles
      {
        std::vector<std::vector<int4>> lo(nl), lf(nl), ld(nl);
        for (const int4& t : ft) {
          const int32_t sn = t.x & 0x1fffffff, kind = t.x & (3 << 29);
          const int32_t l = h.sn_level[sn];
          (kind == KO ? lo : kind == KF ? lf : ld)[l].push_back(t);
        }
        for (int64_t l = nl - 1; l >= 0; --l) {
          bt.insert(bt.end(), lo[l].begin(), lo[l].end());
          bt.insert(bt.end(), lf[l].begin(), lf[l].end());
          bt.insert(bt.end(), ld[l].begin(), ld[l].end());
        }
      }
      init[NF] = 0; init[NB2] = 0;
      // claim order: the start order of a simulated list schedule (see list_schedule)
      {
        const int nwf = pdk::sparse_grid(true), nwb = pdk::sparse_grid(false);
        auto entries = [&](const int4& t) -> double {
          const int32_t sn = t.x & 0x1fffffff, kind = t.x & (3 << 29), nc = ncol(sn), nr = nrow(sn);
          if (kind == KF) return 0.5 * nc * (nc + 1.0) + (double)nr * nc;
          const double cols = std::min(64, nc - t.z);
          if (kind == KD) {
            const double rws = std::min(64, nc - t.y);
            return t.y == t.z ? 0.5 * rws * (rws + 1.0) : rws * cols;
          }
          return std::min(64, nr - t.y) * cols;
        };
        auto reorder = [&](std::vector<int4>& tl, bool fwd) {
          TaskGraph gr;
          const int nt = (int)tl.size();
          gr.nt = nt;
          const int nn = nt + 2 * (int)nsn;
          gr.dur.resize(nt);
          gr.out.assign(nn, {});
          gr.indeg.assign(nn, 0);
          auto edge = [&](int a, int b) { gr.out[a].push_back(b); ++gr.indeg[b]; };
          // fwd: group A(s) = FIN (the inputs of every task of s)
          // bwd: group A(s) = UD (s's u done: every task of s)
          auto A = [&](int32_t sn) { return nt + sn; };
          for (int i = 0; i < nt; ++i) {
            const int4& t = tl[i];
            const int32_t sn = t.x & 0x1fffffff, kind = t.x & (3 << 29);
            gr.dur[i] = 3.0 + 5.0 * entries(t) / 4096.0;   // us: a traced run gave ~8 us per full off tile, ~6.7 per diagonal tile, ~5 per fused task
            auto each_target = [&](auto fn) {
              for (int64_t q = tptr[t.w]; q < tptr[t.w + 1]; ++q) fn(tg[q]);
            };
            if (fwd) {
              edge(A(sn), i);
              if (kind != KD) each_target([&](int32_t a) { edge(i, A(a)); });
            } else {
              if (kind != KD) each_target([&](int32_t a) { edge(A(a), i); });
              edge(i, A(sn));
            }
          }
          const std::vector<int> ord = list_schedule(gr, fwd ? nwf : nwb);
          if ((int)ord.size() != nt) return;   // keep the level order
          std::vector<int4> out(nt);
          for (int k = 0; k < nt; ++k) out[k] = tl[ord[k]];
          tl.swap(out);
        };
        reorder(ft, true);
        reorder(bt, false);
      }
      CK(dupload(s, &sf_ftasks, ft.data(), ft.size()));
      CK(dupload(s, &sf_btasks, bt.data(), bt.size()));
      CK(dupload(s, &sf_tptr, tptr.data(), tptr.size()));
      CK(dupload(s, &sf_tgt, tg.data(), std::max<size_t>(tg.size(), 1)));
      CK(dupload(s, &sf_cnt_init, init.data(), init.size()));
      CK(dupload(s, &sf_cnt, init.data(), init.size()));
      sf.n_ftasks = (int64_t)ft.size(); sf.n_btasks = (int64_t)bt.size();
      sf.ftasks = sf_ftasks; sf.btasks = sf_btasks; sf.tgt_ptr = sf_tptr; sf.tgt = sf_tgt;
      sf.cnt = sf_cnt; sf.cnt_init = sf_cnt_init;
      sf.cnt_fin = FIN; sf.cnt_ydone = YD; sf.cnt_next_f = NF; sf.cnt_zpend = ZP; sf.cnt_udone = UD; sf.cnt_next_b = NB2;
      sf.grid_f = pdk::sparse_grid(true);
      sf.grid_b = pdk::sparse_grid(false);
    }
    sf.n1 = n1; sf.nfree = nfree; sf.nsn = h.nsn; sf.nlevels = nl;
    sf.col0 = sn_col0; sf.rowptr = sn_rowptr; sf.rows = rows; sf.valptr = sn_valptr; sf.L = Lval;
  }
  CK(dalloc(s, &b, 3 * nfree));
  CK(dalloc(s, &yv, 3 * nfree));
  CK(dalloc(s, &u, 3 * nfree));
  CK(dalloc(s, &z, 3 * nfree));
  // dense block
  CK(dalloc(s, &Sigma0, (size_t)m * m));
  {   // the numeric phase: L_1, L_21 and Sigma_0 (Section 3.1, Eq. 9) on the device
    std::string e2;
    const double t2 = now_ms();
    const int r2 = pdk::numeric_factor(h, Lval, Sigma0, stream, &e2);
    numeric_ms = now_ms() - t2;
    if (r2 != 0) {
      err = e2;
      return (pd_status)r2;
    }
  }
  CK(dupload(s, &b22_ptr, h.B22.colptr.data(), h.B22.colptr.size()));
  CK(dupload(s, &b22_row, h.B22.row.data(), h.B22.row.size()));
  CK(dupload(s, &b22_val, h.B22.val.data(), h.B22.val.size()));
  CK(dalloc(s, &H, (size_t)mp * mp));
  {
    int lo_prio = 0, hi_prio = 0;
    CK(cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio));
    CK(cudaStreamCreateWithPriority(&la.side, cudaStreamNonBlocking, lo_prio));
    CK(cudaStreamCreateWithPriority(&fstream, cudaStreamNonBlocking, hi_prio));
    CK(cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ev_fac, cudaEventDisableTiming));
    la.ev_panel.resize(mp / 64);
    la.ev_rest.resize(mp / 64);
    for (size_t i = 0; i < la.ev_panel.size(); ++i) {
      CK(cudaEventCreateWithFlags(&la.ev_panel[i], cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&la.ev_rest[i], cudaEventDisableTiming));
    }
  }
  CK(dalloc(s, &Linv, (size_t)mp * 64));
  CK(dalloc(s, &g, 3 * m));
  CK(dalloc(s, &u0, 3 * m));
  CK(dalloc(s, &u2, 3 * m));
  CK(dalloc(s, &Sau, 3 * m));
  CK(dalloc(s, &U2, 3 * m));
  CK(dalloc(s, &u_last, 3 * m));
  CK(cudaMemset(u_last, 0, sizeof(double) * 3 * m));
  X_rest_h.assign(in.X, in.X + 3 * n);
  CK(dalloc(s, &work, 6 * mp));
  CK(dalloc(s, &trsv_cnt, 2 + 2 * (mp / 64)));
  CK(dalloc(s, &status, 4));
  sf.status = status;
  CK(cudaMemset(status, 0, sizeof(int) * 4));
  CK(cudaMallocHost(&status_h, sizeof(int) * 4));
  CK(cudaMallocHost(&x2_host, sizeof(double) * 3 * m));
  CK(dalloc(s, &x2_dev, 3 * m));
  stats.n_nodes = n; stats.n_tets = E; stats.n_free = nfree; stats.n1 = n1; stats.m = m;
  stats.n_alpha = alpha.count; stats.n_beta = beta.count;
  stats.n_supernodes = h.nsn; stats.n_levels = h.nlevels; stats.nnz_L = h.nnzL;
  CK(cudaDeviceSynchronize());
  return PD_OK;
}

// Algorithm 1 for one time step.
pd_status pd_solver::step(int outer_iters, pd_contact_cb cb, void* user) {
  pd_solver* s = this;
  prefactored = false;
  double t0 = now_ms();
  const int64_t launches0 = pdk::g_launches;
  marks.clear();
  ev_used = 0;
  CK(cudaMemsetAsync(status, 0, sizeof(int) * 4, stream));
  CK(cudaMemcpyAsync(x_save, x, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, stream));
  CK(cudaMemcpyAsync(v_save, v, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, stream));
  if (dirichlet_pending) {
    pdk::scatter_rows(nd, d_dirichlet, dpos, x, stream);
    dirichlet_pending = false;
  }
  if (dt > 0) {
    CK(cudaMemcpyAsync(x_n, x_save, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, stream));
    // inertia target y = x_n + dt v_n, in factor order
    pdk::gather_rows(nfree, d_node_of_pos, x_save, y_in, stream);
    pdk::gather_rows(nfree, d_node_of_pos, v, tmp3, stream);
    pdk::axpby(3 * nfree, dt, tmp3, 1.0, y_in, stream);
  }
  pd_status result = PD_OK;
  int64_t inner_total = 0, refine_total = 0;
  // 4.1 detection: on the device, or through the host callback
  auto detect = [&]() -> pd_status {
    if (!cb && detector) {
      tbegin(3);
      if (detector == 1)
        pdk::detect_spheres(det_n, det_a, d_region, x, nsph, det_sph, det_stiffness, c_idx, c_w, c_t, c_s, stream);
      else if (detector == 2)
        pdk::detect_pairs(det_n, det_a, det_nb, det_b, d_region, x, det_gap, det_stiffness, c_idx, c_w, c_t, c_s,
                          stream);
      else
        pdk::detect_tris(tri, d_region, x, c_idx, c_w, c_t, c_s, stream);
      tend();
      k = det_n;
    }
    if (cb) {
      pdk::gather_rows(m, d_region, x, x2_dev, stream);
      CK(cudaMemcpyAsync(x2_host, x2_dev, sizeof(double) * 3 * m, cudaMemcpyDeviceToHost, stream));
      CK(cudaStreamSynchronize(stream));
      pd_status cr = cb(user, x2_host, this);
      if (cr != PD_OK) {
        if (err.empty()) err = "contact callback returned an error";
        return cr;
      }
    }
    return PD_OK;
  };
  for (int it = 0; it < outer_iters && result == PD_OK; ++it) {
    // the first inner iteration's detection and refactorisation read only x_2
    // and the springs, so they are issued before steps 1-3 and the factor
    // stream overlaps the alpha local step and the forward substitution
    result = detect();
    if (result != PD_OK) break;
    result = refactor();
    if (result != PD_OK) break;
    prefactored = true;
    // 1-2: R_alpha and the alpha forces f_1, f_2^(alpha) (+ x_1 inertia)
    tbegin(0);
    pdk::polar_forces(alpha.count, alpha.tets, alpha.Dm, alpha.w, x, alpha.fe, nullptr, stream, &sl);
    pdk::gather_forces(nfree, alpha.gptr, alpha.gslot, alpha.fe, b, nullptr, mass_h2, x, y_in,
                       d_node_of_pos, n1, stream);
    tend();
    // 3: forward substitution; b[n1..] becomes f~_2 = y_2
    tbegin(1);
    pdk::sparse_forward(sf, b, yv, stream);
    tend();
    double* ft2 = b + 3 * n1;
    CK(cudaMemsetAsync(U2, 0, sizeof(double) * 3 * m, stream));
    for (int j = 0; j < opt.inner_iters; ++j) {
      if (j > 0) {
        pd_status dr = detect();
        if (dr != PD_OK) { result = dr; break; }
      }
      // 4.2, 4.4: R_beta, g = f~_2 + f_2^(beta) (+ x_2 inertia) + f_2^(col)
      tbegin(3);
      pdk::polar_forces(beta.count, beta.tets, beta.Dm, beta.w, x, beta.fe, nullptr, stream, &sl);
      pdk::gather_forces(m, beta.gptr, beta.gslot, beta.fe, g, ft2, mass_h2 ? mass_h2 + n1 : nullptr, x,
                         y_in ? y_in + 3 * n1 : nullptr, d_region, m, stream);
      pdk::contact_forces(k, c_idx, c_w, c_t, c_s, d_region, x, g, stream);
      tend();
      // 4.3, 4.5: H = Sigma_alpha + A22^beta + C22; solve H u2 = g
      pd_status r = region_solve(g, nullptr, u2);
      if (r != PD_OK) { result = r; break; }
      refine_total += last_refine;
      // 4.6, 4.7: x2 += u2; f~_2 -= Sigma_alpha u2 (= Sigma_0 u2 - A22^beta u2 - M2/dt^2 u2).
      // The low-precision and PCG forms take Sigma_0 u2 from the FP32 pair their
      // residuals use (double-float, FP64-accurate, 12 instead of 8 bytes per
      // entry pair but on the FP32 pipes); the FP64 form from Sigma_0 in FP64.
      tbegin(5);
      if (precision == PD_FP64 || !pdm::sigma_product(this, u2, Sau)) pdk::symv3(Sigma0, m, u2, Sau, stream);
      pdk::spmv3(m, b22_ptr, b22_row, b22_val, u2, -1.0, Sau, stream);
      pdk::inner_update(m, u2, Sau, d_region, x, U2, ft2, stream);
      tend();
      ++inner_total;
    }
    if (result != PD_OK) break;
    // 5: backward substitution u_1 = L_1^-T (y_1 - L_21^T U_2); x_1 += u_1
    tbegin(6);
    CK(cudaMemcpyAsync(u + 3 * n1, U2, sizeof(double) * 3 * m, cudaMemcpyDeviceToDevice, stream));
    pdk::sparse_backward(sf, yv, u, z, stream);
    pdk::apply_interior(n1, u, d_node_of_pos, x, stream);
    tend();
    stats.outer_done = it + 1;
  }
  cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess && result == PD_OK) {
    err = std::string("kernel launch: ") + cudaGetErrorString(ce);
    result = PD_ERR_CUDA;
  }
  // no factor-stream work of this step may outlive it (error paths included)
  cudaStreamWaitEvent(stream, ev_fac, 0);
  if (result == PD_OK) result = check_status();
  if (result == PD_OK && dt > 0) {
    pdk::axpby(3 * n, 1.0 / dt, x, 0.0, v, stream);
    pdk::axpby(3 * n, -1.0 / dt, x_n, 1.0, v, stream);
  }
  if (result != PD_OK) {  // roll back to the state before the call
    prefactored = false;
    cudaMemcpyAsync(x, x_save, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, stream);
    cudaMemcpyAsync(v, v_save, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, stream);
    cudaStreamSynchronize(stream);
    return result;
  }
  double ph[9];
  prefactored = false;
  tcollect(ph);
  stats.ms_local_alpha = ph[0]; stats.ms_forward = ph[1]; stats.ms_contact_update = ph[2];
  stats.ms_local_beta = ph[3]; stats.ms_factor_solve = ph[4]; stats.ms_bookkeeping = ph[5];
  stats.ms_backward = ph[6]; stats.ms_refactor = ph[8];
  CK(cudaStreamSynchronize(stream));
  stats.ms_step = now_ms() - t0;
  stats.inner_done = inner_total;
  stats.kernel_launches = pdk::g_launches - launches0;
  stats.contacts = k;
  stats.refine_iters = (int)refine_total;
  stats.residual = last_residual;
  return PD_OK;
}
