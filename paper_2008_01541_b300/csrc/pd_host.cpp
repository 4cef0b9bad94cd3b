// Host-only entry point: the partial Cholesky of pd_setup without a device.
#include <cstring>
#include <string>

#include "host_setup.h"
#include "pd.h"

extern "C" pd_status pd_host_schur(const pd_mesh* mesh, const pd_material* mat, double dt,
                                   const int32_t* region, int64_t m, const int32_t* dirichlet,
                                   int64_t nd, double* sigma_out, char* info, int64_t info_len) {
  if (!mesh || !mat || (!region && m > 0) || (!dirichlet && nd > 0) || (!sigma_out && m > 0)) return PD_ERR_INVALID_ARG;
  pdh::Input in;
  in.n = mesh->n_nodes; in.E = mesh->n_tets; in.X = mesh->rest_pos; in.tets = mesh->tets;
  in.mu = mat->mu; in.mu_prime = mat->mu_prime; in.kappa = mat->kappa; in.density = mat->density; in.dt = dt;
  in.region = region; in.m = m; in.dirichlet = dirichlet; in.nd = nd;
  pdh::Setup s;
  std::string err;
  int st = pdh::build(in, s, &err);
  const std::string& msg = st ? err : s.log;
  if (info && info_len > 0) {
    size_t k = std::min<size_t>(msg.size(), (size_t)info_len - 1);
    std::memcpy(info, msg.data(), k);
    info[k] = 0;
  }
  if (st) return (pd_status)st;
  std::memcpy(sigma_out, s.Sigma0.data(), sizeof(double) * m * m);
  return PD_OK;
}
