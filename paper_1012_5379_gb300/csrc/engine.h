// Host engine: problem handles, problem groups and the solve drivers.
#pragma once
#include <string>
#include <vector>

#include "../../include/helm.h"
#include "helm_internal.h"

namespace helm {

// Thread-local last error text (capi.cpp).
void set_error(const std::string& msg);

struct HostLevel {
  int n = 0, P = 0;
  size_t np = 0;            // P^d
  int ntiles = 0;           // marching tiles per problem
  int nflat = 0;            // flat-kernel tiles per problem
  void* b = nullptr;
  void* xa = nullptr;
  void* xb = nullptr;
  void* r0 = nullptr;
  void* p[SMAX] = {nullptr, nullptr, nullptr, nullptr};
  void* coef = nullptr;     // 3n complex (a | d | c) in the preconditioner precision
  double2* coef64 = nullptr;// the same in FP64
  float* phi = nullptr;     // padded phi or nullptr
  double phic = 0.0;
  void* sc = nullptr;          // SweepScalarsT<R> of the preconditioner precision
  double* part = nullptr;
};

struct Handle {
  int dim = 2, n = 0, prec = HELM_C64;
  int nu1 = 1, nu2 = 1, s = 3, coarsest = 3, restart = 0, maxit = 400, m = 0;
  double theta_beta = 0, theta_gamma = 0.5, ecs = 0.125, k = 0;
  bool has_phi = false;
  TileCfg cfg{8};
  std::vector<HostLevel> lev;
  double2* lu = nullptr;
  int* piv = nullptr;
  int lu_m = 0;
  double2* hcoef = nullptr;   // 3n FP64 coefficients of H
  // outer FGMRES storage
  size_t vs = 0;
  double2* bpad = nullptr;
  double2* xpad = nullptr;
  double2* w = nullptr;
  double2* V = nullptr;
  void* Z = nullptr;
  double2* Hm = nullptr;
  double2* g = nullptr;
  double* cs = nullptr;
  double2* sn = nullptr;
  double2* y = nullptr;
  double2* hcol = nullptr;
  double* vscale = nullptr;
  double* opart = nullptr;
  OuterState* st = nullptr;
  int chunks = 1;
  int ntiles0 = 1;
  int last_j = 0;              // outer iteration index at the last state read
  size_t bytes = 0;
  std::vector<void*> allocs;
  void* group_cache = nullptr;   // single-problem group (engine-owned)
  ~Handle();
};

int setup_handle(const helm_grid* grid, const float* phi, double k, double theta_beta, const helm_opts* opts,
                 cudaStream_t st, Handle** out);
int precond_apply(Handle* h, const void* r, void* z, int prec, cudaStream_t st);
int apply_operator(Handle* h, int which, const void* v, void* w, int prec, cudaStream_t st);
int precond_apply_noalloc(const helm_grid* grid, double k, double theta_beta, const helm_opts* opts,
                          const void* r, void* z, int prec, cudaStream_t st);
int solve_group(Handle* const* hs, int count, const double* const* b, double* const* x, double tol,
                helm_info* infos, cudaStream_t st);

}  // namespace helm
