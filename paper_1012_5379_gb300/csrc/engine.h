// Host engine: problem handles, problem groups and the solve drivers.
#pragma once
#include <sstream>
#include <string>
#include <utility>
#include <array>
#include <complex>
#include <vector>

#include "../../include/helm.h"
#include "helm_internal.h"

namespace helm {

// Thread-local last error text (capi.cpp).
void set_error(const std::string& msg);

// Return the failing CUDA call's status as HELM_ENOMEM / HELM_ECUDA with its text.
#define CUDA_TRY(expr)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      std::ostringstream os_;                                                            \
      os_ << #expr << ": " << cudaGetErrorString(e_) << " (" << __FILE__ << ":" << __LINE__ << ")"; \
      set_error(os_.str());                                                              \
      return e_ == cudaErrorMemoryAllocation ? HELM_ENOMEM : HELM_ECUDA;                 \
    }                                                                                    \
  } while (0)

// Return a failing helm status.
#define TRY(expr)                 \
  do {                            \
    int r_ = (expr);              \
    if (r_ != HELM_OK) return r_; \
  } while (0)

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
  const CUtensorMap* tm = nullptr;  // TMA maps (2D complex64 grid-wide levels), device memory
  double* part = nullptr;
};

struct Handle {
  int dim = 2, n = 0, prec = HELM_C64;
  int nu1 = 1, nu2 = 1, s = 3, coarsest = 3, restart = 0, maxit = 400, m = 0;
  double theta_beta = 0, theta_gamma = 0.5, ecs = 0.125, k = 0;
  int ecs_sides = 0;              // HELM_ECS_BOTH or HELM_ECS_HIGH
  double csl_eps = 0;             // complex shift of M: L - (1 + i csl_eps) phi
  int smoother = 0;               // HELM_SMOOTHER_GMRES or HELM_SMOOTHER_POLY
  int basis = 0;                  // HELM_BASIS_AUTO, HELM_BASIS_F64 or HELM_BASIS_DF (outer Krylov basis)
  std::vector<std::array<std::complex<double>, 3>> polyw;  // Richardson weights per smoothed level
  bool has_phi = false;
  TileCfg cfg{8};
  std::vector<HostLevel> lev;
  double2* lu = nullptr;
  int* piv = nullptr;
  int lu_m = 0;
  double2* hcoef = nullptr;   // 3n FP64 coefficients of H
  float4* hcoef_df = nullptr; // the same as double-floats (hi + lo, rounded to nearest)
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
  unsigned* dcnt = nullptr;   // the multi-dot's group counters
  OuterState* st = nullptr;
  int chunks = 1;
  int ntiles0 = 1;
  int last_j = 0;              // outer iteration index at the last state read
  size_t bytes = 0;
  std::vector<void*> allocs;
  void* group_cache = nullptr;   // single-problem group (engine-owned)
  // page-locked staging of the small uploads that re-target the handle and start a
  // problem (pageable sources would make an upload wait for the stream's queued work):
  // the outer state, the coarsest LU and pivots, each level's coefficients (FP64 and
  // the preconditioner precision), at fixed offsets
  char* stage = nullptr;
  size_t stage_lu = 0, stage_piv = 0;
  std::vector<size_t> stage_coef;  // per level: FP64 block, then the level-precision block
  ~Handle();
};

int setup_handle(const helm_grid* grid, const float* phi, double k, double theta_beta, const helm_opts* opts,
                 cudaStream_t st, Handle** out);
int precond_apply(Handle* h, const void* r, void* z, int prec, cudaStream_t st);
int apply_operator(Handle* h, int which, const void* v, void* w, int prec, cudaStream_t st);
int autotune(const helm_grid* grid, const float* phi, double k, double theta_beta, const helm_opts* opts, int reps,
             const char* path, double* default_ms, double* tuned_ms, cudaStream_t st);
int precond_apply_noalloc(const helm_grid* grid, double k, double theta_beta, const helm_opts* opts,
                          const void* r, void* z, int prec, cudaStream_t st);
int multidot(int basis, const double2* V, int nvec, size_t npts, const double2* w, double2* h_host,
             cudaStream_t st);
// Problems iterated together, joining and leaving between outer iterations.
struct BatchRunner;
BatchRunner* runner_create(int prec);
void runner_destroy(BatchRunner* r);
int runner_add(BatchRunner* r, Handle* h, const double2* b_dense, double tol, cudaStream_t st);
int runner_iterate(BatchRunner* r, cudaStream_t st);
int runner_collect(BatchRunner* r, cudaStream_t st, std::vector<std::pair<Handle*, OuterState>>* done);
int runner_size(const BatchRunner* r);
int runner_finish(Handle* h, const OuterState& s, double2* x_dense, cudaStream_t st, helm_info* info);
struct Server;
int serve_start(const helm_serve_opts* opts, Server** out);
int serve_submit(Server* s, int dim, int n, double k, double theta_beta, const double* b_host, double* x_host,
                 double tol, long long* ticket);
int serve_poll(Server* s, long long ticket, helm_info* info, double* latency);
int serve_wait(Server* s, long long ticket, double timeout_s, helm_info* info, double* latency);
int serve_stats(Server* s, helm_serve_counters* out);
// Group (re)builds, V-cycle graph captures and the host seconds spent in both.
void build_stats(long long* groups, long long* graphs, double* seconds);
int serve_stop(Server* s);
int retarget_handle(Handle* h, double k, double theta_beta, cudaStream_t st);
size_t estimate_handle_bytes(int dim, int n, int prec, int s, int restart, int maxit, int coarsest);
int solve_group(Handle* const* hs, int count, const double* const* b, double* const* x, double tol,
                helm_info* infos, cudaStream_t st);

}  // namespace helm
