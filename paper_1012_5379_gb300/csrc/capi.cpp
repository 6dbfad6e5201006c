// extern "C" boundary of libhelm.so (include/helm.h).  Every entry point validates
// its arguments, catches C++ exceptions and reports failures through a status code
// and a thread-local message.
#include <cuda_runtime.h>

#include <exception>
#include <new>
#include <algorithm>
#include <vector>
#include <string>

#include <cmath>

#include "../../include/helm.h"
#include "geometry.h"
#include "engine.h"
#include "profiler.h"
#include <cstring>

namespace helm {
static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }
}  // namespace helm

using helm::Handle;

#define HELM_GUARD(...)                                   \
  try {                                                   \
    helm::set_error("");                                  \
    __VA_ARGS__                                           \
  } catch (const std::bad_alloc&) {                       \
    helm::set_error("host allocation failed");            \
    return HELM_ENOMEM;                                   \
  } catch (const std::exception& e) {                     \
    helm::set_error(e.what());                            \
    return HELM_ECUDA;                                    \
  } catch (...) {                                         \
    helm::set_error("unknown exception");                 \
    return HELM_ECUDA;                                    \
  }

struct helm_handle {
  Handle* h;
};
struct helm_server {
  helm::Server* s;
};

extern "C" {

int helm_setup(const helm_grid* grid, const float* phi, double k, double theta_beta, const helm_opts* opts,
               void* stream, helm_handle** out) {
  HELM_GUARD({
    if (!out) { helm::set_error("out must not be NULL"); return HELM_EINVAL; }
    *out = nullptr;
    Handle* h = nullptr;
    int rc = helm::setup_handle(grid, phi, k, theta_beta, opts, (cudaStream_t)stream, &h);
    if (rc != HELM_OK) return rc;
    *out = new helm_handle{h};
    return HELM_OK;
  })
}

void helm_destroy(helm_handle* h) {
  if (!h) return;
  try {
    delete h->h;
  } catch (...) {
  }
  delete h;
}

int helm_precond_apply(helm_handle* h, const void* r, void* z, int prec, void* stream) {
  HELM_GUARD({
    if (!h) { helm::set_error("NULL handle"); return HELM_EINVAL; }
    return helm::precond_apply(h->h, r, z, prec, (cudaStream_t)stream);
  })
}

int helm_apply_operator(helm_handle* h, int which, const void* v, void* w, int prec, void* stream) {
  HELM_GUARD({
    if (!h) { helm::set_error("NULL handle"); return HELM_EINVAL; }
    if (which != 0 && which != 1) { helm::set_error("which must be 0 (M) or 1 (H)"); return HELM_EINVAL; }
    return helm::apply_operator(h->h, which, v, w, prec, (cudaStream_t)stream);
  })
}

int helm_solve(helm_handle* h, const double* b, double* x, double tol, helm_info* info, void* stream) {
  HELM_GUARD({
    if (!h) { helm::set_error("NULL handle"); return HELM_EINVAL; }
    Handle* hs[1] = {h->h};
    const double* bs[1] = {b};
    double* xs[1] = {x};
    return helm::solve_group(hs, 1, bs, xs, tol, info, (cudaStream_t)stream);
  })
}

int helm_solve_host(helm_handle* h, const double* b_host, double* x_host, double tol, helm_info* info,
                    void* stream) {
  HELM_GUARD({
    if (!h || !b_host || !x_host) { helm::set_error("NULL argument"); return HELM_EINVAL; }
    Handle* hh = h->h;
    const size_t npts = hh->dim == 3 ? (size_t)hh->n * hh->n * hh->n : (size_t)hh->n * hh->n;
    const size_t bytes = npts * 2 * sizeof(double);
    cudaStream_t st = (cudaStream_t)stream;
    double *db = nullptr, *dx = nullptr;
    if (cudaMalloc(&db, bytes) != cudaSuccess || cudaMalloc(&dx, bytes) != cudaSuccess) {
      cudaFree(db);
      helm::set_error("device allocation for host solve failed");
      return HELM_ENOMEM;
    }
    int rc = HELM_OK;
    if (cudaMemcpyAsync(db, b_host, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(dx, 0, bytes, st) != cudaSuccess) {
      helm::set_error("host to device copy failed");
      rc = HELM_ECUDA;
    }
    if (rc == HELM_OK) {
      Handle* hs[1] = {hh};
      const double* bs[1] = {db};
      double* xs[1] = {dx};
      rc = helm::solve_group(hs, 1, bs, xs, tol, info, st);
      if (rc == HELM_OK || rc == HELM_ENOCONV || rc == HELM_ENUMERIC) {
        if (cudaMemcpyAsync(x_host, dx, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
          helm::set_error("device to host copy failed");
          rc = HELM_ECUDA;
        }
      }
    }
    cudaFree(db);
    cudaFree(dx);
    return rc;
  })
}

int helm_batch_solve(helm_handle* const* hs, int count, const double* const* b, double* const* x, double tol,
                     helm_info* infos, void* stream) {
  HELM_GUARD({
    if (!hs || count <= 0) { helm::set_error("empty batch"); return HELM_EINVAL; }
    std::vector<Handle*> inner(count);
    for (int i = 0; i < count; ++i) {
      if (!hs[i]) { helm::set_error("NULL handle in batch"); return HELM_EINVAL; }
      inner[i] = hs[i]->h;
    }
    return helm::solve_group(inner.data(), count, b, x, tol, infos, (cudaStream_t)stream);
  })
}

int helm_batch_solve_host(helm_handle* const* hs, int count, const double* const* b_host, double* const* x_host,
                          double tol, helm_info* infos, void* stream) {
  HELM_GUARD({
    if (!hs || count <= 0 || !b_host || !x_host) { helm::set_error("empty batch or NULL arrays"); return HELM_EINVAL; }
    std::vector<Handle*> inner(count);
    std::vector<size_t> off(count + 1, 0);
    for (int i = 0; i < count; ++i) {
      if (!hs[i] || !b_host[i] || !x_host[i]) { helm::set_error("NULL handle or vector in batch"); return HELM_EINVAL; }
      inner[i] = hs[i]->h;
      const size_t n = inner[i]->n;
      off[i + 1] = off[i] + (inner[i]->dim == 3 ? n * n * n : n * n) * 2;
    }
    cudaStream_t st = (cudaStream_t)stream;
    double* dev = nullptr;
    if (cudaMalloc(&dev, 2 * off[count] * sizeof(double)) != cudaSuccess) {
      helm::set_error("device allocation for host batch failed");
      return HELM_ENOMEM;
    }
    std::vector<const double*> db(count);
    std::vector<double*> dx(count);
    int rc = HELM_OK;
    for (int i = 0; i < count && rc == HELM_OK; ++i) {
      db[i] = dev + off[i];
      dx[i] = dev + off[count] + off[i];
      const size_t bytes = (off[i + 1] - off[i]) * sizeof(double);
      if (cudaMemcpyAsync((void*)db[i], b_host[i], bytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
          cudaMemsetAsync(dx[i], 0, bytes, st) != cudaSuccess) {
        helm::set_error("host to device copy failed");
        rc = HELM_ECUDA;
      }
    }
    if (rc == HELM_OK) {
      rc = helm::solve_group(inner.data(), count, db.data(), dx.data(), tol, infos, st);
      if (rc == HELM_OK || rc == HELM_ENOCONV || rc == HELM_ENUMERIC) {
        for (int i = 0; i < count; ++i)
          if (cudaMemcpyAsync(x_host[i], dx[i], (off[i + 1] - off[i]) * sizeof(double), cudaMemcpyDeviceToHost, st) !=
              cudaSuccess)
            rc = HELM_ECUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) rc = HELM_ECUDA;
        if (rc == HELM_ECUDA) helm::set_error("device to host copy failed");
      }
    }
    cudaFree(dev);
    return rc;
  })
}

int helm_workspace_bytes(const helm_handle* h, size_t* bytes) {
  if (!h || !bytes) { helm::set_error("NULL argument"); return HELM_EINVAL; }
  *bytes = h->h->bytes;
  return HELM_OK;
}

int helm_levels(const helm_handle* h, int* nlevels, int* sizes, int max_sizes) {
  if (!h || !nlevels) { helm::set_error("NULL argument"); return HELM_EINVAL; }
  const auto& lev = h->h->lev;
  *nlevels = (int)lev.size();
  if (sizes)
    for (int i = 0; i < (int)lev.size() && i < max_sizes; ++i) sizes[i] = lev[i].n;
  return HELM_OK;
}

int helm_autotune(const helm_grid* grid, const float* phi, double k, double theta_beta, const helm_opts* opts,
                  int reps, const char* path, double* default_ms, double* tuned_ms, void* stream) {
  HELM_GUARD({
    if (!grid) { helm::set_error("grid must not be NULL"); return HELM_EINVAL; }
    return helm::autotune(grid, phi, k, theta_beta, opts, reps, path, default_ms, tuned_ms, (cudaStream_t)stream);
  })
}

int helm_multidot(int basis, const double* V, int nvec, size_t npts, const double* w, double* h, void* stream) {
  HELM_GUARD({
    return helm::multidot(basis, (const double2*)V, nvec, npts, (const double2*)w, (double2*)h,
                          (cudaStream_t)stream);
  })
}

int helm_set_barrier_timeout(double seconds) {
  HELM_GUARD({
    if (!(seconds >= 0.0 && seconds <= 60.0)) { helm::set_error("seconds must be in [0, 60]"); return HELM_EINVAL; }
    helm::set_barrier_limit_ns((unsigned long long)(seconds * 1e9));
    return HELM_OK;
  })
}

int helm_tuning_load(const char* path) {
  HELM_GUARD({
    std::string err;
    const int rc = helm::tune_load(path, &err);
    if (rc != HELM_OK) helm::set_error(err);
    return rc;
  })
}

int helm_tuning_get(const char* pass, int dim, int P, int prec, int J, int* v) {
  HELM_GUARD({
    if (!pass || !v) { helm::set_error("NULL argument"); return HELM_EINVAL; }
    const std::string p(pass);
    const int tp = p == "arnoldi" ? helm::TP_ARNOLDI : p == "restrict" ? helm::TP_RESTRICT
                 : p == "prolong" ? helm::TP_PROLONG : p == "persist" ? helm::TP_PERSIST
                 : p == "zplanes" ? helm::TP_ZPLANES : -1;
    if (tp < 0) { helm::set_error("pass must be arnoldi, restrict, prolong, persist or zplanes"); return HELM_EINVAL; }
    if (prec != HELM_C64 && prec != HELM_C128) { helm::set_error("prec must be HELM_C64 or HELM_C128"); return HELM_EINVAL; }
    helm::TuneChoice c;
    if (!helm::tune_get(tp, dim, P, prec == HELM_C128 ? 16 : 8, J, &c)) return 0;
    for (int i = 0; i < helm::TUNE_NV; ++i) v[i] = c.v[i];
    return 1;
  })
}

int helm_precond_precision(const helm_handle* h, int* prec) {
  if (!h || !prec) { helm::set_error("NULL argument"); return HELM_EINVAL; }
  *prec = h->h->prec;
  return HELM_OK;
}

int helm_poly_smoother(double k, double h, double theta_beta, double theta_gamma, int dim, double* phi,
                       double* w) {
  HELM_GUARD({
    if (!phi || !w) { helm::set_error("NULL argument"); return HELM_EINVAL; }
    if (!(std::isfinite(k) && h > 0 && std::isfinite(h) && theta_beta >= 0 && theta_gamma > theta_beta &&
          theta_gamma < M_PI / 2 && (dim == 2 || dim == 3))) {
      helm::set_error("need finite k, h > 0, 0 <= theta_beta < theta_gamma < pi/2, dim 2 or 3");
      return HELM_EINVAL;
    }
    helm::cplx ws[3];
    if (!helm::poly_smoother(k, h, theta_beta, theta_gamma, dim, phi, ws)) {
      helm::set_error("no stable third-degree polynomial smoother for this k, h and theta_beta");
      return HELM_EINVAL;
    }
    for (int j = 0; j < 3; ++j) {
      w[2 * j] = ws[j].real();
      w[2 * j + 1] = ws[j].imag();
    }
    return HELM_OK;
  })
}

int helm_axis_coefficients(int n, double ecs_frac, int ecs_sides, double theta_gamma, double theta_beta,
                           double* a, double* d, double* c) {
  HELM_GUARD({
    if (!a || !d || !c) { helm::set_error("NULL argument"); return HELM_EINVAL; }
    const bool both = ecs_sides == HELM_ECS_BOTH;
    if (!(n >= 1 && (both || ecs_sides == HELM_ECS_HIGH) && ecs_frac > 0 && ecs_frac < (both ? 0.5 : 1.0) &&
          theta_gamma >= 0 && theta_gamma < M_PI / 2 && theta_beta >= 0 && theta_beta < M_PI / 2)) {
      helm::set_error("need n >= 1, a valid ecs_sides and ecs_frac, angles in [0, pi/2)");
      return HELM_EINVAL;
    }
    std::vector<helm::cplx> va, vd, vc;
    helm::stencil_coefficients(helm::grid_spacings(n, ecs_frac, theta_gamma, theta_beta, both), va, vd, vc);
    for (int i = 0; i < n; ++i) {
      a[2 * i] = va[i].real();
      a[2 * i + 1] = va[i].imag();
      d[2 * i] = vd[i].real();
      d[2 * i + 1] = vd[i].imag();
      c[2 * i] = vc[i].real();
      c[2 * i + 1] = vc[i].imag();
    }
    return HELM_OK;
  })
}

int helm_precond_apply_noalloc(const helm_grid* grid, double k, double theta_beta, const helm_opts* opts,
                               const void* r, void* z, int prec, void* stream) {
  HELM_GUARD({ return helm::precond_apply_noalloc(grid, k, theta_beta, opts, r, z, prec, (cudaStream_t)stream); })
}

int helm_serve_start(const helm_serve_opts* opts, helm_server** out) {
  HELM_GUARD({
    if (!out) { helm::set_error("out must not be NULL"); return HELM_EINVAL; }
    *out = nullptr;
    helm::Server* s = nullptr;
    int rc = helm::serve_start(opts, &s);
    if (rc != HELM_OK) return rc;
    *out = new helm_server{s};
    return HELM_OK;
  })
}

int helm_serve_submit(helm_server* s, int dim, int n, double k, double theta_beta, const double* b_host,
                      double* x_host, double tol, long long* ticket) {
  HELM_GUARD({
    if (!s) { helm::set_error("NULL server"); return HELM_EINVAL; }
    return helm::serve_submit(s->s, dim, n, k, theta_beta, b_host, x_host, tol, ticket);
  })
}

int helm_serve_poll(helm_server* s, long long ticket, helm_info* info, double* latency_s) {
  HELM_GUARD({
    if (!s) { helm::set_error("NULL server"); return HELM_EINVAL; }
    return helm::serve_poll(s->s, ticket, info, latency_s);
  })
}

int helm_serve_wait(helm_server* s, long long ticket, double timeout_s, helm_info* info, double* latency_s) {
  HELM_GUARD({
    if (!s) { helm::set_error("NULL server"); return HELM_EINVAL; }
    return helm::serve_wait(s->s, ticket, timeout_s, info, latency_s);
  })
}

int helm_serve_stats(helm_server* s, helm_serve_counters* out) {
  HELM_GUARD({
    if (!s) { helm::set_error("NULL server"); return HELM_EINVAL; }
    return helm::serve_stats(s->s, out);
  })
}

int helm_serve_stop(helm_server* s) {
  HELM_GUARD({
    if (!s) return HELM_OK;
    int rc = helm::serve_stop(s->s);
    delete s;
    return rc;
  })
}

unsigned long long helm_launch_count(void) { return helm::launch_count(); }

int helm_profile_begin(const char* prefix) {
  HELM_GUARD({
    helm::profile_begin(prefix ? prefix : "");
    return HELM_OK;
  })
}

int helm_profile_end(char* buf, size_t cap) {
  HELM_GUARD({
    if (!buf || cap == 0) { helm::set_error("buf must be non-NULL with cap > 0"); return HELM_EINVAL; }
    std::string js = helm::profile_end();
    const size_t n = std::min(js.size(), cap - 1);
    std::memcpy(buf, js.data(), n);
    buf[n] = 0;
    return HELM_OK;
  })
}

const char* helm_last_error(void) { return helm::g_last_error.c_str(); }

}  // extern "C"
