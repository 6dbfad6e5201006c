// The autotuner of the V-cycle's launch choices (tune.cpp holds the table).
//
// For one problem's hierarchy on the current device it times whole V-cycles
// (helm_precond_apply) while one choice at a time takes each of its candidates:
// coordinate descent from the built-in defaults, finest level first.  A candidate
// replaces the current choice when the V-cycle gets faster by more than 0.5%, which
// keeps run-to-run noise from deciding.  Choices:
//   2D levels: tiles per CTA of the Arnoldi passes (each step J), of the residual +
//     restriction pass and of the prolongation pass (1, 2, 4, 8);
//   3D levels without the TMA-fed passes (pitch below 128, or complex128): the planes
//     each CTA of the plain passes marches (2, 4, 8, 16);
//   3D complex64 levels of pitch 128..1024: the TMA-fed Arnoldi pass of each step J
//     off, or on with 2..8 plane slots in flight, 2 or 4 points per thread in y, and
//     the level shared as one piece per resident CTA or as 1, 2 or 4 z pieces per
//     column.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <memory>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/helm.h"
#include "engine.h"
#include "helm_internal.h"

namespace helm {

namespace {

struct Knob {
  int pass, dim, P, prec, J;
  std::vector<TuneChoice> cands;
};

TuneChoice tc(int a, int b = 0, int c = 0, int d = 0) {
  TuneChoice t;
  t.v[0] = a;
  t.v[1] = b;
  t.v[2] = c;
  t.v[3] = d;
  return t;
}

// shared memory of the 3D TMA-fed pass with `stages` plane slots of 72 x (8 qy + 2)
// float boxes, against the per-CTA limit (the static part is below 30 KB)
bool tma3_fits(int J, int qy, int stages) {
  const size_t box = ((size_t)36 * (8 * qy + 2) * 8 + 127) / 128 * 128;
  return (size_t)stages * J * box + 30 * 1024 <= 227 * 1024;
}

// Milliseconds per V-cycle: the best of three trials of `reps` cycles each.
int time_vcycles(Handle* h, const void* r, void* z, int reps, cudaStream_t st, double* ms) {
  cudaEvent_t a = nullptr, b = nullptr;
  CUDA_TRY(cudaEventCreate(&a));
  CUDA_TRY(cudaEventCreate(&b));
  double best = 1e30;
  int rc = HELM_OK;
  for (int w = 0; w < 2 && rc == HELM_OK; ++w) rc = precond_apply(h, r, z, HELM_C64, st);  // warm-up, capture
  for (int t = 0; t < 3 && rc == HELM_OK; ++t) {
    cudaEventRecord(a, st);
    for (int i = 0; i < reps && rc == HELM_OK; ++i) rc = precond_apply(h, r, z, HELM_C64, st);
    cudaEventRecord(b, st);
    if (cudaEventSynchronize(b) != cudaSuccess) rc = HELM_ECUDA;
    float e = 0.f;
    cudaEventElapsedTime(&e, a, b);
    best = std::min(best, (double)e / reps);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc == HELM_OK) rc = vcycle_take_error() ? HELM_ETIMEOUT : HELM_OK;
  *ms = best;
  return rc;
}

}  // namespace

int autotune(const helm_grid* grid, const float* phi, double k, double theta_beta, const helm_opts* opts, int reps,
             const char* path, double* default_ms, double* tuned_ms, cudaStream_t st) {
  if (reps < 1) reps = 10;
  helm_opts o{};
  if (opts) o = *opts;
  o.maxit = 1;
  o.restart = 0;
  Handle* raw = nullptr;
  TRY(setup_handle(grid, phi, k, theta_beta, &o, st, &raw));
  std::unique_ptr<Handle> h(raw);
  const int dim = h->dim, n = h->n;
  const int eb = h->prec == HELM_C128 ? 16 : 8;
  if (h->smoother != HELM_SMOOTHER_GMRES) { set_error("the autotuner tunes the GMRES(s) V-cycle"); return HELM_EINVAL; }
  // input: a fixed pseudo-random complex64 field (a linear congruential sequence)
  const size_t npts = dim == 3 ? (size_t)n * n * n : (size_t)n * n;
  std::vector<float2> hr(npts);
  uint64_t s = 0x9e3779b97f4a7c15ull;
  for (auto& v : hr) {
    s = s * 6364136223846793005ull + 1442695040888963407ull;
    v.x = (float)((double)(s >> 11) / 9007199254740992.0 - 0.5);
    s = s * 6364136223846793005ull + 1442695040888963407ull;
    v.y = (float)((double)(s >> 11) / 9007199254740992.0 - 0.5);
  }
  void* r = nullptr;
  void* z = nullptr;
  CUDA_TRY(cudaMalloc(&r, npts * sizeof(float2)));
  if (cudaMalloc(&z, npts * sizeof(float2)) != cudaSuccess) {
    cudaFree(r);
    set_error("autotune: cannot allocate the output");
    return HELM_ENOMEM;
  }
  struct Free {
    void* a;
    void* b;
    ~Free() { cudaFree(a); cudaFree(b); }
  } fr{r, z};
  CUDA_TRY(cudaMemcpy(r, hr.data(), npts * sizeof(float2), cudaMemcpyHostToDevice));

  // the choices of this hierarchy's grid-wide levels
  const int thr = dim == 2 ? 31 : 7;
  std::vector<Knob> knobs;
  for (const HostLevel& L : h->lev) {
    if (L.n <= thr) continue;
    const int P = L.P;
    if (dim == 3 && !(eb == 8 && L.tm && P >= 128 && P <= 1024 && P % 32 == 0)) {
      // plain 3D passes: planes per CTA march
      Knob kz{TP_ZPLANES, 3, P, eb, 0, {}};
      for (int z : {2, 4, 8, 16})
        if (z <= P) kz.cands.push_back(tc(z));
      knobs.push_back(kz);
    }
    if (dim == 2) {
      for (int J = 1; J <= h->s; ++J) knobs.push_back({TP_ARNOLDI, 2, P, eb, J, {tc(1), tc(2), tc(4), tc(8)}});
      knobs.push_back({TP_RESTRICT, 2, P, eb, 0, {tc(1), tc(2), tc(4), tc(8)}});
      knobs.push_back({TP_PROLONG, 2, P, eb, 0, {tc(1), tc(2), tc(4), tc(8)}});
    } else if (eb == 8 && L.tm && P >= 128 && P <= 1024 && P % 32 == 0) {
      for (int J = 1; J <= h->s; ++J) {
        Knob kb{TP_ARNOLDI, 3, P, eb, J, {tc(0, 2, 0, 2)}};
        for (int qy : {2, 4}) {
          if (qy == 4 && J > 2) continue;
          for (int stg : {2, 3, 4, 6, 8}) {
            if (!tma3_fits(J, qy, stg)) continue;
            for (int pieces : {0, 1, 2, 4}) kb.cands.push_back(tc(1, stg, pieces, qy));
          }
        }
        knobs.push_back(kb);
      }
      Knob kr{TP_RESTRICT, 3, P, eb, 0, {tc(0, 2, 0, 2)}};
      for (int stg : {2, 3, 4})
        if (tma3_fits(h->s + 1, 2, stg))
          for (int pieces : {0, 1, 2, 4}) kr.cands.push_back(tc(1, stg, pieces, 2));
      knobs.push_back(kr);
      Knob kp{TP_PROLONG, 3, P, eb, 0, {tc(0, 2, 0, 2)}};
      for (int qy : {2, 4})
        for (int stg : {2, 3, 4, 6, 8}) {
          if (!tma3_fits(1, qy, stg)) continue;
          for (int pieces : {0, 1, 2, 4}) kp.cands.push_back(tc(1, stg, pieces, qy));
        }
      knobs.push_back(kp);
    }
  }
  // start from the defaults: this hierarchy's entries leave the table
  for (const Knob& kb : knobs) tune_set(kb.pass, kb.dim, kb.P, kb.prec, kb.J, nullptr);
  double base = 0;
  TRY(time_vcycles(h.get(), r, z, reps, st, &base));
  double best = base;
  int tried = 0;
  for (const Knob& kb : knobs) {
    TuneChoice keep{};
    bool have = false;  // the default stays unless a candidate wins
    for (const TuneChoice& c : kb.cands) {
      tune_set(kb.pass, kb.dim, kb.P, kb.prec, kb.J, &c);
      double t = 0;
      TRY(time_vcycles(h.get(), r, z, reps, st, &t));
      ++tried;
      if (t < best * (1.0 - 0.005)) {
        best = t;
        keep = c;
        have = true;
      }
    }
    tune_set(kb.pass, kb.dim, kb.P, kb.prec, kb.J, have ? &keep : nullptr);
  }
  double fin = 0;
  TRY(time_vcycles(h.get(), r, z, reps, st, &fin));
  if (default_ms) *default_ms = base;
  if (tuned_ms) *tuned_ms = fin;
  if (path) {
    std::ostringstream rec;
    rec << "{\"dim\": " << dim << ", \"n\": " << n << ", \"prec\": \"" << (eb == 8 ? "c64" : "c128")
        << "\", \"theta_beta\": " << theta_beta << ", \"field\": " << (phi ? "true" : "false")
        << ", \"reps\": " << reps << ", \"choices\": " << knobs.size() << ", \"candidates_timed\": " << tried
        << ", \"default_ms_per_vcycle\": " << base << ", \"tuned_ms_per_vcycle\": " << fin << "}";
    std::string err;
    if (tune_write(path, rec.str(), &err) != HELM_OK) {
      set_error(err);
      return HELM_EINVAL;
    }
  }
  return HELM_OK;
}

}  // namespace helm
