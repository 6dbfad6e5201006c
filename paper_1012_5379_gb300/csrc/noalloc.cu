// helm_precond_apply_noalloc: one V-cycle for small grids without any device
// allocation.
//
// Some callers cannot let a library call cudaMalloc: applications whose device memory
// is reserved up front by a framework's pooling allocator (a cudaMalloc behind its
// back can fail or fragment the pool), and latency-critical loops where the implicit
// device synchronisation of cudaMalloc/cudaFree is not acceptable.  This entry point
// keeps all of its working memory (level vectors, coefficients, sweep scalars,
// descriptors, the coarsest LU factors) in one file-scope __device__ array of fixed
// size, and launches the same kernels as the allocating path (the input kernel, the
// single-CTA coarse-cycle kernel run from the finest level, the output kernel) on
// descriptors that point into that array.  Host-side set-up uses fixed-size stack
// arrays only.
#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <cstring>
#include <mutex>
#include <sstream>

#include "../../include/helm.h"
#include "engine.h"
#include "helm_internal.h"
#include "profiler.h"

namespace helm {

// Every GPU that loads the library holds this array until the process exits.
constexpr size_t NOALLOC_BYTES = (size_t)4 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

namespace {

constexpr int MAX_DEVICES = 64;
constexpr int MAX_LEVELS = 12;
constexpr int MAX_N = 255;        // per-axis interior nodes accepted before the size check
constexpr int MAX_COARSE = 32;    // unknowns of the coarsest dense solve (stack arrays)
typedef std::complex<double> cd;

void* g_scratch_addr[MAX_DEVICES] = {nullptr};
std::mutex g_scratch_mu;

// Device address of the scratch array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is resolved once per
// device with that device current and then cached.
int scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e)); return HELM_ECUDA; }
  if (dev < 0 || dev >= MAX_DEVICES) { set_error("device ordinal out of range for the scratch table"); return HELM_EINVAL; }
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error(std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
      return HELM_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return HELM_OK;
}

// Complex spacings of the stretched grid (per-interval segment integrals of the
// stretching factor) and the three-point coefficients, written into caller arrays.
double overlap(double a, double b, double lo, double hi) {
  return std::fmax(0.0, std::fmin(b, hi) - std::fmax(a, lo));
}
void level_coefficients(int n, double ecs, double tg, double tb, cd* a, cd* d, cd* c) {
  const double h = 1.0 / (n + 1);
  const cd eg = std::polar(1.0, tg), eb = std::polar(1.0, tb);
  auto sp = [&](int i) {
    const double x0 = i * h, x1 = (i + 1) * h;
    return eg * (overlap(x0, x1, 0.0, ecs) + overlap(x0, x1, 1.0 - ecs, 1.0)) + eb * overlap(x0, x1, ecs, 1.0 - ecs);
  };
  for (int i = 0; i < n; ++i) {
    const cd hl = sp(i), hr = sp(i + 1);
    const cd t = 2.0 / (hl + hr);
    a[i] = -t / hl;
    c[i] = -t / hr;
    d[i] = t * (1.0 / hl + 1.0 / hr);
  }
}

// A bump allocator over the scratch array (offsets only, 256-byte aligned).
struct Carve {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) / 256 * 256;
    return o;
  }
};

#define NA_CUDA(expr)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (expr);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));                    \
      return HELM_ECUDA;                                                                \
    }                                                                                   \
  } while (0)

template <typename C>
int run_noalloc(const helm_grid* grid, double k, double theta_beta, int nu1, int nu2, int s, int coarsest,
                const void* r, void* z, int prec, cudaStream_t st) {
  const int dim = grid->dim, n = grid->n;
  const double ecs = grid->ecs_frac > 0 ? grid->ecs_frac : 0.125;
  const double tg = grid->theta_gamma;
  // level sizes
  int sizes[MAX_LEVELS];
  int nlev = 0;
  sizes[nlev++] = n;
  while (sizes[nlev - 1] > coarsest && (sizes[nlev - 1] + 1) % 2 == 0) {
    if (nlev == MAX_LEVELS) { set_error("too many levels"); return HELM_EINVAL; }
    sizes[nlev] = (sizes[nlev - 1] + 1) / 2 - 1;
    ++nlev;
  }
  const int nc = sizes[nlev - 1];
  const int m = dim == 3 ? nc * nc * nc : nc * nc;
  if (m > MAX_COARSE) { set_error("coarsest grid has more than 32 unknowns (n+1 needs a larger power of two)"); return HELM_EINVAL; }
  // carve the scratch: descriptors, scalars, partial slots, LU, then per-level data
  Carve cv;
  const size_t o_lev = cv.take(sizeof(LevelDev<C>) * nlev);
  const size_t o_lu = cv.take(sizeof(CoarseLU));
  typedef SweepScalarsT<typename RealOf<C>::T> SS;
  const size_t o_sc = cv.take(sizeof(SS) * nlev);
  const size_t o_part = cv.take(sizeof(double) * NPART);
  const size_t o_lum = cv.take(sizeof(double2) * m * m);
  const size_t o_piv = cv.take(sizeof(int) * m);
  const size_t zero_end = cv.off;  // scalars and partial slots start at zero
  size_t o_coef[MAX_LEVELS], o_vec[MAX_LEVELS];
  size_t np[MAX_LEVELS];
  for (int l = 0; l < nlev; ++l) {
    const size_t P = sizes[l] + 1;
    np[l] = dim == 3 ? P * P * P : P * P;
    o_coef[l] = cv.take(3 * sizeof(C) * sizes[l]);
    o_vec[l] = cv.take((4 + s) * sizeof(C) * np[l]);
  }
  if (cv.off > NOALLOC_BYTES) {
    std::ostringstream os;
    os << "grid needs " << cv.off << " bytes of scratch, the allocation-free entry point has " << NOALLOC_BYTES;
    set_error(os.str());
    return HELM_EINVAL;
  }
  void* base_v = nullptr;
  int rc = scratch_address(&base_v);
  if (rc != HELM_OK) return rc;
  char* base = (char*)base_v;

  // clear descriptors, scalars, partial slots and every level vector: nothing of the
  // previous call's contents may leak into this one
  NA_CUDA(cudaMemsetAsync(base, 0, cv.off, st));

  // descriptors and coefficients (host stack buffers; pageable copies are staged
  // before cudaMemcpyAsync returns)
  LevelDev<C> desc[MAX_LEVELS];
  std::memset(desc, 0, sizeof(desc));
  for (int l = 0; l < nlev; ++l) {
    const int nl = sizes[l];
    LevelDev<C>& d = desc[l];
    d.n = nl;
    d.P = nl + 1;
    d.s = s;
    d.ntiles = 1;
    C* v = (C*)(base + o_vec[l]);
    d.b = v;
    d.xa = v + np[l];
    d.xb = v + 2 * np[l];
    d.r0 = v + 3 * np[l];
    for (int j = 0; j < s; ++j) d.p[j] = v + (4 + j) * np[l];
    const C* cf = (const C*)(base + o_coef[l]);
    d.ca = cf;
    d.cd = cf + nl;
    d.cc = cf + 2 * nl;
    d.phi = nullptr;
    d.phic = k * k;
    d.phir = (typename RealOf<C>::T)d.phic;
    d.sc = (SS*)(base + o_sc) + l;
    d.part = (double*)(base + o_part);
    {
      cd a[MAX_N], dd[MAX_N], c[MAX_N];
      level_coefficients(nl, ecs, tg, theta_beta, a, dd, c);
      C host[3 * MAX_N];
      for (int i = 0; i < nl; ++i) {
        host[i].x = a[i].real(); host[i].y = a[i].imag();
        host[nl + i].x = dd[i].real(); host[nl + i].y = dd[i].imag();
        host[2 * nl + i].x = c[i].real(); host[2 * nl + i].y = c[i].imag();
      }
      NA_CUDA(cudaMemcpyAsync(base + o_coef[l], host, 3 * sizeof(C) * nl, cudaMemcpyHostToDevice, st));
    }
  }
  for (int l = 0; l + 1 < nlev; ++l) {
    desc[l].nc = desc[l + 1].n;
    desc[l].Pc = desc[l + 1].P;
    desc[l].bc = desc[l + 1].b;
    desc[l].xcb = desc[l + 1].xb;
    desc[l].scc = desc[l + 1].sc;
  }
  NA_CUDA(cudaMemcpyAsync(base + o_lev, desc, sizeof(LevelDev<C>) * nlev, cudaMemcpyHostToDevice, st));

  // coarsest dense operator, LU with partial pivoting (FP64, on the stack)
  {
    cd a[MAX_COARSE], dd[MAX_COARSE], c[MAX_COARSE];
    level_coefficients(nc, ecs, tg, theta_beta, a, dd, c);
    cd A[MAX_COARSE * MAX_COARSE];
    for (int i = 0; i < m * m; ++i) A[i] = 0.0;
    const int zn = dim == 3 ? nc : 1;
    for (int zz = 0; zz < zn; ++zz)
      for (int yy = 0; yy < nc; ++yy)
        for (int xx = 0; xx < nc; ++xx) {
          const int row = (zz * nc + yy) * nc + xx;
          A[row * m + row] = dd[xx] + dd[yy] + (dim == 3 ? dd[zz] : cd(0, 0)) - k * k;
          if (xx > 0) A[row * m + row - 1] = a[xx];
          if (xx + 1 < nc) A[row * m + row + 1] = c[xx];
          if (yy > 0) A[row * m + row - nc] = a[yy];
          if (yy + 1 < nc) A[row * m + row + nc] = c[yy];
          if (dim == 3 && zz > 0) A[row * m + row - nc * nc] = a[zz];
          if (dim == 3 && zz + 1 < nc) A[row * m + row + nc * nc] = c[zz];
        }
    int perm[MAX_COARSE];
    for (int i = 0; i < m; ++i) perm[i] = i;
    for (int col = 0; col < m; ++col) {
      int piv = col;
      for (int i = col + 1; i < m; ++i)
        if (std::abs(A[i * m + col]) > std::abs(A[piv * m + col])) piv = i;
      if (std::abs(A[piv * m + col]) == 0.0) { set_error("coarsest operator is singular"); return HELM_ENUMERIC; }
      if (piv != col) {
        for (int j = 0; j < m; ++j) std::swap(A[col * m + j], A[piv * m + j]);
        std::swap(perm[col], perm[piv]);
      }
      for (int i = col + 1; i < m; ++i) {
        const cd l = A[i * m + col] / A[col * m + col];
        A[i * m + col] = l;
        for (int j = col + 1; j < m; ++j) A[i * m + j] -= l * A[col * m + j];
      }
    }
    double2 Ad[MAX_COARSE * MAX_COARSE];
    for (int i = 0; i < m * m; ++i) Ad[i] = make_double2(A[i].real(), A[i].imag());
    NA_CUDA(cudaMemcpyAsync(base + o_lum, Ad, sizeof(double2) * m * m, cudaMemcpyHostToDevice, st));
    NA_CUDA(cudaMemcpyAsync(base + o_piv, perm, sizeof(int) * m, cudaMemcpyHostToDevice, st));
    CoarseLU lu;
    lu.m = m;
    lu.nlev = nlev;
    lu.lu = (const double2*)(base + o_lum);
    lu.piv = (const int*)(base + o_piv);
    NA_CUDA(cudaMemcpyAsync(base + o_lu, &lu, sizeof(lu), cudaMemcpyHostToDevice, st));
  }
  (void)zero_end;

  const LevelDev<C>* dlev = (const LevelDev<C>*)(base + o_lev);
  {
    Launch L("noalloc.load", st, 0, 0);
    launch_load_input<C>(dim, dlev, 1, r, prec, st);
  }
  {
    Launch L("noalloc.cycle", st, 0, 0);
    launch_coarse<C>(dim, dlev, nlev, nlev, (const CoarseLU*)(base + o_lu), 1, nu1, nu2, st);
  }
  {
    Launch L("noalloc.store", st, 0, 0);
    launch_store_output<C>(dim, n, dlev, z, prec, st);
  }
  NA_CUDA(cudaGetLastError());
  return HELM_OK;
}

}  // namespace

int precond_apply_noalloc(const helm_grid* grid, double k, double theta_beta, const helm_opts* opts,
                          const void* r, void* z, int prec, cudaStream_t st) {
  if (!grid || !r || !z) { set_error("grid, r and z must not be NULL"); return HELM_EINVAL; }
  if (grid->dim != 2 && grid->dim != 3) { set_error("dim must be 2 or 3"); return HELM_EINVAL; }
  if (grid->n < 1 || grid->n > MAX_N) { set_error("n out of range for the allocation-free entry point"); return HELM_EINVAL; }
  const double ecs = grid->ecs_frac > 0 ? grid->ecs_frac : 0.125;
  if (!(ecs < 0.5)) { set_error("ecs_frac must be in (0, 0.5)"); return HELM_EINVAL; }
  if (grid->ecs_sides != HELM_ECS_BOTH) { set_error("the allocation-free entry point takes layers on both sides only"); return HELM_EINVAL; }
  if (!(grid->theta_gamma >= 0 && grid->theta_gamma < M_PI / 2)) { set_error("theta_gamma must be in [0, pi/2)"); return HELM_EINVAL; }
  if (!(theta_beta >= 0 && theta_beta < M_PI / 2)) { set_error("theta_beta must be in [0, pi/2)"); return HELM_EINVAL; }
  if (!std::isfinite(k)) { set_error("k must be finite"); return HELM_EINVAL; }
  if (prec != HELM_C64 && prec != HELM_C128) { set_error("prec must be HELM_C64 or HELM_C128"); return HELM_EINVAL; }
  helm_opts o{};
  if (opts) o = *opts;
  const int nu1 = o.nu1 > 0 ? o.nu1 : (opts && o.nu1 == 0 && o.nu2 > 0 ? 0 : 1);
  const int nu2 = o.nu2 > 0 ? o.nu2 : (opts && o.nu2 == 0 && o.nu1 > 0 ? 0 : 1);
  const int s = o.s > 0 ? o.s : 3;
  const int coarsest = o.coarsest_n > 0 ? o.coarsest_n : 3;
  const int iprec = o.precond_prec ? o.precond_prec : HELM_C64;
  if (s > SMAX || nu1 > 8 || nu2 > 8) { set_error("s must be in 1..4 and nu1, nu2 <= 8"); return HELM_EINVAL; }
  if (iprec != HELM_C64 && iprec != HELM_C128) { set_error("precond_prec must be HELM_C64 or HELM_C128"); return HELM_EINVAL; }
  if (o.csl_eps != 0.0) { set_error("the allocation-free entry point has no complex shift (csl_eps must be 0)"); return HELM_EINVAL; }
  if (o.smoother != HELM_SMOOTHER_GMRES) { set_error("the allocation-free entry point smooths with GMRES(s) only"); return HELM_EINVAL; }
  return iprec == HELM_C128
             ? run_noalloc<double2>(grid, k, theta_beta, nu1, nu2, s, coarsest, r, z, prec, st)
             : run_noalloc<float2>(grid, k, theta_beta, nu1, nu2, s, coarsest, r, z, prec, st);
}

}  // namespace helm
