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
// descriptors that point into that array.  The set-up data (descriptors, stencil
// coefficients, the coarsest LU factors) is built on the host by the same geometry
// routines as helm_setup's and reaches the array as the arguments of small staging
// kernels, so no host buffer outlives the call and nothing waits for the stream.
#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <cstring>
#include <mutex>
#include <sstream>
#include <vector>

#include "../../include/helm.h"
#include "engine.h"
#include "geometry.h"
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
constexpr int MAX_COARSE = 32;    // unknowns of the coarsest dense solve

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

// Set-up bytes reach the scratch array as kernel arguments: a launch copies its
// arguments when it is enqueued, so the host block may be a stack buffer and the call
// never waits for the stream (a pageable cudaMemcpyAsync would).  One launch carries
// STAGE_CHUNK bytes, which keeps the argument block under the classic 4 KB limit.
constexpr int STAGE_CHUNK = 4032;
struct StageChunk {
  unsigned long long off;  // byte offset into the scratch array
  int nbytes;
  int pad;
  unsigned char data[STAGE_CHUNK];
};
static_assert(sizeof(StageChunk) <= 4096, "staging argument block above 4 KB");

__global__ void k_noalloc_stage(StageChunk c) {
  for (int i = threadIdx.x; i < c.nbytes; i += blockDim.x) g_noalloc_scratch[c.off + i] = c.data[i];
}

// Copy [src, src + bytes) to scratch offset `off` with staging launches on `st`.
int stage_bytes(const void* src, size_t bytes, size_t off, cudaStream_t st) {
  const unsigned char* p = static_cast<const unsigned char*>(src);
  StageChunk c;
  for (size_t done = 0; done < bytes; done += STAGE_CHUNK) {
    const size_t nb = bytes - done < (size_t)STAGE_CHUNK ? bytes - done : (size_t)STAGE_CHUNK;
    c.off = off + done;
    c.nbytes = (int)nb;
    c.pad = 0;
    std::memcpy(c.data, p + done, nb);
    Launch L("noalloc.stage", st, 0, 0);
    k_noalloc_stage<<<1, 256, 0, st>>>(c);
    NA_CUDA(cudaGetLastError());
  }
  return HELM_OK;
}

template <typename C>
int run_noalloc(const helm_grid* grid, double k, double theta_beta, int nu1, int nu2, int s, int coarsest,
                const void* r, void* z, int prec, cudaStream_t st) {
  const int dim = grid->dim, n = grid->n;
  const double ecs = grid->ecs_frac > 0 ? grid->ecs_frac : 0.125;
  const double tg = grid->theta_gamma;
  const std::vector<int> sizes = level_sizes(n, coarsest);  // helm_setup's hierarchy
  const int nlev = (int)sizes.size();
  if (nlev > MAX_LEVELS) { set_error("too many levels"); return HELM_EINVAL; }
  const int nc = sizes[nlev - 1];
  const int m = dim == 3 ? nc * nc * nc : nc * nc;
  if (m > MAX_COARSE) { set_error("coarsest grid has more than 32 unknowns (n+1 needs a larger power of two)"); return HELM_EINVAL; }
  // carve the scratch: descriptors, LU record, LU factors, pivots and coefficients
  // (the staged set-up block, contiguous), then scalars, partial slots and vectors
  Carve cv;
  const size_t o_lev = cv.take(sizeof(LevelDev<C>) * nlev);
  const size_t o_lu = cv.take(sizeof(CoarseLU));
  const size_t o_lum = cv.take(sizeof(double2) * m * m);
  const size_t o_piv = cv.take(sizeof(int) * m);
  size_t o_coef[MAX_LEVELS], o_vec[MAX_LEVELS], np[MAX_LEVELS];
  for (int l = 0; l < nlev; ++l) o_coef[l] = cv.take(3 * sizeof(C) * sizes[l]);
  const size_t setup_end = cv.off;
  typedef SweepScalarsT<typename RealOf<C>::T> SS;
  const size_t o_sc = cv.take(sizeof(SS) * nlev);
  const size_t o_part = cv.take(sizeof(double) * NPART);
  for (int l = 0; l < nlev; ++l) {
    const size_t P = sizes[l] + 1;
    np[l] = dim == 3 ? P * P * P : P * P;
    o_vec[l] = cv.take((4 + s) * sizeof(C) * np[l]);
  }
  if (cv.off > NOALLOC_BYTES) {
    std::ostringstream os;
    os << "grid needs " << cv.off << " bytes of scratch, the allocation-free entry point has " << NOALLOC_BYTES;
    set_error(os.str());
    return HELM_EINVAL;
  }
  // the set-up block is assembled on the host (bounded by MAX_N and MAX_COARSE)
  constexpr size_t SETUP_MAX = 64 * 1024;
  if (setup_end > SETUP_MAX) { set_error("set-up block of the allocation-free entry point too large"); return HELM_EINVAL; }
  void* base_v = nullptr;
  int rc = scratch_address(&base_v);
  if (rc != HELM_OK) return rc;
  char* base = (char*)base_v;
  alignas(16) static thread_local unsigned char blk[SETUP_MAX];
  std::memset(blk, 0, setup_end);

  // stencil coefficients of every level (helm_setup's geometry)
  for (int l = 0; l < nlev; ++l) {
    std::vector<cplx> a, d, c;
    stencil_coefficients(grid_spacings(sizes[l], ecs, tg, theta_beta, true), a, d, c);
    C* host = reinterpret_cast<C*>(blk + o_coef[l]);
    const int nl = sizes[l];
    for (int i = 0; i < nl; ++i) {
      host[i].x = a[i].real(); host[i].y = a[i].imag();
      host[nl + i].x = d[i].real(); host[nl + i].y = d[i].imag();
      host[2 * nl + i].x = c[i].real(); host[2 * nl + i].y = c[i].imag();
    }
  }
  // descriptors pointing into the scratch array
  LevelDev<C>* desc = reinterpret_cast<LevelDev<C>*>(blk + o_lev);
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
  }
  for (int l = 0; l + 1 < nlev; ++l) {
    desc[l].nc = desc[l + 1].n;
    desc[l].Pc = desc[l + 1].P;
    desc[l].bc = desc[l + 1].b;
    desc[l].xcb = desc[l + 1].xb;
    desc[l].scc = desc[l + 1].sc;
  }
  // coarsest dense operator and its LU with partial pivoting (helm_setup's routines)
  {
    std::vector<cplx> a, d, c;
    stencil_coefficients(grid_spacings(nc, ecs, tg, theta_beta, true), a, d, c);
    std::vector<cplx> A = dense_operator(dim, nc, a, d, c, std::vector<double>(m, k * k));
    std::vector<int> perm;
    if (!lu_factor(A, m, perm)) { set_error("coarsest operator is singular"); return HELM_ENUMERIC; }
    double2* Ad = reinterpret_cast<double2*>(blk + o_lum);
    for (int i = 0; i < m * m; ++i) Ad[i] = make_double2(A[i].real(), A[i].imag());
    int* pv = reinterpret_cast<int*>(blk + o_piv);
    for (int i = 0; i < m; ++i) pv[i] = perm[i];
    CoarseLU* lu = reinterpret_cast<CoarseLU*>(blk + o_lu);
    lu->m = m;
    lu->nlev = nlev;
    lu->lu = (const double2*)(base + o_lum);
    lu->piv = (const int*)(base + o_piv);
  }

  // clear scalars, partial slots and every level vector (nothing of the previous
  // call's contents may leak into this one), then stage the set-up block
  NA_CUDA(cudaMemsetAsync(base + setup_end, 0, cv.off - setup_end, st));
  TRY(stage_bytes(blk, setup_end, 0, st));

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
