// Host engine: builds the CSG hierarchy of a problem (Sec. 3.1, Prop. 3.1), groups
// problems for batched launches, and drives the V-cycle (Sec. 3.1-3.2) and the outer
// flexible GMRES (Sec. 5).
#include "engine.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <sstream>

#include "geometry.h"
#include "poly.h"
#include "profiler.h"

namespace helm {

static size_t elem_bytes(int prec) { return prec == HELM_C128 ? sizeof(double2) : sizeof(float2); }


static int sm_count_host() {
  static const int sms = [] {  // thread-safe initialisation
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) v = 1;
    return v;
  }();
  return sms;
}

// Sizes of the tiles of the outer stencil passes: 2D warps march `rows` rows, chosen to
// give about four CTAs per SM on a single problem; 3D CTAs march 8, 16 or 32 planes
// (pitch below 128, below 256, from 256: longer marches amortise the z halo; 255^3:
// 352 us at 16 planes, 328 us at 32).
static TileCfg default_tiles(int dim, int P) {
  TileCfg c;
  if (dim == 2) {
    int rows = (int)((long long)P * P / (32LL * WARPS2 * 608));
    rows = std::max(2, std::min(32, rows & ~1));
    c.rows = rows;
  } else {
    c.rows = P >= 256 ? 32 : (P >= 128 ? 16 : 8);
  }
  return c;
}

// Largest level size run by the coarse sub-cycle kernel (one CTA per problem with the
// levels staged in shared memory) instead of grid-wide launches.
static int coarse_threshold(int dim) { return dim == 2 ? 31 : 7; }

// Tiles of the finest tile configuration (2 rows / planes per march).
static int max_tiles(int dim, int P) {
  TileCfg c;
  c.rows = 2;
  return tiles_per_problem(dim, P, c);
}

template <typename T>
static int dev_alloc(Handle* h, T** p, size_t bytes) {
  void* q = nullptr;
  CUDA_TRY(cudaMalloc(&q, std::max<size_t>(bytes, 16)));
  h->allocs.push_back(q);
  h->bytes += bytes;
  *p = reinterpret_cast<T*>(q);
  return HELM_OK;
}

// Coefficients of M on level l for angle theta_beta (both precisions), and phi.
static int upload_level_coefficients(Handle* h, int l, double theta_beta, cudaStream_t st) {
  HostLevel& L = h->lev[l];
  std::vector<cplx> a, d, c;
  stencil_coefficients(grid_spacings(L.n, h->ecs, h->theta_gamma, theta_beta, h->ecs_sides == HELM_ECS_BOTH), a, d, c);
  // Complex shift of M (constant k): the diagonal's extra -i eps k^2 is spread over the
  // d axes' diagonal coefficients (every point's diagonal adds one per axis), so the
  // kernels' -phi stays real and nothing else changes.
  if (h->csl_eps != 0.0) {
    const cplx per_axis(0.0, -h->csl_eps * h->k * h->k / h->dim);
    for (auto& v : d) v += per_axis;
  }
  double2* c64 = reinterpret_cast<double2*>(h->stage + h->stage_coef[l]);
  for (int i = 0; i < L.n; ++i) {
    c64[i] = make_double2(a[i].real(), a[i].imag());
    c64[L.n + i] = make_double2(d[i].real(), d[i].imag());
    c64[2 * L.n + i] = make_double2(c[i].real(), c[i].imag());
  }
  CUDA_TRY(cudaMemcpyAsync(L.coef64, c64, 3 * L.n * sizeof(double2), cudaMemcpyHostToDevice, st));
  if (h->prec == HELM_C128) {
    CUDA_TRY(cudaMemcpyAsync(L.coef, c64, 3 * L.n * sizeof(double2), cudaMemcpyHostToDevice, st));
  } else {
    float2* c32 = reinterpret_cast<float2*>(c64 + 3 * L.n);
    for (int i = 0; i < 3 * L.n; ++i) c32[i] = make_float2((float)c64[i].x, (float)c64[i].y);
    CUDA_TRY(cudaMemcpyAsync(L.coef, c32, 3 * L.n * sizeof(float2), cudaMemcpyHostToDevice, st));
  }
  return HELM_OK;
}

// Dense FP64 LU (partial pivoting) of the coarsest operator, uploaded.
static int factor_coarsest(Handle* h, double theta_beta, cudaStream_t st) {
  const HostLevel& Lc = h->lev.back();
  const int cm = h->lu_m;
  std::vector<cplx> a, d, c;
  stencil_coefficients(grid_spacings(Lc.n, h->ecs, h->theta_gamma, theta_beta, h->ecs_sides == HELM_ECS_BOTH), a, d, c);
  std::vector<double> phic(cm, Lc.phic);
  if (Lc.phi) {
    std::vector<float> pad(Lc.np);
    CUDA_TRY(cudaMemcpyAsync(pad.data(), Lc.phi, Lc.np * sizeof(float), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    for (int z = 0; z < (h->dim == 3 ? Lc.n : 1); ++z)
      for (int y = 0; y < Lc.n; ++y)
        for (int x = 0; x < Lc.n; ++x) phic[(z * Lc.n + y) * Lc.n + x] = pad[((size_t)z * Lc.P + y) * Lc.P + x];
  }
  std::vector<cplx> A = dense_operator(h->dim, Lc.n, a, d, c, phic, cplx(1.0, h->csl_eps));
  std::vector<int> perm;
  if (!lu_factor(A, cm, perm)) { set_error("coarsest operator is singular"); return HELM_ENUMERIC; }
  double2* Ad = reinterpret_cast<double2*>(h->stage + h->stage_lu);
  int* pv = reinterpret_cast<int*>(h->stage + h->stage_piv);
  for (size_t i = 0; i < A.size(); ++i) Ad[i] = make_double2(A[i].real(), A[i].imag());
  for (int i = 0; i < cm; ++i) pv[i] = perm[i];
  CUDA_TRY(cudaMemcpyAsync(h->lu, Ad, A.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(h->piv, pv, cm * sizeof(int), cudaMemcpyHostToDevice, st));
  return HELM_OK;
}

// Richardson weights of the Sec. 4 polynomial smoother on every smoothed level (all
// but the coarsest); a level of n interior nodes has real spacing 1 / (n + 1).
static int compute_poly_weights(Handle* h, const std::vector<int>& sizes) {
  std::vector<std::array<cplx, 3>> ws(sizes.size() > 0 ? sizes.size() - 1 : 0);
  for (size_t l = 0; l + 1 < sizes.size(); ++l) {
    double phi = 0.0;
    cplx w[3];
    if (!poly_smoother(h->k, 1.0 / (sizes[l] + 1), h->theta_beta, h->theta_gamma, h->dim, &phi, w)) {
      std::ostringstream msg;
      msg << "no stable third-degree polynomial smoother on the level n = " << sizes[l]
          << " (theta_beta too small for this k, Sec. 4.5)";
      set_error(msg.str());
      return HELM_EINVAL;
    }
    for (int j = 0; j < 3; ++j) ws[l][j] = w[j];
  }
  h->polyw.swap(ws);
  return HELM_OK;
}

int setup_handle(const helm_grid* grid, const float* phi, double k, double theta_beta, const helm_opts* opts,
                 cudaStream_t st, Handle** out) {
  if (!grid || !out) { set_error("grid and out must not be NULL"); return HELM_EINVAL; }
  tune_load_default();  // the tuned launch choices, read once per process
  std::unique_ptr<Handle> h(new Handle());
  h->dim = grid->dim;
  h->n = grid->n;
  h->ecs = grid->ecs_frac > 0 ? grid->ecs_frac : 0.125;
  h->theta_gamma = grid->theta_gamma;
  h->ecs_sides = grid->ecs_sides;
  h->theta_beta = theta_beta;
  h->k = k;
  h->has_phi = phi != nullptr;
  helm_opts o{};
  if (opts) o = *opts;
  h->nu1 = o.nu1 > 0 ? o.nu1 : (opts && o.nu1 == 0 && o.nu2 > 0 ? 0 : 1);
  h->nu2 = o.nu2 > 0 ? o.nu2 : (opts && o.nu2 == 0 && o.nu1 > 0 ? 0 : 1);
  h->s = o.s > 0 ? o.s : 3;
  h->coarsest = o.coarsest_n > 0 ? o.coarsest_n : 3;
  h->prec = o.precond_prec ? o.precond_prec : HELM_C64;
  if (h->prec == HELM_CAUTO && (h->dim == 2 || h->dim == 3) && h->n >= 1) {
    const double pts = h->dim == 3 ? (double)h->n * h->n * h->n : (double)h->n * h->n;
    h->prec = pts <= HELM_AUTO_C128_POINTS ? HELM_C128 : HELM_C64;
  }
  h->restart = o.restart > 0 ? o.restart : 0;
  h->maxit = o.maxit > 0 ? o.maxit : 400;
  h->csl_eps = o.csl_eps;
  h->smoother = o.smoother;
  h->basis = o.outer_basis;
  if (h->basis != HELM_BASIS_AUTO && h->basis != HELM_BASIS_F64 && h->basis != HELM_BASIS_DF) {
    set_error("outer_basis must be HELM_BASIS_AUTO, HELM_BASIS_F64 or HELM_BASIS_DF");
    return HELM_EINVAL;
  }
  if (h->dim != 2 && h->dim != 3) { set_error("dim must be 2 or 3"); return HELM_EINVAL; }
  if (h->n < 1 || h->n > (h->dim == 2 ? 32767 : 2047)) { set_error("n out of range"); return HELM_EINVAL; }
  if (h->ecs_sides != HELM_ECS_BOTH && h->ecs_sides != HELM_ECS_HIGH) {
    set_error("ecs_sides must be HELM_ECS_BOTH or HELM_ECS_HIGH");
    return HELM_EINVAL;
  }
  if (!(h->ecs > 0 && h->ecs < (h->ecs_sides == HELM_ECS_BOTH ? 0.5 : 1.0))) {
    set_error("ecs_frac must be in (0, 0.5) with layers on both sides, (0, 1) with one");
    return HELM_EINVAL;
  }
  if (!(h->theta_gamma >= 0 && h->theta_gamma < M_PI / 2)) { set_error("theta_gamma must be in [0, pi/2)"); return HELM_EINVAL; }
  if (!(theta_beta >= 0 && theta_beta < M_PI / 2)) { set_error("theta_beta must be in [0, pi/2)"); return HELM_EINVAL; }
  if (h->s > SMAX) { set_error("s must be in 1..4"); return HELM_EINVAL; }
  if (h->nu1 > 8 || h->nu2 > 8) { set_error("nu1, nu2 must be <= 8"); return HELM_EINVAL; }
  if (h->prec != HELM_C64 && h->prec != HELM_C128) { set_error("precond_prec must be HELM_C64, HELM_C128 or HELM_CAUTO"); return HELM_EINVAL; }
  if (!(std::isfinite(h->csl_eps) && h->csl_eps >= 0.0)) { set_error("csl_eps must be finite and >= 0"); return HELM_EINVAL; }
  if (h->csl_eps != 0.0 && phi) { set_error("the complex shift (csl_eps) needs a constant k"); return HELM_EINVAL; }
  if (h->smoother != HELM_SMOOTHER_GMRES && h->smoother != HELM_SMOOTHER_POLY) {
    set_error("smoother must be HELM_SMOOTHER_GMRES or HELM_SMOOTHER_POLY");
    return HELM_EINVAL;
  }
  if (h->smoother == HELM_SMOOTHER_POLY && (phi || h->csl_eps != 0.0 || !(theta_beta < h->theta_gamma))) {
    set_error("the polynomial smoother needs a constant k, csl_eps = 0 and theta_beta < theta_gamma");
    return HELM_EINVAL;
  }
  // the polynomial smoother's steps alternate through p_0 and p_1
  if (h->smoother == HELM_SMOOTHER_POLY && h->s < 2) h->s = 2;
  if (!phi && !std::isfinite(k)) { set_error("k must be finite"); return HELM_EINVAL; }
  const std::vector<int> sizes = level_sizes(h->n, h->coarsest);
  const int nlev = (int)sizes.size();
  const int cm = h->dim == 3 ? sizes.back() * sizes.back() * sizes.back() : sizes.back() * sizes.back();
  if (cm > 128) {
    set_error("coarsest grid has more than 128 unknowns: n+1 must be divisible by a larger power of two, or lower coarsest_n");
    return HELM_EINVAL;
  }
  if (h->smoother == HELM_SMOOTHER_POLY) TRY(compute_poly_weights(h.get(), sizes));
  h->m = h->restart > 0 ? std::min(h->restart, h->maxit) : h->maxit;
  if (h->m > HELM_MAX_BASIS) {
    set_error("Krylov basis length min(restart, maxit) exceeds HELM_MAX_BASIS");
    return HELM_EINVAL;
  }
  const size_t eb = elem_bytes(h->prec);

  // ------------------------------------------------ page-locked upload staging
  {
    auto r256 = [](size_t b) { return (b + 255) / 256 * 256; };
    size_t off = r256(sizeof(OuterState));
    h->stage_lu = off;
    off += r256((size_t)cm * cm * sizeof(double2));
    h->stage_piv = off;
    off += r256((size_t)cm * sizeof(int));
    h->stage_coef.resize(nlev);
    for (int l = 0; l < nlev; ++l) {
      h->stage_coef[l] = off;
      off += r256(3 * (size_t)sizes[l] * (sizeof(double2) + eb));
    }
    void* p = nullptr;
    CUDA_TRY(cudaMallocHost(&p, off));
    h->stage = static_cast<char*>(p);
  }
  // ------------------------------------------------ levels
  h->lev.resize(nlev);
  for (int l = 0; l < nlev; ++l) {
    HostLevel& L = h->lev[l];
    L.n = sizes[l];
    L.P = L.n + 1;
    L.np = h->dim == 3 ? (size_t)L.P * L.P * L.P : (size_t)L.P * L.P;
    const TileCfg cfg = default_tiles(h->dim, L.P);
    if (l == 0) h->cfg = cfg;
    L.ntiles = vtiles(h->dim, L.P);
    // flat passes: one wave of four CTAs per SM at most (their occupancy), so every CTA
    // streams an equal share and no partial second wave trails
    L.nflat = (int)std::max<size_t>(1, std::min<size_t>(std::min(1024, 4 * sm_count_host()), (L.np + 1023) / 1024));
    TRY(dev_alloc(h.get(), &L.b, L.np * eb));
    TRY(dev_alloc(h.get(), &L.xa, L.np * eb));
    TRY(dev_alloc(h.get(), &L.xb, L.np * eb));
    TRY(dev_alloc(h.get(), &L.r0, L.np * eb));
    for (int j = 0; j < h->s; ++j) TRY(dev_alloc(h.get(), &L.p[j], L.np * eb));
    for (void* v : {L.b, L.xa, L.xb, L.r0}) CUDA_TRY(cudaMemsetAsync(v, 0, L.np * eb, st));
    for (int j = 0; j < h->s; ++j) CUDA_TRY(cudaMemsetAsync(L.p[j], 0, L.np * eb, st));
    const size_t scb = h->prec == HELM_C128 ? sizeof(SweepScalarsT<double>) : sizeof(SweepScalarsT<float>);
    TRY(dev_alloc(h.get(), &L.sc, scb));
    CUDA_TRY(cudaMemsetAsync(L.sc, 0, scb, st));
    // partial slots: one per tile of the marching passes, per flat-pass CTA, and per
    // share of the 3D TMA-fed pass
    size_t nparts = std::max<size_t>(std::max(L.ntiles, L.nflat), 1);
    if (h->dim == 3) {
      TileCfg finest;  // the most tiles a tuned plane count (2) gives
      finest.rows = 2;
      nparts = std::max<size_t>(nparts, std::max<size_t>(TMA3_MAX_UNITS, tiles_per_problem(3, L.P, finest)));
    }
    TRY(dev_alloc(h.get(), &L.part, nparts * NPART * sizeof(double)));
    // TMA maps of the raw vectors the complex64 Arnoldi passes stream
    // (3D: two sets, for column tiles of 16 and of 32 rows)
    if (h->prec == HELM_C64 && L.P >= 64 && (h->dim == 2 || L.P % 32 == 0)) {
      const int nmaps = h->dim == 2 ? TM_COUNT : 2 * TM_COUNT;
      std::vector<CUtensorMap> maps(nmaps);
      const void* vecs[TM_COUNT] = {};
      vecs[TM_B] = L.b;
      vecs[TM_R0] = L.r0;
      vecs[TM_XB] = L.xb;
      for (int j = 0; j < h->s; ++j) vecs[TM_P0 + j] = L.p[j];
      const bool encoded = h->dim == 2 ? encode_level_tmaps(L.P, vecs, TM_COUNT, maps.data())
                                       : encode_level_tmaps3(L.P, 18, vecs, TM_COUNT, maps.data()) &&
                                             encode_level_tmaps3(L.P, 34, vecs, TM_COUNT, maps.data() + TM_COUNT);
      if (encoded) {
        CUtensorMap* dtm = nullptr;
        TRY(dev_alloc(h.get(), &dtm, nmaps * sizeof(CUtensorMap)));
        CUDA_TRY(cudaMemcpyAsync(dtm, maps.data(), nmaps * sizeof(CUtensorMap), cudaMemcpyHostToDevice, st));
        L.tm = dtm;
      }
    }
    // coefficients of M on this level (rediscretisation with spacing 2^l h)
    TRY(dev_alloc(h.get(), &L.coef64, 3 * L.n * sizeof(double2)));
    TRY(dev_alloc(h.get(), &L.coef, 3 * L.n * eb));
    TRY(upload_level_coefficients(h.get(), l, theta_beta, st));
    // phi sampled at this level's nodes (node x of level l is fine node (x+1) 2^l - 1)
    if (phi) {
      TRY(dev_alloc(h.get(), &L.phi, L.np * sizeof(float)));
      scatter_phi(h->dim, L.n, 1 << l, h->n, phi, L.phi, st);
      CUDA_TRY(cudaGetLastError());
    } else {
      L.phic = k * k;
    }
  }
  // ------------------------------------------------ coarsest LU (FP64)
  h->lu_m = cm;
  TRY(dev_alloc(h.get(), &h->lu, (size_t)cm * cm * sizeof(double2)));
  TRY(dev_alloc(h.get(), &h->piv, cm * sizeof(int)));
  TRY(factor_coarsest(h.get(), theta_beta, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  // ------------------------------------------------ H and the outer storage
  {
    const HostLevel& L0 = h->lev[0];
    std::vector<cplx> a, d, c;
    stencil_coefficients(grid_spacings(h->n, h->ecs, h->theta_gamma, 0.0, h->ecs_sides == HELM_ECS_BOTH), a, d, c);
    std::vector<double2> hc(3 * h->n);
    for (int i = 0; i < h->n; ++i) {
      hc[i] = make_double2(a[i].real(), a[i].imag());
      hc[h->n + i] = make_double2(d[i].real(), d[i].imag());
      hc[2 * h->n + i] = make_double2(c[i].real(), c[i].imag());
    }
    TRY(dev_alloc(h.get(), &h->hcoef, hc.size() * sizeof(double2)));
    CUDA_TRY(cudaMemcpyAsync(h->hcoef, hc.data(), hc.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
    std::vector<float4> hcf(hc.size());
    auto split = [](double v, float* hi, float* lo) {
      *hi = (float)v;
      *lo = (float)(v - (double)*hi);
    };
    for (size_t i = 0; i < hc.size(); ++i) {
      split(hc[i].x, &hcf[i].x, &hcf[i].y);
      split(hc[i].y, &hcf[i].z, &hcf[i].w);
    }
    TRY(dev_alloc(h.get(), &h->hcoef_df, hcf.size() * sizeof(float4)));
    CUDA_TRY(cudaMemcpyAsync(h->hcoef_df, hcf.data(), hcf.size() * sizeof(float4), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaStreamSynchronize(st));  // hc and hcf are host staging of this frame
    h->vs = L0.np;
    h->ntiles0 = L0.ntiles;
    h->chunks = outer_chunks(h->vs);
    const int m = h->m;
    TRY(dev_alloc(h.get(), &h->bpad, h->vs * sizeof(double2)));
    TRY(dev_alloc(h.get(), &h->xpad, h->vs * sizeof(double2)));
    TRY(dev_alloc(h.get(), &h->w, h->vs * sizeof(double2)));
    TRY(dev_alloc(h.get(), &h->V, (size_t)(m + 1) * h->vs * sizeof(double2)));
    TRY(dev_alloc(h.get(), &h->Z, (size_t)m * h->vs * eb));
    TRY(dev_alloc(h.get(), &h->Hm, (size_t)(m + 1) * m * sizeof(double2)));
    TRY(dev_alloc(h.get(), &h->g, (size_t)(m + 1) * sizeof(double2)));
    TRY(dev_alloc(h.get(), &h->cs, (size_t)(m + 1) * sizeof(double)));
    TRY(dev_alloc(h.get(), &h->sn, (size_t)(m + 1) * sizeof(double2)));
    TRY(dev_alloc(h.get(), &h->y, (size_t)(m + 1) * sizeof(double2)));
    TRY(dev_alloc(h.get(), &h->hcol, (size_t)(m + 1) * sizeof(double2)));
    TRY(dev_alloc(h.get(), &h->vscale, (size_t)(m + 1) * sizeof(double)));
    const size_t op = std::max<size_t>(std::max<size_t>((size_t)max_tiles(h->dim, L0.P) * NPART,
                                                        (size_t)h->chunks * NPART),
                                       outer_part_doubles(h->chunks, m));
    TRY(dev_alloc(h.get(), &h->opart, op * sizeof(double)));
    CUDA_TRY(cudaMemsetAsync(h->opart, 0, op * sizeof(double), st));
    const int nct = outer_dot_counters(h->chunks);
    TRY(dev_alloc(h.get(), &h->dcnt, (size_t)nct * sizeof(unsigned)));
    CUDA_TRY(cudaMemsetAsync(h->dcnt, 0, (size_t)nct * sizeof(unsigned), st));
    TRY(dev_alloc(h.get(), &h->st, sizeof(OuterState)));
    CUDA_TRY(cudaMemsetAsync(h->w, 0, h->vs * sizeof(double2), st));
    CUDA_TRY(cudaMemsetAsync(h->st, 0, sizeof(OuterState), st));
  }
  CUDA_TRY(cudaStreamSynchronize(st));
  *out = h.release();
  return HELM_OK;
}

// ------------------------------------------------------------------ groups
template <typename C>
static LevelDev<C> make_leveldev(const Handle& h, int l) {
  const HostLevel& L = h.lev[l];
  LevelDev<C> d;
  std::memset(&d, 0, sizeof(d));
  d.n = L.n;
  d.P = L.P;
  d.ntiles = L.ntiles;
  d.s = h.s;
  d.b = (C*)L.b;
  d.xa = (C*)L.xa;
  d.xb = (C*)L.xb;
  d.r0 = (C*)L.r0;
  for (int j = 0; j < SMAX; ++j) d.p[j] = (C*)L.p[j];
  d.ca = (const C*)L.coef;
  d.cd = (const C*)L.coef + L.n;
  d.cc = (const C*)L.coef + 2 * L.n;
  d.phi = L.phi;
  d.phic = L.phic;
  d.phir = (typename RealOf<C>::T)L.phic;
  typedef SweepScalarsT<typename RealOf<C>::T> SS;
  d.sc = (SS*)L.sc;
  d.part = L.part;
  d.tm = L.tm;
  if (l + 1 < (int)h.lev.size()) {
    const HostLevel& Lc = h.lev[l + 1];
    d.nc = Lc.n;
    d.Pc = Lc.P;
    d.bc = (C*)Lc.b;
    d.xcb = (const C*)Lc.xb;
    d.scc = (SS*)Lc.sc;
  }
  return d;
}

template <typename C>
static OuterDev<C> make_outerdev(const Handle& h) {
  OuterDev<C> o;
  std::memset(&o, 0, sizeof(o));
  o.n = h.n;
  o.P = h.n + 1;
  o.ntiles = h.ntiles0;
  o.ca = h.hcoef;
  o.cd = h.hcoef + h.n;
  o.cc = h.hcoef + 2 * h.n;
  o.cdf = h.hcoef_df;
  o.phi = h.lev[0].phi;
  o.phic = h.lev[0].phic;
  o.bpad = h.bpad;
  o.xpad = h.xpad;
  o.w = h.w;
  o.V = h.V;
  o.Z = (C*)h.Z;
  o.b0 = (C*)h.lev[0].b;
  o.zout = (const C*)h.lev[0].xb;
  o.s = h.s;
  o.vs = h.vs;
  o.Hm = h.Hm;
  o.g = h.g;
  o.cs = h.cs;
  o.sn = h.sn;
  o.y = h.y;
  o.hcol = h.hcol;
  o.vscale = h.vscale;
  o.part = h.opart;
  o.gcnt = h.dcnt;
  o.st = h.st;
  o.sc0 = (SweepScalarsT<typename RealOf<C>::T>*)h.lev[0].sc;
  return o;
}

template <typename C>
struct Group {
  int dim = 2, nu1 = 1, nu2 = 1, s = 3, Lmax = 0, tc = 0, nprob = 0;
  int smoother = HELM_SMOOTHER_GMRES;
  TileCfg cfg{8};
  std::vector<Handle*> hs;
  struct Depth {
    int n = 0, cnt = 0, ntiles = 0, nflat = 0;
    bool tma = true;  // every problem at this depth has TMA maps
    TileCfg cfg{8};
    LevelDev<C>* d = nullptr;
    C* pw = nullptr;  // polynomial smoother: three Richardson weights per problem
  };
  std::vector<Depth> depth;      // t < tc
  LevelDev<C>* dcoarse = nullptr;  // [prob][Lmax - tc]
  int nlev_c = 0;
  size_t coarse_smem = 0;          // dynamic shared memory of the staged coarse kernel (0: global)
  CoarseLU* dlu = nullptr;
  struct Sub {
    int n = 0, cnt = 0, ntiles = 0, chunks = 1, m = 1;
    TileCfg cfg{8};
    OuterDev<C>* d = nullptr;
    std::vector<Handle*> members;
    double sum_j1 = 0;   // sum of (j + 1) over members at the last state read (profiling)
  };
  std::vector<Sub> outer;
  LevelDev<C>* lev0 = nullptr;   // level-0 descriptors of all problems (single problem: [0])
  int lev0_nflat = 1;
  GridBar* gbar = nullptr;       // grid barrier of the persistent segments
  int tp = 0;                    // first depth of the persistent segments (tc: none)
  void* dmem = nullptr;
  bool owns = true;              // dmem and cap_stream belong to the group (not to an arena)
  // the V-cycle captured as a CUDA graph (re-captured when profiling starts or stops)
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t vexec = nullptr;
  int vexec_gen = -1;
  int vkernels = 0;
  int direct_runs = 0;           // V-cycles launched directly (before the graph is captured)
  std::vector<GraphRec> vrecs;
  ~Group() {
    if (vexec) cudaGraphExecDestroy(vexec);
    release(vrecs);
    if (owns && cap_stream) cudaStreamDestroy(cap_stream);
    if (owns && dmem) cudaFree(dmem);
  }
};

// Device memory for the descriptor arrays of successive groups, grown only, and the
// stream their V-cycles are captured on: a set whose membership changes often
// rebuilds its group without cudaFree (which would wait for every stream of the
// device) and without creating streams.
struct GroupArena {
  void* p = nullptr;
  size_t cap = 0;
  void* hp = nullptr;      // page-locked staging of the descriptor uploads (same layout as p)
  size_t hcap = 0;
  cudaStream_t cap_stream = nullptr;
  ~GroupArena() {
    if (p) cudaFree(p);
    if (hp) cudaFreeHost(hp);
    if (cap_stream) cudaStreamDestroy(cap_stream);
  }
};

template <typename C>
static int build_group(Handle* const* hs, int count, cudaStream_t st, Group<C>* g, GroupArena* arena = nullptr) {
  g->hs.assign(hs, hs + count);
  g->nprob = count;
  const Handle& h0 = *hs[0];
  g->dim = h0.dim;
  g->nu1 = h0.nu1;
  g->nu2 = h0.nu2;
  g->s = h0.s;
  g->smoother = h0.smoother;
  g->cfg = h0.cfg;
  for (int p = 0; p < count; ++p) {
    const Handle& h = *hs[p];
    if (h.dim != h0.dim || h.prec != h0.prec || h.nu1 != h0.nu1 || h.nu2 != h0.nu2 || h.s != h0.s ||
        h.smoother != h0.smoother || h.lev.back().n != h0.lev.back().n) {
      set_error("batched problems must share dim, precision, nu1, nu2, s, the smoother and the coarsest size");
      return HELM_EINVAL;
    }
    g->Lmax = std::max(g->Lmax, (int)h.lev.size());
  }
  std::vector<int> off(count);
  int maxoff = 0;
  for (int p = 0; p < count; ++p) {
    off[p] = g->Lmax - (int)hs[p]->lev.size();
    maxoff = std::max(maxoff, off[p]);
  }
  // first depth handled by the single-CTA coarse kernel
  int tthr = g->Lmax - 1;
  {
    // sizes by depth (from the deepest-reaching problem)
    const Handle* big = nullptr;
    for (int p = 0; p < count; ++p) if (off[p] == 0) big = hs[p];
    for (int t = 0; t < g->Lmax; ++t)
      if (big->lev[t].n <= coarse_threshold(g->dim)) { tthr = t; break; }
  }
  // the split depends on the level sizes only, never on the other problems: a problem
  // whose finest level is already coarse runs its whole cycle in the coarse kernel
  g->tc = std::min(tthr, g->Lmax - 1);
  // the polynomial smoother runs every level but the coarsest grid-wide; the coarse
  // kernel then only solves the coarsest level
  if (g->smoother == HELM_SMOOTHER_POLY) g->tc = g->Lmax - 1;
  g->nlev_c = g->Lmax - g->tc;
  (void)maxoff;
  {
    // shared-memory footprint of the coarse levels (a function of the level sizes only)
    const Handle* big = nullptr;
    for (int p = 0; p < count; ++p) if (off[p] == 0) big = hs[p];
    size_t bytes = 0;
    for (int t = g->tc; t < g->Lmax; ++t) bytes += (size_t)(4 + g->s) * big->lev[t].np * sizeof(C);
    g->coarse_smem = (g->nlev_c <= MAX_COARSE_LEVELS_HOST && bytes <= 200 * 1024) ? bytes : 0;
  }
  // tile config of a group: the first problem's
  for (int p = 0; p < count; ++p)
    if (hs[p]->cfg.rows != g->cfg.rows && off[p] == 0) g->cfg = hs[p]->cfg;
  // host descriptor arrays
  std::vector<std::vector<LevelDev<C>>> dep(g->tc);
  std::vector<std::vector<C>> pws(g->tc);
  g->depth.resize(g->tc);
  for (int t = 0; t < g->tc; ++t) {
    for (int p = 0; p < count; ++p) {
      if (off[p] > t) continue;
      const int l = t - off[p];
      dep[t].push_back(make_leveldev<C>(*hs[p], l));
      if (g->smoother == HELM_SMOOTHER_POLY)
        for (int j = 0; j < 3; ++j) {
          const cplx wj = hs[p]->polyw[l][j];
          C v;
          v.x = (decltype(v.x))wj.real();
          v.y = (decltype(v.y))wj.imag();
          pws[t].push_back(v);
        }
      typename Group<C>::Depth& D = g->depth[t];
      const HostLevel& L = hs[p]->lev[l];
      if (D.cnt > 0 && D.n != L.n) { set_error("batched problems must have n + 1 a power of two"); return HELM_EINVAL; }
      D.n = L.n;
      D.cnt += 1;
      D.tma = D.tma && L.tm != nullptr;
      D.nflat = L.nflat;
      D.cfg.rows = g->dim == 3 ? tuned_zchunk(L.P, (int)sizeof(C)) : zchunk(L.P);
      D.cfg.P = L.P;
      D.ntiles = g->dim == 3 ? tiles_per_problem(3, L.P, D.cfg) : L.ntiles;
    }
  }
  std::vector<LevelDev<C>> coarse;
  std::vector<CoarseLU> lus;
  for (int p = 0; p < count; ++p) {
    // the problem's coarse levels (depths t0 .. Lmax-1) first, then padding up to the stride
    const int t0 = std::max(g->tc, off[p]);
    const int coarsest = (int)hs[p]->lev.size() - 1;
    for (int k = 0; k < g->nlev_c; ++k) {
      const int t = t0 + k;
      coarse.push_back(make_leveldev<C>(*hs[p], t < g->Lmax ? t - off[p] : coarsest));
    }
    CoarseLU c;
    c.nlev = g->Lmax - t0;
    c.m = hs[p]->lu_m;
    c.lu = hs[p]->lu;
    c.piv = hs[p]->piv;
    lus.push_back(c);
  }
  std::vector<LevelDev<C>> lev0;
  for (int p = 0; p < count; ++p) lev0.push_back(make_leveldev<C>(*hs[p], 0));
  g->lev0_nflat = hs[0]->lev[0].nflat;
  // outer subgroups by top size
  std::vector<std::vector<OuterDev<C>>> subs;
  for (int p = 0; p < count; ++p) {
    const Handle& h = *hs[p];
    int si = -1;
    for (size_t q = 0; q < g->outer.size(); ++q) if (g->outer[q].n == h.n) si = (int)q;
    if (si < 0) {
      typename Group<C>::Sub S;
      S.n = h.n;
      S.cfg = h.cfg;
      S.ntiles = tiles_per_problem(g->dim, h.n + 1, h.cfg);
      S.chunks = h.chunks;
      S.m = h.m;
      g->outer.push_back(S);
      subs.emplace_back();
      si = (int)g->outer.size() - 1;
    }
    g->outer[si].cnt += 1;
    g->outer[si].members.push_back(hs[p]);
    g->outer[si].m = std::max(g->outer[si].m, h.m);
    subs[si].push_back(make_outerdev<C>(h));
  }
  // one device allocation for every descriptor array
  size_t bytes = 0;
  for (int t = 0; t < g->tc; ++t) bytes += dep[t].size() * sizeof(LevelDev<C>) + pws[t].size() * sizeof(C) + 64;
  bytes += coarse.size() * sizeof(LevelDev<C>) + lus.size() * sizeof(CoarseLU) + lev0.size() * sizeof(LevelDev<C>);
  for (auto& v : subs) bytes += v.size() * sizeof(OuterDev<C>);
  bytes += 64 * (g->tc + subs.size() + 4);
  if (arena) {
    // the caller guarantees that no launch of the previous group is still in flight
    if (arena->cap < bytes) {
      if (arena->p) CUDA_TRY(cudaFree(arena->p));
      arena->p = nullptr;
      arena->cap = 0;
      CUDA_TRY(cudaMalloc(&arena->p, 2 * bytes));
      arena->cap = 2 * bytes;
    }
    if (arena->hcap < bytes) {
      if (arena->hp) CUDA_TRY(cudaFreeHost(arena->hp));
      arena->hp = nullptr;
      arena->hcap = 0;
      CUDA_TRY(cudaMallocHost(&arena->hp, 2 * bytes));
      arena->hcap = 2 * bytes;
    }
    if (!arena->cap_stream) CUDA_TRY(cudaStreamCreateWithFlags(&arena->cap_stream, cudaStreamNonBlocking));
    g->owns = false;
    g->dmem = arena->p;
    g->cap_stream = arena->cap_stream;
  } else {
    CUDA_TRY(cudaMalloc(&g->dmem, bytes));
  }
  // Arena groups upload from the arena's page-locked staging: the copies then never wait
  // for the work already queued on the stream (a set's stream may carry request
  // inputs and results), and the previous group's copies have completed, since its
  // iteration has.  Other groups upload from pageable memory and synchronise below.
  char* cur = (char*)g->dmem;
  char* hstage = arena ? static_cast<char*>(arena->hp) : nullptr;
  auto put = [&](const void* src, size_t nb) -> void* {
    void* dst = cur;
    if (nb) {
      const void* from = src;
      if (hstage) {
        char* hs = hstage + (cur - (char*)g->dmem);
        std::memcpy(hs, src, nb);
        from = hs;
      }
      cudaMemcpyAsync(dst, from, nb, cudaMemcpyHostToDevice, st);
    }
    cur += (nb + 63) / 64 * 64;
    return dst;
  };
  for (int t = 0; t < g->tc; ++t) g->depth[t].d = (LevelDev<C>*)put(dep[t].data(), dep[t].size() * sizeof(LevelDev<C>));
  for (int t = 0; t < g->tc; ++t)
    if (!pws[t].empty()) g->depth[t].pw = (C*)put(pws[t].data(), pws[t].size() * sizeof(C));
  g->dcoarse = (LevelDev<C>*)put(coarse.data(), coarse.size() * sizeof(LevelDev<C>));
  g->dlu = (CoarseLU*)put(lus.data(), lus.size() * sizeof(CoarseLU));
  g->lev0 = (LevelDev<C>*)put(lev0.data(), lev0.size() * sizeof(LevelDev<C>));
  for (size_t q = 0; q < subs.size(); ++q) g->outer[q].d = (OuterDev<C>*)put(subs[q].data(), subs[q].size() * sizeof(OuterDev<C>));
  const GridBar gb0{0u, 0u};
  g->gbar = (GridBar*)put(&gb0, sizeof(GridBar));
  // the persistent segments: the deepest run of grid-wide levels that qualify
  // (bounded by the pass list's capacity: a depth records nu1 (s + 1) passes going down
  // and 1 + nu2 (s + 1) coming up)
  g->tp = g->tc;
  const int per_depth = std::max(g->nu1 == 0 ? 1 : g->nu1 * (g->s + 1), 1 + g->nu2 * (g->s + 1));
  if (g->smoother == HELM_SMOOTHER_GMRES)
    while (g->tp > 0 && (g->tc - g->tp + 1) * per_depth <= SEQ_MAX &&
           persist_level(g->dim, g->depth[g->tp - 1].n + 1, (int)sizeof(C)))
      --g->tp;
  CUDA_TRY(cudaGetLastError());
  if (!arena) CUDA_TRY(cudaStreamSynchronize(st));
  return HELM_OK;
}

// One V(nu1, nu2) cycle from a zero guess on every problem of the group (Sec. 3.1).
// Algorithmic bytes per launch count every vector the pass must read or write once
// (E bytes per complex value), plus 4 bytes per point for a phi field.
// One V(nu1, nu2) cycle with the polynomial smoother of Sec. 4: every level but the
// coarsest grid-wide.  A sweep is three Richardson steps; the steps of a sweep go
// through the level's p_0 / p_1 vectors and the last one lands in x_a (pre-smoothing,
// the prolongation's input) or x_b (post-smoothing, the level's output).
template <typename C>
static void run_vcycle_poly(const Group<C>& g, cudaStream_t st) {
  const int dim = g.dim;
  const double E = sizeof(C);
  const double cf = 1.0 / (dim == 3 ? 8.0 : 4.0);
  auto sweeps = [&](const typename Group<C>::Depth& D, int nsw, int first_src, int last_dst, bool fine) {
    const double pts = (double)D.cnt * (dim == 3 ? (double)(D.n + 1) * (D.n + 1) * (D.n + 1) : (double)(D.n + 1) * (D.n + 1));
    const int steps = 3 * nsw;
    for (int k = 0; k < steps; ++k) {
      const int src = k == 0 ? first_src : (k % 2 == 1 ? POLY_P0 : POLY_P1);
      const int dst = k == steps - 1 ? last_dst : (k % 2 == 0 ? POLY_P0 : POLY_P1);
      Launch L(fine ? "vc.poly.l0" : "vc.poly.lc", st, pts * E * (src == POLY_NONE ? 2.0 : 3.0), 0);
      launch_poly_step<C>(dim, D.d, D.pw, D.cnt, D.nflat, src, dst, k % 3, st);
    }
  };
  for (int t = 0; t < g.tc; ++t) {
    const auto& D = g.depth[t];
    const double pts = (double)D.cnt * (dim == 3 ? (double)(D.n + 1) * (D.n + 1) * (D.n + 1) : (double)(D.n + 1) * (D.n + 1));
    const bool fine = (t == 0);
    if (g.nu1 == 0) {
      Launch L(fine ? "vc.poly.l0" : "vc.poly.lc", st, pts * E, 0);
      launch_poly_step<C>(dim, D.d, D.pw, D.cnt, D.nflat, POLY_NONE, POLY_XA, -1, st);  // x_a = 0
    } else {
      sweeps(D, g.nu1, POLY_NONE, POLY_XA, fine);
    }
    Launch L(fine ? "vc.restrict.l0" : "vc.restrict.lc", st, pts * E * (3.0 + cf), 0, 2);
    launch_poly_restrict<C>(dim, D.d, D.cnt, D.nflat, POLY_XA, st);
  }
  {
    Launch L("vc.coarse", st, 0, 0);
    if (g.coarse_smem > 0)
      launch_coarse_smem<C>(dim, g.dcoarse, g.nlev_c, g.nlev_c, g.dlu, g.nprob, g.nu1, g.nu2, g.coarse_smem, st);
    else
      launch_coarse_cluster<C>(dim, g.dcoarse, g.nlev_c, g.dlu, g.nprob, g.nu1, g.nu2, st);
  }
  for (int t = g.tc - 1; t >= 0; --t) {
    const auto& D = g.depth[t];
    const double pts = (double)D.cnt * (dim == 3 ? (double)(D.n + 1) * (D.n + 1) * (D.n + 1) : (double)(D.n + 1) * (D.n + 1));
    const bool fine = (t == 0);
    {
      Launch L(fine ? "vc.prolong.l0" : "vc.prolong.lc", st, pts * E * (2.0 + cf), 0);
      launch_prolong<C>(dim, false, D.d, D.cnt, D.nflat, D.cfg, false, st);  // x_b = x_a + P e_c
    }
    if (g.nu2 > 0) sweeps(D, g.nu2, POLY_XB, POLY_XB, fine);
  }
}

template <typename C>
static void run_vcycle(const Group<C>& g, cudaStream_t st) {
  if (g.smoother == HELM_SMOOTHER_POLY) {
    run_vcycle_poly<C>(g, st);
    return;
  }
  const int dim = g.dim;
  const double E = sizeof(C);
  const double cf = 1.0 / (dim == 3 ? 8.0 : 4.0);
  // The depths t >= g.tp run as two persistent launches (descent, ascent): their passes
  // are recorded instead of launched; bytes counts their algorithmic bytes.
  PassSeq seq;
  seq.npass = 0;
  double seq_bytes = 0;
  auto flush = [&](const char* name) {
    if (seq.npass == 0) return;
    Launch L(name, st, seq_bytes, 0);
    launch_seq<C>(dim, seq, g.gbar, barrier_limit_ns(), st);
    seq.npass = 0;
    seq_bytes = 0;
  };
  for (int t = 0; t < g.tc; ++t) {
    const auto& D = g.depth[t];
    const double pts = (double)D.cnt * (dim == 3 ? (double)(D.n + 1) * (D.n + 1) * (D.n + 1) : (double)(D.n + 1) * (D.n + 1));
    const bool fine = (t == 0);
    const bool rec = t >= g.tp;
    const double ph = g.hs[0]->has_phi ? 4.0 : 0.0;
    if (g.nu1 == 0) {
      if (rec) {
        record_restrict<C>(seq, dim, D.d, D.cnt, D.ntiles, D.cfg, true, true, true);
        seq_bytes += pts * E * (2.0 + cf);
        continue;
      }
      Launch L(fine ? "vc.restrict.l0" : "vc.restrict.lc", st, pts * E * (2.0 + cf), 0);
      launch_restrict<C>(dim, D.d, D.cnt, D.ntiles, D.cfg, true, true, true, st, D.tma, 1);
      continue;
    }
    for (int sw = 0; sw < g.nu1; ++sw) {
      for (int J = 1; J <= g.s; ++J) {
        if (rec) {
          record_arnoldi<C>(seq, dim, J, D.d, D.cnt, D.ntiles, D.cfg, sw == 0, true);
          seq_bytes += pts * (E * (J + 1) + ph);
          continue;
        }
        Launch L(fine ? "vc.arnoldi.l0" : "vc.arnoldi.lc", st, pts * (E * (J + 1) + ph), pts * (8.0 * (2 * dim + 1) + 8.0 * J + 4));
        launch_arnoldi<C>(dim, J, D.d, D.cnt, D.ntiles, D.cfg, sw == 0, true, D.tma, st);
      }
      if (sw < g.nu1 - 1) {
        if (rec) {
          record_update<C>(seq, dim, UPD_RESIDUAL, D.d, D.cnt, D.nflat, sw == 0, 0, sw == 0);
          seq_bytes += pts * E * (g.s + 3.0 + (sw == 0 ? 0 : 1));
          continue;
        }
        Launch L(fine ? "vc.update.l0" : "vc.update.lc", st, pts * E * (g.s + 3.0 + (sw == 0 ? 0 : 1)), 0);
        launch_update_flat<C>(dim, UPD_RESIDUAL, D.d, D.cnt, D.nflat, sw == 0, 0, sw == 0, st);
      } else {
        if (rec) {
          record_restrict<C>(seq, dim, D.d, D.cnt, D.ntiles, D.cfg, sw == 0, sw == 0, false);
          seq_bytes += pts * E * (g.s + 2.0 + cf + (sw == 0 ? 0 : 1));
          continue;
        }
        Launch L(fine ? "vc.restrict.l0" : "vc.restrict.lc", st, pts * E * (g.s + 2.0 + cf + (sw == 0 ? 0 : 1)), 0);
        launch_restrict<C>(dim, D.d, D.cnt, D.ntiles, D.cfg, sw == 0, sw == 0, false, st, D.tma, g.s + 1);
      }
    }
  }
  flush("vc.seq.down");
  {
    Launch L("vc.coarse", st, 0, 0);
    if (g.coarse_smem > 0)
      launch_coarse_smem<C>(dim, g.dcoarse, g.nlev_c, g.nlev_c, g.dlu, g.nprob, g.nu1, g.nu2, g.coarse_smem, st);
    else
      launch_coarse_cluster<C>(dim, g.dcoarse, g.nlev_c, g.dlu, g.nprob, g.nu1, g.nu2, st);
  }
  for (int t = g.tc - 1; t >= 0; --t) {
    const auto& D = g.depth[t];
    const double pts = (double)D.cnt * (dim == 3 ? (double)(D.n + 1) * (D.n + 1) * (D.n + 1) : (double)(D.n + 1) * (D.n + 1));
    const bool fine = (t == 0);
    const bool rec = t >= g.tp;
    if (!rec) flush("vc.seq.up");
    const double ph = g.hs[0]->has_phi ? 4.0 : 0.0;
    const double pbytes = g.nu2 > 0 ? pts * (E * (4.0 + cf) + ph) : pts * E * (2.0 + cf);
    if (rec) {
      record_prolong<C>(seq, dim, g.nu2 > 0, D.d, D.cnt, g.nu2 > 0 ? D.ntiles : D.nflat, D.cfg);
      seq_bytes += pbytes;
    } else {
      Launch L(fine ? "vc.prolong.l0" : "vc.prolong.lc", st, pbytes, 0,
               prolong_kernels(dim, g.nu2 > 0, (int)sizeof(C), D.tma, D.cfg.P));
      launch_prolong<C>(dim, g.nu2 > 0, D.d, D.cnt, g.nu2 > 0 ? D.ntiles : D.nflat, D.cfg, D.tma, st);
    }
    for (int sw = 0; sw < g.nu2; ++sw) {
      const bool last = (sw == g.nu2 - 1);
      for (int J = 1; J <= g.s; ++J) {
        const bool store = J < g.s || !last;
        if (rec) {
          record_arnoldi<C>(seq, dim, J, D.d, D.cnt, D.ntiles, D.cfg, false, store);
          seq_bytes += pts * (E * (J + (store ? 1 : 0)) + ph);
          continue;
        }
        Launch L(fine ? "vc.arnoldi.l0" : "vc.arnoldi.lc", st, pts * (E * (J + (store ? 1 : 0)) + ph),
                 pts * (8.0 * (2 * dim + 1) + 8.0 * J + 4));
        launch_arnoldi<C>(dim, J, D.d, D.cnt, D.ntiles, D.cfg, false, store, D.tma, st);
      }
      if (rec) {
        record_update<C>(seq, dim, last ? UPD_XONLY : UPD_RESIDUAL, D.d, D.cnt, D.nflat, false, 1, false);
        seq_bytes += pts * E * (last ? g.s + 2.0 : g.s + 4.0);
        continue;
      }
      Launch L(fine ? "vc.update.l0" : "vc.update.lc", st, pts * E * (last ? g.s + 2.0 : g.s + 4.0), 0);
      launch_update_flat<C>(dim, last ? UPD_XONLY : UPD_RESIDUAL, D.d, D.cnt, D.nflat, false, 1, false, st);
    }
  }
  flush("vc.seq.up");
}

// Host work of group (re)builds and V-cycle graph captures, for the serving counters.
static std::atomic<long long> g_group_builds{0}, g_graph_builds{0}, g_build_ns{0};
struct BuildTimer {
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  ~BuildTimer() {
    g_build_ns += std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - t0).count();
  }
};
void build_stats(long long* groups, long long* graphs, double* seconds) {
  *groups = g_group_builds.load();
  *graphs = g_graph_builds.load();
  *seconds = 1e-9 * (double)g_build_ns.load();
}

// The V-cycle as one CUDA graph: captured once per group on a private stream (and
// again whenever profiling starts or stops, so timed launches become event nodes),
// replayed on the caller's stream.
template <typename C>
static int run_vcycle_graph(Group<C>& g, cudaStream_t st) {
  const int gen = profile_generation();
  if (!g.vexec || g.vexec_gen != gen) {
    BuildTimer timer;
    g_graph_builds += 1;
    if (g.vexec) { cudaGraphExecDestroy(g.vexec); g.vexec = nullptr; }
    release(g.vrecs);
    g.vkernels = 0;
    if (!g.cap_stream) CUDA_TRY(cudaStreamCreateWithFlags(&g.cap_stream, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    capture_sink_begin(&g.vrecs, &g.vkernels);
    cudaError_t e = cudaStreamBeginCapture(g.cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      run_vcycle<C>(g, g.cap_stream);
      e = cudaStreamEndCapture(g.cap_stream, &graph);
    }
    capture_sink_end();
    CUDA_TRY(e);
    e = cudaGraphInstantiate(&g.vexec, graph, 0);
    cudaGraphDestroy(graph);
    CUDA_TRY(e);
    g.vexec_gen = gen;
  }
  CUDA_TRY(cudaGraphLaunch(g.vexec, st));
  count_launches(g.vkernels);
  return HELM_OK;
}

template <typename C>
static const LevelDev<C>* level0_desc(const Group<C>& g) {
  return g.lev0;
}

template <typename C>
static Group<C>* cached_group(Handle* h, cudaStream_t st, int* rc) {
  if (!h->group_cache) {
    Group<C>* g = new Group<C>();
    Handle* hs[1] = {h};
    *rc = build_group<C>(hs, 1, st, g);
    if (*rc != HELM_OK) { delete g; return nullptr; }
    h->group_cache = g;
  }
  *rc = HELM_OK;
  return (Group<C>*)h->group_cache;
}

template <typename C>
static int precond_apply_t(Handle* h, const void* r, void* z, int prec, cudaStream_t st) {
  int rc;
  Group<C>* g = cached_group<C>(h, st, &rc);
  if (!g) return rc;
  {
    Launch L("io.load", st, 0, 0);
    launch_load_input<C>(h->dim, g->lev0, g->lev0_nflat, r, prec, st);
  }
  run_vcycle<C>(*g, st);
  {
    Launch L("io.store", st, 0, 0);
    launch_store_output<C>(h->dim, h->n, g->lev0, z, prec, st);
  }
  CUDA_TRY(cudaGetLastError());
  return HELM_OK;
}

int precond_apply(Handle* h, const void* r, void* z, int prec, cudaStream_t st) {
  if (!h || !r || !z) { set_error("NULL argument"); return HELM_EINVAL; }
  if (prec != HELM_C64 && prec != HELM_C128) { set_error("prec must be HELM_C64 or HELM_C128"); return HELM_EINVAL; }
  return h->prec == HELM_C128 ? precond_apply_t<double2>(h, r, z, prec, st) : precond_apply_t<float2>(h, r, z, prec, st);
}

int apply_operator(Handle* h, int which, const void* v, void* w, int prec, cudaStream_t st) {
  if (!h || !v || !w) { set_error("NULL argument"); return HELM_EINVAL; }
  if (prec != HELM_C64 && prec != HELM_C128) { set_error("prec must be HELM_C64 or HELM_C128"); return HELM_EINVAL; }
  const HostLevel& L0 = h->lev[0];
  const double2* c = which == 1 ? h->hcoef : L0.coef64;
  Launch L("io.apply", st, 0, 0);
  apply_operator_dense(h->dim, h->n, c, c + h->n, c + 2 * h->n, L0.phi, L0.phic, v, w, prec, st);
  CUDA_TRY(cudaGetLastError());
  return HELM_OK;
}

// h_i = <v_i, w>, i < nvec, on caller data through the outer multi-dot pass (k_dots)
// with the basis held in the arithmetic `basis` selects: the accuracy of the FGMRES
// orthogonalisation checked apart from a solve.
int multidot(int basis, const double2* V, int nvec, size_t npts, const double2* w, double2* h_host,
             cudaStream_t st) {
  if (!V || !w || !h_host) { set_error("NULL argument"); return HELM_EINVAL; }
  if (basis != HELM_BASIS_F64 && basis != HELM_BASIS_DF) { set_error("basis must be HELM_BASIS_F64 or HELM_BASIS_DF"); return HELM_EINVAL; }
  if (nvec < 1 || nvec > HELM_MAX_BASIS + 1) { set_error("nvec must be in 1..HELM_MAX_BASIS + 1"); return HELM_EINVAL; }
  if (npts < 1 || npts > ((size_t)1 << 34)) { set_error("npts must be in 1..2^34"); return HELM_EINVAL; }
  const int m = nvec;  // column j = nvec - 1 of an (m + 1) x m Hessenberg matrix
  const int chunks = outer_chunks(npts);
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t bV = al((size_t)nvec * npts * sizeof(double2)), bw = al(npts * sizeof(double2));
  const size_t bst = al(sizeof(OuterState)), bpart = al(outer_part_doubles(chunks, m) * sizeof(double));
  const size_t bH = al((size_t)(m + 1) * m * sizeof(double2)), bcol = al((size_t)(m + 1) * sizeof(double2));
  const size_t bsc = al((size_t)(m + 1) * sizeof(double)), bod = al(sizeof(OuterDev<float2>));
  const size_t bct = al((size_t)outer_dot_counters(chunks) * sizeof(unsigned));
  char* base = nullptr;
  if (cudaMalloc(&base, bV + bw + bst + bpart + bH + bcol + bsc + bod + bct) != cudaSuccess) {
    cudaGetLastError();
    set_error("multidot: cannot allocate the workspace");
    return HELM_ENOMEM;
  }
  struct Free {
    void* p;
    ~Free() { cudaFree(p); }
  } fr{base};
  char* q = base;
  auto take = [&](size_t b) { char* r = q; q += b; return r; };
  double2* Vb = (double2*)take(bV);
  double2* wb = (double2*)take(bw);
  OuterState* dst = (OuterState*)take(bst);
  double* part = (double*)take(bpart);
  double2* Hm = (double2*)take(bH);
  double2* hcol = (double2*)take(bcol);
  double* vscale = (double*)take(bsc);
  OuterDev<float2>* od = (OuterDev<float2>*)take(bod);
  unsigned* gcnt = (unsigned*)take(bct);
  const int df = basis == HELM_BASIS_DF;
  basis_store(V, Vb, (size_t)nvec * npts, df, st);
  basis_store(w, wb, npts, df, st);
  CUDA_TRY(cudaMemsetAsync(part, 0, bpart, st));
  CUDA_TRY(cudaMemsetAsync(gcnt, 0, bct, st));
  OuterState s0;
  std::memset(&s0, 0, sizeof(s0));
  s0.j = nvec - 1;
  s0.m = m;
  s0.df = df;
  std::vector<double> ones((size_t)m + 1, 1.0);
  OuterDev<float2> o;
  std::memset(&o, 0, sizeof(o));
  o.vs = npts;
  o.V = Vb;
  o.w = wb;
  o.Hm = Hm;
  o.hcol = hcol;
  o.vscale = vscale;
  o.part = part;
  o.gcnt = gcnt;
  o.st = dst;
  // host staging lives on this frame: the stream is synchronised before it returns
  CUDA_TRY(cudaMemcpyAsync(dst, &s0, sizeof(s0), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(vscale, ones.data(), ones.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(od, &o, sizeof(o), cudaMemcpyHostToDevice, st));
  {
    Launch L("out.dots", st, 0, 0);
    outer_dots<float2>(od, 1, chunks, m, npts, st);
  }
  CUDA_TRY(cudaMemcpyAsync(h_host, hcol, (size_t)nvec * sizeof(double2), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  CUDA_TRY(cudaGetLastError());
  return HELM_OK;
}

// ------------------------------------------------------------------ FGMRES driver
// Outer kernels: bytes and flops per point of each pass (j+1 basis vectors).
template <typename C>
static double sub_points(const typename Group<C>::Sub& o, int dim) {
  const double P = o.n + 1;
  return (double)o.cnt * (dim == 3 ? P * P * P : P * P);
}

// A group's first V-cycles are launched directly; the graph is captured once the group
// has lived that long (serving and batches rebuild groups whenever membership changes,
// and a capture costs more host time than a few direct launches).
constexpr int GRAPH_AFTER = 3;

template <typename C>
static int run_iteration(Group<C>& g, cudaStream_t st) {
  if (g.direct_runs < GRAPH_AFTER) {
    run_vcycle<C>(g, st);
    g.direct_runs += 1;
  } else {
    TRY(run_vcycle_graph<C>(g, st));
  }
  const double E = sizeof(C);
  for (const auto& o : g.outer) {
    Launch L("out.apply_h", st, sub_points<C>(o, g.dim) * (16.0 + 2 * E + (g.hs[0]->has_phi ? 4.0 : 0.0)),
             sub_points<C>(o, g.dim) * (8.0 * (2 * g.dim + 1) + 4));
    outer_apply_h<C>(g.dim, o.d, o.cnt, o.ntiles, o.cfg, st);
  }
  for (const auto& o : g.outer) {
    const double pts1 = sub_points<C>(o, g.dim) / o.cnt;
    Launch L("out.dots", st, pts1 * 16.0 * (o.sum_j1 + o.cnt), pts1 * 8.0 * o.sum_j1);
    outer_dots<C>(o.d, o.cnt, o.chunks, o.m, (size_t)(sub_points<C>(o, g.dim) / o.cnt), st);
  }
  for (const auto& o : g.outer) {
    const double pts1 = sub_points<C>(o, g.dim) / o.cnt;
    Launch L("out.vnew", st, pts1 * (16.0 * (o.sum_j1 + 2 * o.cnt) + E * o.cnt), pts1 * 8.0 * (o.sum_j1 + o.cnt));
    outer_vnew<C>(o.d, o.cnt, o.chunks, o.m, false, st);
  }
  return HELM_OK;
}

// Cycle end (acts only on problems whose cycle ended): y = R^{-1} g, x += Z y, true
// residual, and v_0 of the next cycle.
template <typename C>
static void run_cycle_end(const Group<C>& g, cudaStream_t st) {
  Launch L("out.cycle_end", st, 0, 0, 4 * (int)g.outer.size());
  for (const auto& o : g.outer) outer_backsolve<C>(o.d, o.cnt, st);
  for (const auto& o : g.outer) outer_solution<C>(o.d, o.cnt, o.chunks, o.m, st);
  for (const auto& o : g.outer) outer_residual<C>(g.dim, o.d, o.cnt, o.ntiles, o.cfg, st);
  for (const auto& o : g.outer) outer_vnew<C>(o.d, o.cnt, o.chunks, o.m, true, st);
}

// ------------------------------------------------------------------ active sets
// Problems iterated together.  A problem joins with begin_problem (its state asks
// for the true residual first) and leaves when its state says done; the group and
// its V-cycle graph are rebuilt when membership changes.
static int begin_problem(Handle* h, const double2* b_dense, const double2* x_dense, double tol, cudaStream_t st) {
  {
    Launch L("io.convert", st, 0, 0, x_dense ? 2 : 1);
    convert_dense_to_padded_c128(h->dim, h->n, b_dense, h->bpad, st);
    if (x_dense) convert_dense_to_padded_c128(h->dim, h->n, x_dense, h->xpad, st);
  }
  if (!x_dense) CUDA_TRY(cudaMemsetAsync(h->xpad, 0, h->vs * sizeof(double2), st));
  OuterState& s0 = *reinterpret_cast<OuterState*>(h->stage);
  std::memset(&s0, 0, sizeof(s0));
  s0.m = h->m;
  s0.maxit = h->maxit;
  s0.tol = tol;
  const double pts = h->dim == 3 ? (double)h->n * h->n * h->n : (double)h->n * h->n;
  s0.df = h->basis == HELM_BASIS_DF ||
          (h->basis == HELM_BASIS_AUTO && tol >= HELM_BASIS_DF_MIN_TOL && pts > HELM_AUTO_C128_POINTS);
  s0.bnorm = -1.0;
  s0.need_residual = 1;
  CUDA_TRY(cudaMemcpyAsync(h->st, &s0, sizeof(s0), cudaMemcpyHostToDevice, st));
  h->last_j = 0;
  CUDA_TRY(cudaGetLastError());
  return HELM_OK;
}

static int finish_problem(Handle* h, const OuterState& s, double2* x_dense, cudaStream_t st, helm_info* info) {
  if (s.bnorm == 0.0) {
    // b = 0: the solution is x = 0 whatever the initial guess
    const size_t npts = h->dim == 3 ? (size_t)h->n * h->n * h->n : (size_t)h->n * h->n;
    CUDA_TRY(cudaMemsetAsync(x_dense, 0, npts * sizeof(double2), st));
  } else {
    Launch L("io.convert", st, 0, 0);
    convert_padded_to_dense_c128(h->dim, h->n, h->xpad, x_dense, st);
  }
  const int status = s.done == 1 ? HELM_OK : (s.done == 3 ? HELM_ENUMERIC : HELM_ENOCONV);
  if (info) {
    info->iters = s.iters;
    info->restarts = s.restarts;
    info->rel_res_est = s.rel_est;
    info->rel_res_true = s.rel_true;
    info->status = status;
    info->basis = s.df ? HELM_BASIS_DF : HELM_BASIS_F64;
  }
  CUDA_TRY(cudaGetLastError());
  return status;
}

template <typename C>
struct ActiveSet {
  std::vector<Handle*> members;
  std::unique_ptr<Group<C>> own;
  Group<C>* g = nullptr;
  GroupArena* arena = nullptr;  // set: groups are built in it, never from a handle's cache
  bool dirty = true;       // membership changed since the group was built
  bool fresh = false;      // members joined: run their first cycle end before iterating
  Group<C>* graph_pending = nullptr;
  OuterState* pin = nullptr;
  size_t pin_cap = 0;
  size_t n_read = 0;       // members whose state the last iterate() enqueued for reading
  // device copies: the members' state pointers (uploaded at each rebuild) and the
  // gathered states
  OuterState** d_src = nullptr;
  OuterState* d_stage = nullptr;
  OuterState** h_src = nullptr;  // page-locked source of d_src
  size_t d_cap = 0;
  ~ActiveSet() {
    if (pin) cudaFreeHost(pin);
    if (h_src) cudaFreeHost(h_src);
    if (d_src) cudaFree(d_src);
    if (d_stage) cudaFree(d_stage);
  }

  void add(Handle* h) {
    members.push_back(h);
    dirty = true;
    fresh = true;
  }
  int rebuild(cudaStream_t st) {
    BuildTimer timer;
    g_group_builds += 1;
    own.reset();
    g = nullptr;
    dirty = false;
    if (members.size() == 1 && !arena) {
      int rc;
      g = cached_group<C>(members[0], st, &rc);
      return rc;
    }
    own.reset(new Group<C>());
    g = own.get();
    return build_group<C>(members.data(), (int)members.size(), st, g, arena);
  }
  // The members' state pointers on the device, for the per-iteration gather.
  int upload_state_pointers(cudaStream_t st) {
    if (d_cap < members.size()) {
      if (d_src) CUDA_TRY(cudaFree(d_src));
      if (d_stage) CUDA_TRY(cudaFree(d_stage));
      if (h_src) CUDA_TRY(cudaFreeHost(h_src));
      d_src = nullptr;
      d_stage = nullptr;
      h_src = nullptr;
      d_cap = std::max<size_t>(2 * members.size(), 16);
      CUDA_TRY(cudaMalloc(&d_src, d_cap * sizeof(OuterState*)));
      CUDA_TRY(cudaMalloc(&d_stage, d_cap * sizeof(OuterState)));
      CUDA_TRY(cudaMallocHost(&h_src, d_cap * sizeof(OuterState*)));
    }
    // the previous upload from h_src has completed: the set's last iteration has
    for (size_t p = 0; p < members.size(); ++p) h_src[p] = members[p]->st;
    CUDA_TRY(cudaMemcpyAsync(d_src, h_src, members.size() * sizeof(OuterState*), cudaMemcpyHostToDevice, st));
    return HELM_OK;
  }
  // Enqueue one outer iteration of every member (plus the first cycle end of new
  // members), the gather of the members' states and their copy to pinned host memory.
  int iterate(cudaStream_t st) {
    n_read = 0;
    if (members.empty()) return HELM_OK;
    if (dirty) {
      TRY(rebuild(st));
      TRY(upload_state_pointers(st));
    }
    if (fresh) {
      run_cycle_end<C>(*g, st);
      fresh = false;
    }
    for (auto& o : g->outer) {
      o.sum_j1 = 0;
      for (Handle* m : o.members) o.sum_j1 += m->last_j + 1;
    }
    TRY(run_iteration<C>(*g, st));
    run_cycle_end<C>(*g, st);
    CUDA_TRY(cudaGetLastError());
    graph_pending = g;
    if (pin_cap < members.size()) {
      if (pin) CUDA_TRY(cudaFreeHost(pin));
      pin = nullptr;
      pin_cap = std::max<size_t>(2 * members.size(), 16);
      CUDA_TRY(cudaMallocHost(&pin, sizeof(OuterState) * pin_cap));
    }
    {
      Launch L("io.state", st, 0, 0);
      gather_states(d_src, d_stage, (int)members.size(), st);
    }
    CUDA_TRY(cudaMemcpyAsync(pin, d_stage, members.size() * sizeof(OuterState), cudaMemcpyDeviceToHost, st));
    n_read = members.size();
    return HELM_OK;
  }
  // Wait for the last iterate() (synchronises st); finished members move to `done`.
  // Members added since that iterate() stay.
  int collect(cudaStream_t st, std::vector<std::pair<Handle*, OuterState>>* done) {
    if (n_read == 0) return HELM_OK;
    CUDA_TRY(cudaStreamSynchronize(st));
    if (graph_pending) {
      harvest(graph_pending->vrecs);  // timed V-cycle launches of the replay just completed
      graph_pending = nullptr;
    }
    std::vector<Handle*> still;
    for (size_t p = 0; p < members.size(); ++p) {
      if (p >= n_read) { still.push_back(members[p]); continue; }
      members[p]->last_j = pin[p].j;
      if (pin[p].done) done->push_back({members[p], pin[p]});
      else still.push_back(members[p]);
    }
    n_read = 0;
    if (still.size() != members.size()) {
      members = still;
      dirty = true;
    }
    return HELM_OK;
  }
};

// Side streams per host thread for batched solves.
constexpr int MAX_SETS = 4;
static cudaStream_t side_stream(int k) {
  thread_local cudaStream_t s[MAX_SETS] = {nullptr, nullptr, nullptr, nullptr};
  if (!s[k]) cudaStreamCreateWithFlags(&s[k], cudaStreamNonBlocking);
  return s[k];
}

// Batched solve.  The batch is split into two (fewer than 8 problems) or MAX_SETS sets
// that iterate on their own streams: one set's latency-bound V-cycle levels run beside another's FP64-bound
// outer passes.  Each problem's arithmetic does not depend on the grouping, so results
// are the same as in one group or alone.
template <typename C>
static int solve_t(Handle* const* hs, int count, const double* const* b, double* const* x, double tol,
                   helm_info* infos, cudaStream_t st) {
  // measured on GB300: two sets for a handful of problems, four for larger batches
  const int nsets = count >= 8 ? MAX_SETS : std::max(1, std::min(count, 2));
  cudaStream_t sts[MAX_SETS];
  sts[0] = st;
  for (int k = 1; k < nsets; ++k) {
    sts[k] = side_stream(k);
    if (!sts[k]) { set_error("cudaStreamCreate failed"); return HELM_ECUDA; }
  }
  ActiveSet<C> sets[MAX_SETS];
  for (int p = 0; p < count; ++p) {
    TRY(begin_problem(hs[p], (const double2*)b[p], (const double2*)x[p], tol, st));
    sets[p % nsets].add(hs[p]);
  }
  cudaEvent_t ev = nullptr;
  if (nsets > 1) {  // the side streams start after the inputs are in place
    CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CUDA_TRY(cudaEventRecord(ev, st));
    for (int k = 1; k < nsets; ++k) CUDA_TRY(cudaStreamWaitEvent(sts[k], ev, 0));
  }
  std::vector<std::pair<Handle*, OuterState>> done;
  int max_maxit = 0;
  for (int p = 0; p < count; ++p) max_maxit = std::max(max_maxit, hs[p]->maxit);
  // The first iterate() runs every problem's initial residual before its first
  // V-cycle.  Each half is relaunched as soon as its own iteration has finished, so
  // the two drift into different phases.
  int rc = HELM_OK;
  bool inflight[MAX_SETS] = {false, false, false, false};
  int rounds[MAX_SETS] = {0, 0, 0, 0};
  const int guard = 2 * max_maxit + 4;
  while (rc == HELM_OK) {
    bool busy = false;
    for (int k = 0; k < nsets && rc == HELM_OK; ++k) {
      if (inflight[k]) {
        const cudaError_t q = nsets == 1 ? cudaSuccess : cudaStreamQuery(sts[k]);
        if (q == cudaErrorNotReady) { busy = true; continue; }
        if (q != cudaSuccess) { set_error(cudaGetErrorString(q)); rc = HELM_ECUDA; break; }
        rc = sets[k].collect(sts[k], &done);
        inflight[k] = false;
      }
      if (rc == HELM_OK && !sets[k].members.empty() && rounds[k] <= guard) {
        rc = sets[k].iterate(sts[k]);
        inflight[k] = true;
        rounds[k] += 1;
        busy = true;
      }
    }
    if (!busy) break;
  }
  if (nsets > 1) {  // the main stream continues after the side streams' work
    for (int k = 1; k < nsets && rc == HELM_OK; ++k) {
      cudaError_t e = cudaEventRecord(ev, sts[k]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev, 0);
      if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); rc = HELM_ECUDA; }
    }
    cudaEventDestroy(ev);
  }
  TRY(rc);
  if (vcycle_take_error()) {
    set_error("a V-cycle kernel's bounded wait ran out (its tile copies, or the persistent segment's grid barrier)");
    return HELM_ETIMEOUT;
  }
  for (int k = 0; k < nsets; ++k)
    for (Handle* h : sets[k].members) {  // only on a failed guard: report what they have
      OuterState s;
      CUDA_TRY(cudaMemcpy(&s, h->st, sizeof(s), cudaMemcpyDeviceToHost));
      done.push_back({h, s});
    }
  int rc_all = HELM_OK;
  for (int p = 0; p < count; ++p) {
    for (auto& d : done) {
      if (d.first != hs[p]) continue;
      const int status = finish_problem(hs[p], d.second, (double2*)x[p], st, infos ? infos + p : nullptr);
      if (status != HELM_OK && rc_all == HELM_OK) rc_all = status;
    }
  }
  CUDA_TRY(cudaStreamSynchronize(st));
  return rc_all;
}

// ------------------------------------------------------------------ runners (serving)
struct BatchRunner {
  int prec;
  GroupArena arena;
  ActiveSet<float2> s64;
  ActiveSet<double2> s128;
};
BatchRunner* runner_create(int prec) {
  BatchRunner* r = new BatchRunner();
  r->prec = prec;
  r->s64.arena = &r->arena;
  r->s128.arena = &r->arena;
  return r;
}
void runner_destroy_groups(BatchRunner* r) {
  r->s64.own.reset();
  r->s128.own.reset();
}
void runner_destroy(BatchRunner* r) {
  runner_destroy_groups(r);  // groups before the arena they live in
  delete r;
}
int runner_add(BatchRunner* r, Handle* h, const double2* b_dense, double tol, cudaStream_t st) {
  TRY(begin_problem(h, b_dense, nullptr, tol, st));
  if (r->prec == HELM_C128) r->s128.add(h);
  else r->s64.add(h);
  return HELM_OK;
}
int runner_iterate(BatchRunner* r, cudaStream_t st) {
  return r->prec == HELM_C128 ? r->s128.iterate(st) : r->s64.iterate(st);
}
int runner_collect(BatchRunner* r, cudaStream_t st, std::vector<std::pair<Handle*, OuterState>>* done) {
  return r->prec == HELM_C128 ? r->s128.collect(st, done) : r->s64.collect(st, done);
}
int runner_size(const BatchRunner* r) {
  return (int)(r->prec == HELM_C128 ? r->s128.members.size() : r->s64.members.size());
}
int runner_finish(Handle* h, const OuterState& s, double2* x_dense, cudaStream_t st, helm_info* info) {
  return finish_problem(h, s, x_dense, st, info);
}

int solve_group(Handle* const* hs, int count, const double* const* b, double* const* x, double tol,
                helm_info* infos, cudaStream_t st) {
  if (!hs || count <= 0 || !b || !x) { set_error("invalid batch arguments"); return HELM_EINVAL; }
  if (!(tol > 0.0) || !std::isfinite(tol)) { set_error("tol must be positive"); return HELM_EINVAL; }
  for (int p = 0; p < count; ++p)
    if (!hs[p] || !b[p] || !x[p]) { set_error("NULL handle or vector in batch"); return HELM_EINVAL; }
  const int prec = hs[0]->prec;
  return prec == HELM_C128 ? solve_t<double2>(hs, count, b, x, tol, infos, st)
                           : solve_t<float2>(hs, count, b, x, tol, infos, st);
}

static void destroy_group_cache(Handle* h);

// Point an existing handle at a new constant wavenumber and CSG angle (same grid,
// precision and options): the hierarchy buffers are reused, coefficients, phi and the
// coarsest LU are recomputed.
int retarget_handle(Handle* h, double k, double theta_beta, cudaStream_t st) {
  if (!(theta_beta >= 0 && theta_beta < M_PI / 2) || !std::isfinite(k)) {
    set_error("theta_beta must be in [0, pi/2) and k finite");
    return HELM_EINVAL;
  }
  if (h->has_phi) { set_error("a handle built with a phi field cannot be retargeted"); return HELM_EINVAL; }
  if (h->smoother == HELM_SMOOTHER_POLY) {
    const double k0 = h->k, tb0 = h->theta_beta;
    h->k = k;
    h->theta_beta = theta_beta;
    std::vector<int> sizes;
    for (const auto& L : h->lev) sizes.push_back(L.n);
    const int rc = compute_poly_weights(h, sizes);
    if (rc != HELM_OK) {
      h->k = k0;
      h->theta_beta = tb0;
      return rc;
    }
  }
  h->k = k;
  h->theta_beta = theta_beta;
  for (int l = 0; l < (int)h->lev.size(); ++l) {
    h->lev[l].phic = k * k;
    TRY(upload_level_coefficients(h, l, theta_beta, st));
  }
  TRY(factor_coarsest(h, theta_beta, st));
  destroy_group_cache(h);  // its descriptors carry the old phi
  return HELM_OK;
}

// Device bytes helm_setup allocates for these parameters (admission control).
size_t estimate_handle_bytes(int dim, int n, int prec, int s, int restart, int maxit, int coarsest) {
  const std::vector<int> sizes = level_sizes(n, coarsest > 0 ? coarsest : 3);
  const size_t eb = prec == HELM_C128 ? sizeof(double2) : sizeof(float2);
  size_t bytes = 0;
  for (int nl : sizes) {
    const size_t P = nl + 1, np = dim == 3 ? P * P * P : P * P;
    bytes += (4 + (size_t)s) * np * eb + 3 * nl * (eb + sizeof(double2)) + 4096;
  }
  const size_t P0 = n + 1, vs = dim == 3 ? P0 * P0 * P0 : P0 * P0;
  const size_t m = restart > 0 ? std::min(restart, maxit) : maxit;
  bytes += 3 * vs * sizeof(double2) + (m + 1) * vs * sizeof(double2) + m * vs * eb + (m + 1) * (m + 8) * 16;
  bytes += outer_part_doubles(outer_chunks(vs), (int)m) * sizeof(double);
  bytes += (size_t)outer_dot_counters(outer_chunks(vs)) * sizeof(unsigned);
  return bytes;
}

static void destroy_group_cache(Handle* h) {
  if (!h->group_cache) return;
  if (h->prec == HELM_C128) delete (Group<double2>*)h->group_cache;
  else delete (Group<float2>*)h->group_cache;
  h->group_cache = nullptr;
}

Handle::~Handle() {
  destroy_group_cache(this);
  for (void* p : allocs) cudaFree(p);
  if (stage) cudaFreeHost(stage);
}

}  // namespace helm
