// V-cycle kernels of the GMRES(s)-smoothed multigrid for M^CSG (Sec. 3.1).
//
// The grid-wide passes are shared-memory tile kernels (tiles.cuh).
// A kernel of Arnoldi step J never stores v_J: it forms v_J on the fly from the raw
// vectors R_0..R_{J-1} with the sweep's FP64 coefficients (v_J = sum Cf[J][k] R_k),
// applies M, stores p_J = M v_J and reduces <R_k, p_J> and ||p_J||^2 per problem in a
// fixed order.  The last CTA of each problem turns the sums into the next Arnoldi
// coefficients or the least-squares solution (device_common.cuh).
#pragma once
#include "device_common.cuh"

namespace helm {

// ------------------------------------------------------------------ indexing
__device__ __forceinline__ bool inside(int x, int y, int z, int n) {
  return (unsigned)x < (unsigned)n && (unsigned)y < (unsigned)n && (unsigned)z < (unsigned)n;
}
__device__ __forceinline__ size_t pidx(int x, int y, int z, int P) {
  return ((size_t)z * P + y) * (size_t)P + x;
}
// Bounds-checked load; NC = true uses the read-only path and is only for buffers no
// thread writes during the kernel.
template <typename C, bool NC = true>
__device__ __forceinline__ C ldc(const C* p, int x, int y, int z, int n, int P) {
  if (!inside(x, y, z, n)) return czero<C>();
  return NC ? __ldg(p + pidx(x, y, z, P)) : p[pidx(x, y, z, P)];
}

// 1D coefficients of the axis at index i (zero outside)
template <typename C>
struct Coef3 { C a, d, c; };
template <typename C>
__device__ __forceinline__ Coef3<C> ldcoef(const LevelDev<C>& L, int i) {
  Coef3<C> r;
  if ((unsigned)i < (unsigned)L.n) { r.a = __ldg(L.ca + i); r.d = __ldg(L.cd + i); r.c = __ldg(L.cc + i); }
  else { r.a = r.d = r.c = czero<C>(); }
  return r;
}

template <typename C>
__device__ __forceinline__ typename CT<C>::R phi_at(const LevelDev<C>& L, int x, int y, int z) {
  typedef typename CT<C>::R R;
  return L.phi ? (R)__ldg(L.phi + pidx(x, y, z, L.P)) : L.phir;
}

// What a tile loop's stencil reads of its level, copied once into registers: the 1D
// coefficients (one array of 3n: a, then d, then c), the phi field or its constant,
// and the sizes.  (Read through the descriptor, these fields are fetched again for
// every point.)
template <typename C>
struct StencilRegs {
  typedef typename CT<C>::R R;
  const C* coef3;
  const float* phi;
  R phic;
  int n, P;
  __device__ __forceinline__ explicit StencilRegs(const LevelDev<C>& L)
      : coef3(L.ca), phi(L.phi), phic(L.phir), n(L.n), P(L.P) {}
  __device__ __forceinline__ Coef3<C> coef(int i) const {
    Coef3<C> r;
    if ((unsigned)i < (unsigned)n) {
      r.a = __ldg(coef3 + i);
      r.d = __ldg(coef3 + n + i);
      r.c = __ldg(coef3 + 2 * n + i);
    } else {
      r.a = r.d = r.c = czero<C>();
    }
    return r;
  }
  __device__ __forceinline__ R phi_at(int x, int y, int z) const {
    return phi ? (R)__ldg(phi + pidx(x, y, z, P)) : phic;
  }
};

// ------------------------------------------------------------------ prolongation
// Vertex-centred bi/trilinear interpolation of the coarser output at fine node i:
// odd i -> coarse (i-1)/2 with weight 1; even i -> coarse i/2-1 and i/2 with 1/2.
template <typename C, bool NC = true>
__device__ __forceinline__ C interp(const C* xcb, int n, int nc, int Pc, int x, int y, int z, int dim) {
  typedef typename CT<C>::R R;
  C acc = czero<C>();
  if (!inside(x, y, z, n)) return acc;
  int ix[2], iy[2], iz[2];
  R wx, wy, wz;
  int nx, ny, nz;
  if (x & 1) { ix[0] = x >> 1; nx = 1; wx = 1; } else { ix[0] = (x >> 1) - 1; ix[1] = x >> 1; nx = 2; wx = 0.5; }
  if (y & 1) { iy[0] = y >> 1; ny = 1; wy = 1; } else { iy[0] = (y >> 1) - 1; iy[1] = y >> 1; ny = 2; wy = 0.5; }
  if (dim == 3) {
    if (z & 1) { iz[0] = z >> 1; nz = 1; wz = 1; } else { iz[0] = (z >> 1) - 1; iz[1] = z >> 1; nz = 2; wz = 0.5; }
  } else { iz[0] = 0; nz = 1; wz = 1; }
  const R w = wx * wy * wz;
  for (int c = 0; c < nz; ++c)
    for (int b = 0; b < ny; ++b)
      for (int a = 0; a < nx; ++a) acc = cadd(acc, ldc<C, NC>(xcb, ix[a], iy[b], iz[c], nc, Pc));
  return cscale(acc, w);
}
template <typename C, bool NC = true>
__device__ __forceinline__ C interp(const LevelDev<C>& L, int x, int y, int z, int dim) {
  return interp<C, NC>(L.xcb, L.n, L.nc, L.Pc, x, y, z, dim);
}

// ------------------------------------------------------------------ sweep end
// Coefficients of the sweep's update, staged in registers.
template <typename C>
struct UpdCoef {
  int m;
  C xc[SMAX + 1], rc[SMAX + 1];
  const C* Rk[SMAX + 1];
};
template <typename C>
__device__ __forceinline__ UpdCoef<C> load_upd(const LevelDev<C>& L, int r0_is_b) {
  UpdCoef<C> u;
  const auto* sc = L.sc;
  u.m = sc->m;
#pragma unroll
  for (int k = 0; k <= SMAX; ++k) {
    u.xc[k] = sc->xcoef[k];
    u.rc[k] = sc->rcoef[k];
    u.Rk[k] = (k == 0) ? (r0_is_b ? L.b : L.r0) : L.p[k - 1];
  }
  return u;
}
// x-increment and residual at a point: dx = sum_{k<m} xc[k] R_k and, if want_r,
// r = sum_{k<=m} rc[k] R_k.
template <typename C, bool NC = true>
__device__ __forceinline__ void upd_point(const UpdCoef<C>& u, int x, int y, int z, int n, int P,
                                          C& dx, C& r, bool want_r = true) {
  dx = czero<C>();
  r = czero<C>();
#pragma unroll
  for (int k = 0; k <= SMAX; ++k) {
    if (k < u.m || (want_r && k == u.m)) {
      C v = ldc<C, NC>(u.Rk[k], x, y, z, n, P);
      if (k < u.m) dx = cfma(u.xc[k], v, dx);
      r = cfma(u.rc[k], v, r);
    }
  }
}

// Pointwise end of a sweep: x += dx (in place on xa or xb, or from zero) and, in
// residual mode, r0 <- r (in place) with ||r||^2 starting the next sweep.  Every
// vector is zero at the padding positions, so this is a plain stream over the padded
// index (UF_U points per thread and round; 2 when a point reads four or more raw
// vectors).  The body is instantiated per number of raw vectors M (uniform: the
// sweep's length), so every load of a round is issued before the first is used.
constexpr int UF_U = 4;
template <typename C, int M, bool WANT_R>
__device__ __forceinline__ void update_flat_body(const UpdCoef<C>& u, C* xo, C* r0out, size_t npts, size_t i_beg,
                                                 size_t stride, bool x_from_zero, typename CT<C>::R& acc) {
  constexpr int NV = WANT_R ? M + 1 : M;  // raw vectors read per point
  constexpr int UF = NV >= 4 ? 2 : UF_U;  // points per thread and round (registers)
  for (size_t i0 = i_beg; i0 < npts; i0 += UF * stride) {
    C v[UF][NV > 0 ? NV : 1], xv[UF];
#pragma unroll
    for (int q = 0; q < UF; ++q) {
      const size_t i = i0 + q * stride;
      xv[q] = czero<C>();
      if (i < npts) {
#pragma unroll
        for (int k = 0; k < NV; ++k) v[q][k] = u.Rk[k][i];
        if (!x_from_zero) xv[q] = xo[i];
      }
    }
#pragma unroll
    for (int q = 0; q < UF; ++q) {
      const size_t i = i0 + q * stride;
      if (i >= npts) continue;
      C dx = czero<C>();
#pragma unroll
      for (int k = 0; k < M; ++k) dx = cfma(u.xc[k], v[q][k], dx);
      xo[i] = cadd(xv[q], dx);
      if (WANT_R) {
        C r = czero<C>();
#pragma unroll
        for (int k = 0; k <= M; ++k) r = cfma(u.rc[k], v[q][k < NV ? k : 0], r);
        r0out[i] = r;
        acc += cabs2(r);
      }
    }
  }
}

template <typename C>
__device__ __forceinline__ void update_pass_body(const LevelDev<C>* __restrict__ levs, int ntiles, int dim, int mode, int r0_is_b, int xsel,
              int x_from_zero, int vblk) {
  __shared__ typename CT<C>::R sm[32];
  const int prob = vblk / ntiles, tile = vblk - prob * ntiles;
  const LevelDev<C>& L = levs[prob];
  const int P = L.P;
  pdl_wait();
  const UpdCoef<C> u = load_upd(L, r0_is_b);
  C* xo = xsel ? L.xb : L.xa;
  C* r0out = L.r0;
  const size_t npts = dim == 3 ? (size_t)P * P * P : (size_t)P * P;
  const bool want_r = (mode == UPD_RESIDUAL);
  const size_t stride = (size_t)ntiles * block_threads();
  const size_t i_beg = (size_t)tile * block_threads() + flat_tid();
  const bool xz = x_from_zero != 0;
  typename CT<C>::R acc = 0;
  switch (u.m) {  // uniform over the grid
#define HELM_UF_CASE(MM)                                                                    \
    case MM:                                                                                \
      if (want_r) update_flat_body<C, MM, true>(u, xo, r0out, npts, i_beg, stride, xz, acc); \
      else update_flat_body<C, MM, false>(u, xo, r0out, npts, i_beg, stride, xz, acc);       \
      break;
    HELM_UF_CASE(0)
    HELM_UF_CASE(1)
    HELM_UF_CASE(2)
    HELM_UF_CASE(3)
    HELM_UF_CASE(4)
#undef HELM_UF_CASE
    default: break;
  }
  static_assert(SMAX == 4, "update_flat_body is instantiated for m = 0..4");
  if (!want_r) return;
  typename CT<C>::R red[1] = {acc}, tot[1];
  pdl_trigger();  // the main work is done: let the next pass launch
  if (grid_sum_last<1>(red, L.part, tile, ntiles, &L.sc->counter, sm, tot)) {
    if (flat_tid() == 0) sweep_begin(L.sc, tot[0], L.s);
  }
}
template <typename C>
__global__ void __launch_bounds__(256, sizeof(C) == 16 ? 2 : 4)
k_update_flat(const LevelDev<C>* __restrict__ levs, int ntiles, int dim, int mode, int r0_is_b, int xsel,
              int x_from_zero) {
  update_pass_body<C>(levs, ntiles, dim, mode, r0_is_b, xsel, x_from_zero, blockIdx.x);
}

// Level-0 input: b <- src (natural layout, any precision), ||b||^2 starts the first
// sweep.
template <typename Cin, typename C>
__global__ void __launch_bounds__(256)
k_load_input(const LevelDev<C>* __restrict__ levs, int ntiles, int dim, const Cin* __restrict__ src) {
  __shared__ typename CT<C>::R sm[32];
  const int prob = blockIdx.x / ntiles, tile = blockIdx.x - prob * ntiles;
  const LevelDev<C>& L = levs[prob];
  const int n = L.n, P = L.P;
  pdl_wait();
  // CTAs take rows (z, y) of the padded layout in turn; threads stride along x
  const int nrows = dim == 3 ? P * P : P;
  C* const b = L.b;
  typename CT<C>::R acc = 0;
  for (int row = tile; row < nrows; row += ntiles) {
    const int y = dim == 3 ? row % P : row, z = dim == 3 ? row / P : 0;
    const bool rin = y < n && z < n;
    const size_t base = (size_t)row * P, sbase = ((size_t)z * n + y) * n;
    for (int x = threadIdx.x; x < P; x += blockDim.x) {
      C v = czero<C>();
      if (rin && x < n) v = to_c<C>(src[sbase + x]);
      b[base + x] = v;
      acc += cabs2(v);
    }
  }
  typename CT<C>::R red[1] = {acc}, tot[1];
  pdl_trigger();  // the main work is done: let the next pass launch
  if (grid_sum_last<1>(red, L.part, tile, ntiles, &L.sc->counter, sm, tot)) {
    if (flat_tid() == 0) sweep_begin(L.sc, tot[0], L.s);
  }
}

// Level-0 output: dst (natural layout, any precision) <- xb.
template <typename C, typename Cout>
__global__ void __launch_bounds__(256)
k_store_output(const LevelDev<C>* __restrict__ levs, int dim, Cout* __restrict__ dst) {
  pdl_trigger();
  const LevelDev<C>& L = levs[0];
  const int n = L.n, P = L.P;
  pdl_wait();
  // CTAs take rows (z, y) of the natural layout in turn; threads stride along x
  const int nrows = dim == 3 ? n * n : n;
  const C* const xb = L.xb;
  for (int row = blockIdx.x; row < nrows; row += gridDim.x) {
    const int y = dim == 3 ? row % n : row, z = dim == 3 ? row / n : 0;
    const size_t dbase = (size_t)row * n, sbase = ((size_t)z * P + y) * P;
    for (int x = threadIdx.x; x < n; x += blockDim.x) dst[dbase + x] = to_c<Cout>(xb[sbase + x]);
  }
}

// ------------------------------------------------------------------ coarse correction
// Coarse correction without post-smoothing (nu2 = 0): x_b = x_a + P e_c, pointwise.
template <typename C, bool NC = true>
__device__ __forceinline__ void prolong_flat_body(const LevelDev<C>* __restrict__ levs, int ntiles, int dim, int vblk) {
  pdl_trigger();
  const int prob = vblk / ntiles, tile = vblk - prob * ntiles;
  const LevelDev<C>& L = levs[prob];
  const int n = L.n, P = L.P;
  pdl_wait();
  const size_t npts = dim == 3 ? (size_t)P * P * P : (size_t)P * P;
  for (size_t i = (size_t)tile * block_threads() + flat_tid(); i < npts; i += (size_t)ntiles * block_threads()) {
    const int x = (int)(i % P), y = (int)((i / P) % P), z = dim == 3 ? (int)(i / ((size_t)P * P)) : 0;
    C v = czero<C>();
    if (inside(x, y, z, n)) v = cadd(L.xa[i], interp<C, NC>(L, x, y, z, dim));
    L.xb[i] = v;
  }
}
template <typename C>
__global__ void __launch_bounds__(256)
k_prolong_flat(const LevelDev<C>* __restrict__ levs, int ntiles, int dim) {
  prolong_flat_body<C>(levs, ntiles, dim, blockIdx.x);
}

// ------------------------------------------------------------------ coarse levels
// The sub-cycle of the coarse levels (sizes where a grid-wide launch is all latency)
// runs on a "team" per problem: one CTA, or a thread-block cluster whose CTAs act as
// one block.  Every pass is a team-wide loop over the level's points; sync() orders
// all of the team's global-memory accesses; sum() totals per-thread values in a fixed
// order and leaves the totals with thread 0 of every CTA, which then runs the small
// sweep algebra on its CTA's own copy of the sweep scalars (bitwise the same in every
// CTA, so no further exchange is needed).  The coarsest level is a dense FP64 LU solve
// by one warp.
struct CtaTeam {
  __device__ __forceinline__ int rank() const { return 0; }
  __device__ __forceinline__ unsigned gtid() const { return (unsigned)flat_tid(); }
  __device__ __forceinline__ unsigned gnth() const { return (unsigned)block_threads(); }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
  template <int NV, typename T>
  __device__ __forceinline__ void sum(T (&v)[NV], T* sm) { block_sum<NV, T>(v, sm); }
};

constexpr int CLUSTER_MAX = 16;
constexpr int TEAM_NV = 2 * SMAX + 1;  // most values one team sum carries
constexpr int CB_U = 4;                // points per thread per step of the team loops

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_size() {
  unsigned n;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(n));
  return n;
}
// Every thread of every CTA of the cluster; release/acquire at cluster scope.
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Load a word of CTA `rank`'s shared memory at the address of `p` in this CTA's.
__device__ __forceinline__ float ld_dsmem(const float* p, unsigned rank) {
  unsigned a = (unsigned)__cvta_generic_to_shared(p), ra;
  float v;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(ra) : "memory");
  return v;
}
__device__ __forceinline__ double ld_dsmem(const double* p, unsigned rank) {
  unsigned a = (unsigned)__cvta_generic_to_shared(p), ra;
  double v;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(ra) : "memory");
  return v;
}

// `slots` is this CTA's [2][CLUSTER_MAX][TEAM_NV] doubles of shared memory.  The two
// halves alternate between sums: a CTA can only rewrite a half after every CTA has
// passed the barrier that follows the reads of the previous sum in it.
struct ClusterTeam {
  unsigned r, n;
  double* slots;
  int buf;
  __device__ __forceinline__ explicit ClusterTeam(double* s) : r(cluster_rank()), n(cluster_size()), slots(s), buf(0) {}
  __device__ __forceinline__ int rank() const { return (int)r; }
  __device__ __forceinline__ unsigned gtid() const { return r * (unsigned)block_threads() + (unsigned)flat_tid(); }
  __device__ __forceinline__ unsigned gnth() const { return n * (unsigned)block_threads(); }
  __device__ __forceinline__ void sync() const { cluster_sync(); }
  template <int NV, typename T>
  __device__ __forceinline__ void sum(T (&v)[NV], T* sm) {
    block_sum<NV, T>(v, sm);
    T* half = reinterpret_cast<T*>(slots + (size_t)buf * CLUSTER_MAX * TEAM_NV);
    if (flat_tid() == 0)
#pragma unroll
      for (int i = 0; i < NV; ++i) half[r * NV + i] = v[i];
    cluster_sync();
    if (flat_tid() < 32) {  // lane q reads rank q's sums, a fixed butterfly adds them
      const unsigned q = (unsigned)flat_tid();
#pragma unroll
      for (int i = 0; i < NV; ++i) v[i] = q < n ? ld_dsmem(half + q * NV + i, q) : (T)0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int i = 0; i < NV; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    }
    buf ^= 1;
  }
};

template <typename C>
__device__ void cblock_stencil_apply(const LevelDev<C>& L, const C* v, int x, int y, int z, int dim, C& out) {
  const int n = L.n, P = L.P;
  const Coef3<C> cx = ldcoef(L, x), cy = ldcoef(L, y);
  C v0 = v[pidx(x, y, z, P)];
  C diag = cadd(cx.d, cy.d);
  C p = czero<C>();
  p = cfma(cx.a, ldc<C, false>(v, x - 1, y, z, n, P), p);
  p = cfma(cx.c, ldc<C, false>(v, x + 1, y, z, n, P), p);
  p = cfma(cy.a, ldc<C, false>(v, x, y - 1, z, n, P), p);
  p = cfma(cy.c, ldc<C, false>(v, x, y + 1, z, n, P), p);
  if (dim == 3) {
    const Coef3<C> cz = ldcoef(L, z);
    diag = cadd(diag, cz.d);
    p = cfma(cz.a, ldc<C, false>(v, x, y, z - 1, n, P), p);
    p = cfma(cz.c, ldc<C, false>(v, x, y, z + 1, n, P), p);
  }
  diag.x -= phi_at(L, x, y, z);
  out = cfma(diag, v0, p);
}

// Coordinates of padded index i (coarse levels have fewer than 2^32 points).
__device__ __forceinline__ void cblock_coords(unsigned i, unsigned P, int dim, int& x, int& y, int& z) {
  const unsigned q = i / P;
  x = (int)(i - q * P);
  if (dim == 3) {
    const unsigned zz = q / P;
    y = (int)(q - zz * P);
    z = (int)zz;
  } else {
    y = (int)q;
    z = 0;
  }
}
__device__ __forceinline__ unsigned cblock_npts(int P, int dim) {
  return dim == 3 ? (unsigned)P * P * P : (unsigned)P * P;
}

// One GMRES(s) sweep on level L by the team.  R_0 is b (r0_is_b) or r0; x is updated
// in place in xo (or written from zero).  `tmp` holds v_J.  At the end, in residual
// mode r0 <- r_new and the next sweep starts; in restrict mode the residual is left in
// `tmp` for the caller.
template <typename C, typename Team>
__device__ void cblock_sweep(Team& team, const LevelDev<C>& L, int dim, int r0_is_b, C* xo, int x_from_zero, C* tmp,
                             int end_mode, typename CT<C>::R* sm) {
  typedef typename CT<C>::R R;
  auto* sc = L.sc;
  const int P = L.P, n = L.n;
  const unsigned npts = cblock_npts(P, dim);
  const unsigned gt = team.gtid(), gn = team.gnth();
  const C* R0 = r0_is_b ? L.b : L.r0;
  for (int J = 1; J <= SMAX; ++J) {
    __syncthreads();  // this CTA's sweep scalars are final
    if (sc->m < J) break;  // the same in every CTA of the team
    // v_J = sum_k Cf[J][k] R_k (each point by the thread that owns it in every pass;
    // CB_U points at a time, all loads before the stores)
    C cf[SMAX];
    for (int k = 0; k < J; ++k) cf[k] = sc->Cf[J][k];
    for (unsigned i0 = gt; i0 < npts; i0 += CB_U * gn) {
      C v[CB_U];
#pragma unroll
      for (int u = 0; u < CB_U; ++u) {
        const unsigned i = i0 + u * gn;
        v[u] = czero<C>();
        if (i < npts)
          for (int k = 0; k < J; ++k) v[u] = cfma(cf[k], (k == 0 ? R0 : L.p[k - 1])[i], v[u]);
      }
#pragma unroll
      for (int u = 0; u < CB_U; ++u)
        if (i0 + u * gn < npts) tmp[i0 + u * gn] = v[u];
    }
    team.sync();
    R red[2 * SMAX + 1];
    for (int q = 0; q < 2 * SMAX + 1; ++q) red[q] = (R)0;
    C acc[SMAX];
    for (int k = 0; k < SMAX; ++k) acc[k] = czero<C>();
    R accn = 0;
    for (unsigned i0 = gt; i0 < npts; i0 += CB_U * gn) {
      C p[CB_U];
#pragma unroll
      for (int u = 0; u < CB_U; ++u) {
        const unsigned i = i0 + u * gn;
        p[u] = czero<C>();
        if (i < npts) {
          int x, y, z;
          cblock_coords(i, (unsigned)P, dim, x, y, z);
          if (inside(x, y, z, n)) {
            cblock_stencil_apply(L, tmp, x, y, z, dim, p[u]);
            for (int k = 0; k < J; ++k) acc[k] = cdotacc((k == 0 ? R0 : L.p[k - 1])[i], p[u], acc[k]);
            accn += cabs2(p[u]);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < CB_U; ++u)
        if (i0 + u * gn < npts) L.p[J - 1][i0 + u * gn] = p[u];
    }
    for (int k = 0; k < J; ++k) { red[2 * k] = acc[k].x; red[2 * k + 1] = acc[k].y; }
    red[2 * J] = accn;
    team.sum(red, sm);  // also separates this pass's reads of tmp from the next pass's writes
    if (flat_tid() == 0) sweep_after_pass_rt<R>(sc, J, red);
  }
  __syncthreads();
  const int m = sc->m;
  C xc[SMAX + 1], rc[SMAX + 1];
  for (int k = 0; k <= SMAX; ++k) { xc[k] = sc->xcoef[k]; rc[k] = sc->rcoef[k]; }
  R accr = 0;
  for (unsigned i0 = gt; i0 < npts; i0 += CB_U * gn) {
    C xn[CB_U], r[CB_U];
#pragma unroll
    for (int u = 0; u < CB_U; ++u) {
      const unsigned i = i0 + u * gn;
      C dx = czero<C>();
      r[u] = czero<C>();
      xn[u] = czero<C>();
      if (i < npts) {
        for (int k = 0; k <= m; ++k) {
          C v = (k == 0 ? R0 : L.p[k - 1])[i];
          if (k < m) dx = cfma(xc[k], v, dx);
          r[u] = cfma(rc[k], v, r[u]);
        }
        xn[u] = cadd(x_from_zero ? czero<C>() : xo[i], dx);
      }
    }
#pragma unroll
    for (int u = 0; u < CB_U; ++u) {
      const unsigned i = i0 + u * gn;
      if (i >= npts) continue;
      xo[i] = xn[u];
      if (end_mode == UPD_RESIDUAL) { L.r0[i] = r[u]; accr += cabs2(r[u]); }
      if (end_mode == UPD_RESTRICT) tmp[i] = r[u];
    }
  }
  if (end_mode == UPD_RESIDUAL) {
    R red[1] = {accr};
    team.sum(red, sm);
    if (flat_tid() == 0) sweep_begin(sc, red[0], L.s);
  }
  team.sync();
}

// The whole sub-cycle of levels Ls[0..nlev-1] (Ls[nlev-1] the coarsest, solved by
// LU) on one team; the level vectors may live in global or shared memory (plain
// loads only), the sweep scalars are the CTA's own.  `sm` needs 32 * (2 SMAX + 1)
// doubles.
// The coarsest LU factors are staged in shared memory (lu_sm, lu_cap complex values)
// when they fit: the triangular solves read one factor per step of a serial chain,
// and from global memory every step waited for an L2 round trip.
constexpr int LU_STAGE = 1024;  // up to 32 coarsest unknowns (3^3 in 3D, 3^2 .. 5^2 in 2D)
template <typename C, typename Team>
__device__ void coarse_cycle(Team& team, const LevelDev<C>* Ls, int nlev, const CoarseLU& lu, int nu1, int nu2,
                             int dim, double* smd, double2* lu_sm = nullptr, int lu_cap = 0) {
  typedef typename CT<C>::R R;
  R* sm = reinterpret_cast<R*>(smd);
  const unsigned gt = team.gtid(), gn = team.gnth();
  const int tid = flat_tid(), nth = block_threads();
  const bool staged = lu_sm && lu.m * lu.m <= lu_cap;
  if (staged) {
    for (int i = tid; i < lu.m * lu.m; i += nth) lu_sm[i] = lu.lu[i];
    __syncthreads();
  }
  const double2* const LUf = staged ? lu_sm : lu.lu;
  // descent
  for (int l = 0; l < nlev - 1; ++l) {
    const LevelDev<C>& L = Ls[l];
    const int P = L.P;
    const unsigned npts = cblock_npts(P, dim);
    if (nu1 == 0) {
      for (unsigned i = gt; i < npts; i += gn) { L.xa[i] = czero<C>(); L.xb[i] = L.b[i]; }
    } else {
      for (int sw = 0; sw < nu1; ++sw)
        cblock_sweep(team, L, dim, sw == 0, L.xa, sw == 0, L.xb, sw == nu1 - 1 ? UPD_RESTRICT : UPD_RESIDUAL, sm);
    }
    team.sync();
    // b_c = FW(r) with r in xb
    const int Pc = L.Pc, nc = L.nc;
    const unsigned ncpts = cblock_npts(Pc, dim);
    R acc = 0;
    for (unsigned i0 = gt; i0 < ncpts; i0 += CB_U * gn) {
      C out[CB_U];
#pragma unroll
      for (int u = 0; u < CB_U; ++u) {
        const unsigned i = i0 + u * gn;
        out[u] = czero<C>();
        if (i >= ncpts) continue;
        int X, Y, Z;
        cblock_coords(i, (unsigned)Pc, dim, X, Y, Z);
        if (inside(X, Y, Z, nc)) {
          const int fx = 2 * X + 1, fy = 2 * Y + 1, fz = dim == 3 ? 2 * Z + 1 : 0;
          const int dz0 = dim == 3 ? -1 : 0, dz1 = dim == 3 ? 1 : 0;
          for (int dz = dz0; dz <= dz1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
              for (int dx = -1; dx <= 1; ++dx) {
                R wgt = (R)((dx == 0 ? 0.5 : 0.25) * (dy == 0 ? 0.5 : 0.25) * (dim == 3 ? (dz == 0 ? 0.5 : 0.25) : 1.0));
                out[u] = cadd(out[u], cscale(ldc<C, false>((const C*)L.xb, fx + dx, fy + dy, fz + dz, L.n, P), wgt));
              }
          acc += cabs2(out[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < CB_U; ++u)
        if (i0 + u * gn < ncpts) L.bc[i0 + u * gn] = out[u];
    }
    R red[1] = {acc};
    team.sum(red, sm);
    if (tid == 0) sweep_begin(L.scc, red[0], L.s);
    team.sync();
  }
  // coarsest: dense LU solve in FP64 by warp 0 of the first CTA, which also writes x
  {
    const LevelDev<C>& L = Ls[nlev - 1];
    const int m = lu.m, P = L.P, n = L.n;
    double2* yv = reinterpret_cast<double2*>(smd);  // m <= 144 complex values
    if (team.rank() == 0) {
      if (tid < 32) {
        for (int i = tid; i < m; i += 32) {
          const int src = lu.piv[i];
          int sx = src % n, sy = (src / n) % n, sz = dim == 3 ? src / (n * n) : 0;
          yv[i] = to_d(L.b[pidx(sx, sy, sz, P)]);
        }
        // reciprocals of U's diagonal, all at once (a complex FP64 division is a long
        // dependent chain on this part's 1/64-rate FP64 pipe; the backward sweep then
        // multiplies instead of dividing m times in series)
        double2* const inv = staged && m * m + m <= lu_cap ? lu_sm + (size_t)m * m : nullptr;
        if (inv)
          for (int i = tid; i < m; i += 32) inv[i] = ddiv(make_double2(1.0, 0.0), LUf[(size_t)i * m + i]);
        __syncwarp();
        for (int k = 0; k < m; ++k) {  // forward, unit lower
          const double2 yk = yv[k];
          __syncwarp();
          for (int i = k + 1 + tid; i < m; i += 32) yv[i] = csub(yv[i], cmul(LUf[(size_t)i * m + k], yk));
          __syncwarp();
        }
        for (int k = m - 1; k >= 0; --k) {  // backward
          if (tid == 0) yv[k] = inv ? cmul(yv[k], inv[k]) : ddiv(yv[k], LUf[(size_t)k * m + k]);
          __syncwarp();
          const double2 yk = yv[k];
          for (int i = tid; i < k; i += 32) yv[i] = csub(yv[i], cmul(LUf[(size_t)i * m + k], yk));
          __syncwarp();
        }
      }
      __syncthreads();
      const unsigned npts = cblock_npts(P, dim);
      for (unsigned i = tid; i < npts; i += nth) {
        int x, y, z;
        cblock_coords(i, (unsigned)P, dim, x, y, z);
        C v = czero<C>();
        if (inside(x, y, z, n)) v = from_d<C>(yv[(z * n + y) * n + x]);
        L.xb[i] = v;
      }
    }
    team.sync();
  }
  // ascent
  for (int l = nlev - 2; l >= 0; --l) {
    const LevelDev<C>& L = Ls[l];
    const int P = L.P, n = L.n;
    const unsigned npts = cblock_npts(P, dim);
    for (unsigned i0 = gt; i0 < npts; i0 += CB_U * gn) {
      C xv[CB_U];
#pragma unroll
      for (int u = 0; u < CB_U; ++u) {
        const unsigned i = i0 + u * gn;
        xv[u] = czero<C>();
        if (i >= npts) continue;
        int x, y, z;
        cblock_coords(i, (unsigned)P, dim, x, y, z);
        if (inside(x, y, z, n)) xv[u] = cadd(L.xa[i], interp<C, false>(L, x, y, z, dim));
      }
#pragma unroll
      for (int u = 0; u < CB_U; ++u)
        if (i0 + u * gn < npts) L.xb[i0 + u * gn] = xv[u];
    }
    team.sync();
    if (nu2 > 0) {
      R acc = 0;
      for (unsigned i0 = gt; i0 < npts; i0 += CB_U * gn) {
        C r[CB_U];
#pragma unroll
        for (int u = 0; u < CB_U; ++u) {
          const unsigned i = i0 + u * gn;
          r[u] = czero<C>();
          if (i >= npts) continue;
          int x, y, z;
          cblock_coords(i, (unsigned)P, dim, x, y, z);
          if (inside(x, y, z, n)) {
            C p;
            cblock_stencil_apply(L, (const C*)L.xb, x, y, z, dim, p);
            r[u] = csub(L.b[i], p);
            acc += cabs2(r[u]);
          }
        }
#pragma unroll
        for (int u = 0; u < CB_U; ++u)
          if (i0 + u * gn < npts) L.r0[i0 + u * gn] = r[u];
      }
      R red[1] = {acc};
      team.sum(red, sm);
      if (tid == 0) sweep_begin(L.sc, red[0], L.s);
      team.sync();
      for (int sw = 0; sw < nu2; ++sw)
        cblock_sweep(team, L, dim, 0, L.xb, 0, L.xa, sw == nu2 - 1 ? UPD_XONLY : UPD_RESIDUAL, sm);
    }
  }
}


// ------------------------------------------------------------------ polynomial smoother (Sec. 4)
template <typename C>
__device__ __forceinline__ C* poly_vec(const LevelDev<C>& L, int sel) {
  switch (sel) {
    case 1: return L.xa;
    case 2: return L.xb;
    case 3: return L.p[0];
    case 4: return L.p[1];
    default: return nullptr;
  }
}

// Padded coordinates of flat index i (64-bit: the largest levels exceed 2^32 points).
__device__ __forceinline__ void flat_coords(size_t i, int P, int dim, int& x, int& y, int& z) {
  const size_t q = i / (size_t)P;
  x = (int)(i - q * (size_t)P);
  if (dim == 3) {
    const size_t zz = q / (size_t)P;
    y = (int)(q - zz * (size_t)P);
    z = (int)zz;
  } else {
    y = (int)q;
    z = 0;
  }
}

// One Richardson step of the polynomial smoother: dst = src + w (b - M src), zero at
// the padding; src POLY_NONE is the zero vector (dst = w b); wsel < 0 writes zero.
template <typename C>
__global__ void __launch_bounds__(256)
k_poly_step(const LevelDev<C>* __restrict__ levs, const C* __restrict__ pw, int ntiles, int dim, int src, int dst,
            int wsel) {
  const int prob = blockIdx.x / ntiles, tile = blockIdx.x - prob * ntiles;
  const LevelDev<C>& L = levs[prob];
  pdl_wait();
  const int n = L.n, P = L.P;
  const C w = wsel >= 0 ? pw[3 * prob + wsel] : czero<C>();
  const C* xin = poly_vec(L, src);
  C* xout = poly_vec(L, dst);
  const C* b = L.b;
  const size_t npts = dim == 3 ? (size_t)P * P * P : (size_t)P * P;
  for (size_t i = (size_t)tile * blockDim.x + threadIdx.x; i < npts; i += (size_t)ntiles * blockDim.x) {
    int x, y, z;
    flat_coords(i, P, dim, x, y, z);
    C v = czero<C>();
    if (wsel >= 0 && inside(x, y, z, n)) {
      C mv = czero<C>(), xi = czero<C>();
      if (xin) {
        cblock_stencil_apply(L, xin, x, y, z, dim, mv);
        xi = xin[i];
      }
      v = cadd(xi, cmul(w, csub(b[i], mv)));
    }
    xout[i] = v;
  }
}

// r0 = b - M src on a level (src POLY_NONE: r0 = b), zero at the padding.
template <typename C>
__global__ void __launch_bounds__(256)
k_poly_residual(const LevelDev<C>* __restrict__ levs, int ntiles, int dim, int src) {
  const int prob = blockIdx.x / ntiles, tile = blockIdx.x - prob * ntiles;
  const LevelDev<C>& L = levs[prob];
  pdl_wait();
  const int n = L.n, P = L.P;
  const C* xin = poly_vec(L, src);
  const size_t npts = dim == 3 ? (size_t)P * P * P : (size_t)P * P;
  for (size_t i = (size_t)tile * blockDim.x + threadIdx.x; i < npts; i += (size_t)ntiles * blockDim.x) {
    int x, y, z;
    flat_coords(i, P, dim, x, y, z);
    C r = czero<C>();
    if (inside(x, y, z, n)) {
      C mv = czero<C>();
      if (xin) cblock_stencil_apply(L, xin, x, y, z, dim, mv);
      r = csub(L.b[i], mv);
    }
    L.r0[i] = r;
  }
}

// b_c = full weighting of r0 ((1/4, 1/2, 1/4) per axis around fine node 2I + 1), zero at
// the coarse padding.
template <typename C>
__global__ void __launch_bounds__(256)
k_poly_fw(const LevelDev<C>* __restrict__ levs, int ntiles, int dim) {
  typedef typename CT<C>::R R;
  const int prob = blockIdx.x / ntiles, tile = blockIdx.x - prob * ntiles;
  const LevelDev<C>& L = levs[prob];
  pdl_wait();
  const int n = L.n, P = L.P, nc = L.nc, Pc = L.Pc;
  const size_t ncpts = dim == 3 ? (size_t)Pc * Pc * Pc : (size_t)Pc * Pc;
  for (size_t i = (size_t)tile * blockDim.x + threadIdx.x; i < ncpts; i += (size_t)ntiles * blockDim.x) {
    int X, Y, Z;
    flat_coords(i, Pc, dim, X, Y, Z);
    C out = czero<C>();
    if (inside(X, Y, Z, nc)) {
      const int fx = 2 * X + 1, fy = 2 * Y + 1, fz = dim == 3 ? 2 * Z + 1 : 0;
      const int dz0 = dim == 3 ? -1 : 0, dz1 = dim == 3 ? 1 : 0;
      for (int dz = dz0; dz <= dz1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            const R wgt = (R)((dx == 0 ? 0.5 : 0.25) * (dy == 0 ? 0.5 : 0.25) * (dim == 3 ? (dz == 0 ? 0.5 : 0.25) : 1.0));
            out = cadd(out, cscale(ldc<C, false>((const C*)L.r0, fx + dx, fy + dy, fz + dz, n, P), wgt));
          }
    }
    L.bc[i] = out;
  }
}

// Coarse sub-cycle with the levels in global memory (any size).
template <typename C>
__global__ void __launch_bounds__(512)
k_coarse(const LevelDev<C>* __restrict__ levs_all, int nlev, int lev_stride, const CoarseLU* __restrict__ lus,
         int nu1, int nu2, int dim) {
  __shared__ double sm[32 * (2 * SMAX + 1)];
  __shared__ double2 lu_sm[LU_STAGE];
  pdl_trigger();
  pdl_wait();
  const int prob = blockIdx.x;
  CtaTeam team;
  coarse_cycle<C>(team, levs_all + (size_t)prob * lev_stride, nlev, lus[prob], nu1, nu2, dim, sm, lu_sm, LU_STAGE);
}

// Coarse sub-cycle with every level's vectors, descriptors and sweep scalars staged
// in shared memory; only the top coarse level's right-hand side (and its sweep state)
// comes from global memory and only its result goes back.
constexpr int MAX_COARSE_LEVELS = MAX_COARSE_LEVELS_HOST;
template <typename C>
__global__ void __launch_bounds__(512)
k_coarse_smem(const LevelDev<C>* __restrict__ levs_all, int nlev, int lev_stride, const CoarseLU* __restrict__ lus,
              int nu1, int nu2, int dim) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double sm[32 * (2 * SMAX + 1)];
  __shared__ LevelDev<C> Ls[MAX_COARSE_LEVELS];
  __shared__ SweepScalarsT<typename CT<C>::R> Ss[MAX_COARSE_LEVELS];
  __shared__ double2 lu_sm[LU_STAGE];
  pdl_trigger();
  const int prob = blockIdx.x;
  const LevelDev<C>* G = levs_all + (size_t)prob * lev_stride;
  const int tid = flat_tid(), nth = block_threads();
  pdl_wait();
  nlev = lus[prob].nlev;  // this problem's coarse levels (<= the stride)
  if (tid == 0) {
    C* cur = reinterpret_cast<C*>(smraw);
    for (int l = 0; l < nlev; ++l) {
      Ls[l] = G[l];
      const size_t np = dim == 3 ? (size_t)G[l].P * G[l].P * G[l].P : (size_t)G[l].P * G[l].P;
      Ls[l].b = cur; cur += np;
      Ls[l].xa = cur; cur += np;
      Ls[l].xb = cur; cur += np;
      Ls[l].r0 = cur; cur += np;
      for (int j = 0; j < G[l].s; ++j) { Ls[l].p[j] = cur; cur += np; }
      Ls[l].sc = &Ss[l];
    }
    for (int l = 0; l + 1 < nlev; ++l) {
      Ls[l].bc = Ls[l + 1].b;
      Ls[l].xcb = Ls[l + 1].xb;
      Ls[l].scc = &Ss[l + 1];
    }
  }
  __syncthreads();
  {
    const size_t np0 = dim == 3 ? (size_t)G[0].P * G[0].P * G[0].P : (size_t)G[0].P * G[0].P;
    for (size_t i = tid; i < np0; i += nth) Ls[0].b[i] = G[0].b[i];
    const int* src = reinterpret_cast<const int*>(G[0].sc);
    int* dst = reinterpret_cast<int*>(&Ss[0]);
    const int words = sweep_words<typename CT<C>::R>();
    for (int i = tid; i < words; i += nth) dst[i] = src[i];
  }
  __syncthreads();
  CtaTeam team;
  coarse_cycle<C>(team, Ls, nlev, lus[prob], nu1, nu2, dim, sm, lu_sm, LU_STAGE);
  __syncthreads();
  {
    const size_t np0 = dim == 3 ? (size_t)G[0].P * G[0].P * G[0].P : (size_t)G[0].P * G[0].P;
    for (size_t i = tid; i < np0; i += nth) G[0].xb[i] = Ls[0].xb[i];
  }
}

// Coarse sub-cycle on one thread-block cluster per problem (clusters are consecutive
// blocks along x): the level vectors stay in global memory, every CTA holds its own
// copy of the descriptors and sweep scalars.  Problem p runs lus[p].nlev levels.
constexpr int CLUSTER_THREADS = 512;
template <typename C>
__global__ void __launch_bounds__(CLUSTER_THREADS)
k_coarse_cluster(const LevelDev<C>* __restrict__ levs_all, int lev_stride, const CoarseLU* __restrict__ lus,
                 int nu1, int nu2, int dim) {
  __shared__ double sm[32 * (2 * SMAX + 1)];
  __shared__ double slots[2 * CLUSTER_MAX * TEAM_NV];
  __shared__ LevelDev<C> Ls[MAX_COARSE_LEVELS];
  __shared__ SweepScalarsT<typename CT<C>::R> Ss[MAX_COARSE_LEVELS];
  pdl_trigger();
  ClusterTeam team(slots);
  const int prob = blockIdx.x / (int)team.n;
  const CoarseLU lu = lus[prob];
  const int nlev = lu.nlev;
  const LevelDev<C>* G = levs_all + (size_t)prob * lev_stride;
  const int tid = flat_tid(), nth = block_threads();
  pdl_wait();
  if (tid == 0) {
    for (int l = 0; l < nlev; ++l) {
      Ls[l] = G[l];
      Ls[l].sc = &Ss[l];
    }
    for (int l = 0; l + 1 < nlev; ++l) Ls[l].scc = &Ss[l + 1];
  }
  {
    const int* src = reinterpret_cast<const int*>(G[0].sc);
    int* dst = reinterpret_cast<int*>(&Ss[0]);
    const int words = sweep_words<typename CT<C>::R>();
    for (int i = tid; i < words; i += nth) dst[i] = __ldcg(src + i);
  }
  __syncthreads();
  coarse_cycle<C>(team, Ls, nlev, lu, nu1, nu2, dim, sm);
  team.sync();  // no CTA leaves while another may still read its shared memory
}

}  // namespace helm
