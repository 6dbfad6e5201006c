// Shared-memory tile kernels of the grid-wide V-cycle passes (Sec. 3.1).
//
// 2D: a CTA of 32 x 8 threads owns a 64 x 16 tile; each thread owns four points
//     (x0 + lx + 32a, y0 + ly + 8b).  Threads load the raw vectors at their own points
//     (keeping them in registers for the dot products) and write the formed vector
//     into a (16+2) x (64+2) shared tile; the 164 halo points are loaded by the first
//     164 threads.  The stencil then reads shared memory only.
// 3D: a CTA of 32 x 8 threads owns a 32 x 8 column block and marches `zc` planes in
//     z.  Plane tiles (8+2) x (32+2) live in a 4-slot shared ring: the plane loaded in
//     iteration z sits in slot (z+1)&3, the stencil of plane z reads slots (z-1)&3,
//     z&3, (z+1)&3, and a slot read in iteration z is next overwritten in iteration
//     z+2, after iteration z+1's barrier, so one __syncthreads per plane suffices.
#pragma once
#include "vcycle.cuh"

namespace helm {

constexpr int T2X = 64, T2Y = 16;
constexpr int T3X = 32, T3Y = 8;
constexpr int HALO2 = 2 * (T2X + 2) + 2 * T2Y;  // 164
constexpr int HALO3 = 2 * (T3X + 2) + 2 * T3Y;  // 84

// h-th halo point of a TX x TY tile in local coordinates (-1..TX, -1..TY):
// top row, bottom row, left column, right column.
template <int TX, int TY>
__device__ __forceinline__ void halo_coord(int h, int& hx, int& hy) {
  if (h < TX + 2) { hx = h - 1; hy = -1; return; }
  h -= TX + 2;
  if (h < TX + 2) { hx = h - 1; hy = TY; return; }
  h -= TX + 2;
  if (h < TY) { hx = -1; hy = h; return; }
  h -= TY;
  hx = TX;
  hy = h;
}

template <typename C>
__device__ __forceinline__ C stencil5(const Coef3<C>& cx, const Coef3<C>& cy, typename CT<C>::R phi, C v0, C vl,
                                      C vr, C vs, C vn) {
  C diag = cadd(cx.d, cy.d);
  diag.x -= phi;
  C p = cmul(diag, v0);
  p = cfma(cx.a, vl, p);
  p = cfma(cx.c, vr, p);
  p = cfma(cy.a, vs, p);
  return cfma(cy.c, vn, p);
}

// ------------------------------------------------------------------ Arnoldi step J
// Complex128 holds twice the registers per raw vector: two CTAs per SM.
template <typename C, int J>
__global__ void __launch_bounds__(256, sizeof(C) == 16 ? 2 : (J <= 2 ? 4 : 3))
k_arnoldi_t2(const LevelDev<C>* __restrict__ levs, int ntiles, int tpc, int r0_is_b, int store_p) {
  typedef typename CT<C>::R R;
  __shared__ C vt[T2Y + 2][T2X + 2];
  __shared__ R sm[32 * (2 * J + 1)];
  const int nunits = ceil_div(ntiles, tpc);
  const int prob = blockIdx.x / nunits, unit = blockIdx.x - prob * nunits;
  const LevelDev<C>& L = levs[prob];
  auto* sc = L.sc;
  pdl_wait();
  if (sc->m < J) return;  // earlier breakdown or empty sweep: uniform for the problem
  const int n = L.n, P = L.P;
  const int ntx = ceil_div(P, T2X);
  const int lx = threadIdx.x, ly = threadIdx.y, tid = ly * 32 + lx;
  const StencilRegs<C> S(L);
  C* const pJ = L.p[J - 1];
  const C* Rk[J];
  C cf[J];
#pragma unroll
  for (int k = 0; k < J; ++k) {
    Rk[k] = (k == 0) ? (r0_is_b ? L.b : L.r0) : L.p[k - 1];
    cf[k] = sc->Cf[J][k];
  }
  C acc[J];
#pragma unroll
  for (int k = 0; k < J; ++k) acc[k] = czero<C>();
  R accn = 0;
  const int t_end = min(ntiles, (unit + 1) * tpc);
#pragma unroll 1
  for (int tile = unit * tpc; tile < t_end; ++tile) {
    const int x0 = (tile % ntx) * T2X, y0 = (tile / ntx) * T2Y;
    C raw[4][J];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int ox = lx + 32 * (q & 1), oy = ly + 8 * (q >> 1);
      C v = czero<C>();
#pragma unroll
      for (int k = 0; k < J; ++k) {
        raw[q][k] = ldc(Rk[k], x0 + ox, y0 + oy, 0, n, P);
        v = cfma(cf[k], raw[q][k], v);
      }
      vt[oy + 1][ox + 1] = v;
    }
    if (tid < HALO2) {
      int hx, hy;
      halo_coord<T2X, T2Y>(tid, hx, hy);
      C v = czero<C>();
#pragma unroll
      for (int k = 0; k < J; ++k) v = cfma(cf[k], ldc(Rk[k], x0 + hx, y0 + hy, 0, n, P), v);
      vt[hy + 1][hx + 1] = v;
    }
    __syncthreads();
    const Coef3<C> cx0 = S.coef(x0 + lx), cx1 = S.coef(x0 + lx + 32);
    Coef3<C> cy;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int ox = lx + 32 * (q & 1), oy = ly + 8 * (q >> 1);
      const int x = x0 + ox, y = y0 + oy;
      if ((q & 1) == 0) cy = S.coef(y);  // one row per pair of points
      C p = czero<C>();
      if (x < n && y < n) {
        p = stencil5((q & 1) ? cx1 : cx0, cy, S.phi_at(x, y, 0), vt[oy + 1][ox + 1], vt[oy + 1][ox],
                     vt[oy + 1][ox + 2], vt[oy][ox + 1], vt[oy + 2][ox + 1]);
#pragma unroll
        for (int k = 0; k < J; ++k) acc[k] = cdotacc(raw[q][k], p, acc[k]);
        accn += cabs2(p);
      }
      if (store_p && x < P && y < P) pJ[pidx(x, y, 0, P)] = p;
    }
    __syncthreads();  // the next tile rewrites vt
  }
  R red[2 * J + 1];
#pragma unroll
  for (int k = 0; k < J; ++k) { red[2 * k] = acc[k].x; red[2 * k + 1] = acc[k].y; }
  red[2 * J] = accn;
  pdl_trigger();  // the main work is done: let the next pass launch
  grid_sum_sweep<R, J>(red, L.part, unit, nunits, sc, sm);
}

// ------------------------------------------------------------------ Arnoldi step J, TMA (2D, complex64)
// The same pass with the raw vectors streamed by the tensor memory accelerator: a
// 136 x 18 float box per raw vector (the 64 x 16 tile plus halo, from x0 - 2 so that
// the box starts on a 16-byte boundary; out-of-range rows and columns arrive as
// zero, which is the boundary value) lands in shared memory, TMA_STAGES deep: while
// the CTA works on one tile, the next tiles' boxes are in flight.  Every wait is
// bounded; on a timeout the CTA records the error, waits (bounded) for its own copies
// and returns.
constexpr int TMA_BX = T2X + 4, TMA_BY = T2Y + 2;                        // box in complex points
constexpr unsigned TMA_BOX_BYTES = TMA_BX * TMA_BY * 8;                    // 9792
constexpr unsigned TMA_BOX_STRIDE = (TMA_BOX_BYTES + 127) / 128 * 128;     // 9856
constexpr int TMA_STAGES = 2;                                             // tiles in flight per CTA
HELM_HD constexpr unsigned tma_arnoldi_smem(int J) { return (unsigned)TMA_STAGES * J * TMA_BOX_STRIDE; }

template <int J>
__global__ void __launch_bounds__(256, J <= 2 ? 4 : 3)
k_arnoldi_tma2(const LevelDev<float2>* __restrict__ levs, int ntiles, int tpc, int r0_is_b, int store_p) {
  typedef float R;
  typedef float2 C;
  extern __shared__ __align__(128) unsigned char tsm[];
  __shared__ C vt[T2Y + 2][T2X + 2];
  __shared__ R sm[32 * (2 * J + 1)];
  __shared__ __align__(8) uint64_t bar[TMA_STAGES];
  const int nunits = ceil_div(ntiles, tpc);
  const int prob = blockIdx.x / nunits, unit = blockIdx.x - prob * nunits;
  const LevelDev<C>& L = levs[prob];
  auto* sc = L.sc;
  const int lx = threadIdx.x, ly = threadIdx.y, tid = ly * 32 + lx;
  if (tid == 0) {
#pragma unroll
    for (int q = 0; q < TMA_STAGES; ++q) mbar_init(&bar[q], 1);
    mbar_fence_init();
  }
  pdl_wait();
  if (sc->m < J) return;  // earlier breakdown or empty sweep: uniform for the problem
  const int n = L.n, P = L.P;
  const int ntx = ceil_div(P, T2X);
  const StencilRegs<C> S(L);
  C* const pJ = L.p[J - 1];
  const CUtensorMap* tm[J];
  C cf[J];
#pragma unroll
  for (int k = 0; k < J; ++k) {
    tm[k] = L.tm + (k == 0 ? (r0_is_b ? TM_B : TM_R0) : TM_P0 + k - 1);
    cf[k] = sc->Cf[J][k];
  }
  if (tid == 0)
#pragma unroll
    for (int k = 0; k < J; ++k) tmap_acquire(tm[k]);
  __syncthreads();  // initialised barriers
  const int t_beg = unit * tpc, t_end = min(ntiles, (unit + 1) * tpc);
  auto issue = [&](int t, int stage) {
    const int x0 = (t % ntx) * T2X, y0 = (t / ntx) * T2Y;
    mbar_expect_tx(&bar[stage], J * TMA_BOX_BYTES);
#pragma unroll
    for (int k = 0; k < J; ++k)
      tma_load_2d(tsm + (stage * J + k) * TMA_BOX_STRIDE, tm[k], 2 * (x0 - 2), y0 - 1, &bar[stage]);
  };
  if (tid == 0)
    for (int q = 0; q < TMA_STAGES - 1 && t_beg + q < t_end; ++q) issue(t_beg + q, q);
  C acc[J];
#pragma unroll
  for (int k = 0; k < J; ++k) acc[k] = czero<C>();
  R accn = 0;
  bool ok = true;
  int it = 0;
#pragma unroll 1
  for (int tile = t_beg; tile < t_end; ++tile, ++it) {
    const int stage = it % TMA_STAGES;
    // the stage of tile it + STAGES - 1 is the one tile it - 1 released at its end
    if (tid == 0 && tile + TMA_STAGES - 1 < t_end)
      issue(tile + TMA_STAGES - 1, (it + TMA_STAGES - 1) % TMA_STAGES);
    const bool mine = mbar_wait(&bar[stage], (unsigned)((it / TMA_STAGES) & 1));
    if (!__syncthreads_and(mine)) { ok = false; break; }
    const C* box[J];
#pragma unroll
    for (int k = 0; k < J; ++k) box[k] = reinterpret_cast<const C*>(tsm + (stage * J + k) * TMA_BOX_STRIDE);
    // v_J on the tile plus halo: vt[r][c] is the point (x0 - 1 + c, y0 - 1 + r), box
    // column c + 1.  Each thread forms its own four points and keeps their raw values
    // for the dot products; the first HALO2 threads form the halo.
    C raw[4][J];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int ox = lx + 32 * (q & 1), oy = ly + 8 * (q >> 1);
      C v = czero<C>();
#pragma unroll
      for (int k = 0; k < J; ++k) {
        raw[q][k] = box[k][(oy + 1) * TMA_BX + ox + 2];
        v = cfma(cf[k], raw[q][k], v);
      }
      vt[oy + 1][ox + 1] = v;
    }
    if (tid < HALO2) {
      int hx, hy;
      halo_coord<T2X, T2Y>(tid, hx, hy);
      C v = czero<C>();
#pragma unroll
      for (int k = 0; k < J; ++k) v = cfma(cf[k], box[k][(hy + 1) * TMA_BX + hx + 2], v);
      vt[hy + 1][hx + 1] = v;
    }
    __syncthreads();
    const int x0 = (tile % ntx) * T2X, y0 = (tile / ntx) * T2Y;
    const Coef3<C> cx0 = S.coef(x0 + lx), cx1 = S.coef(x0 + lx + 32);
    Coef3<C> cy;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int ox = lx + 32 * (q & 1), oy = ly + 8 * (q >> 1);
      const int x = x0 + ox, y = y0 + oy;
      if ((q & 1) == 0) cy = S.coef(y);  // one row per pair of points
      C p = czero<C>();
      if (x < n && y < n) {
        p = stencil5((q & 1) ? cx1 : cx0, cy, S.phi_at(x, y, 0), vt[oy + 1][ox + 1], vt[oy + 1][ox],
                     vt[oy + 1][ox + 2], vt[oy][ox + 1], vt[oy + 2][ox + 1]);
#pragma unroll
        for (int k = 0; k < J; ++k) acc[k] = cdotacc(raw[q][k], p, acc[k]);
        accn += cabs2(p);
      }
      if (store_p && x < P && y < P) pJ[pidx(x, y, 0, P)] = p;
    }
    __syncthreads();  // vt and this stage are free for reuse
  }
  if (!ok) {
    if (tid == 0) {
      atomicExch(&g_vcycle_error, 1);
      // the copies of this CTA that may still be landing (bounded)
      for (int u = it; u < it + TMA_STAGES && t_beg + u < t_end; ++u)
        mbar_wait(&bar[u % TMA_STAGES], (unsigned)((u / TMA_STAGES) & 1));
    }
    __syncthreads();
    return;
  }
  R red[2 * J + 1];
#pragma unroll
  for (int k = 0; k < J; ++k) { red[2 * k] = acc[k].x; red[2 * k + 1] = acc[k].y; }
  red[2 * J] = accn;
  pdl_trigger();  // the main work is done: let the next pass launch
  grid_sum_sweep<R, J>(red, L.part, unit, nunits, sc, sm);
}

template <typename C, int J>
__global__ void __launch_bounds__(256)
k_arnoldi_t3(const LevelDev<C>* __restrict__ levs, int ntiles, int zc, int r0_is_b, int store_p) {
  typedef typename CT<C>::R R;
  __shared__ C vb[4][T3Y + 2][T3X + 2];
  __shared__ R sm[32 * (2 * J + 1)];
  const int prob = blockIdx.x / ntiles, tile = blockIdx.x - prob * ntiles;
  const LevelDev<C>& L = levs[prob];
  auto* sc = L.sc;
  pdl_wait();
  if (sc->m < J) return;
  const int n = L.n, P = L.P;
  const int ntx = ceil_div(P, T3X), nty = ceil_div(P, T3Y);
  const int x0 = (tile % ntx) * T3X, y0 = ((tile / ntx) % nty) * T3Y;
  const int zbeg = (tile / (ntx * nty)) * zc, zend = min(zbeg + zc, P);
  const int lx = threadIdx.x, ly = threadIdx.y, tid = ly * 32 + lx;
  const int x = x0 + lx, y = y0 + ly;
  const C* Rk[J];
  C cf[J];
#pragma unroll
  for (int k = 0; k < J; ++k) {
    Rk[k] = (k == 0) ? (r0_is_b ? L.b : L.r0) : L.p[k - 1];
    cf[k] = sc->Cf[J][k];
  }
  const bool halo = tid < HALO3;
  int hx = 0, hy = 0;
  if (halo) halo_coord<T3X, T3Y>(tid, hx, hy);
  auto load_plane = [&](int z, C* raw) {
    C v = czero<C>();
#pragma unroll
    for (int k = 0; k < J; ++k) {
      const C r = ldc(Rk[k], x, y, z, n, P);
      if (raw) raw[k] = r;
      v = cfma(cf[k], r, v);
    }
    vb[z & 3][ly + 1][lx + 1] = v;
    if (halo) {
      C w = czero<C>();
#pragma unroll
      for (int k = 0; k < J; ++k) w = cfma(cf[k], ldc(Rk[k], x0 + hx, y0 + hy, z, n, P), w);
      vb[z & 3][hy + 1][hx + 1] = w;
    }
  };
  const Coef3<C> cx = ldcoef(L, x), cy = ldcoef(L, y);
  C acc[J];
#pragma unroll
  for (int k = 0; k < J; ++k) acc[k] = czero<C>();
  R accn = 0;
  if (zbeg < P) {
    C rawc[J], rawn[J];
    load_plane(zbeg - 1, nullptr);
    load_plane(zbeg, rawc);
    for (int z = zbeg; z < zend; ++z) {
      load_plane(z + 1, rawn);
      __syncthreads();
      const int s0 = z & 3;
      C p = czero<C>();
      if (inside(x, y, z, n)) {
        const Coef3<C> cz = ldcoef(L, z);
        p = stencil5(cx, cy, phi_at(L, x, y, z), vb[s0][ly + 1][lx + 1], vb[s0][ly + 1][lx], vb[s0][ly + 1][lx + 2],
                     vb[s0][ly][lx + 1], vb[s0][ly + 2][lx + 1]);
        p = cfma(cz.d, vb[s0][ly + 1][lx + 1], p);
        p = cfma(cz.a, vb[(z - 1) & 3][ly + 1][lx + 1], p);
        p = cfma(cz.c, vb[(z + 1) & 3][ly + 1][lx + 1], p);
#pragma unroll
        for (int k = 0; k < J; ++k) acc[k] = cdotacc(rawc[k], p, acc[k]);
        accn += cabs2(p);
      }
      if (store_p && x < P && y < P) L.p[J - 1][pidx(x, y, z, P)] = p;
#pragma unroll
      for (int k = 0; k < J; ++k) rawc[k] = rawn[k];
    }
  }
  R red[2 * J + 1];
#pragma unroll
  for (int k = 0; k < J; ++k) { red[2 * k] = acc[k].x; red[2 * k + 1] = acc[k].y; }
  red[2 * J] = accn;
  pdl_trigger();  // the main work is done: let the next pass launch
  grid_sum_sweep<R, J>(red, L.part, tile, ntiles, sc, sm);
}

// ------------------------------------------------------------------ end of pre-smoothing
// x_a = x + dx, r = R_0 - sum y_j p_j and b_c = FW(r), ||b_c||^2 starts the coarser
// level's first sweep.  Tiles sit at even fine offsets, so a 64 x 16 fine tile maps
// onto a 32 x 8 coarse tile (one coarse point per thread); r is formed on the tile
// plus one row/column above (x0+64, y0+16).
// The tiles of one CTA with the sweep's raw-vector count M fixed, so that every load
// of a tile (M + 1 raw vectors and x at four points per thread) is issued before the
// first is used.
template <typename C, int M>
__device__ __forceinline__ void restrict_tiles(const LevelDev<C>& L, const UpdCoef<C>& u, int unit, int tpc,
                                               int ntiles, int x_from_zero, C (*rt)[T2X + 1],
                                               typename CT<C>::R& acc) {
  typedef typename CT<C>::R R;
  const int n = L.n, P = L.P, nc = L.nc, Pc = L.Pc;
  const int ntx = ceil_div(P, T2X);
  const int lx = threadIdx.x, ly = threadIdx.y, tid = ly * 32 + lx;
  C* const xa = L.xa;
  C* const bc = L.bc;
  const int t_end = min(ntiles, (unit + 1) * tpc);
#pragma unroll 1
  for (int tile = unit * tpc; tile < t_end; ++tile) {
    const int x0 = (tile % ntx) * T2X, y0 = (tile / ntx) * T2Y;
    constexpr int QB = M >= 3 ? 2 : 4;  // points whose loads are in flight together (registers)
#pragma unroll
    for (int q0 = 0; q0 < 4; q0 += QB) {
      C v[QB][M + 1], xv[QB];
#pragma unroll
      for (int b = 0; b < QB; ++b) {
        const int q = q0 + b;
        const int x = x0 + lx + 32 * (q & 1), y = y0 + ly + 8 * (q >> 1);
#pragma unroll
        for (int k = 0; k <= M; ++k) v[b][k] = ldc(u.Rk[k], x, y, 0, n, P);
        xv[b] = (x_from_zero || x >= n || y >= n) ? czero<C>() : xa[pidx(x, y, 0, P)];
      }
#pragma unroll
      for (int b = 0; b < QB; ++b) {
        const int q = q0 + b;
        const int ox = lx + 32 * (q & 1), oy = ly + 8 * (q >> 1);
        const int x = x0 + ox, y = y0 + oy;
        C dx = czero<C>(), r = czero<C>();
#pragma unroll
        for (int k = 0; k < M; ++k) dx = cfma(u.xc[k], v[b][k], dx);
#pragma unroll
        for (int k = 0; k <= M; ++k) r = cfma(u.rc[k], v[b][k], r);
        if (x < P && y < P) xa[pidx(x, y, 0, P)] = (x < n && y < n) ? cadd(xv[b], dx) : czero<C>();
        rt[oy][ox] = r;
      }
    }
    if (tid < T2X + 1 + T2Y) {
      const int hx = tid < T2X + 1 ? tid : T2X;
      const int hy = tid < T2X + 1 ? T2Y : tid - (T2X + 1);
      C r = czero<C>();
#pragma unroll
      for (int k = 0; k <= M; ++k) r = cfma(u.rc[k], ldc(u.Rk[k], x0 + hx, y0 + hy, 0, n, P), r);
      rt[hy][hx] = r;
    }
    __syncthreads();
    const int fx = 2 * lx + 1, fy = 2 * ly + 1;
    C out = czero<C>();
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx)
        out = cadd(out, cscale(rt[fy + dy][fx + dx], (R)((dx == 0 ? 0.5 : 0.25) * (dy == 0 ? 0.5 : 0.25))));
    const int Ix = x0 / 2 + lx, Iy = y0 / 2 + ly;
    if (Ix < Pc && Iy < Pc) {
      const bool valid = Ix < nc && Iy < nc;
      bc[pidx(Ix, Iy, 0, Pc)] = valid ? out : czero<C>();
      if (valid) acc += cabs2(out);
    }
    __syncthreads();  // the next tile rewrites rt
  }
}

template <typename C>
__global__ void __launch_bounds__(256, sizeof(C) == 16 ? 2 : 3)
k_restrict_t2(const LevelDev<C>* __restrict__ levs, int ntiles, int tpc, int r0_is_b, int x_from_zero,
              int nosmooth) {
  typedef typename CT<C>::R R;
  __shared__ C rt[T2Y + 1][T2X + 1];
  __shared__ R sm[32];
  const int nunits = ceil_div(ntiles, tpc);
  const int prob = blockIdx.x / nunits, unit = blockIdx.x - prob * nunits;
  const LevelDev<C>& L = levs[prob];
  pdl_wait();
  UpdCoef<C> u = load_upd(L, r0_is_b);
  if (nosmooth) { u.m = 0; u.rc[0] = CT<C>::make(1, 0); }
  R acc = 0;
  switch (u.m) {  // uniform over the grid
    case 0: restrict_tiles<C, 0>(L, u, unit, tpc, ntiles, x_from_zero, rt, acc); break;
    case 1: restrict_tiles<C, 1>(L, u, unit, tpc, ntiles, x_from_zero, rt, acc); break;
    case 2: restrict_tiles<C, 2>(L, u, unit, tpc, ntiles, x_from_zero, rt, acc); break;
    case 3: restrict_tiles<C, 3>(L, u, unit, tpc, ntiles, x_from_zero, rt, acc); break;
    case 4: restrict_tiles<C, 4>(L, u, unit, tpc, ntiles, x_from_zero, rt, acc); break;
    default: break;
  }
  static_assert(SMAX == 4, "restrict_tiles is instantiated for m = 0..4");
  R red[1] = {acc}, tot[1];
  pdl_trigger();  // the main work is done: let the next pass launch
  if (grid_sum_last<1>(red, L.part, unit, nunits, &L.sc->counter, sm, tot)) {
    if (flat_tid() == 0) sweep_begin(L.scc, tot[0], L.s);
  }
}

// The z-march of one 3D restriction tile with the sweep's raw-vector count M fixed:
// the next plane's raw values (own point and halo point) and x are loaded before the
// current plane is processed, so each plane's loads overlap the previous plane's work.
template <typename C, int M>
__device__ __forceinline__ void restrict3_march(const LevelDev<C>& L, const UpdCoef<C>& u, int x0, int y0, int zbeg,
                                                int zend, int x_from_zero, C (*rb)[T3Y + 1][T3X + 1],
                                                typename CT<C>::R& acc) {
  typedef typename CT<C>::R R;
  const int n = L.n, P = L.P, nc = L.nc, Pc = L.Pc;
  const int lx = threadIdx.x, ly = threadIdx.y, tid = ly * 32 + lx;
  const int x = x0 + lx, y = y0 + ly;
  const bool halo = tid < T3X + 1 + T3Y;
  const int hx = tid < T3X + 1 ? tid : T3X;
  const int hy = tid < T3X + 1 ? T3Y : tid - (T3X + 1);
  const bool emit = tid < (T3X / 2) * (T3Y / 2);
  const int cx = tid % (T3X / 2), cy = tid / (T3X / 2);
  C* const xa = L.xa;
  C* const bc = L.bc;
  C vn[M + 1], hn[M + 1], xn;
  auto load = [&](int z) {
#pragma unroll
    for (int k = 0; k <= M; ++k) vn[k] = ldc(u.Rk[k], x, y, z, n, P);
    xn = (x_from_zero || !inside(x, y, z, n)) ? czero<C>() : xa[pidx(x, y, z, P)];
    if (halo) {
#pragma unroll
      for (int k = 0; k <= M; ++k) hn[k] = ldc(u.Rk[k], x0 + hx, y0 + hy, z, n, P);
    }
  };
  load(zbeg);
  for (int z = zbeg; z <= zend; ++z) {
    C vc[M + 1], hc[M + 1];
    const C xc = xn;
#pragma unroll
    for (int k = 0; k <= M; ++k) { vc[k] = vn[k]; hc[k] = hn[k]; }
    if (z < zend) load(z + 1);
    C dx = czero<C>(), r = czero<C>();
#pragma unroll
    for (int k = 0; k < M; ++k) dx = cfma(u.xc[k], vc[k], dx);
#pragma unroll
    for (int k = 0; k <= M; ++k) r = cfma(u.rc[k], vc[k], r);
    if (z < zend && x < P && y < P) xa[pidx(x, y, z, P)] = inside(x, y, z, n) ? cadd(xc, dx) : czero<C>();
    rb[z & 3][ly][lx] = r;
    if (halo) {
      C r2 = czero<C>();
#pragma unroll
      for (int k = 0; k <= M; ++k) r2 = cfma(u.rc[k], hc[k], r2);
      rb[z & 3][hy][hx] = r2;
    }
    __syncthreads();
    if ((z & 1) == 0 && z > zbeg && emit) {
      const int fx = 2 * cx + 1, fy = 2 * cy + 1;
      C out = czero<C>();
#pragma unroll
      for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
          for (int ddx = -1; ddx <= 1; ++ddx) {
            const R wgt = (R)((ddx == 0 ? 0.5 : 0.25) * (dy == 0 ? 0.5 : 0.25) * (dz == 0 ? 0.5 : 0.25));
            out = cadd(out, cscale(rb[(z - 1 + dz) & 3][fy + dy][fx + ddx], wgt));
          }
      const int Ix = x0 / 2 + cx, Iy = y0 / 2 + cy, Iz = z / 2 - 1;
      if (Ix < Pc && Iy < Pc && Iz < Pc) {
        const bool valid = Ix < nc && Iy < nc && Iz < nc;
        bc[pidx(Ix, Iy, Iz, Pc)] = valid ? out : czero<C>();
        if (valid) acc += cabs2(out);
      }
    }
  }
}

template <typename C>
__global__ void __launch_bounds__(256)
k_restrict_t3(const LevelDev<C>* __restrict__ levs, int ntiles, int zc, int r0_is_b, int x_from_zero, int nosmooth) {
  typedef typename CT<C>::R R;
  __shared__ C rb[4][T3Y + 1][T3X + 1];
  __shared__ R sm[32];
  const int prob = blockIdx.x / ntiles, tile = blockIdx.x - prob * ntiles;
  const LevelDev<C>& L = levs[prob];
  const int P = L.P;
  pdl_wait();
  const int ntx = ceil_div(P, T3X), nty = ceil_div(P, T3Y);
  const int x0 = (tile % ntx) * T3X, y0 = ((tile / ntx) % nty) * T3Y;
  const int zbeg = (tile / (ntx * nty)) * zc, zend = min(zbeg + zc, P);
  UpdCoef<C> u = load_upd(L, r0_is_b);
  if (nosmooth) { u.m = 0; u.rc[0] = CT<C>::make(1, 0); }
  R acc = 0;
  if (zbeg < P) {
    switch (u.m) {  // uniform over the grid
      case 0: restrict3_march<C, 0>(L, u, x0, y0, zbeg, zend, x_from_zero, rb, acc); break;
      case 1: restrict3_march<C, 1>(L, u, x0, y0, zbeg, zend, x_from_zero, rb, acc); break;
      case 2: restrict3_march<C, 2>(L, u, x0, y0, zbeg, zend, x_from_zero, rb, acc); break;
      case 3: restrict3_march<C, 3>(L, u, x0, y0, zbeg, zend, x_from_zero, rb, acc); break;
      case 4: restrict3_march<C, 4>(L, u, x0, y0, zbeg, zend, x_from_zero, rb, acc); break;
      default: break;
    }
  }
  R red[1] = {acc}, tot[1];
  pdl_trigger();  // the main work is done: let the next pass launch
  if (grid_sum_last<1>(red, L.part, tile, ntiles, &L.sc->counter, sm, tot)) {
    if (flat_tid() == 0) sweep_begin(L.scc, tot[0], L.s);
  }
}

// ------------------------------------------------------------------ coarse correction
// x_b = x_a + P e_c, r0 = b - M x_b, ||r0||^2 starts post-smoothing.
template <typename C>
__global__ void __launch_bounds__(256)
k_prolong_t2(const LevelDev<C>* __restrict__ levs, int ntiles, int tpc) {
  typedef typename CT<C>::R R;
  __shared__ C vt[T2Y + 2][T2X + 2];
  __shared__ R sm[32];
  const int nunits = ceil_div(ntiles, tpc);
  const int prob = blockIdx.x / nunits, unit = blockIdx.x - prob * nunits;
  const LevelDev<C>& L = levs[prob];
  const int n = L.n, P = L.P;
  pdl_wait();
  const int ntx = ceil_div(P, T2X);
  const int lx = threadIdx.x, ly = threadIdx.y, tid = ly * 32 + lx;
  const StencilRegs<C> S(L);
  const C* const xa = L.xa;
  const C* const xcb = L.xcb;
  const C* const bv = L.b;
  C* const xb = L.xb;
  C* const r0 = L.r0;
  const int nc = L.nc, Pc = L.Pc;
  auto form = [&](int xx, int yy) -> C {
    return cadd(ldc(xa, xx, yy, 0, n, P), interp(xcb, n, nc, Pc, xx, yy, 0, 2));
  };
  R acc = 0;
  const int t_end = min(ntiles, (unit + 1) * tpc);
#pragma unroll 1
  for (int tile = unit * tpc; tile < t_end; ++tile) {
    const int x0 = (tile % ntx) * T2X, y0 = (tile / ntx) * T2Y;
    C bq[4];  // b at the owned points, loaded with the first phase's reads
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int ox = lx + 32 * (q & 1), oy = ly + 8 * (q >> 1);
      bq[q] = ldc(bv, x0 + ox, y0 + oy, 0, n, P);
      vt[oy + 1][ox + 1] = form(x0 + ox, y0 + oy);
    }
    if (tid < HALO2) {
      int hx, hy;
      halo_coord<T2X, T2Y>(tid, hx, hy);
      vt[hy + 1][hx + 1] = form(x0 + hx, y0 + hy);
    }
    __syncthreads();
    const Coef3<C> cx0 = S.coef(x0 + lx), cx1 = S.coef(x0 + lx + 32);
    Coef3<C> cy;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int ox = lx + 32 * (q & 1), oy = ly + 8 * (q >> 1);
      const int x = x0 + ox, y = y0 + oy;
      if ((q & 1) == 0) cy = S.coef(y);  // one row per pair of points
      if (x < P && y < P) {
        C r = czero<C>(), xo = czero<C>();
        if (x < n && y < n) {
          const C p = stencil5((q & 1) ? cx1 : cx0, cy, S.phi_at(x, y, 0), vt[oy + 1][ox + 1], vt[oy + 1][ox],
                               vt[oy + 1][ox + 2], vt[oy][ox + 1], vt[oy + 2][ox + 1]);
          r = csub(bq[q], p);
          xo = vt[oy + 1][ox + 1];
          acc += cabs2(r);
        }
        xb[pidx(x, y, 0, P)] = xo;
        r0[pidx(x, y, 0, P)] = r;
      }
    }
    __syncthreads();  // the next tile rewrites vt
  }
  R red[1] = {acc}, tot[1];
  pdl_trigger();  // the main work is done: let the next pass launch
  if (grid_sum_last<1>(red, L.part, unit, nunits, &L.sc->counter, sm, tot)) {
    if (flat_tid() == 0) sweep_begin(L.sc, tot[0], L.s);
  }
}

template <typename C>
__global__ void __launch_bounds__(256)
k_prolong_t3(const LevelDev<C>* __restrict__ levs, int ntiles, int zc) {
  typedef typename CT<C>::R R;
  __shared__ C vb[4][T3Y + 2][T3X + 2];
  __shared__ R sm[32];
  const int prob = blockIdx.x / ntiles, tile = blockIdx.x - prob * ntiles;
  const LevelDev<C>& L = levs[prob];
  const int n = L.n, P = L.P;
  pdl_wait();
  const int ntx = ceil_div(P, T3X), nty = ceil_div(P, T3Y);
  const int x0 = (tile % ntx) * T3X, y0 = ((tile / ntx) % nty) * T3Y;
  const int zbeg = (tile / (ntx * nty)) * zc, zend = min(zbeg + zc, P);
  const int lx = threadIdx.x, ly = threadIdx.y, tid = ly * 32 + lx;
  const int x = x0 + lx, y = y0 + ly;
  const bool halo = tid < HALO3;
  int hx = 0, hy = 0;
  if (halo) halo_coord<T3X, T3Y>(tid, hx, hy);
  auto form = [&](int xx, int yy, int zz) -> C {
    return cadd(ldc((const C*)L.xa, xx, yy, zz, n, P), interp(L, xx, yy, zz, 3));
  };
  auto load_plane = [&](int z) {
    vb[z & 3][ly + 1][lx + 1] = form(x, y, z);
    if (halo) vb[z & 3][hy + 1][hx + 1] = form(x0 + hx, y0 + hy, z);
  };
  const Coef3<C> cx = ldcoef(L, x), cy = ldcoef(L, y);
  R acc = 0;
  if (zbeg < P) {
    load_plane(zbeg - 1);
    load_plane(zbeg);
    C bnext = ldc((const C*)L.b, x, y, zbeg, n, P);  // b of the next plane, loaded a plane ahead
    for (int z = zbeg; z < zend; ++z) {
      const C bcur = bnext;
      load_plane(z + 1);
      if (z + 1 < zend) bnext = ldc((const C*)L.b, x, y, z + 1, n, P);
      __syncthreads();
      const int s0 = z & 3;
      if (x < P && y < P) {
        C r = czero<C>(), xo = czero<C>();
        if (inside(x, y, z, n)) {
          const Coef3<C> cz = ldcoef(L, z);
          C p = stencil5(cx, cy, phi_at(L, x, y, z), vb[s0][ly + 1][lx + 1], vb[s0][ly + 1][lx], vb[s0][ly + 1][lx + 2],
                         vb[s0][ly][lx + 1], vb[s0][ly + 2][lx + 1]);
          p = cfma(cz.d, vb[s0][ly + 1][lx + 1], p);
          p = cfma(cz.a, vb[(z - 1) & 3][ly + 1][lx + 1], p);
          p = cfma(cz.c, vb[(z + 1) & 3][ly + 1][lx + 1], p);
          r = csub(bcur, p);
          xo = vb[s0][ly + 1][lx + 1];
          acc += cabs2(r);
        }
        L.xb[pidx(x, y, z, P)] = xo;
        L.r0[pidx(x, y, z, P)] = r;
      }
    }
  }
  R red[1] = {acc}, tot[1];
  pdl_trigger();  // the main work is done: let the next pass launch
  if (grid_sum_last<1>(red, L.part, tile, ntiles, &L.sc->counter, sm, tot)) {
    if (flat_tid() == 0) sweep_begin(L.sc, tot[0], L.s);
  }
}

}  // namespace helm
