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
template <typename C, int J, bool NC = true>
__device__ __forceinline__ void arnoldi_t2_body(const LevelDev<C>* __restrict__ levs, int ntiles, int tpc, int r0_is_b, int store_p, int vblk) {
  typedef typename CT<C>::R R;
  __shared__ C vt[T2Y + 2][T2X + 2];
  __shared__ R sm[32 * (2 * J + 1)];
  const int nunits = ceil_div(ntiles, tpc);
  const int prob = vblk / nunits, unit = vblk - prob * nunits;
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
        raw[q][k] = ldc<C, NC>(Rk[k], x0 + ox, y0 + oy, 0, n, P);
        v = cfma(cf[k], raw[q][k], v);
      }
      vt[oy + 1][ox + 1] = v;
    }
    if (tid < HALO2) {
      int hx, hy;
      halo_coord<T2X, T2Y>(tid, hx, hy);
      C v = czero<C>();
#pragma unroll
      for (int k = 0; k < J; ++k) v = cfma(cf[k], ldc<C, NC>(Rk[k], x0 + hx, y0 + hy, 0, n, P), v);
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
template <typename C, int J>
__global__ void __launch_bounds__(256, sizeof(C) == 16 ? 2 : (J <= 2 ? 4 : 3))
k_arnoldi_t2(const LevelDev<C>* __restrict__ levs, int ntiles, int tpc, int r0_is_b, int store_p) {
  arnoldi_t2_body<C, J>(levs, ntiles, tpc, r0_is_b, store_p, blockIdx.x);
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

template <typename C, int J, bool NC = true>
__device__ __forceinline__ void arnoldi_t3_body(const LevelDev<C>* __restrict__ levs, int ntiles, int zc, int r0_is_b, int store_p, int vblk) {
  typedef typename CT<C>::R R;
  __shared__ C vb[4][T3Y + 2][T3X + 2];
  __shared__ R sm[32 * (2 * J + 1)];
  const int prob = vblk / ntiles, tile = vblk - prob * ntiles;
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
  // A plane's raw values are fetched into registers one iteration before they are
  // combined into v_J and stored to the ring, so the loads of plane z + 2 are in flight
  // during iteration z's barrier and arithmetic (these levels are small and L2-resident:
  // the pass is bound by the latency of its dependent plane steps, not by bandwidth).
  auto fetch = [&](int z, C* raw, C* hraw) {
#pragma unroll
    for (int k = 0; k < J; ++k) {
      raw[k] = ldc<C, NC>(Rk[k], x, y, z, n, P);
      hraw[k] = halo ? ldc<C, NC>(Rk[k], x0 + hx, y0 + hy, z, n, P) : czero<C>();
    }
  };
  auto store_plane = [&](int z, const C* raw, const C* hraw) {
    C v = czero<C>();
#pragma unroll
    for (int k = 0; k < J; ++k) v = cfma(cf[k], raw[k], v);
    vb[z & 3][ly + 1][lx + 1] = v;
    if (halo) {
      C w = czero<C>();
#pragma unroll
      for (int k = 0; k < J; ++k) w = cfma(cf[k], hraw[k], w);
      vb[z & 3][hy + 1][hx + 1] = w;
    }
  };
  const Coef3<C> cx = ldcoef(L, x), cy = ldcoef(L, y);
  C acc[J];
#pragma unroll
  for (int k = 0; k < J; ++k) acc[k] = czero<C>();
  R accn = 0;
  if (zbeg < P) {
    C rawc[J], rawn[J], rawnn[J], hc[J], hn[J], hnn[J];
    fetch(zbeg - 1, rawc, hc);
    store_plane(zbeg - 1, rawc, hc);
    fetch(zbeg, rawc, hc);
    store_plane(zbeg, rawc, hc);
    fetch(zbeg + 1, rawn, hn);
    for (int z = zbeg; z < zend; ++z) {
      store_plane(z + 1, rawn, hn);
      fetch(z + 2, rawnn, hnn);  // z + 2 <= P: in bounds, zero past n
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
      for (int k = 0; k < J; ++k) {
        rawc[k] = rawn[k];
        rawn[k] = rawnn[k];
        hn[k] = hnn[k];
      }
    }
  }
  R red[2 * J + 1];
#pragma unroll
  for (int k = 0; k < J; ++k) { red[2 * k] = acc[k].x; red[2 * k + 1] = acc[k].y; }
  red[2 * J] = accn;
  pdl_trigger();  // the main work is done: let the next pass launch
  grid_sum_sweep<R, J>(red, L.part, tile, ntiles, sc, sm);
}
template <typename C, int J>
__global__ void __launch_bounds__(256)
k_arnoldi_t3(const LevelDev<C>* __restrict__ levs, int ntiles, int zc, int r0_is_b, int store_p) {
  arnoldi_t3_body<C, J>(levs, ntiles, zc, r0_is_b, store_p, blockIdx.x);
}

// ------------------------------------------------------------------ Arnoldi step J, TMA (3D, complex64)
// The 3D pass with the raw vectors streamed by the tensor memory accelerator.  A CTA of
// 32 x 8 threads works on columns of 32 x 8 QY points (QY points per thread, rows ly,
// ly + 8, ...).  The level's work is the sequence of (column, plane) pairs, column by
// column in z order, and CTA `unit` of a problem takes the `unit`-th of `nunits`
// equal contiguous shares of it (whole columns, or pieces at its ends; with nunits a
// multiple of the column count every share is one piece of one column, and CTAs on
// neighbouring columns march the same planes at the same time, so a tile's halo is
// read from L2).  For every plane z - 1 .. z_end of each column piece, one 72 x
// (8 QY + 2) x 1 float box per raw vector (the columns plus a one-point halo in x and
// y, starting two points left of the tile so that the box starts on a 16-byte
// boundary; out-of-range parts arrive as zero, the boundary value) lands in a ring of
// `stages` plane slots, so several planes' copies are in flight while the CTA forms
// v_J of the newest plane.  Each thread keeps v_J of its own points on three
// consecutive planes in registers (the stencil's z neighbours) and writes the newest
// plane into a 3-slot shared ring for the x and y neighbours: the slot written in
// iteration f was last read in iteration f - 2, before iteration f - 1's barrier, so
// one barrier per plane suffices.  Every wait is bounded; on a timeout the CTA records
// the error, waits (bounded) for its own copies and returns.
constexpr int TM3_TX = 32;
constexpr int TM3_TY2 = 16;                                                  // tile height at two points per thread
constexpr int TM3_BX = TM3_TX + 4;                                          // box width in complex points
HELM_HD constexpr int tm3_ty(int QY) { return 8 * QY; }
HELM_HD constexpr unsigned tm3_box_bytes(int QY) { return TM3_BX * (8 * QY + 2) * 8; }
HELM_HD constexpr unsigned tm3_box_stride(int QY) { return (tm3_box_bytes(QY) + 127) / 128 * 128; }
HELM_HD constexpr unsigned tma3_arnoldi_smem(int J, int QY, int stages) {
  return (unsigned)stages * J * tm3_box_stride(QY);
}
// (column, plane) pairs and columns of a level of pitch P (a multiple of 32)
HELM_HD inline int tma3_cols(int P, int QY) { return (P / TM3_TX) * (P / tm3_ty(QY)); }
HELM_HD inline long long tma3_work(int P, int QY) { return (long long)tma3_cols(P, QY) * P; }

// Walks the planes a CTA loads: z = zs - 1 .. ze of each column piece, in order.
struct Tma3Cursor {
  int col, z, ze;
  __device__ __forceinline__ void start(int g0, int g1, int P) {
    col = g0 / P;
    z = g0 - col * P - 1;
    ze = min(P, g1 - col * P);
  }
  // to the next plane: 1 in the same piece, 2 at the start of the next column's piece,
  // 0 when the plane just passed was the last of the share
  __device__ __forceinline__ int advance(int g1, int P) {
    if (z < ze) { ++z; return 1; }
    ++col;
    if (col * P >= g1) return 0;
    z = -1;
    ze = min(P, g1 - col * P);
    return 2;
  }
};

template <int J, int QY, bool RESID>
__global__ void __launch_bounds__(256, (J == 1 && QY == 2) ? 3 : 2)
k_stencil_tma3(const LevelDev<float2>* __restrict__ levs, int nunits, int stages, int r0_is_b, int store_p) {
  typedef float R;
  typedef float2 C;
  constexpr int TY = 8 * QY;
  constexpr int BY = TY + 2;
  constexpr unsigned BOX = tm3_box_bytes(QY), STRIDE = tm3_box_stride(QY);
  constexpr int HALO = 2 * (TM3_TX + 2) + 2 * TY;
  extern __shared__ __align__(128) unsigned char tsm[];
  __shared__ C vr[3][BY][TM3_TX + 2];
  __shared__ R sm[32 * (2 * J + 1)];
  __shared__ __align__(8) uint64_t bar[TM3_STAGES_MAX];
  const int prob = blockIdx.x / nunits, unit = blockIdx.x - prob * nunits;
  const LevelDev<C>& L = levs[prob];
  auto* sc = L.sc;
  const int lx = threadIdx.x, ly = threadIdx.y, tid = ly * 32 + lx;
  if (tid == 0) {
    for (int q = 0; q < stages; ++q) mbar_init(&bar[q], 1);
    mbar_fence_init();
  }
  pdl_wait();
  if (!RESID && sc->m < J) return;  // earlier breakdown or empty sweep: uniform for the problem
  const int n = L.n, P = L.P;
  const int ntx = P / TM3_TX;
  const long long work = tma3_work(P, QY);
  const int g0 = (int)(work * unit / nunits), g1 = (int)(work * (unit + 1) / nunits);
  const StencilRegs<C> S(L);
  C* const pJ = L.p[J - 1];
  const CUtensorMap* tm[J];
  C cf[J];
  const CUtensorMap* maps = L.tm + (QY == 4 ? TM_COUNT : 0);
#pragma unroll
  for (int k = 0; k < J; ++k) {
    if (RESID) {
      tm[k] = maps + TM_XB;
      cf[k] = make_float2(1.f, 0.f);
    } else {
      tm[k] = maps + (k == 0 ? (r0_is_b ? TM_B : TM_R0) : TM_P0 + k - 1);
      cf[k] = sc->Cf[J][k];
    }
  }
  if (tid == 0)
#pragma unroll
    for (int k = 0; k < J; ++k) tmap_acquire(tm[k]);
  __syncthreads();  // initialised barriers
  // producer (thread 0): issues the planes of the share in order into the stage ring
  Tma3Cursor pc;
  pc.start(g0, g1, P);
  bool pmore = true;
  int pstage = 0, issued = 0;
  auto issue_next = [&]() {
    const int x0 = (pc.col % ntx) * TM3_TX, y0 = (pc.col / ntx) * TY;
    mbar_expect_tx(&bar[pstage], J * BOX);
#pragma unroll
    for (int k = 0; k < J; ++k)
      tma_load_3d(tsm + (pstage * J + k) * STRIDE, tm[k], 2 * (x0 - 2), y0 - 1, pc.z, &bar[pstage]);
    pstage = pstage + 1 == stages ? 0 : pstage + 1;
    ++issued;
    pmore = pc.advance(g1, P) != 0;
  };
  if (tid == 0)
    for (int q = 0; q < stages && pmore; ++q) issue_next();
  int hx = 0, hy = 0;
  const bool halo = tid < HALO;
  if (halo) halo_coord<TM3_TX, TY>(tid, hx, hy);
  C acc[J];
#pragma unroll
  for (int k = 0; k < J; ++k) acc[k] = czero<C>();
  R accn = 0;
  C rawp[QY][J];          // own raw values of the previous plane
  C vprev[QY], vcur[QY];  // own v_J two planes and one plane back
  Coef3<C> cx, cy[QY];
  int x0 = 0, y0 = 0;
  unsigned off = 0;       // padded index of the thread's first point in plane 0
  // consumer: walks the same planes
  Tma3Cursor cc;
  cc.start(g0, g1, P);
  int u = 0, cstage = 0, rslot = 0, consumed = 0;
  unsigned cphase = 0;
  bool ok = true, more = true;
#pragma unroll 1
  while (more) {
    if (u == 0) {
      x0 = (cc.col % ntx) * TM3_TX;
      y0 = (cc.col / ntx) * TY;
      cx = S.coef(x0 + lx);
#pragma unroll
      for (int q = 0; q < QY; ++q) cy[q] = S.coef(y0 + ly + 8 * q);
      off = (unsigned)(y0 + ly) * P + x0 + lx;
    }
    // the stencil of this iteration works on plane z = cc.z - 1 (from the third plane
    // of a piece on); its phi is fetched before the wait (in bounds: z < P)
    const int z = cc.z - 1;
    const unsigned pz = off + (unsigned)z * P * P;
    R ph[QY];
    C bq[QY];  // residual mode: b at the stencil plane, fetched with phi
#pragma unroll
    for (int q = 0; q < QY; ++q) {
      ph[q] = (u >= 2 && S.phi) ? __ldg(S.phi + pz + 8 * q * P) : S.phic;
      if (RESID) bq[q] = u >= 2 ? __ldg(L.b + pz + 8 * q * P) : czero<C>();
    }
    const bool mine = mbar_wait(&bar[cstage], cphase);
    const C* box[J];
#pragma unroll
    for (int k = 0; k < J; ++k) box[k] = reinterpret_cast<const C*>(tsm + (cstage * J + k) * STRIDE);
    C (*vs)[TM3_TX + 2] = vr[rslot];
    C rawn[QY][J], vnew[QY];
#pragma unroll
    for (int q = 0; q < QY; ++q) {
      const int oy = ly + 8 * q;
      C v = czero<C>();
#pragma unroll
      for (int k = 0; k < J; ++k) {
        rawn[q][k] = box[k][(oy + 1) * TM3_BX + lx + 2];
        v = cfma(cf[k], rawn[q][k], v);
      }
      vnew[q] = v;
      vs[oy + 1][lx + 1] = v;
    }
    if (halo) {
      C v = czero<C>();
#pragma unroll
      for (int k = 0; k < J; ++k) v = cfma(cf[k], box[k][(hy + 1) * TM3_BX + hx + 2], v);
      vs[hy + 1][hx + 1] = v;
    }
    if (!__syncthreads_and(mine)) { ok = false; break; }
    ++consumed;
    // every thread is done with this stage: refill it with the next plane
    if (tid == 0 && pmore) issue_next();
    if (u >= 2) {
      const Coef3<C> cz = S.coef(z);
      C (*vc)[TM3_TX + 2] = vr[rslot == 0 ? 2 : rslot - 1];
      const bool zin = z < n && x0 + lx < n;
#pragma unroll
      for (int q = 0; q < QY; ++q) {
        const int oy = ly + 8 * q;
        C p = czero<C>();
        if (zin && y0 + oy < n) {
          p = stencil5(cx, cy[q], ph[q], vcur[q], vc[oy + 1][lx], vc[oy + 1][lx + 2], vc[oy][lx + 1],
                       vc[oy + 2][lx + 1]);
          p = cfma(cz.d, vcur[q], p);
          p = cfma(cz.a, vprev[q], p);
          p = cfma(cz.c, vnew[q], p);
          if (RESID) {
            p = csub(bq[q], p);  // r0 = b - M x_b
            accn += cabs2(p);
          } else {
#pragma unroll
            for (int k = 0; k < J; ++k) acc[k] = cdotacc(rawp[q][k], p, acc[k]);
            accn += cabs2(p);
          }
        }
        if (RESID) L.r0[pz + 8 * q * P] = p;
        else if (store_p) pJ[pz + 8 * q * P] = p;
      }
    }
#pragma unroll
    for (int q = 0; q < QY; ++q) {
      vprev[q] = vcur[q];
      vcur[q] = vnew[q];
#pragma unroll
      for (int k = 0; k < J; ++k) rawp[q][k] = rawn[q][k];
    }
    rslot = rslot == 2 ? 0 : rslot + 1;
    if (++cstage == stages) { cstage = 0; cphase ^= 1u; }
    const int step = cc.advance(g1, P);
    more = step != 0;
    u = step == 2 ? 0 : u + 1;
  }
  if (!ok) {
    if (tid == 0) {
      atomicExch(&g_vcycle_error, 1);
      // the copies of this CTA that may still be landing (bounded)
      int st = cstage;
      unsigned ph = cphase;
      for (int g = consumed; g < issued; ++g) {
        mbar_wait(&bar[st], ph);
        if (++st == stages) { st = 0; ph ^= 1u; }
      }
    }
    __syncthreads();
    return;
  }
  pdl_trigger();  // the main work is done: let the next pass launch
  if (RESID) {
    // ||r0||^2 starts the post-smoothing sweep
    R red[1] = {accn}, tot[1];
    if (grid_sum_last<1>(red, L.part, unit, nunits, &sc->counter, sm, tot)) {
      if (flat_tid() == 0) sweep_begin(sc, tot[0], L.s);
    }
    return;
  }
  R red[2 * J + 1];
#pragma unroll
  for (int k = 0; k < J; ++k) { red[2 * k] = acc[k].x; red[2 * k + 1] = acc[k].y; }
  red[2 * J] = accn;
  grid_sum_sweep<R, J>(red, L.part, unit, nunits, sc, sm);
}

// ------------------------------------------------------------------ end of pre-smoothing, TMA (3D, complex64)
// x_a = x + dx, r = R_0 - sum y_j p_j and b_c = FW(r) on a 3D level with the sweep's
// M + 1 raw vectors streamed by TMA: the plane boxes of the Arnoldi pass (72 x 18 x 1
// floats from (x0 - 2, y0 - 1), the same tensor maps) hold the tile's 32 x 16 points and
// the extra column x0 + 32 and row y0 + 16 the full weighting of the tile's 16 x 8 coarse
// points reads.  The CTA's share of the (column, plane) sequence is walked as in the
// Arnoldi pass; r of each plane goes into a 4-slot shared ring, and after every even
// plane z the coarse plane centred on z - 1 is emitted (when z - 1 lies in the piece).
// Iteration f reads slots f - 2 .. f after its barrier; iteration f + 1 writes slot
// (f + 1) & 3 = (f - 3) & 3, last read in iteration f - 1, before iteration f's barrier,
// so one barrier per plane suffices.  Bounded waits as in the Arnoldi pass.
template <typename C, int M>
__device__ __forceinline__ void restrict_tma3_run(const LevelDev<C>& L, const UpdCoef<C>& u, int g0, int g1, int stages,
                                                  int x_from_zero, const CUtensorMap* const* tm, unsigned char* tsm,
                                                  uint64_t* bar, C (*rr)[TM3_TY2 + 1][TM3_TX + 1], typename CT<C>::R& acc,
                                                  bool& ok) {
  typedef typename CT<C>::R R;
  constexpr int NR = M + 1;  // raw vectors
  constexpr unsigned BOX = tm3_box_bytes(2), STRIDE = tm3_box_stride(2);
  const int n = L.n, P = L.P, nc = L.nc, Pc = L.Pc;
  const int ntx = P / TM3_TX;
  const int lx = threadIdx.x, ly = threadIdx.y, tid = ly * 32 + lx;
  // the extra points: row y0 + 16 (x0 .. x0 + 32) and column x0 + 32 (y0 .. y0 + 15)
  const bool extra = tid < (TM3_TX + 1) + TM3_TY2;
  const int ex = tid < TM3_TX + 1 ? tid : TM3_TX;
  const int ey = tid < TM3_TX + 1 ? TM3_TY2 : tid - (TM3_TX + 1);
  const bool emit = tid < (TM3_TX / 2) * (TM3_TY2 / 2);
  const int ecx = tid % (TM3_TX / 2), ecy = tid / (TM3_TX / 2);
  C* const xa = L.xa;
  C* const bc = L.bc;
  Tma3Cursor pc;
  pc.start(g0, g1, P);
  bool pmore = true;
  int pstage = 0, issued = 0;
  auto issue_next = [&]() {
    const int x0 = (pc.col % ntx) * TM3_TX, y0 = (pc.col / ntx) * TM3_TY2;
    mbar_expect_tx(&bar[pstage], NR * BOX);
#pragma unroll
    for (int k = 0; k < NR; ++k)
      tma_load_3d(tsm + (pstage * NR + k) * STRIDE, tm[k], 2 * (x0 - 2), y0 - 1, pc.z, &bar[pstage]);
    pstage = pstage + 1 == stages ? 0 : pstage + 1;
    ++issued;
    pmore = pc.advance(g1, P) != 0;
  };
  if (tid == 0)
    for (int q = 0; q < stages && pmore; ++q) issue_next();
  Tma3Cursor cc;
  cc.start(g0, g1, P);
  int u_ = 0, cstage = 0, f = 0, consumed = 0;
  unsigned cphase = 0;
  int x0 = 0, y0 = 0;
  bool more = true;
#pragma unroll 1
  while (more) {
    if (u_ == 0) {
      x0 = (cc.col % ntx) * TM3_TX;
      y0 = (cc.col / ntx) * TM3_TY2;
    }
    const int z = cc.z;  // the plane loaded in this iteration
    C xv[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int x = x0 + lx, y = y0 + ly + 8 * q;
      xv[q] = (x_from_zero || !inside(x, y, z, n)) ? czero<C>() : xa[pidx(x, y, z, P)];
    }
    const bool mine = mbar_wait(&bar[cstage], cphase);
    const C* box[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) box[k] = reinterpret_cast<const C*>(tsm + (cstage * NR + k) * STRIDE);
    C (*rs)[TM3_TX + 1] = rr[f & 3];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int oy = ly + 8 * q;
      C v[NR];
#pragma unroll
      for (int k = 0; k < NR; ++k) v[k] = box[k][(oy + 1) * TM3_BX + lx + 2];
      C dx = czero<C>(), r = czero<C>();
#pragma unroll
      for (int k = 0; k < M; ++k) dx = cfma(u.xc[k], v[k], dx);
#pragma unroll
      for (int k = 0; k <= M; ++k) r = cfma(u.rc[k], v[k], r);
      rs[oy][lx] = r;
      const int x = x0 + lx, y = y0 + oy;
      if (z >= 0 && z < P && u_ >= 1 && z < cc.ze)  // planes zs .. ze - 1 of the piece
        xa[pidx(x, y, z, P)] = inside(x, y, z, n) ? cadd(xv[q], dx) : czero<C>();
    }
    if (extra) {
      C r = czero<C>();
#pragma unroll
      for (int k = 0; k <= M; ++k) r = cfma(u.rc[k], box[k][(ey + 1) * TM3_BX + ex + 2], r);
      rs[ey][ex] = r;
    }
    if (!__syncthreads_and(mine)) { ok = false; break; }
    ++consumed;
    if (tid == 0 && pmore) issue_next();
    // coarse plane centred on z - 1 (odd), when z - 1 is a plane of the piece
    if (u_ >= 2 && (z & 1) == 0 && emit) {
      const int fx = 2 * ecx + 1, fy = 2 * ecy + 1;
      C out = czero<C>();
#pragma unroll
      for (int dz = -1; dz <= 1; ++dz) {
        C (*rz)[TM3_TX + 1] = rr[(f - 1 + dz) & 3];
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
          for (int ddx = -1; ddx <= 1; ++ddx) {
            const R wgt = (R)((ddx == 0 ? 0.5 : 0.25) * (dy == 0 ? 0.5 : 0.25) * (dz == 0 ? 0.5 : 0.25));
            out = cadd(out, cscale(rz[fy + dy][fx + ddx], wgt));
          }
      }
      const int Ix = x0 / 2 + ecx, Iy = y0 / 2 + ecy, Iz = z / 2 - 1;
      if (Ix < Pc && Iy < Pc && Iz < Pc) {
        const bool valid = Ix < nc && Iy < nc && Iz < nc;
        bc[pidx(Ix, Iy, Iz, Pc)] = valid ? out : czero<C>();
        if (valid) acc += cabs2(out);
      }
    }
    if (++cstage == stages) { cstage = 0; cphase ^= 1u; }
    ++f;
    const int step = cc.advance(g1, P);
    more = step != 0;
    u_ = step == 2 ? 0 : u_ + 1;
  }
  if (!ok && tid == 0) {
    atomicExch(&g_vcycle_error, 1);
    int st = cstage;
    unsigned ph = cphase;
    for (int g = consumed; g < issued; ++g) {
      mbar_wait(&bar[st], ph);
      if (++st == stages) { st = 0; ph ^= 1u; }
    }
  }
}

template <int M_MAX>
__global__ void __launch_bounds__(256, 2)
k_restrict_tma3(const LevelDev<float2>* __restrict__ levs, int nunits, int stages, int r0_is_b, int x_from_zero,
                int nosmooth) {
  typedef float R;
  typedef float2 C;
  extern __shared__ __align__(128) unsigned char tsm[];
  __shared__ C rr[4][TM3_TY2 + 1][TM3_TX + 1];
  __shared__ R sm[32];
  __shared__ __align__(8) uint64_t bar[TM3_STAGES_MAX];
  const int prob = blockIdx.x / nunits, unit = blockIdx.x - prob * nunits;
  const LevelDev<C>& L = levs[prob];
  const int tid = flat_tid();
  if (tid == 0) {
    for (int q = 0; q < stages; ++q) mbar_init(&bar[q], 1);
    mbar_fence_init();
  }
  pdl_wait();
  UpdCoef<C> u = load_upd(L, r0_is_b);
  if (nosmooth) { u.m = 0; u.rc[0] = CT<C>::make(1, 0); }
  const int P = L.P;
  const long long work = tma3_work(P, 2);
  const int g0 = (int)(work * unit / nunits), g1 = (int)(work * (unit + 1) / nunits);
  const CUtensorMap* tm[SMAX + 1];
#pragma unroll
  for (int k = 0; k <= SMAX; ++k)
    tm[k] = L.tm + (k == 0 ? (r0_is_b ? TM_B : TM_R0) : TM_P0 + k - 1);
  if (tid == 0)
    for (int k = 0; k <= u.m; ++k) tmap_acquire(tm[k]);
  __syncthreads();  // initialised barriers
  R acc = 0;
  bool ok = true;
  switch (u.m) {  // uniform over the grid
    case 0: restrict_tma3_run<C, 0>(L, u, g0, g1, stages, x_from_zero, tm, tsm, bar, rr, acc, ok); break;
    case 1: restrict_tma3_run<C, 1>(L, u, g0, g1, stages, x_from_zero, tm, tsm, bar, rr, acc, ok); break;
    case 2: restrict_tma3_run<C, 2>(L, u, g0, g1, stages, x_from_zero, tm, tsm, bar, rr, acc, ok); break;
    case 3: restrict_tma3_run<C, 3>(L, u, g0, g1, stages, x_from_zero, tm, tsm, bar, rr, acc, ok); break;
    default: restrict_tma3_run<C, 4>(L, u, g0, g1, stages, x_from_zero, tm, tsm, bar, rr, acc, ok); break;
  }
  if (!__syncthreads_and(ok)) return;
  R red[1] = {acc}, tot[1];
  pdl_trigger();  // the main work is done: let the next pass launch
  if (grid_sum_last<1>(red, L.part, unit, nunits, &L.sc->counter, sm, tot)) {
    if (flat_tid() == 0) sweep_begin(L.scc, tot[0], L.s);
  }
}

// x_b = x_a + P e_c on a 3D level, in tiles of PR_ROWS full rows at one z: every
// thread issues the loads of x_a at its points of all the tile's rows first; the five
// coarse rows the tile's trilinear interpolation reads (Y = y0/2 - 1 .. y0/2 + 3),
// each already combined over the one or two coarse planes of z with their weight,
// are staged in shared memory, from which every point takes its y and x neighbours.
// The stencil and residual follow in k_stencil_tma3<1, QY, true>.
constexpr int PR_ROWS = 8;
template <typename C, int PR_XPT>  // points per thread per row: P <= 256 PR_XPT
__global__ void __launch_bounds__(256)
k_prolong3_rows(const LevelDev<C>* __restrict__ levs, int nblk) {
  typedef typename CT<C>::R R;
  __shared__ C cr[5][512 + 1];  // coarse rows Y0 + i, index X + 1 (X = -1 is the boundary)
  const int prob = blockIdx.x / nblk, blk = blockIdx.x - prob * nblk;
  const LevelDev<C>& L = levs[prob];
  pdl_wait();
  const int n = L.n, P = L.P, nc = L.nc, Pc = L.Pc;
  const int nyb = P / PR_ROWS;
  const int items = nyb * P;  // (row block, plane) pairs
  const int tid = threadIdx.x;
  for (int it = blk; it < items; it += nblk) {
    const int yb = it % nyb, z = it / nyb;
    const int y0 = yb * PR_ROWS, Y0 = y0 / 2 - 1;
    C xa[PR_ROWS][PR_XPT];
#pragma unroll
    for (int r = 0; r < PR_ROWS; ++r)
#pragma unroll
      for (int k = 0; k < PR_XPT; ++k) xa[r][k] = ldc(L.xa, tid + 256 * k, y0 + r, z, n, P);
    int iz[2], nz;
    R wz;
    if (z & 1) { iz[0] = z >> 1; iz[1] = 0; nz = 1; wz = 1; }
    else { iz[0] = (z >> 1) - 1; iz[1] = z >> 1; nz = 2; wz = 0.5; }
    for (int e = tid; e < 5 * Pc; e += 256) {
      const int i = e / Pc, X = e - i * Pc;
      C a = ldc(L.xcb, X, Y0 + i, iz[0], nc, Pc);
      if (nz == 2) a = cadd(a, ldc(L.xcb, X, Y0 + i, iz[1], nc, Pc));
      cr[i][X + 1] = cscale(a, wz);
    }
    if (tid < 5) cr[tid][0] = czero<C>();
    __syncthreads();
#pragma unroll
    for (int r = 0; r < PR_ROWS; ++r) {
      const int y = y0 + r;
      // coarse rows of y: Y = y >> 1 (odd y, weight 1) or y/2 - 1 and y/2 (even, 1/2 each)
      const int i0 = (y & 1) ? (y >> 1) - Y0 : (y >> 1) - 1 - Y0;
      const bool two = !(y & 1);
#pragma unroll
      for (int k = 0; k < PR_XPT; ++k) {
        const int x = tid + 256 * k;
        if (x >= P) continue;
        C v = czero<C>();
        if (inside(x, y, z, n)) {
          auto row = [&](int X) -> C {  // the y-combined coarse value at X (-1 <= X < Pc)
            return two ? cscale(cadd(cr[i0][X + 1], cr[i0 + 1][X + 1]), (R)0.5) : cr[i0][X + 1];
          };
          const C e = (x & 1) ? row(x >> 1) : cscale(cadd(row((x >> 1) - 1), row(x >> 1)), (R)0.5);
          v = cadd(xa[r][k], e);
        }
        L.xb[pidx(x, y, z, P)] = v;
      }
    }
    __syncthreads();  // the next tile rewrites cr
  }
  pdl_trigger();
}

// ------------------------------------------------------------------ end of pre-smoothing
// x_a = x + dx, r = R_0 - sum y_j p_j and b_c = FW(r), ||b_c||^2 starts the coarser
// level's first sweep.  Tiles sit at even fine offsets, so a 64 x 16 fine tile maps
// onto a 32 x 8 coarse tile (one coarse point per thread); r is formed on the tile
// plus one row/column above (x0+64, y0+16).
// The tiles of one CTA with the sweep's raw-vector count M fixed, so that every load
// of a tile (M + 1 raw vectors and x at four points per thread) is issued before the
// first is used.
template <typename C, int M, bool NC = true>
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
        for (int k = 0; k <= M; ++k) v[b][k] = ldc<C, NC>(u.Rk[k], x, y, 0, n, P);
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
      for (int k = 0; k <= M; ++k) r = cfma(u.rc[k], ldc<C, NC>(u.Rk[k], x0 + hx, y0 + hy, 0, n, P), r);
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

template <typename C, bool NC = true>
__device__ __forceinline__ void restrict_t2_body(const LevelDev<C>* __restrict__ levs, int ntiles, int tpc, int r0_is_b, int x_from_zero,
              int nosmooth, int vblk) {
  typedef typename CT<C>::R R;
  __shared__ C rt[T2Y + 1][T2X + 1];
  __shared__ R sm[32];
  const int nunits = ceil_div(ntiles, tpc);
  const int prob = vblk / nunits, unit = vblk - prob * nunits;
  const LevelDev<C>& L = levs[prob];
  pdl_wait();
  UpdCoef<C> u = load_upd(L, r0_is_b);
  if (nosmooth) { u.m = 0; u.rc[0] = CT<C>::make(1, 0); }
  R acc = 0;
  switch (u.m) {  // uniform over the grid
    case 0: restrict_tiles<C, 0, NC>(L, u, unit, tpc, ntiles, x_from_zero, rt, acc); break;
    case 1: restrict_tiles<C, 1, NC>(L, u, unit, tpc, ntiles, x_from_zero, rt, acc); break;
    case 2: restrict_tiles<C, 2, NC>(L, u, unit, tpc, ntiles, x_from_zero, rt, acc); break;
    case 3: restrict_tiles<C, 3, NC>(L, u, unit, tpc, ntiles, x_from_zero, rt, acc); break;
    case 4: restrict_tiles<C, 4, NC>(L, u, unit, tpc, ntiles, x_from_zero, rt, acc); break;
    default: break;
  }
  static_assert(SMAX == 4, "restrict_tiles is instantiated for m = 0..4");
  R red[1] = {acc}, tot[1];
  pdl_trigger();  // the main work is done: let the next pass launch
  if (grid_sum_last<1>(red, L.part, unit, nunits, &L.sc->counter, sm, tot)) {
    if (flat_tid() == 0) sweep_begin(L.scc, tot[0], L.s);
  }
}
template <typename C>
__global__ void __launch_bounds__(256, sizeof(C) == 16 ? 2 : 3)
k_restrict_t2(const LevelDev<C>* __restrict__ levs, int ntiles, int tpc, int r0_is_b, int x_from_zero,
              int nosmooth) {
  restrict_t2_body<C>(levs, ntiles, tpc, r0_is_b, x_from_zero, nosmooth, blockIdx.x);
}

// The z-march of one 3D restriction tile with the sweep's raw-vector count M fixed:
// the next plane's raw values (own point and halo point) and x are loaded before the
// current plane is processed, so each plane's loads overlap the previous plane's work.
template <typename C, int M, bool NC = true>
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
    for (int k = 0; k <= M; ++k) vn[k] = ldc<C, NC>(u.Rk[k], x, y, z, n, P);
    xn = (x_from_zero || !inside(x, y, z, n)) ? czero<C>() : xa[pidx(x, y, z, P)];
    if (halo) {
#pragma unroll
      for (int k = 0; k <= M; ++k) hn[k] = ldc<C, NC>(u.Rk[k], x0 + hx, y0 + hy, z, n, P);
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

template <typename C, bool NC = true>
__device__ __forceinline__ void restrict_t3_body(const LevelDev<C>* __restrict__ levs, int ntiles, int zc, int r0_is_b, int x_from_zero, int nosmooth, int vblk) {
  typedef typename CT<C>::R R;
  __shared__ C rb[4][T3Y + 1][T3X + 1];
  __shared__ R sm[32];
  const int prob = vblk / ntiles, tile = vblk - prob * ntiles;
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
      case 0: restrict3_march<C, 0, NC>(L, u, x0, y0, zbeg, zend, x_from_zero, rb, acc); break;
      case 1: restrict3_march<C, 1, NC>(L, u, x0, y0, zbeg, zend, x_from_zero, rb, acc); break;
      case 2: restrict3_march<C, 2, NC>(L, u, x0, y0, zbeg, zend, x_from_zero, rb, acc); break;
      case 3: restrict3_march<C, 3, NC>(L, u, x0, y0, zbeg, zend, x_from_zero, rb, acc); break;
      case 4: restrict3_march<C, 4, NC>(L, u, x0, y0, zbeg, zend, x_from_zero, rb, acc); break;
      default: break;
    }
  }
  R red[1] = {acc}, tot[1];
  pdl_trigger();  // the main work is done: let the next pass launch
  if (grid_sum_last<1>(red, L.part, tile, ntiles, &L.sc->counter, sm, tot)) {
    if (flat_tid() == 0) sweep_begin(L.scc, tot[0], L.s);
  }
}
template <typename C>
__global__ void __launch_bounds__(256)
k_restrict_t3(const LevelDev<C>* __restrict__ levs, int ntiles, int zc, int r0_is_b, int x_from_zero, int nosmooth) {
  restrict_t3_body<C>(levs, ntiles, zc, r0_is_b, x_from_zero, nosmooth, blockIdx.x);
}

// ------------------------------------------------------------------ coarse correction
// x_b = x_a + P e_c, r0 = b - M x_b, ||r0||^2 starts post-smoothing.
template <typename C, bool NC = true>
__device__ __forceinline__ void prolong_t2_body(const LevelDev<C>* __restrict__ levs, int ntiles, int tpc, int vblk) {
  typedef typename CT<C>::R R;
  __shared__ C vt[T2Y + 2][T2X + 2];
  __shared__ R sm[32];
  const int nunits = ceil_div(ntiles, tpc);
  const int prob = vblk / nunits, unit = vblk - prob * nunits;
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
    return cadd(ldc<C, NC>(xa, xx, yy, 0, n, P), interp<C, NC>(xcb, n, nc, Pc, xx, yy, 0, 2));
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
      bq[q] = ldc<C, NC>(bv, x0 + ox, y0 + oy, 0, n, P);
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
k_prolong_t2(const LevelDev<C>* __restrict__ levs, int ntiles, int tpc) {
  prolong_t2_body<C>(levs, ntiles, tpc, blockIdx.x);
}

template <typename C, bool NC = true>
__device__ __forceinline__ void prolong_t3_body(const LevelDev<C>* __restrict__ levs, int ntiles, int zc, int vblk) {
  typedef typename CT<C>::R R;
  __shared__ C vb[4][T3Y + 2][T3X + 2];
  __shared__ R sm[32];
  const int prob = vblk / ntiles, tile = vblk - prob * ntiles;
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
    return cadd(ldc<C, NC>((const C*)L.xa, xx, yy, zz, n, P), interp<C, NC>(L, xx, yy, zz, 3));
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
    C bnext = ldc<C, NC>((const C*)L.b, x, y, zbeg, n, P);  // b of the next plane, loaded a plane ahead
    for (int z = zbeg; z < zend; ++z) {
      const C bcur = bnext;
      load_plane(z + 1);
      if (z + 1 < zend) bnext = ldc<C, NC>((const C*)L.b, x, y, z + 1, n, P);
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
template <typename C>
__global__ void __launch_bounds__(256)
k_prolong_t3(const LevelDev<C>* __restrict__ levs, int ntiles, int zc) {
  prolong_t3_body<C>(levs, ntiles, zc, blockIdx.x);
}

}  // namespace helm

namespace helm {

// ------------------------------------------------------------------ persistent V-cycle segments
// The small grid-wide levels of a V-cycle (where every pass is a few microseconds of
// work behind a launch and a reduction) run as one cooperative launch per half cycle:
// the passes of the descent of those levels (or of the ascent) are walked in order, each
// pass's virtual blocks (the blocks of its ordinary launch, for every problem of the
// group) spread over the persistent CTAs, with a grid-wide barrier between passes.
// A virtual block does exactly what the block of the ordinary launch does (the same
// body, the same partial-sum slot, the same last-block reduction), so the results are
// bitwise those of the launch-per-pass schedule.  Vectors written earlier in the same
// launch are read through the coherent path (NC = false: the read-only cache does not
// see another SM's writes within a kernel); the barrier's fences order the passes.
// A CTA waits at most limit_ns (globaltimer) at a barrier; then it records the error
// (the solve reports HELM_ETIMEOUT) and the whole launch returns: never a trap, never
// an endless spin.
__device__ __forceinline__ bool grid_barrier(GridBar* gb, unsigned nblocks, unsigned long long limit_ns) {
  __shared__ int ok;
  __syncthreads();
  if (flat_tid() == 0) {
    ok = 1;
    volatile unsigned* vgen = &gb->gen;
    const unsigned g = *vgen;
    __threadfence();
    if (atomicAdd(&gb->count, 1u) == nblocks - 1u) {
      atomicExch(&gb->count, 0u);
      __threadfence();
      atomicAdd(&gb->gen, 1u);
    } else {
      const unsigned long long t0 = globaltimer_ns();
      while (*vgen == g) {
        if (globaltimer_ns() - t0 > limit_ns) {
          ok = 0;
          atomicExch(&g_vcycle_error, 2);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// Each pass body is called as a separate function, so the persistent kernel needs the
// registers of its largest body only, not of all of them inlined together.
template <typename C, int DIM, int J>
__device__ __noinline__ void seq_arnoldi(const PassDesc d, const LevelDev<C>* levs, int v) {
  if constexpr (DIM == 2) arnoldi_t2_body<C, J, false>(levs, d.ntiles, d.geo, d.f0, d.f1, v);
  else arnoldi_t3_body<C, J, false>(levs, d.ntiles, d.geo, d.f0, d.f1, v);
}
template <typename C, int DIM>
__device__ __noinline__ void seq_restrict(const PassDesc d, const LevelDev<C>* levs, int v) {
  if constexpr (DIM == 2) restrict_t2_body<C, false>(levs, d.ntiles, d.geo, d.f0, d.f1, d.f2, v);
  else restrict_t3_body<C, false>(levs, d.ntiles, d.geo, d.f0, d.f1, d.f2, v);
}
template <typename C, int DIM>
__device__ __noinline__ void seq_prolong(const PassDesc d, const LevelDev<C>* levs, int v) {
  if constexpr (DIM == 2) prolong_t2_body<C, false>(levs, d.ntiles, d.geo, v);
  else prolong_t3_body<C, false>(levs, d.ntiles, d.geo, v);
}
template <typename C, int DIM>
__device__ __noinline__ void seq_update(const PassDesc d, const LevelDev<C>* levs, int v) {
  update_pass_body<C>(levs, d.ntiles, DIM, d.f0, d.f1, d.f2, d.f3, v);
}
template <typename C, int DIM>
__device__ __noinline__ void seq_prolong_flat(const PassDesc d, const LevelDev<C>* levs, int v) {
  prolong_flat_body<C, false>(levs, d.ntiles, DIM, v);
}

// flags: arnoldi f0 = R_0 is b, f1 = store p_J; restrict f0 = R_0 is b, f1 = x from zero,
// f2 = no smoothing; update f0 = mode, f1 = R_0 is b, f2 = x selection, f3 = x from zero
template <typename C, int DIM>
__device__ __forceinline__ void run_pass(const PassDesc& d, const LevelDev<C>* levs, int v) {
  switch (d.kind) {
    case PK_ARNOLDI:
      switch (d.J) {
        case 1: seq_arnoldi<C, DIM, 1>(d, levs, v); break;
        case 2: seq_arnoldi<C, DIM, 2>(d, levs, v); break;
        case 3: seq_arnoldi<C, DIM, 3>(d, levs, v); break;
        default: seq_arnoldi<C, DIM, 4>(d, levs, v); break;
      }
      break;
    case PK_RESTRICT: seq_restrict<C, DIM>(d, levs, v); break;
    case PK_PROLONG: seq_prolong<C, DIM>(d, levs, v); break;
    case PK_UPDATE: seq_update<C, DIM>(d, levs, v); break;
    default: seq_prolong_flat<C, DIM>(d, levs, v); break;
  }
}

// Launched with 32 x 8 threads, the shape of the tile passes (the flat passes index
// threads by their flat index).
template <typename C, int DIM>
__global__ void __launch_bounds__(256, sizeof(C) == 8 ? 2 : 1)
k_vcycle_seq(const __grid_constant__ PassSeq seq, GridBar* gb, unsigned long long limit_ns) {
  for (int q = 0; q < seq.npass; ++q) {
    const PassDesc& d = seq.p[q];
    const LevelDev<C>* levs = reinterpret_cast<const LevelDev<C>*>(d.levs);
    for (int v = blockIdx.x; v < d.nvblk; v += gridDim.x) {
      run_pass<C, DIM>(d, levs, v);
      __syncthreads();  // the next virtual block reuses the pass's shared memory
    }
    if (q + 1 < seq.npass && !grid_barrier(gb, gridDim.x, limit_ns)) return;
  }
}

}  // namespace helm
