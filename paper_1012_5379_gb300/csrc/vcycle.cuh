// V-cycle kernels of the GMRES(s)-smoothed multigrid for M^CSG (Sec. 3.1).
//
// Every grid-level kernel is a marching stencil over the padded layout:
//   2D: a warp owns 32 consecutive x and marches `rows` rows in y; x-neighbours come
//       from warp shuffles (edge lanes load their outside neighbour), y-neighbours
//       from a three-deep register queue.
//   3D: a CTA owns 32 x 8 (x, y) columns plus two halo rows and marches `rows` planes
//       in z; x-neighbours from shuffles, y-neighbours through a double-buffered
//       shared-memory plane, z-neighbours from a register queue.
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
  return L.phi ? (R)__ldg(L.phi + pidx(x, y, z, L.P)) : (R)L.phic;
}

// ------------------------------------------------------------------ prolongation
// Vertex-centred bi/trilinear interpolation of the coarser output at fine node i:
// odd i -> coarse (i-1)/2 with weight 1; even i -> coarse i/2-1 and i/2 with 1/2.
template <typename C, bool NC = true>
__device__ __forceinline__ C interp(const LevelDev<C>& L, int x, int y, int z, int dim) {
  typedef typename CT<C>::R R;
  C acc = czero<C>();
  if (!inside(x, y, z, L.n)) return acc;
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
      for (int a = 0; a < nx; ++a) acc = cadd(acc, ldc<C, NC>(L.xcb, ix[a], iy[b], iz[c], L.nc, L.Pc));
  return cscale(acc, w);
}

// ------------------------------------------------------------------ pass J (2D)
template <typename C, int J>
__global__ void __launch_bounds__(32 * WARPS2)
k_arnoldi2(const LevelDev<C>* __restrict__ levs, int ntiles, int rows, int r0_is_b, int store_p) {
  typedef typename CT<C>::R R;
  __shared__ double sm[32 * (2 * J + 1)];
  const int prob = blockIdx.x / ntiles, tile = blockIdx.x - prob * ntiles;
  const LevelDev<C>& L = levs[prob];
  SweepScalars* sc = L.sc;
  if (sc->m < J) return;  // earlier breakdown or empty sweep: uniform for the problem
  const int n = L.n, P = L.P;
  const int ntx = ceil_div(P, 32);
  const int tx = tile % ntx, ty = tile / ntx;
  const int lane = threadIdx.x, warp = threadIdx.y;
  const int x = tx * 32 + lane;
  const int ybeg = (ty * WARPS2 + warp) * rows;
  const int yend = min(ybeg + rows, P);

  const C* Rk[J];
  C cf[J];
#pragma unroll
  for (int k = 0; k < J; ++k) {
    Rk[k] = (k == 0) ? (r0_is_b ? L.b : L.r0) : L.p[k - 1];
    cf[k] = from_d<C>(sc->Cf[J][k]);
  }
  const Coef3<C> cx = ldcoef(L, x);
  auto form = [&](int xx, int yy, C* raw) -> C {
    C v = czero<C>();
#pragma unroll
    for (int k = 0; k < J; ++k) {
      C r = ldc(Rk[k], xx, yy, 0, n, P);
      if (raw) raw[k] = r;
      v = cfma(cf[k], r, v);
    }
    return v;
  };

  C acc[J];
#pragma unroll
  for (int k = 0; k < J; ++k) acc[k] = czero<C>();
  R accn = 0;
  if (ybeg < P) {
    C raw0[J], rawn[J];
    C vm = form(x, ybeg - 1, nullptr);
    C v0 = form(x, ybeg, raw0);
    for (int y = ybeg; y < yend; ++y) {
      C vp = form(x, y + 1, rawn);
      C vl = shfl_up_c(v0, 1), vr = shfl_down_c(v0, 1);
      if (lane == 0) vl = form(x - 1, y, nullptr);
      if (lane == 31) vr = form(x + 1, y, nullptr);
      C p = czero<C>();
      if (x < n && y < n) {
        const Coef3<C> cy = ldcoef(L, y);
        C diag = cadd(cx.d, cy.d);
        diag.x -= phi_at(L, x, y, 0);
        p = cmul(diag, v0);
        p = cfma(cx.a, vl, p);
        p = cfma(cx.c, vr, p);
        p = cfma(cy.a, vm, p);
        p = cfma(cy.c, vp, p);
#pragma unroll
        for (int k = 0; k < J; ++k) acc[k] = cdotacc(raw0[k], p, acc[k]);
        accn += cabs2(p);
      }
      if (store_p && x < P) L.p[J - 1][pidx(x, y, 0, P)] = p;
      vm = v0;
      v0 = vp;
#pragma unroll
      for (int k = 0; k < J; ++k) raw0[k] = rawn[k];
    }
  }
  double red[2 * J + 1], tot[2 * J + 1];
#pragma unroll
  for (int k = 0; k < J; ++k) { red[2 * k] = acc[k].x; red[2 * k + 1] = acc[k].y; }
  red[2 * J] = accn;
  if (grid_sum_last<2 * J + 1>(red, L.part, tile, ntiles, &sc->counter, sm, tot)) {
    if (flat_tid() == 0) sweep_after_pass(sc, J, tot, SweepTau<C>::v);
  }
}

// ------------------------------------------------------------------ pass J (3D)
template <typename C, int J>
__global__ void __launch_bounds__(32 * (WY3 + 2))
k_arnoldi3(const LevelDev<C>* __restrict__ levs, int ntiles, int rows, int r0_is_b, int store_p) {
  typedef typename CT<C>::R R;
  __shared__ double sm[32 * (2 * J + 1)];
  __shared__ C sv[2][WY3 + 2][32];
  const int prob = blockIdx.x / ntiles, tile = blockIdx.x - prob * ntiles;
  const LevelDev<C>& L = levs[prob];
  SweepScalars* sc = L.sc;
  if (sc->m < J) return;
  const int n = L.n, P = L.P;
  const int ntx = ceil_div(P, 32), nty = ceil_div(P, WY3);
  const int tx = tile % ntx, ty = (tile / ntx) % nty, tz = tile / (ntx * nty);
  const int lane = threadIdx.x, w = threadIdx.y;
  const bool owned = (w >= 1 && w <= WY3);
  const int x = tx * 32 + lane;
  const int y = ty * WY3 - 1 + w;
  const int zbeg = tz * rows;
  const int zend = min(zbeg + rows, P);

  const C* Rk[J];
  C cf[J];
#pragma unroll
  for (int k = 0; k < J; ++k) {
    Rk[k] = (k == 0) ? (r0_is_b ? L.b : L.r0) : L.p[k - 1];
    cf[k] = from_d<C>(sc->Cf[J][k]);
  }
  const Coef3<C> cx = ldcoef(L, x), cy = ldcoef(L, y);
  auto form = [&](int xx, int yy, int zz, C* raw) -> C {
    C v = czero<C>();
#pragma unroll
    for (int k = 0; k < J; ++k) {
      C r = ldc(Rk[k], xx, yy, zz, n, P);
      if (raw) raw[k] = r;
      v = cfma(cf[k], r, v);
    }
    return v;
  };

  C acc[J];
#pragma unroll
  for (int k = 0; k < J; ++k) acc[k] = czero<C>();
  R accn = 0;
  if (zbeg < P) {
    C raw0[J], rawn[J];
    C vm = form(x, y, zbeg - 1, nullptr);
    C v0 = form(x, y, zbeg, raw0);
    for (int z = zbeg; z < zend; ++z) {
      C vp = form(x, y, z + 1, rawn);
      sv[z & 1][w][lane] = v0;
      __syncthreads();
      if (owned) {
        C vs = sv[z & 1][w - 1][lane], vn = sv[z & 1][w + 1][lane];
        C vl = shfl_up_c(v0, 1), vr = shfl_down_c(v0, 1);
        if (lane == 0) vl = form(x - 1, y, z, nullptr);
        if (lane == 31) vr = form(x + 1, y, z, nullptr);
        C p = czero<C>();
        if (x < n && y < n && z < n) {
          const Coef3<C> cz = ldcoef(L, z);
          C diag = cadd(cadd(cx.d, cy.d), cz.d);
          diag.x -= phi_at(L, x, y, z);
          p = cmul(diag, v0);
          p = cfma(cx.a, vl, p);
          p = cfma(cx.c, vr, p);
          p = cfma(cy.a, vs, p);
          p = cfma(cy.c, vn, p);
          p = cfma(cz.a, vm, p);
          p = cfma(cz.c, vp, p);
#pragma unroll
          for (int k = 0; k < J; ++k) acc[k] = cdotacc(raw0[k], p, acc[k]);
          accn += cabs2(p);
        }
        if (store_p && x < P && y < P) L.p[J - 1][pidx(x, y, z, P)] = p;
      }
      vm = v0;
      v0 = vp;
#pragma unroll
      for (int k = 0; k < J; ++k) raw0[k] = rawn[k];
    }
  }
  double red[2 * J + 1], tot[2 * J + 1];
#pragma unroll
  for (int k = 0; k < J; ++k) { red[2 * k] = acc[k].x; red[2 * k + 1] = acc[k].y; }
  red[2 * J] = accn;
  if (grid_sum_last<2 * J + 1>(red, L.part, tile, ntiles, &sc->counter, sm, tot)) {
    if (flat_tid() == 0) sweep_after_pass(sc, J, tot, SweepTau<C>::v);
  }
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
  const SweepScalars* sc = L.sc;
  u.m = sc->m;
#pragma unroll
  for (int k = 0; k <= SMAX; ++k) {
    u.xc[k] = from_d<C>(sc->xcoef[k]);
    u.rc[k] = from_d<C>(sc->rcoef[k]);
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
// residual mode, r0 <- r (in place) with ||r||^2 starting the next sweep.
template <typename C>
__global__ void __launch_bounds__(256)
k_update_flat(const LevelDev<C>* __restrict__ levs, int ntiles, int dim, int mode, int r0_is_b, int xsel,
              int x_from_zero) {
  __shared__ double sm[32];
  const int prob = blockIdx.x / ntiles, tile = blockIdx.x - prob * ntiles;
  const LevelDev<C>& L = levs[prob];
  const int n = L.n, P = L.P;
  const UpdCoef<C> u = load_upd(L, r0_is_b);
  C* xo = xsel ? L.xb : L.xa;
  const size_t npts = dim == 3 ? (size_t)P * P * P : (size_t)P * P;
  const bool want_r = (mode == UPD_RESIDUAL);
  typename CT<C>::R acc = 0;
  for (size_t i = (size_t)tile * blockDim.x + threadIdx.x; i < npts; i += (size_t)ntiles * blockDim.x) {
    const int x = (int)(i % P);
    const int y = (int)((i / P) % P);
    const int z = dim == 3 ? (int)(i / ((size_t)P * P)) : 0;
    C dx, r;
    upd_point<C, false>(u, x, y, z, n, P, dx, r, want_r);
    C xv = x_from_zero ? czero<C>() : xo[i];
    xo[i] = cadd(xv, dx);
    if (want_r) {
      L.r0[i] = r;
      acc += cabs2(r);
    }
  }
  if (!want_r) return;
  double red[1] = {(double)acc}, tot[1];
  if (grid_sum_last<1>(red, L.part, tile, ntiles, &L.sc->counter, sm, tot)) {
    if (flat_tid() == 0) sweep_begin(L.sc, tot[0], L.s);
  }
}

// Level-0 input: b <- src (natural layout, any precision), ||b||^2 starts the first
// sweep.
template <typename Cin, typename C>
__global__ void __launch_bounds__(256)
k_load_input(const LevelDev<C>* __restrict__ levs, int ntiles, int dim, const Cin* __restrict__ src) {
  __shared__ double sm[32];
  const int prob = blockIdx.x / ntiles, tile = blockIdx.x - prob * ntiles;
  const LevelDev<C>& L = levs[prob];
  const int n = L.n, P = L.P;
  const size_t npts = dim == 3 ? (size_t)P * P * P : (size_t)P * P;
  typename CT<C>::R acc = 0;
  for (size_t i = (size_t)tile * blockDim.x + threadIdx.x; i < npts; i += (size_t)ntiles * blockDim.x) {
    const int x = (int)(i % P);
    const int y = (int)((i / P) % P);
    const int z = dim == 3 ? (int)(i / ((size_t)P * P)) : 0;
    C v = czero<C>();
    if (inside(x, y, z, n)) v = from_d<C>(to_d(src[((size_t)z * n + y) * n + x]));
    L.b[i] = v;
    acc += cabs2(v);
  }
  double red[1] = {(double)acc}, tot[1];
  if (grid_sum_last<1>(red, L.part, tile, ntiles, &L.sc->counter, sm, tot)) {
    if (flat_tid() == 0) sweep_begin(L.sc, tot[0], L.s);
  }
}

// Level-0 output: dst (natural layout, any precision) <- xb.
template <typename C, typename Cout>
__global__ void __launch_bounds__(256)
k_store_output(const LevelDev<C>* __restrict__ levs, int dim, Cout* __restrict__ dst) {
  const LevelDev<C>& L = levs[0];
  const int n = L.n, P = L.P;
  const size_t npts = dim == 3 ? (size_t)n * n * n : (size_t)n * n;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < npts; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % n);
    const int y = (int)((i / n) % n);
    const int z = dim == 3 ? (int)(i / ((size_t)n * n)) : 0;
    dst[i] = from_d<Cout>(to_d(L.xb[pidx(x, y, z, P)]));
  }
}

// End of pre-smoothing, fused with full-weighting restriction (2D): x_a = x + dx,
// r = R_0 - sum y_j p_j, b_c = FW(r) on the coarser grid, ||b_c||^2 starts the
// coarse level's first sweep.  A warp covers 32 fine x (16 coarse) and an even run
// of fine rows plus one halo row above.
template <typename C>
__global__ void __launch_bounds__(32 * WARPS2)
k_restrict2(const LevelDev<C>* __restrict__ levs, int ntiles, int rows, int r0_is_b, int x_from_zero,
            int nosmooth) {
  typedef typename CT<C>::R R;
  __shared__ double sm[32];
  const int prob = blockIdx.x / ntiles, tile = blockIdx.x - prob * ntiles;
  const LevelDev<C>& L = levs[prob];
  const int n = L.n, P = L.P, nc = L.nc, Pc = L.Pc;
  const int ntx = ceil_div(P, 32);
  const int tx = tile % ntx, ty = tile / ntx;
  const int lane = threadIdx.x, warp = threadIdx.y;
  const int x = tx * 32 + lane;
  const int ybeg = (ty * WARPS2 + warp) * rows;
  const int yend = min(ybeg + rows, P);
  UpdCoef<C> u = load_upd(L, r0_is_b);
  if (nosmooth) { u.m = 0; u.rc[0] = CT<C>::make(1, 0); }
  R acc = 0;
  if (ybeg < P) {
    C cacc = czero<C>();
    for (int y = ybeg; y <= yend; ++y) {
      C dx, r;
      upd_point(u, x, y, 0, n, P, dx, r);
      if (y < yend && x < P) {
        C xv = x_from_zero ? czero<C>() : L.xa[pidx(x, y, 0, P)];
        L.xa[pidx(x, y, 0, P)] = (x < n && y < n) ? cadd(xv, dx) : czero<C>();
      }
      C rl = shfl_up_c(r, 1), rr = shfl_down_c(r, 1);
      if (lane == 31) {
        C d2;
        upd_point(u, x + 1, y, 0, n, P, d2, rr);
      }
      // horizontal full weighting at odd x
      C rh = cadd(cscale(r, (R)0.5), cscale(cadd(rl, rr), (R)0.25));
      if ((y & 1) == 0) {
        if (y > ybeg) {
          cacc = cadd(cacc, cscale(rh, (R)0.25));
          const int I = (y >> 1) - 1, Ix = x >> 1;
          if ((x & 1) && Ix < Pc) {
            const bool valid = (Ix < nc && I < nc);
            C out = valid ? cacc : czero<C>();
            L.bc[pidx(Ix, I, 0, Pc)] = out;
            if (valid) acc += cabs2(out);
          }
        }
        cacc = cscale(rh, (R)0.25);
      } else {
        cacc = cadd(cacc, cscale(rh, (R)0.5));
      }
    }
  }
  double red[1] = {(double)acc}, tot[1];
  if (grid_sum_last<1>(red, L.part, tile, ntiles, &L.sc->counter, sm, tot)) {
    if (flat_tid() == 0) sweep_begin(L.scc, tot[0], L.s);
  }
}

// 3D version: the CTA's warps 1..WY3+1 cover fine rows y0..y0+WY3 (one halo row);
// horizontal weighting by shuffles, y-weighting through shared memory, z-weighting
// in registers along the march (planes zbeg..zend, the last one a halo).
template <typename C>
__global__ void __launch_bounds__(32 * (WY3 + 2))
k_restrict3(const LevelDev<C>* __restrict__ levs, int ntiles, int rows, int r0_is_b, int x_from_zero,
            int nosmooth) {
  typedef typename CT<C>::R R;
  __shared__ double sm[32];
  __shared__ C srh[2][WY3 + 2][32];
  const int prob = blockIdx.x / ntiles, tile = blockIdx.x - prob * ntiles;
  const LevelDev<C>& L = levs[prob];
  const int n = L.n, P = L.P, nc = L.nc, Pc = L.Pc;
  const int ntx = ceil_div(P, 32), nty = ceil_div(P, WY3);
  const int tx = tile % ntx, ty = (tile / ntx) % nty, tz = tile / (ntx * nty);
  const int lane = threadIdx.x, w = threadIdx.y;
  const bool owned = (w >= 1 && w <= WY3);
  const int x = tx * 32 + lane;
  const int y = ty * WY3 - 1 + w;
  const int zbeg = tz * rows;
  const int zend = min(zbeg + rows, P);
  UpdCoef<C> u = load_upd(L, r0_is_b);
  if (nosmooth) { u.m = 0; u.rc[0] = CT<C>::make(1, 0); }
  R acc = 0;
  if (zbeg < P) {
    C cacc = czero<C>();
    for (int z = zbeg; z <= zend; ++z) {
      C rh = czero<C>();
      if (w >= 1) {
        C dx, r;
        upd_point(u, x, y, z, n, P, dx, r);
        if (owned && z < zend && x < P && y < P) {
          const size_t id = pidx(x, y, z, P);
          C xv = x_from_zero ? czero<C>() : L.xa[id];
          L.xa[id] = inside(x, y, z, n) ? cadd(xv, dx) : czero<C>();
        }
        C rl = shfl_up_c(r, 1), rr = shfl_down_c(r, 1);
        if (lane == 31) {
          C d2;
          upd_point(u, x + 1, y, z, n, P, d2, rr);
        }
        rh = cadd(cscale(r, (R)0.5), cscale(cadd(rl, rr), (R)0.25));
      }
      srh[z & 1][w][lane] = rh;
      __syncthreads();
      // rows y odd (w even, y0 even) own a coarse row
      if (owned && (y & 1)) {
        C ry = cadd(cscale(rh, (R)0.5), cscale(cadd(srh[z & 1][w - 1][lane], srh[z & 1][w + 1][lane]), (R)0.25));
        if ((z & 1) == 0) {
          if (z > zbeg) {
            cacc = cadd(cacc, cscale(ry, (R)0.25));
            const int Iz = (z >> 1) - 1, Iy = y >> 1, Ix = x >> 1;
            if ((x & 1) && Ix < Pc && Iy < Pc) {
              const bool valid = (Ix < nc && Iy < nc && Iz < nc);
              C out = valid ? cacc : czero<C>();
              L.bc[pidx(Ix, Iy, Iz, Pc)] = out;
              if (valid) acc += cabs2(out);
            }
          }
          cacc = cscale(ry, (R)0.25);
        } else {
          cacc = cadd(cacc, cscale(ry, (R)0.5));
        }
      }
    }
  }
  double red[1] = {(double)acc}, tot[1];
  if (grid_sum_last<1>(red, L.part, tile, ntiles, &L.sc->counter, sm, tot)) {
    if (flat_tid() == 0) sweep_begin(L.scc, tot[0], L.s);
  }
}

// ------------------------------------------------------------------ coarse correction
// x_b = x_a + P e_c and r0 = b - M x_b (2D), ||r0||^2 starts post-smoothing.
template <typename C>
__global__ void __launch_bounds__(32 * WARPS2)
k_prolong2(const LevelDev<C>* __restrict__ levs, int ntiles, int rows) {
  typedef typename CT<C>::R R;
  __shared__ double sm[32];
  const int prob = blockIdx.x / ntiles, tile = blockIdx.x - prob * ntiles;
  const LevelDev<C>& L = levs[prob];
  const int n = L.n, P = L.P;
  const int ntx = ceil_div(P, 32);
  const int tx = tile % ntx, ty = tile / ntx;
  const int lane = threadIdx.x, warp = threadIdx.y;
  const int x = tx * 32 + lane;
  const int ybeg = (ty * WARPS2 + warp) * rows;
  const int yend = min(ybeg + rows, P);
  const Coef3<C> cx = ldcoef(L, x);
  auto form = [&](int xx, int yy) -> C {
    return cadd(ldc((const C*)L.xa, xx, yy, 0, n, P), interp(L, xx, yy, 0, 2));
  };
  R acc = 0;
  if (ybeg < P) {
    C vm = form(x, ybeg - 1), v0 = form(x, ybeg);
    for (int y = ybeg; y < yend; ++y) {
      C vp = form(x, y + 1);
      C vl = shfl_up_c(v0, 1), vr = shfl_down_c(v0, 1);
      if (lane == 0) vl = form(x - 1, y);
      if (lane == 31) vr = form(x + 1, y);
      if (x < P) {
        C r = czero<C>(), xo = czero<C>();
        if (x < n && y < n) {
          const Coef3<C> cy = ldcoef(L, y);
          C diag = cadd(cx.d, cy.d);
          diag.x -= phi_at(L, x, y, 0);
          C p = cmul(diag, v0);
          p = cfma(cx.a, vl, p);
          p = cfma(cx.c, vr, p);
          p = cfma(cy.a, vm, p);
          p = cfma(cy.c, vp, p);
          r = csub(__ldg(L.b + pidx(x, y, 0, P)), p);
          xo = v0;
          acc += cabs2(r);
        }
        L.xb[pidx(x, y, 0, P)] = xo;
        L.r0[pidx(x, y, 0, P)] = r;
      }
      vm = v0;
      v0 = vp;
    }
  }
  double red[1] = {(double)acc}, tot[1];
  if (grid_sum_last<1>(red, L.part, tile, ntiles, &L.sc->counter, sm, tot)) {
    if (flat_tid() == 0) sweep_begin(L.sc, tot[0], L.s);
  }
}

template <typename C>
__global__ void __launch_bounds__(32 * (WY3 + 2))
k_prolong3(const LevelDev<C>* __restrict__ levs, int ntiles, int rows) {
  typedef typename CT<C>::R R;
  __shared__ double sm[32];
  __shared__ C sv[2][WY3 + 2][32];
  const int prob = blockIdx.x / ntiles, tile = blockIdx.x - prob * ntiles;
  const LevelDev<C>& L = levs[prob];
  const int n = L.n, P = L.P;
  const int ntx = ceil_div(P, 32), nty = ceil_div(P, WY3);
  const int tx = tile % ntx, ty = (tile / ntx) % nty, tz = tile / (ntx * nty);
  const int lane = threadIdx.x, w = threadIdx.y;
  const bool owned = (w >= 1 && w <= WY3);
  const int x = tx * 32 + lane;
  const int y = ty * WY3 - 1 + w;
  const int zbeg = tz * rows;
  const int zend = min(zbeg + rows, P);
  const Coef3<C> cx = ldcoef(L, x), cy = ldcoef(L, y);
  auto form = [&](int xx, int yy, int zz) -> C {
    return cadd(ldc((const C*)L.xa, xx, yy, zz, n, P), interp(L, xx, yy, zz, 3));
  };
  R acc = 0;
  if (zbeg < P) {
    C vm = form(x, y, zbeg - 1), v0 = form(x, y, zbeg);
    for (int z = zbeg; z < zend; ++z) {
      C vp = form(x, y, z + 1);
      sv[z & 1][w][lane] = v0;
      __syncthreads();
      if (owned) {
        C vs = sv[z & 1][w - 1][lane], vn = sv[z & 1][w + 1][lane];
        C vl = shfl_up_c(v0, 1), vr = shfl_down_c(v0, 1);
        if (lane == 0) vl = form(x - 1, y, z);
        if (lane == 31) vr = form(x + 1, y, z);
        if (x < P && y < P) {
          C r = czero<C>(), xo = czero<C>();
          if (inside(x, y, z, n)) {
            const Coef3<C> cz = ldcoef(L, z);
            C diag = cadd(cadd(cx.d, cy.d), cz.d);
            diag.x -= phi_at(L, x, y, z);
            C p = cmul(diag, v0);
            p = cfma(cx.a, vl, p);
            p = cfma(cx.c, vr, p);
            p = cfma(cy.a, vs, p);
            p = cfma(cy.c, vn, p);
            p = cfma(cz.a, vm, p);
            p = cfma(cz.c, vp, p);
            r = csub(__ldg(L.b + pidx(x, y, z, P)), p);
            xo = v0;
            acc += cabs2(r);
          }
          L.xb[pidx(x, y, z, P)] = xo;
          L.r0[pidx(x, y, z, P)] = r;
        }
      }
      vm = v0;
      v0 = vp;
    }
  }
  double red[1] = {(double)acc}, tot[1];
  if (grid_sum_last<1>(red, L.part, tile, ntiles, &L.sc->counter, sm, tot)) {
    if (flat_tid() == 0) sweep_begin(L.sc, tot[0], L.s);
  }
}

// Coarse correction without post-smoothing (nu2 = 0): x_b = x_a + P e_c, pointwise.
template <typename C>
__global__ void __launch_bounds__(256)
k_prolong_flat(const LevelDev<C>* __restrict__ levs, int ntiles, int dim) {
  const int prob = blockIdx.x / ntiles, tile = blockIdx.x - prob * ntiles;
  const LevelDev<C>& L = levs[prob];
  const int n = L.n, P = L.P;
  const size_t npts = dim == 3 ? (size_t)P * P * P : (size_t)P * P;
  for (size_t i = (size_t)tile * blockDim.x + threadIdx.x; i < npts; i += (size_t)ntiles * blockDim.x) {
    const int x = (int)(i % P), y = (int)((i / P) % P), z = dim == 3 ? (int)(i / ((size_t)P * P)) : 0;
    C v = czero<C>();
    if (inside(x, y, z, n)) v = cadd(L.xa[i], interp(L, x, y, z, dim));
    L.xb[i] = v;
  }
}

// ------------------------------------------------------------------ coarse levels
// One CTA per problem runs the whole sub-cycle of the coarse levels (sizes where a
// grid-wide launch is all latency): every pass is a block-wide loop with
// __syncthreads and fixed-order block reductions; the coarsest level is a dense FP64
// LU solve by one warp.
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

template <typename C>
__device__ __forceinline__ void cblock_coords(size_t i, int P, int dim, int& x, int& y, int& z) {
  x = (int)(i % P);
  y = (int)((i / P) % P);
  z = dim == 3 ? (int)(i / ((size_t)P * P)) : 0;
}

// One GMRES(s) sweep on level L in a single CTA.  R_0 is b (r0_is_b) or r0; x is
// updated in place in xo (or written from zero).  `tmp` holds v_J.  At the end, in
// residual mode r0 <- r_new and the next sweep starts; in restrict mode the residual
// is left in `tmp` for the caller.
template <typename C>
__device__ void cblock_sweep(const LevelDev<C>& L, int dim, int r0_is_b, C* xo, int x_from_zero, C* tmp,
                             int end_mode, double* sm) {
  typedef typename CT<C>::R R;
  SweepScalars* sc = L.sc;
  const int P = L.P, n = L.n;
  const size_t npts = dim == 3 ? (size_t)P * P * P : (size_t)P * P;
  const int tid = flat_tid(), nth = block_threads();
  const C* R0 = r0_is_b ? L.b : L.r0;
  for (int J = 1; J <= SMAX; ++J) {
    __syncthreads();
    if (sc->m < J) break;
    // v_J = sum_k Cf[J][k] R_k
    for (size_t i = tid; i < npts; i += nth) {
      C v = czero<C>();
      for (int k = 0; k < J; ++k) {
        const C* Rk = k == 0 ? R0 : L.p[k - 1];
        v = cfma(from_d<C>(sc->Cf[J][k]), Rk[i], v);
      }
      tmp[i] = v;
    }
    __syncthreads();
    double red[2 * SMAX + 1];
    for (int q = 0; q < 2 * SMAX + 1; ++q) red[q] = 0.0;
    C acc[SMAX];
    for (int k = 0; k < SMAX; ++k) acc[k] = czero<C>();
    R accn = 0;
    for (size_t i = tid; i < npts; i += nth) {
      int x, y, z;
      cblock_coords<C>(i, P, dim, x, y, z);
      C p = czero<C>();
      if (inside(x, y, z, n)) {
        cblock_stencil_apply(L, tmp, x, y, z, dim, p);
        for (int k = 0; k < J; ++k) acc[k] = cdotacc((k == 0 ? R0 : L.p[k - 1])[i], p, acc[k]);
        accn += cabs2(p);
      }
      L.p[J - 1][i] = p;
    }
    for (int k = 0; k < J; ++k) { red[2 * k] = acc[k].x; red[2 * k + 1] = acc[k].y; }
    red[2 * J] = accn;
    block_sum<2 * SMAX + 1>(red, sm);
    if (tid == 0) {
      double tot[2 * SMAX + 1];
      for (int q = 0; q < 2 * SMAX + 1; ++q) tot[q] = red[q];
      sweep_after_pass(sc, J, tot, SweepTau<C>::v);
    }
  }
  __syncthreads();
  const int m = sc->m;
  C xc[SMAX + 1], rc[SMAX + 1];
  for (int k = 0; k <= SMAX; ++k) { xc[k] = from_d<C>(sc->xcoef[k]); rc[k] = from_d<C>(sc->rcoef[k]); }
  __syncthreads();
  R accr = 0;
  for (size_t i = tid; i < npts; i += nth) {
    C dx = czero<C>(), r = czero<C>();
    for (int k = 0; k <= m; ++k) {
      C v = (k == 0 ? R0 : L.p[k - 1])[i];
      if (k < m) dx = cfma(xc[k], v, dx);
      r = cfma(rc[k], v, r);
    }
    xo[i] = cadd(x_from_zero ? czero<C>() : xo[i], dx);
    if (end_mode == UPD_RESIDUAL) { L.r0[i] = r; accr += cabs2(r); }
    if (end_mode == UPD_RESTRICT) tmp[i] = r;
  }
  if (end_mode == UPD_RESIDUAL) {
    double red[1] = {(double)accr};
    block_sum<1>(red, sm);
    if (tid == 0) sweep_begin(sc, red[0], L.s);
  }
  __syncthreads();
}

template <typename C>
__global__ void __launch_bounds__(1024)
k_coarse(const LevelDev<C>* __restrict__ levs_all, int nlev, int lev_stride, const CoarseLU* __restrict__ lus,
         int nu1, int nu2, int dim) {
  typedef typename CT<C>::R R;
  __shared__ double sm[32 * (2 * SMAX + 1)];
  const int prob = blockIdx.x;
  const LevelDev<C>* Ls = levs_all + (size_t)prob * lev_stride;
  const int tid = flat_tid(), nth = block_threads();
  // descent
  for (int l = 0; l < nlev - 1; ++l) {
    const LevelDev<C>& L = Ls[l];
    const int P = L.P;
    const size_t npts = dim == 3 ? (size_t)P * P * P : (size_t)P * P;
    if (nu1 == 0) {
      for (size_t i = tid; i < npts; i += nth) { L.xa[i] = czero<C>(); L.xb[i] = L.b[i]; }
    } else {
      for (int sw = 0; sw < nu1; ++sw)
        cblock_sweep(L, dim, sw == 0, L.xa, sw == 0, L.xb, sw == nu1 - 1 ? UPD_RESTRICT : UPD_RESIDUAL, sm);
    }
    __syncthreads();
    // b_c = FW(r) with r in xb
    const int Pc = L.Pc, nc = L.nc;
    const size_t ncpts = dim == 3 ? (size_t)Pc * Pc * Pc : (size_t)Pc * Pc;
    R acc = 0;
    for (size_t i = tid; i < ncpts; i += nth) {
      int X, Y, Z;
      cblock_coords<C>(i, Pc, dim, X, Y, Z);
      C out = czero<C>();
      if (inside(X, Y, Z, nc)) {
        const int fx = 2 * X + 1, fy = 2 * Y + 1, fz = dim == 3 ? 2 * Z + 1 : 0;
        const int dz0 = dim == 3 ? -1 : 0, dz1 = dim == 3 ? 1 : 0;
        for (int dz = dz0; dz <= dz1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              R wgt = (R)((dx == 0 ? 0.5 : 0.25) * (dy == 0 ? 0.5 : 0.25) * (dim == 3 ? (dz == 0 ? 0.5 : 0.25) : 1.0));
              out = cadd(out, cscale(ldc<C, false>((const C*)L.xb, fx + dx, fy + dy, fz + dz, L.n, P), wgt));
            }
        acc += cabs2(out);
      }
      L.bc[i] = out;
    }
    double red[1] = {(double)acc};
    block_sum<1>(red, sm);
    if (tid == 0) sweep_begin(L.scc, red[0], L.s);
    __syncthreads();
  }
  // coarsest: dense LU solve in FP64 by warp 0
  {
    const LevelDev<C>& L = Ls[nlev - 1];
    const CoarseLU& lu = lus[prob];
    const int m = lu.m, P = L.P, n = L.n;
    double2* yv = reinterpret_cast<double2*>(sm);  // m <= 64 complex values
    if (tid < 32) {
      for (int i = tid; i < m; i += 32) {
        const int src = lu.piv[i];
        int sx = src % n, sy = (src / n) % n, sz = dim == 3 ? src / (n * n) : 0;
        yv[i] = to_d(L.b[pidx(sx, sy, sz, P)]);
      }
      __syncwarp();
      for (int k = 0; k < m; ++k) {  // forward, unit lower
        const double2 yk = yv[k];
        __syncwarp();
        for (int i = k + 1 + tid; i < m; i += 32) yv[i] = csub(yv[i], cmul(lu.lu[(size_t)i * m + k], yk));
        __syncwarp();
      }
      for (int k = m - 1; k >= 0; --k) {  // backward
        if (tid == 0) yv[k] = ddiv(yv[k], lu.lu[(size_t)k * m + k]);
        __syncwarp();
        const double2 yk = yv[k];
        for (int i = tid; i < k; i += 32) yv[i] = csub(yv[i], cmul(lu.lu[(size_t)i * m + k], yk));
        __syncwarp();
      }
    }
    __syncthreads();
    const size_t npts = dim == 3 ? (size_t)P * P * P : (size_t)P * P;
    for (size_t i = tid; i < npts; i += nth) {
      int x, y, z;
      cblock_coords<C>(i, P, dim, x, y, z);
      C v = czero<C>();
      if (inside(x, y, z, n)) v = from_d<C>(yv[(z * n + y) * n + x]);
      L.xb[i] = v;
    }
    __syncthreads();
  }
  // ascent
  for (int l = nlev - 2; l >= 0; --l) {
    const LevelDev<C>& L = Ls[l];
    const int P = L.P, n = L.n;
    const size_t npts = dim == 3 ? (size_t)P * P * P : (size_t)P * P;
    for (size_t i = tid; i < npts; i += nth) {
      int x, y, z;
      cblock_coords<C>(i, P, dim, x, y, z);
      L.xb[i] = inside(x, y, z, n) ? cadd(L.xa[i], interp<C, false>(L, x, y, z, dim)) : czero<C>();
    }
    __syncthreads();
    if (nu2 > 0) {
      R acc = 0;
      for (size_t i = tid; i < npts; i += nth) {
        int x, y, z;
        cblock_coords<C>(i, P, dim, x, y, z);
        C r = czero<C>();
        if (inside(x, y, z, n)) {
          C p;
          cblock_stencil_apply(L, (const C*)L.xb, x, y, z, dim, p);
          r = csub(L.b[i], p);
          acc += cabs2(r);
        }
        L.r0[i] = r;
      }
      double red[1] = {(double)acc};
      block_sum<1>(red, sm);
      if (tid == 0) sweep_begin(L.sc, red[0], L.s);
      __syncthreads();
      for (int sw = 0; sw < nu2; ++sw)
        cblock_sweep(L, dim, 0, L.xb, 0, L.xa, sw == nu2 - 1 ? UPD_XONLY : UPD_RESIDUAL, sm);
    }
  }
}

}  // namespace helm
