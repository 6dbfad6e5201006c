// Outer flexible GMRES in FP64 (Sec. 5: FGMRES [Saad 1993] on H u = b, right-
// preconditioned by one V-cycle on M^CSG; the preconditioned vectors z_j are stored
// because the GMRES-smoothed V-cycle is not a fixed linear operator).
//
// Per iteration j:  w = H z_j (FP64 stencil, z_j in the preconditioner precision)
//                   h_ij = <v_i, w>                      (one multi-dot pass)
//                   u = w - sum h_ij v_i, h_{j+1,j} = ||u|| (explicit, same pass)
//                   Givens update of the least-squares residual |g_{j+1}|
// u is stored unnormalised, v_{j+1} = u / h_{j+1,j} lives as u with a scale factor
// vscale[j+1] applied to every coefficient that touches it; u (in the
// preconditioner precision) is the next V-cycle input.  The explicit norm replaces
// sqrt(||w||^2 - sum |h|^2), whose cancellation made the basis lose orthogonality
// once the preconditioned operator is close to the identity.
// At a cycle end: y = R^{-1} g, x += Z y, true residual b - H x recomputed in FP64.
//
// Basis arithmetic (OuterState::df): binary64, or double-float (dfloat.cuh) for the
// basis V, for w = H z_j as the multi-dot and the update read it, and for their
// products and sums.  The double-float passes run on the FP32 pipe, which issues 64
// instructions where the FP64 pipe issues one; in binary64 the multi-dot and the update
// are bound by the FP64 pipe (4 FMA per point and vector against 16 bytes), in
// double-float by HBM.  With a complex64 preconditioner the stencil forms H z_j in
// double-float from the exact complex64 z_j, and x += Z y accumulates in double-float
// too; the Hessenberg column, the rotations, y, the stored x and Z and the true residual
// stay binary64.
#include <algorithm>

#include "device_common.cuh"
#include "dfloat.cuh"
#include "vcycle.cuh"

namespace helm {

template <typename C>
__device__ __forceinline__ double2 ldd(const C* p, int x, int y, int z, int n, int P) {
  return inside(x, y, z, n) ? to_d(__ldg(p + pidx(x, y, z, P))) : make_double2(0, 0);
}

struct HCoef { double2 a, d, c; };
__device__ __forceinline__ HCoef ldh(const double2* ca, const double2* cd, const double2* cc, int i, int n) {
  HCoef r;
  if ((unsigned)i < (unsigned)n) { r.a = __ldg(ca + i); r.d = __ldg(cd + i); r.c = __ldg(cc + i); }
  else { r.a = r.d = r.c = make_double2(0, 0); }
  return r;
}

// MODE 0: w = b - H x (true residual; also ||b||^2 on the first call)
// MODE 1: w = H z_j, with z_j read from the V-cycle output buffer and archived into Z[j]
template <typename C, int MODE>
__device__ __forceinline__ const C* stencil_src(const OuterDev<C>& O, const OuterState* st);
template <>
__device__ __forceinline__ const float2* stencil_src<float2, 0>(const OuterDev<float2>& O, const OuterState*) { return nullptr; }
template <>
__device__ __forceinline__ const double2* stencil_src<double2, 0>(const OuterDev<double2>& O, const OuterState*) { return nullptr; }
template <>
__device__ __forceinline__ const float2* stencil_src<float2, 1>(const OuterDev<float2>& O, const OuterState*) { return O.zout; }
template <>
__device__ __forceinline__ const double2* stencil_src<double2, 1>(const OuterDev<double2>& O, const OuterState*) { return O.zout; }

template <typename C, int MODE>
__device__ __forceinline__ void outer_stencil_epilogue(const OuterDev<C>& O, OuterState* st, const double* tot) {
  if (MODE == 0) {
    if (st->bnorm < 0.0) st->bnorm = sqrt(tot[1]);
    const double beta = sqrt(tot[0]);
    st->beta = beta;
    st->rel_true = st->bnorm > 0.0 ? beta / st->bnorm : 0.0;
    st->cycle_end = 0;
    st->need_residual = 0;
    st->j = 0;
    if (!isfinite(beta)) { st->done = 3; st->status = -4; }
    else if (st->bnorm == 0.0 || st->rel_true <= st->tol) { st->done = 1; st->status = 0; }
    else if (st->iters >= st->maxit) { st->done = 2; st->status = -3; }
    else {
      for (int i = 0; i <= st->m; ++i) O.g[i] = make_double2(0, 0);
      O.g[0] = make_double2(beta, 0);
      st->hnext = beta;  // v_0 = r / beta
      st->fresh = 1;
    }
  } else {
    st->wnorm2 = tot[0];
  }
}

// ---- w = H z_j in double-float (complex64 z_j, FP32 pipe)
// H's coefficients as double-floats (a, d, c blocks of n), zero outside 0..n-1.
__device__ __forceinline__ float4 ldh_df(const float4* cdf, int which, int i, int n) {
  return (unsigned)i < (unsigned)n ? __ldg(cdf + (size_t)which * n + i) : make_float4(0, 0, 0, 0);
}
__device__ __forceinline__ float2 ldz(const float2* p, int x, int y, int z, int n, int P) {
  return inside(x, y, z, n) ? __ldg(p + pidx(x, y, z, P)) : make_float2(0, 0);
}
__device__ __forceinline__ float2 shfl_f2(float2 v, int d, bool up) {
  return up ? make_float2(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d))
            : make_float2(__shfl_down_sync(0xffffffffu, v.x, d), __shfl_down_sync(0xffffffffu, v.y, d));
}
// One point: diag = d_x + d_y (+ d_z) - phi assembled in double-float, then the five or
// seven products summed with TwoSum; returns the double-float result and adds |w_p|^2
// to (ns, nc).  dxy holds d_x + d_y; the z terms enter only in 3D.
__device__ __forceinline__ float4 hpoint_df(float4 dxy, float4 dz, float phih, float phil, float4 ax, float4 cxr,
                                            float4 ay, float4 cyr, float4 az, float4 czr, float2 v0, float2 vl,
                                            float2 vr, float2 vs, float2 vn, float2 vm, float2 vp, bool three,
                                            float& ns, float& nc) {
  float4 dg = three ? df_cadd(dxy, dz) : dxy;
  const float2 dre = df_add(dg.x, dg.y, -phih, -phil);
  dg.x = dre.x;
  dg.y = dre.y;
  DfAcc a = df_cmul_first(dg, v0);
  df_cmac(a, ax, vl);
  df_cmac(a, cxr, vr);
  df_cmac(a, ay, vs);
  df_cmac(a, cyr, vn);
  if (three) {
    df_cmac(a, az, vm);
    df_cmac(a, czr, vp);
  }
  float hr, lr, hi, li;
  df_two_sum(a.sr, a.cr, hr, lr);
  df_two_sum(a.si, a.ci, hi, li);
  df_mac(ns, nc, hr, lr, hr, lr);
  df_mac(ns, nc, hi, li, hi, li);
  df_renorm(ns, nc);
  return make_float4(hr, lr, hi, li);
}

// 2D rows ybeg..yend-1 of one warp column; returns this thread's share of ||w||^2.  The
// next row's value, phi and the edge lanes' x neighbours are loaded one row ahead, as in
// the 3D pass.
__device__ double hstencil2_df(const OuterDev<float2>& O, const float2* u1, float2* zarch, int x, int ybeg,
                               int yend, int lane) {
  const int n = O.n, P = O.P;
  const float4 ax = ldh_df(O.cdf, 0, x, n), dx = ldh_df(O.cdf, 1, x, n), cxr = ldh_df(O.cdf, 2, x, n);
  const float2 pc = df_split(O.phic);
  const float4 zero = make_float4(0, 0, 0, 0);
  const bool edge = lane == 0 || lane == 31;
  const int xe = lane == 0 ? x - 1 : x + 1;  // the edge lane's neighbour outside the warp
  auto ldphi = [&](int y) -> float {
    return O.phi ? (x < n && y < n ? __ldg(O.phi + pidx(x, y, 0, P)) : 0.0f) : pc.x;
  };
  float ns = 0.0f, nc = 0.0f;
  if (ybeg < P) {
    float2 vm = ldz(u1, x, ybeg - 1, 0, n, P), v0 = ldz(u1, x, ybeg, 0, n, P);
    float ph0 = ldphi(ybeg);
    float2 e0 = edge ? ldz(u1, xe, ybeg, 0, n, P) : make_float2(0, 0);
    for (int y = ybeg; y < yend; ++y) {
      const float2 vp = ldz(u1, x, y + 1, 0, n, P);
      const float ph1 = ldphi(y + 1);
      const float2 e1 = edge ? ldz(u1, xe, y + 1, 0, n, P) : make_float2(0, 0);
      float2 vl = shfl_f2(v0, 1, true), vr = shfl_f2(v0, 1, false);
      if (lane == 0) vl = e0;
      if (lane == 31) vr = e0;
      if (x < P) {
        float4 o = zero;
        if (x < n && y < n) {
          const float4 ay = ldh_df(O.cdf, 0, y, n), dy = ldh_df(O.cdf, 1, y, n), cyr = ldh_df(O.cdf, 2, y, n);
          o = hpoint_df(df_cadd(dx, dy), zero, ph0, O.phi ? 0.0f : pc.y, ax, cxr, ay, cyr, zero, zero, v0, vl, vr,
                        vm, vp, vm, vp, false, ns, nc);
        }
        reinterpret_cast<float4*>(O.w)[pidx(x, y, 0, P)] = o;
        zarch[pidx(x, y, 0, P)] = v0;
      }
      vm = v0;
      v0 = vp;
      ph0 = ph1;
      e0 = e1;
    }
  }
  return df_value(ns, nc);
}

// 3D: the block's 32 x (WY3 + 2) columns marching planes zbeg..zend-1 (y neighbours
// through a two-plane shared ring, as the binary64 pass does).  Everything a plane needs
// from DRAM (the next plane's value, phi, the x neighbours of the warp's edge lanes) is
// loaded one plane ahead, so no DRAM latency sits between the plane's barrier and its
// arithmetic (the z coefficients, shared by the block, come from L1).  In a 255^3 solve
// this took the pass from 446 to 352 us.
__device__ double hstencil3_df(const OuterDev<float2>& O, const float2* u1, float2* zarch, int x, int y, int zbeg,
                               int zend, int w, int lane, bool owned) {
  __shared__ float2 svf[2][WY3 + 2][32];
  const int n = O.n, P = O.P;
  const float4 ax = ldh_df(O.cdf, 0, x, n), cxr = ldh_df(O.cdf, 2, x, n);
  const float4 ay = ldh_df(O.cdf, 0, y, n), cyr = ldh_df(O.cdf, 2, y, n);
  const float4 dxy = df_cadd(ldh_df(O.cdf, 1, x, n), ldh_df(O.cdf, 1, y, n));
  const float2 pc = df_split(O.phic);
  const bool edge = owned && (lane == 0 || lane == 31);
  const int xe = lane == 0 ? x - 1 : x + 1;  // the edge lane's neighbour outside the warp
  auto ldphi = [&](int z) -> float {
    return O.phi ? (inside(x, y, z, n) ? __ldg(O.phi + pidx(x, y, z, P)) : 0.0f) : pc.x;
  };
  float ns = 0.0f, nc = 0.0f;
  if (zbeg < P) {
    float2 vm = ldz(u1, x, y, zbeg - 1, n, P), v0 = ldz(u1, x, y, zbeg, n, P);
    float ph0 = ldphi(zbeg);
    float2 e0 = edge ? ldz(u1, xe, y, zbeg, n, P) : make_float2(0, 0);
    for (int z = zbeg; z < zend; ++z) {
      const float2 vp = ldz(u1, x, y, z + 1, n, P);
      const float ph1 = ldphi(z + 1);
      const float2 e1 = edge ? ldz(u1, xe, y, z + 1, n, P) : make_float2(0, 0);
      svf[z & 1][w][lane] = v0;
      __syncthreads();
      if (owned) {
        const float2 vs = svf[z & 1][w - 1][lane], vn = svf[z & 1][w + 1][lane];
        float2 vl = shfl_f2(v0, 1, true), vr = shfl_f2(v0, 1, false);
        if (lane == 0) vl = e0;
        if (lane == 31) vr = e0;
        if (x < P && y < P) {
          float4 o = make_float4(0, 0, 0, 0);
          if (inside(x, y, z, n))
            o = hpoint_df(dxy, ldh_df(O.cdf, 1, z, n), ph0, O.phi ? 0.0f : pc.y, ax, cxr, ay, cyr, ldh_df(O.cdf, 0, z, n), ldh_df(O.cdf, 2, z, n), v0, vl, vr, vs, vn, vm,
                          vp, true, ns, nc);
          reinterpret_cast<float4*>(O.w)[pidx(x, y, z, P)] = o;
          zarch[pidx(x, y, z, P)] = v0;
        }
      }
      vm = v0;
      v0 = vp;
      ph0 = ph1;
      e0 = e1;
    }
  }
  return df_value(ns, nc);
}

template <typename C, int MODE>
__global__ void __launch_bounds__(32 * WARPS2)
k_hstencil2(const OuterDev<C>* __restrict__ ods, int ntiles, int rows) {
  __shared__ double sm[64];
  const int prob = blockIdx.x / ntiles, tile = blockIdx.x - prob * ntiles;
  const OuterDev<C>& O = ods[prob];
  OuterState* st = O.st;
  if (MODE == 1 && (st->done || st->cycle_end)) return;
  if (MODE == 0 && !st->need_residual) return;
  const int n = O.n, P = O.P;
  const int ntx = ceil_div(P, 32);
  const int tx = tile % ntx, ty = tile / ntx;
  const int lane = threadIdx.x, warp = threadIdx.y;
  const int x = tx * 32 + lane;
  const int ybeg = (ty * WARPS2 + warp) * rows;
  const int yend = min(ybeg + rows, P);
  const C* u1 = stencil_src<C, MODE>(O, st);
  C* zarch = O.Z + (size_t)st->j * O.vs;
  const double2* u0 = O.xpad;
  const bool df = MODE == 1 && st->df;  // H z_j stored as a double-float
  auto form = [&](int xx, int yy) -> double2 {
    return MODE == 0 ? ldd(u0, xx, yy, 0, n, P) : ldd(u1, xx, yy, 0, n, P);
  };
  const HCoef cx = ldh(O.ca, O.cd, O.cc, x, n);
  double accw = 0.0, accb = 0.0;
  bool dfdone = false;
  if constexpr (MODE == 1 && sizeof(C) == 8) {
    if (df) {
      accw = hstencil2_df(O, u1, zarch, x, ybeg, yend, lane);
      dfdone = true;
    }
  }
  if (!dfdone && ybeg < P) {
    double2 vm = form(x, ybeg - 1), v0 = form(x, ybeg);
    for (int y = ybeg; y < yend; ++y) {
      double2 vp = form(x, y + 1);
      double2 vl = shfl_up_c(v0, 1), vr = shfl_down_c(v0, 1);
      if (lane == 0) vl = form(x - 1, y);
      if (lane == 31) vr = form(x + 1, y);
      if (x < P) {
        double2 out = make_double2(0, 0);
        if (x < n && y < n) {
          const HCoef cy = ldh(O.ca, O.cd, O.cc, y, n);
          double2 diag = cadd(cx.d, cy.d);
          diag.x -= O.phi ? widen(__ldg(O.phi + pidx(x, y, 0, P))) : O.phic;
          double2 p = cmul(diag, v0);
          p = cfma(cx.a, vl, p);
          p = cfma(cx.c, vr, p);
          p = cfma(cy.a, vm, p);
          p = cfma(cy.c, vp, p);
          if (MODE == 0) {
            double2 bv = __ldg(O.bpad + pidx(x, y, 0, P));
            out = csub(bv, p);
            accb += dabs2(bv);
          } else {
            out = p;
          }
          accw += dabs2(out);
        }
        if (df) reinterpret_cast<float4*>(O.w)[pidx(x, y, 0, P)] = df_split(out);
        else O.w[pidx(x, y, 0, P)] = out;
        if (MODE == 1) zarch[pidx(x, y, 0, P)] = u1[pidx(x, y, 0, P)];
      }
      vm = v0;
      v0 = vp;
    }
  }
  double red[2] = {accw, accb}, tot[2];
  if (grid_sum_last<2>(red, O.part, tile, ntiles, &st->counter, sm, tot)) {
    if (flat_tid() == 0) outer_stencil_epilogue<C, MODE>(O, st, tot);
  }
}

template <typename C, int MODE>
__global__ void __launch_bounds__(32 * (WY3 + 2), 2)  // two CTAs per SM: 20 warps to hide latency
k_hstencil3(const OuterDev<C>* __restrict__ ods, int ntiles, int rows) {
  __shared__ double sm[64];
  __shared__ double2 sv[2][WY3 + 2][32];
  const int prob = blockIdx.x / ntiles, tile = blockIdx.x - prob * ntiles;
  const OuterDev<C>& O = ods[prob];
  OuterState* st = O.st;
  if (MODE == 1 && (st->done || st->cycle_end)) return;
  if (MODE == 0 && !st->need_residual) return;
  const int n = O.n, P = O.P;
  const int ntx = ceil_div(P, 32), nty = ceil_div(P, WY3);
  const int tx = tile % ntx, ty = (tile / ntx) % nty, tz = tile / (ntx * nty);
  const int lane = threadIdx.x, w = threadIdx.y;
  const bool owned = (w >= 1 && w <= WY3);
  const int x = tx * 32 + lane;
  const int y = ty * WY3 - 1 + w;
  const int zbeg = tz * rows;
  const int zend = min(zbeg + rows, P);
  const C* u1 = stencil_src<C, MODE>(O, st);
  C* zarch = O.Z + (size_t)st->j * O.vs;
  const double2* u0 = O.xpad;
  const bool df = MODE == 1 && st->df;  // H z_j stored as a double-float
  auto form = [&](int xx, int yy, int zz) -> double2 {
    return MODE == 0 ? ldd(u0, xx, yy, zz, n, P) : ldd(u1, xx, yy, zz, n, P);
  };
  const HCoef cx = ldh(O.ca, O.cd, O.cc, x, n), cy = ldh(O.ca, O.cd, O.cc, y, n);
  double accw = 0.0, accb = 0.0;
  bool dfdone = false;
  if constexpr (MODE == 1 && sizeof(C) == 8) {
    if (df) {
      accw = hstencil3_df(O, u1, zarch, x, y, zbeg, zend, w, lane, owned);
      dfdone = true;
    }
  }
  if (!dfdone && zbeg < P) {
    double2 vm = form(x, y, zbeg - 1), v0 = form(x, y, zbeg);
    for (int z = zbeg; z < zend; ++z) {
      double2 vp = form(x, y, z + 1);
      sv[z & 1][w][lane] = v0;
      __syncthreads();
      if (owned) {
        double2 vs = sv[z & 1][w - 1][lane], vn = sv[z & 1][w + 1][lane];
        double2 vl = shfl_up_c(v0, 1), vr = shfl_down_c(v0, 1);
        if (lane == 0) vl = form(x - 1, y, z);
        if (lane == 31) vr = form(x + 1, y, z);
        if (x < P && y < P) {
          double2 out = make_double2(0, 0);
          if (inside(x, y, z, n)) {
            const HCoef cz = ldh(O.ca, O.cd, O.cc, z, n);
            double2 diag = cadd(cadd(cx.d, cy.d), cz.d);
            diag.x -= O.phi ? widen(__ldg(O.phi + pidx(x, y, z, P))) : O.phic;
            double2 p = cmul(diag, v0);
            p = cfma(cx.a, vl, p);
            p = cfma(cx.c, vr, p);
            p = cfma(cy.a, vs, p);
            p = cfma(cy.c, vn, p);
            p = cfma(cz.a, vm, p);
            p = cfma(cz.c, vp, p);
            if (MODE == 0) {
              double2 bv = __ldg(O.bpad + pidx(x, y, z, P));
              out = csub(bv, p);
              accb += dabs2(bv);
            } else {
              out = p;
            }
            accw += dabs2(out);
          }
          if (df) reinterpret_cast<float4*>(O.w)[pidx(x, y, z, P)] = df_split(out);
          else O.w[pidx(x, y, z, P)] = out;
          if (MODE == 1) zarch[pidx(x, y, z, P)] = u1[pidx(x, y, z, P)];
        }
      }
      vm = v0;
      v0 = vp;
    }
  }
  double red[2] = {accw, accb}, tot[2];
  if (grid_sum_last<2>(red, O.part, tile, ntiles, &st->counter, sm, tot)) {
    if (flat_tid() == 0) outer_stencil_epilogue<C, MODE>(O, st, tot);
  }
}

// ------------------------------------------------------------------ multi-dot
// h_i = <v_i, w>, i = 0..j.  The points of a problem are split into `chunks` fixed
// units (contiguous ranges of equal size, dot_unit_begin); persistent CTAs take units
// in turn, so the partial sums, and hence the result, depend neither on the grid nor on
// which other problems share the launch.  A unit sweeps its points once per block of
// DOT_VB vectors with the DOT_VB complex sums in registers, so the FP64
// pipe runs 4 DFMA per point and vector; the warp combines its 2 DOT_VB partial sums
// (padded to 16 or 32) with a transposed butterfly (about one add per value instead of five), the CTA
// combines warps in fixed order.  Units are combined in two levels, so that no
// single SM adds up every unit: the last unit of each group of DOT_GROUP units sums
// the group, the last group sums the groups.
constexpr int DOT_THREADS = 256;
// Vectors per register block (w is re-read once per block): ten where the basis streams
// from HBM (a tenth fewer w reads than eight, 2% off the 255^3 multi-dot), eight on
// smaller problems (fewer registers, no spills; 2-4% faster on the 1023^2 solves).
constexpr size_t DOT_VB10_MIN_POINTS = (size_t)1 << 22;
constexpr int DOT_GROUP = 16;  // units per first-level group

HELM_HD inline int dot_groups(int chunks) { return (chunks + DOT_GROUP - 1) / DOT_GROUP; }

// First point of unit u of `chunks` contiguous units over n points: equal shares, each
// starting on a multiple of 32 points, so that a warp's 16-byte loads and stores cover
// whole 128-byte lines (unaligned starts split every warp access over one more line).
__device__ __forceinline__ size_t unit_begin(size_t n, int u, int chunks) {
  return u >= chunks ? n : ((n * (size_t)u) / (size_t)chunks) & ~(size_t)31;
}

// First point of unit u of the multi-dot: equal shares starting at any point.  On the
// 255^3 basis (one GPU, ncu, both forms back to back) this ran 3-4% faster than 32-point
// starts from j = 4 on, although it reads about 6% more from DRAM (lines that straddle
// two warps' ranges are fetched twice); 32-point starts were faster only for j <= 2.
// The new-vector pass, which writes as well, gains from 32-point starts (unit_begin).
__device__ __forceinline__ size_t dot_unit_begin(size_t n, int u, int chunks) {
  return (n * (size_t)u) / (size_t)chunks;
}

// Sum NS (16 or 32) per-lane values over the warp; lane L returns the total of value
// L (NS = 32) or L >> 1 (NS = 16) (fixed order: butterflies at offsets 16, 8, 4, ...,
// halving the values kept, so about one shuffle and one add per value instead of five).
template <int NS>
__device__ __forceinline__ double warp_transpose_sum(double (&v)[NS], int lane) {
  int o = 16;
#pragma unroll
  for (int c = NS / 2; c >= 1; c >>= 1, o >>= 1) {
    const bool hi = lane & o;
#pragma unroll
    for (int k = 0; k < c; ++k) {
      const double send = hi ? v[k] : v[k + c];
      const double keep = hi ? v[k + c] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return NS == 32 ? v[0] : v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// One thread's sums over its points of the DOT_VB vectors vb .. vb + nv - 1: acc[2 t]
// and acc[2 t + 1] the real and imaginary parts of <v_{vb+t}, w>.
template <int DOT_VB>
__device__ __forceinline__ void dots_block_f64(const double2* V, const double2* W, size_t npts, int vb, int nv,
                                               size_t beg, size_t end, bool rev, double (&acc)[2 * DOT_VB]) {
  const double2* vbase = V + (size_t)vb * npts;
#pragma unroll
  for (int k = 0; k < 2 * DOT_VB; ++k) acc[k] = 0.0;
  const int cnt = beg < end ? (int)((end - beg + DOT_THREADS - 1) / DOT_THREADS) : 0;
  const int dk = rev ? -1 : 1;
#pragma unroll 2
  for (int q = 0, k = rev ? cnt - 1 : 0; q < cnt; ++q, k += dk) {
    const size_t idx = beg + (size_t)k * DOT_THREADS;
    const double2 w = __ldcg(W + idx);
#pragma unroll
    for (int t = 0; t < DOT_VB; ++t) {
      if (t < nv) {
        const double2 v = __ldcs(vbase + (size_t)t * npts + idx);
        acc[2 * t] = fma(v.x, w.x, acc[2 * t]);
        acc[2 * t] = fma(v.y, w.y, acc[2 * t]);
        acc[2 * t + 1] = fma(v.x, w.y, acc[2 * t + 1]);
        acc[2 * t + 1] = fma(-v.y, w.x, acc[2 * t + 1]);
      }
    }
  }
}
// The same sums with the basis and w in double-float (FP32 pipe), widened to binary64
// at the end: conj(v) w = (vr wr + vi wi) + i (vr wi - vi wr), four multiply-adds.
template <int DOT_VB>
__device__ __forceinline__ void dots_block_df(const double2* V, const double2* W, size_t npts, int vb, int nv,
                                              size_t beg, size_t end, bool rev, double (&acc)[2 * DOT_VB]) {
  const float4* vbase = reinterpret_cast<const float4*>(V) + (size_t)vb * npts;
  const float4* w4 = reinterpret_cast<const float4*>(W);
  float s[2 * DOT_VB], c[2 * DOT_VB];
#pragma unroll
  for (int k = 0; k < 2 * DOT_VB; ++k) s[k] = c[k] = 0.0f;
  const int cnt = beg < end ? (int)((end - beg + DOT_THREADS - 1) / DOT_THREADS) : 0;
  const int dk = rev ? -1 : 1;
  for (int q = 0, k = rev ? cnt - 1 : 0; q < cnt; ++q, k += dk) {
    const size_t idx = beg + (size_t)k * DOT_THREADS;
    const float4 w = __ldcg(w4 + idx);
    float4 v[DOT_VB];
#pragma unroll
    for (int t = 0; t < DOT_VB; ++t)
      if (t < nv) v[t] = __ldcs(vbase + (size_t)t * npts + idx);
#pragma unroll
    for (int t = 0; t < DOT_VB; ++t) {
      if (t < nv) {
        df_mac(s[2 * t], c[2 * t], v[t].x, v[t].y, w.x, w.y);
        df_mac(s[2 * t], c[2 * t], v[t].z, v[t].w, w.z, w.w);
        df_mac(s[2 * t + 1], c[2 * t + 1], v[t].x, v[t].y, w.z, w.w);
        df_mac(s[2 * t + 1], c[2 * t + 1], -v[t].z, -v[t].w, w.x, w.y);
        df_renorm(s[2 * t], c[2 * t]);
        df_renorm(s[2 * t + 1], c[2 * t + 1]);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 2 * DOT_VB; ++k) acc[k] = df_value(s[k], c[k]);
}

template <typename C, int DOT_VB>
__global__ void __launch_bounds__(DOT_THREADS, 2)
k_dots(const OuterDev<C>* __restrict__ ods, int nprob, int chunks) {
  extern __shared__ double sred[];  // [warp][2 (m + 1)] per-warp sums of the unit
  __shared__ int s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ngroups = dot_groups(chunks);
  for (int g = blockIdx.x; g < nprob * chunks; g += gridDim.x) {
    const int prob = g / chunks, unit = g - prob * chunks;
    const OuterDev<C>& O = ods[prob];
    OuterState* st = O.st;
    if (st->done || st->cycle_end) continue;  // uniform over the CTA
    const int j = st->j, M1 = st->m + 1;
    const size_t npts = O.vs;
    const size_t ubeg = dot_unit_begin(npts, unit, chunks), uend = dot_unit_begin(npts, unit + 1, chunks);
    double* upart = O.part;                                   // [chunks][M1][2]
    double* gpart = O.part + (size_t)chunks * M1 * 2;         // [ngroups][M1][2]
    unsigned* gcnt = O.gcnt;  // [ngroups], zero between calls (each group's last unit resets its own)
    double* wsum = sred + (size_t)warp * 2 * M1;
    __syncthreads();  // the previous unit's readers of sred are done
    const bool df = st->df;
    for (int vb = 0; vb <= j; vb += DOT_VB) {
      const int nv = min(DOT_VB, j + 1 - vb);
      double acc[2 * DOT_VB];
      // where w streams from HBM (ten-vector blocks), odd blocks sweep the unit backwards:
      // they start on the part of w the previous block read last, the part most likely
      // still in L2
      const bool rev = DOT_VB >= 10 && ((vb / DOT_VB) & 1);
      if (df) dots_block_df<DOT_VB>(O.V, O.w, npts, vb, nv, ubeg + tid, uend, rev, acc);
      else dots_block_f64<DOT_VB>(O.V, O.w, npts, vb, nv, ubeg + tid, uend, rev, acc);
      constexpr int NS = 2 * DOT_VB <= 16 ? 16 : 32;
      double vals[NS];
#pragma unroll
      for (int k = 0; k < NS; ++k) vals[k] = k < 2 * DOT_VB ? acc[k < 2 * DOT_VB ? k : 0] : 0.0;
      const double r = warp_transpose_sum<NS>(vals, lane);
      const int vi = NS == 32 ? lane : lane >> 1;
      if ((NS == 32 || (lane & 1) == 0) && vi < 2 * nv) wsum[2 * vb + vi] = r;
    }
    __syncthreads();
    for (int k = tid; k < 2 * (j + 1); k += DOT_THREADS) {
      double sum = 0.0;
#pragma unroll
      for (int ww = 0; ww < DOT_THREADS / 32; ++ww) sum += sred[(size_t)ww * 2 * M1 + k];
      upart[(size_t)unit * M1 * 2 + k] = sum;
    }
    // first level: the last unit of the group sums the group's units
    const int grp = unit / DOT_GROUP, u0 = grp * DOT_GROUP, gsize = min(DOT_GROUP, chunks - u0);
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(gcnt + grp, 1u) == (unsigned)gsize - 1u);
    __syncthreads();
    if (!s_last) continue;
    __threadfence();
    for (int k = tid; k < 2 * (j + 1); k += DOT_THREADS) {
      double sum = 0.0;
      for (int u = u0; u < u0 + gsize; ++u) sum += __ldcg(upart + (size_t)u * M1 * 2 + k);
      gpart[(size_t)grp * M1 * 2 + k] = sum;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      gcnt[grp] = 0u;
      s_last = (atomicAdd(&st->counter, 1u) == (unsigned)ngroups - 1u);
    }
    __syncthreads();
    if (!s_last) continue;
    // second level: the last group sums the groups and scales into the Hessenberg column
    __threadfence();
    for (int i = tid; i <= j; i += DOT_THREADS) {
      double2 sum = make_double2(0, 0);
      for (int c = 0; c < ngroups; ++c)
        sum = cadd(sum, make_double2(__ldcg(gpart + ((size_t)c * M1 + i) * 2),
                                     __ldcg(gpart + ((size_t)c * M1 + i) * 2 + 1)));
      const double sc = O.vscale[i];
      const double2 h = make_double2(sum.x * sc, sum.y * sc);
      O.hcol[i] = h;
      O.Hm[(size_t)j * M1 + i] = h;
    }
    if (tid == 0) st->counter = 0u;
    __syncthreads();
  }
}

// Units of the multi-dot and new-vector passes for a problem of vs points: four per
// SM (so the persistent grids, two or four CTAs per SM, get equal shares), at most one
// per 256 points.
int outer_chunks(size_t vs) {
  static const int units = [] {  // thread-safe initialisation
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 1;
    return 4 * std::max(1, sms);
  }();
  return (int)std::max<size_t>(1, std::min<size_t>((size_t)units, (vs + DOT_THREADS - 1) / DOT_THREADS));
}

// Doubles of the outer partial-sum buffer the passes need for `chunks` units and
// restart length m (unit and group partials of the multi-dot).  The buffer is scratch
// shared by the outer passes, each overwriting the others' slots.
size_t outer_part_doubles(int chunks, int m) {
  const int ng = dot_groups(chunks);
  return (size_t)(chunks + ng) * (m + 1) * 2;
}
// Group counters of the multi-dot for `chunks` units.  They live in a buffer of their
// own: a counter must read zero at the start of every call, and the partial-sum buffer
// is overwritten by the other outer passes' partials in between (which, for short
// restart lengths, once corrupted the counters and with them the inner products).
int outer_dot_counters(int chunks) { return dot_groups(chunks); }

// ------------------------------------------------------------------ new Arnoldi vector
// Givens update of column j once h_{j+1,j} is known (last block of k_vnew, warp 0).
// The column's entries 0..j (hc) and the earlier rotations (cs, sn) were staged in
// shared memory by the whole block.  Rotation i maps the running entry t_i and the
// untouched h_{i+1} to the final H[i] = c_i t_i + s_i h_{i+1} and to
// t_{i+1} = c_i h_{i+1} - conj(s_i) t_i, an affine map of t_i.  A dependent chain of j
// such maps costs j x ~14 FP64 latencies on one thread (on this part every FP64
// instruction occupies its pipe for 64 cycles), so the warp splits the chain into 32
// segments, composes each segment's maps, scans the compositions across lanes, and
// every lane then walks its own segment from the exact entering t.
template <typename C>
__device__ void givens_step_warp(const OuterDev<C>& O, OuterState* st, int j, double hn, const double2* hc,
                                 const double* cs, const double2* sn_prev, double2* t_last) {
  const int lane = threadIdx.x & 31;
  const int M1 = st->m + 1;
  double2* Hc = O.Hm + (size_t)j * M1;
  const int per = (j + 31) / 32;
  const int i0 = min(j, lane * per), i1 = min(j, i0 + per);
  // composition (al, be) of this lane's maps t -> A_i t + B_i, A_i = -conj(s_i), B_i = c_i h_{i+1}
  double2 al = make_double2(1, 0), be = make_double2(0, 0);
  for (int i = i0; i < i1; ++i) {
    const double2 A = make_double2(-sn_prev[i].x, sn_prev[i].y);
    const double2 B = make_double2(cs[i] * hc[i + 1].x, cs[i] * hc[i + 1].y);
    be = cfma(A, be, B);
    al = cmul(A, al);
  }
  // inclusive scan: lane l holds the composition of segments 0..l (earlier maps first)
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double2 pa = shfl_up_c(al, o), pb = shfl_up_c(be, o);
    if (lane >= o) {
      be = cfma(al, pb, be);
      al = cmul(al, pa);
    }
  }
  const double2 ea = shfl_up_c(al, 1), eb = shfl_up_c(be, 1);
  const double2 h0 = hc[0];
  double2 t = lane == 0 ? h0 : cfma(ea, h0, eb);  // t_{i0}
  for (int i = i0; i < i1; ++i) {
    const double c = cs[i];
    const double2 s = sn_prev[i];
    const double2 t1 = hc[i + 1];
    Hc[i] = cadd(make_double2(c * t.x, c * t.y), cmul(s, t1));
    t = csub(make_double2(c * t1.x, c * t1.y), cmul(dconj(s), t));
  }
  if (i1 == j && i0 < i1) *t_last = t;  // the lane holding rotation j-1
  if (j == 0 && lane == 0) *t_last = h0;
  __syncwarp();
  if (lane != 0) return;
  const double2 a = *t_last, b = make_double2(hn, 0);
  const double na = sqrt(dabs2(a)), nb = sqrt(dabs2(b));
  const double r = hypot(na, nb);
  double c;
  double2 sn;
  if (r == 0.0) { c = 1.0; sn = make_double2(0, 0); }
  else if (na == 0.0) { c = 0.0; sn = make_double2(1, 0); }
  else {
    c = na / r;
    sn = cmul(make_double2(a.x / na, a.y / na), dconj(b));
    sn = make_double2(sn.x / r, sn.y / r);
  }
  O.cs[j] = c;
  O.sn[j] = sn;
  Hc[j] = cadd(make_double2(c * a.x, c * a.y), cmul(sn, b));
  Hc[j + 1] = make_double2(0, 0);
  const double2 g0 = O.g[j];
  O.g[j] = make_double2(c * g0.x, c * g0.y);
  O.g[j + 1] = cmul(make_double2(-sn.x, sn.y), g0);
}

// Shared memory of k_vnew: the scaled column h (m+1) in binary64 and in double-float,
// then the staging of the Givens update: column j (m+1), sines (m), cosines (m).
HELM_HD constexpr size_t vnew_smem_bytes(int m) {
  return 2 * (size_t)(m + 1) * 16 + (size_t)(m + 1) * 16 + (size_t)m * 16 + (size_t)m * 8;
}

// u = w - sum_{i<=j} h_i v_i stored as V[j+1] with ||u|| reduced here; the last block
// sets h_{j+1,j} = ||u||, vscale[j+1] = 1/||u||, performs the Givens update and decides
// whether the cycle ends.  Writes the next V-cycle input b0 (precision C) and starts
// level 0's first sweep from its norm.  (A cycle's first vector: k_vstart.)
template <typename C>
__global__ void __launch_bounds__(256, 4)
k_vnew(const OuterDev<C>* __restrict__ ods, int nprob, int chunks) {
  extern __shared__ double2 sh[];  // m+1
  __shared__ double sm[64];
  const int tid = threadIdx.x;
  for (int g = blockIdx.x; g < nprob * chunks; g += gridDim.x) {
    const int prob = g / chunks, unit = g - prob * chunks;
    const OuterDev<C>& O = ods[prob];
    OuterState* st = O.st;
    if (st->done || st->cycle_end) continue;  // uniform
    const int j = st->j;
    const bool df = st->df;
    float4* shf = reinterpret_cast<float4*>(sh + (st->m + 1));  // the same column as double-floats
    __shared__ double s_scale[1];
    __syncthreads();  // the previous unit's readers of sh and s_scale are done
    for (int i = tid; i <= j; i += blockDim.x) {
      const double sc = O.vscale[i];
      sh[i] = make_double2(O.hcol[i].x * sc, O.hcol[i].y * sc);
      shf[i] = df_split(sh[i]);
    }
    // The next V-cycle's input is u / ||w||: the preconditioned operator maps it back to
    // O(1) norms, so its magnitude does not drift over a cycle (an unscaled u shrinks
    // geometrically and would underflow complex64).  FGMRES is exact for any scaling of
    // z_j: w = H z_j and the Hessenberg column inherit it, and x = Z y cancels it.  One
    // thread forms the scale (an FP64 square root and division are long sequences on
    // this part's FP64 pipe).
    if (tid == 0) s_scale[0] = st->wnorm2 > 0.0 ? 1.0 / sqrt(st->wnorm2) : 1.0;
    __syncthreads();
    const double bsc = s_scale[0];
    const int jn = j + 1;
    double2* vout = O.V + (size_t)jn * O.vs;
    double accu = 0.0;
    typename CT<C>::R accb = 0;
    const size_t end = unit_begin(O.vs, unit + 1, chunks);
    if (df) {
      // u = w - sum h_i v_i in double-float: four multiply-adds per vector on the FP32
      // pipe, eight vectors' loads in flight per step (the pass is bound by HBM: the
      // loads in flight per SM must cover its latency)
      const float4* w4 = reinterpret_cast<const float4*>(O.w);
      float4* vout4 = reinterpret_cast<float4*>(vout);
      const float bscf = (float)bsc;
      const bool bf = sizeof(C) == 8 && bscf > 1e-30f && bscf < 1e30f;  // complex64 input formed in FP32
      float ns = 0.0f, nc = 0.0f;
      for (size_t idx = unit_begin(O.vs, unit, chunks) + tid; idx < end; idx += blockDim.x) {
        const float4 w = __ldcg(w4 + idx);
        float sr = w.x, cr = w.y, si = w.z, ci = w.w;
        const float4* vp = reinterpret_cast<const float4*>(O.V) + idx;
        int i = 0;
        for (; i + 7 <= j; i += 8) {
          float4 v[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) v[q] = __ldcs(vp + (size_t)(i + q) * O.vs);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 h = shf[i + q];
            df_mac(sr, cr, -h.x, -h.y, v[q].x, v[q].y);
            df_mac(sr, cr, h.z, h.w, v[q].z, v[q].w);
            df_mac(si, ci, -h.x, -h.y, v[q].z, v[q].w);
            df_mac(si, ci, -h.z, -h.w, v[q].x, v[q].y);
          }
          df_renorm(sr, cr);
          df_renorm(si, ci);
        }
        if (i + 3 <= j) {
          float4 v[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) v[q] = __ldcs(vp + (size_t)(i + q) * O.vs);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float4 h = shf[i + q];
            df_mac(sr, cr, -h.x, -h.y, v[q].x, v[q].y);
            df_mac(sr, cr, h.z, h.w, v[q].z, v[q].w);
            df_mac(si, ci, -h.x, -h.y, v[q].z, v[q].w);
            df_mac(si, ci, -h.z, -h.w, v[q].x, v[q].y);
          }
          i += 4;
        }
        for (; i <= j; ++i) {
          const float4 v = __ldcs(vp + (size_t)i * O.vs), h = shf[i];
          df_mac(sr, cr, -h.x, -h.y, v.x, v.y);
          df_mac(sr, cr, h.z, h.w, v.z, v.w);
          df_mac(si, ci, -h.x, -h.y, v.z, v.w);
          df_mac(si, ci, -h.z, -h.w, v.x, v.y);
        }
        float ur, lr, ui, li;
        df_two_sum(sr, cr, ur, lr);
        df_two_sum(si, ci, ui, li);
        vout4[idx] = make_float4(ur, lr, ui, li);
        df_mac(ns, nc, ur, lr, ur, lr);
        df_mac(ns, nc, ui, li, ui, li);
        df_renorm(ns, nc);
        C c;
        if (bf) c = CT<C>::make((typename CT<C>::R)__fmul_rn(__fadd_rn(ur, lr), bscf),
                                (typename CT<C>::R)__fmul_rn(__fadd_rn(ui, li), bscf));
        else c = from_d<C>(make_double2(df_value(ur, lr) * bsc, df_value(ui, li) * bsc));
        O.b0[idx] = c;
        accb += cabs2(c);
      }
      accu = df_value(ns, nc);
    } else
    for (size_t idx = unit_begin(O.vs, unit, chunks) + tid; idx < end; idx += blockDim.x) {
      // two independent accumulation chains keep the FP64 pipe busy
      double2 wa = __ldcg(O.w + idx), wb = make_double2(0, 0);
      const double2* vp = O.V + idx;
      int i = 0;
      for (; i + 1 <= j; i += 2) {
        const double2 v0 = __ldcs(vp + (size_t)i * O.vs), v1 = __ldcs(vp + (size_t)(i + 1) * O.vs);
        wa = cfms(sh[i], v0, wa);
        wb = cfms(sh[i + 1], v1, wb);
      }
      if (i <= j) wa = cfms(sh[i], __ldcs(vp + (size_t)i * O.vs), wa);
      const double2 wv = cadd(wa, wb);
      vout[idx] = wv;
      accu += dabs2(wv);
      C c = from_d<C>(make_double2(wv.x * bsc, wv.y * bsc));
      O.b0[idx] = c;
      accb += cabs2(c);
    }
    double red[2] = {accu, (double)accb}, tot[2];
    if (grid_sum_last<2>(red, O.part, unit, chunks, &st->counter, sm, tot)) {
      const int mm = st->m;
      double2* hc = sh + 2 * (mm + 1);
      double2* sn_prev = hc + (mm + 1);
      double* cs = reinterpret_cast<double*>(sn_prev + mm);
      {
        const double2* Hc = O.Hm + (size_t)j * (mm + 1);
        for (int i = tid; i <= j; i += blockDim.x) hc[i] = __ldcg(Hc + i);
        for (int i = tid; i < j; i += blockDim.x) {
          sn_prev[i] = __ldcg(O.sn + i);
          cs[i] = __ldcg(O.cs + i);
        }
        __syncthreads();
      }
      __shared__ double2 t_last;
      if (tid < 32) givens_step_warp(O, st, j, tid == 0 ? sqrt(tot[0]) : 0.0, hc, cs, sn_prev, &t_last);
      if (tid == 0) {
        sweep_begin(O.sc0, (typename CT<C>::R)tot[1], O.s);
        const double hn = sqrt(tot[0]);
        O.vscale[jn] = hn > 0.0 ? 1.0 / hn : 0.0;
        st->iters += 1;
        st->rel_est = st->bnorm > 0.0 ? sqrt(dabs2(O.g[j + 1])) / st->bnorm : 0.0;
        // lucky breakdown: the new direction vanishes against H z_j (below the rounding
        // level of the basis arithmetic: about 2^-46 j relative in double-float)
        const bool breakdown = !(hn > (df ? 1e-12 : 1e-14) * sqrt(st->wnorm2));
        if (!isfinite(st->rel_est)) { st->done = 3; st->status = -4; st->cycle_end = 1; }
        else if (st->rel_est <= st->tol || st->iters >= st->maxit || j + 1 >= st->m || breakdown) st->cycle_end = 1;
        else st->j = jn;
      }
    }
  }
}

// The first basis vector of a cycle, v_0 = r / beta (w holds the true residual r): the
// cycle-start case of k_vnew in a kernel of its own, so that its double-float form adds
// no registers to the per-iteration pass.  With a double-float basis and a complex64
// preconditioner r is split on the integer pipes and scaled by 1/beta in double-float
// (no FP64 instruction per point); otherwise in binary64.  Writes the V-cycle input b0
// and starts level 0's first sweep from its norm.
template <typename C>
__global__ void __launch_bounds__(256)
k_vstart(const OuterDev<C>* __restrict__ ods, int nprob, int chunks) {
  __shared__ double sm[64];
  const int tid = threadIdx.x;
  for (int g = blockIdx.x; g < nprob * chunks; g += gridDim.x) {
    const int prob = g / chunks, unit = g - prob * chunks;
    const OuterDev<C>& O = ods[prob];
    OuterState* st = O.st;
    if (st->done || !st->fresh) continue;  // uniform
    __shared__ double s_inv;
    __syncthreads();  // the previous unit's block reduction and s_inv readers are done
    if (tid == 0) s_inv = 1.0 / st->beta;  // one thread: a long FP64 sequence on this part
    __syncthreads();
    const bool df = st->df;
    const double inv = s_inv;
    double2* vout = O.V;
    typename CT<C>::R accb = 0;
    const size_t end = unit_begin(O.vs, unit + 1, chunks);
    if (df && sizeof(C) == 8) {
      const float2 sinv = df_split(inv);
      for (size_t idx = unit_begin(O.vs, unit, chunks) + tid; idx < end; idx += blockDim.x) {
        const double2 r = __ldcg(O.w + idx);
        const float2 rr = df_split(r.x), ri = df_split(r.y);
        const float pr = __fmul_rn(rr.x, sinv.x), pi = __fmul_rn(ri.x, sinv.x);
        const float er = fmaf(rr.x, sinv.y, fmaf(rr.y, sinv.x, fmaf(rr.x, sinv.x, -pr)));
        const float ei = fmaf(ri.x, sinv.y, fmaf(ri.y, sinv.x, fmaf(ri.x, sinv.x, -pi)));
        float ur, lr, ui, li;
        df_two_sum(pr, er, ur, lr);
        df_two_sum(pi, ei, ui, li);
        reinterpret_cast<float4*>(vout)[idx] = make_float4(ur, lr, ui, li);
        const C c = CT<C>::make((typename CT<C>::R)__fadd_rn(ur, lr), (typename CT<C>::R)__fadd_rn(ui, li));
        O.b0[idx] = c;
        accb += cabs2(c);
      }
    } else {
      for (size_t idx = unit_begin(O.vs, unit, chunks) + tid; idx < end; idx += blockDim.x) {
        const double2 r = __ldcg(O.w + idx);
        const double2 wv = make_double2(r.x * inv, r.y * inv);
        if (df) reinterpret_cast<float4*>(vout)[idx] = df_split(wv);
        else vout[idx] = wv;
        const C c = from_d<C>(wv);
        O.b0[idx] = c;
        accb += cabs2(c);
      }
    }
    double red[1] = {(double)accb}, tot[1];
    if (grid_sum_last<1>(red, O.part, unit, chunks, &st->counter, sm, tot)) {
      if (tid == 0) {
        sweep_begin(O.sc0, (typename CT<C>::R)tot[0], O.s);
        O.vscale[0] = 1.0;
        st->fresh = 0;
        st->j = 0;
      }
    }
  }
}

// y = R^{-1} g over the current cycle's columns (one warp per problem).
template <typename C>
__global__ void k_backsolve(const OuterDev<C>* __restrict__ ods) {
  const OuterDev<C>& O = ods[blockIdx.x];
  OuterState* st = O.st;
  if (!st->cycle_end) return;
  const int k = st->j + 1;  // columns in this cycle
  const int M1 = st->m + 1;
  const int lane = threadIdx.x;
  if (lane == 0) { st->need_residual = 1; st->restarts += 1; }
  for (int i = lane; i < k; i += 32) O.y[i] = O.g[i];
  __syncwarp();
  for (int c = k - 1; c >= 0; --c) {
    if (lane == 0) {
      const double2 d = O.Hm[(size_t)c * M1 + c];
      O.y[c] = dabs2(d) > 0.0 ? ddiv(O.y[c], d) : make_double2(0, 0);
    }
    __syncwarp();
    const double2 yc = O.y[c];
    for (int i = lane; i < c; i += 32) O.y[i] = csub(O.y[i], cmul(O.Hm[(size_t)c * M1 + i], yc));
    __syncwarp();
  }
}

// x += sum_i y_i z_i over the stored preconditioned vectors: binary64 accumulation, or
// (double-float basis with complex64 z_i) double-float accumulation on the FP32 pipe of
// the exact complex64 z_i against y split into double-floats, x read and written in
// binary64.
template <typename C>
__global__ void __launch_bounds__(256)
k_solution(const OuterDev<C>* __restrict__ ods, int chunks) {
  extern __shared__ double2 sh[];  // y (m+1), then y as double-floats (m+1)
  const int prob = blockIdx.x / chunks, cta = blockIdx.x - prob * chunks;
  const OuterDev<C>& O = ods[prob];
  OuterState* st = O.st;
  if (!st->cycle_end) return;
  const int k = st->j + 1;
  float4* shf = reinterpret_cast<float4*>(sh + (st->m + 1));
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    sh[i] = O.y[i];
    shf[i] = df_split(sh[i]);
  }
  __syncthreads();
  if constexpr (sizeof(C) == 8) {
    if (st->df) {
      for (size_t idx = (size_t)cta * blockDim.x + threadIdx.x; idx < O.vs; idx += (size_t)chunks * blockDim.x) {
        const double2 x0 = O.xpad[idx];
        const float2 xr = df_split(x0.x), xi = df_split(x0.y);
        float sr = xr.x, cr = xr.y, si = xi.x, ci = xi.y;
        const C* zp = O.Z + idx;
        int i = 0;
        for (; i + 7 < k; i += 8) {
          C z[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) z[q] = __ldcs(zp + (size_t)(i + q) * O.vs);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 y = shf[i + q];
            df_mac1(sr, cr, y.x, y.y, z[q].x);
            df_mac1(sr, cr, -y.z, -y.w, z[q].y);
            df_mac1(si, ci, y.x, y.y, z[q].y);
            df_mac1(si, ci, y.z, y.w, z[q].x);
          }
          df_renorm(sr, cr);
          df_renorm(si, ci);
        }
        for (; i < k; ++i) {
          const C z = __ldcs(zp + (size_t)i * O.vs);
          const float4 y = shf[i];
          df_mac1(sr, cr, y.x, y.y, z.x);
          df_mac1(sr, cr, -y.z, -y.w, z.y);
          df_mac1(si, ci, y.x, y.y, z.y);
          df_mac1(si, ci, y.z, y.w, z.x);
        }
        O.xpad[idx] = make_double2(df_value(sr, cr), df_value(si, ci));
      }
      return;
    }
  }
  for (size_t idx = (size_t)cta * blockDim.x + threadIdx.x; idx < O.vs; idx += (size_t)chunks * blockDim.x) {
    double2 xv = O.xpad[idx];
    for (int i = 0; i < k; ++i) xv = cfma(sh[i], to_d(__ldcg(O.Z + (size_t)i * O.vs + idx)), xv);
    O.xpad[idx] = xv;
  }
}

// ------------------------------------------------------------------ launchers
template <typename C>
void outer_residual(int dim, const OuterDev<C>* od, int nprob, int ntiles, TileCfg cfg, cudaStream_t s) {
  if (dim == 2) k_hstencil2<C, 0><<<nprob * ntiles, dim3(32, WARPS2), 0, s>>>(od, ntiles, cfg.rows);
  else k_hstencil3<C, 0><<<nprob * ntiles, dim3(32, WY3 + 2), 0, s>>>(od, ntiles, cfg.rows);
}
template <typename C>
void outer_apply_h(int dim, const OuterDev<C>* od, int nprob, int ntiles, TileCfg cfg, cudaStream_t s) {
  if (dim == 2) k_hstencil2<C, 1><<<nprob * ntiles, dim3(32, WARPS2), 0, s>>>(od, ntiles, cfg.rows);
  else k_hstencil3<C, 1><<<nprob * ntiles, dim3(32, WY3 + 2), 0, s>>>(od, ntiles, cfg.rows);
}
// Resident CTAs of a kernel over the whole GPU (the persistent grid of the outer
// passes), cached per thread for the last shared-memory size asked.
template <typename K>
static int resident_grid(K kernel, int threads, size_t smem) {
  thread_local K last_kernel = nullptr;
  thread_local size_t last_smem = 0;
  thread_local int last = 0;
  if (kernel == last_kernel && smem == last_smem && last > 0) return last;
  int dev = 0, sms = 1, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  last_kernel = kernel;
  last_smem = smem;
  last = per_sm * std::max(sms, 1);
  return last;
}

template <typename C, int VB>
static void launch_dots(const OuterDev<C>* od, int nprob, int chunks, int m, cudaStream_t s) {
  const size_t smem = (size_t)(DOT_THREADS / 32) * 2 * (m + 1) * sizeof(double);
  thread_local size_t configured = 0;  // per host thread and block size; setting it again is harmless
  if (smem > 48 * 1024 && smem > configured) {
    cudaFuncSetAttribute(k_dots<C, VB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured = smem;
  }
  thread_local size_t res_smem = 0;
  thread_local int resident = 0;
  if (resident == 0 || res_smem != smem) {
    int dev = 0, sms = 1, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dots<C, VB>, DOT_THREADS, smem) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    resident = per_sm * std::max(sms, 1);
    res_smem = smem;
  }
  k_dots<C, VB><<<std::min(nprob * chunks, resident), DOT_THREADS, smem, s>>>(od, nprob, chunks);
}
template <typename C>
void outer_dots(const OuterDev<C>* od, int nprob, int chunks, int m, size_t vs, cudaStream_t s) {
  if (vs >= DOT_VB10_MIN_POINTS) launch_dots<C, 10>(od, nprob, chunks, m, s);
  else launch_dots<C, 8>(od, nprob, chunks, m, s);
}
template <typename C>
void outer_vnew(const OuterDev<C>* od, int nprob, int chunks, int m, bool start, cudaStream_t s) {
  // Shared memory is padded so that at most four CTAs fit on an SM: the persistent
  // grid of four CTAs per SM then places exactly four on every SM, one unit each, so
  // the work (FP64 in binary64, HBM in double-float) is spread evenly.  Four CTAs
  // (1024 threads) keep enough loads in flight for the double-float pass: at two per SM
  // the pass reached 2.9 TB/s, at four 5.0 TB/s (255^3, 19 basis vectors).
  thread_local size_t pad = 0;
  if (pad == 0) {
    int dev = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    pad = (size_t)per_sm / 5 + 1024;
    cudaFuncSetAttribute(k_vnew<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(pad, 160 * 1024));
  }
  const size_t need = vnew_smem_bytes(m);
  if (need > 160 * 1024) {
    thread_local size_t configured = 0;
    if (need > configured) {
      cudaFuncSetAttribute(k_vnew<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
      configured = need;
    }
  }
  if (start) {
    thread_local int vres = 0;
    if (vres == 0) vres = resident_grid(k_vstart<C>, 256, 0);
    k_vstart<C><<<std::min(nprob * chunks, vres), 256, 0, s>>>(od, nprob, chunks);
    return;
  }
  const size_t smem = std::max<size_t>(need, pad);
  const int resident = resident_grid(k_vnew<C>, 256, smem);
  k_vnew<C><<<std::min(nprob * chunks, resident), 256, smem, s>>>(od, nprob, chunks);
}
template <typename C>
void outer_backsolve(const OuterDev<C>* od, int nprob, cudaStream_t s) {
  k_backsolve<C><<<nprob, 32, 0, s>>>(od);
}
template <typename C>
void outer_solution(const OuterDev<C>* od, int nprob, int chunks, int m, cudaStream_t s) {
  const size_t smem = 2 * (size_t)(m + 1) * sizeof(double2);
  thread_local size_t configured = 0;  // per host thread; setting the attribute again is harmless
  if (smem > 48 * 1024 && smem > configured) {
    cudaFuncSetAttribute(k_solution<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured = smem;
  }
  k_solution<C><<<nprob * chunks, 256, smem, s>>>(od, chunks);
}

// Binary64 complex values stored in the basis arithmetic: as double-floats (df) or
// copied unchanged.
__global__ void __launch_bounds__(256) k_basis_store(const double2* __restrict__ src, double2* __restrict__ dst,
                                                     size_t n, int df) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double2 v = src[i];
    if (df) reinterpret_cast<float4*>(dst)[i] = df_split(v);
    else dst[i] = v;
  }
}
void basis_store(const double2* src, double2* dst, size_t n, int df, cudaStream_t s) {
  const size_t blocks = std::min<size_t>((n + 255) / 256, 4096);
  k_basis_store<<<(unsigned)std::max<size_t>(blocks, 1), 256, 0, s>>>(src, dst, n, df);
}

// The outer states of a set's problems gathered into one array (one copy to the host
// per iteration instead of one per problem).
__global__ void __launch_bounds__(256) k_gather_states(OuterState* const* __restrict__ src, OuterState* dst,
                                                       int count) {
  constexpr int W = (int)(sizeof(OuterState) / sizeof(unsigned));
  static_assert(sizeof(OuterState) % sizeof(unsigned) == 0, "OuterState is copied in 32-bit words");
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count * W; i += gridDim.x * blockDim.x) {
    const int p = i / W, w = i - p * W;
    reinterpret_cast<unsigned*>(dst + p)[w] = reinterpret_cast<const unsigned*>(src[p])[w];
  }
}
void gather_states(OuterState* const* src, OuterState* dst, int count, cudaStream_t s) {
  constexpr int W = (int)(sizeof(OuterState) / sizeof(unsigned));
  k_gather_states<<<std::max(1, std::min(64, (count * W + 255) / 256)), 256, 0, s>>>(src, dst, count);
}

#define HELM_OUTER_INST(C)                                                                              \
  template void outer_residual<C>(int, const OuterDev<C>*, int, int, TileCfg, cudaStream_t);           \
  template void outer_apply_h<C>(int, const OuterDev<C>*, int, int, TileCfg, cudaStream_t);            \
  template void outer_dots<C>(const OuterDev<C>*, int, int, int, size_t, cudaStream_t);                \
  template void outer_vnew<C>(const OuterDev<C>*, int, int, int, bool, cudaStream_t);                  \
  template void outer_backsolve<C>(const OuterDev<C>*, int, cudaStream_t);                             \
  template void outer_solution<C>(const OuterDev<C>*, int, int, int, cudaStream_t);
HELM_OUTER_INST(float2)
HELM_OUTER_INST(double2)

}  // namespace helm
