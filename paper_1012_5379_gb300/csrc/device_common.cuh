// Device helpers: complex arithmetic on float2/double2, deterministic block and
// grid reductions, and the FP64 scalar algebra of one GMRES(s) smoothing sweep.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include "helm_internal.h"

namespace helm {

// ------------------------------------------------------------------ complex
template <typename C> struct CT;
template <> struct CT<float2> {
  typedef float R;
  __device__ __forceinline__ static float2 make(float a, float b) { return make_float2(a, b); }
};
template <> struct CT<double2> {
  typedef double R;
  __device__ __forceinline__ static double2 make(double a, double b) { return make_double2(a, b); }
};

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
// a * b
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a * b + c
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
// conj(a) * b + c
__device__ __forceinline__ float2 cdotacc(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(a.x, b.x, fmaf(a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(-a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 cdotacc(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, fma(a.y, b.y, c.x)), fma(a.x, b.y, fma(-a.y, b.x, c.y)));
}
__device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }
__device__ __forceinline__ double cabs2(double2 a) { return fma(a.x, a.x, a.y * a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

template <typename C> __device__ __forceinline__ C czero() { return CT<C>::make(0, 0); }
template <typename C> __device__ __forceinline__ C from_d(double2 v) {
  return CT<C>::make((typename CT<C>::R)v.x, (typename CT<C>::R)v.y);
}
__device__ __forceinline__ double2 to_d(float2 v) { return make_double2(v.x, v.y); }
__device__ __forceinline__ double2 to_d(double2 v) { return v; }

__device__ __forceinline__ double2 dconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double dabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double2 ddiv(double2 a, double2 b) {
  double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

__device__ __forceinline__ float2 shfl_up_c(float2 v, int d) {
  return make_float2(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d));
}
__device__ __forceinline__ double2 shfl_up_c(double2 v, int d) {
  return make_double2(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d));
}
__device__ __forceinline__ float2 shfl_down_c(float2 v, int d) {
  return make_float2(__shfl_down_sync(0xffffffffu, v.x, d), __shfl_down_sync(0xffffffffu, v.y, d));
}
__device__ __forceinline__ double2 shfl_down_c(double2 v, int d) {
  return make_double2(__shfl_down_sync(0xffffffffu, v.x, d), __shfl_down_sync(0xffffffffu, v.y, d));
}

// ------------------------------------------------------------------ reductions
__device__ __forceinline__ int flat_tid() { return threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z); }
__device__ __forceinline__ int block_threads() { return blockDim.x * blockDim.y * blockDim.z; }

// Sum NV doubles over the block in a fixed order; thread 0 ends with the totals.
// `sm` needs 32 * NV doubles.  Every thread of the block must call it.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sm) {
  const int tid = flat_tid(), lane = tid & 31, warp = tid >> 5, nw = (block_threads() + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) sm[warp * NV + i] = v[i];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = lane < nw ? sm[lane * NV + i] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int i = 0; i < NV; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  }
  __syncthreads();
}

// Write this block's NV partial sums to slot `tile`, then report whether this block
// is the last of `ntiles` blocks of its problem to arrive.  If so, the returned
// block reduces all slots in a fixed order (independent of arrival order) and
// thread 0 holds the totals in `tot`.
template <int NV>
__device__ __forceinline__ bool grid_sum_last(double (&v)[NV], double* part, int tile, int ntiles,
                                              unsigned int* counter, double* sm, double (&tot)[NV]) {
  __shared__ int s_last;
  block_sum<NV>(v, sm);
  const int tid = flat_tid();
  if (tid == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) part[(size_t)tile * NPART + i] = v[i];
    __threadfence();
    unsigned int prev = atomicAdd(counter, 1u);
    s_last = (prev == (unsigned)ntiles - 1u);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = 0.0;
  for (int t = tid; t < ntiles; t += block_threads())
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] += __ldcg(part + (size_t)t * NPART + i);
  block_sum<NV>(acc, sm);
#pragma unroll
  for (int i = 0; i < NV; ++i) tot[i] = acc[i];
  if (tid == 0) *counter = 0u;
  return true;
}

// ------------------------------------------------------------------ sweep algebra
// Breakdown threshold on ||w||^2 / ||p_J||^2 after projection: below it the
// Pythagorean norm is rounding noise of the working precision.
template <typename C> struct SweepTau;
template <> struct SweepTau<float2> { static constexpr double v = 1e-5; };
template <> struct SweepTau<double2> { static constexpr double v = 1e-24; };

// Start a sweep whose initial residual R_0 has squared norm beta2.
__device__ inline void sweep_begin(SweepScalars* sc, double beta2, int s) {
  sc->s = s;
  sc->beta2 = beta2;
  for (int i = 0; i <= SMAX; ++i) {
    sc->xcoef[i] = make_double2(0, 0);
    sc->rcoef[i] = make_double2(0, 0);
    for (int j = 0; j <= SMAX; ++j) {
      sc->G[i][j] = make_double2(0, 0);
      sc->Cf[i][j] = make_double2(0, 0);
    }
    for (int j = 0; j < SMAX; ++j) sc->Hh[i][j] = make_double2(0, 0);
  }
  sc->rcoef[0] = make_double2(1, 0);
  if (!isfinite(beta2)) {
    sc->status = 1;
    sc->m = 0;
    return;
  }
  if (!(beta2 > 0.0)) {
    sc->m = 0;
    return;
  }
  sc->m = s;
  sc->G[0][0] = make_double2(beta2, 0);
  sc->Cf[1][0] = make_double2(1.0 / sqrt(beta2), 0);
}

// min || beta e1 - Hbar y || for the (m+1) x m Hessenberg matrix, complex Givens.
__device__ inline void sweep_lstsq(const double2 (*Hh)[SMAX], int m, double beta, double2* y) {
  double2 R[SMAX + 1][SMAX];
  double2 g[SMAX + 1];
  for (int i = 0; i <= m; ++i) {
    g[i] = make_double2(i == 0 ? beta : 0.0, 0);
    for (int j = 0; j < m; ++j) R[i][j] = Hh[i][j];
  }
  for (int j = 0; j < m; ++j) {
    double2 a = R[j][j], b = R[j + 1][j];
    double na = sqrt(dabs2(a)), nb = sqrt(dabs2(b));
    double r = hypot(na, nb);
    double c;
    double2 s;
    if (r == 0.0) { c = 1.0; s = make_double2(0, 0); }
    else if (na == 0.0) { c = 0.0; s = make_double2(1, 0); }
    else {
      c = na / r;
      double2 ph = make_double2(a.x / na, a.y / na);
      s = cmul(ph, dconj(b));
      s = make_double2(s.x / r, s.y / r);
    }
    for (int l = j; l < m; ++l) {
      double2 t0 = R[j][l], t1 = R[j + 1][l];
      R[j][l] = cadd(make_double2(c * t0.x, c * t0.y), cmul(s, t1));
      R[j + 1][l] = csub(make_double2(c * t1.x, c * t1.y), cmul(dconj(s), t0));
    }
    double2 g0 = g[j];
    g[j] = make_double2(c * g0.x, c * g0.y);
    g[j + 1] = cmul(make_double2(-s.x, s.y), g0);  // -conj(s) g0
  }
  for (int j = m - 1; j >= 0; --j) {
    double2 acc = g[j];
    for (int l = j + 1; l < m; ++l) acc = csub(acc, cmul(R[j][l], y[l]));
    y[j] = (dabs2(R[j][j]) > 0.0) ? ddiv(acc, R[j][j]) : make_double2(0, 0);
  }
}

// After Arnoldi pass J: red[2k..2k+1] = <R_k, p_J> (k < J), red[2J] = ||p_J||^2.
__device__ inline void sweep_after_pass(SweepScalars* sc, int J, const double* red, double tau) {
  double2 g[SMAX];
  for (int k = 0; k < J; ++k) {
    g[k] = make_double2(red[2 * k], red[2 * k + 1]);
    sc->G[k][J] = g[k];
  }
  const double gg = red[2 * J];
  sc->G[J][J] = make_double2(gg, 0);
  double2 h[SMAX + 1];
  double hs = 0.0;
  for (int i = 1; i <= J; ++i) {
    double2 acc = make_double2(0, 0);
    for (int k = 0; k < i; ++k) acc = cadd(acc, cmul(dconj(sc->Cf[i][k]), g[k]));
    h[i] = acc;
    sc->Hh[i - 1][J - 1] = acc;
    hs += dabs2(acc);
  }
  if (!isfinite(gg) || !isfinite(hs)) sc->status = 1;
  const double w2 = gg - hs;
  const double hn = w2 > 0.0 ? sqrt(w2) : 0.0;
  sc->Hh[J][J - 1] = make_double2(hn, 0);
  const bool breakdown = !(w2 > tau * gg);
  if (breakdown || J == sc->s) {
    const int m = J;
    sc->m = m;
    double2 y[SMAX];
    sweep_lstsq(sc->Hh, m, sqrt(sc->beta2), y);
    for (int k = 0; k <= SMAX; ++k) { sc->xcoef[k] = make_double2(0, 0); sc->rcoef[k] = make_double2(0, 0); }
    for (int jj = 1; jj <= m; ++jj)
      for (int k = 0; k < jj; ++k) sc->xcoef[k] = cadd(sc->xcoef[k], cmul(y[jj - 1], sc->Cf[jj][k]));
    sc->rcoef[0] = make_double2(1, 0);
    for (int jj = 1; jj <= m; ++jj) sc->rcoef[jj] = make_double2(-y[jj - 1].x, -y[jj - 1].y);
  } else {
    const double inv = 1.0 / hn;
    for (int k = 0; k < J; ++k) {
      double2 acc = make_double2(0, 0);
      for (int i = k + 1; i <= J; ++i) acc = cadd(acc, cmul(h[i], sc->Cf[i][k]));
      sc->Cf[J + 1][k] = make_double2(-acc.x * inv, -acc.y * inv);
    }
    sc->Cf[J + 1][J] = make_double2(inv, 0);
  }
}

}  // namespace helm
