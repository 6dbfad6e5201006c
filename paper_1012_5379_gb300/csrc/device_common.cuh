// Device helpers: complex arithmetic on float2/double2, deterministic block and
// grid reductions, and the scalar algebra of one GMRES(s) smoothing sweep.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stddef.h>
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
// c - a * b in four FMAs
__device__ __forceinline__ double2 cfms(double2 a, double2 b, double2 c) {
  return make_double2(fma(-a.x, b.x, fma(a.y, b.y, c.x)), fma(-a.x, b.y, fma(-a.y, b.x, c.y)));
}
__device__ __forceinline__ float2 cfms(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(-a.x, b.x, fmaf(a.y, b.y, c.x)), fmaf(-a.x, b.y, fmaf(-a.y, b.x, c.y)));
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
// binary32 -> binary64 widening (exact) on the integer pipes: the sign is kept, the
// exponent re-biased by 1023 - 127 = 896 and the 23 fraction bits moved to the top of
// the 52-bit field.  Zero, subnormals, infinities and NaNs take the converting
// instruction, which on this part issues to the FP64 pipe (the bound of the outer
// passes); normal numbers need none.
__device__ __forceinline__ double widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if (e - 1u >= 254u) return (double)f;
  const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u >> 3) & 0xfffffu);
  return __hiloint2double((int)hi, (int)(u << 29));
}
__device__ __forceinline__ double2 to_d(float2 v) { return make_double2(widen(v.x), widen(v.y)); }
__device__ __forceinline__ double2 to_d(double2 v) { return v; }
// Change of complex type (exact unless it narrows).
template <typename Cout> __device__ __forceinline__ Cout to_c(float2 v);
template <> __device__ __forceinline__ float2 to_c<float2>(float2 v) { return v; }
template <> __device__ __forceinline__ double2 to_c<double2>(float2 v) { return to_d(v); }
template <typename Cout> __device__ __forceinline__ Cout to_c(double2 v) { return from_d<Cout>(v); }

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

// ------------------------------------------------------------------ dependent launch
// Programmatic dependent launch: a kernel lets the next kernel in the stream start
// launching at once (its CTAs then run their prologue), and waits for the previous
// kernel's completion and memory before reading anything that kernel wrote.  Both
// are no-ops for a kernel launched without the programmatic attribute.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ------------------------------------------------------------------ TMA and mbarriers
// Error flag of the V-cycle kernels: set when a bounded wait ran out (each
// translation unit has its own; the host reads the complex64 one after a solve).
static __device__ int g_vcycle_error = 0;

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// Make initialised barriers visible to the async (TMA) proxy.
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n\tfence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
// Non-blocking test of the phase `parity` of a barrier.
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for the phase `parity` of a barrier for at most one second (wall clock, and at
// most 2^24 polls): false if it did not complete.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  if (mbar_test_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  for (int it = 0; it < (1 << 24); ++it) {
    __nanosleep(32);
    if (mbar_test_wait(bar, parity)) return true;
    if ((it & 255) == 255 && globaltimer_ns() - t0 > 1000000000ull) return false;
  }
  return false;
}
__device__ __forceinline__ void tmap_acquire(const CUtensorMap* tm) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tm) : "memory");
}
// 2D tiled TMA load of the box at element coordinates (c0, c1) into shared memory,
// completing on `bar`.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int c0, int c1, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_addr(dst)), "l"(tm), "r"(c0), "r"(c1), "r"(smem_addr(bar))
      : "memory");
}

// 3D tiled TMA load of the box at element coordinates (c0, c1, c2).
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int c0, int c1, int c2, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_addr(dst)), "l"(tm), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
      : "memory");
}

// ------------------------------------------------------------------ reductions
__device__ __forceinline__ int flat_tid() { return threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z); }
__device__ __forceinline__ int block_threads() { return blockDim.x * blockDim.y * blockDim.z; }

// Sum NV doubles over the block in a fixed order; thread 0 ends with the totals.
// `sm` needs 32 * NV doubles.  Every thread of the block must call it.
template <int NV, typename T>
__device__ __forceinline__ void block_sum(T (&v)[NV], T* sm) {
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
    for (int i = 0; i < NV; ++i) v[i] = lane < nw ? sm[lane * NV + i] : (T)0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int i = 0; i < NV; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  }
  __syncthreads();
}

// Per-thread sums of the partial slots t = tid, tid + threads, ... in a fixed order;
// four slots' loads are in flight before their adds.
template <int NV, typename T>
__device__ __forceinline__ void sum_partials(const T* part, int ntiles, T (&acc)[NV]) {
  const int tid = flat_tid(), nt = block_threads();
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = (T)0;
  for (int t0 = tid; t0 < ntiles; t0 += 4 * nt) {
    T v[4][NV];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int t = t0 + u * nt;
#pragma unroll
      for (int i = 0; i < NV; ++i) v[u][i] = t < ntiles ? __ldcg(part + (size_t)t * NPART + i) : (T)0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int i = 0; i < NV; ++i) acc[i] += v[u][i];
  }
}

// Write this block's NV partial sums to slot `tile`, then report whether this block
// is the last of `ntiles` blocks of its problem to arrive.  If so, the returned
// block reduces all slots in a fixed order (independent of arrival order) and
// thread 0 holds the totals in `tot`.
// Partial slots, the block sums and the final sum are all in T: FP32 for the
// complex64 V-cycle, FP64 elsewhere.
template <int NV, typename T>
__device__ __forceinline__ bool grid_sum_last(T (&v)[NV], void* partv, int tile, int ntiles,
                                              unsigned int* counter, T* sm, T (&tot)[NV]) {
  __shared__ int s_last;
  T* part = reinterpret_cast<T*>(partv);
  block_sum<NV, T>(v, sm);
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
  T acc[NV];
  sum_partials<NV, T>(part, ntiles, acc);
  block_sum<NV, T>(acc, sm);
#pragma unroll
  for (int i = 0; i < NV; ++i) tot[i] = acc[i];
  if (tid == 0) *counter = 0u;
  return true;
}

// ------------------------------------------------------------------ sweep algebra
// Breakdown threshold on ||w||^2 / ||p_J||^2 after projection: below it the
// Pythagorean norm is rounding noise of the working precision.
template <typename T> struct SweepTau;
template <> struct SweepTau<float> { static constexpr float v = 1e-5f; };
template <> struct SweepTau<double> { static constexpr double v = 1e-24; };

__device__ __forceinline__ float2 fconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ double2 fconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ float fabs2(float2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double fabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ float2 fdiv(float2 a, float2 b) {
  const float d = 1.0f / (b.x * b.x + b.y * b.y);
  return make_float2((a.x * b.x + a.y * b.y) * d, (a.y * b.x - a.x * b.y) * d);
}
__device__ __forceinline__ double2 fdiv(double2 a, double2 b) { return ddiv(a, b); }

template <typename T>
__device__ __forceinline__ int sweep_words() {
  return (int)(offsetof(SweepScalarsT<T>, counter) / sizeof(int));
}

// Start a sweep whose initial residual R_0 has squared norm beta2.  Only the fields
// a sweep reads before writing are set (one thread).
template <typename T>
__device__ inline void sweep_begin(SweepScalarsT<T>* sc, T beta2, int s) {
  typedef typename CplxOf<T>::T CR;
  sc->s = s;
  sc->beta2 = beta2;
  sc->rcoef[0] = CT<CR>::make(1, 0);
  if (!isfinite(beta2)) {
    sc->status = 1;
    sc->m = 0;
    return;
  }
  if (!(beta2 > (T)0)) {
    sc->m = 0;
    return;
  }
  sc->m = s;
  sc->Cf[1][0] = CT<CR>::make((T)1 / sqrt(beta2), 0);
}

// The sweep algebra works on register copies: every field it reads is loaded before
// anything is computed (one memory latency instead of a chain), and the results are
// stored at the end.

// min || beta e1 - Hbar y || for the (M+1) x M Hessenberg matrix hh, complex Givens.
// M is a compile-time constant so every array stays in registers.
template <typename T, int M>
__device__ __forceinline__ void sweep_lstsq(const typename CplxOf<T>::T (&hh)[SMAX + 1][SMAX], T beta,
                                            typename CplxOf<T>::T* y) {
  typedef typename CplxOf<T>::T CR;
  CR R[M + 1][M];
  CR g[M + 1];
#pragma unroll
  for (int i = 0; i <= M; ++i) {
    g[i] = CT<CR>::make(i == 0 ? beta : (T)0, 0);
#pragma unroll
    for (int j = 0; j < M; ++j) R[i][j] = (i <= j + 1) ? hh[i][j] : CT<CR>::make(0, 0);
  }
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const CR a = R[j][j], b = R[j + 1][j];
    const T na = sqrt(fabs2(a)), nb = sqrt(fabs2(b));
    const T r = sqrt(na * na + nb * nb);
    T c;
    CR s;
    if (r == (T)0) { c = 1; s = CT<CR>::make(0, 0); }
    else if (na == (T)0) { c = 0; s = CT<CR>::make(1, 0); }
    else {
      const T inv_na = (T)1 / na, inv_r = (T)1 / r;
      c = na * inv_r;
      s = cmul(CT<CR>::make(a.x * inv_na, a.y * inv_na), fconj(b));
      s = CT<CR>::make(s.x * inv_r, s.y * inv_r);
    }
#pragma unroll
    for (int l = j; l < M; ++l) {
      const CR t0 = R[j][l], t1 = R[j + 1][l];
      R[j][l] = cadd(CT<CR>::make(c * t0.x, c * t0.y), cmul(s, t1));
      R[j + 1][l] = csub(CT<CR>::make(c * t1.x, c * t1.y), cmul(fconj(s), t0));
    }
    const CR g0 = g[j];
    g[j] = CT<CR>::make(c * g0.x, c * g0.y);
    g[j + 1] = cmul(CT<CR>::make(-s.x, s.y), g0);  // -conj(s) g0
  }
#pragma unroll
  for (int j = M - 1; j >= 0; --j) {
    CR acc = g[j];
#pragma unroll
    for (int l = j + 1; l < M; ++l) acc = csub(acc, cmul(R[j][l], y[l]));
    y[j] = (fabs2(R[j][j]) > (T)0) ? fdiv(acc, R[j][j]) : CT<CR>::make(0, 0);
  }
}

// Least-squares solution of the sweep and its update coefficients over the raw
// vectors: x += sum_{k<M} xcoef[k] R_k, r = sum_{k<=M} rcoef[k] R_k.
template <typename T, int M>
__device__ __forceinline__ void sweep_finish(SweepScalarsT<T>* sc, const typename CplxOf<T>::T (&hh)[SMAX + 1][SMAX],
                                             const typename CplxOf<T>::T (&cf)[SMAX + 1][SMAX], T beta2) {
  typedef typename CplxOf<T>::T CR;
  CR y[M];
  sweep_lstsq<T, M>(hh, sqrt(beta2), y);
  CR xc[SMAX + 1], rc[SMAX + 1];
#pragma unroll
  for (int k = 0; k <= SMAX; ++k) { xc[k] = CT<CR>::make(0, 0); rc[k] = CT<CR>::make(0, 0); }
#pragma unroll
  for (int k = 0; k < M; ++k) {
    CR acc = CT<CR>::make(0, 0);
#pragma unroll
    for (int jj = k + 1; jj <= M; ++jj) acc = cadd(acc, cmul(y[jj - 1], cf[jj][k]));
    xc[k] = acc;
  }
  rc[0] = CT<CR>::make(1, 0);
#pragma unroll
  for (int jj = 1; jj <= M; ++jj) rc[jj] = CT<CR>::make(-y[jj - 1].x, -y[jj - 1].y);
  sc->m = M;
#pragma unroll
  for (int k = 0; k <= SMAX; ++k) { sc->xcoef[k] = xc[k]; sc->rcoef[k] = rc[k]; }
}

// After Arnoldi pass J: red[2k..2k+1] = <R_k, p_J> (k < J), red[2J] = ||p_J||^2.
// Works on `sc` in any memory space (the kernels pass a shared-memory copy).
template <typename T, int J>
__device__ __forceinline__ void sweep_after_pass(SweepScalarsT<T>* sc, const T* red) {
  typedef typename CplxOf<T>::T CR;
  // every field the algebra reads, loaded first
  CR cf[SMAX + 1][SMAX], hh[SMAX + 1][SMAX];
#pragma unroll
  for (int i = 1; i <= J; ++i)
#pragma unroll
    for (int k = 0; k < i; ++k) cf[i][k] = sc->Cf[i][k];
#pragma unroll
  for (int j = 0; j + 1 < J; ++j)
#pragma unroll
    for (int i = 0; i <= j + 1; ++i) hh[i][j] = sc->Hh[i][j];
  const int s = sc->s;
  const T beta2 = sc->beta2;
  CR g[J];
#pragma unroll
  for (int k = 0; k < J; ++k) g[k] = CT<CR>::make(red[2 * k], red[2 * k + 1]);
  const T gg = red[2 * J];
  CR h[J + 1];
  T hs = 0;
#pragma unroll
  for (int i = 1; i <= J; ++i) {
    CR acc = CT<CR>::make(0, 0);
#pragma unroll
    for (int k = 0; k < i; ++k) acc = cadd(acc, cmul(fconj(cf[i][k]), g[k]));
    h[i] = acc;
    hh[i - 1][J - 1] = acc;
    hs += fabs2(acc);
  }
  if (!isfinite(gg) || !isfinite(hs)) sc->status = 1;
  const T w2 = gg - hs;
  const T hn = w2 > (T)0 ? sqrt(w2) : (T)0;
  hh[J][J - 1] = CT<CR>::make(hn, 0);
  const bool breakdown = !(w2 > SweepTau<T>::v * gg);
  if (breakdown || J == s) {
    sweep_finish<T, J>(sc, hh, cf, beta2);
  } else if (J < SMAX) {
    const T inv = (T)1 / hn;
    CR cn[J + 1];
#pragma unroll
    for (int k = 0; k < J; ++k) {
      CR acc = CT<CR>::make(0, 0);
#pragma unroll
      for (int i = k + 1; i <= J; ++i) acc = cadd(acc, cmul(h[i], cf[i][k]));
      cn[k] = CT<CR>::make(-acc.x * inv, -acc.y * inv);
    }
    cn[J] = CT<CR>::make(inv, 0);
#pragma unroll
    for (int i = 0; i <= J; ++i) sc->Hh[i][J - 1] = hh[i][J - 1];
#pragma unroll
    for (int k = 0; k <= J; ++k) sc->Cf[J + 1][k] = cn[k];
  }
}

// Runtime-J dispatch (coarse single-CTA cycle).
template <typename T>
__device__ inline void sweep_after_pass_rt(SweepScalarsT<T>* sc, int J, const T* red) {
  switch (J) {
    case 1: sweep_after_pass<T, 1>(sc, red); break;
    case 2: sweep_after_pass<T, 2>(sc, red); break;
    case 3: sweep_after_pass<T, 3>(sc, red); break;
    default: sweep_after_pass<T, 4>(sc, red); break;
  }
}

// End of an Arnoldi pass: publish this block's sums; the last block of the problem
// loads the sweep state and all partial sums with their loads in flight together,
// runs the algebra on one thread in shared memory and writes the state back.  Every
// thread of the block must call it.
template <typename T, int J>
__device__ inline void grid_sum_sweep(T (&v)[2 * J + 1], void* partv, int tile, int ntiles,
                                      SweepScalarsT<T>* sc, T* sm) {
  constexpr int NV = 2 * J + 1;
  constexpr int WPT = 2;  // sweep-state words per thread (the state is < 2 x 256 words)
  __shared__ int s_last;
  __shared__ SweepScalarsT<T> ls;
  __shared__ T stot[NV];
  T* part = reinterpret_cast<T*>(partv);
  block_sum<NV, T>(v, sm);
  const int tid = flat_tid(), nt = block_threads();
  if (tid == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) part[(size_t)tile * NPART + i] = v[i];
    __threadfence();
    s_last = (atomicAdd(&sc->counter, 1u) == (unsigned)ntiles - 1u);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  int* gsrc = reinterpret_cast<int*>(sc);
  int* sdst = reinterpret_cast<int*>(&ls);
  const int words = sweep_words<T>();
  int w[WPT];
#pragma unroll
  for (int q = 0; q < WPT; ++q) w[q] = tid + q * nt < words ? __ldcg(gsrc + tid + q * nt) : 0;
  T acc[NV];
  sum_partials<NV, T>(part, ntiles, acc);
#pragma unroll
  for (int q = 0; q < WPT; ++q)
    if (tid + q * nt < words) sdst[tid + q * nt] = w[q];
  block_sum<NV, T>(acc, sm);
  if (tid == 0) {
    sc->counter = 0u;
#pragma unroll
    for (int i = 0; i < NV; ++i) stot[i] = acc[i];
    sweep_after_pass<T, J>(&ls, stot);
  }
  __syncthreads();
  for (int i = tid; i < words; i += nt) gsrc[i] = sdst[i];
}

}  // namespace helm
