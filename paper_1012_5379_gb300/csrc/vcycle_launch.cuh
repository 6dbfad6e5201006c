// Host launchers of the V-cycle kernels, instantiated once per precision in
// vcycle_c64.cu and vcycle_c128.cu (two translation units compile in parallel).
#pragma once
#include "tiles.cuh"
#include <algorithm>
#include <type_traits>
#include "../../include/helm.h"
#include "poly.h"

namespace helm {

// Launch with programmatic stream serialisation: the kernel may start while its
// predecessor finishes and synchronises with it through griddepcontrol.wait.  The
// passes that end in a grid reduction signal their dependents only after their main
// work, so waiting dependents never hold SM slots the predecessor's later waves need;
// the launch latency and the dependent's prologue then overlap the predecessor's
// reduction tail.
static inline int sm_count() {
  // initialised once, thread-safely (serving and callers' threads launch concurrently)
  static const int n = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 1;
    return v;
  }();
  return n;
}
template <typename... KArgs, typename... Args>
static inline void pdl_launch(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// Tiles per CTA of a 2D pass for one problem of `ntiles` tiles: each CTA pays a fixed
// cost (its reduction, the atomic, the ramp; about half a tile's time on GB300) plus
// the cost of its tiles, so t tiles per CTA take ceil(ntiles / (t slots)) rounds of
// (1/2 + t) tile times; the smallest such t up to 8 wins.  A function of the level size and of the kernel's
// residency on the device only (it fixes the order of the pass's partial sums).
template <typename K>
static int tiles_per_cta(K kernel, int ntiles, size_t smem = 0) {
  static thread_local K last_kernel = nullptr;
  static thread_local int slots = 0;
  if (kernel != last_kernel) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, smem) != cudaSuccess || per_sm < 1)
      per_sm = 1;
    slots = per_sm * sm_count();
    last_kernel = kernel;
  }
  int best = 1;
  long long best_cost = -1;
  for (int t = 1; t <= 8; t *= 2) {
    const long long rounds = (ntiles + (long long)t * slots - 1) / ((long long)t * slots);
    const long long cost = rounds * (1 + 2 * t);
    if (best_cost < 0 || cost < best_cost) { best = t; best_cost = cost; }
  }
  return best;
}

constexpr int TMA_MIN_TILES = 16384;  // 2D levels of 4095^2 and larger

template <int J>
static void arnoldi_tma2(const LevelDev<float2>* levs, int nprob, int ntiles, bool r0_is_b, bool store_p,
                         cudaStream_t st) {
  const size_t smem = tma_arnoldi_smem(J);
  thread_local bool configured = false;  // the attribute is per function; setting it again is harmless
  if (!configured) {
    cudaFuncSetAttribute(k_arnoldi_tma2<J>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured = true;
  }
  const int t = tiles_per_cta(k_arnoldi_tma2<J>, ntiles, smem);
  pdl_launch(k_arnoldi_tma2<J>, dim3(nprob * ceil_div(ntiles, t)), dim3(32, 8), smem, st, levs, ntiles, t,
             r0_is_b ? 1 : 0, store_p ? 1 : 0);
}

template <typename C, int J>
static void arnoldi_J(int dim, const LevelDev<C>* levs, int grid, int ntiles, TileCfg cfg, bool r0_is_b,
                      bool store_p, bool tma, cudaStream_t st) {
  if constexpr (std::is_same<C, float2>::value) {
    // the TMA pipeline pays off on levels that stream from HBM; smaller levels are
    // latency-bound and L2-resident
    if (dim == 2 && tma && ntiles >= TMA_MIN_TILES) {
      arnoldi_tma2<J>(levs, grid / ntiles, ntiles, r0_is_b, store_p, st);
      return;
    }
  }
  if (dim == 2) {
    const int t = tiles_per_cta(k_arnoldi_t2<C, J>, ntiles);
    pdl_launch(k_arnoldi_t2<C, J>, dim3(grid / ntiles * ceil_div(ntiles, t)), dim3(dim3(32, 8)), 0, st, levs, ntiles, t,
               r0_is_b, store_p);
  }
  else
    pdl_launch(k_arnoldi_t3<C, J>, dim3(grid), dim3(dim3(32, 8)), 0, st, levs, ntiles, cfg.rows, r0_is_b, store_p);
}

template <typename C>
void launch_arnoldi(int dim, int J, const LevelDev<C>* levs, int nprob, int ntiles, TileCfg cfg, bool r0_is_b,
                    bool store_p, bool tma, cudaStream_t st) {
  const int grid = nprob * ntiles;
  switch (J) {
    case 1: arnoldi_J<C, 1>(dim, levs, grid, ntiles, cfg, r0_is_b, store_p, tma, st); break;
    case 2: arnoldi_J<C, 2>(dim, levs, grid, ntiles, cfg, r0_is_b, store_p, tma, st); break;
    case 3: arnoldi_J<C, 3>(dim, levs, grid, ntiles, cfg, r0_is_b, store_p, tma, st); break;
    default: arnoldi_J<C, 4>(dim, levs, grid, ntiles, cfg, r0_is_b, store_p, tma, st); break;
  }
}

template <typename C>
void launch_restrict(int dim, const LevelDev<C>* levs, int nprob, int ntiles, TileCfg cfg, bool r0_is_b,
                     bool x_from_zero, bool nosmooth, cudaStream_t st) {
  if (dim == 2)
    pdl_launch(k_restrict_t2<C>, dim3(nprob * ceil_div(ntiles, tiles_per_cta(k_restrict_t2<C>, ntiles))),
               dim3(dim3(32, 8)), 0, st, levs, ntiles, tiles_per_cta(k_restrict_t2<C>, ntiles), r0_is_b, x_from_zero,
               nosmooth);
  else
    pdl_launch(k_restrict_t3<C>, dim3(nprob * ntiles), dim3(dim3(32, 8)), 0, st, levs, ntiles, cfg.rows, r0_is_b, x_from_zero, nosmooth);
}

template <typename C>
void launch_update_flat(int dim, UpdateMode mode, const LevelDev<C>* levs, int nprob, int ntiles, bool r0_is_b,
                        int xsel, bool x_from_zero, cudaStream_t st) {
  pdl_launch(k_update_flat<C>, dim3(nprob * ntiles), dim3(256), 0, st, levs, ntiles, dim, (int)mode, r0_is_b, xsel, x_from_zero);
}

template <typename C>
void launch_prolong(int dim, bool with_residual, const LevelDev<C>* levs, int nprob, int ntiles, TileCfg cfg,
                    cudaStream_t st) {
  if (!with_residual) {
    pdl_launch(k_prolong_flat<C>, dim3(nprob * ntiles), dim3(256), 0, st, levs, ntiles, dim);
  } else if (dim == 2) {
    pdl_launch(k_prolong_t2<C>, dim3(nprob * ceil_div(ntiles, tiles_per_cta(k_prolong_t2<C>, ntiles))),
               dim3(dim3(32, 8)), 0, st, levs, ntiles, tiles_per_cta(k_prolong_t2<C>, ntiles));
  } else {
    pdl_launch(k_prolong_t3<C>, dim3(nprob * ntiles), dim3(dim3(32, 8)), 0, st, levs, ntiles, cfg.rows);
  }
}

template <typename C>
void launch_coarse(int dim, const LevelDev<C>* levs, int nlev, int lev_stride, const CoarseLU* lus, int nprob,
                   int nu1, int nu2, cudaStream_t st) {
  pdl_launch(k_coarse<C>, dim3(nprob), dim3(512), 0, st, levs, nlev, lev_stride, lus, nu1, nu2, dim);
}

template <typename C>
void launch_coarse_smem(int dim, const LevelDev<C>* levs, int nlev, int lev_stride, const CoarseLU* lus, int nprob,
                        int nu1, int nu2, size_t smem_bytes, cudaStream_t st) {
  // the static part (descriptors, sweep scalars) counts against the same limit: allow
  // the largest dynamic part the device offers, once per host thread
  thread_local bool configured = false;
  if (!configured) {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (cudaFuncGetAttributes(&fa, k_coarse_smem<C>) == cudaSuccess && optin > (int)fa.sharedSizeBytes)
      cudaFuncSetAttribute(k_coarse_smem<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    configured = true;
  }
  pdl_launch(k_coarse_smem<C>, dim3(nprob), dim3(512), smem_bytes, st, levs, nlev, lev_stride, lus, nu1, nu2, dim);
}

// Cluster size of the coarse sub-cycle: the largest power of two up to CLUSTER_MAX
// that the device can make resident (a constant of the device, so a problem's result
// does not depend on the other problems of its launch).
template <typename C>
static int coarse_cluster_size() {
  // the largest cluster the device can place, found once (thread-safe initialisation)
  static const int csize = [] {
    cudaFuncSetAttribute(k_coarse_cluster<C>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    int found = 0;
    for (int c = CLUSTER_MAX; c >= 1 && found == 0; c >>= 1) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(c);
      cfg.blockDim = dim3(CLUSTER_THREADS);
      cudaLaunchAttribute at;
      at.id = cudaLaunchAttributeClusterDimension;
      at.val.clusterDim.x = c;
      at.val.clusterDim.y = 1;
      at.val.clusterDim.z = 1;
      cfg.attrs = &at;
      cfg.numAttrs = 1;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, k_coarse_cluster<C>, &cfg) == cudaSuccess && nclusters > 0)
        found = c;
    }
    cudaGetLastError();
    return found == 0 ? 1 : found;
  }();
  return csize;
}

template <typename C>
void launch_coarse_cluster(int dim, const LevelDev<C>* levs, int lev_stride, const CoarseLU* lus, int nprob,
                           int nu1, int nu2, cudaStream_t st) {
  const int c = coarse_cluster_size<C>();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nprob * c);
  cfg.blockDim = dim3(CLUSTER_THREADS);
  cfg.stream = st;
  cudaLaunchAttribute at;
  at.id = cudaLaunchAttributeClusterDimension;
  at.val.clusterDim.x = c;
  at.val.clusterDim.y = 1;
  at.val.clusterDim.z = 1;
  cfg.attrs = &at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_coarse_cluster<C>, levs, lev_stride, lus, nu1, nu2, dim);
}

template <typename C>
void launch_load_input(int dim, const LevelDev<C>* levs, int ntiles, const void* src, int in_prec, cudaStream_t st) {
  if (in_prec == HELM_C128)
    pdl_launch(k_load_input<double2, C>, dim3(ntiles), dim3(256), 0, st, levs, ntiles, dim, (const double2*)src);
  else
    pdl_launch(k_load_input<float2, C>, dim3(ntiles), dim3(256), 0, st, levs, ntiles, dim, (const float2*)src);
}

template <typename C>
void launch_store_output(int dim, int n, const LevelDev<C>* levs, void* dst, int out_prec, cudaStream_t st) {
  const size_t npts = dim == 3 ? (size_t)n * n * n : (size_t)n * n;
  const int grid = (int)std::min<size_t>((npts + 255) / 256, 4096);
  if (out_prec == HELM_C128)
    pdl_launch(k_store_output<C, double2>, dim3(grid), dim3(256), 0, st, levs, dim, (double2*)dst);
  else
    pdl_launch(k_store_output<C, float2>, dim3(grid), dim3(256), 0, st, levs, dim, (float2*)dst);
}

template <typename C>
void launch_poly_step(int dim, const LevelDev<C>* levs, const C* pw, int nprob, int nflat, int src, int dst,
                      int wsel, cudaStream_t st) {
  pdl_launch(k_poly_step<C>, dim3(nprob * nflat), dim3(256), 0, st, levs, pw, nflat, dim, src, dst, wsel);
}

template <typename C>
void launch_poly_restrict(int dim, const LevelDev<C>* levs, int nprob, int nflat, int src, cudaStream_t st) {
  pdl_launch(k_poly_residual<C>, dim3(nprob * nflat), dim3(256), 0, st, levs, nflat, dim, src);
  pdl_launch(k_poly_fw<C>, dim3(nprob * nflat), dim3(256), 0, st, levs, nflat, dim);
}

#define HELM_VCYCLE_INST(C)                                                                                   \
  template void launch_arnoldi<C>(int, int, const LevelDev<C>*, int, int, TileCfg, bool, bool, bool, cudaStream_t); \
  template void launch_restrict<C>(int, const LevelDev<C>*, int, int, TileCfg, bool, bool, bool,           \
                                    cudaStream_t);                                                          \
  template void launch_update_flat<C>(int, UpdateMode, const LevelDev<C>*, int, int, bool, int, bool,         \
                                      cudaStream_t);                                                          \
  template void launch_prolong<C>(int, bool, const LevelDev<C>*, int, int, TileCfg, cudaStream_t);            \
  template void launch_coarse<C>(int, const LevelDev<C>*, int, int, const CoarseLU*, int, int, int,           \
                                 cudaStream_t);                                                               \
  template void launch_coarse_smem<C>(int, const LevelDev<C>*, int, int, const CoarseLU*, int, int, int, size_t, \
                                      cudaStream_t);                                                          \
  template void launch_coarse_cluster<C>(int, const LevelDev<C>*, int, const CoarseLU*, int, int, int,       \
                                         cudaStream_t);                                                       \
  template void launch_load_input<C>(int, const LevelDev<C>*, int, const void*, int, cudaStream_t);           \
  template void launch_store_output<C>(int, int, const LevelDev<C>*, void*, int, cudaStream_t);              \
  template void launch_poly_step<C>(int, const LevelDev<C>*, const C*, int, int, int, int, int, cudaStream_t); \
  template void launch_poly_restrict<C>(int, const LevelDev<C>*, int, int, int, cudaStream_t);

}  // namespace helm
