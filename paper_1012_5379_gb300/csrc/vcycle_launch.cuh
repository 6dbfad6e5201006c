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
static void arnoldi_tma2(const LevelDev<float2>* levs, int nprob, int ntiles, int P, bool r0_is_b, bool store_p,
                         cudaStream_t st) {
  const size_t smem = tma_arnoldi_smem(J);
  thread_local bool configured = false;  // the attribute is per function; setting it again is harmless
  if (!configured) {
    cudaFuncSetAttribute(k_arnoldi_tma2<J>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured = true;
  }
  const int t = tuned_tpc(TP_ARNOLDI, P, 8, J, tiles_per_cta(k_arnoldi_tma2<J>, ntiles, smem));
  pdl_launch(k_arnoldi_tma2<J>, dim3(nprob * ceil_div(ntiles, t)), dim3(32, 8), smem, st, levs, ntiles, t,
             r0_is_b ? 1 : 0, store_p ? 1 : 0);
}

// The 3D TMA-fed Arnoldi pass: planes per z-march, plane slots in flight and tiles per
// CTA of a level of pitch P (tuned table, else these defaults).

template <int J, int QY, bool RESID>
static void stencil_tma3_q(const LevelDev<float2>* levs, int nprob, int P, const Tma3Params& tp, bool r0_is_b,
                           bool store_p, cudaStream_t st) {
  const size_t smem = tma3_arnoldi_smem(J, QY, tp.stages);
  // per host thread: the largest dynamic shared memory set so far, and the residency
  // of the last configuration
  thread_local size_t configured = 0;
  thread_local int occ_stages = -1, occ = 1;
  if (configured < smem) {
    cudaFuncSetAttribute(k_stencil_tma3<J, QY, RESID>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured = smem;
  }
  if (occ_stages != tp.stages) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_stencil_tma3<J, QY, RESID>, 256, smem) != cudaSuccess ||
        occ < 1)
      occ = 1;
    occ_stages = tp.stages;
  }
  // shares of the level's (column, plane) sequence: column pieces, or one per resident
  // CTA (a function of the level size and the device only: it fixes the order of the
  // partial sums)
  const long long cols = tma3_cols(P, QY);
  long long units = tp.pieces > 0 ? cols * std::min(tp.pieces, P) : (long long)occ * sm_count();
  units = std::max<long long>(1, std::min<long long>(units, std::min<long long>(TMA3_MAX_UNITS, cols * P)));
  const int nunits = (int)units;
  pdl_launch(k_stencil_tma3<J, QY, RESID>, dim3(nprob * nunits), dim3(32, 8), smem, st, levs, nunits, tp.stages,
             r0_is_b ? 1 : 0, store_p ? 1 : 0);
}

template <int J>
static void arnoldi_tma3(const LevelDev<float2>* levs, int nprob, int P, bool r0_is_b, bool store_p,
                         cudaStream_t st) {
  const Tma3Params tp = tma3_params(TP_ARNOLDI, J, P);
  if constexpr (J <= 2) {
    if (tp.qy == 4) {
      stencil_tma3_q<J, 4, false>(levs, nprob, P, tp, r0_is_b, store_p, st);
      return;
    }
  }
  stencil_tma3_q<J, 2, false>(levs, nprob, P, tp, r0_is_b, store_p, st);
}

// Coarse correction and post-smoothing residual of a 3D complex64 level in two passes:
// x_b = x_a + P e_c row by row, then r0 = b - M x_b with x_b streamed by TMA.
static void prolong_tma3(const LevelDev<float2>* levs, int nprob, int P, cudaStream_t st) {
  const Tma3Params tp = tma3_params(TP_PROLONG, 0, P);
  const int nblk = std::max(1, std::min(8 * sm_count() / std::max(nprob, 1), (P / PR_ROWS) * P));
  if (P <= 256)
    pdl_launch(k_prolong3_rows<float2, 1>, dim3(nprob * nblk), dim3(256), 0, st, levs, nblk);
  else if (P <= 512)
    pdl_launch(k_prolong3_rows<float2, 2>, dim3(nprob * nblk), dim3(256), 0, st, levs, nblk);
  else
    pdl_launch(k_prolong3_rows<float2, 4>, dim3(nprob * nblk), dim3(256), 0, st, levs, nblk);
  if (tp.qy == 4)
    stencil_tma3_q<1, 4, true>(levs, nprob, P, tp, false, false, st);
  else
    stencil_tma3_q<1, 2, true>(levs, nprob, P, tp, false, false, st);
}

template <typename C, int J>
static void arnoldi_J(int dim, const LevelDev<C>* levs, int grid, int ntiles, TileCfg cfg, bool r0_is_b,
                      bool store_p, bool tma, cudaStream_t st) {
  if constexpr (std::is_same<C, float2>::value) {
    // the TMA pipeline pays off on levels that stream from HBM; smaller levels are
    // latency-bound and L2-resident
    if (dim == 2 && tma && ntiles >= TMA_MIN_TILES) {
      arnoldi_tma2<J>(levs, grid / ntiles, ntiles, cfg.P, r0_is_b, store_p, st);
      return;
    }
    if (dim == 3 && tma && cfg.P >= TMA3_MIN_P && cfg.P <= TMA3_MAX_P && tma3_params(TP_ARNOLDI, J, cfg.P).enabled) {
      arnoldi_tma3<J>(levs, grid / ntiles, cfg.P, r0_is_b, store_p, st);
      return;
    }
  }
  if (dim == 2) {
    const int t = tuned_tpc(TP_ARNOLDI, cfg.P, (int)sizeof(C), J, tiles_per_cta(k_arnoldi_t2<C, J>, ntiles));
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

// The TMA-fed 3D restriction (complex64 levels of pitch 128..1024 with tensor maps).
static void restrict_tma3(const LevelDev<float2>* levs, int nprob, int P, bool r0_is_b, bool x_from_zero,
                          bool nosmooth, int nraw, cudaStream_t st) {
  const Tma3Params tp = tma3_params(TP_RESTRICT, 0, P);
  const size_t smem = (size_t)tp.stages * nraw * tm3_box_stride(2);
  thread_local size_t configured = 0;
  thread_local int occ_key = -1, occ = 1;
  if (configured < smem) {
    cudaFuncSetAttribute(k_restrict_tma3<SMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured = smem;
  }
  const int key = tp.stages * 16 + nraw;
  if (occ_key != key) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_restrict_tma3<SMAX>, 256, smem) != cudaSuccess || occ < 1)
      occ = 1;
    occ_key = key;
  }
  const long long cols = tma3_cols(P, 2);
  long long units = tp.pieces > 0 ? cols * std::min(tp.pieces, P) : (long long)occ * sm_count();
  units = std::max<long long>(1, std::min<long long>(units, std::min<long long>(TMA3_MAX_UNITS, cols * P)));
  pdl_launch(k_restrict_tma3<SMAX>, dim3(nprob * (int)units), dim3(32, 8), smem, st, levs, (int)units, tp.stages,
             r0_is_b ? 1 : 0, x_from_zero ? 1 : 0, nosmooth ? 1 : 0);
}

template <typename C>
void launch_restrict(int dim, const LevelDev<C>* levs, int nprob, int ntiles, TileCfg cfg, bool r0_is_b,
                     bool x_from_zero, bool nosmooth, cudaStream_t st, bool tma, int nraw) {
  if constexpr (std::is_same<C, float2>::value) {
    if (dim == 3 && tma && cfg.P >= TMA3_MIN_P && cfg.P <= TMA3_MAX_P && tma3_params(TP_RESTRICT, 0, cfg.P).enabled) {
      restrict_tma3(levs, nprob, cfg.P, r0_is_b, x_from_zero, nosmooth, nraw, st);
      return;
    }
  }
  if (dim == 2) {
    const int t = tuned_tpc(TP_RESTRICT, cfg.P, (int)sizeof(C), 0, tiles_per_cta(k_restrict_t2<C>, ntiles));
    pdl_launch(k_restrict_t2<C>, dim3(nprob * ceil_div(ntiles, t)), dim3(dim3(32, 8)), 0, st, levs, ntiles, t, r0_is_b,
               x_from_zero, nosmooth);
  } else
    pdl_launch(k_restrict_t3<C>, dim3(nprob * ntiles), dim3(dim3(32, 8)), 0, st, levs, ntiles, cfg.rows, r0_is_b, x_from_zero, nosmooth);
}

template <typename C>
void launch_update_flat(int dim, UpdateMode mode, const LevelDev<C>* levs, int nprob, int ntiles, bool r0_is_b,
                        int xsel, bool x_from_zero, cudaStream_t st) {
  pdl_launch(k_update_flat<C>, dim3(nprob * ntiles), dim3(256), 0, st, levs, ntiles, dim, (int)mode, r0_is_b, xsel, x_from_zero);
}

template <typename C>
void launch_prolong(int dim, bool with_residual, const LevelDev<C>* levs, int nprob, int ntiles, TileCfg cfg,
                    bool tma, cudaStream_t st) {
  if constexpr (std::is_same<C, float2>::value) {
    if (prolong_kernels(dim, with_residual, (int)sizeof(C), tma, cfg.P) == 2) {
      prolong_tma3(levs, nprob, cfg.P, st);
      return;
    }
  }
  if (!with_residual) {
    pdl_launch(k_prolong_flat<C>, dim3(nprob * ntiles), dim3(256), 0, st, levs, ntiles, dim);
  } else if (dim == 2) {
    const int t = tuned_tpc(TP_PROLONG, cfg.P, (int)sizeof(C), 0, tiles_per_cta(k_prolong_t2<C>, ntiles));
    pdl_launch(k_prolong_t2<C>, dim3(nprob * ceil_div(ntiles, t)), dim3(dim3(32, 8)), 0, st, levs, ntiles, t);
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

// ------------------------------------------------------------------ persistent segments
// The recorders append the pass an ordinary launch would run (the same launch
// parameters, so the same partial-sum order) to a pass list instead of launching it.
static inline void seq_push(PassSeq& q, const void* levs, int kind, int J, int ntiles, int geo, int f0, int f1, int f2,
                            int f3, int nvblk) {
  if (q.npass >= SEQ_MAX) return;  // the caller sizes its lists (checked by the engine)
  PassDesc& d = q.p[q.npass++];
  d.levs = levs;
  d.kind = kind;
  d.J = J;
  d.ntiles = ntiles;
  d.geo = geo;
  d.f0 = f0;
  d.f1 = f1;
  d.f2 = f2;
  d.f3 = f3;
  d.nvblk = nvblk;
}

template <typename C, int J>
static void record_arnoldi_J(PassSeq& q, int dim, const LevelDev<C>* levs, int nprob, int ntiles, TileCfg cfg,
                             bool r0_is_b, bool store_p) {
  if (dim == 2) {
    const int t = tuned_tpc(TP_ARNOLDI, cfg.P, (int)sizeof(C), J, tiles_per_cta(k_arnoldi_t2<C, J>, ntiles));
    seq_push(q, levs, PK_ARNOLDI, J, ntiles, t, r0_is_b, store_p, 0, 0, nprob * ceil_div(ntiles, t));
  } else {
    seq_push(q, levs, PK_ARNOLDI, J, ntiles, cfg.rows, r0_is_b, store_p, 0, 0, nprob * ntiles);
  }
}

template <typename C>
void record_arnoldi(PassSeq& q, int dim, int J, const LevelDev<C>* levs, int nprob, int ntiles, TileCfg cfg,
                    bool r0_is_b, bool store_p) {
  switch (J) {
    case 1: record_arnoldi_J<C, 1>(q, dim, levs, nprob, ntiles, cfg, r0_is_b, store_p); break;
    case 2: record_arnoldi_J<C, 2>(q, dim, levs, nprob, ntiles, cfg, r0_is_b, store_p); break;
    case 3: record_arnoldi_J<C, 3>(q, dim, levs, nprob, ntiles, cfg, r0_is_b, store_p); break;
    default: record_arnoldi_J<C, 4>(q, dim, levs, nprob, ntiles, cfg, r0_is_b, store_p); break;
  }
}

template <typename C>
void record_restrict(PassSeq& q, int dim, const LevelDev<C>* levs, int nprob, int ntiles, TileCfg cfg, bool r0_is_b,
                     bool x_from_zero, bool nosmooth) {
  if (dim == 2) {
    const int t = tuned_tpc(TP_RESTRICT, cfg.P, (int)sizeof(C), 0, tiles_per_cta(k_restrict_t2<C>, ntiles));
    seq_push(q, levs, PK_RESTRICT, 0, ntiles, t, r0_is_b, x_from_zero, nosmooth, 0, nprob * ceil_div(ntiles, t));
  } else {
    seq_push(q, levs, PK_RESTRICT, 0, ntiles, cfg.rows, r0_is_b, x_from_zero, nosmooth, 0, nprob * ntiles);
  }
}

template <typename C>
void record_update(PassSeq& q, int dim, UpdateMode mode, const LevelDev<C>* levs, int nprob, int ntiles, bool r0_is_b,
                   int xsel, bool x_from_zero) {
  (void)dim;
  seq_push(q, levs, PK_UPDATE, 0, ntiles, 0, (int)mode, r0_is_b, xsel, x_from_zero, nprob * ntiles);
}

template <typename C>
void record_prolong(PassSeq& q, int dim, bool with_residual, const LevelDev<C>* levs, int nprob, int ntiles,
                    TileCfg cfg) {
  if (!with_residual) {
    seq_push(q, levs, PK_PROLONG_FLAT, 0, ntiles, 0, 0, 0, 0, 0, nprob * ntiles);
  } else if (dim == 2) {
    const int t = tuned_tpc(TP_PROLONG, cfg.P, (int)sizeof(C), 0, tiles_per_cta(k_prolong_t2<C>, ntiles));
    seq_push(q, levs, PK_PROLONG, 0, ntiles, t, 0, 0, 0, 0, nprob * ceil_div(ntiles, t));
  } else {
    seq_push(q, levs, PK_PROLONG, 0, ntiles, cfg.rows, 0, 0, 0, 0, nprob * ntiles);
  }
}

// One cooperative launch of the pass list: every CTA resident (the grid barrier needs
// it), at most as many CTAs as the largest pass has virtual blocks.
template <typename C>
int launch_seq(int dim, const PassSeq& q, GridBar* gb, unsigned long long limit_ns, cudaStream_t st) {
  if (q.npass == 0) return 0;
  void (*kern)(const PassSeq, GridBar*, unsigned long long) = dim == 2 ? k_vcycle_seq<C, 2> : k_vcycle_seq<C, 3>;
  thread_local void (*last)(const PassSeq, GridBar*, unsigned long long) = nullptr;
  thread_local int occ = 1;
  if (kern != last) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, 0) != cudaSuccess || occ < 1) occ = 1;
    last = kern;
  }
  int maxv = 1;
  for (int i = 0; i < q.npass; ++i) maxv = std::max(maxv, q.p[i].nvblk);
  const int grid = std::max(1, std::min(maxv, occ * sm_count()));
  cudaError_t e = cudaMemsetAsync(gb, 0, sizeof(GridBar), st);
  if (e != cudaSuccess) return (int)e;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(32, 8);  // the tile passes' shape; the flat passes use the flat thread index
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, kern, q, gb, limit_ns);
  return (int)e;
}

#define HELM_VCYCLE_INST(C)                                                                                   \
  template void launch_arnoldi<C>(int, int, const LevelDev<C>*, int, int, TileCfg, bool, bool, bool, cudaStream_t); \
  template void launch_restrict<C>(int, const LevelDev<C>*, int, int, TileCfg, bool, bool, bool,           \
                                    cudaStream_t, bool, int);                                               \
  template void launch_update_flat<C>(int, UpdateMode, const LevelDev<C>*, int, int, bool, int, bool,         \
                                      cudaStream_t);                                                          \
  template void launch_prolong<C>(int, bool, const LevelDev<C>*, int, int, TileCfg, bool, cudaStream_t);      \
  template void launch_coarse<C>(int, const LevelDev<C>*, int, int, const CoarseLU*, int, int, int,           \
                                 cudaStream_t);                                                               \
  template void launch_coarse_smem<C>(int, const LevelDev<C>*, int, int, const CoarseLU*, int, int, int, size_t, \
                                      cudaStream_t);                                                          \
  template void launch_coarse_cluster<C>(int, const LevelDev<C>*, int, const CoarseLU*, int, int, int,       \
                                         cudaStream_t);                                                       \
  template void launch_load_input<C>(int, const LevelDev<C>*, int, const void*, int, cudaStream_t);           \
  template void launch_store_output<C>(int, int, const LevelDev<C>*, void*, int, cudaStream_t);              \
  template void launch_poly_step<C>(int, const LevelDev<C>*, const C*, int, int, int, int, int, cudaStream_t); \
  template void launch_poly_restrict<C>(int, const LevelDev<C>*, int, int, int, cudaStream_t);                \
  template void record_arnoldi<C>(PassSeq&, int, int, const LevelDev<C>*, int, int, TileCfg, bool, bool);      \
  template void record_restrict<C>(PassSeq&, int, const LevelDev<C>*, int, int, TileCfg, bool, bool, bool);    \
  template void record_update<C>(PassSeq&, int, UpdateMode, const LevelDev<C>*, int, int, bool, int, bool);    \
  template void record_prolong<C>(PassSeq&, int, bool, const LevelDev<C>*, int, int, TileCfg);                 \
  template int launch_seq<C>(int, const PassSeq&, GridBar*, unsigned long long, cudaStream_t);

}  // namespace helm
