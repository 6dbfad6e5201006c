// Host launchers of the V-cycle kernels, instantiated once per precision in
// vcycle_c64.cu and vcycle_c128.cu (two translation units compile in parallel).
#pragma once
#include "vcycle.cuh"
#include <algorithm>
#include "../../include/helm.h"

namespace helm {

template <typename C, int J>
static void arnoldi_J(int dim, const LevelDev<C>* levs, int grid, int ntiles, TileCfg cfg, bool r0_is_b,
                      bool store_p, cudaStream_t st) {
  if (dim == 2)
    k_arnoldi2<C, J><<<grid, dim3(32, WARPS2), 0, st>>>(levs, ntiles, cfg.rows, r0_is_b, store_p);
  else
    k_arnoldi3<C, J><<<grid, dim3(32, WY3 + 2), 0, st>>>(levs, ntiles, cfg.rows, r0_is_b, store_p);
}

template <typename C>
void launch_arnoldi(int dim, int J, const LevelDev<C>* levs, int nprob, int ntiles, TileCfg cfg, bool r0_is_b,
                    bool store_p, cudaStream_t st) {
  const int grid = nprob * ntiles;
  switch (J) {
    case 1: arnoldi_J<C, 1>(dim, levs, grid, ntiles, cfg, r0_is_b, store_p, st); break;
    case 2: arnoldi_J<C, 2>(dim, levs, grid, ntiles, cfg, r0_is_b, store_p, st); break;
    case 3: arnoldi_J<C, 3>(dim, levs, grid, ntiles, cfg, r0_is_b, store_p, st); break;
    default: arnoldi_J<C, 4>(dim, levs, grid, ntiles, cfg, r0_is_b, store_p, st); break;
  }
}

template <typename C>
void launch_restrict(int dim, const LevelDev<C>* levs, int nprob, int ntiles, TileCfg cfg, bool r0_is_b,
                     bool x_from_zero, bool nosmooth, cudaStream_t st) {
  if (dim == 2)
    k_restrict2<C><<<nprob * ntiles, dim3(32, WARPS2), 0, st>>>(levs, ntiles, cfg.rows, r0_is_b, x_from_zero,
                                                                nosmooth);
  else
    k_restrict3<C><<<nprob * ntiles, dim3(32, WY3 + 2), 0, st>>>(levs, ntiles, cfg.rows, r0_is_b, x_from_zero,
                                                                 nosmooth);
}

template <typename C>
void launch_update_flat(int dim, UpdateMode mode, const LevelDev<C>* levs, int nprob, int ntiles, bool r0_is_b,
                        int xsel, bool x_from_zero, cudaStream_t st) {
  k_update_flat<C><<<nprob * ntiles, 256, 0, st>>>(levs, ntiles, dim, (int)mode, r0_is_b, xsel, x_from_zero);
}

template <typename C>
void launch_prolong(int dim, bool with_residual, const LevelDev<C>* levs, int nprob, int ntiles, TileCfg cfg,
                    cudaStream_t st) {
  if (!with_residual) {
    k_prolong_flat<C><<<nprob * ntiles, 256, 0, st>>>(levs, ntiles, dim);
  } else if (dim == 2) {
    k_prolong2<C><<<nprob * ntiles, dim3(32, WARPS2), 0, st>>>(levs, ntiles, cfg.rows);
  } else {
    k_prolong3<C><<<nprob * ntiles, dim3(32, WY3 + 2), 0, st>>>(levs, ntiles, cfg.rows);
  }
}

template <typename C>
void launch_coarse(int dim, const LevelDev<C>* levs, int nlev, int lev_stride, const CoarseLU* lus, int nprob,
                   int nu1, int nu2, cudaStream_t st) {
  k_coarse<C><<<nprob, 1024, 0, st>>>(levs, nlev, lev_stride, lus, nu1, nu2, dim);
}

template <typename C>
void launch_load_input(int dim, const LevelDev<C>* levs, int ntiles, const void* src, int in_prec, cudaStream_t st) {
  if (in_prec == HELM_C128)
    k_load_input<double2, C><<<ntiles, 256, 0, st>>>(levs, ntiles, dim, (const double2*)src);
  else
    k_load_input<float2, C><<<ntiles, 256, 0, st>>>(levs, ntiles, dim, (const float2*)src);
}

template <typename C>
void launch_store_output(int dim, int n, const LevelDev<C>* levs, void* dst, int out_prec, cudaStream_t st) {
  const size_t npts = dim == 3 ? (size_t)n * n * n : (size_t)n * n;
  const int grid = (int)std::min<size_t>((npts + 255) / 256, 4096);
  if (out_prec == HELM_C128)
    k_store_output<C, double2><<<grid, 256, 0, st>>>(levs, dim, (double2*)dst);
  else
    k_store_output<C, float2><<<grid, 256, 0, st>>>(levs, dim, (float2*)dst);
}

#define HELM_VCYCLE_INST(C)                                                                                   \
  template void launch_arnoldi<C>(int, int, const LevelDev<C>*, int, int, TileCfg, bool, bool, cudaStream_t); \
  template void launch_restrict<C>(int, const LevelDev<C>*, int, int, TileCfg, bool, bool, bool,           \
                                    cudaStream_t);                                                          \
  template void launch_update_flat<C>(int, UpdateMode, const LevelDev<C>*, int, int, bool, int, bool,         \
                                      cudaStream_t);                                                          \
  template void launch_prolong<C>(int, bool, const LevelDev<C>*, int, int, TileCfg, cudaStream_t);            \
  template void launch_coarse<C>(int, const LevelDev<C>*, int, int, const CoarseLU*, int, int, int,           \
                                 cudaStream_t);                                                               \
  template void launch_load_input<C>(int, const LevelDev<C>*, int, const void*, int, cudaStream_t);           \
  template void launch_store_output<C>(int, int, const LevelDev<C>*, void*, int, cudaStream_t);

}  // namespace helm
