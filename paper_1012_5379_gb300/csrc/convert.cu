// Layout conversions between the natural (n^d) and padded ((n+1)^d) layouts, the
// sampling of a phi field onto coarse levels, and a plain natural-layout operator
// apply used by helm_apply_operator.
#include "vcycle.cuh"
#include "../../include/helm.h"
#include <algorithm>

namespace helm {

static int grid_for(size_t npts) { return (int)std::min<size_t>((npts + 255) / 256, 8192); }

__global__ void k_dense_to_padded(int dim, int n, const double2* __restrict__ src, double2* __restrict__ dst) {
  const int P = n + 1;
  const size_t npts = dim == 3 ? (size_t)P * P * P : (size_t)P * P;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < npts; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % P), y = (int)((i / P) % P), z = dim == 3 ? (int)(i / ((size_t)P * P)) : 0;
    dst[i] = inside(x, y, z, n) ? src[((size_t)z * n + y) * n + x] : make_double2(0, 0);
  }
}

__global__ void k_padded_to_dense(int dim, int n, const double2* __restrict__ src, double2* __restrict__ dst) {
  const int P = n + 1;
  const size_t npts = dim == 3 ? (size_t)n * n * n : (size_t)n * n;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < npts; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % n), y = (int)((i / n) % n), z = dim == 3 ? (int)(i / ((size_t)n * n)) : 0;
    dst[i] = src[pidx(x, y, z, P)];
  }
}

// Level node x (0-based) sits on fine node (x + 1) * stride - 1.
__global__ void k_scatter_phi(int dim, int n, int stride, int nf, const float* __restrict__ phi_f,
                              float* __restrict__ dst) {
  const int P = n + 1;
  const size_t npts = dim == 3 ? (size_t)P * P * P : (size_t)P * P;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < npts; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % P), y = (int)((i / P) % P), z = dim == 3 ? (int)(i / ((size_t)P * P)) : 0;
    float v = 0.0f;
    if (inside(x, y, z, n)) {
      const size_t fx = (size_t)(x + 1) * stride - 1, fy = (size_t)(y + 1) * stride - 1;
      const size_t fz = dim == 3 ? (size_t)(z + 1) * stride - 1 : 0;
      v = phi_f[(fz * nf + fy) * nf + fx];
    }
    dst[i] = v;
  }
}

template <typename C>
__global__ void k_apply_dense(int dim, int n, const double2* __restrict__ ca, const double2* __restrict__ cd,
                              const double2* __restrict__ cc, const float* __restrict__ phi, double phic,
                              const C* __restrict__ v, C* __restrict__ w) {
  const size_t npts = dim == 3 ? (size_t)n * n * n : (size_t)n * n;
  auto at = [&](int x, int y, int z) -> C {
    return inside(x, y, z, n) ? v[((size_t)z * n + y) * n + x] : czero<C>();
  };
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < npts; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % n), y = (int)((i / n) % n), z = dim == 3 ? (int)(i / ((size_t)n * n)) : 0;
    C diag = cadd(from_d<C>(cd[x]), from_d<C>(cd[y]));
    C p = czero<C>();
    p = cfma(from_d<C>(ca[x]), at(x - 1, y, z), p);
    p = cfma(from_d<C>(cc[x]), at(x + 1, y, z), p);
    p = cfma(from_d<C>(ca[y]), at(x, y - 1, z), p);
    p = cfma(from_d<C>(cc[y]), at(x, y + 1, z), p);
    if (dim == 3) {
      diag = cadd(diag, from_d<C>(cd[z]));
      p = cfma(from_d<C>(ca[z]), at(x, y, z - 1), p);
      p = cfma(from_d<C>(cc[z]), at(x, y, z + 1), p);
    }
    diag.x -= phi ? (typename CT<C>::R)phi[pidx(x, y, z, n + 1)] : (typename CT<C>::R)phic;
    w[i] = cfma(diag, v[i], p);
  }
}

void convert_dense_to_padded_c128(int dim, int n, const double2* src, double2* dst, cudaStream_t st) {
  const size_t P = n + 1;
  k_dense_to_padded<<<grid_for(dim == 3 ? P * P * P : P * P), 256, 0, st>>>(dim, n, src, dst);
}
void convert_padded_to_dense_c128(int dim, int n, const double2* src, double2* dst, cudaStream_t st) {
  const size_t nn = n;
  k_padded_to_dense<<<grid_for(dim == 3 ? nn * nn * nn : nn * nn), 256, 0, st>>>(dim, n, src, dst);
}
void scatter_phi(int dim, int n_level, int stride, int n_fine, const float* phi_f, float* dst, cudaStream_t st) {
  const size_t P = n_level + 1;
  k_scatter_phi<<<grid_for(dim == 3 ? P * P * P : P * P), 256, 0, st>>>(dim, n_level, stride, n_fine, phi_f, dst);
}
void apply_operator_dense(int dim, int n, const double2* ca, const double2* cd, const double2* cc,
                          const float* phi_pad, double phic, const void* v, void* w, int prec, cudaStream_t st) {
  const size_t nn = n;
  const int grid = grid_for(dim == 3 ? nn * nn * nn : nn * nn);
  if (prec == HELM_C128)
    k_apply_dense<double2><<<grid, 256, 0, st>>>(dim, n, ca, cd, cc, phi_pad, phic, (const double2*)v, (double2*)w);
  else
    k_apply_dense<float2><<<grid, 256, 0, st>>>(dim, n, ca, cd, cc, phi_pad, phic, (const float2*)v, (float2*)w);
}

}  // namespace helm
