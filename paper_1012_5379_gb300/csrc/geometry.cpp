// Host geometry of the complex stretched grids (Sec. 2, Eq. csggrid) and the dense
// LU of the coarsest operator.
#include "geometry.h"

#include <algorithm>
#include <cmath>

namespace helm {

// Length of [a, b] inside [lo, hi].
static double overlap(double a, double b, double lo, double hi) {
  return std::max(0.0, std::min(b, hi) - std::max(a, lo));
}

// h_i = integral over [x_i, x_{i+1}] of the stretching factor: e^{i theta_gamma} in
// the layers [0, w] and [1 - w, 1] (both sides, Remark 2.2), e^{i theta_beta} in the
// interior (Eq. csggrid).  An interval that straddles a turning point gets the exact
// mixed value.
std::vector<cplx> grid_spacings(int n, double ecs, double theta_gamma, double theta_beta) {
  const double h = 1.0 / (n + 1);
  const cplx eg = std::polar(1.0, theta_gamma), eb = std::polar(1.0, theta_beta);
  std::vector<cplx> sp(n + 1);
  for (int i = 0; i <= n; ++i) {
    const double a = i * h, b = (i + 1) * h;
    sp[i] = eg * (overlap(a, b, 0.0, ecs) + overlap(a, b, 1.0 - ecs, 1.0)) + eb * overlap(a, b, ecs, 1.0 - ecs);
  }
  return sp;
}

// Non-uniform three-point second difference (Shortley-Weller), sign of -d^2/dz^2:
//   (L u)_i = -2/(hl+hr) [ (u_{i+1}-u_i)/hr - (u_i-u_{i-1})/hl ]
void stencil_coefficients(const std::vector<cplx>& sp, std::vector<cplx>& a, std::vector<cplx>& d,
                          std::vector<cplx>& c) {
  const int n = (int)sp.size() - 1;
  a.resize(n);
  d.resize(n);
  c.resize(n);
  for (int i = 0; i < n; ++i) {
    const cplx hl = sp[i], hr = sp[i + 1];
    const cplx two_over_sum = 2.0 / (hl + hr);
    a[i] = -two_over_sum / hl;
    c[i] = -two_over_sum / hr;
    d[i] = two_over_sum * (1.0 / hl + 1.0 / hr);
  }
}

// Dense matrix of M = sum_axes L_axis - diag(phi) on an n^dim grid (natural order).
std::vector<cplx> dense_operator(int dim, int n, const std::vector<cplx>& a, const std::vector<cplx>& d,
                                 const std::vector<cplx>& c, const std::vector<double>& phi, cplx shift) {
  const int m = dim == 3 ? n * n * n : n * n;
  std::vector<cplx> A((size_t)m * m, cplx(0, 0));
  for (int z = 0; z < (dim == 3 ? n : 1); ++z)
    for (int y = 0; y < n; ++y)
      for (int x = 0; x < n; ++x) {
        const int row = (z * n + y) * n + x;
        cplx diag = d[x] + d[y] + (dim == 3 ? d[z] : cplx(0, 0)) - shift * phi[row];
        A[(size_t)row * m + row] += diag;
        auto add = [&](int xx, int yy, int zz, cplx v) {
          if (xx < 0 || yy < 0 || zz < 0 || xx >= n || yy >= n || zz >= n) return;
          A[(size_t)row * m + (zz * n + yy) * n + xx] += v;
        };
        add(x - 1, y, z, a[x]);
        add(x + 1, y, z, c[x]);
        add(x, y - 1, z, a[y]);
        add(x, y + 1, z, c[y]);
        if (dim == 3) {
          add(x, y, z - 1, a[z]);
          add(x, y, z + 1, c[z]);
        }
      }
  return A;
}

// In-place LU with partial pivoting: perm[i] = original row now at row i.
bool lu_factor(std::vector<cplx>& A, int m, std::vector<int>& perm) {
  perm.resize(m);
  for (int i = 0; i < m; ++i) perm[i] = i;
  for (int k = 0; k < m; ++k) {
    int piv = k;
    double best = std::abs(A[(size_t)k * m + k]);
    for (int i = k + 1; i < m; ++i) {
      const double v = std::abs(A[(size_t)i * m + k]);
      if (v > best) { best = v; piv = i; }
    }
    if (best == 0.0) return false;
    if (piv != k) {
      for (int j = 0; j < m; ++j) std::swap(A[(size_t)k * m + j], A[(size_t)piv * m + j]);
      std::swap(perm[k], perm[piv]);
    }
    const cplx inv = 1.0 / A[(size_t)k * m + k];
    for (int i = k + 1; i < m; ++i) {
      const cplx l = A[(size_t)i * m + k] * inv;
      A[(size_t)i * m + k] = l;
      for (int j = k + 1; j < m; ++j) A[(size_t)i * m + j] -= l * A[(size_t)k * m + j];
    }
  }
  return true;
}

std::vector<int> level_sizes(int n, int coarsest) {
  std::vector<int> s{n};
  while (s.back() > coarsest && (s.back() + 1) % 2 == 0) s.push_back((s.back() + 1) / 2 - 1);
  return s;
}

}  // namespace helm
