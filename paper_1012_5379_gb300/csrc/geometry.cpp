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
// mixed value.  low_layer = false drops the layer at x = 0: homogeneous Dirichlet on
// that edge of the interior, the layer only at the far end (Eq. csggrid as printed;
// Benchmark 3 of Sec. 5 has Dirichlet south and west edges, layers north and east).
std::vector<cplx> grid_spacings(int n, double ecs, double theta_gamma, double theta_beta, bool low_layer) {
  const double h = 1.0 / (n + 1);
  const cplx eg = std::polar(1.0, theta_gamma), eb = std::polar(1.0, theta_beta);
  const double lo = low_layer ? ecs : 0.0;
  std::vector<cplx> sp(n + 1);
  for (int i = 0; i <= n; ++i) {
    const double a = i * h, b = (i + 1) * h;
    sp[i] = eg * (overlap(a, b, 0.0, lo) + overlap(a, b, 1.0 - ecs, 1.0)) + eb * overlap(a, b, lo, 1.0 - ecs);
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

namespace helm {

// ------------------------------------------------------------------ polynomial smoother
// Third-degree polynomial smoother of Sec. 4 on a level of real spacing h.  The
// spectrum's bounding triangle (Prop. 3.1) has vertices t0 = -k^2,
// t1 = t0 + 4d e^{-2i theta_beta} / h^2, t2 = t0 + 4d e^{-2i theta_gamma} / h^2.
// p(t) = c0 + c1 s + c2 s^2 + c3 s^3 (s = t - t0) with p(t0) = e^{i phi},
// p(t1) = p(t2) = 0 and p(0) = 1: c0 = e^{i phi} and (c1, c2, c3) = e - e^{i phi} f
// (Eq. coefficients_solution), e and f solving the 3 x 3 Vandermonde system in the
// nodes s = -t0, t1 - t0, t2 - t0 with right-hand sides (1, 0, 0) and (1, 1, 1).
// phi: the midpoint of the longest arc (0.05 degree grid) meeting the first-order
// condition Re(e^{-i phi} c1 e^{-2i theta_beta}) < 0 (Eq. firstorder_varphi, with the
// sign of phi of its derivation) and the second-order condition
// |c1|^2 + 2 Re(e^{-i phi} c2 e^{-4i theta_beta}) < 0 (Eq. secondorder_varphi); 0 where
// the first-order condition holds for every phi; none otherwise.  The smoother is then
// three Richardson steps with the reciprocals of p's roots.

// Solve the 3 x 3 complex system V x = r by Gaussian elimination with partial pivoting.
static void solve3(cplx V[3][3], cplx r[3], cplx x[3]) {
  for (int c = 0; c < 3; ++c) {
    int p = c;
    for (int i = c + 1; i < 3; ++i)
      if (std::abs(V[i][c]) > std::abs(V[p][c])) p = i;
    if (p != c) {
      for (int j = 0; j < 3; ++j) std::swap(V[c][j], V[p][j]);
      std::swap(r[c], r[p]);
    }
    for (int i = c + 1; i < 3; ++i) {
      const cplx m = V[i][c] / V[c][c];
      for (int j = c; j < 3; ++j) V[i][j] -= m * V[c][j];
      r[i] -= m * r[c];
    }
  }
  for (int i = 2; i >= 0; --i) {
    cplx acc = r[i];
    for (int j = i + 1; j < 3; ++j) acc -= V[i][j] * x[j];
    x[i] = acc / V[i][i];
  }
}

bool poly_smoother(double k, double h, double theta_beta, double theta_gamma, int dim, double* phi_out,
                   cplx w_out[3]) {
  const cplx t0(-k * k, 0.0);
  const cplx t1 = t0 + 4.0 * dim * std::polar(1.0, -2.0 * theta_beta) / (h * h);
  const cplx t2 = t0 + 4.0 * dim * std::polar(1.0, -2.0 * theta_gamma) / (h * h);
  const cplx nodes[3] = {-t0, t1 - t0, t2 - t0};
  cplx e[3], f[3];
  for (int rhs = 0; rhs < 2; ++rhs) {
    cplx V[3][3], r[3];
    for (int i = 0; i < 3; ++i) {
      cplx pw = nodes[i];
      for (int j = 0; j < 3; ++j) {
        V[i][j] = pw;
        pw *= nodes[i];
      }
      r[i] = rhs == 0 ? cplx(i == 0 ? 1.0 : 0.0, 0.0) : cplx(1.0, 0.0);
    }
    solve3(V, r, rhs == 0 ? e : f);
  }
  const cplx w1 = std::polar(1.0, -2.0 * theta_beta), w2 = std::polar(1.0, -4.0 * theta_beta);
  const int NG = 7200;  // 0.05 degree steps
  std::vector<char> first(NG), both(NG);
  bool any = false, all_first = true, all_both = true;
  for (int g = 0; g < NG; ++g) {
    const double ph = g * (2.0 * M_PI / NG);
    const cplx z = std::polar(1.0, ph), zi = std::conj(z);
    const cplx c1 = e[0] - z * f[0], c2 = e[1] - z * f[1];
    first[g] = std::real(zi * c1 * w1) < 0.0;
    both[g] = first[g] && (std::norm(c1) + 2.0 * std::real(zi * c2 * w2) < 0.0);
    any = any || both[g];
    all_first = all_first && first[g];
    all_both = all_both && both[g];
  }
  double phi;
  if (any && !all_both) {
    int start = 0;
    while (both[start]) ++start;  // an infeasible grid point: no arc wraps past it
    int best = 0, best_at = 0, run = 0, run_at = 0;
    for (int i = 0; i < NG; ++i) {
      if (both[(start + i) % NG]) {
        if (run == 0) run_at = i;
        ++run;
        if (run > best) { best = run; best_at = run_at; }
      } else {
        run = 0;
      }
    }
    const double mid = std::fmod(start + best_at + 0.5 * (best - 1), (double)NG);
    phi = mid * (2.0 * M_PI / NG);
  } else if (all_both || all_first) {
    phi = 0.0;
  } else {
    return false;
  }
  // p's roots in s (Durand-Kerner on the monic cubic), then w_j = 1 / (t0 + s_j)
  const cplx z = std::polar(1.0, phi);
  const cplx c[4] = {z, e[0] - z * f[0], e[1] - z * f[1], e[2] - z * f[2]};
  const cplx a0 = c[0] / c[3], a1 = c[1] / c[3], a2 = c[2] / c[3];
  auto mono = [&](cplx s) { return ((s + a2) * s + a1) * s + a0; };
  const double rad = 1.0 + std::max({std::abs(a0), std::abs(a1), std::abs(a2)});
  cplx s[3] = {rad * std::polar(1.0, 0.4), rad * std::polar(1.0, 0.4 + 2.0 * M_PI / 3),
               rad * std::polar(1.0, 0.4 + 4.0 * M_PI / 3)};
  for (int it = 0; it < 500; ++it) {
    double moved = 0.0;
    for (int i = 0; i < 3; ++i) {
      cplx den(1.0, 0.0);
      for (int j = 0; j < 3; ++j)
        if (j != i) den *= (s[i] - s[j]);
      const cplx step = mono(s[i]) / den;
      s[i] -= step;
      moved = std::max(moved, std::abs(step) / std::max(1.0, std::abs(s[i])));
    }
    if (moved < 1e-15) break;
  }
  for (int i = 0; i < 3; ++i) w_out[i] = 1.0 / (t0 + s[i]);
  // a fixed order (real part, then imaginary part): the steps commute in exact arithmetic
  std::sort(w_out, w_out + 3, [](const cplx& a, const cplx& b) {
    return a.real() < b.real() || (a.real() == b.real() && a.imag() < b.imag());
  });
  *phi_out = phi;
  return true;
}

}  // namespace helm
