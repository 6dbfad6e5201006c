// Host geometry of the complex stretched grids and the coarsest dense LU.
#pragma once
#include <complex>
#include <vector>

namespace helm {

typedef std::complex<double> cplx;

// Complex spacings of one axis (n + 1 intervals of the unit box); low_layer = false
// keeps the ECS layer at the far end only (Dirichlet edge at x = 0).
std::vector<cplx> grid_spacings(int n, double ecs, double theta_gamma, double theta_beta, bool low_layer = true);
void stencil_coefficients(const std::vector<cplx>& sp, std::vector<cplx>& a, std::vector<cplx>& d,
                          std::vector<cplx>& c);
// Dense matrix of L - shift * diag(phi) on n^dim nodes (shift 1: CSG; 1 + i eps: CSL variant).
std::vector<cplx> dense_operator(int dim, int n, const std::vector<cplx>& a, const std::vector<cplx>& d,
                                 const std::vector<cplx>& c, const std::vector<double>& phi, cplx shift = cplx(1, 0));
bool lu_factor(std::vector<cplx>& A, int m, std::vector<int>& perm);
// Third-degree polynomial smoother of a level (Sec. 4): its mapping angle phi and the
// weights w of the three Richardson steps x <- x + w_j (b - M x); false if no stable
// polynomial exists under the first- and second-order conditions.
bool poly_smoother(double k, double h, double theta_beta, double theta_gamma, int dim, double* phi, cplx w[3]);
std::vector<int> level_sizes(int n, int coarsest);

}  // namespace helm
