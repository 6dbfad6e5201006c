// The V-cycle passes of the third-degree polynomial smoother (Sec. 4): Richardson steps
// x_out = x_in + w (b - M x_in), the residual r0 = b - M x and its full-weighting
// restriction.  Flat passes over every problem of a depth (grid = problems x flat
// CTAs); each problem's three weights are `pw[3 * problem .. + 2]`.
#pragma once
#include <cuda_runtime.h>

#include "helm_internal.h"

namespace helm {

// Level vectors a step reads or writes (POLY_NONE: the zero vector / none).
enum PolySel { POLY_NONE = 0, POLY_XA = 1, POLY_XB = 2, POLY_P0 = 3, POLY_P1 = 4 };

// dst = src + w_j (b - M src); wsel < 0 writes zero.
template <typename C>
void launch_poly_step(int dim, const LevelDev<C>* levs, const C* pw, int nprob, int nflat, int src, int dst,
                      int wsel, cudaStream_t st);
// r0 = b - M src (src POLY_NONE: r0 = b), then b_c = full weighting of r0.
template <typename C>
void launch_poly_restrict(int dim, const LevelDev<C>* levs, int nprob, int nflat, int src, cudaStream_t st);

}  // namespace helm
