// Host-side icosahedral grid of the THOR dynamical core (Sec. 2 of
// Mendonca et al. 2016): construction, spring dynamics, centroid relocation,
// metric terms, and the per-column stencil weights the device kernels apply.
// Everything here is float64 and runs once per grid, off the hot path.
#pragma once

#include <cstdint>
#include <vector>

namespace thor {

struct SpringParams {
  double beta = 1.15, alpha = 1.0, k = 1.0, dt = 0.01, tol = 1e-5;
  int max_iter = 100000;
};

// Column numbering: 10 rhombi of n x n owned points (n = 2^glevel), column
// index r*n*n + j*n + i for rhombus r and lattice point (i, j), then the north
// pole (10 n^2) and the south pole (10 n^2 + 1).
struct HostGrid {
  int glevel = 0, n = 1, ncol = 0, nv = 0;
  double radius = 0, z_top = 0;
  std::vector<double> P;          // ncol*3 cell centres, unit sphere
  std::vector<int> nbr;           // ncol*6 counter-clockwise, -1 padded
  std::vector<int> nn;            // ncol: 5 or 6
  std::vector<int> tri;           // ntri*3 counter-clockwise triangles
  std::vector<int> ring_tri;      // ncol*6: triangle (c, nbr[k], nbr[k+1])
  std::vector<double> corner;     // ntri*3 control-volume vertices C
  std::vector<double> area;       // ncol control-volume areas A_c
  // Linear stencils on the unit sphere over the 7 points (self, nbr[0..5]):
  //   div(F)(c)  = sum_j w_div[c][j] . F(n_j)        (Eqs. int_grid, flx_div, div_gauss)
  //   grad(s)(c) = sum_j w_grad[c][j] s(n_j)          (Eq. grad + Eq. proj_h)
  //   lap(s)(c)  = sum_j w_lap[c][j] s(n_j)           (Sec. 4 Laplacian)
  std::vector<double> w_div;      // ncol*7*3
  std::vector<double> w_grad;     // ncol*7*3
  std::vector<double> w_lap;      // ncol*7
  int spring_iters = 0, spring_converged = 0;
  int ntri() const { return (int)tri.size() / 3; }
};

// Returns 0 on success, a negative THOR status otherwise.
int build_grid(int glevel, int nv, double radius, double z_top, const SpringParams& sp,
               bool modified, HostGrid& g);

}  // namespace thor
