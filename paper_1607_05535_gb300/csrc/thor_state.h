// Handle structs behind the C ABI, shared by the translation units.
#pragma once

#include <memory>

#include "grid.h"
#include "thor_impl.cuh"

struct thor_mlp;

struct thor_grid {
  thor::HostGrid h;
};

// learned closure attached to a state (thor_closure_attach)
struct ClosureBinding {
  thor_mlp* net = nullptr;
  const float *in_mean = nullptr, *in_std = nullptr, *out_mean = nullptr, *out_std = nullptr;
  float *x = nullptr, *y = nullptr;   // per-state feature / output buffers
  int period = 1;                     // large steps per closure window
  long long counter = 0;              // large steps since attach
};

// zonal band means accumulated over time (thor_zonal_accumulate)
struct ZonalAcc {
  int nlat = 0;                       // bands (0: nothing allocated)
  int* band = nullptr;                // [colp] band of every column
  double* basis = nullptr;            // [6][colp] east and north unit vectors
  double* tmp = nullptr;              // [nv][nlat][9] sums of one state
  double* acc = nullptr;              // [nv][nlat][9] accumulated band means and covariances
  double* wsum = nullptr;             // [nv][colp] time sum of w at the centres of every cell
  long long samples = 0;
};

struct thor_state {
  thor_grid* grid = nullptr;
  int precision = THOR_FP64;
  int check_finite = 0;
  ClosureBinding closure;
  ZonalAcc zonal;
  std::unique_ptr<thor::ImplBase> impl;
};

namespace thor {
int closure_large_step(thor_state* s, int n_small, double dt);   // thor_mlp.cu
void closure_release(thor_state* s);
void zonal_release(ZonalAcc& z);                                  // thor_climate.cu
}
