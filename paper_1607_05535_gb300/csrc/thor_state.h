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

struct thor_state {
  thor_grid* grid = nullptr;
  int precision = THOR_FP64;
  int check_finite = 0;
  ClosureBinding closure;
  std::unique_ptr<thor::ImplBase> impl;
};

namespace thor {
int closure_large_step(thor_state* s, int n_small, double dt);   // thor_mlp.cu
void closure_release(thor_state* s);
}
