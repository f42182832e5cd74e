// Device state of one atmosphere and the typed implementation behind the C
// ABI. R = double (THOR_FP64) or float (THOR_MIXED).
#pragma once

#include <vector>

#include "thor_kernels.cuh"

namespace thor {

// Derived fields and intermediates
template <typename R>
struct Work {
  R *pp, *Tp, *theta;              // p', T', theta at the centres
  R *vx, *vy, *vz;                 // full 3-D velocity at the centres
  R *vhx, *vhy, *vhz;              // horizontal velocity M / rho
  R *vr;                           // W / rho at the interfaces
  R *qrho, *qvx, *qvy, *qvz, *qT;  // K_d lap(.) (times rho) for the hyperdiffusion
  R *qvr;                          // interfaces
  R *dd;                           // 3-D divergence (small step)
  R *gx, *gy, *gz;                 // its horizontal gradient
};

// Slow tendencies and small-step coefficients of a stage
template <typename R>
struct Slow {
  R *smx, *smy, *smz, *srho, *sth, *dsc, *acr, *pi;  // centres
  R *sw, *thi;                                        // interfaces
};

// Small-step perturbations Phi* = Phi - Phi^(s)
template <typename R>
struct Pert {
  R *rho, *mx, *my, *mz, *th, *p;  // centres
  R *w;                            // interfaces
};

struct ImplBase {
  virtual ~ImplBase() { prof_clear(); }
  virtual int step(int n_large, int n_small, double dt) = 0;
  virtual int diag(double* out8, long long* nonfinite) = 0;
  virtual int get(int field, double* host, size_t n) = 0;
  virtual int set(int field, const double* host, size_t n) = 0;
  long long launches = 0;
  int kchunk = 8;                      // levels per thread in the stencil kernels
  // per-kernel event timing (off unless enabled)
  cudaStream_t stream = nullptr;
  bool prof_on = false;
  std::vector<cudaEvent_t> prof_ev;   // pairs (start, stop)
  std::vector<int> prof_id;           // kernel id of each pair
  size_t prof_used = 0;
  void prof_clear() {
    for (cudaEvent_t e : prof_ev) cudaEventDestroy(e);
    prof_ev.clear();
    prof_id.clear();
    prof_used = 0;
  }
  // bracket one launch: call with begin = true before and false after
  void mark(int id, bool begin) {
    if (!prof_on) return;
    if (begin) {
      if (prof_used == prof_id.size()) {
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        prof_ev.push_back(a);
        prof_ev.push_back(b);
        prof_id.push_back(id);
      }
      prof_id[prof_used] = id;
      cudaEventRecord(prof_ev[2 * prof_used], stream);
    } else {
      cudaEventRecord(prof_ev[2 * prof_used + 1], stream);
      ++prof_used;
    }
  }
  int prof_read(int id, double* ms, long long* n) {
    if (cudaStreamSynchronize(stream)) return -3;
    double t = 0;
    long long c = 0;
    for (size_t i = 0; i < prof_used; ++i)
      if (prof_id[i] == id) {
        float x = 0;
        if (cudaEventElapsedTime(&x, prof_ev[2 * i], prof_ev[2 * i + 1])) return -3;
        t += x;
        ++c;
      }
    *ms = t;
    *n = c;
    return 0;
  }
};

template <typename R>
struct Impl : ImplBase {
  Geo<R> G;
  Vert V;
  VR<R> U;
  Phys ph;
  Xf<R> Xt, Xst;
  Work<R> T;
  Slow<R> SL;
  Pert<R> P;
  int hyper = 1, divdamp = 1, forcing = 0;
  double diff_D = 0, dbar4 = 0, hj_dT = 300.0;
  // device allocations
  void* arena = nullptr;
  double* staging = nullptr;       // canonical-order float64 transfer buffer
  double* red = nullptr;           // reduction partials
  int red_blocks = 0;

  ~Impl() override;
  void launch_2d(int nplanes, int kchunk, dim3& grid) const;
  int large_step(double dt, int n_small);
  int step(int n_large, int n_small, double dt) override {
    for (int i = 0; i < n_large; ++i) {
      int rc = large_step(dt, n_small);
      if (rc) return rc;
    }
    return 0;
  }
  int diag(double* out8, long long* nonfinite) override;
  int get(int field, double* host, size_t n) override;
  int set(int field, const double* host, size_t n) override;
};

}  // namespace thor
