// Device state of one atmosphere and the typed implementation behind the C
// ABI. R = double (THOR_FP64) or float (THOR_MIXED).
#pragma once

#include <cuda.h>

#include <memory>
#include <vector>

#include "thor_kernels.cuh"

namespace thor {

// L2 eviction priorities of the small-step kernels (THOR_TUNE_L2_HINTS);
// 0 on success
int set_l2_mode(int mode);

// Derived fields and intermediates
template <typename R>
struct Work {
  // packed [nv][colp][4] planes (one 16-byte gather per neighbour, ld4):
  // v4 = the full 3-D velocity and theta, vh4 = the horizontal velocity
  // M / rho and T', q4 = K_d lap(v_h) rho (x, y, z) and K_d lap(rho)
  R *v4, *vh4, *q4;
  R *pp, *theta;                   // p', theta at the centres
  R *vr;                           // W / rho at the interfaces
  R *wc;                           // W / rho at the centres (shallow atmosphere)
  R *qT;                           // K_d lap(T') rho for the hyperdiffusion
  R *qvr;                          // interfaces
  R *dd;                           // 3-D divergence (small step)
  R *dd0;                          // 3-D divergence of X^t (first small step of every stage)
  R *lp;                           // [nv][colp][2]: the Laplacian of that D and the cell's p*
  R *ca, *cb, *cc;                 // per-cell parts of the column equations (a, b, c)
  R *dhm;                          // horizontal divergence of the new M*
  R *psurf;                        // [colp] surface pressure (physics)
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
  R *rho, *th, *p;                 // centres
  R *m4;                           // [nv][colp][4]: M* (x, y, z) and theta of the stage state
  R *w;                            // interfaces
};

// TMA descriptors of the planes the staged column solve reads (float storage):
// each a 2-D map (x = column, y = plane) with a box of 32 columns x all planes
struct SolveMaps {
  CUtensorMap w, sw, cc, ca, thi, cb, pp, th_t, th_s, dsc, dhm;   // float
  CUtensorMap q, inv, cf, junction;                             // float64 factors
};

// Everything the kernels of one state need, as one record: a device array of
// these lets one launch step an ensemble of states of different sizes,
// planets and time steps.
template <typename R>
struct Member {
  Geo<R> G;
  VR<R> U;
  Phys ph;
  Xf<R> Xt, Xst;
  Xf<R> XtL;                       // low parts of a compensated X^t (null pointers: none)
  Work<R> T;
  Slow<R> SL;
  Pert<R> P;
  Fac<R> F;
  double dt, hj_dT;
  double dts[3];                   // small-step length of each RK stage
  R Kd;                            // hyperdiffusion coefficient for this dt
  int nsub[3];                     // small steps of each RK stage
  int hyper, divdamp, forcing, shallow;
  const SolveMaps* smap;           // device copy of the staged-solve descriptors (or null)
  int* err;                        // the state's device error flag
};

// device buffer of the energy fixer and budget: two diagnostics reductions
// (kDiagBlocks + 1 rows of 8 each), dT in float64, dT in the storage type
constexpr size_t kFixBufBytes = (size_t)(2 * (512 + 1) * 8 + 2) * sizeof(double);

struct ImplBase {
  virtual ~ImplBase() {
    prof_clear();
    if (fixbuf) cudaFree(fixbuf);
    if (budget) cudaFree(budget);
    if (budget_count) cudaFree(budget_count);
  }
  virtual void reset_graph() = 0;      // drop the captured step (its launches changed)
  virtual int step(int n_large, int n_small, double dt) = 0;
  virtual int diag(double* out8, long long* nonfinite) = 0;
  virtual int get(int field, double* host, size_t n) = 0;
  virtual int set(int field, const double* host, size_t n) = 0;
  // the four prognostic fields (RHO, MOM, W, RHOTHETA) with one synchronisation
  virtual int get_all(double* const host[4]) = 0;
  virtual int set_all(const double* const host[4]) = 0;
  virtual void set_graph(bool on) = 0;
  // compensated state (THOR_TUNE_COMPENSATED): on = 1 adds zeroed low parts
  // to the prognostic fields of a float state, on = 0 drops them (the state
  // rounds to its float parts); -1 for a float64 state
  virtual int set_compensated(int on) = 0;
  virtual bool anelastic() const = 0;
  int compensated = 0;
  long long launches = 0;
  int kchunk = 2;                      // levels per thread in the stencil kernels
  int block = kBlock;                  // threads (columns) per block of the stencil kernels
  int solve_tma = 1;                   // TMA-staged column solve where available
  int level_split = 1;                 // small-step stencils in two level halves on two streams
  int rk_stages = 3;                   // RK3 stages a large step runs (THOR_TUNE_RK_STAGES; tests)
  int* dev_err = nullptr;              // device flag: 1 = a bounded device wait timed out
  // energy fixer and budget (thor_tune THOR_TUNE_ENERGY_FIXER / THOR_TUNE_BUDGET)
  int energy_fix = 0;
  int budget_cap = 0;                  // large steps the budget can hold (0: not recording)
  double* fixbuf = nullptr;            // two diagnostics reductions, dT (float64 and storage type)
  double* budget = nullptr;            // [budget_cap][8]
  int* budget_count = nullptr;         // rows recorded
  // FNV-1a hash of what the stored deviations are relative to: the
  // reference column and vertical tables, the planet and the switches
  // (checkpoints record it and refuse to load into another)
  unsigned long long ref_hash = 0;
  // copy the prognostic fields to / from a device buffer of state_bytes()
  virtual size_t state_bytes() const = 0;
  virtual int save_state(void* dst) = 0;
  virtual int load_state(const void* src) = 0;
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
  Fac<R> F;
  // low parts of X^t when compensated (null pointers otherwise): the value
  // of a field is hi + lo, with |lo| at most half a unit in the last place of
  // hi; the stage state is stored as floats
  Xf<R> XtL{};
  void* lo_buf = nullptr;
  // anelastic switch: float64 work planes of the pressure solve, the
  // horizontal diagonal of its operator per column, solver limits
  void* an_buf = nullptr;
  double* an_dh = nullptr;
  int an_max_iter = 500;
  double an_tol = 1e-13;
  int an_last_iters = 0;
  int anelastic_step(double dt);
  int hyper = 1, divdamp = 1, forcing = 0;
  int shallow = 0;                 // shallow-atmosphere approximation (thor_init.shallow)
  double diff_D = 0, dbar4 = 0, hj_dT = 300.0;
  // device allocations
  void* arena = nullptr;
  double* staging = nullptr;       // canonical-order float64 transfer buffer (room for all four fields)
  double* red = nullptr;           // reduction partials
  int red_blocks = 0;

  int use_graph = 1;
  void set_graph(bool on) override {
    use_graph = on;
    if (!on) drop_graph();
  }
  void reset_graph() override { drop_graph(); }
  ~Impl() override;
  void launch_2d(int nplanes, int kchunk, dim3& grid) const;
  int large_step(double dt, int n_small);
  // CUDA graph of one large step, replayed while (dt, n_small, kchunk) stay
  // the same; used on a non-default stream when no profiling is recorded
  cudaGraphExec_t graph_exec = nullptr;
  double graph_dt = 0;
  int graph_n = 0, graph_kc = 0, graph_bs = 0, graph_tma = -1, graph_energy = -1, graph_stages = -1,
      graph_cmp = -1;
  std::unique_ptr<SolveMaps> smaps;   // null where the staged solve does not apply
  // second stream for the kernels of a stage that run beside others, forked
  // from and joined to the state's stream by events (null: everything on the
  // state's stream)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join0 = nullptr;
  // the small steps' stencils over the upper levels run on side2 beside the
  // lower levels on the state's stream (THOR_TUNE_LEVEL_SPLIT)
  cudaStream_t side2 = nullptr;
  cudaEvent_t ev_s1 = nullptr, ev_s2 = nullptr;
  // whole-state transfers: one event per field between its conversion (on
  // the state's stream) and its copy (on the side stream)
  cudaEvent_t ev_x[4] = {nullptr, nullptr, nullptr, nullptr};
  int build_solve_maps();
  cudaError_t launch_solve_tma(dim3 grid, int stage, const Xf<R>& Xo, const Xf<R>& XsL, const Xf<R>& XoL,
                               double dtau, int want_div, int last);
  long long graph_launches = 0;
  void drop_graph() {
    if (graph_exec) cudaGraphExecDestroy(graph_exec);
    graph_exec = nullptr;
  }
  int energy_key() const { return energy_fix * 2 + (budget_cap > 0 ? 1 : 0); }
  int step(int n_large, int n_small, double dt) override {
    if (ph.anelastic) {                  // host-driven solver iterations: no graph
      for (int i = 0; i < n_large; ++i) {
        int rc = anelastic_step(dt);
        if (rc) return rc;
      }
      return 0;
    }
    if (use_graph && stream != nullptr && !prof_on && n_large > 0) {
      if (!graph_exec || graph_dt != dt || graph_n != n_small || graph_kc != kchunk || graph_bs != block ||
          graph_tma != solve_tma || graph_energy != energy_key() || graph_stages != rk_stages ||
          graph_cmp != compensated) {
        drop_graph();
        cudaGraph_t g = nullptr;
        long long before = launches;
        if (cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal)) return -3;
        int rc = large_step(dt, n_small);
        cudaError_t e = cudaStreamEndCapture(stream, &g);
        if (rc || e) {
          if (g) cudaGraphDestroy(g);
          launches = before;
          return -3;
        }
        e = cudaGraphInstantiate(&graph_exec, g, 0);
        cudaGraphDestroy(g);
        graph_launches = launches - before;
        launches = before;
        if (e) {
          graph_exec = nullptr;
          return -3;
        }
        graph_dt = dt;
        graph_n = n_small;
        graph_kc = kchunk;
        graph_bs = block;
        graph_tma = solve_tma;
        graph_energy = energy_key();
        graph_stages = rk_stages;
        graph_cmp = compensated;
      }
      for (int i = 0; i < n_large; ++i) {
        if (cudaGraphLaunch(graph_exec, stream)) return -3;
        launches += graph_launches;
      }
      return 0;
    }
    for (int i = 0; i < n_large; ++i) {
      int rc = large_step(dt, n_small);
      if (rc) return rc;
    }
    return 0;
  }
  int diag(double* out8, long long* nonfinite) override;
  int get(int field, double* host, size_t n) override;
  int set(int field, const double* host, size_t n) override;
  int get_all(double* const host[4]) override;
  int set_all(const double* const host[4]) override;
  // queue one field (copy on cs, default the state's stream), no synchronisation
  int set_async(int field, const double* host, double* buf, cudaStream_t cs = nullptr);
  int set_compensated(int on) override;
  bool anelastic() const override { return ph.anelastic != 0; }
  // rho, M (3), rho theta: nv planes each; W: nv + 1 planes (and the same
  // again for the low parts of a compensated state); buf in device or host
  // memory (unified addressing)
  size_t state_bytes() const override {
    return (size_t)(6 * G.nv + 1) * G.colp * sizeof(R) * (compensated ? 2 : 1);
  }
  int copy_state(char* buf, bool save) {
    const size_t plane = (size_t)G.colp * sizeof(R), c = G.nv * plane;
    R* f[12] = {Xt.rho, Xt.mx, Xt.my, Xt.mz, Xt.th, Xt.w, XtL.rho, XtL.mx, XtL.my, XtL.mz, XtL.th, XtL.w};
    size_t off = 0;
    for (int i = 0; i < (compensated ? 12 : 6); ++i) {
      const size_t bytes = i % 6 == 5 ? c + plane : c;
      cudaError_t e = save ? cudaMemcpyAsync(buf + off, f[i], bytes, cudaMemcpyDefault, stream)
                           : cudaMemcpyAsync(f[i], buf + off, bytes, cudaMemcpyDefault, stream);
      if (e) return -3;
      off += bytes;
    }
    return 0;
  }
  int save_state(void* dst) override { return copy_state(static_cast<char*>(dst), true); }
  int load_state(const void* src) override { return copy_state(static_cast<char*>(const_cast<void*>(src)), false); }
  // this state's entry of an ensemble member table
  Member<R> member(double dt, int n_small) const {
    Member<R> m;
    m.G = G;
    m.U = U;
    m.ph = ph;
    m.Xt = Xt;
    m.Xst = Xst;
    m.XtL = XtL;
    m.T = T;
    m.SL = SL;
    m.P = P;
    m.F = F;
    m.dt = dt;
    m.hj_dT = hj_dT;
    m.dts[0] = dt / 3.0;
    m.dts[1] = m.dts[2] = dt / n_small;
    m.nsub[0] = 1;
    m.nsub[1] = n_small / 2;
    m.nsub[2] = n_small;
    m.Kd = (R)(diff_D * dbar4 / dt);
    m.hyper = hyper;
    m.divdamp = divdamp;
    m.forcing = forcing;
    m.shallow = shallow;
    m.smap = nullptr;
    m.err = dev_err;
    return m;
  }
};

// Launch plan of an ensemble large step (device member table and block maps
// built on the host; see ensemble_large_step)
template <typename R>
struct EnsPlan {
  const Member<R>* M = nullptr;
  const int2* map = nullptr;        // stencil blocks: (member, local block)
  const int2* mapc = nullptr;       // 32-column blocks of the column kernels
  int nv = 0, kchunk = 2, block = kBlock;
  int nblk = 0, nblkc = 0;          // all members
  int maxsub[3] = {0, 0, 0};
  std::vector<int> active[3], activec[3];  // blocks of the members still stepping at small step j
  int any_hyper = 0, any_divdamp = 0, any_forcing = 0;
  int staged = 0;                   // every member runs the TMA-staged column solve
  // the small steps' stencils in two level halves, the upper on side2,
  // forked and joined by ev_a / ev_b (null side2: one chain)
  cudaStream_t side2 = nullptr;
  cudaEvent_t ev_a = nullptr, ev_b = nullptr;
};

template <typename R>
int ensemble_large_step(const EnsPlan<R>& E, cudaStream_t stream, long long* launches);

}  // namespace thor
