// Ensembles of independent atmospheres stepped together, and the launch-shape
// autotuner.
//
// An ensemble holds states of different grid levels, planets and time steps
// (same level count and precision). Every kernel of the large step is one
// launch over all members: a block map sends each block of the launch to a
// (member, local block) pair, and a device table holds each member's arrays
// and constants (Member<R>). Members are ordered by decreasing n_small, so
// the members still inside their small-step loop form a prefix of the maps.
// On a non-default stream the whole ensemble large step is captured once as
// a CUDA graph and replayed.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "../../include/thor.h"
#include "thor_state.h"

namespace thor {

struct EnsBase {
  virtual ~EnsBase() {}
  virtual int step(int n_large, const int* n_small, const double* dt) = 0;
  virtual void drop_graph() = 0;
  long long launches = 0;
  int kchunk = 2, block = kBlock, use_graph = 1;
};

template <typename R>
struct EnsImpl : EnsBase {
  std::vector<Impl<R>*> mem;          // creation order
  std::vector<cudaStream_t> streams;  // distinct member streams other than the ensemble's
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // the upper level halves of the small steps' stencils (a graph branch)
  cudaStream_t side2 = nullptr;
  cudaEvent_t ev_a = nullptr, ev_b = nullptr;
  EnsPlan<R> plan;
  Member<R>* dM = nullptr;
  SolveMaps* dmaps = nullptr;          // members' staged-solve descriptors, in plan order
  int2 *dmap = nullptr, *dmapc = nullptr;
  size_t cap_map = 0, cap_mapc = 0;
  // plan key
  bool planned = false;
  std::vector<int> key_n;
  std::vector<double> key_dt;
  std::vector<const void*> key_lo;    // members' low-part planes (compensated state) at planning
  int key_kc = 0, key_bs = 0;
  cudaGraphExec_t gexec = nullptr;
  long long graph_launches = 0;

  ~EnsImpl() override {
    drop_graph();
    if (dM) cudaFree(dM);
    if (dmaps) cudaFree(dmaps);
    if (dmap) cudaFree(dmap);
    if (dmapc) cudaFree(dmapc);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (side2) {
      cudaStreamSynchronize(side2);
      cudaStreamDestroy(side2);
    }
    if (ev_a) cudaEventDestroy(ev_a);
    if (ev_b) cudaEventDestroy(ev_b);
  }
  void drop_graph() override {
    if (gexec) cudaGraphExecDestroy(gexec);
    gexec = nullptr;
  }

  int build_plan(const int* n_small, const double* dt) {
    const int n = (int)mem.size();
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n_small[a] > n_small[b]; });
    std::vector<Member<R>> tab(n);
    std::vector<int2> map, mapc;
    std::vector<int> nb(n), nbc(n);
    EnsPlan<R> p;
    p.nv = mem[0]->G.nv;
    p.kchunk = kchunk;
    p.block = block;
    p.side2 = side2;
    p.ev_a = ev_a;
    p.ev_b = ev_b;
    for (int q = 0; q < n; ++q) {
      const int i = order[q];
      const Impl<R>* I = mem[i];
      tab[q] = I->member(dt[i], n_small[i]);
      nb[q] = (I->G.ncol + block - 1) / block;
      nbc[q] = (I->G.ncol + 31) / 32;
      for (int b = 0; b < nb[q]; ++b) map.push_back(make_int2(q, b));
      for (int b = 0; b < nbc[q]; ++b) mapc.push_back(make_int2(q, b));
      p.any_hyper |= I->hyper;
      p.any_divdamp |= I->divdamp;
      p.any_forcing |= I->forcing != 0;
    }
    p.nblk = (int)map.size();
    p.nblkc = (int)mapc.size();
    // staged column solve when every member has its descriptors
    std::vector<SolveMaps> smaps;
    p.staged = 1;
    for (int q = 0; q < n; ++q) {
      const Impl<R>* I = mem[order[q]];
      if (!I->solve_tma || !I->smaps) {
        p.staged = 0;
        break;
      }
      smaps.push_back(*I->smaps);
    }
    for (int s = 0; s < 3; ++s) {
      p.maxsub[s] = tab[0].nsub[s];
      for (int j = 0; j < p.maxsub[s]; ++j) {
        int a = 0, ac = 0;
        for (int q = 0; q < n && tab[q].nsub[s] > j; ++q) {
          a += nb[q];
          ac += nbc[q];
        }
        p.active[s].push_back(a);
        p.activec[s].push_back(ac);
      }
    }
    drop_graph();
    // the previous plan's launches may still read the old tables
    if (cudaStreamSynchronize(stream)) return THOR_ECUDA;
    if (!dM && cudaMalloc(&dM, n * sizeof(Member<R>))) return THOR_ENOMEM;
    if (map.size() > cap_map) {
      if (dmap) cudaFree(dmap);
      dmap = nullptr;
      if (cudaMalloc(&dmap, map.size() * sizeof(int2))) return THOR_ENOMEM;
      cap_map = map.size();
    }
    if (mapc.size() > cap_mapc) {
      if (dmapc) cudaFree(dmapc);
      dmapc = nullptr;
      if (cudaMalloc(&dmapc, mapc.size() * sizeof(int2))) return THOR_ENOMEM;
      cap_mapc = mapc.size();
    }
    if (p.staged) {
      if (!dmaps && cudaMalloc(&dmaps, n * sizeof(SolveMaps))) return THOR_ENOMEM;
      if (cudaMemcpy(dmaps, smaps.data(), n * sizeof(SolveMaps), cudaMemcpyHostToDevice)) return THOR_ECUDA;
      for (int q = 0; q < n; ++q) tab[q].smap = dmaps + q;
    }
    if (cudaMemcpy(dM, tab.data(), n * sizeof(Member<R>), cudaMemcpyHostToDevice) ||
        cudaMemcpy(dmap, map.data(), map.size() * sizeof(int2), cudaMemcpyHostToDevice) ||
        cudaMemcpy(dmapc, mapc.data(), mapc.size() * sizeof(int2), cudaMemcpyHostToDevice))
      return THOR_ECUDA;
    p.M = dM;
    p.map = dmap;
    p.mapc = dmapc;
    plan = std::move(p);
    key_n.assign(n_small, n_small + n);
    key_dt.assign(dt, dt + n);
    key_kc = kchunk;
    key_bs = block;
    key_lo.clear();
    for (const Impl<R>* I : mem) key_lo.push_back(I->XtL.rho);
    planned = true;
    return THOR_OK;
  }

  int step(int n_large, const int* n_small, const double* dt) override {
    const int n = (int)mem.size();
    bool lo_same = key_lo.size() == mem.size();
    for (size_t i = 0; lo_same && i < mem.size(); ++i) lo_same = key_lo[i] == mem[i]->XtL.rho;
    if (!planned || key_kc != kchunk || key_bs != block || !std::equal(key_n.begin(), key_n.end(), n_small) ||
        !std::equal(key_dt.begin(), key_dt.end(), dt) || !lo_same) {
      int rc = build_plan(n_small, dt);
      if (rc) return rc;
    }
    (void)n;
    // order against work already queued on the members' own streams
    for (cudaStream_t ms : streams) {
      if (cudaEventRecord(ev_in, ms) || cudaStreamWaitEvent(stream, ev_in, 0)) return THOR_ECUDA;
    }
    if (use_graph && stream != nullptr && n_large > 0) {
      if (!gexec) {
        cudaGraph_t g = nullptr;
        long long l = 0;
        if (cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal)) return THOR_ECUDA;
        int rc = ensemble_large_step<R>(plan, stream, &l);
        cudaError_t e = cudaStreamEndCapture(stream, &g);
        if (rc || e) {
          if (g) cudaGraphDestroy(g);
          return THOR_ECUDA;
        }
        e = cudaGraphInstantiate(&gexec, g, 0);
        cudaGraphDestroy(g);
        if (e) {
          gexec = nullptr;
          return THOR_ECUDA;
        }
        graph_launches = l;
      }
      for (int i = 0; i < n_large; ++i) {
        if (cudaGraphLaunch(gexec, stream)) return THOR_ECUDA;
        launches += graph_launches;
      }
    } else {
      for (int i = 0; i < n_large; ++i) {
        int rc = ensemble_large_step<R>(plan, stream, &launches);
        if (rc) return THOR_ECUDA;
      }
    }
    if (cudaEventRecord(ev_out, stream)) return THOR_ECUDA;
    for (cudaStream_t ms : streams)
      if (cudaStreamWaitEvent(ms, ev_out, 0)) return THOR_ECUDA;
    return THOR_OK;
  }
};

// Times `steps` large steps (after one untimed step, which also captures a
// graph where one is used) for every candidate launch shape, restoring the
// prognostic state before each candidate and at the end; leaves the fastest
// shape set.
template <typename Run, typename Set, typename Save>
int autotune_loop(cudaStream_t st, int steps, Run run, Set set, Save save_restore, int* best_kc, int* best_bs,
                  double* best_ms) {
  // levels per thread and block sizes that need not divide the level and
  // column counts (3 levels and 128 columns win at glevel 6 x 32 levels)
  static const int kcs[] = {1, 2, 3, 4, 6, 8};
  static const int bss[] = {64, 96, 128, 192, 256};
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) || cudaEventCreate(&b)) return THOR_ECUDA;
  int rc = save_restore(true);
  double best = -1.0;
  int bk = 2, bb = kBlock;
  for (int kc : kcs) {
    for (int bs : bss) {
      if (rc) break;
      set(kc, bs);
      rc = run(1);
      if (!rc && cudaEventRecord(a, st)) rc = THOR_ECUDA;
      if (!rc) rc = run(steps);
      if (!rc && cudaEventRecord(b, st)) rc = THOR_ECUDA;
      float ms = 0.f;
      if (!rc && (cudaEventSynchronize(b) || cudaEventElapsedTime(&ms, a, b))) rc = THOR_ECUDA;
      if (!rc) rc = save_restore(false);
      if (!rc && (best < 0 || ms < best)) {
        best = ms;
        bk = kc;
        bb = bs;
      }
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc) return rc;
  set(bk, bb);
  if (best_kc) *best_kc = bk;
  if (best_bs) *best_bs = bb;
  if (best_ms) *best_ms = best / steps;
  return THOR_OK;
}

}  // namespace thor

struct thor_ensemble {
  std::vector<thor_state*> members;
  int precision = THOR_FP64;
  cudaStream_t stream = nullptr;
  std::unique_ptr<thor::EnsBase> impl;
};

namespace {

template <typename R>
int make_ens(thor_ensemble* E) {
  using namespace thor;
  auto impl = std::make_unique<EnsImpl<R>>();
  impl->stream = E->stream;
  for (thor_state* s : E->members) {
    impl->mem.push_back(static_cast<Impl<R>*>(s->impl.get()));
    cudaStream_t ms = s->impl->stream;
    if (ms != E->stream && std::find(impl->streams.begin(), impl->streams.end(), ms) == impl->streams.end())
      impl->streams.push_back(ms);
  }
  if (cudaEventCreateWithFlags(&impl->ev_in, cudaEventDisableTiming) ||
      cudaEventCreateWithFlags(&impl->ev_out, cudaEventDisableTiming))
    return THOR_ECUDA;
  // optional: without it the stencils run as one chain
  if (cudaStreamCreateWithFlags(&impl->side2, cudaStreamNonBlocking) ||
      cudaEventCreateWithFlags(&impl->ev_a, cudaEventDisableTiming) ||
      cudaEventCreateWithFlags(&impl->ev_b, cudaEventDisableTiming)) {
    cudaGetLastError();
    if (impl->side2) cudaStreamDestroy(impl->side2);
    impl->side2 = nullptr;
  }
  E->impl = std::move(impl);
  return THOR_OK;
}

int check_steps(const thor_ensemble* E, int n_large, const int* n_small, const double* dt) {
  if (!E || n_large < 0 || !n_small || !dt) return THOR_EINVAL;
  for (size_t i = 0; i < E->members.size(); ++i) {
    if (n_small[i] < 2 || (n_small[i] % 2) || !(dt[i] > 0)) return THOR_EINVAL;
    if (E->members[i]->closure.net || E->members[i]->impl->anelastic()) return THOR_EINVAL;
  }
  return THOR_OK;
}

}  // namespace

extern "C" {

int thor_ensemble_create(thor_state* const* members, int n, void* stream, thor_ensemble** out) {
  if (!members || !out || n < 1 || n > THOR_ENSEMBLE_MAX) return THOR_EINVAL;
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!members[i]) return THOR_EINVAL;
    if (members[i]->precision != members[0]->precision || members[i]->grid->h.nv != members[0]->grid->h.nv)
      return THOR_EINVAL;
    for (int j = 0; j < i; ++j)
      if (members[j] == members[i]) return THOR_EINVAL;
  }
  auto E = std::make_unique<thor_ensemble>();
  E->members.assign(members, members + n);
  E->precision = members[0]->precision;
  E->stream = static_cast<cudaStream_t>(stream);
  int rc = E->precision == THOR_FP64 ? make_ens<double>(E.get()) : make_ens<float>(E.get());
  if (rc) return rc;
  *out = E.release();
  return THOR_OK;
}

int thor_ensemble_step(thor_ensemble* E, int n_large, const int* n_small, const double* dt) {
  int rc = check_steps(E, n_large, n_small, dt);
  if (rc) return rc;
  if (n_large == 0) return THOR_OK;
  return E->impl->step(n_large, n_small, dt);
}

int thor_ensemble_info(const thor_ensemble* E, int* n_members, long long* launches) {
  if (!E) return THOR_EINVAL;
  if (n_members) *n_members = (int)E->members.size();
  if (launches) *launches = E->impl->launches;
  return THOR_OK;
}

int thor_ensemble_tune(thor_ensemble* E, int knob, int value) {
  if (!E) return THOR_EINVAL;
  if (knob == THOR_TUNE_KCHUNK) {
    if (value < 1 || value > 256) return THOR_EINVAL;
    E->impl->kchunk = value;
    return THOR_OK;
  }
  if (knob == THOR_TUNE_BLOCK) {
    if (value < 32 || value > thor::kMaxBlock || value % 32) return THOR_EINVAL;
    E->impl->block = value;
    return THOR_OK;
  }
  if (knob == THOR_TUNE_GRAPH) {
    E->impl->use_graph = value != 0;
    if (!value) E->impl->drop_graph();
    return THOR_OK;
  }
  return THOR_EINVAL;
}

void thor_ensemble_destroy(thor_ensemble* E) {
  if (!E) return;
  if (E->stream) cudaStreamSynchronize(E->stream);
  else cudaDeviceSynchronize();
  delete E;
}

int thor_autotune(thor_state* s, int n_small, double dt, int steps, int* kchunk, int* block, double* ms_per_step) {
  using namespace thor;
  if (!s || n_small < 2 || (n_small % 2) || !(dt > 0) || steps < 1) return THOR_EINVAL;
  ImplBase* I = s->impl.get();
  void* buf = nullptr;
  if (cudaMalloc(&buf, I->state_bytes())) return THOR_ENOMEM;
  auto run = [&](int k) { return I->step(k, n_small, dt) ? THOR_ECUDA : THOR_OK; };
  auto set = [&](int kc, int bs) {
    I->kchunk = kc;
    I->block = bs;
  };
  auto sr = [&](bool save) { return (save ? I->save_state(buf) : I->load_state(buf)) ? THOR_ECUDA : THOR_OK; };
  int rc = autotune_loop(I->stream, steps, run, set, sr, kchunk, block, ms_per_step);
  cudaStreamSynchronize(I->stream);
  cudaFree(buf);
  return rc;
}

int thor_ensemble_autotune(thor_ensemble* E, const int* n_small, const double* dt, int steps, int* kchunk,
                           int* block, double* ms_per_step) {
  using namespace thor;
  int rc = check_steps(E, 1, n_small, dt);
  if (rc || steps < 1) return rc ? rc : THOR_EINVAL;
  const size_t n = E->members.size();
  std::vector<void*> bufs(n, nullptr);
  for (size_t i = 0; i < n; ++i)
    if (cudaMalloc(&bufs[i], E->members[i]->impl->state_bytes())) {
      for (void* b : bufs)
        if (b) cudaFree(b);
      return THOR_ENOMEM;
    }
  EnsBase* I = E->impl.get();
  // member copies run on the members' streams; order them with the ensemble's
  auto sync_all = [&]() {
    for (thor_state* m : E->members)
      if (cudaStreamSynchronize(m->impl->stream)) return THOR_ECUDA;
    return cudaStreamSynchronize(E->stream) ? THOR_ECUDA : THOR_OK;
  };
  auto run = [&](int k) { return I->step(k, n_small, dt); };
  auto set = [&](int kc, int bs) {
    I->kchunk = kc;
    I->block = bs;
  };
  auto sr = [&](bool save) {
    int r = sync_all();
    for (size_t i = 0; i < n && !r; ++i) {
      ImplBase* M = E->members[i]->impl.get();
      r = (save ? M->save_state(bufs[i]) : M->load_state(bufs[i])) ? THOR_ECUDA : THOR_OK;
    }
    return r ? r : sync_all();
  };
  rc = autotune_loop(E->stream, steps, run, set, sr, kchunk, block, ms_per_step);
  sync_all();
  for (void* b : bufs) cudaFree(b);
  return rc;
}

}  // extern "C"
