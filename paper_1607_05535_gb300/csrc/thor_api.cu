// C ABI of libthor (declared in include/thor.h): handles, initial state,
// field transfer in the canonical order, diagnostics.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "../../include/thor.h"
#include "grid.h"
#include "thor_impl.cuh"
#include "thor_reduce.cuh"

#include "thor_state.h"

namespace thor {
template <typename R>
int col_kernel_setup(int nv);   // thor_step.cu: opt the column kernel into its shared memory
// thor_anelastic.cu: the pressure solve of the anelastic switch
std::vector<double> anelastic_hdiag(const HostGrid& h);
template <typename R>
int anelastic_setup(Impl<R>& I, const std::vector<double>& hdiag);
namespace {

inline int colp_of(int ncol) { return (ncol + kBlock - 1) / kBlock * kBlock; }
constexpr int kNumVertCentre = 12, kNumVert = 19;   // float64 vertical arrays (centres, total)

uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// ------------------------------------------------------------ transfers

// canonical float64 [ncol][nv(+1)][ncomp] -> device planes, reference removed;
// with low planes l0.. (a compensated state) the value is split into its
// storage-type part and the remainder
template <typename R>
__global__ void k_from_canonical(const double* src, int ncol, int colp, int nlev, int ncomp,
                                 const double* ref, R* d0, R* d1, R* d2, R* l0, R* l1, R* l2, int zero_ends) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  int k = blockIdx.y;
  if (c >= ncol) return;
  R* dst[3] = {d0, d1, d2};
  R* low[3] = {l0, l1, l2};
  for (int j = 0; j < ncomp; ++j) {
    double v = src[((size_t)c * nlev + k) * ncomp + j];
    if (ref) v -= ref[k];
    if (zero_ends && (k == 0 || k == nlev - 1)) v = 0.0;
    const R hi = (R)v;
    dst[j][(size_t)k * colp + c] = hi;
    if (low[j]) low[j][(size_t)k * colp + c] = (R)(v - (double)hi);
  }
}

// device planes -> canonical float64; field selects the reconstruction; XL:
// the low parts of a compensated state (null: none)
template <typename R>
__global__ void k_to_canonical(double* dst, Geo<R> G, Vert V, Phys ph, Xf<R> X, Xf<R> XL, int field) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  int k = blockIdx.y;
  if (c >= G.ncol) return;
  const int S = G.colp, nv = G.nv;
  size_t i = (size_t)k * S + c;
  auto val = [&](const R* hi, const R* lo) { return lo ? (double)hi[i] + (double)lo[i] : (double)hi[i]; };
  switch (field) {
    case THOR_FIELD_RHO:
      dst[(size_t)c * nv + k] = V.rhob[k] + val(X.rho, XL.rho);
      break;
    case THOR_FIELD_MOM:
      dst[((size_t)c * nv + k) * 3 + 0] = val(X.mx, XL.mx);
      dst[((size_t)c * nv + k) * 3 + 1] = val(X.my, XL.my);
      dst[((size_t)c * nv + k) * 3 + 2] = val(X.mz, XL.mz);
      break;
    case THOR_FIELD_W:
      dst[(size_t)c * (nv + 1) + k] = val(X.w, XL.w);
      break;
    case THOR_FIELD_RHOTHETA:
      dst[(size_t)c * nv + k] = V.thb[k] + val(X.th, XL.th);
      break;
    case THOR_FIELD_PRESSURE:
    case THOR_FIELD_TEMPERATURE: {
      double thp = val(X.th, XL.th);
      double p = V.pb[k] + V.pb[k] * expm1(ph.gamma * log1p(thp / V.thb[k]));
      if (field == THOR_FIELD_PRESSURE) {
        dst[(size_t)c * nv + k] = p;
      } else {
        double rho = V.rhob[k] + val(X.rho, XL.rho);
        dst[(size_t)c * nv + k] = p / (rho * ph.Rd);
      }
      break;
    }
  }
}

// The bounded mbarrier wait of the staged solve and of the tensor-core GEMM,
// on a barrier of one expected arrival: with arrive = 0 nothing arrives and
// the wait must give up after limit_ns; with arrive = 1 the thread arrives
// first and the wait must succeed. out = 1 if the wait gave up, else 0.
__global__ void k_wait_probe(int arrive, unsigned long long limit_ns, int* out) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  mbar_init_fence();
  if (arrive) mbar_arrive(&bar);
  *out = mbar_wait(&bar, 0, limit_ns) ? 0 : 1;
}


// ------------------------------------------------------------ allocation

struct Carver {
  char* base;
  size_t off = 0;
  template <typename T>
  T* take(size_t n) {
    size_t bytes = (n * sizeof(T) + 255) / 256 * 256;
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += bytes;
    return p;
  }
};

// the VR arrays in a fixed order (all allocated with nv + 1 entries)
template <typename R>
std::vector<const R**> vr_slots(VR<R>& U) {
  return {&U.inv_rc, &U.inv_rc2, &U.sv, &U.ri2, &U.wlo, &U.whi, &U.clo, &U.chi, &U.inv_dzc,
          &U.rhob, &U.thb, &U.pb, &U.Tb, &U.Rb, &U.zc, &U.sq_lo, &U.sq_hi};
}

template <typename R>
void carve(Carver& cv, Impl<R>& I, int ncol, int nv) {
  const size_t S = (size_t)colp_of(ncol);
  const size_t C = S * nv, F = S * (nv + 1);
  auto X = [&](Xf<R>& x) {
    x.rho = cv.take<R>(C); x.mx = cv.take<R>(C); x.my = cv.take<R>(C); x.mz = cv.take<R>(C);
    x.th = cv.take<R>(C); x.w = cv.take<R>(F);
  };
  X(I.Xt);
  X(I.Xst);
  Work<R>& T = I.T;
  R** cen[] = {&T.pp, &T.theta, &T.qT, &T.dd, &T.dd0, &T.ca, &T.cb, &T.cc, &T.dhm};
  for (R** p : cen) *p = cv.take<R>(C);
  T.v4 = cv.take<R>(4 * C);
  T.vh4 = cv.take<R>(4 * C);
  T.q4 = cv.take<R>(4 * C);
  T.vr = cv.take<R>(F);
  T.qvr = cv.take<R>(F);
  T.wc = cv.take<R>(C);
  T.psurf = cv.take<R>(S);
  Slow<R>& SL = I.SL;
  R** sc[] = {&SL.smx, &SL.smy, &SL.smz, &SL.srho, &SL.sth, &SL.dsc, &SL.acr, &SL.pi};
  for (R** p : sc) *p = cv.take<R>(C);
  SL.sw = cv.take<R>(F);
  SL.thi = cv.take<R>(F);
  Pert<R>& P = I.P;
  R** pc[] = {&P.rho, &P.th, &P.p};
  for (R** p : pc) *p = cv.take<R>(C);
  P.m4 = cv.take<R>(4 * C);
  T.lp = cv.take<R>(2 * C);
  P.w = cv.take<R>(F);
  I.F.inv = cv.take<double>(F);
  I.F.cf = cv.take<double>(F);
  I.F.q = cv.take<double>(F);
  I.F.junction = cv.take<double>(S);
  // tables
  I.G.nbr = cv.take<int>(6 * S);
  I.G.wdiv = cv.take<R>(28 * S);
  I.G.wgrad = cv.take<R>(28 * S);
  I.G.wlap = cv.take<R>(7 * S);
  I.G.rhat = cv.take<R>(3 * S);
  I.G.gcor = cv.take<R>(3 * S);
  I.G.sinlat = cv.take<R>(S);
  I.G.coslat = cv.take<R>(S);
  I.G.xdir = cv.take<R>(S);
  I.G.area = cv.take<double>(S);
  const double** vp[] = {&I.V.rc, &I.V.dz, &I.V.clo, &I.V.chi, &I.V.zc, &I.V.rhob, &I.V.thb, &I.V.pb,
                         &I.V.Tb, &I.V.sv, &I.V.sq_lo, &I.V.sq_hi};
  for (const double** p : vp) *p = cv.take<double>(nv);
  const double** vi[] = {&I.V.ri, &I.V.dzc, &I.V.wlo, &I.V.whi, &I.V.Rb, &I.V.ri2, &I.V.inv_dzc};
  for (const double** p : vi) *p = cv.take<double>(nv + 1);
  for (const R** p : vr_slots(I.U)) *p = cv.take<R>(nv + 1);
  I.U.iw = cv.take<R>(4 * (size_t)(nv + 1));
  I.U.cw = cv.take<R>(4 * (size_t)nv);
  I.U.ij0 = cv.take<int>(nv + 1);
  I.U.cj0 = cv.take<int>(nv);
  I.staging = cv.take<double>((size_t)ncol * (6 * nv + 1));    // rho, 3 x rho v_h, W, rho theta
  I.red = cv.take<double>((size_t)(kDiagBlocks + 1) * 8);
  I.dev_err = cv.take<int>(64);
}

// Vertical grid, reference column and initial state in float64 on the host.
struct HostSetup {
  // rc dz clo chi zc rhob thb pb Tb sv sq_lo sq_hi | ri dzc wlo whi Rb ri2 inv_dzc
  std::vector<double> vert[kNumVert];
  std::vector<double> rho, th;    // canonical [ncol][nv]
  // order-k Lagrange tables of the explicit vertical interpolations
  std::vector<double> iw, cw;     // [4][nv + 1], [4][nv]
  std::vector<int> ij0, cj0;      // [nv + 1], [nv]
};
template <typename R>
int upload_tables(Impl<R>& I, const HostGrid& h, const std::vector<double>* vert, const HostSetup* lag,
                  cudaStream_t st) {
  const int ncol = h.ncol, S = colp_of(ncol), nv = h.nv;
  std::vector<int> nbr(6 * (size_t)S, 0);
  std::vector<R> wdiv(28 * (size_t)S, 0), wgrad(28 * (size_t)S, 0), wlap(7 * (size_t)S, 0),
      rhat(3 * (size_t)S, 0), gcor(3 * (size_t)S, 0), sl(S, 0), cl(S, 0), clon(S, 0);
  std::vector<double> area(S, 0.0);
  for (int c = 0; c < ncol; ++c) {
    for (int j = 0; j < 6; ++j) {
      int q = h.nbr[6 * c + j];
      nbr[(size_t)j * S + c] = q < 0 ? c : q;
    }
    for (int j = 0; j < 7; ++j) {
      const size_t q = ((size_t)j * S + c) * 4;        // packed [7][colp][4]
      for (int d = 0; d < 3; ++d) {
        wdiv[q + d] = (R)h.w_div[21 * c + 3 * j + d];
        wgrad[q + d] = (R)h.w_grad[21 * c + 3 * j + d];
      }
      wgrad[q + 3] = (R)h.w_lap[7 * c + j];
      wdiv[q + 3] = (R)h.w_lap[7 * c + j];
      wlap[(size_t)j * S + c] = (R)h.w_lap[7 * c + j];
    }
    for (int d = 0; d < 3; ++d) gcor[(size_t)d * S + c] = (R)(h.w_grad[21 * c + d] - h.w_div[21 * c + d]);
    double x = h.P[3 * c], y = h.P[3 * c + 1], z = h.P[3 * c + 2];
    rhat[c] = (R)x;
    rhat[S + c] = (R)y;
    rhat[2 * S + c] = (R)z;
    double lat = std::asin(std::fmax(-1.0, std::fmin(1.0, z)));
    sl[c] = (R)std::sin(lat);
    cl[c] = (R)std::cos(lat);
    clon[c] = (R)x;   // cos(lon) cos(lat), well defined at the poles
    area[c] = h.area[c];
  }
  auto up = [&](const void* dst, const void* src, size_t bytes) {
    return cudaMemcpyAsync(const_cast<void*>(dst), src, bytes, cudaMemcpyHostToDevice, st);
  };
  cudaError_t e = cudaSuccess;
  e = e ? e : up(I.G.nbr, nbr.data(), nbr.size() * sizeof(int));
  e = e ? e : up(I.G.wdiv, wdiv.data(), wdiv.size() * sizeof(R));
  e = e ? e : up(I.G.wgrad, wgrad.data(), wgrad.size() * sizeof(R));
  e = e ? e : up(I.G.wlap, wlap.data(), wlap.size() * sizeof(R));
  e = e ? e : up(I.G.rhat, rhat.data(), rhat.size() * sizeof(R));
  e = e ? e : up(I.G.gcor, gcor.data(), gcor.size() * sizeof(R));
  e = e ? e : up(I.G.sinlat, sl.data(), sl.size() * sizeof(R));
  e = e ? e : up(I.G.coslat, cl.data(), cl.size() * sizeof(R));
  e = e ? e : up(I.G.xdir, clon.data(), clon.size() * sizeof(R));
  e = e ? e : up(I.G.area, area.data(), area.size() * sizeof(double));
  const double* vp[] = {I.V.rc, I.V.dz, I.V.clo, I.V.chi, I.V.zc, I.V.rhob, I.V.thb, I.V.pb, I.V.Tb,
                        I.V.sv, I.V.sq_lo, I.V.sq_hi, I.V.ri, I.V.dzc, I.V.wlo, I.V.whi, I.V.Rb,
                        I.V.ri2, I.V.inv_dzc};
  for (int j = 0; j < kNumVert; ++j) {
    size_t cnt = j < kNumVertCentre ? nv : nv + 1;
    e = e ? e : up(vp[j], vert[j].data(), cnt * sizeof(double));
  }
  // storage-type copies with the reciprocals precomputed
  {
    const std::vector<double>& rc = vert[0];
    std::vector<std::vector<R>> vr(17, std::vector<R>(nv + 1, R(0)));
    for (int k = 0; k < nv; ++k) {
      vr[0][k] = (R)(1.0 / rc[k]);
      vr[1][k] = (R)(1.0 / (rc[k] * rc[k]));
      vr[2][k] = (R)vert[9][k];
      vr[6][k] = (R)vert[2][k];
      vr[7][k] = (R)vert[3][k];
      vr[9][k] = (R)vert[5][k];
      vr[10][k] = (R)vert[6][k];
      vr[11][k] = (R)vert[7][k];
      vr[12][k] = (R)vert[8][k];
      vr[14][k] = (R)vert[4][k];
      vr[15][k] = (R)vert[10][k];
      vr[16][k] = (R)vert[11][k];
    }
    for (int i = 0; i <= nv; ++i) {
      vr[3][i] = (R)vert[17][i];
      vr[4][i] = (R)vert[14][i];
      vr[5][i] = (R)vert[15][i];
      vr[8][i] = (R)vert[18][i];
      vr[13][i] = (R)vert[16][i];
    }
    std::vector<const R**> slots = vr_slots(I.U);
    for (int j = 0; j < 17; ++j) e = e ? e : up(*slots[j], vr[j].data(), (nv + 1) * sizeof(R));
    std::vector<R> iw(lag->iw.begin(), lag->iw.end()), cw(lag->cw.begin(), lag->cw.end());
    e = e ? e : up(I.U.iw, iw.data(), iw.size() * sizeof(R));
    e = e ? e : up(I.U.cw, cw.data(), cw.size() * sizeof(R));
    e = e ? e : up(I.U.ij0, lag->ij0.data(), lag->ij0.size() * sizeof(int));
    e = e ? e : up(I.U.cj0, lag->cj0.data(), lag->cj0.size() * sizeof(int));
    if (e) return THOR_ECUDA;
    if (cudaStreamSynchronize(st)) return THOR_ECUDA;   // host vectors die here
  }
  if (e) return THOR_ECUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? THOR_OK : THOR_ECUDA;
}

}  // namespace

// ------------------------------------------------------------ Impl methods

template <typename R>
Impl<R>::~Impl() {
  drop_graph();
  if (side) {
    cudaStreamSynchronize(side);
    cudaStreamDestroy(side);
  }
  if (side2) {
    cudaStreamSynchronize(side2);
    cudaStreamDestroy(side2);
  }
  if (ev_s1) cudaEventDestroy(ev_s1);
  if (ev_s2) cudaEventDestroy(ev_s2);
  if (ev_fork) cudaEventDestroy(ev_fork);
  if (ev_join) cudaEventDestroy(ev_join);
  if (ev_join0) cudaEventDestroy(ev_join0);
  for (cudaEvent_t e : ev_x)
    if (e) cudaEventDestroy(e);
  if (arena) cudaFree(arena);
  if (lo_buf) cudaFree(lo_buf);
  if (an_buf) cudaFree(an_buf);
}

// the element count of a field in the canonical layout of thor_state_get
static size_t field_count(int field, int ncol, int nv) {
  return field == THOR_FIELD_MOM ? (size_t)ncol * nv * 3 : field == THOR_FIELD_W ? (size_t)ncol * (nv + 1)
                                                                                 : (size_t)ncol * nv;
}

template <typename R>
int Impl<R>::get(int field, double* host, size_t n) {
  const int nv = G.nv;
  const size_t need = field_count(field, G.ncol, nv);
  if (field < 0 || field > THOR_FIELD_TEMPERATURE || n != need || !host) return THOR_EINVAL;
  int nlev = field == THOR_FIELD_W ? nv + 1 : nv;
  dim3 grid((G.ncol + 127) / 128, nlev);
  k_to_canonical<R><<<grid, 128, 0, stream>>>(staging, G, V, ph, Xt, XtL, field);
  ++launches;
  if (cudaMemcpyAsync(host, staging, need * sizeof(double), cudaMemcpyDeviceToHost, stream)) return THOR_ECUDA;
  return cudaStreamSynchronize(stream) == cudaSuccess ? THOR_OK : THOR_ECUDA;
}

template <typename R>
int Impl<R>::set(int field, const double* host, size_t n) {
  if (!host || n != field_count(field, G.ncol, G.nv)) return THOR_EINVAL;
  const int rc = set_async(field, host, staging);
  if (rc) return rc;
  return cudaStreamSynchronize(stream) == cudaSuccess ? THOR_OK : THOR_ECUDA;
}

// All four fields: with the side stream, the copies run back to back on it
// and each field's conversion on the state's stream waits for its own copy
// (set) or the copy waits for its conversion (get), so conversions overlap
// the other fields' copies; every field has its own region of the staging
// buffer.
template <typename R>
int Impl<R>::set_all(const double* const host[4]) {
  for (int f = 0; f < 4; ++f)
    if (!host[f]) return THOR_EINVAL;
  size_t off = 0;
  if (side) {
    // the side stream must not overwrite staging before the state's stream is done with it
    if (cudaEventRecord(ev_x[0], stream) || cudaStreamWaitEvent(side, ev_x[0], 0)) return THOR_ECUDA;
  }
  for (int f = 0; f < 4; ++f) {
    const int rc = set_async(f, host[f], staging + off, side);
    if (rc) return rc;
    off += field_count(f, G.ncol, G.nv);
  }
  return cudaStreamSynchronize(stream) == cudaSuccess ? THOR_OK : THOR_ECUDA;
}

template <typename R>
int Impl<R>::get_all(double* const host[4]) {
  for (int f = 0; f < 4; ++f)
    if (!host[f]) return THOR_EINVAL;
  size_t off = 0;
  for (int f = 0; f < 4; ++f) {
    const size_t n = field_count(f, G.ncol, G.nv);
    dim3 grid((G.ncol + 127) / 128, f == THOR_FIELD_W ? G.nv + 1 : G.nv);
    k_to_canonical<R><<<grid, 128, 0, stream>>>(staging + off, G, V, ph, Xt, XtL, f);
    ++launches;
    cudaStream_t cs = stream;
    if (side) {
      if (cudaEventRecord(ev_x[f], stream) || cudaStreamWaitEvent(side, ev_x[f], 0)) return THOR_ECUDA;
      cs = side;
    }
    if (cudaMemcpyAsync(host[f], staging + off, n * sizeof(double), cudaMemcpyDeviceToHost, cs)) return THOR_ECUDA;
    off += n;
  }
  if (side && cudaStreamSynchronize(side)) return THOR_ECUDA;
  return cudaStreamSynchronize(stream) == cudaSuccess ? THOR_OK : THOR_ECUDA;
}

// copy (on cs, the state's stream by default) and convert (on the state's
// stream, after the copy) one field
template <typename R>
int Impl<R>::set_async(int field, const double* host, double* buf, cudaStream_t cs) {
  const int nv = G.nv;
  int nlev = nv, ncomp = 1, zero_ends = 0;
  const double* ref = nullptr;
  R *d0 = nullptr, *d1 = nullptr, *d2 = nullptr, *l0 = nullptr, *l1 = nullptr, *l2 = nullptr;
  switch (field) {
    case THOR_FIELD_RHO: ref = V.rhob; d0 = Xt.rho; l0 = XtL.rho; break;
    case THOR_FIELD_MOM:
      ncomp = 3; d0 = Xt.mx; d1 = Xt.my; d2 = Xt.mz; l0 = XtL.mx; l1 = XtL.my; l2 = XtL.mz;
      break;
    case THOR_FIELD_W: nlev = nv + 1; zero_ends = 1; d0 = Xt.w; l0 = XtL.w; break;
    case THOR_FIELD_RHOTHETA: ref = V.thb; d0 = Xt.th; l0 = XtL.th; break;
    default: return THOR_EINVAL;
  }
  const size_t n = (size_t)G.ncol * nlev * ncomp;
  if (!cs) cs = stream;
  if (cudaMemcpyAsync(buf, host, n * sizeof(double), cudaMemcpyHostToDevice, cs)) return THOR_ECUDA;
  if (cs != stream) {
    if (cudaEventRecord(ev_x[field], cs) || cudaStreamWaitEvent(stream, ev_x[field], 0)) return THOR_ECUDA;
  }
  dim3 grid((G.ncol + 127) / 128, nlev);
  k_from_canonical<R><<<grid, 128, 0, stream>>>(buf, G.ncol, G.colp, nlev, ncomp, ref, d0, d1, d2, l0, l1, l2,
                                                zero_ends);
  ++launches;
  return cudaGetLastError() == cudaSuccess ? THOR_OK : THOR_ECUDA;
}

template <typename R>
int Impl<R>::diag(double* out8, long long* nonfinite) {
  k_diag_partial<R><<<kDiagBlocks, kDiagThreads, 0, stream>>>(G, V, ph, Xt, XtL, red);
  k_diag_final<<<1, 256, 0, stream>>>(red, kDiagBlocks);
  launches += 2;
  double h[8];
  int flag = 0;
  if (cudaMemcpyAsync(h, red + kDiagBlocks * 8, sizeof(h), cudaMemcpyDeviceToHost, stream)) return THOR_ECUDA;
  if (cudaMemcpyAsync(&flag, dev_err, sizeof(int), cudaMemcpyDeviceToHost, stream)) return THOR_ECUDA;
  if (cudaStreamSynchronize(stream)) return THOR_ECUDA;
  if (flag) return THOR_ETIMEOUT;
  for (int j = 0; j < 8; ++j) out8[j] = h[j];
  *nonfinite = (long long)h[7];
  return THOR_OK;
}

// the low parts of a compensated float X^t: on allocates them zeroed (the
// state's value is unchanged), off frees them (the value rounds to the float
// parts); float64 states need none
template <typename R>
int Impl<R>::set_compensated(int on) {
  if (sizeof(R) == sizeof(double) || ph.anelastic) return on ? THOR_EINVAL : THOR_OK;
  if ((on != 0) == (compensated != 0)) return THOR_OK;
  if (cudaStreamSynchronize(stream)) return THOR_ECUDA;
  drop_graph();
  if (!on) {
    cudaFree(lo_buf);
    lo_buf = nullptr;
    XtL = Xf<R>{};
    compensated = 0;
    return THOR_OK;
  }
  const size_t S = G.colp, C = S * G.nv, F = S * (G.nv + 1);
  const size_t per = 5 * C + F;                 // rho, M (3), rho theta, W
  if (cudaMalloc(&lo_buf, per * sizeof(R))) {
    lo_buf = nullptr;
    return THOR_ENOMEM;
  }
  if (cudaMemsetAsync(lo_buf, 0, per * sizeof(R), stream) || cudaStreamSynchronize(stream)) {
    cudaFree(lo_buf);
    lo_buf = nullptr;
    return THOR_ECUDA;
  }
  R* b = static_cast<R*>(lo_buf);
  auto lay = [&](Xf<R>& x, R* p) {
    x.rho = p; x.mx = p + C; x.my = p + 2 * C; x.mz = p + 3 * C; x.th = p + 4 * C; x.w = p + 5 * C;
  };
  lay(XtL, b);
  compensated = 1;
  return THOR_OK;
}

template Impl<double>::~Impl();
template Impl<float>::~Impl();
template int Impl<double>::get(int, double*, size_t);
template int Impl<float>::get(int, double*, size_t);
template int Impl<double>::set(int, const double*, size_t);
template int Impl<float>::set(int, const double*, size_t);
template int Impl<double>::diag(double*, long long*);
template int Impl<double>::set_compensated(int);
template int Impl<float>::set_compensated(int);
template int Impl<float>::diag(double*, long long*);

namespace {


// Sec. 2.1 with k + 1 nodes (reading L-1): the k + 1 consecutive nodes
// nearest the target, from target - ceil((k + 1) / 2) up, shifted inward at
// the ends; `target` is the first of the n nodes above the target altitude.
// L_j(zh) = prod_{i != j} (zh - z_i) / (z_j - z_i).
static void lagrange_row(const std::vector<double>& nodes, double zh, int target, int k, int& j0, double w[4]) {
  const int n = (int)nodes.size();
  j0 = std::min(std::max(target - (k + 2) / 2, 0), n - k - 1);
  for (int j = 0; j < 4; ++j) w[j] = 0.0;
  for (int j = 0; j <= k; ++j) {
    double l = 1.0;
    for (int i = 0; i <= k; ++i)
      if (i != j) l *= (zh - nodes[j0 + i]) / (nodes[j0 + j] - nodes[j0 + i]);
    w[j] = l;
  }
}

// The start column of Sec. 6.1's Held-Suarez run: every layer at the
// equatorial T_eq of its own pressure, max(200, (315 - 10 ln(p/p0)) (p/p0)^kappa)
// with p0 = 1e5 Pa, in the discrete hydrostatic balance of the reference
// column below. Layer by layer from the ground, T_k is the fixed point of
// T -> T_eq(p_k(T)), p_k(T) the balanced pressure over layer k-1; returns
// false when a layer does not settle to 1e-12 K.
static bool held_suarez_column(const std::vector<double>& zc, const std::vector<double>& dzc,
                               const std::vector<double>& wlo, const std::vector<double>& whi, double p_surf,
                               double g, double Rd, double kappa, std::vector<double>& T, std::vector<double>& p) {
  const int nv = (int)zc.size();
  auto teq = [&](double pp) {
    const double s = pp / 1.0e5;
    return std::fmax(200.0, (315.0 - 10.0 * std::log(s)) * std::pow(s, kappa));
  };
  auto balanced = [&](int k, double Tk) {
    if (k == 0) return p_surf * std::exp(-g * zc[0] / (Rd * Tk));
    return p[k - 1] * (1.0 - g * dzc[k] * wlo[k] / (Rd * T[k - 1])) / (1.0 + g * dzc[k] * whi[k] / (Rd * Tk));
  };
  for (int k = 0; k < nv; ++k) {
    double t = k == 0 ? 315.0 : T[k - 1];
    bool settled = false;
    for (int it = 0; it < 1000 && !settled; ++it) {
      const double tn = teq(balanced(k, t));
      settled = std::fabs(tn - t) <= 1e-12;
      t = tn;
    }
    if (!settled) return false;
    T[k] = t;
    p[k] = balanced(k, t);
  }
  return true;
}

int host_setup(const HostGrid& h, const thor_planet& pl, const thor_init& in, HostSetup& hs) {
  const int nv = h.nv, ncol = h.ncol;
  std::vector<double> zi(nv + 1), zc(nv);
  const double step = h.z_top / nv;
  for (int i = 0; i < nv; ++i) zi[i] = i * step;
  zi[nv] = h.z_top;
  for (int k = 0; k < nv; ++k) zc[k] = 0.5 * (zi[k] + zi[k + 1]);
  {
    const int k = in.vorder > 1 ? in.vorder : 1;
    hs.iw.assign(4 * (size_t)(nv + 1), 0.0);
    hs.cw.assign(4 * (size_t)nv, 0.0);
    hs.ij0.assign(nv + 1, 0);
    hs.cj0.assign(nv, 0);
    double w[4];
    for (int m = 1; m < nv; ++m) {
      lagrange_row(zc, zi[m], m, k, hs.ij0[m], w);
      for (int j = 0; j < 4; ++j) hs.iw[(size_t)j * (nv + 1) + m] = w[j];
    }
    for (int c = 0; c < nv; ++c) {
      lagrange_row(zi, zc[c], c + 1, k, hs.cj0[c], w);
      for (int j = 0; j < 4; ++j) hs.cw[(size_t)j * nv + c] = w[j];
    }
  }
  auto& rc = hs.vert[0]; auto& dz = hs.vert[1]; auto& clo = hs.vert[2]; auto& chi = hs.vert[3];
  auto& zcv = hs.vert[4]; auto& rhob = hs.vert[5]; auto& thb = hs.vert[6]; auto& pb = hs.vert[7];
  auto& Tb = hs.vert[8]; auto& sv = hs.vert[9]; auto& sq_lo = hs.vert[10]; auto& sq_hi = hs.vert[11];
  auto& ri = hs.vert[12]; auto& dzc = hs.vert[13]; auto& wlo = hs.vert[14]; auto& whi = hs.vert[15];
  auto& Rb = hs.vert[16]; auto& ri2 = hs.vert[17]; auto& inv_dzc = hs.vert[18];
  for (int j = 0; j < kNumVertCentre; ++j) hs.vert[j].assign(nv, 0.0);
  for (int j = kNumVertCentre; j < kNumVert; ++j) hs.vert[j].assign(nv + 1, 0.0);
  const double deep = in.shallow ? 0.0 : 1.0;   // shallow atmosphere: r = radius everywhere
  for (int k = 0; k < nv; ++k) {
    rc[k] = h.radius + deep * zc[k];
    dz[k] = zi[k + 1] - zi[k];
    clo[k] = (zc[k] - zi[k + 1]) / (zi[k] - zi[k + 1]);
    chi[k] = (zc[k] - zi[k]) / (zi[k + 1] - zi[k]);
    zcv[k] = zc[k];
  }
  for (int i = 0; i <= nv; ++i) {
    ri[i] = h.radius + deep * zi[i];
    ri2[i] = ri[i] * ri[i];
  }
  for (int k = 0; k < nv; ++k) {
    sv[k] = 1.0 / (rc[k] * rc[k] * dz[k]);
    sq_lo[k] = ri2[k] * sv[k];
    sq_hi[k] = ri2[k + 1] * sv[k];
  }
  for (int i = 1; i < nv; ++i) {
    dzc[i] = zc[i] - zc[i - 1];
    inv_dzc[i] = 1.0 / dzc[i];
    wlo[i] = (zi[i] - zc[i]) / (zc[i - 1] - zc[i]);
    whi[i] = (zi[i] - zc[i - 1]) / (zc[i] - zc[i - 1]);
  }
  const double g = pl.gravity, Rd = pl.Rd;
  const double gamma = pl.cp / (pl.cp - Rd);
  // discretely balanced reference column, isothermal at T0 or the
  // Held-Suarez start: (p_i - p_i-1)/dzc + g (wlo rho_i-1 + whi rho_i) = 0
  // with rho = p/(Rd T)
  std::vector<double> Tcol(nv, in.T0);
  if (in.profile == THOR_PROFILE_HELD_SUAREZ) {
    if (!held_suarez_column(zc, dzc, wlo, whi, in.p_surf, g, Rd, Rd / pl.cp, Tcol, pb)) return THOR_ENOTCONV;
  } else {
    pb[0] = in.p_surf * std::exp(-g * zc[0] / (Rd * in.T0));
    for (int i = 1; i < nv; ++i)
      pb[i] = pb[i - 1] * (1.0 - g * dzc[i] * wlo[i] / (Rd * in.T0)) / (1.0 + g * dzc[i] * whi[i] / (Rd * in.T0));
  }
  for (int k = 0; k < nv; ++k) {
    rhob[k] = pb[k] / (Rd * Tcol[k]);
    thb[k] = pl.p_ref / Rd * std::pow(pb[k] / pl.p_ref, 1.0 / gamma);
    Tb[k] = pb[k] / (rhob[k] * Rd);
  }
  for (int i = 1; i < nv; ++i)
    Rb[i] = -(pb[i] - pb[i - 1]) / dzc[i] - g * (wlo[i] * rhob[i - 1] + whi[i] * rhob[i]);
  hs.rho.assign((size_t)ncol * nv, 0.0);
  hs.th.assign((size_t)ncol * nv, 0.0);
  for (int c = 0; c < ncol; ++c)
    for (int k = 0; k < nv; ++k) {
      double T = Tcol[k];
      if (in.noise_amp > 0.0) {
        uint64_t z = splitmix64(in.seed ^ ((uint64_t)c * (uint64_t)nv + (uint64_t)k));
        double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
        T = Tcol[k] + in.noise_amp * (2.0 * u - 1.0);
      }
      if (in.anelastic) {
        // anelastic start: rho stays the reference column; the temperature
        // perturbation at fixed pressure is a theta' = theta0 dT / T
        hs.rho[(size_t)c * nv + k] = rhob[k];
        hs.th[(size_t)c * nv + k] = thb[k] * (1.0 + (T - Tcol[k]) / Tcol[k]);
      } else {
        hs.rho[(size_t)c * nv + k] = pb[k] / (Rd * T);
        hs.th[(size_t)c * nv + k] = thb[k];
      }
    }
  return THOR_OK;
}

template <typename R>
int make_impl(thor_grid* grid, const thor_planet& pl, const thor_init& in, cudaStream_t st,
              std::unique_ptr<ImplBase>& out) {
  const HostGrid& h = grid->h;
  auto I = std::make_unique<Impl<R>>();
  I->stream = st;
  I->G.ncol = h.ncol;
  I->G.colp = colp_of(h.ncol);
  I->G.nv = h.nv;
  I->ph.Rd = pl.Rd;
  I->ph.cp = pl.cp;
  I->ph.cv = pl.cp - pl.Rd;
  I->ph.gamma = pl.cp / (pl.cp - pl.Rd);
  I->ph.kappa = pl.Rd / pl.cp;
  I->ph.g = pl.gravity;
  I->ph.omega = pl.omega;
  I->ph.p_ref = pl.p_ref;
  I->ph.inv_Rd = 1.0 / I->ph.Rd;
  I->ph.inv_gamma = 1.0 / I->ph.gamma;
  I->ph.two_omega = 2.0 * I->ph.omega;
  I->ph.Rd_f = (float)I->ph.Rd;
  I->ph.inv_Rd_f = (float)I->ph.inv_Rd;
  I->ph.gamma_f = (float)I->ph.gamma;
  I->ph.inv_gamma_f = (float)I->ph.inv_gamma;
  I->ph.kappa_f = (float)I->ph.kappa;
  I->ph.g_f = (float)I->ph.g;
  I->ph.two_omega_f = (float)I->ph.two_omega;
  I->ph.hydrostatic = in.hydrostatic ? 1 : 0;
  I->ph.vorder = in.vorder > 1 ? in.vorder : 1;
  I->ph.anelastic = in.anelastic ? 1 : 0;
  I->ph.delta = in.hydrostatic ? 0.0 : 1.0;
  I->ph.delta_f = (float)I->ph.delta;
  I->hyper = in.hyperdiffusion ? 1 : 0;
  I->divdamp = in.divergence_damping ? 1 : 0;
  I->shallow = in.shallow ? 1 : 0;
  I->forcing = in.forcing;
  I->hj_dT = in.hj_dT;
  I->diff_D = pl.diff_D;
  double dbar = std::sqrt(2.0 * M_PI / 5.0) * pl.radius / std::pow(2.0, h.glevel);
  I->dbar4 = dbar * dbar * dbar * dbar;
  Carver dry{nullptr};
  carve(dry, *I, h.ncol, h.nv);
  void* arena = nullptr;
  if (cudaMalloc(&arena, dry.off) != cudaSuccess) return THOR_ENOMEM;
  if (cudaMemsetAsync(arena, 0, dry.off, st) != cudaSuccess) {
    cudaFree(arena);
    return THOR_ECUDA;
  }
  I->arena = arena;
  Carver real{static_cast<char*>(arena)};
  carve(real, *I, h.ncol, h.nv);
  if (col_kernel_setup<R>(h.nv)) return THOR_ECUDA;
  if (I->build_solve_maps()) return THOR_ECUDA;
  // side stream for the stage kernels that run beside others (optional:
  // without it everything runs on the state's stream)
  if (cudaStreamCreateWithFlags(&I->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&I->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&I->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&I->ev_join0, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&I->ev_x[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&I->ev_x[1], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&I->ev_x[2], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&I->ev_x[3], cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (I->side) cudaStreamDestroy(I->side);
    I->side = nullptr;
  }
  // third stream for the upper levels of the small steps' stencils
  // (THOR_TUNE_LEVEL_SPLIT; optional as well)
  if (cudaStreamCreateWithFlags(&I->side2, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&I->ev_s1, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&I->ev_s2, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (I->side2) cudaStreamDestroy(I->side2);
    I->side2 = nullptr;
  }
  HostSetup hs;
  int rc = host_setup(h, pl, in, hs);
  if (rc) return rc;
  {
    unsigned long long x = 1469598103934665603ull;           // FNV-1a, 64 bit
    auto mix = [&x](const void* p, size_t n) {
      const unsigned char* b = static_cast<const unsigned char*>(p);
      for (size_t i = 0; i < n; ++i) x = (x ^ b[i]) * 1099511628211ull;
    };
    for (int v = 0; v < kNumVert; ++v) mix(hs.vert[v].data(), hs.vert[v].size() * sizeof(double));
    const double pv[7] = {pl.radius, pl.omega, pl.gravity, pl.Rd, pl.cp, pl.p_ref, pl.diff_D};
    mix(pv, sizeof(pv));
    const int sw[5] = {in.shallow, in.hydrostatic, in.forcing, in.vorder > 1 ? in.vorder : 1, in.anelastic ? 1 : 0};
    mix(sw, sizeof(sw));
    I->ref_hash = x;
  }
  rc = upload_tables(*I, h, hs.vert, &hs, st);
  if (rc) return rc;
  if (in.anelastic) {
    rc = anelastic_setup(*I, anelastic_hdiag(h));
    if (rc) return rc;
  }
  rc = I->set(THOR_FIELD_RHO, hs.rho.data(), hs.rho.size());
  if (rc) return rc;
  rc = I->set(THOR_FIELD_RHOTHETA, hs.th.data(), hs.th.size());
  if (rc) return rc;
  out = std::move(I);
  return THOR_OK;
}

}  // namespace
}  // namespace thor

// ====================================================================== ABI

extern "C" {

const char* thor_strerror(int s) {
  switch (s) {
    case THOR_OK: return "ok";
    case THOR_EINVAL: return "invalid argument";
    case THOR_ENOMEM: return "out of memory";
    case THOR_ECUDA: return "CUDA runtime error";
    case THOR_ENONFINITE: return "non-finite state";
    case THOR_ETIMEOUT: return "device wait timed out";
    case THOR_ENOTCONV: return "not converged";
    default: return "unknown status";
  }
}

int thor_grid_create(int glevel, int nv, double radius, double z_top, const thor_spring* spring,
                     thor_grid** out) {
  if (!out || glevel < 0 || glevel > 10 || nv < 2 || nv > 256 || !(radius > 0) || !(z_top > 0))
    return THOR_EINVAL;
  thor::SpringParams sp;
  if (spring) {
    if (!(spring->dt > 0) || spring->max_iter < 0) return THOR_EINVAL;
    sp.beta = spring->beta;
    sp.alpha = spring->alpha;
    sp.k = spring->k;
    sp.dt = spring->dt;
    sp.tol = spring->tol;
    sp.max_iter = spring->max_iter;
  }
  thor_grid* g = new (std::nothrow) thor_grid;
  if (!g) return THOR_ENOMEM;
  int rc = thor::build_grid(glevel, nv, radius, z_top, sp, true, g->h);
  if (rc) {
    delete g;
    return rc;
  }
  *out = g;
  return THOR_OK;
}

int thor_grid_info(const thor_grid* g, int* ncol, int* nv, int* npent, int* iters, int* conv) {
  if (!g) return THOR_EINVAL;
  if (ncol) *ncol = g->h.ncol;
  if (nv) *nv = g->h.nv;
  if (npent) {
    int c = 0;
    for (int x : g->h.nn) c += x == 5;
    *npent = c;
  }
  if (iters) *iters = g->h.spring_iters;
  if (conv) *conv = g->h.spring_converged;
  return THOR_OK;
}

int thor_grid_points(const thor_grid* g, double* xyz, size_t n) {
  if (!g || !xyz || n != (size_t)3 * g->h.ncol) return THOR_EINVAL;
  std::memcpy(xyz, g->h.P.data(), n * sizeof(double));
  return THOR_OK;
}

int thor_grid_neighbours(const thor_grid* g, int* nbr, size_t n) {
  if (!g || !nbr || n != (size_t)6 * g->h.ncol) return THOR_EINVAL;
  std::memcpy(nbr, g->h.nbr.data(), n * sizeof(int));
  return THOR_OK;
}

int thor_grid_areas(const thor_grid* g, double* area, size_t n) {
  if (!g || !area || n != (size_t)g->h.ncol) return THOR_EINVAL;
  std::memcpy(area, g->h.area.data(), n * sizeof(double));
  return THOR_OK;
}

int thor_grid_coarse_map(const thor_grid* fine, const thor_grid* coarse, int* map, size_t n) {
  if (!fine || !coarse || !map || n != (size_t)fine->h.ncol) return THOR_EINVAL;
  const std::vector<double>& F = fine->h.P;
  const std::vector<double>& C = coarse->h.P;
  const std::vector<int>& nb = coarse->h.nbr;
  const int nc = coarse->h.ncol;
  auto dot = [&](int i, int c) { return F[3 * i] * C[3 * c] + F[3 * i + 1] * C[3 * c + 1] + F[3 * i + 2] * C[3 * c + 2]; };
  // greedy ascent of the dot product over the neighbour graph
  auto walk = [&](int i, int c) {
    double best = dot(i, c);
    for (int it = 0; it < nc; ++it) {
      int next = -1;
      for (int k = 0; k < 6; ++k) {
        const int q = nb[6 * c + k];
        if (q < 0) continue;
        const double d = dot(i, q);
        if (d > best) {
          best = d;
          next = q;
        }
      }
      if (next < 0) break;
      c = next;
    }
    return c;
  };
  // no point of the second ring beats c (the walk's end is the global
  // nearest centre unless the grid is badly distorted)
  auto local_ok = [&](int i, int c) {
    const double d0 = dot(i, c);
    for (int k = 0; k < 6; ++k) {
      const int q = nb[6 * c + k];
      if (q < 0) continue;
      for (int l = 0; l < 6; ++l) {
        const int r = nb[6 * q + l];
        if (r >= 0 && dot(i, r) > d0) return false;
      }
    }
    return true;
  };
  int c = 0;
  for (int i = 0; i < (int)n; ++i) {
    c = walk(i, c);
    if (!local_ok(i, c)) {
      int bc = 0;
      for (int q = 1; q < nc; ++q)
        if (dot(i, q) > dot(i, bc)) bc = q;
      c = bc;
    }
    map[i] = c;
  }
  return THOR_OK;
}

void thor_grid_destroy(thor_grid* g) { delete g; }

int thor_state_init(thor_grid* grid, const thor_planet* pl, const thor_init* in, void* stream,
                    thor_state** out) {
  if (!grid || !pl || !in || !out) return THOR_EINVAL;
  if (!(pl->radius > 0) || std::fabs(pl->radius - grid->h.radius) > 1e-9 * grid->h.radius ||
      !(pl->Rd > 0) || !(pl->cp > pl->Rd) || !(pl->gravity > 0) || !(pl->p_ref > 0) || !(pl->diff_D >= 0) ||
      !(in->T0 > 0 || in->profile == THOR_PROFILE_HELD_SUAREZ) || !(in->p_surf > 0) || !(in->noise_amp >= 0) ||
      in->profile < THOR_PROFILE_ISOTHERMAL || in->profile > THOR_PROFILE_HELD_SUAREZ || in->forcing < 0 ||
      in->vorder < 0 || in->vorder > 3 || grid->h.nv < (in->vorder > 1 ? in->vorder : 1) + 1 ||
      (in->anelastic && in->hydrostatic) ||
      in->forcing > 2 ||
      (in->precision != THOR_FP64 && in->precision != THOR_MIXED) || grid->h.nv > thor::kMaxNv)
    return THOR_EINVAL;
  thor_state* s = new (std::nothrow) thor_state;
  if (!s) return THOR_ENOMEM;
  s->grid = grid;
  s->precision = in->precision;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = in->precision == THOR_FP64 ? thor::make_impl<double>(grid, *pl, *in, st, s->impl)
                                      : thor::make_impl<float>(grid, *pl, *in, st, s->impl);
  // mixed states keep X^t as compensated float pairs unless switched off
  if (!rc && in->precision == THOR_MIXED && !in->anelastic) rc = s->impl->set_compensated(1);
  if (rc) {
    delete s;
    return rc;
  }
  *out = s;
  return THOR_OK;
}

int thor_step(thor_state* s, int n_large, int n_small, double dt) {
  if (!s || n_large < 0 || n_small < 2 || (n_small % 2) || !(dt > 0)) return THOR_EINVAL;
  int rc = THOR_OK;
  if (s->closure.net) {
    for (int i = 0; i < n_large && !rc; ++i) rc = thor::closure_large_step(s, n_small, dt);
  } else {
    rc = s->impl->step(n_large, n_small, dt);
  }
  if (rc || !s->check_finite) return rc;
  double v[8];
  long long nf = 0;
  rc = s->impl->diag(v, &nf);
  if (rc) return rc;
  return nf ? THOR_ENONFINITE : THOR_OK;
}

namespace {
// header of a raw checkpoint
struct CkptHeader {
  char magic[8];
  int precision, ncol, nv, colp;
  unsigned long long payload;
  unsigned long long ref_hash;    // the saving state's reference (ImplBase::ref_hash)
  long long closure_steps;        // large steps since its closure was attached
  char pad[16];
};
static_assert(sizeof(CkptHeader) == 64, "checkpoint header is 64 bytes");
const char kCkptMagic[8] = {'T', 'H', 'O', 'R', 'C', 'K', 'P', '2'};
}  // namespace

int thor_wait_selftest(int arrive, unsigned int limit_us, int* gave_up) {
  if (!gave_up || limit_us < 1 || limit_us > 2000000) return THOR_EINVAL;
  int* d = nullptr;
  if (cudaMalloc(&d, sizeof(int))) return THOR_ENOMEM;
  int h = -1;
  thor::k_wait_probe<<<1, 32>>>(arrive ? 1 : 0, 1000ull * limit_us, d);
  cudaError_t e = cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e) return THOR_ECUDA;
  *gave_up = h;
  return THOR_OK;
}

int thor_checkpoint_bytes(const thor_state* s, size_t* bytes) {
  if (!s || !bytes) return THOR_EINVAL;
  *bytes = sizeof(CkptHeader) + s->impl->state_bytes();
  return THOR_OK;
}

int thor_checkpoint_save(thor_state* s, void* buf, size_t bytes) {
  if (!s || !buf) return THOR_EINVAL;
  const size_t payload = s->impl->state_bytes();
  if (bytes != sizeof(CkptHeader) + payload) return THOR_EINVAL;
  CkptHeader h{};
  std::memcpy(h.magic, kCkptMagic, 8);
  h.precision = s->precision;
  h.ncol = s->grid->h.ncol;
  h.nv = s->grid->h.nv;
  h.colp = thor::colp_of(h.ncol);
  h.payload = payload;
  h.ref_hash = s->impl->ref_hash;
  h.closure_steps = s->closure.counter;
  char* p = static_cast<char*>(buf);
  if (cudaMemcpy(p, &h, sizeof(h), cudaMemcpyDefault)) return THOR_ECUDA;
  if (s->impl->save_state(p + sizeof(h))) return THOR_ECUDA;
  return cudaStreamSynchronize(s->impl->stream) ? THOR_ECUDA : THOR_OK;
}

int thor_checkpoint_load(thor_state* s, const void* buf, size_t bytes) {
  if (!s || !buf) return THOR_EINVAL;
  const size_t payload = s->impl->state_bytes();
  if (bytes != sizeof(CkptHeader) + payload) return THOR_EINVAL;
  CkptHeader h{};
  if (cudaMemcpy(&h, buf, sizeof(h), cudaMemcpyDefault)) return THOR_ECUDA;
  if (std::memcmp(h.magic, kCkptMagic, 8) || h.precision != s->precision || h.ncol != s->grid->h.ncol ||
      h.nv != s->grid->h.nv || h.payload != payload || h.ref_hash != s->impl->ref_hash || h.closure_steps < 0)
    return THOR_EINVAL;
  if (s->impl->load_state(static_cast<const char*>(buf) + sizeof(h))) return THOR_ECUDA;
  s->closure.counter = h.closure_steps;        // resume inside the same closure window
  return cudaStreamSynchronize(s->impl->stream) ? THOR_ECUDA : THOR_OK;
}

int thor_diag(thor_state* s, thor_diag_t* out) {
  if (!s || !out) return THOR_EINVAL;
  double v[8];
  long long nf = 0;
  int rc = s->impl->diag(v, &nf);
  if (rc) return rc;
  out->mass = v[0];
  out->energy = v[1];
  out->aam = v[2];
  out->mean_T = v[3] / v[4];
  out->max_vh = v[5];
  out->max_w = v[6];
  out->nonfinite = nf;
  return THOR_OK;
}

int thor_state_get(thor_state* s, int field, double* host, size_t n) {
  if (!s) return THOR_EINVAL;
  return s->impl->get(field, host, n);
}

int thor_state_set(thor_state* s, int field, const double* host, size_t n) {
  if (!s) return THOR_EINVAL;
  return s->impl->set(field, host, n);
}

int thor_state_get_all(thor_state* s, double* rho, double* mom, double* w, double* rhotheta, int ncol, int nv) {
  if (!s || ncol != s->grid->h.ncol || nv != s->grid->h.nv) return THOR_EINVAL;
  double* const host[4] = {rho, mom, w, rhotheta};
  return s->impl->get_all(host);
}

int thor_state_set_all(thor_state* s, const double* rho, const double* mom, const double* w, const double* rhotheta,
                       int ncol, int nv) {
  if (!s || ncol != s->grid->h.ncol || nv != s->grid->h.nv) return THOR_EINVAL;
  const double* const host[4] = {rho, mom, w, rhotheta};
  return s->impl->set_all(host);
}

int thor_launch_count(const thor_state* s, long long* count) {
  if (!s || !count) return THOR_EINVAL;
  *count = s->impl->launches;
  return THOR_OK;
}

int thor_tune(thor_state* s, int knob, int value) {
  if (!s) return THOR_EINVAL;
  if (knob == THOR_TUNE_KCHUNK) {
    if (value < 1 || value > 256) return THOR_EINVAL;
    s->impl->kchunk = value;
    return THOR_OK;
  }
  if (knob == THOR_TUNE_GRAPH) {
    s->impl->set_graph(value != 0);
    return THOR_OK;
  }
  if (knob == THOR_TUNE_CHECK_FINITE) {
    s->check_finite = value != 0;
    return THOR_OK;
  }
  if (knob == THOR_TUNE_BLOCK) {
    if (value < 32 || value > thor::kMaxBlock || value % 32) return THOR_EINVAL;
    s->impl->block = value;
    return THOR_OK;
  }
  if (knob == THOR_TUNE_SOLVE_TMA) {
    s->impl->solve_tma = value != 0;
    return THOR_OK;
  }
  if (knob == THOR_TUNE_COMPENSATED) return s->impl->set_compensated(value != 0);
  if (knob == THOR_TUNE_LEVEL_SPLIT) {
    s->impl->level_split = value != 0;
    s->impl->reset_graph();
    return THOR_OK;
  }
  if (knob == THOR_TUNE_L2_HINTS) {
    if (value < 0 || value > 3) return THOR_EINVAL;
    return thor::set_l2_mode(value) ? THOR_ECUDA : THOR_OK;
  }
  if (knob == THOR_TUNE_RK_STAGES) {
    if (value < 1 || value > 3) return THOR_EINVAL;
    s->impl->rk_stages = value;
    s->impl->reset_graph();
    return THOR_OK;
  }
  if (knob == THOR_TUNE_ENERGY_FIXER || knob == THOR_TUNE_BUDGET) {
    thor::ImplBase* I = s->impl.get();
    if (knob == THOR_TUNE_BUDGET && (value < 0 || value > (1 << 24))) return THOR_EINVAL;
    if (cudaStreamSynchronize(I->stream)) return THOR_ECUDA;   // no step still uses the buffers
    if (!I->fixbuf && value && cudaMalloc(&I->fixbuf, thor::kFixBufBytes)) return THOR_ENOMEM;
    if (knob == THOR_TUNE_ENERGY_FIXER) {
      I->energy_fix = value != 0;
    } else {
      if (I->budget) cudaFree(I->budget);
      I->budget = nullptr;
      I->budget_cap = 0;
      if (value) {
        if (!I->budget_count && cudaMalloc(&I->budget_count, sizeof(int))) return THOR_ENOMEM;
        if (cudaMalloc(&I->budget, (size_t)value * 8 * sizeof(double))) return THOR_ENOMEM;
        if (cudaMemset(I->budget_count, 0, sizeof(int))) return THOR_ECUDA;
        I->budget_cap = value;
      }
    }
    I->reset_graph();
    return THOR_OK;
  }
  return THOR_EINVAL;
}

int thor_budget_read(thor_state* s, double* out, int max_rows, int* n_rows) {
  if (!s || !n_rows || max_rows < 0 || (max_rows > 0 && !out)) return THOR_EINVAL;
  thor::ImplBase* I = s->impl.get();
  *n_rows = 0;
  if (!I->budget_cap) return THOR_OK;
  int n = 0;
  if (cudaMemcpyAsync(&n, I->budget_count, sizeof(int), cudaMemcpyDeviceToHost, I->stream) ||
      cudaStreamSynchronize(I->stream))
    return THOR_ECUDA;
  n = std::min(n, max_rows);
  if (n > 0 && cudaMemcpy(out, I->budget, (size_t)n * 8 * sizeof(double), cudaMemcpyDeviceToHost))
    return THOR_ECUDA;
  *n_rows = n;
  return THOR_OK;
}

int thor_profile(thor_state* s, int enable) {
  if (!s) return THOR_EINVAL;
  s->impl->prof_used = 0;
  s->impl->prof_on = enable != 0;
  return THOR_OK;
}

int thor_profile_read(thor_state* s, int kernel, double* total_ms, long long* launches) {
  if (!s || !total_ms || !launches || kernel < 0 || kernel >= THOR_K_COUNT) return THOR_EINVAL;
  return s->impl->prof_read(kernel, total_ms, launches) ? THOR_ECUDA : THOR_OK;
}

void thor_state_destroy(thor_state* s) {
  if (!s) return;
  thor::closure_release(s);
  if (s->impl) cudaStreamSynchronize(s->impl->stream);
  thor::zonal_release(s->zonal);
  delete s;
}

}  // extern "C"
