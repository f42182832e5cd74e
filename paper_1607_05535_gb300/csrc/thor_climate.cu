// Zonal band means of a state on the GPU (Sec. 6.1: the Held-Suarez and
// hot-Jupiter climates are judged by zonal and time averages of the wind and
// temperature, the mass stream function and the eddy fluxes [u'v'], [v'T']).
//
// A zonal mean on the icosahedral grid is the volume-weighted mean over the
// cells of one level whose latitude falls in one of nlat equal bands (band
// b = floor((lat + pi/2 + 1e-9) / pi * nlat), the north pole in the last
// band).
// thor_zonal_accumulate reduces the current state to per-(level, band) sums
// of V, V u, V v, V T, V p, V uv, V vT, V uu, V vv (float64, shared-memory
// band histograms per block, then global atomics), turns them into the
// band means and covariances of that state and adds them to the state's
// time accumulator; thor_zonal_read returns the accumulated sums. At the two
// polar cells east and north are undefined and u = v = 0. The same pass adds
// every cell's vertical velocity at its centre, w = (W interpolated to the
// centre) / rho, to a per-cell time sum: the time mean [w] behind the
// grid-imprinting map [w*] of Sec. 6.1 (thor_zonal_read_w).
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/thor.h"
#include "thor_state.h"

namespace thor {
namespace {

constexpr int kZonalThreads = 256;
constexpr int kZonalQ = 9;    // weight, u, v, T, p, uv, vT, uu, vv

template <typename R>
__global__ void __launch_bounds__(kZonalThreads)
    k_zonal_partial(Geo<R> G, Vert V, Phys ph, Xf<R> X, Xf<R> XL, const int* __restrict__ band,
                    const double* __restrict__ basis, int nlat, double* __restrict__ tmp,
                    double* __restrict__ wsum) {
  extern __shared__ double hist[];                 // [nlat][kZonalQ]
  const int k = blockIdx.y, S = G.colp;
  for (int t = threadIdx.x; t < nlat * kZonalQ; t += blockDim.x) hist[t] = 0.0;
  __syncthreads();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < G.ncol) {
    const size_t i = (size_t)k * S + c;
    // the full value of a field: a compensated state adds its low part XL
    auto val = [&](const R* hi, const R* lo, size_t j) { return lo ? (double)hi[j] + (double)lo[j] : (double)hi[j]; };
    const double rho = V.rhob[k] + val(X.rho, XL.rho, i);
    const double p = V.pb[k] + V.pb[k] * expm1(ph.gamma * log1p(val(X.th, XL.th, i) / V.thb[k]));
    const double T = p / (rho * ph.Rd);
    const double vx = val(X.mx, XL.mx, i) / rho, vy = val(X.my, XL.my, i) / rho, vz = val(X.mz, XL.mz, i) / rho;
    const double u = vx * basis[c] + vy * basis[S + c] + vz * basis[2 * S + c];
    const double v = vx * basis[3 * S + c] + vy * basis[4 * S + c] + vz * basis[5 * S + c];
    wsum[i] += (V.clo[k] * val(X.w, XL.w, i) + V.chi[k] * val(X.w, XL.w, i + S)) / rho;
    const double w = G.area[c] * V.rc[k] * V.rc[k] * V.dz[k];
    const double q[kZonalQ] = {w, w * u, w * v, w * T, w * p, w * u * v, w * v * T, w * u * u, w * v * v};
    double* h = hist + band[c] * kZonalQ;
#pragma unroll
    for (int j = 0; j < kZonalQ; ++j) atomicAdd(h + j, q[j]);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nlat * kZonalQ; t += blockDim.x)
    if (hist[t] != 0.0) atomicAdd(tmp + (size_t)k * nlat * kZonalQ + t, hist[t]);
}

// per (level, band): the state's band means and covariances added to acc,
// the sums cleared for the next state
__global__ void k_zonal_finish(int n, double* __restrict__ tmp, double* __restrict__ acc) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  double* s = tmp + (size_t)t * kZonalQ;
  double* a = acc + (size_t)t * kZonalQ;
  const double W = s[0];
  if (W > 0.0) {
    const double mu = s[1] / W, mv = s[2] / W, mT = s[3] / W, mp = s[4] / W;
    a[0] += W;
    a[1] += mu;
    a[2] += mv;
    a[3] += mT;
    a[4] += mp;
    a[5] += s[5] / W - mu * mv;
    a[6] += s[6] / W - mv * mT;
    a[7] += s[7] / W - mu * mu;
    a[8] += s[8] / W - mv * mv;
  }
  for (int j = 0; j < kZonalQ; ++j) s[j] = 0.0;
}

template <typename R>
int zonal_launch(thor_state* s) {
  auto* I = static_cast<Impl<R>*>(s->impl.get());
  ZonalAcc& z = s->zonal;
  const int nv = I->G.nv;
  dim3 grid((I->G.ncol + kZonalThreads - 1) / kZonalThreads, nv);
  const size_t smem = (size_t)z.nlat * kZonalQ * sizeof(double);
  k_zonal_partial<R><<<grid, kZonalThreads, smem, I->stream>>>(I->G, I->V, I->ph, I->Xt, I->XtL, z.band, z.basis, z.nlat,
                                                                z.tmp, z.wsum);
  const int n = nv * z.nlat;
  k_zonal_finish<<<(n + 255) / 256, 256, 0, I->stream>>>(n, z.tmp, z.acc);
  I->launches += 2;
  return cudaGetLastError() == cudaSuccess ? THOR_OK : THOR_ECUDA;
}

// (re)allocates the accumulator for nlat bands: band index and east/north
// unit vectors of every column (host, float64, from the grid points), sums
// and accumulator cleared
int zonal_setup(thor_state* s, int nlat) {
  ZonalAcc& z = s->zonal;
  zonal_release(z);
  const HostGrid& h = s->grid->h;
  const int ncol = h.ncol, nv = h.nv, S = (ncol + kBlock - 1) / kBlock * kBlock;
  std::vector<int> band(S, 0);
  std::vector<double> basis(6 * (size_t)S, 0.0);
  for (int c = 0; c < ncol; ++c) {
    const double x = h.P[3 * c], y = h.P[3 * c + 1], zz = h.P[3 * c + 2];
    const double lon = std::atan2(y, x), lat = std::asin(std::fmax(-1.0, std::fmin(1.0, zz)));
    // 1e-9 rad: a cell on a band edge (the equatorial cells) goes north,
    // whatever the last bits of its coordinates
    int b = (int)std::floor((lat + 0.5 * M_PI + 1e-9) / M_PI * nlat);
    band[c] = b < nlat ? (b < 0 ? 0 : b) : nlat - 1;
    if (std::hypot(x, y) < 1e-9) continue;   // a polar cell: east and north undefined, u = v = 0
    basis[c] = -std::sin(lon);
    basis[S + c] = std::cos(lon);
    basis[2 * S + c] = 0.0;
    basis[3 * S + c] = -std::sin(lat) * std::cos(lon);
    basis[4 * S + c] = -std::sin(lat) * std::sin(lon);
    basis[5 * S + c] = std::cos(lat);
  }
  const size_t nq = (size_t)nv * nlat * kZonalQ;
  const size_t nw = (size_t)nv * S;
  if (cudaMalloc(&z.band, S * sizeof(int)) || cudaMalloc(&z.basis, basis.size() * sizeof(double)) ||
      cudaMalloc(&z.tmp, nq * sizeof(double)) || cudaMalloc(&z.acc, nq * sizeof(double)) ||
      cudaMalloc(&z.wsum, nw * sizeof(double))) {
    zonal_release(z);
    return THOR_ENOMEM;
  }
  if (cudaMemcpy(z.band, band.data(), S * sizeof(int), cudaMemcpyHostToDevice) ||
      cudaMemcpy(z.basis, basis.data(), basis.size() * sizeof(double), cudaMemcpyHostToDevice) ||
      cudaMemset(z.tmp, 0, nq * sizeof(double)) || cudaMemset(z.acc, 0, nq * sizeof(double)) ||
      cudaMemset(z.wsum, 0, nw * sizeof(double))) {
    zonal_release(z);
    return THOR_ECUDA;
  }
  z.nlat = nlat;
  z.samples = 0;
  return THOR_OK;
}

}  // namespace

void zonal_release(ZonalAcc& z) {
  if (z.band) cudaFree(z.band);
  if (z.basis) cudaFree(z.basis);
  if (z.tmp) cudaFree(z.tmp);
  if (z.acc) cudaFree(z.acc);
  if (z.wsum) cudaFree(z.wsum);
  z = ZonalAcc{};
}

}  // namespace thor

extern "C" {

int thor_zonal_accumulate(thor_state* s, int nlat) {
  if (!s || nlat < 1 || nlat > 360) return THOR_EINVAL;   // the band histogram fits 48 KB of shared memory
  if (s->zonal.nlat != nlat) {
    if (cudaStreamSynchronize(s->impl->stream)) return THOR_ECUDA;
    const int rc = thor::zonal_setup(s, nlat);
    if (rc) return rc;
  }
  const int rc = s->precision == THOR_FP64 ? thor::zonal_launch<double>(s) : thor::zonal_launch<float>(s);
  if (rc == THOR_OK) ++s->zonal.samples;
  return rc;
}

int thor_zonal_read(thor_state* s, int nlat, double* out, size_t n, int reset, long long* samples) {
  if (!s || !samples) return THOR_EINVAL;
  const size_t need = (size_t)s->grid->h.nv * nlat * 9;
  if (nlat < 1 || !out || n != need) return THOR_EINVAL;
  if (s->zonal.nlat != nlat) {
    std::memset(out, 0, need * sizeof(double));
    *samples = 0;
    return THOR_OK;
  }
  if (cudaStreamSynchronize(s->impl->stream) ||
      cudaMemcpy(out, s->zonal.acc, need * sizeof(double), cudaMemcpyDeviceToHost))
    return THOR_ECUDA;
  *samples = s->zonal.samples;
  if (reset) {
    const size_t colp = (size_t)(s->grid->h.ncol + thor::kBlock - 1) / thor::kBlock * thor::kBlock;
    if (cudaMemset(s->zonal.acc, 0, need * sizeof(double)) ||
        cudaMemset(s->zonal.wsum, 0, (size_t)s->grid->h.nv * colp * sizeof(double)))
      return THOR_ECUDA;
    s->zonal.samples = 0;
  }
  return THOR_OK;
}

int thor_zonal_read_w(thor_state* s, int nlat, double* out, size_t n, long long* samples) {
  if (!s || !samples || !out) return THOR_EINVAL;
  const int ncol = s->grid->h.ncol, nv = s->grid->h.nv;
  if (nlat < 1 || n != (size_t)ncol * nv) return THOR_EINVAL;
  if (s->zonal.nlat != nlat || s->zonal.samples == 0) {
    std::memset(out, 0, n * sizeof(double));
    *samples = 0;
    return THOR_OK;
  }
  const size_t S = (size_t)(ncol + thor::kBlock - 1) / thor::kBlock * thor::kBlock;
  std::vector<double> buf((size_t)nv * S);
  if (cudaStreamSynchronize(s->impl->stream) ||
      cudaMemcpy(buf.data(), s->zonal.wsum, buf.size() * sizeof(double), cudaMemcpyDeviceToHost))
    return THOR_ECUDA;
  const double inv = 1.0 / (double)s->zonal.samples;
  for (int c = 0; c < ncol; ++c)
    for (int k = 0; k < nv; ++k) out[(size_t)c * nv + k] = buf[k * S + c] * inv;
  *samples = s->zonal.samples;
  return THOR_OK;
}

}  // extern "C"
