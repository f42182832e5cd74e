// Global diagnostics of one state in float64 (Sec. 3: dry mass, total energy,
// axial angular momentum; extrema and a non-finite count): a grid-stride
// pass with compensated (Kahan) sums per thread, a block tree, then one
// warp per quantity over the block partials. Shared by thor_diag and by the
// energy budget and fixer inside the large step; internal linkage in every
// translation unit that includes it.
#pragma once

#include "thor_impl.cuh"

namespace thor {
namespace {

constexpr int kDiagBlocks = 512;
static_assert(kFixBufBytes == (size_t)(2 * (kDiagBlocks + 1) * 8 + 2) * sizeof(double), "fixer buffer size");
constexpr int kDiagThreads = 256;

struct Kahan {
  double s = 0, c = 0;
  __device__ void add(double x) {
    double y = x - c;
    double t = s + y;
    c = (t - s) - y;
    s = t;
  }
};

// partial sums per block: mass, energy, aam, sum V T, sum V, max vh, max w, nonfinite
// XL: the low parts of a compensated state (null pointers: none)
template <typename R>
__global__ void __launch_bounds__(kDiagThreads) k_diag_partial(Geo<R> G, Vert V, Phys ph, Xf<R> X, Xf<R> XL,
                                                               double* part) {
  const int S = G.colp, nv = G.nv;
  const long long ncell = (long long)G.ncol * nv;
  Kahan mass, en, aam, vt, vs;
  double mvh = 0, mw = 0;
  double nf = 0;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < ncell;
       q += (long long)gridDim.x * blockDim.x) {
    int k = (int)(q / G.ncol), c = (int)(q % G.ncol);
    size_t i = (size_t)k * S + c;
    const bool cmp = XL.rho != nullptr;
    auto val = [&](const R* hi, const R* lo, size_t j) {
      return cmp ? (double)hi[j] + (double)lo[j] : (double)hi[j];
    };
    double rx = G.rhat[c], ry = G.rhat[S + c], rz = G.rhat[2 * S + c];
    const double rhop = val(X.rho, XL.rho, i), thp = val(X.th, XL.th, i);
    double rho = V.rhob[k] + rhop;
    double th = V.thb[k] + thp;
    double p = V.pb[k] + V.pb[k] * expm1(ph.gamma * log1p(thp / V.thb[k]));
    double Temp = p / (rho * ph.Rd);
    double wlo = val(X.w, XL.w, i), whi = val(X.w, XL.w, i + S);
    double wc = V.clo[k] * wlo + V.chi[k] * whi;
    const double mhx = val(X.mx, XL.mx, i), mhy = val(X.my, XL.my, i), mhz = val(X.mz, XL.mz, i);
    double mx = mhx + wc * rx, my = mhy + wc * ry, mz = mhz + wc * rz;
    double vol = G.area[c] * V.rc[k] * V.rc[k] * V.dz[k];
    mass.add(vol * rho);
    en.add(vol * (rho * ph.cv * Temp + 0.5 * (mx * mx + my * my + mz * mz) / rho + rho * ph.g * V.zc[k]));
    double r = V.rc[k];
    aam.add(vol * (r * (rx * my - ry * mx) + rho * ph.omega * r * r * (rx * rx + ry * ry)));
    vt.add(vol * Temp);
    vs.add(vol);
    double hx = mhx / rho, hy = mhy / rho, hz = mhz / rho;
    mvh = fmax(mvh, sqrt(hx * hx + hy * hy + hz * hz));
    if (k >= 1) {
      double rif = V.wlo[k] * (V.rhob[k - 1] + val(X.rho, XL.rho, i - S)) + V.whi[k] * rho;
      mw = fmax(mw, fabs(wlo / rif));
    }
    double vals[6] = {(double)X.rho[i], (double)X.mx[i], (double)X.my[i], (double)X.mz[i], th, (double)X.w[i]};
    for (int j = 0; j < 6; ++j)
      if (!isfinite(vals[j])) nf += 1.0;
    if (k == nv - 1 && !isfinite((double)X.w[i + S])) nf += 1.0;
  }
  __shared__ double sh[8][kDiagThreads];
  double mine[8] = {mass.s, en.s, aam.s, vt.s, vs.s, mvh, mw, nf};
  for (int j = 0; j < 8; ++j) sh[j][threadIdx.x] = mine[j];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int j = 0; j < 8; ++j) {
        double a = sh[j][threadIdx.x], b = sh[j][threadIdx.x + w];
        sh[j][threadIdx.x] = (j == 5 || j == 6) ? fmax(a, b) : a + b;
      }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int j = 0; j < 8; ++j) part[blockIdx.x * 8 + j] = sh[j][0];
}

// One warp per quantity: every lane sums a strided share of the block
// partials (compensated), then lane 0 adds the 32 lane sums in order
// (compensated); extrema by max, the non-finite count by plain addition.
__global__ void __launch_bounds__(256) k_diag_final(double* part, int nblocks) {
  const int j = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ double lanes[8][32];
  const bool is_max = j == 5 || j == 6, is_count = j == 7;
  double s = 0.0, comp = 0.0;
  for (int b = lane; b < nblocks; b += 32) {
    const double x = part[b * 8 + j];
    if (is_max) {
      s = fmax(s, x);
    } else if (is_count) {
      s += x;
    } else {
      const double y = x - comp, t = s + y;
      comp = (t - s) - y;
      s = t;
    }
  }
  lanes[j][lane] = s;
  __syncwarp();
  if (lane == 0) {
    double o = 0.0, cm = 0.0;
    for (int l = 0; l < 32; ++l) {
      const double x = lanes[j][l];
      if (is_max) {
        o = fmax(o, x);
      } else if (is_count) {
        o += x;
      } else {
        const double y = x - cm, t = o + y;
        cm = (t - o) - y;
        o = t;
      }
    }
    part[nblocks * 8 + j] = o;
  }
}

}  // namespace
}  // namespace thor
