// Kernels of one large step (Sec. 3-5 of Mendonca et al. 2016) and their
// launch sequence. Thread mapping for the stencil kernels: one thread per
// column, looping over a chunk of levels, so that the per-column stencil
// weights are loaded once and reused across the chunk; blockIdx.y selects the
// chunk. The vertical solve runs one thread per column over all levels.
#include "../../include/thor.h"
#include "thor_impl.cuh"

namespace thor {

// ---------------------------------------------------------------- slow terms

// Pointwise derived quantities at the stage state: p', T', theta, the full
// 3-D velocity, v_h = M/rho (centres) and v_r = W/rho (interfaces).
template <typename R>
__global__ void k_derived(Geo<R> G, Vert V, Phys ph, Xf<R> X, Work<R> T, int kchunk) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= G.ncol) return;
  const int S = G.colp;
  R rx = G.rhat[c], ry = G.rhat[S + c], rz = G.rhat[2 * S + c];
  int k0 = blockIdx.y * kchunk, k1 = min(G.nv + 1, k0 + kchunk);
  for (int k = k0; k < k1; ++k) {
    if (k < G.nv) {
      int i = k * S + c;
      R rho = (R)V.rhob[k] + X.rho[i];
      R thp = X.th[i];
      R pp = eos_dev<R>((R)V.pb[k], (R)V.thb[k], thp, (R)ph.gamma);
      R p = (R)V.pb[k] + pp;
      R Temp = p / (rho * (R)ph.Rd);
      R wc = (R)V.clo[k] * X.w[i] + (R)V.chi[k] * X.w[i + S];
      R inv = R(1) / rho;
      R mx = X.mx[i], my = X.my[i], mz = X.mz[i];
      T.pp[i] = pp;
      T.Tp[i] = Temp - (R)V.Tb[k];
      T.theta[i] = ((R)V.thb[k] + thp) * inv;
      T.vx[i] = (mx + wc * rx) * inv;
      T.vy[i] = (my + wc * ry) * inv;
      T.vz[i] = (mz + wc * rz) * inv;
      T.vhx[i] = mx * inv;
      T.vhy[i] = my * inv;
      T.vhz[i] = mz * inv;
    }
    if (k >= 1 && k < G.nv) {
      int i = k * S + c;
      R rlo = (R)V.rhob[k - 1] + X.rho[i - S], rhi = (R)V.rhob[k] + X.rho[i];
      R rif = (R)V.wlo[k] * rlo + (R)V.whi[k] * rhi;
      T.vr[i] = X.w[i] / rif;
    } else if (k == 0 || k == G.nv) {
      T.vr[k * S + c] = 0;
    }
  }
}

// First Laplacians of the hyperdiffusion (Sec. 4), already multiplied by
// K_d and, for the momentum and temperature terms, by rho.
template <typename R>
__global__ void k_lap1(Geo<R> G, Vert V, Xf<R> X, Work<R> T, R Kd, int kchunk) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= G.ncol) return;
  const int S = G.colp;
  Nbr7 nb = load_nbr(G, c);
  W7<R> wl = load_w7(G.wlap, S, c);
  int k0 = blockIdx.y * kchunk, k1 = min(G.nv + 1, k0 + kchunk);
  for (int k = k0; k < k1; ++k) {
    if (k < G.nv) {
      int o = k * S;
      R inv_r2 = R(1.0 / (V.rc[k] * V.rc[k]));
      R rho = (R)V.rhob[k] + X.rho[o + c];
      T.qrho[o + c] = Kd * apply7(wl, nb, X.rho + o) * inv_r2;
      R rk = rho * Kd * inv_r2;
      T.qvx[o + c] = rk * apply7(wl, nb, T.vhx + o);
      T.qvy[o + c] = rk * apply7(wl, nb, T.vhy + o);
      T.qvz[o + c] = rk * apply7(wl, nb, T.vhz + o);
      T.qT[o + c] = rk * apply7(wl, nb, T.Tp + o);
    }
    if (k >= 1 && k < G.nv) {
      int o = k * S;
      R rlo = (R)V.rhob[k - 1] + X.rho[o - S + c], rhi = (R)V.rhob[k] + X.rho[o + c];
      R rif = (R)V.wlo[k] * rlo + (R)V.whi[k] * rhi;
      T.qvr[o + c] = rif * Kd * apply7(wl, nb, T.vr + o) * R(1.0 / (V.ri[k] * V.ri[k]));
    } else if (k == 0 || k == G.nv) {
      T.qvr[k * S + c] = 0;
    }
  }
}

// Slow tendencies at the centres (right-hand sides of Eqs. mom2, dens2, pt2):
// S_M = -grad_h p - A_h - C_h + F_M, S_rho = -div(M) - div(W) + F_rho,
// S_th = F_th - div(theta M) - div(theta W), plus Dsc = div(M) + div(W) of the
// stage state (divergence damping), the radial advection+Coriolis and
// Pi = gamma p / rho theta.
template <typename R>
__global__ void k_slow(Geo<R> G, Vert V, Phys ph, Xf<R> X, Work<R> T, Slow<R> SL, int hyper,
                       int kchunk) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= G.ncol) return;
  const int S = G.colp;
  Nbr7 nb = load_nbr(G, c);
  W7x3<R> wd = load_w7x3(G.wdiv, S, c);
  W7x3<R> wg = load_w7x3(G.wgrad, S, c);
  W7<R> wl = load_w7(G.wlap, S, c);
  R rx = G.rhat[c], ry = G.rhat[S + c], rz = G.rhat[2 * S + c];
  const R two_om = R(2.0 * ph.omega);
  int k0 = blockIdx.y * kchunk, k1 = min(G.nv, k0 + kchunk);
  for (int k = k0; k < k1; ++k) {
    const int o = k * S, i = o + c;
    const R inv_r = R(1.0 / V.rc[k]);
    const R inv_r2 = R(1.0 / (V.rc[k] * V.rc[k]));
    const R qlo = (R)(V.ri[k] * V.ri[k]), qhi = (R)(V.ri[k + 1] * V.ri[k + 1]);
    const R sv = R(1.0 / (V.rc[k] * V.rc[k] * V.dz[k]));
    R rho = (R)V.rhob[k] + X.rho[i];
    R thfull = (R)V.thb[k] + X.th[i];
    R p = (R)V.pb[k] + T.pp[i];

    // hyperdiffusion (Sec. 4)
    R Frho = 0, FMx = 0, FMy = 0, FMz = 0, Fth = 0;
    if (hyper) {
      Frho = -apply7(wl, nb, T.qrho + o) * inv_r2;
      FMx = -apply7(wl, nb, T.qvx + o) * inv_r2;
      FMy = -apply7(wl, nb, T.qvy + o) * inv_r2;
      FMz = -apply7(wl, nb, T.qvz + o) * inv_r2;
      project(rx, ry, rz, FMx, FMy, FMz);
      R Fp = -(R)ph.Rd * apply7(wl, nb, T.qT + o) * inv_r2;
      Fth = thfull / ((R)ph.gamma * p) * Fp;
    }

    // advection div(rho v v_j) of the Cartesian components (Sec. 3)
    const R* vs[3] = {T.vx, T.vy, T.vz};
    R A[3];
    R wlo_w = X.w[i], whi_w = X.w[i + S];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      R ah = div7_scaled(wd, nb, vs[j] + o, X.mx + o, X.my + o, X.mz + o) * inv_r;
      R vlo = 0, vhi = 0;
      if (k >= 1) vlo = (R)V.wlo[k] * vs[j][i - S] + (R)V.whi[k] * vs[j][i];
      if (k + 1 < G.nv) vhi = (R)V.wlo[k + 1] * vs[j][i] + (R)V.whi[k + 1] * vs[j][i + S];
      A[j] = ah + (qhi * whi_w * vhi - qlo * wlo_w * vlo) * sv;
    }
    // Coriolis 2 Omega z x (rho v) with the full momentum
    R wc = (R)V.clo[k] * wlo_w + (R)V.chi[k] * whi_w;
    R mx = X.mx[i], my = X.my[i], mz = X.mz[i];
    R fx = mx + wc * rx, fy = my + wc * ry;
    A[0] += -two_om * fy;
    A[1] += two_om * fx;
    R acr = A[0] * rx + A[1] * ry + A[2] * rz;
    R ahx = A[0] - acr * rx, ahy = A[1] - acr * ry, ahz = A[2] - acr * rz;

    R gx, gy, gz;
    grad7(wg, nb, T.pp + o, gx, gy, gz);
    R smx = -gx * inv_r - ahx + FMx, smy = -gy * inv_r - ahy + FMy, smz = -gz * inv_r - ahz + FMz;
    project(rx, ry, rz, smx, smy, smz);
    SL.smx[i] = smx;
    SL.smy[i] = smy;
    SL.smz[i] = smz;

    R dh = div7(wd, nb, X.mx + o, X.my + o, X.mz + o) * inv_r;
    R dv = (qhi * whi_w - qlo * wlo_w) * sv;
    SL.srho[i] = -dh - dv + Frho;
    SL.dsc[i] = dh + dv;

    R dht = div7_scaled(wd, nb, T.theta + o, X.mx + o, X.my + o, X.mz + o) * inv_r;
    R thlo = 0, thhi = 0;
    if (k >= 1) thlo = (R)V.wlo[k] * T.theta[i - S] + (R)V.whi[k] * T.theta[i];
    if (k + 1 < G.nv) thhi = (R)V.wlo[k + 1] * T.theta[i] + (R)V.whi[k + 1] * T.theta[i + S];
    R dvt = (qhi * thhi * whi_w - qlo * thlo * wlo_w) * sv;
    SL.sth[i] = Fth - dht - dvt;
    SL.acr[i] = acr;
    SL.pi[i] = (R)ph.gamma * p / thfull;
  }
}

// Slow tendency of the vertical momentum at the interior interfaces
// (right-hand side of Eq. momr2) and theta at the interfaces.
template <typename R>
__global__ void k_slow_w(Geo<R> G, Vert V, Phys ph, Xf<R> X, Work<R> T, Slow<R> SL, int hyper,
                         int kchunk) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= G.ncol) return;
  const int S = G.colp;
  Nbr7 nb = load_nbr(G, c);
  W7<R> wl = load_w7(G.wlap, S, c);
  int k0 = blockIdx.y * kchunk, k1 = min(G.nv + 1, k0 + kchunk);
  for (int k = k0; k < k1; ++k) {
    const int i = k * S + c;
    if (k == 0 || k == G.nv) {
      SL.sw[i] = 0;
      SL.thi[i] = 0;
      continue;
    }
    R wlo = (R)V.wlo[k], whi = (R)V.whi[k];
    R FW = 0;
    if (hyper) FW = -apply7(wl, nb, T.qvr + k * S) * R(1.0 / (V.ri[k] * V.ri[k]));
    R sw = (R)V.Rb[k] - (T.pp[i] - T.pp[i - S]) / (R)V.dzc[k]
         - (R)ph.g * (wlo * X.rho[i - S] + whi * X.rho[i])
         - (wlo * SL.acr[i - S] + whi * SL.acr[i]) + FW;
    SL.sw[i] = sw;
    SL.thi[i] = wlo * T.theta[i - S] + whi * T.theta[i];
  }
}

// Perturbations at the start of a stage: Phi* = Phi^t - Phi^(s); p* from the
// nonlinear Eq. theta_to_p.
template <typename R>
__global__ void k_stage_init(Geo<R> G, Vert V, Phys ph, Xf<R> Xt, Xf<R> Xs, Work<R> T, Pert<R> P,
                             int kchunk) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= G.ncol) return;
  const int S = G.colp;
  int k0 = blockIdx.y * kchunk, k1 = min(G.nv + 1, k0 + kchunk);
  for (int k = k0; k < k1; ++k) {
    int i = k * S + c;
    if (k < G.nv) {
      P.rho[i] = Xt.rho[i] - Xs.rho[i];
      P.mx[i] = Xt.mx[i] - Xs.mx[i];
      P.my[i] = Xt.my[i] - Xs.my[i];
      P.mz[i] = Xt.mz[i] - Xs.mz[i];
      P.th[i] = Xt.th[i] - Xs.th[i];
      R ppt = eos_dev<R>((R)V.pb[k], (R)V.thb[k], Xt.th[i], (R)ph.gamma);
      P.p[i] = ppt - T.pp[i];
    }
    P.w[i] = Xt.w[i] - Xs.w[i];
  }
}

// ---------------------------------------------------------------- small step

// 3-D divergence of the total momentum (divergence damping, Sec. 4)
template <typename R>
__global__ void k_ss_div(Geo<R> G, Vert V, Slow<R> SL, Pert<R> P, Work<R> T, int kchunk) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= G.ncol) return;
  const int S = G.colp;
  Nbr7 nb = load_nbr(G, c);
  W7x3<R> wd = load_w7x3(G.wdiv, S, c);
  int k0 = blockIdx.y * kchunk, k1 = min(G.nv, k0 + kchunk);
  for (int k = k0; k < k1; ++k) {
    const int o = k * S, i = o + c;
    R dh = div7(wd, nb, P.mx + o, P.my + o, P.mz + o) * R(1.0 / V.rc[k]);
    R dv = ((R)(V.ri[k + 1] * V.ri[k + 1]) * P.w[i + S] - (R)(V.ri[k] * V.ri[k]) * P.w[i])
         * R(1.0 / (V.rc[k] * V.rc[k] * V.dz[k]));
    T.dd[i] = SL.dsc[i] + dh + dv;
  }
}

template <typename R>
__global__ void k_ss_grad(Geo<R> G, Vert V, Work<R> T, int kchunk) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= G.ncol) return;
  const int S = G.colp;
  Nbr7 nb = load_nbr(G, c);
  W7x3<R> wg = load_w7x3(G.wgrad, S, c);
  int k0 = blockIdx.y * kchunk, k1 = min(G.nv, k0 + kchunk);
  for (int k = k0; k < k1; ++k) {
    const int o = k * S, i = o + c;
    R gx, gy, gz;
    grad7(wg, nb, T.dd + o, gx, gy, gz);
    R inv_r = R(1.0 / V.rc[k]);
    T.gx[i] = gx * inv_r;
    T.gy[i] = gy * inv_r;
    T.gz[i] = gz * inv_r;
  }
}

// Eq. mom2 with the divergence damping: M* <- proj(M* + dtau(-grad p* + DD + S_M))
template <typename R>
__global__ void k_ss_mom(Geo<R> G, Vert V, Slow<R> SL, Pert<R> P, Work<R> T, R dtau, R Kd,
                         int divdamp, int kchunk) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= G.ncol) return;
  const int S = G.colp;
  Nbr7 nb = load_nbr(G, c);
  W7x3<R> wg = load_w7x3(G.wgrad, S, c);
  W7<R> wl = load_w7(G.wlap, S, c);
  R rx = G.rhat[c], ry = G.rhat[S + c], rz = G.rhat[2 * S + c];
  int k0 = blockIdx.y * kchunk, k1 = min(G.nv, k0 + kchunk);
  for (int k = k0; k < k1; ++k) {
    const int o = k * S, i = o + c;
    R inv_r = R(1.0 / V.rc[k]);
    R ddx = 0, ddy = 0, ddz = 0;
    if (divdamp) {
      R s = -Kd * R(1.0 / (V.rc[k] * V.rc[k]));
      ddx = s * apply7(wl, nb, T.gx + o);
      ddy = s * apply7(wl, nb, T.gy + o);
      ddz = s * apply7(wl, nb, T.gz + o);
      project(rx, ry, rz, ddx, ddy, ddz);
    }
    R gx, gy, gz;
    grad7(wg, nb, P.p + o, gx, gy, gz);
    R mx = P.mx[i] + dtau * (-gx * inv_r + ddx + SL.smx[i]);
    R my = P.my[i] + dtau * (-gy * inv_r + ddy + SL.smy[i]);
    R mz = P.mz[i] + dtau * (-gz * inv_r + ddz + SL.smz[i]);
    project(rx, ry, rz, mx, my, mz);
    P.mx[i] = mx;
    P.my[i] = my;
    P.mz[i] = mz;
  }
}

// HE-VI column step: Eqs. dens2 and pt2 substituted into Eq. momr2 give a
// tridiagonal system in W* at the interior interfaces (rigid lid W* = 0 at
// the bottom and top), solved by the Thomas algorithm in float64; then
// Eq. dens2, Eq. pt2 and the nonlinear Eq. theta_to_p with the new W*.
template <typename R>
__global__ void __launch_bounds__(kBlock) k_ss_col(Geo<R> G, Vert V, Phys ph, Xf<R> Xs, Slow<R> SL,
                                                   Pert<R> P, Work<R> T, double dtau) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= G.ncol) return;
  const int S = G.colp, nv = G.nv;
  Nbr7 nb = load_nbr(G, c);
  W7x3<R> wd = load_w7x3(G.wdiv, S, c);
  double a[kMaxNv], b[kMaxNv], cc[kMaxNv];
  double cp_[kMaxNv + 1], dp_[kMaxNv + 1];
  const R rdt = (R)dtau;
  for (int k = 0; k < nv; ++k) {
    const int o = k * S, i = o + c;
    R inv_r = R(1.0 / V.rc[k]);
    R dh = div7(wd, nb, P.mx + o, P.my + o, P.mz + o) * inv_r;
    R dht = div7_scaled(wd, nb, T.theta + o, P.mx + o, P.my + o, P.mz + o) * inv_r;
    R ak = P.rho[i] + rdt * (SL.srho[i] - dh);
    R thk = P.th[i];
    R bk = thk + rdt * (SL.sth[i] - dht);
    a[k] = (double)ak;
    b[k] = (double)bk;
    cc[k] = (double)P.p[i] + (double)SL.pi[i] * ((double)bk - (double)thk);
  }
  // forward elimination over the interior interfaces 1..nv-1
  const double g = ph.g, dt2 = dtau * dtau;
  double wprev_c = 0.0, wprev_d = 0.0;
  for (int m = 1; m < nv; ++m) {
    const int i = m * S + c;
    double s_lo = 1.0 / (V.rc[m - 1] * V.rc[m - 1] * V.dz[m - 1]);
    double s_hi = 1.0 / (V.rc[m] * V.rc[m] * V.dz[m]);
    double q = V.ri[m] * V.ri[m];
    double th_m = (double)SL.thi[i];
    double pi_lo = (double)SL.pi[i - S], pi_hi = (double)SL.pi[i];
    double wlo = V.wlo[m], whi = V.whi[m], inv_dzc = 1.0 / V.dzc[m];
    double lower = 0.0, upper = 0.0;
    if (m > 1) {
      double qm = V.ri[m - 1] * V.ri[m - 1];
      double thm = (double)SL.thi[i - S];
      lower = -dt2 * inv_dzc * pi_lo * s_lo * qm * thm + dt2 * g * wlo * s_lo * qm;
    }
    if (m < nv - 1) {
      double qp = V.ri[m + 1] * V.ri[m + 1];
      double thp = (double)SL.thi[i + S];
      upper = -dt2 * inv_dzc * pi_hi * s_hi * qp * thp - dt2 * g * whi * s_hi * qp;
    }
    double diag = 1.0 + dt2 * inv_dzc * q * th_m * (pi_hi * s_hi + pi_lo * s_lo)
                - dt2 * g * q * (wlo * s_lo - whi * s_hi);
    double rhs = (double)P.w[i] + dtau * (double)SL.sw[i] - dtau * inv_dzc * (cc[m] - cc[m - 1])
               - dtau * g * (wlo * a[m - 1] + whi * a[m]);
    double den = diag - lower * wprev_c;
    double inv = 1.0 / den;
    double cm = upper * inv;
    double dm = (rhs - lower * wprev_d) * inv;
    cp_[m] = cm;
    dp_[m] = dm;
    wprev_c = cm;
    wprev_d = dm;
  }
  // back substitution; cp_/dp_ now hold W*
  double wnext = 0.0;
  for (int m = nv - 1; m >= 1; --m) {
    double wm = dp_[m] - cp_[m] * wnext;
    dp_[m] = wm;
    wnext = wm;
  }
  dp_[0] = 0.0;
  dp_[nv] = 0.0;
  const double gamma = ph.gamma;
  for (int k = 0; k < nv; ++k) {
    const int i = k * S + c;
    double s = 1.0 / (V.rc[k] * V.rc[k] * V.dz[k]);
    double qlo = V.ri[k] * V.ri[k], qhi = V.ri[k + 1] * V.ri[k + 1];
    double wl = dp_[k], wh = dp_[k + 1];
    double thl = k > 0 ? (double)SL.thi[i] : 0.0;
    double thh = k + 1 < nv ? (double)SL.thi[i + S] : 0.0;
    double rho_new = a[k] - dtau * s * (qhi * wh - qlo * wl);
    double th_new = b[k] - dtau * s * (qhi * thh * wh - qlo * thl * wl);
    P.rho[i] = (R)rho_new;
    P.th[i] = (R)th_new;
    // p* = EOS(Th^(s) + Th*) - p^(s) = p^(s) ((1 + Th*/Th^(s))^gamma - 1)
    R ps = (R)V.pb[k] + T.pp[i];
    R ths = (R)V.thb[k] + Xs.th[i];
    P.p[i] = ps * rexpm1<R>((R)gamma * rlog1p<R>((R)th_new / ths));
    if (k >= 1) P.w[i] = (R)dp_[k];
  }
}

// Phi^(s+1) = Phi^(s) + Phi*
template <typename R>
__global__ void k_stage_end(Geo<R> G, Xf<R> Xs, Pert<R> P, Xf<R> Xo, int kchunk) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= G.ncol) return;
  const int S = G.colp;
  int k0 = blockIdx.y * kchunk, k1 = min(G.nv + 1, k0 + kchunk);
  for (int k = k0; k < k1; ++k) {
    int i = k * S + c;
    if (k < G.nv) {
      Xo.rho[i] = Xs.rho[i] + P.rho[i];
      Xo.mx[i] = Xs.mx[i] + P.mx[i];
      Xo.my[i] = Xs.my[i] + P.my[i];
      Xo.mz[i] = Xs.mz[i] + P.mz[i];
      Xo.th[i] = Xs.th[i] + P.th[i];
    }
    Xo.w[i] = Xs.w[i] + P.w[i];
  }
}

// ---------------------------------------------------------------- physics

// Sec. 5 backward-Euler friction (Eq. im_eq_v) and Newtonian relaxation
// (Eq. im_eq_t) with the Sec. 6.1 Held-Suarez or Sec. 6.2 hot-Jupiter
// coefficients; sigma = p / p_s with p_s extrapolated hydrostatically at the
// lowest layer's temperature.
template <typename R>
__global__ void k_physics(Geo<R> G, Vert V, Phys ph, Xf<R> X, int forcing, double dt, double hj_dT) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= G.ncol) return;
  const int S = G.colp;
  const R gamma = (R)ph.gamma;
  R sl = G.sinlat[c], cl = G.coslat[c], clon = G.coslon[c];
  R p0 = (R)V.pb[0] + eos_dev<R>((R)V.pb[0], (R)V.thb[0], X.th[c], gamma);
  R T0 = p0 / (((R)V.rhob[0] + X.rho[c]) * (R)ph.Rd);
  R ps = p0 * rexp<R>((R)(ph.g * V.zc[0]) / ((R)ph.Rd * T0));
  const R rdt = (R)dt;
  for (int k = 0; k < G.nv; ++k) {
    const int i = k * S + c;
    R rhop = X.rho[i];
    R rho = (R)V.rhob[k] + rhop;
    R p = (R)V.pb[k] + eos_dev<R>((R)V.pb[k], (R)V.thb[k], X.th[i], gamma);
    R Temp = p / (rho * (R)ph.Rd);
    R sigma = p / ps;
    R Kv, KT, Teq;
    if (forcing == 1) {
      const R day = R(86400.0);
      const R kf = R(1) / day, ka = R(1) / (R(40) * day), ks = R(1) / (R(4) * day);
      const R sb = R(0.7), p00 = R(1.0e5);
      R ramp = (sigma - sb) / (R(1) - sb);
      ramp = ramp > R(0) ? ramp : R(0);
      Kv = kf * ramp;
      R c2 = cl * cl;
      KT = ka + (ks - ka) * ramp * c2 * c2;
      R pr = p / p00;
      Teq = (R(315) - R(60) * sl * sl - R(10) * rlog<R>(pr) * c2) * rpow<R>(pr, (R)ph.kappa);
      Teq = Teq > R(200) ? Teq : R(200);
    } else {
      const R ss = R(0.12), zs = R(2.0e6), Ts = R(1600), Gt = R(2.0e-4), dTs = R(10);
      R z = (R)V.zc[k];
      R Tv, bt;
      if (z <= zs) {
        R h = Gt * (z - zs) / R(2);
        Tv = Ts - Gt * (zs + (z - zs) / R(2)) + rsqrt_<R>(h * h + dTs * dTs);
        bt = (R)sin(M_PI * (double)((sigma - ss) / (R(2) * (R(1) - ss))));
      } else {
        Tv = Ts - Gt * zs + dTs;
        bt = 0;
      }
      Kv = 0;
      KT = R(1) / R(1.5e5);
      Teq = Tv + bt * (R)hj_dT * clon * cl;
    }
    R fr = R(1) / (R(1) + Kv * rdt);
    X.mx[i] *= fr;
    X.my[i] *= fr;
    X.mz[i] *= fr;
    R Tn = (Temp + KT * rdt * Teq) / (R(1) + KT * rdt);
    // rho theta at fixed rho: Th/Th_bar = ((rho/rho_bar)(T/T_bar))^(1/gamma)
    R lr = rlog1p<R>(rhop / (R)V.rhob[k]) + rlog<R>(Tn / (R)V.Tb[k]);
    X.th[i] = (R)V.thb[k] * rexpm1<R>(lr / gamma);
  }
}

// ---------------------------------------------------------------- driver

template <typename R>
void Impl<R>::launch_2d(int nplanes, int kchunk, dim3& grid) const {
  grid = dim3((G.ncol + kBlock - 1) / kBlock, (nplanes + kchunk - 1) / kchunk);
}

template <typename R>
int Impl<R>::large_step(double dt, int n_small) {
  const int kc = kchunk;
  dim3 g2, g2i;
  launch_2d(G.nv, kc, g2);
  launch_2d(G.nv + 1, kc, g2i);
  dim3 g1((G.ncol + kBlock - 1) / kBlock);
  const R Kd = (R)(diff_D * dbar4 / dt);
  const double dts[3] = {dt / 3.0, dt / n_small, dt / n_small};
  const int nsub[3] = {1, n_small / 2, n_small};
  for (int s = 0; s < 3; ++s) {
    Xf<R> Xs = s == 0 ? Xt : Xst;
    mark(THOR_K_DERIVED, true);
    k_derived<R><<<g2i, kBlock, 0, stream>>>(G, V, ph, Xs, T, kc);
    mark(THOR_K_DERIVED, false);
    ++launches;
    if (hyper) {
      mark(THOR_K_LAP1, true);
      k_lap1<R><<<g2i, kBlock, 0, stream>>>(G, V, Xs, T, Kd, kc);
      mark(THOR_K_LAP1, false);
      ++launches;
    }
    mark(THOR_K_SLOW, true);
    k_slow<R><<<g2, kBlock, 0, stream>>>(G, V, ph, Xs, T, SL, hyper, kc);
    mark(THOR_K_SLOW, false);
    mark(THOR_K_SLOW_W, true);
    k_slow_w<R><<<g2i, kBlock, 0, stream>>>(G, V, ph, Xs, T, SL, hyper, kc);
    mark(THOR_K_SLOW_W, false);
    mark(THOR_K_STAGE_INIT, true);
    k_stage_init<R><<<g2i, kBlock, 0, stream>>>(G, V, ph, Xt, Xs, T, P, kc);
    mark(THOR_K_STAGE_INIT, false);
    launches += 3;
    for (int j = 0; j < nsub[s]; ++j) {
      if (divdamp) {
        mark(THOR_K_SS_DIV, true);
        k_ss_div<R><<<g2, kBlock, 0, stream>>>(G, V, SL, P, T, kc);
        mark(THOR_K_SS_DIV, false);
        mark(THOR_K_SS_GRAD, true);
        k_ss_grad<R><<<g2, kBlock, 0, stream>>>(G, V, T, kc);
        mark(THOR_K_SS_GRAD, false);
        launches += 2;
      }
      mark(THOR_K_SS_MOM, true);
      k_ss_mom<R><<<g2, kBlock, 0, stream>>>(G, V, SL, P, T, (R)dts[s], Kd, divdamp, kc);
      mark(THOR_K_SS_MOM, false);
      mark(THOR_K_SS_COL, true);
      k_ss_col<R><<<g1, kBlock, 0, stream>>>(G, V, ph, Xs, SL, P, T, dts[s]);
      mark(THOR_K_SS_COL, false);
      launches += 2;
    }
    Xf<R> Xo = s == 2 ? Xt : Xst;
    mark(THOR_K_STAGE_END, true);
    k_stage_end<R><<<g2i, kBlock, 0, stream>>>(G, Xs, P, Xo, kc);
    mark(THOR_K_STAGE_END, false);
    ++launches;
  }
  if (forcing != 0) {
    mark(THOR_K_PHYSICS, true);
    k_physics<R><<<g1, kBlock, 0, stream>>>(G, V, ph, Xt, forcing, dt, hj_dT);
    mark(THOR_K_PHYSICS, false);
    ++launches;
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

template void Impl<double>::launch_2d(int, int, dim3&) const;
template void Impl<float>::launch_2d(int, int, dim3&) const;
template int Impl<double>::large_step(double, int);
template int Impl<float>::large_step(double, int);

}  // namespace thor
