// Kernels of one large step (Sec. 3-5 of Mendonca et al. 2016) and their
// launch sequence.
//
// Stencil kernels: one thread per column, looping over a chunk of levels, so
// the per-column stencil weights are loaded once per chunk; the block's
// second index picks the chunk. A warp covers 32 consecutive columns of one
// level, so every field access is a coalesced (or neighbour-shifted) row of
// one plane.
//
// The vertical solve is split: k_ss_flux (a stencil kernel like the others)
// forms the per-cell parts of the column equations, and k_ss_solve runs the
// float64 tridiagonal elimination with two warps per 32 columns.
#include "../../include/thor.h"
#include "thor_impl.cuh"
#include "thor_reduce.cuh"

#include <utility>

namespace thor {

// ---------------------------------------------------------------- launch helper

template <typename... K, typename... A>
cudaError_t launch_k(void (*kern)(K...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...);
}

// Each step of the method is a device function over one block of columns
// (block indices passed in); the kernels below run it either for one state
// (block indices from the launch grid) or for a whole ensemble of states in
// one launch (block -> (member, local block) from a block map).


// ---------------------------------------------------------------- slow terms

// Pointwise derived quantities at the stage state: p', T', theta, the full
// 3-D velocity, v_h = M/rho (centres) and v_r = W/rho (interfaces); the
// velocities go into packed planes with theta (v4) and T' (vh4) beside them,
// the fields the next stencils gather together.
// HO: the order-k interpolation of the explicit terms (thor_init.vorder > 1)
template <typename R, bool HO = false>
__device__ __forceinline__ void d_derived(const Geo<R>& G, const VR<R>& U, const Phys& ph, const Xf<R>& X, const Work<R>& T, int shallow, int kchunk,
                                          int bx, int by) {
  int c = bx * blockDim.x + threadIdx.x;
  if (c >= G.ncol) return;
  const int S = G.colp;
  const R gamma = pc<R>(ph.gamma, ph.gamma_f), inv_Rd = pc<R>(ph.inv_Rd, ph.inv_Rd_f);
  R rx = ld(G.rhat + (c)), ry = ld(G.rhat + (S + c)), rz = ld(G.rhat + (2 * S + c));
  int k0 = by * kchunk, k1 = min(G.nv + 1, k0 + kchunk);
#pragma unroll 2
  for (int k = k0; k < k1; ++k) {
    if (k < G.nv) {
      int i = k * S + c;
      R rho = ld(U.rhob + (k)) + ld(X.rho + (i));
      R thp = ld(X.th + (i));
      R pp = eos_dev<R>(ld(U.pb + (k)), ld(U.thb + (k)), thp, gamma);
      R p = ld(U.pb + (k)) + pp;
      R inv = R(1) / rho;
      R Temp = p * inv * inv_Rd;
      R wc = HO ? vint_centre(U, X.w, k, c, S, G.nv)
                           : ld(U.clo + (k)) * ld(X.w + (i)) + ld(U.chi + (k)) * ld(X.w + (i + S));
      R mx = ld(X.mx + (i)), my = ld(X.my + (i)), mz = ld(X.mz + (i));
      const R theta = (ld(U.thb + (k)) + thp) * inv;
      T.pp[i] = pp;
      T.theta[i] = theta;
      st4(T.v4, i, (mx + wc * rx) * inv, (my + wc * ry) * inv, (mz + wc * rz) * inv, theta);
      st4(T.vh4, i, mx * inv, my * inv, mz * inv, Temp - ld(U.Tb + (k)));
      if (shallow) T.wc[i] = wc * inv;
    }
    if (k >= 1 && k < G.nv) {
      int i = k * S + c;
      R rlo = ld(U.rhob + (k - 1)) + ld(X.rho + (i - S)), rhi = ld(U.rhob + (k)) + ld(X.rho + (i));
      if constexpr (HO)
        T.vr[i] = ld(X.w + (i)) / vint_iface(U, X.rho, U.rhob, k, c, S, G.nv);
      else
        T.vr[i] = ld(X.w + (i)) / (ld(U.wlo + (k)) * rlo + ld(U.whi + (k)) * rhi);
    } else if (k == 0 || k == G.nv) {
      T.vr[k * S + c] = 0;
    }
  }
}

// First Laplacians of the hyperdiffusion (Sec. 4), already multiplied by
// K_d and, for the momentum and temperature terms, by rho.
template <typename R, bool HO = false>
__device__ __forceinline__ void d_lap1(const Geo<R>& G, const VR<R>& U, const Xf<R>& X, const Work<R>& T, R Kd, int kchunk, int bx, int by,
                                       int kend) {
  int c = bx * blockDim.x + threadIdx.x;
  if (c >= G.ncol) return;
  const int S = G.colp;
  Nbr7 nb = load_nbr(G, c);
  W7<R> wl = load_w7(G.wlap, S, c);
  int k0 = by * kchunk, k1 = min(kend, k0 + kchunk);
#pragma unroll 2
  for (int k = k0; k < k1; ++k) {
    if (k < G.nv) {
      int o = k * S;
      R inv_r2 = ld(U.inv_rc2 + (k));
      R rho = ld(U.rhob + (k)) + ld(X.rho + (o + c));
      R rk = rho * Kd * inv_r2;
      const Q4<R> lv = apply7x4(wl, nb, T.vh4, o);       // lap of v_h (x, y, z) and of T'
      st4(T.q4, o + c, rk * lv.x, rk * lv.y, rk * lv.z, Kd * apply7(wl, nb, X.rho + o) * inv_r2);
      T.qT[o + c] = rk * lv.w;
    }
    if (k >= 1 && k < G.nv) {
      int o = k * S;
      R rlo = ld(U.rhob + (k - 1)) + ld(X.rho + (o - S + c)), rhi = ld(U.rhob + (k)) + ld(X.rho + (o + c));
      R rif = HO ? vint_iface(U, X.rho, U.rhob, k, c, S, G.nv) : ld(U.wlo + (k)) * rlo + ld(U.whi + (k)) * rhi;
      T.qvr[o + c] = rif * Kd * apply7(wl, nb, T.vr + o) / ld(U.ri2 + (k));
    } else if (k == 0 || k == G.nv) {
      T.qvr[k * S + c] = 0;
    }
  }
}

// Slow tendencies at the centres (right-hand sides of Eqs. mom2, dens2, pt2):
// S_M = -grad_h p - A_h - C_h + F_M, S_rho = -div(M) - div(W) + F_rho,
// S_th = F_th - div(theta M) - div(theta W), plus Dsc = div(M) + div(W) of the
// stage state (divergence damping), the radial advection+Coriolis and
// Pi = gamma p / rho theta. In the first stage (stage state = X^t) Dsc is also
// kept in d0: it is the divergence D that the first small step of every
// stage damps, since there M^(s) + M* = M^t and W^(s) + W* = W^t.
// SH: the shallow-atmosphere approximation of Sec. 3 (r = A in the tables;
// here the traditional Coriolis, 2 Omega sin(lat) r x M on the horizontal
// momentum only, and the horizontal velocity and w advected without the
// metric terms the approximation drops)
template <typename R, bool SH = false, bool HO = false>
__device__ __forceinline__ void d_slow(const Geo<R>& G, const VR<R>& U, const Phys& ph, const Xf<R>& X, const Work<R>& T, const Slow<R>& SL, int hyper,
                                            R* d0, int kchunk, int bx, int by, int kend) {
  int c = bx * blockDim.x + threadIdx.x;
  if (c >= G.ncol) return;
  const int S = G.colp;
  Nbr7 nb = load_nbr(G, c);
  // the divergence and Laplacian weights; the gradient of p below is taken
  // with the divergence weights plus the centre correction, unprojected
  // (S_M is projected as a whole)
  W7x3<R> wd;
  W7<R> wl;
  load_w7x3_lap(G.wdiv, S, c, wd, wl);
  const R gcx = ld(G.gcor + (c)), gcy = ld(G.gcor + (S + c)), gcz = ld(G.gcor + (2 * S + c));
  R rx = ld(G.rhat + (c)), ry = ld(G.rhat + (S + c)), rz = ld(G.rhat + (2 * S + c));
  const R two_om = pc<R>(ph.two_omega, ph.two_omega_f), gamma = pc<R>(ph.gamma, ph.gamma_f),
          Rd = pc<R>(ph.Rd, ph.Rd_f);
  int k0 = by * kchunk, k1 = min(kend, k0 + kchunk);
  constexpr int kUnroll = sizeof(R) == sizeof(float) ? 2 : 1;   // float64: registers
#pragma unroll kUnroll
  for (int k = k0; k < k1; ++k) {
    const int o = k * S, i = o + c;
    const R inv_r = ld(U.inv_rc + (k)), inv_r2 = ld(U.inv_rc2 + (k));
    const R sql = ld(U.sq_lo + (k)), sqh = ld(U.sq_hi + (k));
    R thfull = ld(U.thb + (k)) + ld(X.th + (i));
    R p = ld(U.pb + (k)) + ld(T.pp + (i));

    // one pass over the 7-point neighbourhood, each neighbour value loaded
    // once: the edge flux f = w . M of the momentum (shared by the continuity,
    // advection and rho-theta divergences), the pressure gradient and the
    // second Laplacians of the hyperdiffusion
    R sa0 = 0, sa1 = 0, sa2 = 0, sa3 = 0, sdh = 0, sdt = 0, gx = 0, gy = 0, gz = 0;
    R hr = 0, hx = 0, hy = 0, hz = 0, hT = 0;
    // advected velocity (packed with theta or T'): the full 3-D one, or (SH)
    // the horizontal one and w
    const R* av4 = SH ? T.vh4 : T.v4;
#pragma unroll
    for (int j = 0; j < 7; ++j) {
      const int q = o + nb.n[j];
      const R f = wd.x[j] * ld(X.mx + q) + wd.y[j] * ld(X.my + q) + wd.z[j] * ld(X.mz + q);
      const Q4<R> av = ld4(av4, (size_t)q);
      sa0 += av.x * f;
      sa1 += av.y * f;
      sa2 += av.z * f;
      if constexpr (SH) sa3 += ld(T.wc + q) * f;
      sdh += f;
      sdt += (SH ? ld(T.theta + q) : av.w) * f;
      const R pq = ld(T.pp + q);
      gx += wd.x[j] * pq;
      gy += wd.y[j] * pq;
      gz += wd.z[j] * pq;
      if (j == 0) {
        gx += gcx * pq;
        gy += gcy * pq;
        gz += gcz * pq;
      }
      if (hyper) {
        const Q4<R> hq = ld4(T.q4, (size_t)q);
        hr += wl.v[j] * hq.w;
        hx += wl.v[j] * hq.x;
        hy += wl.v[j] * hq.y;
        hz += wl.v[j] * hq.z;
        hT += wl.v[j] * ld(T.qT + q);
      }
    }

    // hyperdiffusion (Sec. 4)
    R Frho = 0, FMx = 0, FMy = 0, FMz = 0, Fth = 0;
    if (hyper) {
      Frho = -hr * inv_r2;
      FMx = -hx * inv_r2;
      FMy = -hy * inv_r2;
      FMz = -hz * inv_r2;
      project(rx, ry, rz, FMx, FMy, FMz);
      R Fp = -Rd * hT * inv_r2;
      Fth = thfull / (gamma * p) * Fp;
    }

    // advection div(rho v v_j) of the Cartesian components (Sec. 3)
    const R sa[3] = {sa0, sa1, sa2};
    R A[3];
    R wlo_w = ld(X.w + (i)), whi_w = ld(X.w + (i + S));
    // the advected velocity at the cell's lower and upper interfaces
    Q4<R> vl = {0, 0, 0, 0}, vh = {0, 0, 0, 0};
    if constexpr (HO) {
      if (k >= 1) vl = vint_iface4(U, av4, k, c, S, G.nv);
      if (k + 1 < G.nv) vh = vint_iface4(U, av4, k + 1, c, S, G.nv);
    } else {
      const Q4<R> v0 = ld4(av4, (size_t)i);
      if (k >= 1) {
        const Q4<R> vm = ld4(av4, (size_t)(i - S));
        const R a = ld(U.wlo + (k)), b = ld(U.whi + (k));
        vl = {a * vm.x + b * v0.x, a * vm.y + b * v0.y, a * vm.z + b * v0.z, 0};
      }
      if (k + 1 < G.nv) {
        const Q4<R> vp = ld4(av4, (size_t)(i + S));
        const R a = ld(U.wlo + (k + 1)), b = ld(U.whi + (k + 1));
        vh = {a * v0.x + b * vp.x, a * v0.y + b * vp.y, a * v0.z + b * vp.z, 0};
      }
    }
    const R vlo3[3] = {vl.x, vl.y, vl.z}, vhi3[3] = {vh.x, vh.y, vh.z};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      R ah = sa[j] * inv_r;
      A[j] = ah + sqh * whi_w * vhi3[j] - sql * wlo_w * vlo3[j];
    }
    R acr, ahx, ahy, ahz;
    if constexpr (SH) {
      // traditional Coriolis f r x M_h, f = 2 Omega sin(lat); w advected as a scalar
      const R mx = ld(X.mx + (i)), my = ld(X.my + (i)), mz = ld(X.mz + (i)), f = two_om * rz;
      A[0] += f * (ry * mz - rz * my);
      A[1] += f * (rz * mx - rx * mz);
      A[2] += f * (rx * my - ry * mx);
      R wlo_c = 0, whi_c = 0;
      if constexpr (HO) {
        if (k >= 1) wlo_c = vint_iface(U, (const R*)T.wc, (const R*)nullptr, k, c, S, G.nv);
        if (k + 1 < G.nv) whi_c = vint_iface(U, (const R*)T.wc, (const R*)nullptr, k + 1, c, S, G.nv);
      } else {
        if (k >= 1) wlo_c = ld(U.wlo + (k)) * ld(T.wc + (i - S)) + ld(U.whi + (k)) * ld(T.wc + (i));
        if (k + 1 < G.nv) whi_c = ld(U.wlo + (k + 1)) * ld(T.wc + (i)) + ld(U.whi + (k + 1)) * ld(T.wc + (i + S));
      }
      acr = sa3 * inv_r + sqh * whi_w * whi_c - sql * wlo_w * wlo_c;
      const R d = A[0] * rx + A[1] * ry + A[2] * rz;
      ahx = A[0] - d * rx;
      ahy = A[1] - d * ry;
      ahz = A[2] - d * rz;
    } else {
      // Coriolis 2 Omega z x (rho v) with the full momentum
      R wc = HO ? vint_centre(U, X.w, k, c, S, G.nv) : ld(U.clo + (k)) * wlo_w + ld(U.chi + (k)) * whi_w;
      R mx = ld(X.mx + (i)), my = ld(X.my + (i));
      R fx = mx + wc * rx, fy = my + wc * ry;
      A[0] += -two_om * fy;
      A[1] += two_om * fx;
      acr = A[0] * rx + A[1] * ry + A[2] * rz;
      ahx = A[0] - acr * rx;
      ahy = A[1] - acr * ry;
      ahz = A[2] - acr * rz;
    }

    // the anelastic switch leaves the pressure force to the projection
    const R pgr = ph.anelastic ? R(0) : inv_r;
    R smx = -gx * pgr - ahx + FMx, smy = -gy * pgr - ahy + FMy, smz = -gz * pgr - ahz + FMz;
    project(rx, ry, rz, smx, smy, smz);
    SL.smx[i] = smx;
    SL.smy[i] = smy;
    SL.smz[i] = smz;

    R dh = sdh * inv_r;
    R dv = sqh * whi_w - sql * wlo_w;
    SL.srho[i] = -dh - dv + Frho;
    SL.dsc[i] = dh + dv;
    if (d0) d0[i] = dh + dv;

    R dht = sdt * inv_r;
    R thlo = 0, thhi = 0;
    if (k >= 1) thlo = ld(U.wlo + (k)) * ld(T.theta + (i - S)) + ld(U.whi + (k)) * ld(T.theta + (i));
    if (k + 1 < G.nv) thhi = ld(U.wlo + (k + 1)) * ld(T.theta + (i)) + ld(U.whi + (k + 1)) * ld(T.theta + (i + S));
    R dvt = sqh * thhi * whi_w - sql * thlo * wlo_w;
    SL.sth[i] = Fth - dht - dvt;
    SL.acr[i] = acr;
    SL.pi[i] = gamma * p / thfull;
  }
}

// Slow tendency of the vertical momentum at the interior interfaces
// (right-hand side of Eq. momr2) and theta at the interfaces; with init, on
// the same (column, level) grid, also the perturbations at the start of the
// stage: Phi* = Phi^t - Phi^(s), p* from the nonlinear Eq. theta_to_p.
// XtL (init only): the low parts of a compensated X^t (null pointers when X
// is X^t itself or the state is not compensated); the stage state is stored
// as floats
template <typename R, bool HO = false>
__device__ __forceinline__ void d_slow_w(const Geo<R>& G, const VR<R>& U, const Phys& ph, const Xf<R>& Xt, const Xf<R>& X, const Work<R>& T, const Slow<R>& SL,
                                         const Pert<R>& P, int hyper, int init, int kchunk, int bx, int by,
                                         const Xf<R>& XtL = Xf<R>{}) {
  int c = bx * blockDim.x + threadIdx.x;
  if (c >= G.ncol) return;
  const int S = G.colp;
  Nbr7 nb = load_nbr(G, c);
  W7<R> wl = load_w7(G.wlap, S, c);
  const R g = pc<R>(ph.g, ph.g_f), gamma = pc<R>(ph.gamma, ph.gamma_f);
  int k0 = by * kchunk, k1 = min(G.nv + 1, k0 + kchunk);
#pragma unroll 2
  for (int k = k0; k < k1; ++k) {
    const int i = k * S + c;
    // stage start (unless k_stage_init does it)
    auto dif = [&](const R* a, const R* b, const R* al) {
      R d = ld(a + (i)) - ld(b + (i));
      if (al) d += ld(al + (i));
      return d;
    };
    if (init && k < G.nv) {
      P.rho[i] = dif(Xt.rho, X.rho, XtL.rho);
      st4(P.m4, i, dif(Xt.mx, X.mx, XtL.mx), dif(Xt.my, X.my, XtL.my), dif(Xt.mz, X.mz, XtL.mz),
          ld(T.theta + (i)));
      P.th[i] = dif(Xt.th, X.th, XtL.th);
      const R tht = XtL.th ? ld(Xt.th + (i)) + ld(XtL.th + (i)) : ld(Xt.th + (i));
      R ppt = eos_dev<R>(ld(U.pb + (k)), ld(U.thb + (k)), tht, gamma);
      P.p[i] = ppt - ld(T.pp + (i));
    }
    if (init) P.w[i] = dif(Xt.w, X.w, XtL.w);
    // slow terms of Eq. momr2
    if (k == 0 || k == G.nv) {
      SL.sw[i] = 0;
      SL.thi[i] = 0;
      continue;
    }
    R wlo = ld(U.wlo + (k)), whi = ld(U.whi + (k));
    R sw;
    if (ph.anelastic) {
      // Ogura-Phillips buoyancy g rho0_i (theta' / theta0)_i, theta' / theta0 =
      // Th' / Th_bar at rho = rho_bar, both interpolated linearly
      sw = g * (wlo * ld(U.rhob + (k - 1)) + whi * ld(U.rhob + (k)))
           * (wlo * ld(X.th + (i - S)) / ld(U.thb + (k - 1)) + whi * ld(X.th + (i)) / ld(U.thb + (k)));
    } else {
      sw = ld(U.Rb + (k)) - (ld(T.pp + (i)) - ld(T.pp + (i - S))) * ld(U.inv_dzc + (k))
           - g * (wlo * ld(X.rho + (i - S)) + whi * ld(X.rho + (i)));
    }
    // the vertical advection, Coriolis and diffusion of W are part of the
    // inertia that the hydrostatic switch drops
    if (!ph.hydrostatic) {
      R FW = 0;
      if (hyper) FW = -apply7(wl, nb, T.qvr + k * S) / ld(U.ri2 + (k));
      const R acr_i = HO ? vint_iface(U, (const R*)SL.acr, (const R*)nullptr, k, c, S, G.nv)
                                    : wlo * ld(SL.acr + (i - S)) + whi * ld(SL.acr + (i));
      sw = sw - acr_i + FW;
    }
    SL.sw[i] = sw;
    SL.thi[i] = wlo * ld(T.theta + (i - S)) + whi * ld(T.theta + (i));
  }
}

// The perturbations at the start of a stage on their own (the state's step
// runs this beside the slow terms): Phi* = Phi^t - Phi^(s), p* from the
// nonlinear Eq. theta_to_p; all zero in the first stage, where Phi^(s) =
// Phi^t and p^(s) = EOS(Th^t). M* goes into the packed plane with theta of
// the stage state beside it (the column fluxes gather both). XtL: the low
// parts of a compensated X^t (null pointers: none), XL those of the stage
// state (null: stored as floats), so that Phi^t - Phi^(s) is taken from the
// full values.
template <typename R>
__device__ __forceinline__ void d_stage_init(const Geo<R>& G, const VR<R>& U, const Phys& ph, const Xf<R>& Xt, const Xf<R>& X, const Work<R>& T, const Pert<R>& P,
                                             const Xf<R>& XtL, const Xf<R>& XL, int zero, int kchunk, int bx, int by) {
  int c = bx * blockDim.x + threadIdx.x;
  if (c >= G.ncol) return;
  const int S = G.colp;
  const R gamma = pc<R>(ph.gamma, ph.gamma_f);
  const bool cmp = XtL.rho != nullptr;
  int k0 = by * kchunk, k1 = min(G.nv + 1, k0 + kchunk);
#pragma unroll 2
  for (int k = k0; k < k1; ++k) {
    const int i = k * S + c;
    // Phi^t - Phi^(s) of one field (the stage state of a compensated state
    // is stored as floats, XL null, except in the first stage where it is
    // X^t itself and the perturbations are zero)
    auto dif = [&](const R* a, const R* b, const R* al, const R* bl) {
      R d = ld(a + i) - ld(b + i);
      if (cmp) d += bl ? ld(al + i) - ld(bl + i) : ld(al + i);
      return d;
    };
    if (k < G.nv) {
      if (zero) {
        P.rho[i] = P.th[i] = P.p[i] = R(0);
        st4(P.m4, i, R(0), R(0), R(0), ld(T.theta + (i)));
      } else {
        P.rho[i] = dif(Xt.rho, X.rho, XtL.rho, XL.rho);
        st4(P.m4, i, dif(Xt.mx, X.mx, XtL.mx, XL.mx), dif(Xt.my, X.my, XtL.my, XL.my),
            dif(Xt.mz, X.mz, XtL.mz, XL.mz), ld(T.theta + (i)));
        P.th[i] = dif(Xt.th, X.th, XtL.th, XL.th);
        const R tht = cmp ? ld(Xt.th + (i)) + ld(XtL.th + (i)) : ld(Xt.th + (i));
        R ppt = eos_dev<R>(ld(U.pb + (k)), ld(U.thb + (k)), tht, gamma);
        P.p[i] = ppt - ld(T.pp + (i));
      }
    }
    P.w[i] = zero ? R(0) : dif(Xt.w, X.w, XtL.w, XL.w);
  }
}

// ---------------------------------------------------------------- small step

// L2 eviction priorities of the small step's planes (thor_tune
// THOR_TUNE_L2_HINTS): bit 0 loads the stage constants evict-first, bit 1
// keeps the perturbations and the split's intermediates evict-last. Default
// 3 (both): at glevel 6 x 32 levels the large step takes 1.368 ms, against
// 1.373 with the constants' hint alone and 1.402 without hints. Float64
// states keep their perturbations at the normal priority whatever the mode:
// their set is twice the size, and held evict-last it slowed the float64
// large step from 9.85 to 11.1 ms.
__constant__ int c_l2mode = 3;
__device__ __forceinline__ uint64_t pol_stream() { return l2_policy((c_l2mode & 1) ? kL2First : kL2Normal); }
template <typename R = float>
__device__ __forceinline__ uint64_t pol_keep() {
  return l2_policy(sizeof(R) == sizeof(float) && (c_l2mode & 2) ? kL2Last : kL2Normal);
}
int set_l2_mode(int mode) { return cudaMemcpyToSymbol(c_l2mode, &mode, sizeof mode) == cudaSuccess ? 0 : -1; }

template <typename R>
// Divergence damping, first stencil (Sec. 4, reading R5: the damping is
// -K_d grad_h(lap D)): the Laplacian of the 3-D divergence D of the total
// momentum, D = d0 in the first small step of a stage and later the D the
// previous column step formed; stored packed with the cell's p* (the
// momentum step gathers both)
__device__ __forceinline__ void d_ss_lapd(const Geo<R>& G, const VR<R>& U, const Work<R>& T, const R* dsrc, const R* pstar, int kchunk,
                                          int bx, int by) {
  int c = bx * blockDim.x + threadIdx.x;
  if (c >= G.ncol) return;
  const int S = G.colp;
  const uint64_t pk = pol_keep<R>();
  Nbr7 nb = load_nbr(G, c);
  W7<R> wl = load_w7(G.wlap, S, c);
  int k0 = by * kchunk, k1 = min(G.nv, k0 + kchunk);
#pragma unroll 2
  for (int k = k0; k < k1; ++k) {
    const int o = k * S, i = o + c;
    R l = 0;
#pragma unroll
    for (int j = 0; j < 7; ++j) l += wl.v[j] * ldh(dsrc + (o + nb.n[j]), pk);
    st2h(T.lp, i, l * ld(U.inv_rc2 + (k)), ldh(pstar + (i), pk), pk);
  }
}

// Eq. mom2 with the divergence damping: M* <- proj(M* + dtau(-grad p* + DD + S_M));
// in the last small step of a stage also M^(s+1) = M^(s) + M* into Xo (which
// may be Xs itself: each cell reads its own Xs value before writing it), with
// the low parts XsL -> XoL of a compensated state (null: none)
template <typename R>
__device__ __forceinline__ void d_ss_mom(const Geo<R>& G, const VR<R>& U, const Slow<R>& SL, const Pert<R>& P, const Work<R>& T, R dtau, R Kd,
                                            int divdamp, const Xf<R>& Xs, const Xf<R>& Xo, const Xf<R>& XsL, const Xf<R>& XoL, int last,
                                            int kchunk, int bx, int by) {
  int c = bx * blockDim.x + threadIdx.x;
  if (c >= G.ncol) return;
  const int S = G.colp;
  const uint64_t ps = pol_stream(), pk = pol_keep<R>();
  Nbr7 nb = load_nbr(G, c);
  W7x3<R> wg = load_w7x3(G.wgrad, S, c);
  R rx = ld(G.rhat + (c)), ry = ld(G.rhat + (S + c)), rz = ld(G.rhat + (2 * S + c));
  int k0 = by * kchunk, k1 = min(G.nv, k0 + kchunk);
#pragma unroll 2
  for (int k = k0; k < k1; ++k) {
    const int o = k * S, i = o + c;
    R inv_r = ld(U.inv_rc + (k));
    R ddx = 0, ddy = 0, ddz = 0;
    R gx = 0, gy = 0, gz = 0;
    if (divdamp) {
      // one packed gather per neighbour: the Laplacian of D and p*, both
      // through the (projected) gradient weights
      R ax = 0, ay = 0, az = 0;
#pragma unroll
      for (int j = 0; j < 7; ++j) {
        const Q2<R> q = ld2h(T.lp, (size_t)(o + nb.n[j]), pk);
        ax += wg.x[j] * q.x;
        ay += wg.y[j] * q.x;
        az += wg.z[j] * q.x;
        gx += wg.x[j] * q.y;
        gy += wg.y[j] * q.y;
        gz += wg.z[j] * q.y;
      }
      R s = -Kd * inv_r;
      ddx = s * ax;
      ddy = s * ay;
      ddz = s * az;
    } else {
      grad7(wg, nb, P.p + o, gx, gy, gz);
    }
    const Q4<R> m = ld4h(P.m4, (size_t)i, pk);
    R mx = m.x + dtau * (fmar<R>(-gx, inv_r, ddx) + ldh(SL.smx + (i), ps));
    R my = m.y + dtau * (fmar<R>(-gy, inv_r, ddy) + ldh(SL.smy + (i), ps));
    R mz = m.z + dtau * (fmar<R>(-gz, inv_r, ddz) + ldh(SL.smz + (i), ps));
    project(rx, ry, rz, mx, my, mz);
    st4h(P.m4, i, mx, my, mz, m.w, pk);
    if (last) {          // end of the stage: M^(s+1) = M^(s) + M*
      if (XoL.mx) {
        comp_add<R>(Xs.mx, XsL.mx, Xo.mx, XoL.mx, i, mx);
        comp_add<R>(Xs.my, XsL.my, Xo.my, XoL.my, i, my);
        comp_add<R>(Xs.mz, XsL.mz, Xo.mz, XoL.mz, i, mz);
      } else {
        Xo.mx[i] = ld(Xs.mx + (i)) + mx;
        Xo.my[i] = ld(Xs.my + (i)) + my;
        Xo.mz[i] = ld(Xs.mz + (i)) + mz;
      }
    }
  }
}

// HE-VI column step, part 1: horizontal fluxes of the new M* and, for every
// cell, the parts of Eqs. dens2 and pt2 that do not involve W*:
//   a_k = rho*_k + dtau (S_rho,k - div_h M*_k)
//   b_k = Th*_k + dtau (S_th,k - div_h(theta M*)_k)
//   c_k = p*_k + Pi_k (b_k - Th*_k)        (p* advanced linearly in Th)
template <typename R>
struct FluxCell {
  R dhm, a, b, c;
};
// the four values of cell i = o + column (o = level k's plane offset)
template <typename R>
__device__ __forceinline__ FluxCell<R> flux_cell(const W7x3<R>& wd, const Nbr7& nb, const VR<R>& U,
                                                 const Slow<R>& SL, const Pert<R>& P, const Work<R>& T, R dtau,
                                                 int k, int o, int i, uint64_t ps, uint64_t pk) {
  R dh = 0, dht = 0;
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    const Q4<R> m = ld4h(P.m4, (size_t)(o + nb.n[j]), pk);    // M* and theta of the neighbour
    R f = fmar<R>(wd.z[j], m.z, fmar<R>(wd.y[j], m.y, wd.x[j] * m.x));
    dh += f;
    dht += m.w * f;
  }
  const R inv_r = ld(U.inv_rc + (k));
  const R thk = ldh(P.th + (i), pk);
  const R bk = thk + dtau * (ldh(SL.sth + (i), ps) - dht * inv_r);
  FluxCell<R> r;
  r.dhm = dh * inv_r;
  r.a = ldh(P.rho + (i), pk) + dtau * (ldh(SL.srho + (i), ps) - dh * inv_r);
  r.b = bk;
  r.c = ldh(P.p + (i), pk) + ldh(SL.pi + (i), ps) * (bk - thk);
  return r;
}

template <typename R>
__device__ __forceinline__ void d_ss_flux(const Geo<R>& G, const VR<R>& U, const Slow<R>& SL, const Pert<R>& P, const Work<R>& T, R dtau, int kchunk, int bx, int by) {
  int c = bx * blockDim.x + threadIdx.x;
  if (c >= G.ncol) return;
  const int S = G.colp;
  const uint64_t ps = pol_stream(), pk = pol_keep<R>();
  Nbr7 nb = load_nbr(G, c);
  W7x3<R> wd = load_w7x3(G.wdiv, S, c);
  int k0 = by * kchunk, k1 = min(G.nv, k0 + kchunk);
#pragma unroll 2
  for (int k = k0; k < k1; ++k) {
    const int o = k * S, i = o + c;
    const FluxCell<R> f = flux_cell(wd, nb, U, SL, P, T, dtau, k, o, i, ps, pk);
    sth(T.dhm + i, f.dhm, pk);
    sth(T.ca + i, f.a, pk);
    sth(T.cb + i, f.b, pk);
    sth(T.cc + i, f.c, pk);
  }
}

// one row's factors of a float64 state
template <typename R>
__device__ __forceinline__ void fac_store(const Fac<R>& F, int i, double inv, double cf, double q) {
  F.inv[i] = inv;
  F.cf[i] = cf;
  F.q[i] = q;
}

// HE-VI column step, part 2 (matrix). Substituting Eqs. dens2 and pt2 into
// Eq. momr2 gives at the interior interfaces m = 1..nv-1 (rigid lid: W* = 0
// at m = 0 and nv)
//   lo_m W_m-1 + di_m W_m + up_m W_m+1 = rh_m
// with e_k = r^2/(rc_k^2 dz_k) at the bottom (sq_lo) and top (sq_hi)
// interfaces of cell k, th_m = theta at interface m, w-/w+ the Lagrange
// weights of centres m-1, m at interface m:
//   lo_m = -dtau^2/dzc_m Pi_m-1 sq_lo_m-1 th_m-1 + dtau^2 g w- sq_lo_m-1
//   di_m = 1 + dtau^2/dzc_m th_m (Pi_m sq_lo_m + Pi_m-1 sq_hi_m-1)
//            - dtau^2 g (w- sq_hi_m-1 - w+ sq_lo_m)
//   up_m = -dtau^2/dzc_m Pi_m sq_hi_m th_m+1 - dtau^2 g w+ sq_hi_m
// The matrix depends only on the stage state (Pi, theta) and dtau, so it is
// factorised once per RK stage and the factors serve every small step of
// the stage. The factorisation is the matrix half of a two-sided Thomas
// algorithm, in float64 for float64 states and in double-float (df_rcp,
// df_mul_f: pivot reciprocals to about 2^-46) for float-storage states:
// warp 0 eliminates rows 1..p downwards
// (c'_m = up_m / (di_m - lo_m c'_m-1)), warp 1 rows nv-1..p+1 upwards
// (e'_m = lo_m / (di_m - up_m e'_m+1)); the two warps run on different SM
// sub-partitions. Stored per row: the pivot reciprocal, c' or e', and q = lo
// or up times the pivot reciprocal; per column: 1 / (1 - c'_p e'_p+1) for the
// junction rows p, p+1.
template <typename R>
__device__ __forceinline__ void d_ss_factor(const Geo<R>& G, const VR<R>& U, const Phys& ph, const Slow<R>& SL, const Fac<R>& F,
                                            double dtau, int bx, int by) {
  const int nv = G.nv, S = G.colp, N = nv - 1;
  const int tx = threadIdx.x & 31, half = threadIdx.x >> 5;
  const int c = bx * 32 + tx;
  const bool valid = c < G.ncol;
  const int cs = valid ? c : 0;          // padding lanes compute on column 0 and store nothing
  const int p = N / 2 > 0 ? N / 2 : 1;
  const R g = pc<R>(ph.g, ph.g_f), dt2 = (R)(dtau * dtau), delta = pc<R>(ph.delta, ph.delta_f);
  __shared__ double sj[2][32];
  // the matrix row m in the storage type
  auto coef_r = [&](int m, R& lo, R& di, R& up) {
    const int i = m * S + cs;
    const R pi_lo = ld(SL.pi + (i - S)), pi_hi = ld(SL.pi + i);
    const R wlo = ld(U.wlo + m), whi = ld(U.whi + m), dtz = dt2 * ld(U.inv_dzc + m);
    const R ql = ld(U.sq_lo + (m - 1)), qh = ld(U.sq_hi + (m - 1));   // cell m-1
    const R pl = ld(U.sq_lo + m), ph_ = ld(U.sq_hi + m);              // cell m
    const R th_m = ld(SL.thi + i);
    R lower = 0, upper = 0;
    if (m > 1) lower = (-dtz * pi_lo * ld(SL.thi + (i - S)) + dt2 * g * wlo) * ql;
    if (m < N) upper = (-dtz * pi_hi * ld(SL.thi + (i + S)) - dt2 * g * whi) * ph_;
    lo = lower;
    up = upper;
    di = delta + dtz * th_m * (pi_hi * pl + pi_lo * qh) - dt2 * g * (wlo * qh - whi * pl);
  };
  if constexpr (sizeof(R) == sizeof(float)) {
    // float storage: the factorisation in double-float on the float32 pipes
    // (the float coefficients are exact pairs), stored as pairs
    __shared__ float2 sj2[2][32];
    float2* Finv = reinterpret_cast<float2*>(F.inv);
    float2* Fcf = reinterpret_cast<float2*>(F.cf);
    float2* Fq = reinterpret_cast<float2*>(F.q);
    float2 last = make_float2(0.f, 0.f);
    if (half == 0) {
      for (int m = 1; m <= p; ++m) {
        R lo, di, up;
        coef_r(m, lo, di, up);
        const float2 inv = df_rcp(df_fms(di, 0.f, make_float2(lo, 0.f), last));
        last = df_mul_f(up, inv);
        if (valid) {
          Finv[m * S + c] = inv;
          Fcf[m * S + c] = last;
          Fq[m * S + c] = df_mul_f(lo, inv);
        }
      }
    } else {
      for (int m = N; m > p; --m) {
        R lo, di, up;
        coef_r(m, lo, di, up);
        const float2 inv = df_rcp(df_fms(di, 0.f, make_float2(up, 0.f), last));
        last = df_mul_f(lo, inv);
        if (valid) {
          Finv[m * S + c] = inv;
          Fcf[m * S + c] = last;
          Fq[m * S + c] = df_mul_f(up, inv);
        }
      }
    }
    sj2[half][tx] = last;    // c'_p (warp 0) and e'_p+1 (warp 1)
    __syncthreads();
    if (half == 0 && valid)
      reinterpret_cast<float2*>(F.junction)[c] =
          p < N ? df_rcp(df_fms(1.f, 0.f, sj2[0][tx], sj2[1][tx])) : make_float2(1.f, 0.f);
    return;
  }
  auto coef = [&](int m, double& lo, double& di, double& up) {
    R l, d, u;
    coef_r(m, l, d, u);
    lo = l;
    di = d;
    up = u;
  };
  auto inv_of = [](double den) { return 1.0 / den; };
  double last = 0.0;
  if (half == 0) {
    for (int m = 1; m <= p; ++m) {
      double lo, di, up;
      coef(m, lo, di, up);
      const double inv = inv_of(di - lo * last);
      last = up * inv;
      if (valid) fac_store(F, m * S + c, inv, last, lo * inv);
    }
  } else {
    for (int m = N; m > p; --m) {
      double lo, di, up;
      coef(m, lo, di, up);
      const double inv = inv_of(di - up * last);
      last = lo * inv;
      if (valid) fac_store(F, m * S + c, inv, last, up * inv);
    }
  }
  sj[half][tx] = last;     // c'_p (warp 0) and e'_p+1 (warp 1)
  __syncthreads();
  if (half == 0 && valid) F.junction[c] = p < N ? 1.0 / (1.0 - sj[0][tx] * sj[1][tx]) : 1.0;
}

// End of an RK stage for one cell of the column step: Phi^(s+1) = Phi^(s) +
// Phi* for rho, rho theta and W (the momentum in k_ss_mom), into Xo, which may
// be Xs itself (each cell reads its own Xs values before writing them). The
// lid and surface interfaces keep W^(s) + W*, as the interior ones.
// XsL, XoL: the low parts of a compensated state (null: none), updated
// with comp_add so that the stage end does not round the state.
template <typename R>
__device__ __forceinline__ void stage_end_cell(const Xf<R>& Xs, const Xf<R>& Xo, const Xf<R>& XsL, const Xf<R>& XoL,
                                               const Pert<R>& P, R rho_new, R th_new, R w_new, int k, int i, int S,
                                               int nv) {
  if (XoL.rho) {
    comp_add<R>(Xs.rho, XsL.rho, Xo.rho, XoL.rho, i, rho_new);
    comp_add<R>(Xs.th, XsL.th, Xo.th, XoL.th, i, th_new);
    if (k >= 1) comp_add<R>(Xs.w, XsL.w, Xo.w, XoL.w, i, w_new);
    if (k == 0) comp_add<R>(Xs.w, XsL.w, Xo.w, XoL.w, i, ld(P.w + i));
    if (k == nv - 1) comp_add<R>(Xs.w, XsL.w, Xo.w, XoL.w, i + S, ld(P.w + (i + S)));
    return;
  }
  Xo.rho[i] = ld(Xs.rho + i) + rho_new;
  Xo.th[i] = ld(Xs.th + i) + th_new;
  if (k >= 1) Xo.w[i] = ld(Xs.w + i) + w_new;
  if (k == 0) Xo.w[i] = ld(Xs.w + i) + ld(P.w + i);
  if (k == nv - 1) Xo.w[i + S] = ld(Xs.w + (i + S)) + ld(P.w + (i + S));
}

// the solved W* of row o of the direct solve's shared array: a float64
// value, or for float storage the float in the first word of the row
template <typename R>
__device__ __forceinline__ R solved_w(const double* sdp, int o) {
  if constexpr (sizeof(R) == sizeof(double))
    return sdp[o];
  else
    return reinterpret_cast<const float2*>(sdp)[o].x;
}

// HE-VI column step, part 3 (every small step). The right-hand side
//   rh_m = W*_m + dtau S_W,m - dtau/dzc_m (c_m - c_m-1) - dtau g (w- a_m-1 + w+ a_m)
// goes through the stored factors (d'_m = rh_m / piv_m - q_m d'_m-1
// downwards, f'_m = rh_m / piv_m - q_m f'_m+1 upwards: one dependent
// multiply-add per row, the product rh_m / piv_m off the chain; then the
// junction rows x_p = (d'_p - c'_p f'_p+1) / (1 - c'_p e'_p+1),
// x_p+1 = f'_p+1 - e'_p+1 x_p, then back substitution outwards), in float64
// for float64 states and in double-float for float-storage states; then
// rho* and Th* follow from Eqs. dens2 and pt2 and p* from the nonlinear Eq.
// theta_to_p. One block = 32 columns x 2 warps.
template <typename R>
__device__ __forceinline__ void d_ss_solve(const Geo<R>& G, const VR<R>& U, const Phys& ph, const Xf<R>& Xs, const Slow<R>& SL,
                                            const Pert<R>& P, const Work<R>& T, const Fac<R>& F, double dtau,
                                            int want_div, const Xf<R>& Xo, const Xf<R>& XsL, const Xf<R>& XoL, int last, int bx,
                                            int by) {
  extern __shared__ double sm[];
  const int nv = G.nv, S = G.colp, N = nv - 1;
  const int tx = threadIdx.x & 31, half = threadIdx.x >> 5;
  const int c = bx * 32 + tx;
  const bool valid = c < G.ncol;
  const int cs = valid ? c : 0;          // padding lanes read column 0 and store nothing
  double* sdp = sm;                      // [nv + 1][32] d' / f', then W
  double* sx = sdp + (nv + 1) * 32;      // [2][32] junction values
  double* scf = sx + 64;                 // [nv + 1][32] c' / e', fetched during the sweeps
  const int p = N / 2 > 0 ? N / 2 : 1;
  const R rdt = (R)dtau, g = pc<R>(ph.g, ph.g_f), delta = pc<R>(ph.delta, ph.delta_f);

  auto rhs_r = [&](int m) {
    const int i = m * S + cs;
    const R wlo = ld(U.wlo + m), whi = ld(U.whi + m);
    return delta * ld(P.w + i) + rdt * ld(SL.sw + i) - rdt * ld(U.inv_dzc + m) * (ld(T.cc + i) - ld(T.cc + (i - S)))
           - rdt * g * (wlo * ld(T.ca + (i - S)) + whi * ld(T.ca + i));
  };
  if constexpr (sizeof(R) == sizeof(float)) {
    // float storage: the elimination in double-float, the same operations
    // in the same order as the staged solve (solve_sweeps); W* (float) over
    // the first word of each row of sdp
    const float2* Fq = reinterpret_cast<const float2*>(F.q);
    const float2* Finv = reinterpret_cast<const float2*>(F.inv);
    const float2* Fcf = reinterpret_cast<const float2*>(F.cf);
    float2* dp2 = reinterpret_cast<float2*>(sdp);
    float2* sx2 = reinterpret_cast<float2*>(sx);
    float2* cf2 = reinterpret_cast<float2*>(scf);
    if (half == 0) {
      float2 d1 = make_float2(0.f, 0.f);
#pragma unroll 4
      for (int m = 1; m <= p; ++m) {
        const int i = m * S + cs;
        cf2[m * 32 + tx] = Fcf[i];
        d1 = df_sweep(rhs_r(m), Finv[i], Fq[i], d1);
        dp2[m * 32 + tx] = d1;
      }
    } else {
      float2 f1 = make_float2(0.f, 0.f);
#pragma unroll 4
      for (int m = N; m > p; --m) {
        const int i = m * S + cs;
        cf2[m * 32 + tx] = Fcf[i];
        f1 = df_sweep(rhs_r(m), Finv[i], Fq[i], f1);
        dp2[m * 32 + tx] = f1;
      }
    }
    __syncthreads();
    if (half == 0) {
      float2 xp, xq = make_float2(0.f, 0.f);
      if (p < N) {
        const float2 dp_ = dp2[p * 32 + tx], fq = dp2[(p + 1) * 32 + tx];
        xp = df_mul(df_fms(dp_.x, dp_.y, cf2[p * 32 + tx], fq), reinterpret_cast<const float2*>(F.junction)[cs]);
        xq = df_fms(fq.x, fq.y, cf2[(p + 1) * 32 + tx], xp);
      } else {
        xp = dp2[p * 32 + tx];
      }
      sx2[tx] = xp;
      sx2[32 + tx] = xq;
    }
    __syncthreads();
    if (half == 0) {
      float2 x = sx2[tx];
      dp2[p * 32 + tx] = make_float2(df_to_float(x), 0.f);
      for (int m = p - 1; m >= 1; --m) {
        const float2 d = dp2[m * 32 + tx];
        x = df_fms(d.x, d.y, cf2[m * 32 + tx], x);
        dp2[m * 32 + tx] = make_float2(df_to_float(x), 0.f);
      }
      dp2[tx] = make_float2(0.f, 0.f);             // bottom interface
    } else {
      float2 x = sx2[32 + tx];
      if (p < N) dp2[(p + 1) * 32 + tx] = make_float2(df_to_float(x), 0.f);
      for (int m = p + 2; m <= N; ++m) {
        const float2 d = dp2[m * 32 + tx];
        x = df_fms(d.x, d.y, cf2[m * 32 + tx], x);
        dp2[m * 32 + tx] = make_float2(df_to_float(x), 0.f);
      }
      dp2[nv * 32 + tx] = make_float2(0.f, 0.f);    // top interface
    }
  } else {
    // float64 storage: the elimination in float64
    auto rhs = [&](int m) { return (double)rhs_r(m); };
    if (half == 0) {
      double d1 = 0.0;
#pragma unroll 4
      for (int m = 1; m <= p; ++m) {
        const int i = m * S + cs;
        scf[m * 32 + tx] = ld(F.cf + i);
        d1 = fma(-ld(F.q + i), d1, rhs(m) * ld(F.inv + i));
        sdp[m * 32 + tx] = d1;
      }
    } else {
      double f1 = 0.0;
#pragma unroll 4
      for (int m = N; m > p; --m) {
        const int i = m * S + cs;
        scf[m * 32 + tx] = ld(F.cf + i);
        f1 = fma(-ld(F.q + i), f1, rhs(m) * ld(F.inv + i));
        sdp[m * 32 + tx] = f1;
      }
    }
    __syncthreads();
    if (half == 0) {
      double xp, xq = 0.0;
      if (p < N) {
        const double cp_ = scf[p * 32 + tx], eq = scf[(p + 1) * 32 + tx];
        const double dp_ = sdp[p * 32 + tx], fq = sdp[(p + 1) * 32 + tx];
        xp = (dp_ - cp_ * fq) * ld(F.junction + cs);
        xq = fq - eq * xp;
      } else {
        xp = sdp[p * 32 + tx];
      }
      sx[tx] = xp;
      sx[32 + tx] = xq;
    }
    __syncthreads();
    // back substitution, each warp over its own rows
    if (half == 0) {
      double x = sx[tx];
      sdp[p * 32 + tx] = x;
      for (int m = p - 1; m >= 1; --m) {
        x = sdp[m * 32 + tx] - scf[m * 32 + tx] * x;
        sdp[m * 32 + tx] = x;
      }
      sdp[tx] = 0.0;                 // bottom interface
    } else {
      double x = sx[32 + tx];
      if (p < N) sdp[(p + 1) * 32 + tx] = x;
      for (int m = p + 2; m <= N; ++m) {
        x = sdp[m * 32 + tx] - scf[m * 32 + tx] * x;
        sdp[m * 32 + tx] = x;
      }
      sdp[nv * 32 + tx] = 0.0;       // top interface
    }
  }
  __syncthreads();
  // Eqs. dens2, pt2, theta_to_p with the new W*; the two warps share the levels
  if (valid) {
    const R gamma = pc<R>(ph.gamma, ph.gamma_f);
#pragma unroll 4
    for (int k = half; k < nv; k += 2) {
      const int i = k * S + c;
      const R wl = solved_w<R>(sdp, k * 32 + tx), wh = solved_w<R>(sdp, (k + 1) * 32 + tx);
      const R thl = k > 0 ? ld(SL.thi + i) : R(0);
      const R thh = k + 1 < nv ? ld(SL.thi + (i + S)) : R(0);
      const R el = ld(U.sq_lo + k), eh = ld(U.sq_hi + k);
      R th_new = ld(T.cb + i) - rdt * (eh * thh * wh - el * thl * wl);
      const R rho_new = ld(T.ca + i) - rdt * (eh * wh - el * wl);
      P.rho[i] = rho_new;
      P.th[i] = th_new;
      // p* = EOS(Th^(s) + Th*) - p^(s) = p^(s) ((1 + Th*/Th^(s))^gamma - 1)
      R ps = ld(U.pb + k) + ld(T.pp + i);
      R ths = ld(U.thb + k) + ld(Xs.th + i);
      P.p[i] = ps * rexpm1<R>(gamma * rlog1p<R>(th_new / ths));
      if (k >= 1) P.w[i] = wl;
      // 3-D divergence of the new total momentum, for the next small step's
      // divergence damping: D^(s) + div_h M* (from k_ss_flux) + div_v W*
      if (want_div) T.dd[i] = ld(SL.dsc + i) + ld(T.dhm + i) + (eh * wh - el * wl);
      if (last) stage_end_cell(Xs, Xo, XsL, XoL, P, rho_new, th_new, wl, k, i, S, nv);
    }
  }
}

// ---------------------------------------------------------------- physics

// Sec. 5 backward-Euler friction (Eq. im_eq_v) and Newtonian relaxation
// (Eq. im_eq_t) with the Sec. 6.1 Held-Suarez or Sec. 6.2 hot-Jupiter
// coefficients; sigma = p / p_s with p_s extrapolated hydrostatically at the
// lowest layer's temperature.
// p_s of every column before the physics update, from its lowest layer
// (one thread per column; the update kernel then works on chunks of levels
// and changes the lowest layer's rho theta)
template <typename R>
__device__ __forceinline__ void d_surface_p(const Geo<R>& G, const VR<R>& U, const Phys& ph, const Xf<R>& X, const Work<R>& T, int bx) {
  int c = bx * blockDim.x + threadIdx.x;
  if (c >= G.ncol) return;
  const R gamma = pc<R>(ph.gamma, ph.gamma_f), Rd = pc<R>(ph.Rd, ph.Rd_f);
  R p0 = ld(U.pb + (0)) + eos_dev<R>(ld(U.pb + (0)), ld(U.thb + (0)), ld(X.th + (c)), gamma);
  R T0 = p0 / ((ld(U.rhob + (0)) + ld(X.rho + (c))) * Rd);
  T.psurf[c] = p0 * rexp<R>(pc<R>(ph.g, ph.g_f) * ld(U.zc + (0)) / (Rd * T0));
}

// XL: the low parts of a compensated state (null: none); there the friction
// and the relaxation enter as increments of the state's pairs, the same
// update written as M (1/(1 + K_v dt) - 1) and rho theta at fixed rho
// scaled by (T_new / T)^(1/gamma).
template <typename R>
__device__ __forceinline__ void d_physics(const Geo<R>& G, const VR<R>& U, const Phys& ph, const Xf<R>& X, const Xf<R>& XL, const Work<R>& T, int forcing,
                                          double dt, double hj_dT, int kchunk, int bx, int by) {
  int c = bx * blockDim.x + threadIdx.x;
  if (c >= G.ncol) return;
  const int S = G.colp;
  const R gamma = pc<R>(ph.gamma, ph.gamma_f), inv_gamma = pc<R>(ph.inv_gamma, ph.inv_gamma_f),
          Rd = pc<R>(ph.Rd, ph.Rd_f), kappa = pc<R>(ph.kappa, ph.kappa_f);
  R sl = ld(G.sinlat + (c)), cl = ld(G.coslat + (c)), clcl = ld(G.xdir + (c));
  const R ps = ld(T.psurf + (c));
  const R rdt = (R)dt;
  const int k0 = by * kchunk, k1 = min(G.nv, k0 + kchunk);
  const bool cmp = XL.rho != nullptr;
  for (int k = k0; k < k1; ++k) {
    const int i = k * S + c;
    R rhop = cmp ? ld(X.rho + (i)) + ld(XL.rho + (i)) : ld(X.rho + (i));
    const R thp = cmp ? ld(X.th + (i)) + ld(XL.th + (i)) : ld(X.th + (i));
    R rho = ld(U.rhob + (k)) + rhop;
    R p = ld(U.pb + (k)) + eos_dev<R>(ld(U.pb + (k)), ld(U.thb + (k)), thp, gamma);
    R Temp = p / (rho * Rd);
    R sigma = p / ps;
    R Kv, KT, Teq;
    if (forcing == THOR_FORCING_HELD_SUAREZ) {
      const R day = R(86400.0);
      const R kf = R(1) / day, ka = R(1) / (R(40) * day), ks = R(1) / (R(4) * day);
      const R sb = R(0.7), p00 = R(1.0e5);
      R ramp = (sigma - sb) / (R(1) - sb);
      ramp = ramp > R(0) ? ramp : R(0);
      Kv = kf * ramp;
      R c2 = cl * cl;
      KT = ka + (ks - ka) * ramp * c2 * c2;
      R pr = p / p00;
      Teq = (R(315) - R(60) * sl * sl - R(10) * rlog<R>(pr) * c2) * rpow<R>(pr, kappa);
      Teq = Teq > R(200) ? Teq : R(200);
    } else {
      const R ss = R(0.12), zs = R(2.0e6), Ts = R(1600), Gt = R(2.0e-4), dTs = R(10);
      R z = ld(U.zc + (k));
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
      Teq = Tv + bt * (R)hj_dT * clcl;
    }
    // no friction (K_v = 0: above sigma_b, and everywhere on the hot Jupiter)
    // leaves the momentum as it is, so it is neither read nor written there
    if (cmp) {
      if (Kv != R(0)) {
        const R dfr = -Kv * rdt / (R(1) + Kv * rdt);      // 1 / (1 + K_v dt) - 1
        comp_add<R>(X.mx, XL.mx, X.mx, XL.mx, i, (ld(X.mx + i) + ld(XL.mx + i)) * dfr);
        comp_add<R>(X.my, XL.my, X.my, XL.my, i, (ld(X.my + i) + ld(XL.my + i)) * dfr);
        comp_add<R>(X.mz, XL.mz, X.mz, XL.mz, i, (ld(X.mz + i) + ld(XL.mz + i)) * dfr);
      }
      const R dT = KT * rdt * (Teq - Temp) / (R(1) + KT * rdt);
      const R th = ld(U.thb + (k)) + thp;
      comp_add<R>(X.th, XL.th, X.th, XL.th, i, th * rexpm1<R>(rlog1p<R>(dT / Temp) * inv_gamma));
      continue;
    }
    if (Kv != R(0)) {
      R fr = R(1) / (R(1) + Kv * rdt);
      X.mx[i] *= fr;
      X.my[i] *= fr;
      X.mz[i] *= fr;
    }
    R Tn = (Temp + KT * rdt * Teq) / (R(1) + KT * rdt);
    // rho theta at fixed rho: Th/Th_bar = ((rho/rho_bar)(T/T_bar))^(1/gamma)
    R lr = rlog1p<R>(rhop / ld(U.rhob + (k))) + rlog<R>(Tn / ld(U.Tb + (k)));
    X.th[i] = ld(U.thb + (k)) * rexpm1<R>(lr * inv_gamma);
  }
}

// ---------------------------------------------------------------- energy budget and fixer
//
// Sec. 3 (after Eq. pressure): an energy fixer after Williamson (2009) that
// adjusts the internal energy by the same amount at every grid point. Once per
// large step (reading F-1) the global diagnostics are reduced at the start of
// the step (fin0) and after the three RK3 stages (fin1); the fixer raises the
// temperature of every cell by dT = (E_start - E_dyn) / (c_v sum V rho) at
// fixed rho and momentum, before the physics. The budget records, per large
// step, mass, energy and axial angular momentum at both points and dT.

// one thread: dT (0 without the fixer) into fix[0] (float64) and fixf[0]
// (storage type), and the step's budget row if recording
template <typename R>
__global__ void k_energy_prepare(const double* fin0, const double* fin1, double cv, int do_fix, double* fix,
                                 R* fixf, double* budget, int* count, int cap) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double dT = do_fix ? (fin0[1] - fin1[1]) / (cv * fin1[0]) : 0.0;
  fix[0] = dT;
  fixf[0] = (R)dT;
  if (budget) {
    const int n = *count;
    if (n < cap) {
      double* row = budget + (size_t)n * 8;
      row[0] = fin0[0];
      row[1] = fin0[1];
      row[2] = fin0[2];
      row[3] = fin1[0];
      row[4] = fin1[1];
      row[5] = fin1[2];
      row[6] = dT;
      row[7] = 0.0;
      *count = n + 1;
    }
  }
}

// every cell: T -> T + dT at fixed rho, i.e. rho theta (Eq. pressure, in
// deviation form) scaled by (1 + dT / T)^(1 / gamma)
template <typename R>
__global__ void k_energy_fix(Geo<R> G, VR<R> U, Phys ph, Xf<R> X, Xf<R> XL, const R* fixf, int kchunk) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= G.ncol) return;
  const int S = G.colp;
  const R dT = ld(fixf);
  const R gamma = pc<R>(ph.gamma, ph.gamma_f), inv_gamma = pc<R>(ph.inv_gamma, ph.inv_gamma_f),
          inv_Rd = pc<R>(ph.inv_Rd, ph.inv_Rd_f);
  const int k0 = blockIdx.y * kchunk, k1 = min(G.nv, k0 + kchunk);
  for (int k = k0; k < k1; ++k) {
    const int i = k * S + c;
    const bool cmp = XL.rho != nullptr;
    const R thp = cmp ? ld(X.th + i) + ld(XL.th + i) : ld(X.th + i);
    const R rho = ld(U.rhob + k) + (cmp ? ld(X.rho + i) + ld(XL.rho + i) : ld(X.rho + i));
    const R p = ld(U.pb + k) + eos_dev<R>(ld(U.pb + k), ld(U.thb + k), thp, gamma);
    const R Temp = p / rho * inv_Rd;
    const R th = ld(U.thb + k) + thp;
    const R d = th * rexpm1<R>(rlog1p<R>(dT / Temp) * inv_gamma);
    if (cmp)
      comp_add<R>(X.th, XL.th, X.th, XL.th, i, d);
    else
      X.th[i] = thp + d;
  }
}

// ---------------------------------------------------------------- kernels: one state

template <typename R, bool HO>
__global__ void k_derived(Geo<R> G, VR<R> U, Phys ph, Xf<R> X, Work<R> T, int shallow, int kchunk) {
  d_derived<R, HO>(G, U, ph, X, T, shallow, kchunk, blockIdx.x, blockIdx.y);
}
template <typename R, bool HO>
__global__ void k_lap1(Geo<R> G, VR<R> U, Xf<R> X, Work<R> T, R Kd, int kchunk, int klo, int kend) {
  d_lap1<R, HO>(G, U, X, T, Kd, kchunk, blockIdx.x, blockIdx.y + klo, kend);
}
template <typename R, bool SH, bool HO>
__global__ void __launch_bounds__(kMaxBlock, sizeof(R) == sizeof(float) ? 3 : 2)
    k_slow(Geo<R> G, VR<R> U, Phys ph, Xf<R> X, Work<R> T, Slow<R> SL, int hyper, R* d0, int kchunk, int klo,
           int kend) {
  d_slow<R, SH, HO>(G, U, ph, X, T, SL, hyper, d0, kchunk, blockIdx.x, blockIdx.y + klo, kend);
}
template <typename R, bool HO>
__global__ void k_slow_w(Geo<R> G, VR<R> U, Phys ph, Xf<R> Xt, Xf<R> X, Work<R> T, Slow<R> SL, Pert<R> P, int hyper,
                         int init, int kchunk) {
  d_slow_w<R, HO>(G, U, ph, Xt, X, T, SL, P, hyper, init, kchunk, blockIdx.x, blockIdx.y);
}
template <typename R>
__global__ void k_stage_init(Geo<R> G, VR<R> U, Phys ph, Xf<R> Xt, Xf<R> X, Work<R> T, Pert<R> P, Xf<R> XtL,
                             Xf<R> XL, int zero, int kchunk) {
  d_stage_init<R>(G, U, ph, Xt, X, T, P, XtL, XL, zero, kchunk, blockIdx.x, blockIdx.y);
}
// the small-step stencils take a level range [kchunk * klo, khi) (klo in
// chunks), so that the lower and upper levels can run as separate launches
template <typename R>
__global__ void k_ss_lapd(Geo<R> G, VR<R> U, Work<R> T, const R* dsrc, const R* pstar, int kchunk, int klo,
                          int khi) {
  G.nv = khi;
  d_ss_lapd<R>(G, U, T, dsrc, pstar, kchunk, blockIdx.x, blockIdx.y + klo);
}
// LAST: the last small step of a stage (a separate instantiation, so the
// other small steps carry no registers for the stage end)
template <typename R, bool LAST>
__global__ void k_ss_mom(Geo<R> G, VR<R> U, Slow<R> SL, Pert<R> P, Work<R> T, R dtau, R Kd, int divdamp,
                         Xf<R> Xs, Xf<R> Xo, Xf<R> XsL, Xf<R> XoL, int kchunk, int klo, int khi) {
  G.nv = khi;
  d_ss_mom<R>(G, U, SL, P, T, dtau, Kd, divdamp, Xs, Xo, XsL, XoL, LAST ? 1 : 0, kchunk, blockIdx.x,
              blockIdx.y + klo);
}
template <typename R>
__global__ void k_ss_flux(Geo<R> G, VR<R> U, Slow<R> SL, Pert<R> P, Work<R> T, R dtau, int kchunk, int klo,
                          int khi) {
  G.nv = khi;
  d_ss_flux<R>(G, U, SL, P, T, dtau, kchunk, blockIdx.x, blockIdx.y + klo);
}
template <typename R>
__global__ void __launch_bounds__(64) k_ss_factor(Geo<R> G, VR<R> U, Phys ph, Slow<R> SL, Fac<R> F, double dtau) {
  d_ss_factor<R>(G, U, ph, SL, F, dtau, blockIdx.x, 0);
}
template <typename R>
__global__ void __launch_bounds__(64) k_ss_solve(Geo<R> G, VR<R> U, Phys ph, Xf<R> Xs, Slow<R> SL, Pert<R> P,
                                                 Work<R> T, Fac<R> F, double dtau, int want_div, Xf<R> Xo,
                                                 Xf<R> XsL, Xf<R> XoL, int last) {
  d_ss_solve<R>(G, U, ph, Xs, SL, P, T, F, dtau, want_div, Xo, XsL, XoL, last, blockIdx.x, 0);
}
template <typename R>
__global__ void k_surface_p(Geo<R> G, VR<R> U, Phys ph, Xf<R> X, Work<R> T) {
  d_surface_p<R>(G, U, ph, X, T, blockIdx.x);
}
template <typename R>
__global__ void k_physics(Geo<R> G, VR<R> U, Phys ph, Xf<R> X, Xf<R> XL, Work<R> T, int forcing, double dt,
                          double hj_dT, int kchunk) {
  d_physics<R>(G, U, ph, X, XL, T, forcing, dt, hj_dT, kchunk, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------- staged column solve (float storage)
//
// The column step of d_ss_solve for 32 columns with eight warps. Thread 0
// stages the planes of the elimination (W*, S_W, c, a, the scaled
// off-diagonals q, pivot reciprocals, c'/e', junction factors) into shared
// memory with one
// cp.async.bulk.tensor per array, and asks the copy engine to prefetch the
// planes of the final updates into L2. Warps 0 and 1 then run the two float64
// sweeps out of shared memory (d' overwrites the pivot reciprocal it has just
// used); afterwards all eight warps share the levels of Eqs. dens2, pt2 and
// theta_to_p, whose loads now hit L2. Same operations in the same order as
// d_ss_solve.

constexpr int kSolveWarps = 8;

// one column group's planes in shared memory (32 columns)
struct SolveSm {
  float *w, *sw, *cc, *ca;        // w: W*, then the solved W*
  double *q, *inv, *cf, *junc;    // inv: the pivot reciprocals, then d' and f'
};
__device__ __forceinline__ SolveSm solve_sm(unsigned char* base, int nv) {
  SolveSm s;
  s.w = reinterpret_cast<float*>(base);             // [nv + 1][32]
  s.sw = s.w + (nv + 1) * 32;                       // [nv + 1][32]
  s.cc = s.sw + (nv + 1) * 32;                      // [nv][32]
  s.ca = s.cc + nv * 32;                            // [nv][32]
  s.q = reinterpret_cast<double*>(s.ca + nv * 32);  // [nv + 1][32]
  s.inv = s.q + (nv + 1) * 32;                      // [nv + 1][32]
  s.cf = s.inv + (nv + 1) * 32;                     // [nv + 1][32]
  s.junc = s.cf + (nv + 1) * 32;                    // [32]
  return s;
}
// bytes of one group's planes (a multiple of 128, so every plane and what
// follows them starts 128-byte aligned)
__host__ __device__ __forceinline__ size_t solve_stage_bytes(int nv) {
  return (size_t)(2 * (nv + 1) + 2 * nv) * 128 + (size_t)(3 * (nv + 1) + 1) * 256;
}
size_t solve_tma_smem_bytes(int nv) { return 128 + solve_stage_bytes(nv) + 2 * 256 + sizeof(uint64_t); }

// thread 0 of the copies: the group's elimination planes into s (completing
// on bar) and the planes of its final updates into L2
__device__ __forceinline__ void solve_issue(const SolveSm& s, const SolveMaps& M, int c0, uint64_t* bar, int nv,
                                            int stage0, int want_div) {
  const uint32_t fi = (nv + 1) * 128, fc = nv * 128, di = (nv + 1) * 256;
  const uint64_t ps = pol_stream(), pk = pol_keep();
  mbar_arrive_expect_tx(bar, 2 * fi + 2 * fc + 3 * di + 256);
  tma_load_2d(s.w, &M.w, c0, 0, bar, pk);
  tma_load_2d(s.sw, &M.sw, c0, 0, bar, ps);
  tma_load_2d(s.cc, &M.cc, c0, 0, bar, pk);
  tma_load_2d(s.ca, &M.ca, c0, 0, bar, pk);
  tma_load_2d(s.q, &M.q, c0, 0, bar, ps);
  tma_load_2d(s.inv, &M.inv, c0, 0, bar, ps);
  tma_load_2d(s.cf, &M.cf, c0, 0, bar, ps);
  tma_load_2d(s.junc, &M.junction, c0, 0, bar, ps);
  tma_prefetch_2d(&M.thi, c0, 0, ps);
  tma_prefetch_2d(&M.cb, c0, 0, pk);
  tma_prefetch_2d(&M.pp, c0, 0, ps);
  tma_prefetch_2d(stage0 ? &M.th_t : &M.th_s, c0, 0, ps);
  if (want_div) {
    tma_prefetch_2d(&M.dsc, c0, 0, ps);
    tma_prefetch_2d(&M.dhm, c0, 0, pk);
  }
}

// the two sweeps of one group, sweep 0 (rows 1..p, downwards) or 1 (rows
// nv-1..p+1, upwards) by one warp each, then the junction rows and the back
// substitution; the solved W* over s.w. The elimination runs in
// double-float on the float32 pipes (the factors arrive as double-float
// pairs). The two warps meet at named barrier 1.
__device__ __forceinline__ void solve_sweeps(const SolveSm& s, float2* sx, const VR<float>& U, float rdt, float g,
                                             float delta, int nv, int tx, int sweep) {
  const int N = nv - 1, p = N / 2 > 0 ? N / 2 : 1;
  auto rhs = [&](int m) {
    const int o = m * 32 + tx;
    const float wlo = ld(U.wlo + m), whi = ld(U.whi + m);
    return delta * s.w[o] + rdt * s.sw[o] - rdt * ld(U.inv_dzc + m) * (s.cc[o] - s.cc[o - 32])
           - rdt * g * (wlo * s.ca[o - 32] + whi * s.ca[o]);
  };
  const float2* q = reinterpret_cast<const float2*>(s.q);
  const float2* cf = reinterpret_cast<const float2*>(s.cf);
  float2* sdp = reinterpret_cast<float2*>(s.inv);      // d' / f' over the pivot reciprocals
  float* s_wf = s.w;
  if (sweep == 0) {
    float2 d1 = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int m = 1; m <= p; ++m) {
      const int o = m * 32 + tx;
      d1 = df_sweep(rhs(m), sdp[o], q[o], d1);
      sdp[o] = d1;
    }
  } else {
    float2 f1 = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int m = N; m > p; --m) {
      const int o = m * 32 + tx;
      f1 = df_sweep(rhs(m), sdp[o], q[o], f1);
      sdp[o] = f1;
    }
  }
  asm volatile("bar.sync 1, 64;" ::: "memory");        // the two sweeps only
  if (sweep == 0) {
    const int op = p * 32 + tx;
    float2 xp, xq = make_float2(0.f, 0.f);
    if (p < N) {
      const float2 dp_ = sdp[op], fq = sdp[op + 32];
      xp = df_mul(df_fms(dp_.x, dp_.y, cf[op], fq), reinterpret_cast<const float2*>(s.junc)[tx]);
      xq = df_fms(fq.x, fq.y, cf[op + 32], xp);
    } else {
      xp = sdp[op];
    }
    sx[tx] = xp;
    sx[32 + tx] = xq;
  }
  asm volatile("bar.sync 1, 64;" ::: "memory");
  if (sweep == 0) {
    float2 x = sx[tx];
    s_wf[p * 32 + tx] = df_to_float(x);
    for (int m = p - 1; m >= 1; --m) {
      const float2 d = sdp[m * 32 + tx];
      x = df_fms(d.x, d.y, cf[m * 32 + tx], x);
      s_wf[m * 32 + tx] = df_to_float(x);
    }
    s_wf[tx] = 0.f;
  } else {
    float2 x = sx[32 + tx];
    if (p < N) s_wf[(p + 1) * 32 + tx] = df_to_float(x);
    for (int m = p + 2; m <= N; ++m) {
      const float2 d = sdp[m * 32 + tx];
      x = df_fms(d.x, d.y, cf[m * 32 + tx], x);
      s_wf[m * 32 + tx] = df_to_float(x);
    }
    s_wf[nv * 32 + tx] = 0.f;
  }
}

// Operands of the final updates (Eqs. dens2, pt2, theta_to_p) of one cell
// that do not depend on the solved W*.
struct UpdOps {
  float thl, thh, cb, ps, ths, dsc, dhm;
};
__device__ __forceinline__ UpdOps upd_load(const Geo<float>& G, const VR<float>& U, const Xf<float>& Xs,
                                           const Slow<float>& SL, const Work<float>& T, int want_div, int k,
                                           int c, uint64_t ps, uint64_t pk) {
  const int nv = G.nv, S = G.colp, i = k * S + c;
  UpdOps o;
  o.thl = k > 0 ? ldh(SL.thi + i, ps) : 0.f;
  o.thh = k + 1 < nv ? ldh(SL.thi + (i + S), ps) : 0.f;
  o.cb = ldh(T.cb + i, pk);
  o.ps = ld(U.pb + k) + ldh(T.pp + i, ps);
  o.ths = ld(U.thb + k) + ldh(Xs.th + i, ps);
  o.dsc = want_div ? ldh(SL.dsc + i, ps) : 0.f;
  o.dhm = want_div ? ldh(T.dhm + i, pk) : 0.f;
  return o;
}

// Eqs. dens2, pt2, theta_to_p of one cell with the solved W* (the same
// operations in the same order as d_ss_solve)
__device__ __forceinline__ void upd_apply(const SolveSm& s, const UpdOps& o, const Geo<float>& G,
                                          const VR<float>& U, const Phys& ph, const Xf<float>& Xs,
                                          const Pert<float>& P, const Work<float>& T, float rdt, int want_div,
                                          const Xf<float>& Xo, const Xf<float>& XsL, const Xf<float>& XoL,
                                          int last, int c, int tx, int k, uint64_t pk) {
  const int nv = G.nv, S = G.colp;
  const int q = k * 32 + tx, i = k * S + c;
  const float* s_wf = s.w;
  const float wl = s_wf[q], wh = s_wf[q + 32];
  const float el = ld(U.sq_lo + k), eh = ld(U.sq_hi + k);
  float th_new = o.cb - rdt * (eh * o.thh * wh - el * o.thl * wl);
  const float rho_new = s.ca[q] - rdt * (eh * wh - el * wl);
  sth(P.rho + i, rho_new, pk);
  sth(P.th + i, th_new, pk);
  sth(P.p + i, o.ps * rexpm1<float>(ph.gamma_f * rlog1p<float>(th_new / o.ths)), pk);
  if (k >= 1) sth(P.w + i, wl, pk);
  if (want_div) sth(T.dd + i, o.dsc + o.dhm + (eh * wh - el * wl), pk);
  if (last) stage_end_cell(Xs, Xo, XsL, XoL, P, rho_new, th_new, wl, k, i, S, nv);
}

// M: the state's descriptors, in kernel-parameter or global memory
__device__ __forceinline__ void d_ss_solve_tma(const Geo<float>& G, const VR<float>& U, const Phys& ph,
                                               const SolveMaps& M, int stage0, const Xf<float>& Xs,
                                               const Slow<float>& SL, const Pert<float>& P, const Work<float>& T,
                                               double dtau, int want_div, const Xf<float>& Xo, const Xf<float>& XsL,
                                               const Xf<float>& XoL, int last, int* err, int bx) {
  extern __shared__ unsigned char smraw[];
  const int nv = G.nv;
  const int tid = threadIdx.x, tx = tid & 31, warp = tid >> 5;
  const int c0 = bx * 32, c = c0 + tx;
  unsigned char* base = smraw + ((128u - (smem_u32(smraw) & 127u)) & 127u);
  const SolveSm s = solve_sm(base, nv);
  float2* sx = reinterpret_cast<float2*>(base + solve_stage_bytes(nv));   // [2][32]
  uint64_t* bar = reinterpret_cast<uint64_t*>(sx + 64);

  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (tid == 0) solve_issue(s, M, c0, bar, nv, stage0, want_div);
  if (!__syncthreads_and(mbar_wait(bar, 0))) {
    if (tid == 0) {                      // flag, give the copies a bounded time to land, leave
      atomicExch(err, 1);
      mbar_wait(bar, 0);
    }
    return;
  }
  const float rdt = (float)dtau, g = ph.g_f;
  if (warp < 2) solve_sweeps(s, sx, U, rdt, g, ph.delta_f, nv, tx, warp);
  __syncthreads();
  if (c >= G.ncol) return;
  // the eight warps share the levels of the final updates
  const uint64_t ps = pol_stream(), pk = pol_keep();
#pragma unroll 4
  for (int k = warp; k < nv; k += kSolveWarps)
    upd_apply(s, upd_load(G, U, Xs, SL, T, want_div, k, c, ps, pk), G, U, ph, Xs, P, T, rdt, want_div, Xo, XsL,
              XoL, last, c, tx, k, pk);
}

__global__ void __launch_bounds__(32 * kSolveWarps)
    k_ss_solve_tma(Geo<float> G, VR<float> U, Phys ph, const __grid_constant__ SolveMaps M, int stage0,
                   Xf<float> Xs, Slow<float> SL, Pert<float> P, Work<float> T, double dtau, int want_div,
                   Xf<float> Xo, Xf<float> XsL, Xf<float> XoL, int last, int* err) {
  d_ss_solve_tma(G, U, ph, M, stage0, Xs, SL, P, T, dtau, want_div, Xo, XsL, XoL, last, err, blockIdx.x);
}

// ---------------------------------------------------------------- kernels: ensemble
//
// One launch covers every member: block b of the launch works on local block
// map[b].y of member map[b].x, whose arrays and constants come from the
// member table. Per-member switches (hyperdiffusion, divergence damping,
// forcing) are uniform over a block. s is the RK stage, j the small step.

// The block's member record is copied to shared memory once, and the device
// functions read its fields from there as they need them (by reference), so
// that the record's pointers do not all occupy registers.
template <typename T>
__device__ __forceinline__ const T& stage_record(const T* src, T* dst) {
  static_assert(sizeof(T) % 4 == 0, "record of whole words");
  const uint32_t* a = reinterpret_cast<const uint32_t*>(src);
  uint32_t* b = reinterpret_cast<uint32_t*>(dst);
  for (int w = threadIdx.x; w < (int)(sizeof(T) / 4); w += blockDim.x) b[w] = a[w];
  __syncthreads();
  return *dst;
}

#define THOR_MEMBER()                                   \
  __shared__ Member<R> a_sm;                            \
  const int2 e = map[blockIdx.x];                       \
  const Member<R>& a = stage_record(M + e.x, &a_sm);    \
  const Xf<R>& Xs = s == 0 ? a.Xt : a.Xst

template <typename R>
__global__ void ke_derived(const Member<R>* __restrict__ M, const int2* __restrict__ map, int s, int kchunk) {
  THOR_MEMBER();
  if (a.ph.vorder > 1)
    d_derived<R, true>(a.G, a.U, a.ph, Xs, a.T, a.shallow, kchunk, e.y, blockIdx.y);
  else
    d_derived<R>(a.G, a.U, a.ph, Xs, a.T, a.shallow, kchunk, e.y, blockIdx.y);
}
template <typename R>
__global__ void ke_lap1(const Member<R>* __restrict__ M, const int2* __restrict__ map, int s, int kchunk) {
  THOR_MEMBER();
  if (a.hyper && a.ph.vorder > 1)
    d_lap1<R, true>(a.G, a.U, Xs, a.T, a.Kd, kchunk, e.y, blockIdx.y, a.G.nv + 1);
  else if (a.hyper)
    d_lap1<R>(a.G, a.U, Xs, a.T, a.Kd, kchunk, e.y, blockIdx.y, a.G.nv + 1);
}
template <typename R>
__global__ void __launch_bounds__(kMaxBlock, 2)
    ke_slow(const Member<R>* __restrict__ M, const int2* __restrict__ map, int s, int kchunk) {
  THOR_MEMBER();
  R* d0 = s == 0 && a.divdamp ? a.T.dd0 : nullptr;
  const bool ho = a.ph.vorder > 1;
  if (a.shallow && ho)
    d_slow<R, true, true>(a.G, a.U, a.ph, Xs, a.T, a.SL, a.hyper, d0, kchunk, e.y, blockIdx.y, a.G.nv);
  else if (a.shallow)
    d_slow<R, true>(a.G, a.U, a.ph, Xs, a.T, a.SL, a.hyper, d0, kchunk, e.y, blockIdx.y, a.G.nv);
  else if (ho)
    d_slow<R, false, true>(a.G, a.U, a.ph, Xs, a.T, a.SL, a.hyper, d0, kchunk, e.y, blockIdx.y, a.G.nv);
  else
    d_slow<R, false>(a.G, a.U, a.ph, Xs, a.T, a.SL, a.hyper, d0, kchunk, e.y, blockIdx.y, a.G.nv);
}
template <typename R>
__global__ void ke_slow_w(const Member<R>* __restrict__ M, const int2* __restrict__ map, int s, int kchunk) {
  THOR_MEMBER();
  const Xf<R> XtL = s == 0 ? Xf<R>{} : a.XtL;      // stage 0: X^(s) is X^t, pair and all
  if (a.ph.vorder > 1)
    d_slow_w<R, true>(a.G, a.U, a.ph, a.Xt, Xs, a.T, a.SL, a.P, a.hyper, 1, kchunk, e.y, blockIdx.y, XtL);
  else
    d_slow_w<R>(a.G, a.U, a.ph, a.Xt, Xs, a.T, a.SL, a.P, a.hyper, 1, kchunk, e.y, blockIdx.y, XtL);
}
template <typename R>
__global__ void __launch_bounds__(64)
    ke_ss_factor(const Member<R>* __restrict__ M, const int2* __restrict__ map, int s) {
  THOR_MEMBER();
  d_ss_factor<R>(a.G, a.U, a.ph, a.SL, a.F, a.dts[s], e.y, 0);
}
template <typename R>
// the small-step stencils over levels [kchunk * klo, khi) (as k_ss_*)
__global__ void ke_ss_lapd(const Member<R>* __restrict__ M, const int2* __restrict__ map, int s, int j,
                           int kchunk, int klo, int khi) {
  THOR_MEMBER();
  Geo<R> G = a.G;
  G.nv = khi;
  if (a.divdamp) d_ss_lapd<R>(G, a.U, a.T, j == 0 ? a.T.dd0 : a.T.dd, a.P.p, kchunk, e.y, blockIdx.y + klo);
}
template <typename R>
__global__ void ke_ss_mom(const Member<R>* __restrict__ M, const int2* __restrict__ map, int s, int j,
                          int kchunk, int klo, int khi) {
  THOR_MEMBER();
  Geo<R> G = a.G;
  G.nv = khi;
  d_ss_mom<R>(G, a.U, a.SL, a.P, a.T, (R)a.dts[s], a.Kd, a.divdamp, Xs, s == 2 ? a.Xt : a.Xst,
              s == 0 ? a.XtL : Xf<R>{}, s == 2 ? a.XtL : Xf<R>{}, j + 1 == a.nsub[s], kchunk, e.y,
              blockIdx.y + klo);
}
template <typename R>
__global__ void ke_ss_flux(const Member<R>* __restrict__ M, const int2* __restrict__ map, int s, int kchunk,
                           int klo, int khi) {
  THOR_MEMBER();
  Geo<R> G = a.G;
  G.nv = khi;
  d_ss_flux<R>(G, a.U, a.SL, a.P, a.T, (R)a.dts[s], kchunk, e.y, blockIdx.y + klo);
}
template <typename R>
__global__ void __launch_bounds__(64)
    ke_ss_solve(const Member<R>* __restrict__ M, const int2* __restrict__ map, int s, int j) {
  THOR_MEMBER();
  const int want_div = a.divdamp && j + 1 < a.nsub[s];
  d_ss_solve<R>(a.G, a.U, a.ph, Xs, a.SL, a.P, a.T, a.F, a.dts[s], want_div, s == 2 ? a.Xt : a.Xst,
                s == 0 ? a.XtL : Xf<R>{}, s == 2 ? a.XtL : Xf<R>{}, j + 1 == a.nsub[s], e.y, 0);
}
__global__ void __launch_bounds__(32 * kSolveWarps)
    ke_ss_solve_tma(const Member<float>* __restrict__ M, const int2* __restrict__ map, int s, int j) {
  const int2 e = map[blockIdx.x];
  const Member<float>& a = M[e.x];
  const Xf<float> Xs = s == 0 ? a.Xt : a.Xst;
  const int want_div = a.divdamp && j + 1 < a.nsub[s];
  d_ss_solve_tma(a.G, a.U, a.ph, *a.smap, s == 0, Xs, a.SL, a.P, a.T, a.dts[s], want_div, s == 2 ? a.Xt : a.Xst,
                 s == 0 ? a.XtL : Xf<float>{}, s == 2 ? a.XtL : Xf<float>{}, j + 1 == a.nsub[s], a.err, e.y);
}
template <typename R>
__global__ void ke_surface_p(const Member<R>* __restrict__ M, const int2* __restrict__ map) {
  const int2 e = map[blockIdx.x];
  const Member<R>& a = M[e.x];
  if (a.forcing) d_surface_p<R>(a.G, a.U, a.ph, a.Xt, a.T, e.y);
}
template <typename R>
__global__ void ke_physics(const Member<R>* __restrict__ M, const int2* __restrict__ map, int kchunk) {
  const int2 e = map[blockIdx.x];
  const Member<R>& a = M[e.x];
  if (a.forcing) d_physics<R>(a.G, a.U, a.ph, a.Xt, a.XtL, a.T, a.forcing, a.dt, a.hj_dT, kchunk, e.y, blockIdx.y);
}
#undef THOR_MEMBER

// ---------------------------------------------------------------- driver

template <typename R>
void Impl<R>::launch_2d(int nplanes, int kchunk, dim3& grid) const {
  grid = dim3((G.ncol + block - 1) / block, (nplanes + kchunk - 1) / kchunk);
}

size_t solve_smem_bytes(int nv) { return (size_t)(2 * (nv + 1) + 2) * 32 * sizeof(double); }

// Raise a kernel's dynamic shared-memory limit to at least bytes, never
// lower it: states with different level counts share the kernels, and a
// later state with fewer levels must not take room from an earlier one.
template <typename K>
static bool raise_smem_limit(K* kernel, int bytes) {
  cudaFuncAttributes a{};
  if (cudaFuncGetAttributes(&a, kernel) != cudaSuccess) return false;
  if (a.maxDynamicSharedSizeBytes >= bytes) return true;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess;
}

template <typename R>
int col_kernel_setup(int nv) {
  const int bytes = (int)solve_smem_bytes(nv);
  return raise_smem_limit(k_ss_solve<R>, bytes) && raise_smem_limit(ke_ss_solve<R>, bytes) ? 0 : -3;
}
template int col_kernel_setup<double>(int);
template int col_kernel_setup<float>(int);

template <typename R>
int Impl<R>::large_step(double dt, int n_small) {
  const int kc = kchunk, bs = block;
  dim3 g2, g2i;
  launch_2d(G.nv, kc, g2);
  launch_2d(G.nv + 1, kc, g2i);
  dim3 g1((G.ncol + bs - 1) / bs);
  dim3 gsolve((G.ncol + 31) / 32);
  const size_t solve_smem = solve_smem_bytes(G.nv);
  const bool staged = solve_tma && smaps != nullptr;
  // level halves of the small-step stencils (THOR_TUNE_LEVEL_SPLIT): levels
  // [0, kc * hc) on the state's stream, [kc * hc, nv) on side2
  const bool lsplit = level_split && side != nullptr && !prof_on && side2 != nullptr && G.nv >= 2 * kc;
  const int nch = (G.nv + kc - 1) / kc, hc = lsplit ? nch / 2 : nch;
  dim3 glo(g2.x, hc), ghi(g2.x, nch - hc);
  auto lapd = [&](cudaStream_t st, const R* dsrc, dim3 g, int klo, int khi) -> cudaError_t {
    return launch_k(k_ss_lapd<R>, g, bs, 0, st, G, U, T, dsrc, (const R*)P.p, kc, klo, khi);
  };
  const R Kd = (R)(diff_D * dbar4 / dt);
  const double dts[3] = {dt / 3.0, dt / n_small, dt / n_small};
  const int nsub[3] = {1, n_small / 2, n_small};
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  // Kernels of a stage that do not depend on each other run on two streams
  // (graph branches when captured): after k_derived the stage's perturbations
  // (k_stage_init) and, from the second stage on, the first small step's
  // gradient of D (of X^t, kept from the first stage) run on the side stream
  // beside the slow terms; after k_slow_w the factorisation runs there beside
  // the first small step's stencils. With per-kernel profiling everything
  // stays on the state's stream, in the same order.
  const bool fork = side != nullptr && !prof_on;
  const int nstages = rk_stages;      // 3, or fewer when a test stops the step early
  const bool energy = (energy_fix || budget_cap > 0) && fixbuf != nullptr && nstages == 3;
  double* fin0 = fixbuf + kDiagBlocks * 8;                       // reduction at the step start
  double* part1 = fixbuf + (kDiagBlocks + 1) * 8;
  double* fin1 = part1 + kDiagBlocks * 8;                        // after the dynamics
  double* fixv = fin1 + 8;
  R* fixf = reinterpret_cast<R*>(fixv + 1);
  if (energy) {
    chk(launch_k(k_diag_partial<R>, kDiagBlocks, kDiagThreads, 0, stream, G, V, ph, Xt, XtL, fixbuf));
    chk(launch_k(k_diag_final, 1, 256, 0, stream, fixbuf, kDiagBlocks));
    launches += 2;
  }
  for (int s = 0; s < nstages; ++s) {
    // the last stage run writes X^(s+1) into the state
    Xf<R> Xs = s == 0 ? Xt : Xst, Xo = s == nstages - 1 ? Xt : Xst;
    // low parts of a compensated state: X^t keeps them; a stage state is
    // stored as floats (the next stage's perturbations start from the stored
    // value, so its rounding cancels at the last stage end, which writes X^t
    // as a pair)
    Xf<R> XsL = s == 0 ? XtL : Xf<R>{}, XoL = s == nstages - 1 ? XtL : Xf<R>{};
    cudaStream_t aux = fork ? side : stream;
    mark(THOR_K_DERIVED, true);
    const bool ho = ph.vorder > 1;
    chk(launch_k(ho ? k_derived<R, true> : k_derived<R, false>, g2i, bs, 0, stream, G, U, ph, Xs, T, shallow, kc));
    mark(THOR_K_DERIVED, false);
    ++launches;
    if (fork) {
      chk(cudaEventRecord(ev_fork, stream));
      chk(cudaStreamWaitEvent(side, ev_fork, 0));
    }
    mark(THOR_K_STAGE_INIT, true);
    chk(launch_k(k_stage_init<R>, g2i, bs, 0, aux, G, U, ph, Xt, Xs, T, P, XtL, XsL, (int)(s == 0), kc));
    mark(THOR_K_STAGE_INIT, false);
    ++launches;
    const bool early_grad = divdamp && s > 0;    // D of X^t is ready before the slow terms
    if (early_grad) {
      mark(THOR_K_SS_LAPD, true);
      chk(lapd(aux, (const R*)T.dd0, g2, 0, G.nv));
      mark(THOR_K_SS_LAPD, false);
      ++launches;
    }
    if (fork) chk(cudaEventRecord(ev_join0, side));
    if (hyper) {
      mark(THOR_K_LAP1, true);
      chk(launch_k(ho ? k_lap1<R, true> : k_lap1<R, false>, g2i, bs, 0, stream, G, U, Xs, T, Kd, kc, 0, G.nv + 1));
      mark(THOR_K_LAP1, false);
      ++launches;
    }
    mark(THOR_K_SLOW, true);
    auto slow = shallow ? (ho ? k_slow<R, true, true> : k_slow<R, true, false>)
                        : (ho ? k_slow<R, false, true> : k_slow<R, false, false>);
    chk(launch_k(slow, g2, bs, 0, stream, G, U, ph, Xs, T, SL, hyper,
                 s == 0 && divdamp ? T.dd0 : (R*)nullptr, kc, 0, G.nv));
    mark(THOR_K_SLOW, false);
    ++launches;
    // the vertical momentum's slow term and the factorisation only gate the
    // first column solve: they run on the side stream beside the first
    // small step's stencils
    if (fork) {
      chk(cudaEventRecord(ev_fork, stream));
      chk(cudaStreamWaitEvent(side, ev_fork, 0));
    }
    mark(THOR_K_SLOW_W, true);
    chk(launch_k(ho ? k_slow_w<R, true> : k_slow_w<R, false>, g2i, bs, 0, aux, G, U, ph, Xt, Xs, T, SL, P, hyper, 0,
                 kc));
    mark(THOR_K_SLOW_W, false);
    mark(THOR_K_SS_FACTOR, true);
    chk(launch_k(k_ss_factor<R>, gsolve, 64, 0, aux, G, U, ph, SL, F, dts[s]));
    mark(THOR_K_SS_FACTOR, false);
    if (fork) {
      chk(cudaEventRecord(ev_join, side));
      chk(cudaStreamWaitEvent(stream, ev_join0, 0));
    }
    launches += 2;
    for (int j = 0; j < nsub[s]; ++j) {
      // the last small step of a stage also ends the stage: X^(s+1) = X^(s) + X*
      const int last = j + 1 == nsub[s];
      // the three horizontal stencils over levels [kc * klo, khi) on st
      auto stencils = [&](cudaStream_t st, dim3 g, int klo, int khi) {
        // D: of X^t in the first small step, then from the previous column step
        if (divdamp && !(j == 0 && early_grad)) {
          mark(THOR_K_SS_LAPD, true);
          chk(lapd(st, (const R*)(j == 0 ? T.dd0 : T.dd), g, klo, khi));
          mark(THOR_K_SS_LAPD, false);
          ++launches;
        }
        mark(THOR_K_SS_MOM, true);
        chk(launch_k(last ? k_ss_mom<R, true> : k_ss_mom<R, false>, g, bs, 0, st, G, U, SL, P, T, (R)dts[s], Kd,
                     divdamp, Xs, Xo, XsL, XoL, kc, klo, khi));
        mark(THOR_K_SS_MOM, false);
        mark(THOR_K_SS_FLUX, true);
        chk(launch_k(k_ss_flux<R>, g, bs, 0, st, G, U, SL, P, T, (R)dts[s], kc, klo, khi));
        mark(THOR_K_SS_FLUX, false);
        launches += 2;
      };
      if (lsplit) {
        chk(cudaEventRecord(ev_s1, stream));
        chk(cudaStreamWaitEvent(side2, ev_s1, 0));
        stencils(stream, glo, 0, kc * hc);
        stencils(side2, ghi, hc, G.nv);
        chk(cudaEventRecord(ev_s2, side2));
        chk(cudaStreamWaitEvent(stream, ev_s2, 0));
      } else {
        stencils(stream, g2, 0, G.nv);
      }
      const int want_div = divdamp && !last;
      if (fork && j == 0) chk(cudaStreamWaitEvent(stream, ev_join, 0));
      mark(THOR_K_SS_SOLVE, true);
      if (staged)
        chk(launch_solve_tma(gsolve, s, Xo, XsL, XoL, dts[s], want_div, last));
      else
        chk(launch_k(k_ss_solve<R>, gsolve, 64, solve_smem, stream, G, U, ph, Xs, SL, P, T, F, dts[s],
                     want_div, Xo, XsL, XoL, last));
      mark(THOR_K_SS_SOLVE, false);
      ++launches;
    }
  }
  if (energy) {
    chk(launch_k(k_diag_partial<R>, kDiagBlocks, kDiagThreads, 0, stream, G, V, ph, Xt, XtL, part1));
    chk(launch_k(k_diag_final, 1, 256, 0, stream, part1, kDiagBlocks));
    chk(launch_k(k_energy_prepare<R>, 1, 32, 0, stream, (const double*)fin0, (const double*)fin1, ph.cv,
                 energy_fix, fixv, fixf, budget_cap > 0 ? budget : (double*)nullptr, budget_count, budget_cap));
    launches += 3;
    if (energy_fix) {
      chk(launch_k(k_energy_fix<R>, g2, bs, 0, stream, G, U, ph, Xt, XtL, (const R*)fixf, kc));
      ++launches;
    }
  }
  if (forcing != 0 && nstages == 3) {
    mark(THOR_K_PHYSICS, true);
    chk(launch_k(k_surface_p<R>, g1, bs, 0, stream, G, U, ph, Xt, T));
    chk(launch_k(k_physics<R>, g2, bs, 0, stream, G, U, ph, Xt, XtL, T, forcing, dt, hj_dT, kc));
    mark(THOR_K_PHYSICS, false);
    launches += 2;
  }
  return e == cudaSuccess && cudaGetLastError() == cudaSuccess ? 0 : -3;
}

template <typename R>
int anelastic_project(Impl<R>& I, double dts, const Xf<R>& Xo, int* iters);   // thor_anelastic.cu

// One large step under the anelastic switch (Sec. 3): the three RK3 stages
// of lengths dt/3, dt/2, dt, each the slow terms at the stage state
// (pressure gradient and gravity replaced by the buoyancy) and one
// projection from X^t (thor_anelastic.cu), then the physics.
template <typename R>
int Impl<R>::anelastic_step(double dt) {
  const int kc = kchunk, bs = block;
  dim3 g2, g2i;
  launch_2d(G.nv, kc, g2);
  launch_2d(G.nv + 1, kc, g2i);
  dim3 g1((G.ncol + bs - 1) / bs);
  const R Kd = (R)(diff_D * dbar4 / dt);
  const double dts[3] = {dt / 3.0, dt / 2.0, dt};
  const bool ho = ph.vorder > 1;
  for (int s = 0; s < 3; ++s) {
    Xf<R> Xs = s == 0 ? Xt : Xst, Xo = s == 2 ? Xt : Xst;
    if (launch_k(ho ? k_derived<R, true> : k_derived<R, false>, g2i, bs, 0, stream, G, U, ph, Xs, T, shallow, kc))
      return -3;
    if (hyper && launch_k(ho ? k_lap1<R, true> : k_lap1<R, false>, g2i, bs, 0, stream, G, U, Xs, T, Kd, kc, 0,
                          G.nv + 1))
      return -3;
    auto slow = shallow ? (ho ? k_slow<R, true, true> : k_slow<R, true, false>)
                        : (ho ? k_slow<R, false, true> : k_slow<R, false, false>);
    if (launch_k(slow, g2, bs, 0, stream, G, U, ph, Xs, T, SL, hyper, (R*)nullptr, kc, 0, G.nv) ||
        launch_k(ho ? k_slow_w<R, true> : k_slow_w<R, false>, g2i, bs, 0, stream, G, U, ph, Xt, Xs, T, SL, P,
                 hyper, 0, kc))
      return -3;
    launches += 3 + (hyper ? 1 : 0);
    int it = 0;
    const int rc = anelastic_project(*this, dts[s], Xo, &it);
    an_last_iters = it;
    if (rc) return rc;
  }
  if (forcing != 0) {
    if (launch_k(k_surface_p<R>, g1, bs, 0, stream, G, U, ph, Xt, T) ||
        launch_k(k_physics<R>, g2, bs, 0, stream, G, U, ph, Xt, XtL, T, forcing, dt, hj_dT, kc))
      return -3;
    launches += 2;
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}
template int Impl<double>::anelastic_step(double);
template int Impl<float>::anelastic_step(double);

template <>
cudaError_t Impl<float>::launch_solve_tma(dim3 grid, int stage, const Xf<float>& Xo, const Xf<float>& XsL,
                                          const Xf<float>& XoL, double dtau, int want_div, int last) {
  return launch_k(k_ss_solve_tma, grid, 32 * kSolveWarps, solve_tma_smem_bytes(G.nv), stream, G, U, ph, *smaps,
                  (int)(stage == 0), stage == 0 ? Xt : Xst, SL, P, T, dtau, want_div, Xo, XsL, XoL, last, dev_err);
}
template <>
cudaError_t Impl<double>::launch_solve_tma(dim3, int, const Xf<double>&, const Xf<double>&, const Xf<double>&,
                                           double, int, int) {
  return cudaErrorInvalidValue;
}

// TMA descriptors of the staged solve (float storage only; the float64
// planes would not fit the shared memory of a useful number of blocks)
template <>
int Impl<float>::build_solve_maps() {
  static void* encode_fn = nullptr;
  const size_t smem = solve_tma_smem_bytes(G.nv);
  if (smem > 200 * 1024) return 0;                  // stays on the direct solve
  if (!encode_fn) {
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &encode_fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !encode_fn) {
      encode_fn = nullptr;
      return 0;
    }
  }
  using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  Encode encode = reinterpret_cast<Encode>(encode_fn);
  auto map = std::make_unique<SolveMaps>();
  bool ok = true;
  auto make = [&](CUtensorMap* m, const void* ptr, int planes, bool dbl) {
    const cuuint64_t dims[2] = {(cuuint64_t)G.colp, (cuuint64_t)planes};
    const cuuint64_t strides[1] = {(cuuint64_t)G.colp * (dbl ? 8 : 4)};
    const cuuint32_t box[2] = {32, (cuuint32_t)planes};
    const cuuint32_t es[2] = {1, 1};
    ok = ok && encode(m, dbl ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                      const_cast<void*>(ptr), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  };
  const int nv = G.nv;
  make(&map->w, P.w, nv + 1, false);
  make(&map->sw, SL.sw, nv + 1, false);
  make(&map->thi, SL.thi, nv + 1, false);
  make(&map->cc, T.cc, nv, false);
  make(&map->ca, T.ca, nv, false);
  make(&map->cb, T.cb, nv, false);
  make(&map->pp, T.pp, nv, false);
  make(&map->th_t, Xt.th, nv, false);
  make(&map->th_s, Xst.th, nv, false);
  make(&map->dsc, SL.dsc, nv, false);
  make(&map->dhm, T.dhm, nv, false);
  make(&map->q, F.q, nv + 1, true);
  make(&map->inv, F.inv, nv + 1, true);
  make(&map->cf, F.cf, nv + 1, true);
  make(&map->junction, F.junction, 1, true);
  if (!ok) return 0;
  if (!raise_smem_limit(k_ss_solve_tma, (int)smem) || !raise_smem_limit(ke_ss_solve_tma, (int)smem)) return -3;
  smaps = std::move(map);
  return 0;
}
template <>
int Impl<double>::build_solve_maps() {
  return 0;
}

template void Impl<double>::launch_2d(int, int, dim3&) const;
template void Impl<float>::launch_2d(int, int, dim3&) const;
template int Impl<double>::large_step(double, int);
template int Impl<float>::large_step(double, int);

// One large step of every member of an ensemble, one launch per kernel of
// the sequence above. Members are ordered by decreasing n_small, so the
// members still in their small-step loop at step j of a stage are a prefix
// of the block maps.
template <typename R>
int ensemble_large_step(const EnsPlan<R>& E, cudaStream_t stream, long long* launches) {
  const int kc = E.kchunk, bs = E.block;
  const int yc = (E.nv + kc - 1) / kc, yci = (E.nv + 1 + kc - 1) / kc;
  const size_t solve_smem = solve_smem_bytes(E.nv);
  const Member<R>* M = E.M;
  long long n = 0;
  for (int s = 0; s < 3; ++s) {
    const dim3 g2(E.nblk, yc), g2i(E.nblk, yci);
    ke_derived<R><<<g2i, bs, 0, stream>>>(M, E.map, s, kc);
    if (E.any_hyper) {
      ke_lap1<R><<<g2i, bs, 0, stream>>>(M, E.map, s, kc);
      ++n;
    }
    ke_slow<R><<<g2, bs, 0, stream>>>(M, E.map, s, kc);
    ke_slow_w<R><<<g2i, bs, 0, stream>>>(M, E.map, s, kc);
    ke_ss_factor<R><<<E.nblkc, 64, 0, stream>>>(M, E.mapc, s);
    n += 4;
    for (int j = 0; j < E.maxsub[s]; ++j) {
      const int nb = E.active[s][j], nbc = E.activec[s][j];
      // the stencils over level chunks [c0, c1) on st
      auto stencils = [&](cudaStream_t st, int c0, int c1) {
        const dim3 a2(nb, c1 - c0);
        const int khi = min(E.nv, c1 * kc);
        if (E.any_divdamp) {
          ke_ss_lapd<R><<<a2, bs, 0, st>>>(M, E.map, s, j, kc, c0, khi);
          ++n;
        }
        ke_ss_mom<R><<<a2, bs, 0, st>>>(M, E.map, s, j, kc, c0, khi);
        ke_ss_flux<R><<<a2, bs, 0, st>>>(M, E.map, s, kc, c0, khi);
        n += 2;
      };
      if (E.side2 && yc >= 2) {
        cudaEventRecord(E.ev_a, stream);
        cudaStreamWaitEvent(E.side2, E.ev_a, 0);
        stencils(stream, 0, yc / 2);
        stencils(E.side2, yc / 2, yc);
        cudaEventRecord(E.ev_b, E.side2);
        cudaStreamWaitEvent(stream, E.ev_b, 0);
      } else {
        stencils(stream, 0, yc);
      }
      if constexpr (sizeof(R) == sizeof(float)) {
        if (E.staged)
          ke_ss_solve_tma<<<nbc, 32 * kSolveWarps, solve_tma_smem_bytes(E.nv), stream>>>(M, E.mapc, s, j);
        else
          ke_ss_solve<R><<<nbc, 64, solve_smem, stream>>>(M, E.mapc, s, j);
      } else {
        ke_ss_solve<R><<<nbc, 64, solve_smem, stream>>>(M, E.mapc, s, j);
      }
      ++n;
    }
  }
  if (E.any_forcing) {
    ke_surface_p<R><<<E.nblk, bs, 0, stream>>>(M, E.map);
    ke_physics<R><<<dim3(E.nblk, yc), bs, 0, stream>>>(M, E.map, kc);
    n += 2;
  }
  *launches += n;
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

template int ensemble_large_step<double>(const EnsPlan<double>&, cudaStream_t, long long*);
template int ensemble_large_step<float>(const EnsPlan<float>&, cudaStream_t, long long*);

}  // namespace thor
