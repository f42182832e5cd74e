// Device kernels of the THOR hot path (Mendonca et al. 2016, Sec. 3-5).
//
// Data layout in HBM: every field is a set of planes [level][colp] (colp =
// column count padded to a multiple of 128), so a warp reads 32 consecutive
// columns of one level in one coalesced transaction; interface fields have
// nv+1 planes; the state's Cartesian vectors are three separate scalar
// fields, while intermediates that stencils gather together sit in packed
// [level][colp][4] (or [2]) planes. Columns
// follow the rhombus numbering of the grid, so the six neighbours of an
// interior column sit at offsets +-1, +-n, +-(n+1) in the same plane.
//
// Thermodynamic fields are stored as deviations from a horizontally uniform
// float64 reference column (rho_bar, Th_bar, p_bar = EOS(Th_bar), with the
// reference hydrostatic residual R_bar of the discrete Eq. momr2 kept in
// float64). This is an exact rewrite: with R = double the kernels compute the
// same numbers as the plain equations up to rounding; with R = float the
// large hydrostatic terms never meet in float32.
//
// Operators: per-column float64-derived weights over (self, 6 neighbours),
// divided by the layer radius (horizontal divergence, gradient) or its square
// (Laplacian), Sec. 3 deep atmosphere.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace thor {

constexpr int kBlock = 128;        // columns per block (default; the padding of colp)
constexpr int kMaxBlock = 256;     // largest block of the stencil kernels
constexpr int kMaxNv = 128;        // largest nv the column kernel supports

// Vertical grid and reference column (float64, device global memory)
struct Vert {
  const double* rc;     // [nv]   r at centres
  const double* ri;     // [nv+1] r at interfaces
  const double* dz;     // [nv]   layer thickness
  const double* dzc;    // [nv+1] centre spacing across interface i (1..nv-1)
  const double* wlo;    // [nv+1] Lagrange weight of centre i-1 at interface i
  const double* whi;    // [nv+1] Lagrange weight of centre i at interface i
  const double* clo;    // [nv]   weight of interface k at centre k
  const double* chi;    // [nv]   weight of interface k+1 at centre k
  const double* zc;     // [nv]
  const double* rhob;   // [nv] reference column
  const double* thb;
  const double* pb;
  const double* Tb;
  const double* Rb;     // [nv+1] reference residual -dp_bar/dr - g rho_bar_iface
  const double* sv;     // [nv]   1 / (rc^2 dz): radial divergence factor
  const double* ri2;    // [nv+1] ri^2
  const double* inv_dzc;// [nv+1] 1 / dzc
  const double* sq_lo;  // [nv] ri[k]^2 / (rc^2 dz): weight of the bottom interface in div_v
  const double* sq_hi;  // [nv] ri[k+1]^2 / (rc^2 dz): weight of the top interface
};

// The same vertical quantities in the storage type, with the reciprocals
// precomputed, so no kernel divides by a level constant per cell.
template <typename R>
struct VR {
  const R *inv_rc, *inv_rc2, *sv, *ri2, *wlo, *whi, *clo, *chi, *inv_dzc;
  const R *rhob, *thb, *pb, *Tb, *Rb, *zc;
  const R *sq_lo, *sq_hi;
  // Lagrange interpolation of order k > 1 in the explicit terms (Sec. 2.1):
  // interface m (1..nv-1) from centres ij0[m] + j with weights iw[j][m];
  // centre c from interfaces cj0[c] + j with weights cw[j][c]; j < 4, the
  // weights beyond k zero
  const R *iw, *cw;
  const int *ij0, *cj0;
};

template <typename R>
struct Geo {
  int ncol, colp, nv;
  const int* nbr;       // [6][colp]; slot 5 of a pentagon repeats the column
  const R* wdiv;        // [7][colp][4]: x, y, z and the Laplacian weight of the point
  const R* wgrad;       // [7][colp][4]: x, y, z and the Laplacian weight of the point
  // [3][colp]: wgrad_0 - wdiv_0. The gradient weights are the divergence
  // weights projected on the tangent plane, plus -sum_e l_e n_e / A at the
  // centre point, so grad f = P_h(sum_j wdiv_j f_j + gcor f_0): a kernel
  // that projects its result anyway needs only the divergence weights.
  const R* gcor;
  const R* wlap;        // [7][colp]
  const R* rhat;        // [3][colp]
  const R* sinlat;      // [colp]
  const R* coslat;
  const R* xdir;        // cos(lon) cos(lat) = x of the unit position
  const double* area;   // [colp]
};

struct Phys {
  double Rd, cp, cv, gamma, kappa, g, omega, p_ref;
  double inv_Rd, inv_gamma, two_omega;
  // float copies for the float kernels (a float64 conversion per thread costs
  // an issue slot of the GB300's narrow float64 pipe)
  float Rd_f, inv_Rd_f, gamma_f, inv_gamma_f, kappa_f, g_f, two_omega_f;
  // hydrostatic switch (Sec. 3): delta on the vertical momentum's inertia,
  // 1 for the nonhydrostatic equations, 0 under the hydrostatic approximation
  double delta = 1.0;
  float delta_f = 1.0f;
  int hydrostatic = 0;
  // order k of the vertical interpolation in the explicit terms (1: linear)
  int vorder = 1;
  // anelastic switch (Sec. 3): the slow terms drop the pressure gradient
  // and gravity for the Ogura-Phillips buoyancy; a projection replaces the
  // acoustic small steps
  int anelastic = 0;
};
// the constant in the kernel's storage type
template <typename R> __device__ __forceinline__ R pc(double d, float f);
template <> __device__ __forceinline__ double pc<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float pc<float>(double, float f) { return f; }

// Factors of the per-stage vertical matrix: planes [nv + 1][colp] (rows
// 1..nv-1 used) and one plane for the junction of the two sweeps. Per row:
// the pivot reciprocal, c' (downward sweep) or e' (upward sweep), and q, the
// off-diagonal entry lo (down) or up (up) times the pivot reciprocal. 8
// bytes per entry: float64 values for float64 states, double-float pairs
// (float2) for float-storage states.
template <typename R>
struct Fac {
  double *inv, *cf, *junction, *q;
};

// state in deviation form
template <typename R>
struct Xf {
  R *rho, *mx, *my, *mz, *w, *th;
};

// ------------------------------------------------------------ small helpers

template <typename R> __device__ __forceinline__ R rlog1p(R x);
template <> __device__ __forceinline__ double rlog1p<double>(double x) { return log1p(x); }
template <> __device__ __forceinline__ float rlog1p<float>(float x) { return log1pf(x); }
template <typename R> __device__ __forceinline__ R rexpm1(R x);
template <> __device__ __forceinline__ double rexpm1<double>(double x) { return expm1(x); }
template <> __device__ __forceinline__ float rexpm1<float>(float x) { return expm1f(x); }
template <typename R> __device__ __forceinline__ R rlog(R x);
template <> __device__ __forceinline__ double rlog<double>(double x) { return log(x); }
template <> __device__ __forceinline__ float rlog<float>(float x) { return logf(x); }
template <typename R> __device__ __forceinline__ R rexp(R x);
template <> __device__ __forceinline__ double rexp<double>(double x) { return exp(x); }
template <> __device__ __forceinline__ float rexp<float>(float x) { return expf(x); }
template <typename R> __device__ __forceinline__ R rpow(R x, R y);
template <> __device__ __forceinline__ double rpow<double>(double x, double y) { return pow(x, y); }
template <> __device__ __forceinline__ float rpow<float>(float x, float y) { return powf(x, y); }
template <typename R> __device__ __forceinline__ R rsqrt_(R x);
template <> __device__ __forceinline__ double rsqrt_<double>(double x) { return sqrt(x); }
template <> __device__ __forceinline__ float rsqrt_<float>(float x) { return sqrtf(x); }

// a b + c with one rounding, written out where a sum of two products could
// otherwise be contracted either way (kernels that must agree bit for bit
// then contract alike)
template <typename R> __device__ __forceinline__ R fmar(R a, R b, R c);
template <> __device__ __forceinline__ double fmar<double>(double a, double b, double c) { return fma(a, b, c); }
template <> __device__ __forceinline__ float fmar<float>(float a, float b, float c) { return fmaf(a, b, c); }

// Knuth's TwoSum: s = fl(a + b) and the rounding error e, so that s + e equals
// a + b exactly (no multiplication, so no contraction into an FMA can touch
// it). The compensated state keeps every prognostic field as such a pair.
template <typename R>
__device__ __forceinline__ void two_sum(R a, R b, R& s, R& e) {
  s = a + b;
  const R bv = s - a;
  e = (a - (s - bv)) + (b - bv);
}

// Compensated state update hi/lo += d at element i: the new value
// hi + (lo + d) is split into its float and the float remainder, so the
// state's own rounding is not repeated at every update (only d + lo rounds).
// out_hi / out_lo may be hi / lo themselves (each element is read first).
// A null lo is a zero low part (a stage state stored as floats).
template <typename R>
__device__ __forceinline__ void comp_add(const R* hi, const R* lo, R* out_hi, R* out_lo, size_t i, R d) {
  R s, e;
  two_sum(hi[i], lo ? lo[i] + d : d, s, e);
  out_hi[i] = s;
  out_lo[i] = e;
}

// Eq. pressure in deviation form: EOS(Th_bar (1 + x)) - EOS(Th_bar) with
// x = th'/Th_bar, i.e. p_bar ((1 + x)^gamma - 1)
template <typename R>
__device__ __forceinline__ R eos_dev(R pbar, R thbar, R thp, R gamma) {
  return pbar * rexpm1<R>(gamma * rlog1p<R>(thp / thbar));
}

// Double-float numbers: an unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi) / 2, about 48 significant bits, on the float32 pipes
// (double-double arithmetic of Hida, Li and Bailey 2001, with float words).
// The column elimination of float-storage states runs in this form: its
// row recurrences are chains of dependent operations, and on the GB300 a
// dependent float64 FMA takes 64 cycles per step (a float32 one under 5),
// so a double-float row step (about 18 float32 operations) finishes in
// about a fifth of the time of the float64 one. The error-free parts use
// explicitly rounded intrinsics, which the compiler never contracts into
// FMAs.
//
// (ph + pl) - c x, renormalised: the product's error-free high part by FMA
// (Dekker's TwoProduct), the difference of the high words by Knuth's
// TwoSum, the low words added to the error, then one fast TwoSum
__device__ __forceinline__ float2 df_fms(float ph, float pl, float2 c, float2 x) {
  const float th = __fmul_rn(c.x, x.x);
  const float tl = __fmaf_rn(c.x, x.y, __fmaf_rn(c.y, x.x, __fmaf_rn(c.x, x.x, -th)));
  const float s = __fsub_rn(ph, th);
  const float bb = __fsub_rn(s, ph);
  const float e = __fadd_rn(__fsub_rn(__fsub_rn(ph, __fsub_rn(s, bb)), __fadd_rn(th, bb)), __fsub_rn(pl, tl));
  const float h = __fadd_rn(s, e);
  return make_float2(h, __fsub_rn(e, __fsub_rn(h, s)));
}
// r inv - q d for a float r: the sweep step of the elimination
__device__ __forceinline__ float2 df_sweep(float r, float2 inv, float2 q, float2 d) {
  const float ph = __fmul_rn(r, inv.x);
  const float pl = __fmaf_rn(r, inv.y, __fmaf_rn(r, inv.x, -ph));
  return df_fms(ph, pl, q, d);
}
// a b, renormalised
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  const float h = __fmul_rn(a.x, b.x);
  const float l = __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, __fmaf_rn(a.x, b.x, -h)));
  const float s = __fadd_rn(h, l);
  return make_float2(s, __fsub_rn(l, __fsub_rn(s, h)));
}
// a b for a float a, renormalised
__device__ __forceinline__ float2 df_mul_f(float a, float2 b) {
  const float h = __fmul_rn(a, b.x);
  const float l = __fmaf_rn(a, b.y, __fmaf_rn(a, b.x, -h));
  const float s = __fadd_rn(h, l);
  return make_float2(s, __fsub_rn(l, __fsub_rn(s, h)));
}
// 1 / a: the float reciprocal r of the high word refined by one
// Newton-Raphson step r + r (1 - a r), the residual 1 - a r (about 2^-24)
// formed in double-float; relative error about 2^-46
__device__ __forceinline__ float2 df_rcp(float2 a) {
  const float r = __frcp_rn(a.x);
  const float2 e = df_fms(1.0f, 0.0f, a, make_float2(r, 0.0f));
  const float t = __fmul_rn(r, e.x);
  const float s = __fadd_rn(r, t);
  return make_float2(s, __fsub_rn(t, __fsub_rn(s, r)));
}
// the float nearest to hi + lo (one rounding of the exact sum)
__device__ __forceinline__ float df_to_float(float2 a) { return __fadd_rn(a.x, a.y); }

// read-only load through the non-coherent path: the fields a kernel reads
// are never written by another thread of the same kernel, so the compiler may
// issue these loads early and keep many in flight
template <typename T>
__device__ __forceinline__ T ld(const T* p) { return __ldg(p); }

// L2 eviction priority of single loads and stores (createpolicy with
// .L2::cache_hint). The acoustic small steps of a stage read two kinds of
// planes: stage constants (slow tendencies, Pi, theta, the factors of the
// column matrix), read once per small step, and perturbations and the
// split's intermediates, written by one kernel and read by the next. At
// glevel 6 x 32 levels the two sets together exceed L2; the constants can
// be loaded evict-first and the perturbations kept evict-last, so that the
// second set has the better chance of staying in L2 (the first alone is
// what pays at that size). Hints change where a line lives, never a value.
enum { kL2Normal = 0, kL2First = 1, kL2Last = 2 };
__device__ __forceinline__ uint64_t l2_policy(int prio) {
  uint64_t p;
  if (prio == kL2First)
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  else if (prio == kL2Last)
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  else
    asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// read-only loads (non-coherent path, like ld) with a policy
__device__ __forceinline__ float ldh(const float* p, uint64_t pol) {
  float v;
  asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ double ldh(const double* p, uint64_t pol) {
  double v;
  asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ void sth(float* p, float v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void sth(double* p, double v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v), "l"(pol) : "memory");
}

// Four values of one cell stored together ([level][colp][4] planes), so that
// a stencil gathers them with one 16-byte (float) or two 16-byte (double)
// loads per neighbour instead of four.
template <typename R>
struct Q4 {
  R x, y, z, w;
};
__device__ __forceinline__ Q4<float> ld4(const float* base, size_t cell) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(base) + cell);
  return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ Q4<double> ld4(const double* base, size_t cell) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(base) + 2 * cell);
  const double2 b = __ldg(reinterpret_cast<const double2*>(base) + 2 * cell + 1);
  return {a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ void st4(float* base, size_t cell, float x, float y, float z, float w) {
  reinterpret_cast<float4*>(base)[cell] = make_float4(x, y, z, w);
}
__device__ __forceinline__ void st4(double* base, size_t cell, double x, double y, double z, double w) {
  reinterpret_cast<double2*>(base)[2 * cell] = make_double2(x, y);
  reinterpret_cast<double2*>(base)[2 * cell + 1] = make_double2(z, w);
}
// the same with an L2 policy (l2_policy)
__device__ __forceinline__ Q4<float> ld4h(const float* base, size_t cell, uint64_t pol) {
  Q4<float> v;
  asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
      : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
      : "l"(base + 4 * cell), "l"(pol));
  return v;
}
__device__ __forceinline__ Q4<double> ld4h(const double* base, size_t cell, uint64_t pol) {
  Q4<double> v;
  asm("ld.global.nc.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(v.x), "=d"(v.y) : "l"(base + 4 * cell), "l"(pol));
  asm("ld.global.nc.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(v.z), "=d"(v.w) : "l"(base + 4 * cell + 2), "l"(pol));
  return v;
}
__device__ __forceinline__ void st4h(float* base, size_t cell, float x, float y, float z, float w, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(base + 4 * cell), "f"(x), "f"(y),
               "f"(z), "f"(w), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void st4h(double* base, size_t cell, double x, double y, double z, double w, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;" ::"l"(base + 4 * cell), "d"(x), "d"(y), "l"(pol)
               : "memory");
  asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;" ::"l"(base + 4 * cell + 2), "d"(z), "d"(w),
               "l"(pol)
               : "memory");
}

// two values of one cell stored together ([level][colp][2] planes)
template <typename R>
struct Q2 {
  R x, y;
};
__device__ __forceinline__ Q2<float> ld2(const float* base, size_t cell) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(base) + cell);
  return {v.x, v.y};
}
__device__ __forceinline__ Q2<double> ld2(const double* base, size_t cell) {
  const double2 v = __ldg(reinterpret_cast<const double2*>(base) + cell);
  return {v.x, v.y};
}
__device__ __forceinline__ void st2(float* base, size_t cell, float x, float y) {
  reinterpret_cast<float2*>(base)[cell] = make_float2(x, y);
}
__device__ __forceinline__ void st2(double* base, size_t cell, double x, double y) {
  reinterpret_cast<double2*>(base)[cell] = make_double2(x, y);
}
__device__ __forceinline__ Q2<float> ld2h(const float* base, size_t cell, uint64_t pol) {
  Q2<float> v;
  asm("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(base + 2 * cell), "l"(pol));
  return v;
}
__device__ __forceinline__ Q2<double> ld2h(const double* base, size_t cell, uint64_t pol) {
  Q2<double> v;
  asm("ld.global.nc.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(v.x), "=d"(v.y) : "l"(base + 2 * cell), "l"(pol));
  return v;
}
__device__ __forceinline__ void st2h(float* base, size_t cell, float x, float y, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(base + 2 * cell), "f"(x), "f"(y), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void st2h(double* base, size_t cell, double x, double y, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;" ::"l"(base + 2 * cell), "d"(x), "d"(y), "l"(pol)
               : "memory");
}

struct Nbr7 {
  int n[7];
};

template <typename R>
__device__ __forceinline__ Nbr7 load_nbr(const Geo<R>& G, int c) {
  Nbr7 s;
  s.n[0] = c;
#pragma unroll
  for (int j = 0; j < 6; ++j) s.n[j + 1] = ld(G.nbr + j * G.colp + c);
  return s;
}

template <typename R>
struct W7 {
  R v[7];
};
template <typename R>
struct W7x3 {
  R x[7], y[7], z[7];
};

template <typename R>
__device__ __forceinline__ W7<R> load_w7(const R* w, int colp, int c) {
  W7<R> o;
#pragma unroll
  for (int j = 0; j < 7; ++j) o.v[j] = ld(w + j * colp + c);
  return o;
}
// The 3-vector weights of the seven stencil points of column c, stored
// packed as [7][colp][4] (x, y, z and a fourth value: for the gradient table
// the Laplacian weight of the same point, else 0), so that one 16-byte load
// (two in float64) brings a point's weights.
template <typename R>
__device__ __forceinline__ W7x3<R> load_w7x3(const R* w, int colp, int c) {
  W7x3<R> o;
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    const Q4<R> q = ld4(w, (size_t)j * colp + c);
    o.x[j] = q.x;
    o.y[j] = q.y;
    o.z[j] = q.z;
  }
  return o;
}
// the gradient weights and, from the same loads, the Laplacian weights
template <typename R>
__device__ __forceinline__ void load_w7x3_lap(const R* w, int colp, int c, W7x3<R>& g, W7<R>& l) {
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    const Q4<R> q = ld4(w, (size_t)j * colp + c);
    g.x[j] = q.x;
    g.y[j] = q.y;
    g.z[j] = q.z;
    l.v[j] = q.w;
  }
}

// Order-k Lagrange interpolation (Sec. 2.1) of column c: the centre field f
// at interface m, or the interface field fi at centre k; with ref (one
// value per level) the full value ref + f is interpolated.
template <typename R>
__device__ __forceinline__ R vint_iface(const VR<R>& U, const R* f, const R* ref, int m, int c, int S, int nv) {
  const int j0 = ld(U.ij0 + m);
  R s = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int q = min(j0 + j, nv - 1);
    const R v = ref ? ld(ref + q) + ld(f + (q * S + c)) : ld(f + (q * S + c));
    s += ld(U.iw + (j * (nv + 1) + m)) * v;
  }
  return s;
}
// vint_iface of the four values of a packed plane (no reference column)
template <typename R>
__device__ __forceinline__ Q4<R> vint_iface4(const VR<R>& U, const R* f4, int m, int c, int S, int nv) {
  const int j0 = ld(U.ij0 + m);
  Q4<R> s = {0, 0, 0, 0};
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int q = min(j0 + j, nv - 1);
    const Q4<R> v = ld4(f4, (size_t)q * S + c);
    const R wj = ld(U.iw + (j * (nv + 1) + m));
    s.x += wj * v.x;
    s.y += wj * v.y;
    s.z += wj * v.z;
    s.w += wj * v.w;
  }
  return s;
}
template <typename R>
__device__ __forceinline__ R vint_centre(const VR<R>& U, const R* fi, int k, int c, int S, int nv) {
  const int j0 = ld(U.cj0 + k);
  R s = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int q = min(j0 + j, nv);
    s += ld(U.cw + (j * nv + k)) * ld(fi + (q * S + c));
  }
  return s;
}

// sum_j w_j f(n_j) on one plane
template <typename R>
__device__ __forceinline__ R apply7(const W7<R>& w, const Nbr7& nb, const R* plane) {
  R s = 0;
#pragma unroll
  for (int j = 0; j < 7; ++j) s += w.v[j] * ld(plane + nb.n[j]);
  return s;
}
// the same for the four values of a packed plane at level offset o (each
// sum in the order of apply7)
template <typename R>
__device__ __forceinline__ Q4<R> apply7x4(const W7<R>& w, const Nbr7& nb, const R* packed, int o) {
  Q4<R> s = {0, 0, 0, 0};
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    const Q4<R> v = ld4(packed, (size_t)(o + nb.n[j]));
    s.x += w.v[j] * v.x;
    s.y += w.v[j] * v.y;
    s.z += w.v[j] * v.z;
    s.w += w.v[j] * v.w;
  }
  return s;
}
// sum_j w_j . F(n_j) with F given by three planes
template <typename R>
__device__ __forceinline__ R div7(const W7x3<R>& w, const Nbr7& nb, const R* fx, const R* fy, const R* fz) {
  R s = 0;
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    int q = nb.n[j];
    s += w.x[j] * ld(fx + q) + w.y[j] * ld(fy + q) + w.z[j] * ld(fz + q);
  }
  return s;
}
// sum_j w_j . (a(n_j) F(n_j))
template <typename R>
__device__ __forceinline__ R div7_scaled(const W7x3<R>& w, const Nbr7& nb, const R* a, const R* fx,
                                         const R* fy, const R* fz) {
  R s = 0;
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    int q = nb.n[j];
    R aq = ld(a + q);
    s += aq * (w.x[j] * ld(fx + q) + w.y[j] * ld(fy + q) + w.z[j] * ld(fz + q));
  }
  return s;
}
template <typename R>
__device__ __forceinline__ void grad7(const W7x3<R>& w, const Nbr7& nb, const R* s, R& gx, R& gy, R& gz) {
  gx = gy = gz = 0;
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    R v = ld(s + nb.n[j]);
    gx += w.x[j] * v;
    gy += w.y[j] * v;
    gz += w.z[j] * v;
  }
}
template <typename R>
__device__ __forceinline__ void project(R rx, R ry, R rz, R& x, R& y, R& z) {
  R d = x * rx + y * ry + z * rz;
  x -= d * rx;
  y -= d * ry;
  z -= d * rz;
}

}  // namespace thor

// ------------------------------------------------------------ TMA staging
//
// Thin wrappers over the PTX mbarrier and bulk-tensor instructions. A block
// stages a box of planes into shared memory with cp.async.bulk.tensor; the
// copy engine signals completion on an mbarrier by transaction bytes. Every
// wait is bounded in time, so a copy that never lands ends the kernel with
// an error flag instead of a hang.

constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// makes the initialised barriers visible to the copy engine
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// the one expected arrival, with the byte count the copies will deliver
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// L2 prefetch of a box of a 2-D tensor map (no shared memory, no completion)
__device__ __forceinline__ void tma_prefetch_2d(const void* map, int x, int y) {
  asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global [%0, {%1, %2}];" ::"l"(reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y)
               : "memory");
}
// true once the barrier's phase `parity` has completed; false after limit_ns
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          unsigned long long limit_ns = kWaitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (int i = 0; i < (1 << 26); ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
    __nanosleep(32);
  }
  return false;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// the same two with an L2 policy (thor::l2_policy)
__device__ __forceinline__ void tma_prefetch_2d(const void* map, int x, int y, uint64_t pol) {
  asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.L2::cache_hint [%0, {%1, %2}], %3;" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void tma_load_2d(void* dst, const void* map, int x, int y, uint64_t* bar, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, {%2, "
      "%3}], [%4], %5;" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar)), "l"(pol)
      : "memory");
}
// box of a 2-D tensor map (x = column, y = plane) into shared memory
__device__ __forceinline__ void tma_load_2d(void* dst, const void* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
