// Host-side grid builder (Sec. 2 of Mendonca et al. 2016), float64.
//
// Construction (Sec. 2.1): the icosahedron with two vertices at the poles is
// cut into 10 rhombi of two faces each; every rhombus is refined glevel times
// by recursive edge bisection on an (n+1) x (n+1) lattice (n = 2^glevel), each
// new point being the normalised midpoint of its parent edge. A rhombus owns
// its lattice points 0 <= i, j < n; the points on its two far edges belong to
// the neighbouring rhombi and the two poles are stored last. Lattice triangles
// give the counter-clockwise neighbour rings.
//
// Modified grid (Sec. 2.2): spring dynamics (Eqs. spring_force, spr_vel, dbar)
// with the 12 pentagon centres fixed, then the control-volume vertices are the
// triangle centroids and every centre moves to its control-volume centroid.
// Readings shared with the method's statement: semi-implicit Euler with
// spring constant k, stop when every |v| = |dP/dt| < tol; centroid of a
// spherical polygon = direction of sum_i theta_i (r_i x r_i+1)/|r_i x r_i+1|
// with theta_i the arc angle; spherical triangle areas by the Van Oosterom -
// Strackee formula; edge normals are the great-circle-plane normals of the
// arc C_k -> C_k+1, signed to point away from the cell centre.
//
// Stencils: the operators are linear in the cell values, so each one is
// reduced to per-column weights over the cell and its neighbours:
//   div  (Eqs. int_grid, flx_div, div_gauss),
//   grad (Eq. grad, curvature term included, then Eq. proj_h),
//   lap  (Sec. 4: Eq. grad on every triangle places a gradient at the corner
//         C_k, then Eq. div_gauss of those corner vectors).
#include "grid.h"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace thor {
namespace {

struct V3 {
  double x, y, z;
};
inline V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 operator*(V3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
inline double norm(V3 a) { return std::sqrt(dot(a, a)); }
inline V3 unit(V3 a) { return a * (1.0 / norm(a)); }

double arc(V3 a, V3 b) { return std::atan2(norm(cross(a, b)), dot(a, b)); }

double tri_area(V3 a, V3 b, V3 c) {
  double num = std::fabs(dot(a, cross(b, c)));
  double den = 1.0 + dot(a, b) + dot(b, c) + dot(c, a);
  return 2.0 * std::atan2(num, den);
}

V3 polygon_centroid(const V3* v, int m) {
  V3 acc{0, 0, 0};
  for (int i = 0; i < m; ++i) {
    V3 a = v[i], b = v[(i + 1) % m];
    V3 cr = cross(a, b);
    double s = norm(cr);
    double th = std::atan2(s, dot(a, b));
    acc = acc + cr * (th / s);
  }
  return unit(acc);
}

// outward (away from `inside`) unit normal of the great circle through a, b
V3 arc_normal(V3 a, V3 b, V3 inside) {
  V3 n = unit(cross(a, b));
  return dot(n, inside) > 0 ? n * -1.0 : n;
}

inline V3 getv(const std::vector<double>& a, int i) { return {a[3 * i], a[3 * i + 1], a[3 * i + 2]}; }
inline void setv(std::vector<double>& a, int i, V3 v) {
  a[3 * i] = v.x;
  a[3 * i + 1] = v.y;
  a[3 * i + 2] = v.z;
}

struct Rhombi {
  int n;
  int npole, spole;
  // canonical column of lattice point (i, j) of rhombus r, 0 <= i, j <= n
  int canon(int r, int i, int j) const {
    for (;;) {
      if (i < n && j < n) return r * n * n + j * n + i;
      bool north = r < 5;
      int k = north ? r : r - 5;
      if (i == n) {
        if (north) {            // edge L_k -> U_k+1: south k's i = 0 edge
          r = 5 + k;
          i = 0;
        } else {                // edge S -> L_k+1: south k+1's j = 0 edge, reversed
          if (j == 0) return spole;
          int t = j;
          r = 5 + (k + 1) % 5;
          i = n - t;
          j = 0;
        }
      } else {                  // j == n
        if (north) {            // edge N -> U_k+1: north k+1's i = 0 edge, reversed
          if (i == 0) return npole;
          int t = i;
          r = (k + 1) % 5;
          i = 0;
          j = n - t;
        } else {                // edge U_k+1 -> L_k+1: north k+1's j = 0 edge
          r = (k + 1) % 5;
          j = 0;
        }
      }
    }
  }
};

}  // namespace

int build_grid(int glevel, int nv, double radius, double z_top, const SpringParams& sp,
               bool modified, HostGrid& g) {
  if (glevel < 0 || glevel > 10) return -1;
  const int n = 1 << glevel;
  g.glevel = glevel;
  g.n = n;
  g.nv = nv;
  g.radius = radius;
  g.z_top = z_top;
  const int ncol = 10 * n * n + 2;
  g.ncol = ncol;
  Rhombi rh{n, 10 * n * n, 10 * n * n + 1};

  // icosahedron: north pole, U_k at latitude +atan(1/2) and longitude 72k deg,
  // L_k at latitude -atan(1/2) and longitude 72k + 36 deg, south pole
  const double lat = std::atan(0.5);
  V3 N{0, 0, 1}, S{0, 0, -1}, U[5], L[5];
  for (int k = 0; k < 5; ++k) {
    double lu = 2.0 * M_PI * k / 5.0, ll = lu + M_PI / 5.0;
    U[k] = {std::cos(lat) * std::cos(lu), std::cos(lat) * std::sin(lu), std::sin(lat)};
    L[k] = {std::cos(lat) * std::cos(ll), std::cos(lat) * std::sin(ll), -std::sin(lat)};
  }

  g.P.assign(3 * ncol, 0.0);
  std::vector<V3> lat_pts((n + 1) * (n + 1));
  for (int r = 0; r < 10; ++r) {
    int k = r % 5, k1 = (k + 1) % 5;
    V3 c00, cn0, c0n, cnn;
    if (r < 5) {
      c00 = U[k]; cn0 = L[k]; c0n = N; cnn = U[k1];
    } else {
      c00 = L[k]; cn0 = S; c0n = U[k1]; cnn = L[k1];
    }
    auto at = [&](int i, int j) -> V3& { return lat_pts[j * (n + 1) + i]; };
    at(0, 0) = c00; at(n, 0) = cn0; at(0, n) = c0n; at(n, n) = cnn;
    for (int h = n / 2; h >= 1; h /= 2) {
      for (int j = 0; j <= n; j += h)
        for (int i = 0; i <= n; i += h) {
          bool io = (i / h) % 2, jo = (j / h) % 2;
          if (!io && !jo) continue;
          V3 m;
          if (io && !jo) m = at(i - h, j) + at(i + h, j);
          else if (!io && jo) m = at(i, j - h) + at(i, j + h);
          else m = at(i - h, j - h) + at(i + h, j + h);
          at(i, j) = unit(m);
        }
    }
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) setv(g.P, rh.canon(r, i, j), at(i, j));
  }
  setv(g.P, rh.npole, N);
  setv(g.P, rh.spole, S);

  // triangles, counter-clockwise seen from outside
  g.tri.clear();
  g.tri.reserve(3 * 20 * n * n);
  for (int r = 0; r < 10; ++r)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        int a = rh.canon(r, i, j), b = rh.canon(r, i + 1, j), c = rh.canon(r, i + 1, j + 1),
            d = rh.canon(r, i, j + 1);
        int t[6] = {a, b, c, a, c, d};
        g.tri.insert(g.tri.end(), t, t + 6);
      }
  const int ntri = g.ntri();
  for (int t = 0; t < ntri; ++t) {
    V3 a = getv(g.P, g.tri[3 * t]), b = getv(g.P, g.tri[3 * t + 1]), c = getv(g.P, g.tri[3 * t + 2]);
    if (dot(cross(b - a, c - a), a + b + c) <= 0) return -1;   // orientation invariant
  }

  // neighbour rings from the triangle fans
  std::vector<int> fan_from(6 * ncol, -1), fan_to(6 * ncol, -1), fan_tri(6 * ncol, -1), fan_n(ncol, 0);
  for (int t = 0; t < ntri; ++t)
    for (int v = 0; v < 3; ++v) {
      int a = g.tri[3 * t + v], b = g.tri[3 * t + (v + 1) % 3], c = g.tri[3 * t + (v + 2) % 3];
      int s = fan_n[a]++;
      if (s >= 6) return -1;
      fan_from[6 * a + s] = b;
      fan_to[6 * a + s] = c;
      fan_tri[6 * a + s] = t;
    }
  g.nbr.assign(6 * ncol, -1);
  g.ring_tri.assign(6 * ncol, -1);
  g.nn.assign(ncol, 0);
  for (int c = 0; c < ncol; ++c) {
    int m = fan_n[c];
    if (m != 5 && m != 6) return -1;
    int start = fan_from[6 * c];
    for (int s = 1; s < m; ++s) start = std::min(start, fan_from[6 * c + s]);
    int cur = start;
    for (int k = 0; k < m; ++k) {
      int s = 0;
      while (s < m && fan_from[6 * c + s] != cur) ++s;
      if (s == m) return -1;
      g.nbr[6 * c + k] = cur;
      g.ring_tri[6 * c + k] = fan_tri[6 * c + s];
      cur = fan_to[6 * c + s];
    }
    if (cur != start) return -1;
    g.nn[c] = m;
  }

  // spring dynamics (Sec. 2.2)
  g.spring_iters = 0;
  g.spring_converged = 0;
  if (modified && glevel > 0) {
    const double dbar = sp.beta * 2.0 * M_PI / (10.0 * std::pow(2.0, glevel - 1));
    std::vector<double> vel(3 * ncol, 0.0), Pn(3 * ncol);
    int it = 0;
    while (it < sp.max_iter) {
      double vmax = 0.0;
#pragma omp parallel for schedule(static) reduction(max : vmax)
      for (int c = 0; c < ncol; ++c) {
        V3 p0 = getv(g.P, c);
        if (g.nn[c] == 5) {   // pentagon centres stay fixed
          setv(Pn, c, p0);
          setv(vel, c, V3{0, 0, 0});
          continue;
        }
        V3 f{0, 0, 0};
        for (int k = 0; k < g.nn[c]; ++k) {
          V3 q = getv(g.P, g.nbr[6 * c + k]);
          double d = arc(p0, q);
          V3 t = q - p0 * dot(q, p0);
          f = f + unit(t) * (sp.k * (d - dbar));
        }
        V3 v = getv(vel, c);
        v = v + (f - v * sp.alpha) * sp.dt;
        V3 pn = unit(p0 + v * sp.dt);
        v = v - pn * dot(v, pn);
        setv(Pn, c, pn);
        setv(vel, c, v);
        vmax = std::max(vmax, norm(v));
      }
      g.P.swap(Pn);
      ++it;
      if (sp.tol > 0 && vmax < sp.tol) {
        g.spring_converged = 1;
        break;
      }
    }
    g.spring_iters = it;
  }

  // control-volume vertices at the triangle centroids, then centres to the
  // control-volume centroids (corners fixed)
  g.corner.assign(3 * ntri, 0.0);
  for (int t = 0; t < ntri; ++t) {
    V3 v[3] = {getv(g.P, g.tri[3 * t]), getv(g.P, g.tri[3 * t + 1]), getv(g.P, g.tri[3 * t + 2])};
    setv(g.corner, t, polygon_centroid(v, 3));
  }
  if (modified) {
    std::vector<double> Pm(3 * ncol);
    for (int c = 0; c < ncol; ++c) {
      V3 v[6];
      for (int k = 0; k < g.nn[c]; ++k) v[k] = getv(g.corner, g.ring_tri[6 * c + k]);
      setv(Pm, c, polygon_centroid(v, g.nn[c]));
    }
    g.P.swap(Pm);
  }

  // Eq. int_grid weights per triangle: each vertex weighted by the area of
  // the sub-triangle opposite to it
  std::vector<double> tw(3 * ntri);
  for (int t = 0; t < ntri; ++t) {
    V3 a = getv(g.P, g.tri[3 * t]), b = getv(g.P, g.tri[3 * t + 1]), c = getv(g.P, g.tri[3 * t + 2]);
    V3 C = getv(g.corner, t);
    double wa = tri_area(b, c, C), wb = tri_area(a, c, C), wc = tri_area(a, b, C);
    double s = wa + wb + wc;
    tw[3 * t] = wa / s;
    tw[3 * t + 1] = wb / s;
    tw[3 * t + 2] = wc / s;
  }
  // triangle-gradient coefficients (Sec. 4): grad at C_t = sum_v a[t][v] s_v
  std::vector<double> ta(9 * ntri);
  for (int t = 0; t < ntri; ++t) {
    V3 v[3] = {getv(g.P, g.tri[3 * t]), getv(g.P, g.tri[3 * t + 1]), getv(g.P, g.tri[3 * t + 2])};
    double AT = tri_area(v[0], v[1], v[2]);
    V3 ln[3];
    V3 lsum{0, 0, 0};
    for (int e = 0; e < 3; ++e) {   // edge e joins v[e] and v[e+1]
      V3 u = v[e], w = v[(e + 1) % 3], o = v[(e + 2) % 3];
      ln[e] = arc_normal(u, w, o) * arc(u, w);
      lsum = lsum + ln[e];
    }
    for (int q = 0; q < 3; ++q) {
      // vertex q lies on edges q and q-1
      V3 a = (ln[q] + ln[(q + 2) % 3]) * 0.5 - lsum * tw[3 * t + q];
      a = a * (1.0 / AT);
      ta[9 * t + 3 * q] = a.x;
      ta[9 * t + 3 * q + 1] = a.y;
      ta[9 * t + 3 * q + 2] = a.z;
    }
  }

  g.area.assign(ncol, 0.0);
  g.w_div.assign(21 * ncol, 0.0);
  g.w_grad.assign(21 * ncol, 0.0);
  g.w_lap.assign(7 * ncol, 0.0);
  for (int c = 0; c < ncol; ++c) {
    const int m = g.nn[c];
    V3 p0 = getv(g.P, c);
    auto slot = [&](int id) -> int {
      if (id == c) return 0;
      for (int k = 0; k < m; ++k)
        if (g.nbr[6 * c + k] == id) return 1 + k;
      return -1;
    };
    double A = 0.0;
    for (int k = 0; k < m; ++k) {
      V3 ck = getv(g.corner, g.ring_tri[6 * c + k]), ck1 = getv(g.corner, g.ring_tri[6 * c + (k + 1) % m]);
      A += tri_area(p0, ck, ck1);
    }
    g.area[c] = A;
    V3 wd[7], wg[7];
    double wl[7];
    for (int j = 0; j < 7; ++j) {
      wd[j] = wg[j] = V3{0, 0, 0};
      wl[j] = 0.0;
    }
    V3 lnsum{0, 0, 0};
    for (int k = 0; k < m; ++k) {
      int t0 = g.ring_tri[6 * c + k], t1 = g.ring_tri[6 * c + (k + 1) % m];
      V3 ck = getv(g.corner, t0), ck1 = getv(g.corner, t1);
      V3 nk = arc_normal(ck, ck1, p0);
      double lk = arc(ck, ck1);
      V3 coef = nk * (lk / (2.0 * A));
      lnsum = lnsum + nk * lk;
      for (int t : {t0, t1})
        for (int q = 0; q < 3; ++q) {
          int s = slot(g.tri[3 * t + q]);
          if (s < 0) return -1;
          wd[s] = wd[s] + coef * tw[3 * t + q];
          V3 a{ta[9 * t + 3 * q], ta[9 * t + 3 * q + 1], ta[9 * t + 3 * q + 2]};
          wl[s] += dot(coef, a);
        }
    }
    for (int j = 0; j < 7; ++j) wg[j] = wd[j];
    wg[0] = wg[0] - lnsum * (1.0 / A);
    for (int j = 0; j < 7; ++j) {
      wg[j] = wg[j] - p0 * dot(wg[j], p0);     // Eq. proj_h
      g.w_div[21 * c + 3 * j] = wd[j].x;
      g.w_div[21 * c + 3 * j + 1] = wd[j].y;
      g.w_div[21 * c + 3 * j + 2] = wd[j].z;
      g.w_grad[21 * c + 3 * j] = wg[j].x;
      g.w_grad[21 * c + 3 * j + 1] = wg[j].y;
      g.w_grad[21 * c + 3 * j + 2] = wg[j].z;
      g.w_lap[7 * c + j] = wl[j];
    }
  }
  return 0;
}

}  // namespace thor
