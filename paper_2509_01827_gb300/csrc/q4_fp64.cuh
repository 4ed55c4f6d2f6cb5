// q4_fp64.cuh -- FP64 element arithmetic of the ES-FEM Q4 step.
//
// Every expression keeps one fixed IEEE operation order (the translation
// units that include this header are compiled with -fmad=false), so that the
// FP64 mode is reproducible bit for bit:
//   strain at edge point k (Eq. 4 evaluated at the edge midpoints):
//     exx = sum_a dN_a/dx u_a, eyy = sum_a dN_a/dy v_a,
//     gxy = (sum_a dN_a/dy u_a) + (sum_a dN_a/dx v_a), sums in a = 0..3,
//   stress sigma = D eps (plane Cauchy stress),
//   nodal force of local node a (Eq. 6): (sum_k [dN_a/dx sxx + dN_a/dy sxy])*A_p/4.
// On a rectangle hx*hy the derivatives at the edge midpoints are
// numerator/(2h) with numerators in {0, +-1, +-2}; zero terms are skipped,
// which changes nothing but the sign of an exact zero.
#pragma once

#include "cem_internal.h"

namespace cem {

// dN_a/dx numerators (units 1/(2 hx)) and dN_a/dy numerators (units
// 1/(2 hy)) at the midpoint of local edge k.
__host__ __device__ constexpr int dxn(int k, int a) {
  return k == 0 ? (a == 0 ? -2 : a == 1 ? 2 : 0)
       : k == 2 ? (a == 2 ? 2 : a == 3 ? -2 : 0)
       : (a == 0 || a == 3 ? -1 : 1);
}
__host__ __device__ constexpr int dyn(int k, int a) {
  return (k == 0 || k == 2) ? (a < 2 ? -1 : 1)
       : k == 1 ? (a == 1 ? -2 : a == 2 ? 2 : 0)
       : (a == 0 ? -2 : a == 3 ? 2 : 0);
}

// c * x with c = N / (2h): full = fl(1/h), half = full / 2.
template <int N>
__device__ __forceinline__ double cmul(double full, double half, double x) {
  static_assert(N == 2 || N == -2 || N == 1 || N == -1, "nonzero numerator");
  if constexpr (N == 2) return full * x;
  else if constexpr (N == -2) return -(full * x);
  else if constexpr (N == 1) return half * x;
  else return -(half * x);
}

template <int N0, int N1, int N2, int N3>
__device__ __forceinline__ double dot4(double full, double half, double x0, double x1,
                                       double x2, double x3) {
  double acc = 0.0;
  if constexpr (N0 != 0) acc = acc + cmul<N0>(full, half, x0);
  if constexpr (N1 != 0) acc = acc + cmul<N1>(full, half, x1);
  if constexpr (N2 != 0) acc = acc + cmul<N2>(full, half, x2);
  if constexpr (N3 != 0) acc = acc + cmul<N3>(full, half, x3);
  return acc;
}

template <int K>
__device__ __forceinline__ void strain64(const Geo &g, const double u[4], const double v[4],
                                         double e[3]) {
  e[0] = dot4<dxn(K, 0), dxn(K, 1), dxn(K, 2), dxn(K, 3)>(g.rx, g.rxh, u[0], u[1], u[2], u[3]);
  e[1] = dot4<dyn(K, 0), dyn(K, 1), dyn(K, 2), dyn(K, 3)>(g.ry, g.ryh, v[0], v[1], v[2], v[3]);
  double g1 = dot4<dyn(K, 0), dyn(K, 1), dyn(K, 2), dyn(K, 3)>(g.ry, g.ryh, u[0], u[1], u[2], u[3]);
  double g2 = dot4<dxn(K, 0), dxn(K, 1), dxn(K, 2), dxn(K, 3)>(g.rx, g.rxh, v[0], v[1], v[2], v[3]);
  e[2] = g1 + g2;
}

__device__ __forceinline__ void strain64_rt(const Geo &g, int k, const double u[4],
                                            const double v[4], double e[3]) {
  switch (k) {
    case 0: strain64<0>(g, u, v, e); break;
    case 1: strain64<1>(g, u, v, e); break;
    case 2: strain64<2>(g, u, v, e); break;
    default: strain64<3>(g, u, v, e); break;
  }
}

__device__ __forceinline__ void stress64(const Mat &m, const double e[3], double s[3]) {
  s[0] = m.D11 * e[0] + m.D12 * e[1];
  s[1] = m.D12 * e[0] + m.D11 * e[1];
  s[2] = m.D33 * e[2];
}

// fl(cx * a + cy * b) with zero coefficients skipped.
template <int NX, int NY>
__device__ __forceinline__ double term2(const Geo &g, double a, double b) {
  if constexpr (NX == 0) return cmul<NY>(g.ry, g.ryh, b);
  else if constexpr (NY == 0) return cmul<NX>(g.rx, g.rxh, a);
  else return cmul<NX>(g.rx, g.rxh, a) + cmul<NY>(g.ry, g.ryh, b);
}
// fy term: dN/dy * syy + dN/dx * sxy
template <int NX, int NY>
__device__ __forceinline__ double term2y(const Geo &g, double syy, double sxy) {
  if constexpr (NY == 0) return cmul<NX>(g.rx, g.rxh, sxy);
  else if constexpr (NX == 0) return cmul<NY>(g.ry, g.ryh, syy);
  else return cmul<NY>(g.ry, g.ryh, syy) + cmul<NX>(g.rx, g.rxh, sxy);
}

// Nodal force of local node A from the element's (or piece's) stresses at
// its four edge points s[k] = (sxx, syy, sxy), scaled by qA = A_p/4.
template <int A>
__device__ __forceinline__ void node_force64(const Geo &g, const double s[4][3], double qA,
                                             double &fx, double &fy) {
  double sx = 0.0, sy = 0.0;
  sx = sx + term2<dxn(0, A), dyn(0, A)>(g, s[0][0], s[0][2]);
  sy = sy + term2y<dxn(0, A), dyn(0, A)>(g, s[0][1], s[0][2]);
  sx = sx + term2<dxn(1, A), dyn(1, A)>(g, s[1][0], s[1][2]);
  sy = sy + term2y<dxn(1, A), dyn(1, A)>(g, s[1][1], s[1][2]);
  sx = sx + term2<dxn(2, A), dyn(2, A)>(g, s[2][0], s[2][2]);
  sy = sy + term2y<dxn(2, A), dyn(2, A)>(g, s[2][1], s[2][2]);
  sx = sx + term2<dxn(3, A), dyn(3, A)>(g, s[3][0], s[3][2]);
  sy = sy + term2y<dxn(3, A), dyn(3, A)>(g, s[3][1], s[3][2]);
  fx = sx * qA;
  fy = sy * qA;
}

__device__ __forceinline__ void node_force64_rt(const Geo &g, int a, const double s[4][3],
                                                double qA, double &fx, double &fy) {
  switch (a) {
    case 0: node_force64<0>(g, s, qA, fx, fy); break;
    case 1: node_force64<1>(g, s, qA, fx, fy); break;
    case 2: node_force64<2>(g, s, qA, fx, fy); break;
    default: node_force64<3>(g, s, qA, fx, fy); break;
  }
}

// ----------------------------------------------------------------- geometry
__device__ __forceinline__ int elem_node(const Geo &g, int e, int a) {
  int i = e % g.nx, j = e / g.nx, r = g.nx + 1;
  return a == 0 ? j * r + i : a == 1 ? j * r + i + 1 : a == 2 ? (j + 1) * r + i + 1 : (j + 1) * r + i;
}

__device__ __forceinline__ int elem_neighbor(const Geo &g, int e, int k) {
  int i = e % g.nx, j = e / g.nx;
  return k == 0 ? (j > 0 ? e - g.nx : -1)
       : k == 1 ? (i < g.nx - 1 ? e + 1 : -1)
       : k == 2 ? (j < g.ny - 1 ? e + g.nx : -1)
       : (i > 0 ? e - 1 : -1);
}

__device__ __forceinline__ int elem_edge(const Geo &g, int e, int k) {
  int i = e % g.nx, j = e / g.nx;
  return k == 0 ? j * g.nx + i
       : k == 1 ? g.nh + j * (g.nx + 1) + i + 1
       : k == 2 ? (j + 1) * g.nx + i
       : g.nh + j * (g.nx + 1) + i;
}

// Elements beside edge gid: lo (below / left, its local edge 2 / 1) and hi
// (above / right, its local edge 0 / 3); -1 where there is none.
__device__ __forceinline__ void edge_sides(const Geo &g, int gid, int &lo, int &klo, int &hi,
                                           int &khi) {
  if (gid < g.nh) {
    int j = gid / g.nx, i = gid % g.nx;
    lo = j > 0 ? (j - 1) * g.nx + i : -1;
    klo = 2;
    hi = j < g.ny ? j * g.nx + i : -1;
    khi = 0;
  } else {
    int gg = gid - g.nh, j = gg / (g.nx + 1), i = gg % (g.nx + 1);
    lo = i > 0 ? j * g.nx + i - 1 : -1;
    klo = 1;
    hi = i < g.nx ? j * g.nx + i : -1;
    khi = 3;
  }
}

__device__ __forceinline__ int estatus(const DevState &d, int e) {
  return e < 0 ? ST_OUT : (int)d.estate[e];
}

// Natural coordinates of nodes and edge midpoints.
__host__ __device__ constexpr double xi_n(int a) { return (a == 0 || a == 3) ? -1.0 : 1.0; }
__host__ __device__ constexpr double eta_n(int a) { return a < 2 ? -1.0 : 1.0; }
__host__ __device__ constexpr double xi_g(int k) { return k == 1 ? 1.0 : k == 3 ? -1.0 : 0.0; }
__host__ __device__ constexpr double eta_g(int k) { return k == 0 ? -1.0 : k == 2 ? 1.0 : 0.0; }

}  // namespace cem
