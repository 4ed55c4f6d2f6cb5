// eval_common.cuh -- FP64 energy release rate of the candidate paths of a
// free-surface point (Sec. 2.2) and the Q4 cracking conditions, templated on
// how nodal displacements are read (FP64 arrays or FP32 hi + lo pairs).
// Translation units that include it are compiled with -fmad=false.
#pragma once

#include "cem_internal.h"
#include "q4_fp64.cuh"

namespace cem {

struct U64 {
  const double *x, *y;
  __device__ __forceinline__ double ux(int N) const { return x[N]; }
  __device__ __forceinline__ double uy(int N) const { return y[N]; }
};

struct U32x2 {
  const float4 *u;  // (x.hi, x.lo, y.hi, y.lo)
  __device__ __forceinline__ double ux(int N) const {
    const float4 a = u[N];
    return (double)a.x + (double)a.y;
  }
  __device__ __forceinline__ double uy(int N) const {
    const float4 a = u[N];
    return (double)a.z + (double)a.w;
  }
};

// Own strain of intact element e at its edge k.
template <class UA>
__device__ __forceinline__ void own_strain(const DevState &d, const UA &U, int e, int k,
                                           double eps[3]) {
  double u[4], v[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    int N = elem_node(d.g, e, a);
    u[a] = U.ux(N);
    v[a] = U.uy(N);
  }
  strain64_rt(d.g, k, u, v, eps);
}

// Stress used by intact element e at its edge k: smoothed with an intact
// neighbour (Eqs. 1-2, equal areas: weights 1/2), own strain otherwise.
template <class UA>
__device__ void used_stress(const DevState &d, const UA &U, int e, int k, double s[3]) {
  double eo[3];
  own_strain(d, U, e, k, eo);
  int f = elem_neighbor(d.g, e, k);
  if (estatus(d, f) == ST_INTACT) {
    double ef[3], ep[3];
    own_strain(d, U, f, (k + 2) & 3, ef);
    const double *p1 = e < f ? eo : ef;
    const double *p2 = e < f ? ef : eo;
    for (int c = 0; c < 3; ++c) ep[c] = 0.5 * p1[c] + 0.5 * p2[c];
    stress64(d.mat, ep, s);
  } else {
    stress64(d.mat, eo, s);
  }
}

__device__ __forceinline__ bool is_tip_edge(const DevState &d, int e, int k0) {
  int f = elem_neighbor(d.g, e, k0);
  if (estatus(d, f) != ST_CRACKED) return false;
  int info = d.ck_info[d.crack_of[f]];
  int kf = (k0 + 2) & 3;
  return (info & 3) == kf || ((info >> 2) & 3) == kf;
}

// Reference vector X_N2 - X_N1 of local edge k0 and the unit normal of the
// candidate segment from edge point k0 to edge point k, oriented along it.
__device__ __forceinline__ void candidate_normal(const Geo &g, int k0, int k, double &nx,
                                                 double &ny) {
  double DX = (xi_n((k0 + 1) & 3) - xi_n(k0)) * (0.5 * g.hx);
  double DY = (eta_n((k0 + 1) & 3) - eta_n(k0)) * (0.5 * g.hy);
  double x0 = (xi_g(k0) + 1.0) * (0.5 * g.hx), y0 = (eta_g(k0) + 1.0) * (0.5 * g.hy);
  double xk = (xi_g(k) + 1.0) * (0.5 * g.hx), yk = (eta_g(k) + 1.0) * (0.5 * g.hy);
  double sx = xk - x0, sy = yk - y0;
  double rx = -sy, ry = sx;
  if (rx * DX + ry * DY < 0.0) { rx = -rx; ry = -ry; }
  double len = sqrt(sx * sx + sy * sy);
  nx = rx / len;
  ny = ry / len;
}

// G of the three candidate paths of surface point (e, k0); G[k0] = -1.
// delta_d = (u_N2 - u_N1) H(|x_N2 - x_N1| > |X_N2 - X_N1|), G = delta_d.(sigma n)/2.
template <class UA>
__device__ void eval_G64(const DevState &d, const UA &U, int e, int k0, double G[4]) {
  const Geo &g = d.g;
  int N1 = elem_node(g, e, k0), N2 = elem_node(g, e, (k0 + 1) & 3);
  double DX = (xi_n((k0 + 1) & 3) - xi_n(k0)) * (0.5 * g.hx);
  double DY = (eta_n((k0 + 1) & 3) - eta_n(k0)) * (0.5 * g.hy);
  double dux = U.ux(N2) - U.ux(N1);
  double duy = U.uy(N2) - U.uy(N1);
  double dx = DX + dux, dy = DY + duy;
  double cur2 = dx * dx + dy * dy;
  double ref2 = DX * DX + DY * DY;
  double H = cur2 > ref2 ? 1.0 : 0.0;
  double ddx = dux * H, ddy = duy * H;
  for (int k = 0; k < 4; ++k) {
    if (k == k0) { G[k] = -1.0; continue; }
    double nx, ny;
    candidate_normal(g, k0, k, nx, ny);
    double s[3];
    used_stress(d, U, e, k, s);
    double tx = s[0] * nx + s[2] * ny;
    double ty = s[2] * nx + s[1] * ny;
    G[k] = 0.5 * (ddx * tx + ddy * ty);
  }
}

// Q4 cracking conditions with the split ratio gamma (Sec. 2.2).
__device__ __forceinline__ int q4_rule(const DevState &d, int e, int k0, const double G[4]) {
  double gc = (double)d.gc[e];
  int best = -1, ncand = 0;
  for (int k = 0; k < 4; ++k) {
    if (k == k0 || !(G[k] > gc)) continue;
    ++ncand;
    if (best < 0 || G[k] > G[best]) best = k;
  }
  if (ncand == 0) return -1;
  for (int q = 0; q < 4; ++q) {
    if (q == k0 || q == best || !(G[q] > gc)) continue;
    bool ok = d.mat.gamma_mode == 0 ? (G[best] > d.mat.gamma * (G[best] - G[q]))
                                    : (G[best] > d.mat.gamma * G[q]);
    if (!ok) return -1;
  }
  return best;
}

// Warp-aggregated append of a proposal (ballot + popc); whole warps call it.
__device__ __forceinline__ void append_proposal(const DevState &d, bool has, int key, int edge,
                                                int k, double G) {
  unsigned mask = __ballot_sync(0xffffffffu, has);
  if (!mask) return;
  int lane = threadIdx.x & 31;
  int leader = __ffs(mask) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(&d.cnt->n_prop, __popc(mask));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (has) {
    int pos = base + __popc(mask & ((1u << lane) - 1));
    if (pos < d.prop_cap) {
      d.pr_key[pos] = key;
      d.pr_edge[pos] = edge;
      d.pr_k[pos] = k;
      d.pr_G[pos] = G;
    } else {
      atomicOr(&d.cnt->status, STAT_CAPACITY);
    }
  }
}

}  // namespace cem
