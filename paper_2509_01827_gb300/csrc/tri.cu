// tri.cu -- ES-FEM constant-strain triangles on an unstructured mesh, FP64
// or FP32-mixed (Sec. 2.1, Eqs. 1, 3 and 5; the paper's own element).  No
// cracking.
//
// One step is three kernels:
//   k_tri_strain  element strain eps_e = B_e u_e (constant on the triangle);
//   k_tri_edge    edge strain: the area-weighted average of the two
//                 triangles' strains on an interior edge (Eq. 1), the one
//                 triangle's on a boundary edge; edge stress sigma_g = D eps_g;
//   k_tri_node    per node, the force of every (edge, triangle) incidence,
//                 B_j^T sigma_g A_j / 3 (Eq. 5), gathered in increasing edge
//                 id, then element id, then local node (no atomics), and the
//                 central-difference update with loads and prescribed
//                 velocities.
// The gather lists are built once on the host.  Compiled with -fmad=false
// and summed in the oracle's order, so the FP64 fields are bit-identical to
// it.  The FP32-mixed kernels (suffix 32) keep the displacement as
// compensated float pairs (error-free two-sum), form element strains from
// node differences, and do the rest in FP32 with FP64 energy sums: the FP64
// pipe of this GPU is 1/74 of its FP32 rate, and the FP64 path is bound by it.
// HBM per step (FP64): per element its record (64 B) and node ids (16 B),
// three node gathers and a 32-byte strain write; per edge its elements and
// weights (32 B), two strain gathers and a 32-byte stress write; per node
// its gather list (32 B per incidence, ~18 incidences: the node's b, c and
// the triangle's A/3 stored with the edge id, so a node streams its list and
// gathers only the edge stresses) and ~90 B of node state.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "cem.h"
#include "tri_internal.h"

namespace cem {

namespace {

// four doubles in one 32-byte load (strain or stress: xx, yy, xy, unused)
struct alignas(32) Dbl4 {
  double x, y, z, w;
};

// one (edge, triangle, local node) incidence of a node's gather list: the
// edge whose stress it takes and the node's b, c and the triangle's A/3
struct alignas(32) TriInc {
  int g, pad;
  double b, c, q3;
};

// element record: shape-function derivatives and the area's third
struct alignas(64) TriElem {
  double b[3], c[3];
  double q3;  // A / 3
  double A;
};

// FP32-mixed mode: the same records in single precision
struct alignas(32) TriElem32 {
  float b[3], c[3];
  float q3, A;
};
struct alignas(16) TriInc32 {
  int g;
  float b, c, q3;
};

struct TriDev {
  int nn, ne, ned;
  const int4 *conn;        // [ne] node ids, .w unused
  const TriElem *el;       // [ne]
  const int2 *edge_el;     // [ned] elements (e2 = -1 on the boundary)
  const double2 *edge_w;   // [ned] (w1, w2) area weights
  const double *edge_a;    // [ned] smoothing-domain area (A1 + A2) / 3
  const int *inc_deg;      // [nn] incidences of each node
  const long *slice_off;   // [ceil(nn / 32)] first record of each 32-node slice
  const TriInc *inc;       // gather lists, sliced: record k of node 32 s + l at
                           // slice_off[s] + 32 k + l (a warp's loads coalesce)
  Dbl4 *eps;            // [ne]
  Dbl4 *sig;            // [ned]
  double2 *u, *v;          // [nn]
  const double *m, *minv;  // [nn]
  const double2 *F;        // [nn] Neumann load at unit factor
  const double2 *Vp;       // [nn] prescribed velocity at unit factor
  const unsigned char *lflag, *dmask;
  double *Wn, *Wd;         // [nn]
  double D11, D12, D33;
  double *part;            // energy partials: [grid_edge] SE, then [grid_node] x 3
  // crack evaluation: node coordinates, edge nodes, each element's edges
  const double2 *X;        // [nn]
  const int2 *edge_nodes;  // [ned] (min, max)
  const int4 *elem_edges;  // [ne] edge ids of local edges 0, 1, 2
  // FP32-mixed mode (u as compensated pairs x.hi, x.lo, y.hi, y.lo)
  int precision;
  const TriElem32 *el32;
  const float2 *edge_w32;
  const TriInc32 *inc32;
  float4 *eps32, *sig32, *u4;
  float2 *v2;
  const float *minvf;
  double *rec;             // energy records, 7 doubles each
  int *status;             // non-finite flag
};

constexpr int kTB = 256;

__global__ void k_tri_strain(TriDev d) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d.ne; e += gridDim.x * blockDim.x) {
    const int4 n = d.conn[e];
    const TriElem &r = d.el[e];
    const int nd[3] = {n.x, n.y, n.z};
    double exx = 0.0, eyy = 0.0, gxy = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const double2 u = d.u[nd[i]];
      exx = exx + r.b[i] * u.x;
      eyy = eyy + r.c[i] * u.y;
      gxy = gxy + (r.c[i] * u.x + r.b[i] * u.y);
    }
    d.eps[e] = Dbl4{exx, eyy, gxy, 0.0};
  }
}

// block sum of one double in fixed order, written to out[blockIdx.x]
__device__ __forceinline__ void block_sum_to(double a, double *out) {
  __shared__ double ws[kTB / 32];
  for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) ws[w] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < kTB / 32; ++q) s += ws[q];
    out[blockIdx.x] = s;
  }
  __syncthreads();
}

__global__ void k_tri_edge(TriDev d, int energy) {
  double se = 0.0;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < d.ned; g += gridDim.x * blockDim.x) {
    const int2 el = d.edge_el[g];
    const Dbl4 e1 = d.eps[el.x];
    double ep0, ep1, ep2;
    if (el.y >= 0) {
      const double2 w = d.edge_w[g];
      const Dbl4 e2 = d.eps[el.y];
      ep0 = w.x * e1.x + w.y * e2.x;
      ep1 = w.x * e1.y + w.y * e2.y;
      ep2 = w.x * e1.z + w.y * e2.z;
    } else {
      ep0 = e1.x;
      ep1 = e1.y;
      ep2 = e1.z;
    }
    const double s0 = d.D11 * ep0 + d.D12 * ep1;
    const double s1 = d.D12 * ep0 + d.D11 * ep1;
    const double s2 = d.D33 * ep2;
    d.sig[g] = Dbl4{s0, s1, s2, 0.0};
    if (energy) se += 0.5 * (d.edge_a[g] * (ep0 * s0 + ep1 * s1 + ep2 * s2));
  }
  if (energy) block_sum_to(se, d.part);
}

__global__ void k_tri_node(TriDev d, double lamN, double lamD, double dt, double dtv, int first,
                           int energy, int part_off) {
  double ke = 0.0, wn = 0.0, wd = 0.0;
  bool bad = false;
  for (int N = blockIdx.x * blockDim.x + threadIdx.x; N < d.nn; N += gridDim.x * blockDim.x) {
    double fx = 0.0, fy = 0.0;
    const int deg = d.inc_deg[N];
    const TriInc *rec = d.inc + d.slice_off[N >> 5] + (N & 31);
#pragma unroll 4
    for (int k = 0; k < deg; ++k) {
      const TriInc r = rec[32L * k];
      const Dbl4 s = d.sig[r.g];
      fx = fx + (r.b * s.x + r.c * s.z) * r.q3;
      fy = fy + (r.c * s.y + r.b * s.z) * r.q3;
    }
    const int loaded = d.lflag[N];
    const int dm = d.dmask[N];
    const double2 F = d.F[N];
    const double fex = loaded ? lamN * F.x : 0.0;
    const double fey = loaded ? lamN * F.y : 0.0;
    const double mi = d.minv[N];
    const double ax = (fex - fx) * mi;
    const double ay = (fey - fy) * mi;
    const double2 vo = d.v[N];
    double vxn = vo.x + dtv * ax;
    double vyn = vo.y + dtv * ay;
    if (dm) {
      const double2 V = d.Vp[N];
      if (dm & 1) vxn = lamD * V.x;
      if (dm & 2) vyn = lamD * V.y;
    }
    const double vbx = first ? vo.x : 0.5 * (vo.x + vxn);
    const double vby = first ? vo.y : 0.5 * (vo.y + vyn);
    if (energy) {
      wn += d.Wn[N];
      wd += d.Wd[N];
    }
    if (loaded) d.Wn[N] = d.Wn[N] + dt * (fex * vbx + fey * vby);
    if (dm) {
      const double m = d.m[N];
      const double Rx = m * ((vxn - vo.x) / dtv) - (fex - fx);
      const double Ry = m * ((vyn - vo.y) / dtv) - (fey - fy);
      double w = 0.0;
      if (dm & 1) w = w + Rx * vbx;
      if (dm & 2) w = w + Ry * vby;
      d.Wd[N] = d.Wd[N] + dt * w;
    }
    if (energy) ke += 0.5 * (d.m[N] * (vbx * vbx + vby * vby));
    d.v[N] = make_double2(vxn, vyn);
    const double2 u = d.u[N];
    d.u[N] = make_double2(u.x + dt * vxn, u.y + dt * vyn);
    bad |= !(fabs(vxn) <= DBL_MAX) || !(fabs(vyn) <= DBL_MAX);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(d.status, 1);
  if (energy) {
    block_sum_to(ke, d.part + part_off);
    block_sum_to(wn, d.part + part_off + gridDim.x);
    block_sum_to(wd, d.part + part_off + 2 * gridDim.x);
  }
}

// ------------------------------------------------------ FP32-mixed mode
// (hi, lo) += x, error-free (Knuth's two-sum) with renormalisation: the
// displacement keeps about 48 significant bits without FP64 arithmetic
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float x) {
  const float s = __fadd_rn(hi, x);
  const float bb = __fsub_rn(s, hi);
  const float er = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
  const float l = __fadd_rn(lo, er);
  const float h = __fadd_rn(s, l);
  lo = __fsub_rn(l, __fsub_rn(h, s));
  hi = h;
}

// element strain from the differences of nodes 1 and 2 to node 0, each a
// difference of compensated pairs: b_0 = -(b_1 + b_2), so sum_i b_i u_i =
// b_1 (u_1 - u_0) + b_2 (u_2 - u_0), free of the cancellation of a large
// common displacement
__global__ void k_tri_strain32(TriDev d) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d.ne; e += gridDim.x * blockDim.x) {
    const int4 n = d.conn[e];
    const TriElem32 &r = d.el32[e];
    const float4 U0 = d.u4[n.x], U1 = d.u4[n.y], U2 = d.u4[n.z];
    const float d1x = (U1.x - U0.x) + (U1.y - U0.y), d1y = (U1.z - U0.z) + (U1.w - U0.w);
    const float d2x = (U2.x - U0.x) + (U2.y - U0.y), d2y = (U2.z - U0.z) + (U2.w - U0.w);
    const float exx = r.b[1] * d1x + r.b[2] * d2x;
    const float eyy = r.c[1] * d1y + r.c[2] * d2y;
    const float gxy = (r.c[1] * d1x + r.c[2] * d2x) + (r.b[1] * d1y + r.b[2] * d2y);
    d.eps32[e] = make_float4(exx, eyy, gxy, 0.f);
  }
}

__global__ void k_tri_edge32(TriDev d, int energy) {
  double se = 0.0;
  const float D11 = (float)d.D11, D12 = (float)d.D12, D33 = (float)d.D33;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < d.ned; g += gridDim.x * blockDim.x) {
    const int2 el = d.edge_el[g];
    const float4 e1 = d.eps32[el.x];
    float ep0 = e1.x, ep1 = e1.y, ep2 = e1.z;
    if (el.y >= 0) {
      const float2 w = d.edge_w32[g];
      const float4 e2 = d.eps32[el.y];
      ep0 = w.x * e1.x + w.y * e2.x;
      ep1 = w.x * e1.y + w.y * e2.y;
      ep2 = w.x * e1.z + w.y * e2.z;
    }
    const float s0 = D11 * ep0 + D12 * ep1;
    const float s1 = D12 * ep0 + D11 * ep1;
    const float s2 = D33 * ep2;
    d.sig32[g] = make_float4(s0, s1, s2, 0.f);
    if (energy) se += 0.5 * (d.edge_a[g] * (double)(ep0 * s0 + ep1 * s1 + ep2 * s2));
  }
  if (energy) block_sum_to(se, d.part);
}

__global__ void k_tri_node32(TriDev d, double lamN, double lamD, double dtd, double dtvd,
                             int first, int energy, int part_off) {
  double ke = 0.0, wn = 0.0, wd = 0.0;
  bool bad = false;
  const float dt = (float)dtd, dtv = (float)dtvd;
  for (int N = blockIdx.x * blockDim.x + threadIdx.x; N < d.nn; N += gridDim.x * blockDim.x) {
    float fx = 0.f, fy = 0.f;
    const int deg = d.inc_deg[N];
    const TriInc32 *rec = d.inc32 + d.slice_off[N >> 5] + (N & 31);
#pragma unroll 4
    for (int k = 0; k < deg; ++k) {
      const TriInc32 r = rec[32L * k];
      const float4 s = d.sig32[r.g];
      fx = fx + (r.b * s.x + r.c * s.z) * r.q3;
      fy = fy + (r.c * s.y + r.b * s.z) * r.q3;
    }
    const int loaded = d.lflag[N];
    const int dm = d.dmask[N];
    float fex = 0.f, fey = 0.f;
    if (loaded) {
      const double2 F = d.F[N];
      fex = (float)(lamN * F.x);
      fey = (float)(lamN * F.y);
    }
    const float mi = d.minvf[N];
    const float2 vo = d.v2[N];
    float vxn = vo.x + dtv * ((fex - fx) * mi);
    float vyn = vo.y + dtv * ((fey - fy) * mi);
    if (dm) {
      const double2 V = d.Vp[N];
      if (dm & 1) vxn = (float)(lamD * V.x);
      if (dm & 2) vyn = (float)(lamD * V.y);
    }
    const double vbx = first ? (double)vo.x : 0.5 * ((double)vo.x + (double)vxn);
    const double vby = first ? (double)vo.y : 0.5 * ((double)vo.y + (double)vyn);
    if (energy) {
      wn += d.Wn[N];
      wd += d.Wd[N];
    }
    if (loaded) d.Wn[N] = d.Wn[N] + dtd * ((double)fex * vbx + (double)fey * vby);
    if (dm) {
      const double m = d.m[N], dv = dtvd;
      const double Rx = m * (((double)vxn - (double)vo.x) / dv) - ((double)fex - (double)fx);
      const double Ry = m * (((double)vyn - (double)vo.y) / dv) - ((double)fey - (double)fy);
      double w = 0.0;
      if (dm & 1) w = w + Rx * vbx;
      if (dm & 2) w = w + Ry * vby;
      d.Wd[N] = d.Wd[N] + dtd * w;
    }
    if (energy) ke += 0.5 * (d.m[N] * (vbx * vbx + vby * vby));
    d.v2[N] = make_float2(vxn, vyn);
    float4 U = d.u4[N];
    two_sum_acc(U.x, U.y, dt * vxn);
    two_sum_acc(U.z, U.w, dt * vyn);
    d.u4[N] = U;
    bad |= !(fabsf(vxn) <= FLT_MAX) || !(fabsf(vyn) <= FLT_MAX);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(d.status, 1);
  if (energy) {
    block_sum_to(ke, d.part + part_off);
    block_sum_to(wn, d.part + part_off + gridDim.x);
    block_sum_to(wd, d.part + part_off + 2 * gridDim.x);
  }
}

// ------------------------------------------------------- crack evaluation
// FP64 displacement of node N in either precision
__device__ __forceinline__ double2 node_u64(const TriDev &d, int N) {
  if (d.precision == CEM_FP32_MIXED) {
    const float4 U = d.u4[N];
    return make_double2((double)U.x + (double)U.y, (double)U.z + (double)U.w);
  }
  return d.u[N];
}

// strain of element e from the current displacement, in the oracle's order
__device__ __forceinline__ void elem_strain64(const TriDev &d, int e, double ep[3]) {
  const int4 n = d.conn[e];
  const int nd[3] = {n.x, n.y, n.z};
  const TriElem &r = d.el[e];
  double exx = 0.0, eyy = 0.0, gxy = 0.0;
  for (int i = 0; i < 3; ++i) {
    const double2 u = node_u64(d, nd[i]);
    exx = exx + r.b[i] * u.x;
    eyy = eyy + r.c[i] * u.y;
    gxy = gxy + (r.c[i] * u.x + r.b[i] * u.y);
  }
  ep[0] = exx; ep[1] = eyy; ep[2] = gxy;
}

// Sec. 2.2 for triangles, one thread per surface point (edge g0 of element
// e): delta_d over the point's edge with the stretch test, the energy
// release rate of the path to the midpoint of each of the element's two
// other edges (the edge's smoothed stress on the segment's normal), and the
// decision rule; FP64 in either precision.
__global__ void k_tri_eval(TriDev d, int n, const int *edge, const int *elem, const float *gc,
                           double gamma, int gamma_mode, double *G, int *choice) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const int g0 = edge[q], e = elem[q];
    const int4 cn4 = d.conn[e];
    const int cn[3] = {cn4.x, cn4.y, cn4.z};
    const int2 en = d.edge_nodes[g0];
    int k0 = 0;
    for (int k = 0; k < 3; ++k) {
      const int a = cn[k], b = cn[(k + 1) % 3];
      if ((a == en.x && b == en.y) || (a == en.y && b == en.x)) k0 = k;
    }
    const int N1 = cn[k0], N2 = cn[(k0 + 1) % 3];
    const double2 P1 = d.X[N1], P2 = d.X[N2];
    const double dX = P2.x - P1.x, dY = P2.y - P1.y;
    const double2 u1 = node_u64(d, N1), u2 = node_u64(d, N2);
    const double dux = u2.x - u1.x, duy = u2.y - u1.y;
    const double lx = dX + dux, ly = dY + duy;
    const bool H = lx * lx + ly * ly > dX * dX + dY * dY;
    const double ddx = H ? dux : 0.0, ddy = H ? duy : 0.0;
    const double mx0 = 0.5 * (P1.x + P2.x), my0 = 0.5 * (P1.y + P2.y);
    const int4 ee = d.elem_edges[e];
    const int eds[3] = {ee.x, ee.y, ee.z};
    double Gj[2];
    int kj[2];
    for (int j = 0; j < 2; ++j) {
      const int k = (k0 + 1 + j) % 3;
      kj[j] = k;
      const double2 A = d.X[cn[k]], B = d.X[cn[(k + 1) % 3]];
      const double mx = 0.5 * (A.x + B.x), my = 0.5 * (A.y + B.y);
      const double tx = mx - mx0, ty = my - my0;
      const double L = sqrt(tx * tx + ty * ty);
      double nx = -ty / L, ny = tx / L;
      if (nx * dX + ny * dY < 0) { nx = -nx; ny = -ny; }
      const int g = eds[k];
      const int2 el = d.edge_el[g];
      double ep[3], e1[3], e2[3];
      elem_strain64(d, el.x, e1);
      if (el.y >= 0) {
        elem_strain64(d, el.y, e2);
        const double2 w = d.edge_w[g];
        for (int c = 0; c < 3; ++c) ep[c] = w.x * e1[c] + w.y * e2[c];
      } else {
        for (int c = 0; c < 3; ++c) ep[c] = e1[c];
      }
      const double s0 = d.D11 * ep[0] + d.D12 * ep[1];
      const double s1 = d.D12 * ep[0] + d.D11 * ep[1];
      const double s2 = d.D33 * ep[2];
      const double snx = s0 * nx + s2 * ny, sny = s2 * nx + s1 * ny;
      Gj[j] = 0.5 * (ddx * snx + ddy * sny);
      G[2 * q + j] = Gj[j];
    }
    const double gce = (double)gc[e];
    const bool a0 = Gj[0] > gce, a1 = Gj[1] > gce;
    int pick = -1;
    if (a0 && !a1) {
      pick = 0;
    } else if (a1 && !a0) {
      pick = 1;
    } else if (a0 && a1) {
      const bool p0 = gamma_mode ? Gj[0] > gamma * Gj[1] : Gj[0] > gamma * (Gj[0] - Gj[1]);
      const bool p1 = gamma_mode ? Gj[1] > gamma * Gj[0] : Gj[1] > gamma * (Gj[1] - Gj[0]);
      if (p0 && p1) pick = Gj[1] > Gj[0] ? 1 : (Gj[0] > Gj[1] ? 0 : (kj[0] < kj[1] ? 0 : 1));
      else if (p0) pick = 0;
      else if (p1) pick = 1;
    }
    choice[q] = pick < 0 ? -1 : kj[pick];
  }
}

// one thread: the record (step, t, KE, SE, W_ext, W_dir, U_d = 0) from the
// partials, summed in block order
__global__ void k_tri_record(TriDev d, int ge, int gn, int part_off, int slot, double step,
                             double t) {
  if (threadIdx.x || blockIdx.x) return;
  double se = 0.0, ke = 0.0, wn = 0.0, wd = 0.0;
  for (int b = 0; b < ge; ++b) se += d.part[b];
  for (int b = 0; b < gn; ++b) {
    ke += d.part[part_off + b];
    wn += d.part[part_off + gn + b];
    wd += d.part[part_off + 2 * gn + b];
  }
  double *r = d.rec + 7 * (size_t)slot;
  r[0] = step; r[1] = t; r[2] = ke; r[3] = se; r[4] = wn; r[5] = wd; r[6] = 0.0;
}

int grid_of(long n) {
  const long b = (n + kTB - 1) / kTB;
  return (int)std::max(1L, std::min(b, 152L * 8));
}

double law_eval(int law, double t, double t0, double tau) {
  if (law == CEM_LAW_CONST) return 1.0;
  if (t <= t0) return t / t0;
  if (law == CEM_LAW_RAMP) return 1.0;
  return std::exp(-(t - t0) / tau);
}

}  // namespace

struct TriMesh {
  int nn = 0, ne = 0, ned = 0;
  int device = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  cem_alloc_fn alloc = nullptr;
  cem_free_fn free_fn = nullptr;
  void *ctx = nullptr;
  std::vector<void *> blocks;
  // host geometry
  std::vector<double> X;
  std::vector<int> conn;
  std::vector<TriElem> el;
  std::vector<int> en1, en2, ee1, ee2;
  double hmin = 0.0, dt_factor = 0.5, dt_explicit = 0.0, dt = 0.0;
  double E = 0, nu = 0, rho = 0, D11 = 0, D12 = 0, D33 = 0;
  bool material = false;
  // loads
  std::vector<double2> F, Vp;
  std::vector<unsigned char> lflag, dmask;
  bool neu_set = false, dir_set = false;
  int neu_law = 0, dir_law = 0;
  double neu_t0 = 0, neu_tau = 0, dir_t0 = 0, dir_tau = 0;
  bool loads_dirty = true;
  long step = 0;
  int energy_every = 0;
  long n_rec = 0, rec_cap = 0;
  long launches = 0;
  int ge = 1, gn = 1;
  TriDev d{};
  int *h_status = nullptr;
  int precision = CEM_FP64;
  std::vector<float> gc;  // per element
  double gamma = 1.0;
  int gamma_mode = 0;
  float *d_gc = nullptr;
};

namespace {

void *tri_alloc(TriMesh *t, size_t bytes) {
  void *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (t->alloc) {
    p = t->alloc(bytes, t->ctx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    p = nullptr;
  }
  if (p) {
    t->blocks.push_back(p);
    cudaMemsetAsync(p, 0, bytes, t->st);
  }
  return p;
}

template <class T>
bool tri_alloc_n(TriMesh *t, T *&p, size_t n) {
  p = static_cast<T *>(tri_alloc(t, n * sizeof(T)));
  return p != nullptr;
}

template <class T>
bool upload(TriMesh *t, T *dst, const std::vector<T> &src) {
  return src.empty() || cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(T),
                                        cudaMemcpyHostToDevice, t->st) == cudaSuccess;
}

}  // namespace

void tri_destroy(TriMesh *t) {
  if (!t) return;
  cudaSetDevice(t->device);
  if (t->st) cudaStreamSynchronize(t->st);
  for (void *p : t->blocks) {
    if (t->free_fn) t->free_fn(p, t->ctx);
    else cudaFree(p);
  }
  if (t->h_status) cudaFreeHost(t->h_status);
  if (t->own_stream) cudaStreamDestroy(t->st);
  delete t;
}

TriMesh *tri_create(const cem_tri_mesh_desc *desc, std::string &err) {
  const int nn = desc->n_nodes, ne = desc->n_elems;
  if (nn < 3 || ne < 1 || !desc->X || !desc->conn) {
    err = "need >= 3 nodes, >= 1 element, X and conn";
    return nullptr;
  }
  if (desc->alloc && !desc->free) {
    err = "free is required with alloc";
    return nullptr;
  }
  for (long q = 0; q < 3L * ne; ++q)
    if (desc->conn[q] < 0 || desc->conn[q] >= nn) {
      err = "node id out of range in conn";
      return nullptr;
    }
  TriMesh *t = new TriMesh();
  t->nn = nn;
  t->ne = ne;
  t->X.assign(desc->X, desc->X + 2L * nn);
  t->conn.assign(desc->conn, desc->conn + 3L * ne);
  t->el.resize(ne);
  // geometry in the oracle's order of operations (host compiled without
  // contraction): twice the area, derivatives, the area's third
  double hmin = INFINITY;
  for (int e = 0; e < ne; ++e) {
    const int *n = &t->conn[3L * e];
    double x[3], y[3];
    for (int i = 0; i < 3; ++i) { x[i] = t->X[2L * n[i]]; y[i] = t->X[2L * n[i] + 1]; }
    const double twoA = (x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]);
    if (!(twoA > 0)) {
      err = "element " + std::to_string(e) + " is not counter-clockwise";
      delete t;
      return nullptr;
    }
    TriElem &r = t->el[e];
    r.A = 0.5 * twoA;
    for (int i = 0; i < 3; ++i) {
      const int j = (i + 1) % 3, k = (i + 2) % 3;
      r.b[i] = (y[j] - y[k]) / twoA;
      r.c[i] = (x[k] - x[j]) / twoA;
    }
    r.q3 = r.A / 3.0;
    double Lmax = 0.0;
    for (int i = 0; i < 3; ++i) {
      const int j = (i + 1) % 3;
      const double L = std::sqrt((x[j] - x[i]) * (x[j] - x[i]) + (y[j] - y[i]) * (y[j] - y[i]));
      if (L > Lmax) Lmax = L;
    }
    const double h = twoA / Lmax;
    if (h < hmin) hmin = h;
  }
  t->hmin = hmin;
  // edges: distinct node pairs in increasing (min, max), their elements
  struct Half { int a, b, e, k; };
  std::vector<Half> he((size_t)ne * 3);
  for (int e = 0; e < ne; ++e)
    for (int k = 0; k < 3; ++k) {
      const int a = t->conn[3L * e + k], b = t->conn[3L * e + (k + 1) % 3];
      he[3L * e + k] = Half{std::min(a, b), std::max(a, b), e, k};
    }
  std::sort(he.begin(), he.end(), [](const Half &p, const Half &q) {
    if (p.a != q.a) return p.a < q.a;
    if (p.b != q.b) return p.b < q.b;
    if (p.e != q.e) return p.e < q.e;
    return p.k < q.k;
  });
  for (size_t q = 0; q < he.size();) {
    size_t r = q + 1;
    while (r < he.size() && he[r].a == he[q].a && he[r].b == he[q].b) ++r;
    if (r - q > 2 || he[q].a == he[q].b) {
      err = "an edge has more than two elements";
      delete t;
      return nullptr;
    }
    t->en1.push_back(he[q].a);
    t->en2.push_back(he[q].b);
    t->ee1.push_back(he[q].e);
    t->ee2.push_back(r - q == 2 ? he[q + 1].e : -1);
    q = r;
  }
  t->ned = (int)t->en1.size();
  t->F.assign(nn, make_double2(0.0, 0.0));
  t->Vp.assign(nn, make_double2(0.0, 0.0));
  t->lflag.assign(nn, 0);
  t->dmask.assign(nn, 0);
  if (desc->precision != CEM_FP64 && desc->precision != CEM_FP32_MIXED) {
    err = "bad precision";
    delete t;
    return nullptr;
  }
  t->precision = desc->precision;
  t->dt_factor = desc->dt_factor > 0 ? desc->dt_factor : 0.5;
  t->dt_explicit = desc->dt > 0 ? desc->dt : 0.0;
  t->energy_every = desc->energy_every > 0 ? desc->energy_every : 0;
  t->device = desc->device;
  t->alloc = desc->alloc;
  t->free_fn = desc->free;
  t->ctx = desc->alloc_ctx;
  t->st = (cudaStream_t)desc->cuda_stream;
  cudaError_t ce = cudaSetDevice(t->device);
  if (ce == cudaSuccess && !t->st) {
    ce = cudaStreamCreateWithFlags(&t->st, cudaStreamNonBlocking);
    t->own_stream = ce == cudaSuccess;
  }
  if (ce == cudaSuccess) ce = cudaHostAlloc((void **)&t->h_status, sizeof(int), cudaHostAllocDefault);
  if (ce != cudaSuccess) {
    err = std::string("CUDA set-up failed: ") + cudaGetErrorString(ce);
    tri_destroy(t);
    return nullptr;
  }
  // device arrays
  std::vector<int4> c4(ne);
  for (int e = 0; e < ne; ++e)
    c4[e] = make_int4(t->conn[3L * e], t->conn[3L * e + 1], t->conn[3L * e + 2], 0);
  std::vector<int2> eel(t->ned);
  std::vector<double2> ew(t->ned);
  std::vector<double> ea(t->ned);
  for (int g = 0; g < t->ned; ++g) {
    const int e1 = t->ee1[g], e2 = t->ee2[g];
    eel[g] = make_int2(e1, e2);
    double a = t->el[e1].A / 3.0;
    if (e2 >= 0) {
      const double A1 = t->el[e1].A, A2 = t->el[e2].A;
      ew[g] = make_double2(A1 / (A1 + A2), A2 / (A1 + A2));
      a = a + t->el[e2].A / 3.0;
    } else {
      ew[g] = make_double2(1.0, 0.0);
    }
    ea[g] = a;
  }
  // gather lists: for each node, its (edge, element side, local node)
  // incidences in increasing edge id, then side, then local node
  std::vector<int> cnt(nn + 1, 0);
  for (int g = 0; g < t->ned; ++g)
    for (int side = 0; side < 2; ++side) {
      const int e = side ? t->ee2[g] : t->ee1[g];
      if (e < 0) continue;
      for (int i = 0; i < 3; ++i) cnt[t->conn[3L * e + i] + 1]++;
    }
  for (int N = 0; N < nn; ++N) cnt[N + 1] += cnt[N];
  // sliced layout: the nodes of slice s = N / 32 store their k-th records
  // side by side, 32 per row, as many rows as the slice's largest list
  const int nsl = (nn + 31) / 32;
  std::vector<int> deg(nn);
  std::vector<long> soff(nsl + 1, 0);
  for (int N = 0; N < nn; ++N) deg[N] = cnt[N + 1] - cnt[N];
  for (int sl = 0; sl < nsl; ++sl) {
    int dmax = 0;
    for (int N = 32 * sl; N < std::min(nn, 32 * sl + 32); ++N) dmax = std::max(dmax, deg[N]);
    soff[sl + 1] = soff[sl] + 32L * dmax;
  }
  std::vector<TriInc> inc(std::max(1L, soff[nsl]), TriInc{0, 0, 0.0, 0.0, 0.0});
  std::vector<TriInc32> inc32(t->precision == CEM_FP32_MIXED ? inc.size() : 0, TriInc32{0, 0.f, 0.f, 0.f});
  std::vector<int> fill(nn, 0);
  for (int g = 0; g < t->ned; ++g)
    for (int side = 0; side < 2; ++side) {
      const int e = side ? t->ee2[g] : t->ee1[g];
      if (e < 0) continue;
      for (int i = 0; i < 3; ++i) {
        const int N = t->conn[3L * e + i];
        const long at = soff[N >> 5] + (N & 31) + 32L * fill[N]++;
        inc[at] = TriInc{g, 0, t->el[e].b[i], t->el[e].c[i], t->el[e].q3};
        if (!inc32.empty())
          inc32[at] = TriInc32{g, (float)t->el[e].b[i], (float)t->el[e].c[i], (float)t->el[e].q3};
      }
    }
  soff.pop_back();
  t->ge = grid_of(t->ned);
  t->gn = grid_of(nn);
  TriDev &d = t->d;
  d.nn = nn;
  d.ne = ne;
  d.ned = t->ned;
  int4 *dconn;
  TriElem *del;
  int2 *deel;
  TriInc *dinc;
  double2 *dew, *dF, *dVp;
  double *dea, *dm, *dminv;
  int *ddeg;
  long *dsoff;
  unsigned char *dlf, *ddm;
  bool ok = tri_alloc_n(t, dconn, ne) && tri_alloc_n(t, del, ne) && tri_alloc_n(t, deel, t->ned) &&
            tri_alloc_n(t, dew, t->ned) && tri_alloc_n(t, dea, t->ned) &&
            tri_alloc_n(t, ddeg, (size_t)nn) && tri_alloc_n(t, dsoff, soff.size()) &&
            tri_alloc_n(t, dinc, inc.size()) &&
            tri_alloc_n(t, d.eps, ne) && tri_alloc_n(t, d.sig, t->ned) &&
            tri_alloc_n(t, d.u, nn) && tri_alloc_n(t, d.v, nn) && tri_alloc_n(t, dm, nn) &&
            tri_alloc_n(t, dminv, nn) && tri_alloc_n(t, dF, nn) && tri_alloc_n(t, dVp, nn) &&
            tri_alloc_n(t, dlf, nn) && tri_alloc_n(t, ddm, nn) && tri_alloc_n(t, d.Wn, nn) &&
            tri_alloc_n(t, d.Wd, nn) &&
            tri_alloc_n(t, d.part, (size_t)t->ge + 3 * (size_t)t->gn) &&
            tri_alloc_n(t, d.status, 1);
  if (ok && t->precision == CEM_FP32_MIXED) {
    std::vector<TriElem32> e32(ne);
    for (int e = 0; e < ne; ++e) {
      for (int i = 0; i < 3; ++i) { e32[e].b[i] = (float)t->el[e].b[i]; e32[e].c[i] = (float)t->el[e].c[i]; }
      e32[e].q3 = (float)t->el[e].q3;
      e32[e].A = (float)t->el[e].A;
    }
    std::vector<float2> w32(t->ned);
    for (int g = 0; g < t->ned; ++g) w32[g] = make_float2((float)ew[g].x, (float)ew[g].y);
    TriElem32 *de32;
    float2 *dw32;
    TriInc32 *di32;
    float *dmf;
    ok = tri_alloc_n(t, de32, ne) && tri_alloc_n(t, dw32, t->ned) && tri_alloc_n(t, di32, inc32.size()) &&
         tri_alloc_n(t, d.eps32, ne) && tri_alloc_n(t, d.sig32, t->ned) && tri_alloc_n(t, d.u4, nn) &&
         tri_alloc_n(t, d.v2, nn) && tri_alloc_n(t, dmf, nn) && upload(t, de32, e32) &&
         upload(t, dw32, w32) && upload(t, di32, inc32);
    d.el32 = de32; d.edge_w32 = dw32; d.inc32 = di32; d.minvf = dmf;
  }
  d.precision = t->precision;
  t->rec_cap = 1024;
  ok = ok && tri_alloc_n(t, d.rec, (size_t)t->rec_cap * 7);
  ok = ok && upload(t, dconn, c4) && upload(t, del, t->el) && upload(t, deel, eel) &&
       upload(t, dew, ew) && upload(t, dea, ea) && upload(t, ddeg, deg) && upload(t, dsoff, soff) && upload(t, dinc, inc);
  if (!ok || cudaStreamSynchronize(t->st) != cudaSuccess) {
    err = "device allocation or upload failed";
    tri_destroy(t);
    return nullptr;
  }
  // crack-evaluation tables: coordinates, edge nodes, each element's edges
  {
    std::vector<double2> X2(nn);
    for (int N = 0; N < nn; ++N) X2[N] = make_double2(t->X[2L * N], t->X[2L * N + 1]);
    std::vector<int2> enod(t->ned);
    for (int g = 0; g < t->ned; ++g) enod[g] = make_int2(t->en1[g], t->en2[g]);
    std::vector<int4> eed(ne, make_int4(-1, -1, -1, -1));
    // each element's local edge k is the node pair (conn[k], conn[k+1])
    for (int g = 0; g < t->ned; ++g)
      for (int side = 0; side < 2; ++side) {
        const int e = side ? t->ee2[g] : t->ee1[g];
        if (e < 0) continue;
        for (int k = 0; k < 3; ++k) {
          const int a = t->conn[3L * e + k], b = t->conn[3L * e + (k + 1) % 3];
          if (std::min(a, b) == t->en1[g] && std::max(a, b) == t->en2[g]) (&eed[e].x)[k] = g;
        }
      }
    double2 *dX;
    int2 *dEn;
    int4 *dEe;
    float *dgc;
    t->gc.assign(ne, 3.0f);
    if (!tri_alloc_n(t, dX, nn) || !tri_alloc_n(t, dEn, t->ned) || !tri_alloc_n(t, dEe, ne) ||
        !tri_alloc_n(t, dgc, ne) || !upload(t, dX, X2) || !upload(t, dEn, enod) ||
        !upload(t, dEe, eed) || !upload(t, dgc, t->gc) || cudaStreamSynchronize(t->st) != cudaSuccess) {
      err = "device allocation or upload failed";
      tri_destroy(t);
      return nullptr;
    }
    d.X = dX; d.edge_nodes = dEn; d.elem_edges = dEe;
    t->d_gc = dgc;
  }
  d.conn = dconn; d.el = del; d.edge_el = deel; d.edge_w = dew; d.edge_a = dea;
  d.inc_deg = ddeg; d.slice_off = dsoff; d.inc = dinc; d.m = dm; d.minv = dminv; d.F = dF; d.Vp = dVp;
  d.lflag = dlf; d.dmask = ddm;
  return t;
}

int tri_n_edges(const TriMesh *t) { return t->ned; }

cem_status tri_set_material(TriMesh *t, double E, double nu, double rho, int plane_strain,
                            const float *gc, double gc_uniform, double gamma, int gamma_mode,
                            std::string &err) {
  if (t->material) { err = "material already set"; return CEM_ERR_STATE; }
  if (!(E > 0) || !(nu > -1.0 && nu < 0.5) || !(rho > 0)) { err = "bad material"; return CEM_ERR_ARG; }
  if (gamma_mode < 0 || gamma_mode > 1) { err = "bad gamma mode"; return CEM_ERR_ARG; }
  for (int e = 0; e < t->ne; ++e) t->gc[e] = gc ? gc[e] : (float)gc_uniform;
  t->gamma = gamma;
  t->gamma_mode = gamma_mode;
  if (!upload(t, t->d_gc, t->gc)) { err = "upload failed"; return CEM_ERR_CUDA; }
  t->E = E; t->nu = nu; t->rho = rho;
  double cd;
  if (plane_strain) {
    const double c = E / ((1.0 + nu) * (1.0 - 2.0 * nu));
    t->D11 = c * (1.0 - nu);
    t->D12 = c * nu;
    t->D33 = c * (1.0 - 2.0 * nu) * 0.5;
    cd = std::sqrt((E * (1.0 - nu)) / (rho * ((1.0 + nu) * (1.0 - 2.0 * nu))));
  } else {
    const double c = E / (1.0 - nu * nu);
    t->D11 = c;
    t->D12 = c * nu;
    t->D33 = c * (1.0 - nu) * 0.5;
    cd = std::sqrt(E / (rho * (1.0 - nu * nu)));
  }
  t->d.D11 = t->D11; t->d.D12 = t->D12; t->d.D33 = t->D33;
  t->dt = t->dt_explicit > 0 ? t->dt_explicit : t->dt_factor * t->hmin / cd;
  // lumped masses: rho A / 3 to each node, in increasing element id
  std::vector<double> m(t->nn, 0.0), mi(t->nn, 0.0);
  for (int e = 0; e < t->ne; ++e) {
    const double me = (rho * t->el[e].A) / 3.0;
    for (int i = 0; i < 3; ++i) m[t->conn[3L * e + i]] = m[t->conn[3L * e + i]] + me;
  }
  for (int N = 0; N < t->nn; ++N) mi[N] = m[N] > 0 ? 1.0 / m[N] : 0.0;
  cudaSetDevice(t->device);
  std::vector<float> mif;
  if (t->precision == CEM_FP32_MIXED)
    for (double x : mi) mif.push_back((float)x);
  if (!upload(t, const_cast<double *>(t->d.m), m) || !upload(t, const_cast<double *>(t->d.minv), mi) ||
      (!mif.empty() && !upload(t, const_cast<float *>(t->d.minvf), mif)) ||
      cudaStreamSynchronize(t->st) != cudaSuccess) {
    err = "mass upload failed";
    return CEM_ERR_CUDA;
  }
  t->material = true;
  return CEM_OK;
}

// Neumann loads: each node of a loaded boundary edge of length L gets L/2
// times the traction (pressure: -p times the outward normal of the edge's
// counter-clockwise element side), edges in increasing id; prescribed
// velocities per component on nodes.
cem_status tri_set_bc(TriMesh *t, int kind, int n, const int *items, int comp_mask, int law,
                      double a0, double t0, double tau, std::string &err) {
  if (n < 0 || (n > 0 && !items)) { err = "bad items"; return CEM_ERR_ARG; }
  if (law < 0 || law > 2) { err = "bad law"; return CEM_ERR_ARG; }
  if (law != CEM_LAW_CONST && !(t0 > 0)) { err = "t0 must be > 0"; return CEM_ERR_ARG; }
  if (law == CEM_LAW_RAMP_EXP && !(tau > 0)) { err = "tau must be > 0"; return CEM_ERR_ARG; }
  if (t->step != 0) { err = "loads can only be set before the first step"; return CEM_ERR_STATE; }
  if (kind == CEM_TRACTION || kind == CEM_PRESSURE) {
    if (t->neu_set && (t->neu_law != law || t->neu_t0 != t0 || t->neu_tau != tau)) {
      err = "all Neumann loads share one time law";
      return CEM_ERR_ARG;
    }
    for (int q = 0; q < n; ++q)
      if (items[q] < 0 || items[q] >= t->ned || t->ee2[items[q]] >= 0) {
        err = "edge " + std::to_string(items[q]) + " is not a boundary edge";
        return CEM_ERR_ARG;
      }
    std::vector<int> s(items, items + n);
    std::sort(s.begin(), s.end());
    for (int g : s) {
      const int e = t->ee1[g];
      int a = -1, b = -1;
      for (int k = 0; k < 3; ++k) {
        const int p = t->conn[3L * e + k], q = t->conn[3L * e + (k + 1) % 3];
        if ((p == t->en1[g] && q == t->en2[g]) || (p == t->en2[g] && q == t->en1[g])) { a = p; b = q; }
      }
      const double dx = t->X[2L * b] - t->X[2L * a], dy = t->X[2L * b + 1] - t->X[2L * a + 1];
      const double L = std::sqrt(dx * dx + dy * dy);
      const double ox = dy / L, oy = -dx / L;
      double tx, ty;
      if (kind == CEM_TRACTION) {
        tx = (comp_mask & 1) ? a0 : 0.0;
        ty = (comp_mask & 2) ? a0 : 0.0;
      } else {
        tx = -a0 * ox;
        ty = -a0 * oy;
      }
      const double half = 0.5 * L;
      const int n1 = t->en1[g], n2 = t->en2[g];
      t->F[n1].x = t->F[n1].x + half * tx; t->F[n1].y = t->F[n1].y + half * ty;
      t->F[n2].x = t->F[n2].x + half * tx; t->F[n2].y = t->F[n2].y + half * ty;
      t->lflag[n1] = 1;
      t->lflag[n2] = 1;
    }
    t->neu_set = true; t->neu_law = law; t->neu_t0 = t0; t->neu_tau = tau;
  } else if (kind == CEM_VELOCITY) {
    if (t->dir_set && (t->dir_law != law || t->dir_t0 != t0 || t->dir_tau != tau)) {
      err = "all Dirichlet loads share one time law";
      return CEM_ERR_ARG;
    }
    if ((comp_mask & 3) == 0) { err = "empty component mask"; return CEM_ERR_ARG; }
    for (int q = 0; q < n; ++q)
      if (items[q] < 0 || items[q] >= t->nn) { err = "bad node id"; return CEM_ERR_ARG; }
    for (int q = 0; q < n; ++q) {
      const int N = items[q];
      if (comp_mask & 1) { t->dmask[N] |= 1; t->Vp[N].x = a0; }
      if (comp_mask & 2) { t->dmask[N] |= 2; t->Vp[N].y = a0; }
    }
    t->dir_set = true; t->dir_law = law; t->dir_t0 = t0; t->dir_tau = tau;
  } else {
    err = "bad kind";
    return CEM_ERR_ARG;
  }
  t->loads_dirty = true;
  return CEM_OK;
}

cem_status tri_set_fields(TriMesh *t, int which, const void *data, long n_bytes, int on_device,
                          std::string &err) {
  if (t->step != 0) { err = "fields can only be set before the first step"; return CEM_ERR_STATE; }
  if (which != CEM_FIELD_U && which != CEM_FIELD_V) { err = "field not settable"; return CEM_ERR_ARG; }
  const long n = t->nn;
  if (n_bytes != 16 * n) { err = "expected " + std::to_string(16 * n) + " bytes"; return CEM_ERR_ARG; }
  // caller layout: x[n] then y[n]; device layout: interleaved
  std::vector<double> h(2 * n), il(2 * n);
  cudaSetDevice(t->device);
  if (cudaMemcpy(h.data(), data, 16 * n, on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost) != cudaSuccess) {
    err = "copy failed";
    return CEM_ERR_CUDA;
  }
  for (long N = 0; N < n; ++N) { il[2 * N] = h[N]; il[2 * N + 1] = h[n + N]; }
  cudaError_t ce;
  if (t->precision == CEM_FP32_MIXED) {
    if (which == CEM_FIELD_U) {
      // compensated pairs: hi = the nearest float, lo = the rest
      std::vector<float4> u4(n);
      for (long N = 0; N < n; ++N) {
        const float xh = (float)il[2 * N], yh = (float)il[2 * N + 1];
        u4[N] = make_float4(xh, (float)(il[2 * N] - (double)xh), yh, (float)(il[2 * N + 1] - (double)yh));
      }
      ce = cudaMemcpyAsync(t->d.u4, u4.data(), 16 * n, cudaMemcpyHostToDevice, t->st);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(t->st);
    } else {
      std::vector<float2> v2(n);
      for (long N = 0; N < n; ++N) v2[N] = make_float2((float)il[2 * N], (float)il[2 * N + 1]);
      ce = cudaMemcpyAsync(t->d.v2, v2.data(), 8 * n, cudaMemcpyHostToDevice, t->st);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(t->st);
    }
  } else {
    double2 *dst = which == CEM_FIELD_U ? t->d.u : t->d.v;
    ce = cudaMemcpyAsync(dst, il.data(), 16 * n, cudaMemcpyHostToDevice, t->st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(t->st);
  }
  if (ce != cudaSuccess) {
    err = "upload failed";
    return CEM_ERR_CUDA;
  }
  return CEM_OK;
}

cem_status tri_step(TriMesh *t, int n, std::string &err) {
  if (!t->material) { err = "cem_set_material must come first"; return CEM_ERR_STATE; }
  if (n < 0) { err = "negative step count"; return CEM_ERR_ARG; }
  if (n == 0) return CEM_OK;
  cudaSetDevice(t->device);
  if (t->loads_dirty) {
    if (!upload(t, const_cast<double2 *>(t->d.F), t->F) ||
        !upload(t, const_cast<double2 *>(t->d.Vp), t->Vp) ||
        !upload(t, const_cast<unsigned char *>(t->d.lflag), t->lflag) ||
        !upload(t, const_cast<unsigned char *>(t->d.dmask), t->dmask)) {
      err = "load upload failed";
      return CEM_ERR_CUDA;
    }
    t->loads_dirty = false;
  }
  const int ge = t->ge, gn = t->gn, gs = grid_of(t->ne);
  for (int q = 0; q < n; ++q) {
    const long s = t->step;
    const double dt = t->dt, tt = (double)s * dt;
    const bool energy = t->energy_every > 0 && s % t->energy_every == 0;
    const double lamN = t->neu_set ? law_eval(t->neu_law, tt, t->neu_t0, t->neu_tau) : 0.0;
    const double lamD = t->dir_set ? law_eval(t->dir_law, ((double)s + 0.5) * dt, t->dir_t0, t->dir_tau) : 0.0;
    const double dtv = s == 0 ? 0.5 * dt : dt;
    if (t->precision == CEM_FP32_MIXED) {
      k_tri_strain32<<<gs, kTB, 0, t->st>>>(t->d);
      k_tri_edge32<<<ge, kTB, 0, t->st>>>(t->d, energy ? 1 : 0);
      k_tri_node32<<<gn, kTB, 0, t->st>>>(t->d, lamN, lamD, dt, dtv, s == 0 ? 1 : 0, energy ? 1 : 0, ge);
    } else {
      k_tri_strain<<<gs, kTB, 0, t->st>>>(t->d);
      k_tri_edge<<<ge, kTB, 0, t->st>>>(t->d, energy ? 1 : 0);
      k_tri_node<<<gn, kTB, 0, t->st>>>(t->d, lamN, lamD, dt, dtv, s == 0 ? 1 : 0, energy ? 1 : 0, ge);
    }
    t->launches += 3;
    if (energy) {
      if (t->n_rec == t->rec_cap) {
        // grow the record array (rare): copy into one twice the size
        double *nr;
        if (!tri_alloc_n(t, nr, (size_t)t->rec_cap * 14) ||
            cudaMemcpyAsync(nr, t->d.rec, (size_t)t->rec_cap * 56, cudaMemcpyDeviceToDevice, t->st) != cudaSuccess) {
          err = "record allocation failed";
          return CEM_ERR_CUDA;
        }
        t->d.rec = nr;
        t->rec_cap *= 2;
      }
      k_tri_record<<<1, 32, 0, t->st>>>(t->d, ge, gn, ge, (int)t->n_rec, (double)s, tt);
      t->launches += 1;
      t->n_rec++;
    }
    t->step = s + 1;
  }
  cudaError_t ce = cudaGetLastError();
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(t->h_status, t->d.status, 4, cudaMemcpyDeviceToHost, t->st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(t->st);
  if (ce != cudaSuccess) { err = std::string("step failed: ") + cudaGetErrorString(ce); return CEM_ERR_CUDA; }
  if (*t->h_status) { err = "non-finite displacement or velocity"; return CEM_ERR_NONFINITE; }
  return CEM_OK;
}

cem_status tri_get_fields(TriMesh *t, int which, void *out, long n_bytes, int on_device,
                          std::string &err) {
  cudaSetDevice(t->device);
  const long n = t->nn;
  std::vector<double> h;
  if (which == CEM_FIELD_U || which == CEM_FIELD_V) {
    if (n_bytes < 16 * n) { err = "buffer too small"; return CEM_ERR_ARG; }
    std::vector<double> il(2 * n);
    cudaError_t ce;
    if (t->precision == CEM_FP32_MIXED && which == CEM_FIELD_U) {
      std::vector<float4> u4(n);
      ce = cudaMemcpyAsync(u4.data(), t->d.u4, 16 * n, cudaMemcpyDeviceToHost, t->st);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(t->st);
      for (long N = 0; N < n; ++N) {
        il[2 * N] = (double)u4[N].x + (double)u4[N].y;
        il[2 * N + 1] = (double)u4[N].z + (double)u4[N].w;
      }
    } else if (t->precision == CEM_FP32_MIXED) {
      std::vector<float2> v2(n);
      ce = cudaMemcpyAsync(v2.data(), t->d.v2, 8 * n, cudaMemcpyDeviceToHost, t->st);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(t->st);
      for (long N = 0; N < n; ++N) { il[2 * N] = v2[N].x; il[2 * N + 1] = v2[N].y; }
    } else {
      ce = cudaMemcpyAsync(il.data(), which == CEM_FIELD_U ? t->d.u : t->d.v, 16 * n,
                           cudaMemcpyDeviceToHost, t->st);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(t->st);
    }
    if (ce != cudaSuccess) {
      err = "copy failed";
      return CEM_ERR_CUDA;
    }
    h.resize(2 * n);
    for (long N = 0; N < n; ++N) { h[N] = il[2 * N]; h[n + N] = il[2 * N + 1]; }
  } else if (which == CEM_FIELD_MASS) {
    if (n_bytes < 8 * n) { err = "buffer too small"; return CEM_ERR_ARG; }
    h.resize(n);
    if (cudaMemcpyAsync(h.data(), t->d.m, 8 * n, cudaMemcpyDeviceToHost, t->st) != cudaSuccess ||
        cudaStreamSynchronize(t->st) != cudaSuccess) {
      err = "copy failed";
      return CEM_ERR_CUDA;
    }
  } else if (which == CEM_FIELD_ENERGY) {
    if (n_bytes < 56 * t->n_rec) { err = "buffer too small"; return CEM_ERR_ARG; }
    h.resize(7 * t->n_rec);
    if (t->n_rec &&
        (cudaMemcpyAsync(h.data(), t->d.rec, 56 * t->n_rec, cudaMemcpyDeviceToHost, t->st) != cudaSuccess ||
         cudaStreamSynchronize(t->st) != cudaSuccess)) {
      err = "copy failed";
      return CEM_ERR_CUDA;
    }
  } else {
    err = "field not available on a triangle mesh";
    return CEM_ERR_ARG;
  }
  if (h.empty()) return CEM_OK;
  if (cudaMemcpy(out, h.data(), h.size() * 8, on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost) != cudaSuccess) {
    err = "copy failed";
    return CEM_ERR_CUDA;
  }
  return CEM_OK;
}

cem_status tri_eval_surface(TriMesh *t, int n, const int *edge, const int *elem, double *G,
                            int *choice, std::string &err) {
  if (!t->material) { err = "cem_set_material must come first"; return CEM_ERR_STATE; }
  if (n < 0 || (n > 0 && (!edge || !elem || !G || !choice))) { err = "bad arguments"; return CEM_ERR_ARG; }
  if (n == 0) return CEM_OK;
  for (int q = 0; q < n; ++q) {
    const int g = edge[q], e = elem[q];
    if (g < 0 || g >= t->ned || e < 0 || e >= t->ne || (t->ee1[g] != e && t->ee2[g] != e)) {
      err = "point " + std::to_string(q) + ": not an edge of its element";
      return CEM_ERR_ARG;
    }
  }
  cudaSetDevice(t->device);
  int *dedge = nullptr, *delem = nullptr, *dch = nullptr;
  double *dG = nullptr;
  cudaError_t ce = cudaMallocAsync((void **)&dedge, 4L * n, t->st);
  if (ce == cudaSuccess) ce = cudaMallocAsync((void **)&delem, 4L * n, t->st);
  if (ce == cudaSuccess) ce = cudaMallocAsync((void **)&dch, 4L * n, t->st);
  if (ce == cudaSuccess) ce = cudaMallocAsync((void **)&dG, 16L * n, t->st);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(dedge, edge, 4L * n, cudaMemcpyHostToDevice, t->st);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(delem, elem, 4L * n, cudaMemcpyHostToDevice, t->st);
  if (ce == cudaSuccess) {
    k_tri_eval<<<grid_of(n), kTB, 0, t->st>>>(t->d, n, dedge, delem, t->d_gc, t->gamma,
                                              t->gamma_mode, dG, dch);
    ce = cudaGetLastError();
  }
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(G, dG, 16L * n, cudaMemcpyDeviceToHost, t->st);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(choice, dch, 4L * n, cudaMemcpyDeviceToHost, t->st);
  for (void *p : {(void *)dedge, (void *)delem, (void *)dch, (void *)dG})
    if (p) cudaFreeAsync(p, t->st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(t->st);
  if (ce != cudaSuccess) {
    err = std::string("evaluation failed: ") + cudaGetErrorString(ce);
    return CEM_ERR_CUDA;
  }
  t->launches += 1;
  return CEM_OK;
}

void tri_counts(const TriMesh *t, cem_counts *out) {
  std::memset(out, 0, sizeof *out);
  out->n_nodes = t->nn;
  out->n_elems = t->ne;
  out->n_active = t->ne;
  out->n_energy = t->n_rec;
  out->step = t->step;
  out->dt = t->dt;
  out->t = (double)t->step * t->dt;
  out->kernel_launches = t->launches;
}

}  // namespace cem
