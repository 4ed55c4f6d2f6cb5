// eval_fp32.cu -- surface-point evaluation of the FP32-mixed mode
// (compiled with -fmad=false so that its FP64 re-check uses the same
// operation order as the FP64 mode).
//
// Each free-surface point computes the energy release rate of its three
// candidate paths (Sec. 2.2) in FP32 from the compensated displacement.  If
// any candidate lies within 1e-3 of G_c (|G/G_c - 1| < 1e-3) the point is
// re-evaluated in FP64, so that the threshold decision is the FP64 one.  The
// Q4 cracking rule then runs on the (FP64-widened) values and proposals are
// appended with a warp ballot.
#include <cuda_runtime.h>

#include "cem_internal.h"
#include "eval_common.cuh"
#include "q4_fp64.cuh"

namespace cem {

namespace {

__device__ __forceinline__ float df_diff(float ah, float al, float bh, float bl) {
  return (bh - ah) + (bl - al);
}

// Own FP32 strain of an intact element at its edge k (Eq. 4 at the edge
// point), from its four nodes' displacement pairs in local order.
__device__ __forceinline__ void own_strain32(const Geo &g, const float4 (&q)[4], int k,
                                             float eps[3]) {
  float xh[4], xl[4], yh[4], yl[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    xh[a] = q[a].x; xl[a] = q[a].y; yh[a] = q[a].z; yl[a] = q[a].w;
  }
  const float rx = g.rxf, ry = g.ryf, hx2 = 0.5f * rx, hy2 = 0.5f * ry;
  float au = df_diff(xh[0], xl[0], xh[1], xl[1]), bu = df_diff(xh[3], xl[3], xh[2], xl[2]);
  float cu = df_diff(xh[0], xl[0], xh[3], xl[3]), eu = df_diff(xh[1], xl[1], xh[2], xl[2]);
  float av = df_diff(yh[0], yl[0], yh[1], yl[1]), bv = df_diff(yh[3], yl[3], yh[2], yl[2]);
  float cv = df_diff(yh[0], yl[0], yh[3], yl[3]), ev = df_diff(yh[1], yl[1], yh[2], yl[2]);
  switch (k) {
    case 0: eps[0] = rx * au; eps[1] = hy2 * (cv + ev); eps[2] = hy2 * (cu + eu) + rx * av; break;
    case 1: eps[0] = hx2 * (au + bu); eps[1] = ry * ev; eps[2] = ry * eu + hx2 * (av + bv); break;
    case 2: eps[0] = rx * bu; eps[1] = hy2 * (cv + ev); eps[2] = hy2 * (cu + eu) + rx * bv; break;
    default: eps[0] = hx2 * (au + bu); eps[1] = ry * cv; eps[2] = ry * cu + hx2 * (av + bv); break;
  }
}

// Everything the FP32 evaluation of surface point (e, k0) reads, loaded in
// one level: the displacement pairs of e's nodes, the states of its four
// neighbours, the two far nodes of each neighbour inside the mesh (across
// the edges other than k0) and G_c of e.
struct EvalPatch {
  float4 ue[4];     // e's nodes, local order
  float4 far[4][2]; // neighbour across edge k: its two nodes not on edge k
  int st[4];        // neighbour states (ST_OUT outside the mesh)
  float gc;
};

__device__ __forceinline__ void load_patch(const DevState &d, const U32x2 &U, int e, int k0,
                                           EvalPatch &P) {
  const Geo &g = d.g;
  const int i = e % g.nx, j = e / g.nx, r = g.nx + 1;
  const int n0 = j * r + i, n1 = n0 + 1, n2 = n0 + r + 1, n3 = n0 + r;
  const int nd[4] = {n0, n1, n2, n3};
  // far nodes of the neighbour below, right, above, left
  const int fa[4][2] = {{n0 - r, n1 - r}, {n1 + 1, n2 + 1}, {n2 + r, n3 + r}, {n0 - 1, n3 - 1}};
#pragma unroll
  for (int a = 0; a < 4; ++a) P.ue[a] = U.u[nd[a]];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int f = elem_neighbor(g, e, k);
    P.st[k] = estatus(d, f);
    const bool use = f >= 0 && k != k0;
    P.far[k][0] = use ? U.u[fa[k][0]] : make_float4(0.f, 0.f, 0.f, 0.f);
    P.far[k][1] = use ? U.u[fa[k][1]] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  P.gc = d.gc[e];
}

// The neighbour across edge k in its own local node order.
__device__ __forceinline__ void neighbour_nodes(const EvalPatch &P, int k, float4 (&q)[4]) {
  switch (k) {
    case 0: q[0] = P.far[0][0]; q[1] = P.far[0][1]; q[2] = P.ue[1]; q[3] = P.ue[0]; break;
    case 1: q[0] = P.ue[1]; q[1] = P.far[1][0]; q[2] = P.far[1][1]; q[3] = P.ue[2]; break;
    case 2: q[0] = P.ue[3]; q[1] = P.ue[2]; q[2] = P.far[2][0]; q[3] = P.far[2][1]; break;
    default: q[0] = P.far[3][0]; q[1] = P.ue[0]; q[2] = P.ue[3]; q[3] = P.far[3][1]; break;
  }
}

__device__ __forceinline__ void used_stress32(const DevState &d, const EvalPatch &P, int k,
                                              float s[3]) {
  float e1[3];
  own_strain32(d.g, P.ue, k, e1);
  if (P.st[k] == ST_INTACT) {
    float4 q[4];
    neighbour_nodes(P, k, q);
    float e2[3];
    own_strain32(d.g, q, (k + 2) & 3, e2);
    for (int c = 0; c < 3; ++c) e1[c] = 0.5f * (e1[c] + e2[c]);
  }
  const Mat &m = d.mat;
  s[0] = m.D11f * e1[0] + m.D12f * e1[1];
  s[1] = m.D12f * e1[0] + m.D11f * e1[1];
  s[2] = m.D33f * e1[2];
}

__device__ __forceinline__ void eval_G32(const DevState &d, const EvalPatch &P, int k0,
                                         float G[4]) {
  const Geo &g = d.g;
  const float DX = g.DXf[k0], DY = g.DYf[k0];
  float4 P1 = P.ue[0], P2 = P.ue[1];
#pragma unroll
  for (int a = 1; a < 4; ++a)
    if (a == k0) { P1 = P.ue[a]; P2 = P.ue[(a + 1) & 3]; }
  float dux = df_diff(P1.x, P1.y, P2.x, P2.y);
  float duy = df_diff(P1.z, P1.w, P2.z, P2.w);
  // |x_N2 - x_N1|^2 - |X_N2 - X_N1|^2 without cancellation
  float stretch = 2.f * (DX * dux + DY * duy) + (dux * dux + duy * duy);
  float H = stretch > 0.f ? 1.f : 0.f;
  float ddx = dux * H, ddy = duy * H;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (k == k0) { G[k] = -1.f; continue; }
    const float nx = g.nxf[k0][k], ny = g.nyf[k0][k];
    float s[3];
    used_stress32(d, P, k, s);
    float tx = s[0] * nx + s[2] * ny;
    float ty = s[2] * nx + s[1] * ny;
    G[k] = 0.5f * (ddx * tx + ddy * ty);
  }
}

// FP64 re-evaluation, out of line so that its FP64 instructions are not
// predicated into every surface point's FP32 evaluation.
__device__ __noinline__ void recheck64(const DevState &d, const float4 *u, int e, int k0,
                                       double *G) {
  const U32x2 U{u};
  eval_G64(d, U, e, k0, G);
}

__device__ __forceinline__ void eval32(const DevState &d, VBlk vb, int cur) {
  const int n = d.cnt->n_S;
  const U32x2 U{d.u4[cur]};
  for (int base = vb.x * blockDim.x; base < n; base += vb.gx * blockDim.x) {
    int i = base + threadIdx.x;
    bool has = false;
    int key = 0, edge = 0, kk = -1;
    double Gk = 0.0;
    if (i < n) {
      edge = d.S[i];
      const int info = d.S_info[i];
      if (edge >= 0) {
        key = info;
        int e = key >> 2, k0 = key & 3;
        if (d.mat.scope != 2 || is_tip_edge(d, e, k0)) {
          EvalPatch P;
          load_patch(d, U, e, k0, P);
          float G32[4];
          eval_G32(d, P, k0, G32);
          float gc = P.gc;
          bool near = false;
          for (int k = 0; k < 4; ++k)
            if (k != k0 && fabsf(G32[k] / gc - 1.f) < 1e-3f) near = true;
          double G[4];
          if (near) {
            recheck64(d, d.u4[cur], e, k0, G);  // FP64 re-check near the threshold
          } else {
            for (int k = 0; k < 4; ++k) G[k] = (double)G32[k];
          }
          double gm = -1.0;
          for (int k = 0; k < 4; ++k) gm = fmax(gm, G[k]);
          d.S_G[i] = gm;
          kk = q4_rule(d, e, k0, G);
          if (kk >= 0) { has = true; Gk = G[kk]; }
        }
      }
    }
    append_proposal(d, has, key, edge, kk, Gk);
  }
}

__global__ void __launch_bounds__(256, 4) k_eval32(DevState d, int cur) { eval32(d, hw_vblk(), cur); }

__global__ void __launch_bounds__(256, 4) k_eval32_batch(BatchDev b) {
  __shared__ DevState sd;
  int held = -1, w0, w1;
  const int n = *b.bstep;
  block_range(b.n_eval, w0, w1);
  for (int w = w0; w < w1; ++w) {
    const int4 it = b.w_eval[w];
    stage_member(b.ds, it.x, sd, held);
    if (!member_active(sd, n)) continue;
    eval32(sd, VBlk{it.y, 0, it.w, 1}, member_cur(sd, n));
  }
}

int grid_for(int n, int block, int maxb) {
  int b = (n + block - 1) / block;
  return b < 1 ? 1 : (b > maxb ? maxb : b);
}

}  // namespace

int grid_eval(const DevState &d) { return grid_for(d.list_cap, 256, 152); }

cudaError_t eval32_carveouts() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = match_tile_carveout(k_eval32);
  if (e == cudaSuccess) e = match_tile_carveout(k_eval32_batch);
  if (e == cudaSuccess) done = true;
  return e;
}

cudaError_t launch_eval32(const DevState &d, int cur, cudaStream_t st) {
  cudaError_t e = eval32_carveouts();
  if (e != cudaSuccess) return e;
  k_eval32<<<grid_eval(d), 256, 0, st>>>(d, cur);
  return cudaGetLastError();
}

cudaError_t launch_eval32_batch(const BatchDev &b, cudaStream_t st) {
  cudaError_t e = eval32_carveouts();
  if (e != cudaSuccess) return e;
  k_eval32_batch<<<grid_for(b.n_eval, 1, 1216), 256, 0, st>>>(b);
  return cudaGetLastError();
}

}  // namespace cem
