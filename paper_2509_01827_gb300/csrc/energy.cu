// energy.cu -- FP64 energy records, batched counter read-back and precision
// conversions (compiled with -fmad=false).
//
// An energy record at step n holds KE of the mid-step velocity
// vbar^n = (v^{n-1/2} + v^{n+1/2}) / 2, the strain energy of u^n (each
// element or piece owns A_p/4 of each of its edge points), the external and
// prescribed-velocity work done before step n, and the dissipated energy
// U_d = sum of G_c * segment length over the splits made before step n.
// Per-block partial sums are added in a fixed order, so records are
// reproducible run to run.
#include <cuda_runtime.h>

#include "cem_internal.h"
#include "q4_fp64.cuh"

namespace cem {

namespace {

constexpr int TB = 1024;

__device__ double block_sum(double v) {
  __shared__ double ws[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) ws[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  __syncthreads();
  return r;  // valid in thread 0
}

// Part b of the prologue: chunk b of the loaded/prescribed boundary nodes'
// work and of the splits' dissipated energy, summed by one block of EPRE_TB
// threads into e_pre[3b..3b+2].  The chunking depends only on the counts, so
// a mesh stepped alone and the same mesh in a batch add in the same order.
__device__ __forceinline__ void energy_pre_part(const DevState &d, int b) {
  Counters *c = d.cnt;
  if (c->n_rec >= d.rec_cap) {
    if (b == 0 && threadIdx.x == 0) atomicOr(&c->status, STAT_CAPACITY);
    return;
  }
  const int nbc = d.n_bc, nck = c->n_ck;
  const int kb = (nbc + EPRE - 1) / EPRE, kc = (nck + EPRE - 1) / EPRE;
  const int b0 = b * kb, b1 = min(nbc, b0 + kb), c0 = b * kc, c1 = min(nck, c0 + kc);
  double wn = 0.0, wd = 0.0, ud = 0.0;
  for (int q = b0 + threadIdx.x; q < b1; q += EPRE_TB) {
    const int N = d.bc_nodes[q];
    wn += d.Wn[N];
    wd += d.Wd[N];
  }
  for (int q = c0 + threadIdx.x; q < c1; q += EPRE_TB) ud += d.ck_ud[q];
  wn = block_sum(wn);
  wd = block_sum(wd);
  ud = block_sum(ud);
  if (threadIdx.x == 0) {
    d.e_pre[3 * b] = wn;
    d.e_pre[3 * b + 1] = wd;
    d.e_pre[3 * b + 2] = ud;
  }
}

// The record: step, time, the prologue's sums (work and dissipation before
// the step) and the step's kinetic and strain energy partials.
__device__ __forceinline__ void energy_post(const DevState &d, int nparts) {
  Counters *c = d.cnt;
  int rec = c->n_rec;
  if (rec >= d.rec_cap) return;
  double ke = 0.0, se = 0.0, wn = 0.0, wd = 0.0, ud = 0.0;
  for (int q = threadIdx.x; q < nparts; q += TB) {
    ke += d.e_part[2 * q];
    se += d.e_part[2 * q + 1];
  }
  if (threadIdx.x < EPRE) {
    wn = d.e_pre[3 * threadIdx.x];
    wd = d.e_pre[3 * threadIdx.x + 1];
    ud = d.e_pre[3 * threadIdx.x + 2];
  }
  ke = block_sum(ke);
  se = block_sum(se);
  wn = block_sum(wn);
  wd = block_sum(wd);
  ud = block_sum(ud);
  if (threadIdx.x == 0) {
    double *r = d.erec + (size_t)rec * 7;
    r[0] = (double)c->step;
    r[1] = (double)c->step * d.mat.dt;
    r[2] = ke;
    r[3] = se;
    r[4] = wn;
    r[5] = wd;
    r[6] = ud;
    c->n_rec = rec + 1;
  }
}


__global__ void __launch_bounds__(EPRE_TB) k_energy_pre(DevState d) {
  energy_pre_part(d, blockIdx.x);
}

__global__ void __launch_bounds__(TB) k_energy_post(DevState d, int nparts) {
  energy_post(d, nparts);
}

// batched counterparts: EPRE prologue parts per member; one CTA per member
// for the epilogue
__global__ void __launch_bounds__(EPRE_TB) k_energy_pre_batch(BatchDev b) {
  __shared__ DevState sd;
  int held = -1, w0, w1;
  const int n = *b.bstep;
  block_range(b.n * EPRE, w0, w1);
  for (int w = w0; w < w1; ++w) {
    stage_member(b.ds, w / EPRE, sd, held);
    if (!member_active(sd, n)) continue;
    energy_pre_part(sd, w % EPRE);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(TB) k_energy_post_batch(BatchDev b) {
  __shared__ DevState sd;
  int held = -1;
  const int n = *b.bstep;
  for (int s = blockIdx.x; s < b.n; s += gridDim.x) {
    stage_member(b.ds, s, sd, held);
    if (!member_active(sd, n)) continue;
    energy_post(sd, b.nparts[s]);
    __syncthreads();
  }
}


// copies every member's counters into out[n] (one read-back for the batch)
__global__ void k_gather_counters(BatchDev b, Counters *out) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < b.n; s += gridDim.x * blockDim.x)
    out[s] = *b.ds[s].cnt;
}

__global__ void k_f32_to_f64(DevState d, int cur, double *ux, double *uy, double *vx, double *vy,
                             int n) {
  for (int N = blockIdx.x * blockDim.x + threadIdx.x; N < n; N += gridDim.x * blockDim.x) {
    const float4 U = d.u4[cur][N];
    const float2 V = d.v2[N];
    if (ux) ux[N] = (double)U.x + (double)U.y;
    if (uy) uy[N] = (double)U.z + (double)U.w;
    if (vx) vx[N] = (double)V.x;
    if (vy) vy[N] = (double)V.y;
  }
}

__global__ void k_f64_to_f32(DevState d, int cur, const double *ux, const double *uy,
                             const double *vx, const double *vy, int n) {
  for (int N = blockIdx.x * blockDim.x + threadIdx.x; N < n; N += gridDim.x * blockDim.x) {
    float4 U = d.u4[cur][N];
    float2 V = d.v2[N];
    if (ux) {
      U.x = (float)ux[N];
      U.y = (float)(ux[N] - (double)U.x);
    }
    if (uy) {
      U.z = (float)uy[N];
      U.w = (float)(uy[N] - (double)U.z);
    }
    if (vx) V.x = (float)vx[N];
    if (vy) V.y = (float)vy[N];
    d.u4[cur][N] = U;
    d.v2[N] = V;
  }
}

// ---------------------------------------------------------- element stress
// Mean stress of every element, for the stress contour outputs of Sec. 4: an
// intact element averages over its four edge points the stress its internal
// force uses there (Eqs. 1-2: the own strains of both elements beside an
// edge averaged when both are intact, Eq. 4 at the edge midpoints); a split
// element weights its pieces' mean stresses by the piece areas; an inactive
// element gets 0.  Also the largest principal stress
// sigma1 = (sxx + syy)/2 + sqrt(((sxx - syy)/2)^2 + sxy^2).  FP64 in both
// precisions (the FP32-mixed displacement pairs are summed to doubles).
__device__ __forceinline__ void node_u(const DevState &d, int cur, int N, double &x, double &y) {
  if (d.precision == 0) {
    x = d.ux[cur][N];
    y = d.uy[cur][N];
  } else {
    const float4 U = d.u4[cur][N];
    x = (double)U.x + (double)U.y;
    y = (double)U.z + (double)U.w;
  }
}

__device__ __forceinline__ void elem_u(const DevState &d, int cur, int e, double u[4], double v[4]) {
  const int i = e % d.g.nx, j = e / d.g.nx, r = d.g.nx + 1;
  const int n4[4] = {j * r + i, j * r + i + 1, (j + 1) * r + i + 1, (j + 1) * r + i};
#pragma unroll
  for (int a = 0; a < 4; ++a) node_u(d, cur, n4[a], u[a], v[a]);
}

__global__ void k_element_stress(DevState d, int cur, double *sx, double *sy, double *sxy,
                                 double *s1) {
  const Geo &g = d.g;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < g.ne; e += gridDim.x * blockDim.x) {
    double m[3] = {0.0, 0.0, 0.0};
    const int st = d.estate[e];
    if (st == ST_INTACT) {
      double u[4], v[4], sig[4][3];
      elem_u(d, cur, e, u, v);
      const int i = e % g.nx, j = e / g.nx;
      for (int k = 0; k < 4; ++k) {
        double own[3];
        strain64_rt(g, k, u, v, own);
        const int f = k == 0 ? (j > 0 ? e - g.nx : -1)
                    : k == 1 ? (i < g.nx - 1 ? e + 1 : -1)
                    : k == 2 ? (j < g.ny - 1 ? e + g.nx : -1)
                             : (i > 0 ? e - 1 : -1);
        double ep[3];
        if (f >= 0 && d.estate[f] == ST_INTACT) {
          double uf[4], vf[4], of[3];
          elem_u(d, cur, f, uf, vf);
          strain64_rt(g, (k + 2) % 4, uf, vf, of);
          const double *p1 = e < f ? own : of, *p2 = e < f ? of : own;
          for (int c = 0; c < 3; ++c) ep[c] = 0.5 * p1[c] + 0.5 * p2[c];
        } else {
          for (int c = 0; c < 3; ++c) ep[c] = own[c];
        }
        stress64(d.mat, ep, sig[k]);
      }
      for (int c = 0; c < 3; ++c) m[c] = (((sig[0][c] + sig[1][c]) + sig[2][c]) + sig[3][c]) * 0.25;
    } else if (st == ST_CRACKED) {
      const int ck = d.crack_of[e];
      double mp[2][3];
      for (int p = 0; p < 2; ++p) {
        double u[4], v[4], sig[4][3];
        for (int a = 0; a < 4; ++a) node_u(d, cur, d.ck_node[ck * 8 + p * 4 + a], u[a], v[a]);
        for (int k = 0; k < 4; ++k) {
          double ep[3];
          strain64_rt(g, k, u, v, ep);
          stress64(d.mat, ep, sig[k]);
        }
        for (int c = 0; c < 3; ++c)
          mp[p][c] = (((sig[0][c] + sig[1][c]) + sig[2][c]) + sig[3][c]) * 0.25;
      }
      const double A0 = d.ck_Ap[ck * 2], A1 = d.ck_Ap[ck * 2 + 1];
      for (int c = 0; c < 3; ++c) m[c] = (A0 * mp[0][c] + A1 * mp[1][c]) / (A0 + A1);
    }
    sx[e] = m[0];
    sy[e] = m[1];
    sxy[e] = m[2];
    const double h = 0.5 * (m[0] - m[1]);
    s1[e] = 0.5 * (m[0] + m[1]) + sqrt(h * h + m[2] * m[2]);
  }
}

int grid_for(int n, int block, int maxb) {
  int b = (n + block - 1) / block;
  return b < 1 ? 1 : (b > maxb ? maxb : b);
}

}  // namespace

cudaError_t launch_element_stress(const DevState &d, int cur, double *out4, cudaStream_t st) {
  const int ne = d.g.ne;
  k_element_stress<<<grid_for(ne, 256, 4864), 256, 0, st>>>(d, cur, out4, out4 + ne, out4 + 2 * ne,
                                                           out4 + 3 * (size_t)ne);
  return cudaGetLastError();
}

cudaError_t energy_carveouts() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = match_tile_carveout(k_energy_pre);
  if (e == cudaSuccess) e = match_tile_carveout(k_energy_post);
  if (e == cudaSuccess) e = match_tile_carveout(k_energy_pre_batch);
  if (e == cudaSuccess) e = match_tile_carveout(k_energy_post_batch);
  if (e == cudaSuccess) done = true;
  return e;
}

cudaError_t launch_energy_pre(const DevState &d, cudaStream_t st) {
  cudaError_t e = energy_carveouts();
  if (e != cudaSuccess) return e;
  k_energy_pre<<<EPRE, EPRE_TB, 0, st>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_energy_post(const DevState &d, int nparts, cudaStream_t st) {
  k_energy_post<<<1, TB, 0, st>>>(d, nparts);
  return cudaGetLastError();
}


cudaError_t launch_energy_pre_batch(const BatchDev &b, cudaStream_t st) {
  cudaError_t e = energy_carveouts();
  if (e != cudaSuccess) return e;
  const int items = b.n * EPRE;
  k_energy_pre_batch<<<items < 1216 ? items : 1216, EPRE_TB, 0, st>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_energy_post_batch(const BatchDev &b, cudaStream_t st) {
  k_energy_post_batch<<<b.n < 1216 ? b.n : 1216, TB, 0, st>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_gather_counters(const BatchDev &b, Counters *out, cudaStream_t st) {
  k_gather_counters<<<grid_for(b.n, 128, 64), 128, 0, st>>>(b, out);
  return cudaGetLastError();
}


cudaError_t launch_fp32_to_fp64(const DevState &d, int cur, double *ux, double *uy, double *vx,
                                double *vy, int n, cudaStream_t st) {
  k_f32_to_f64<<<grid_for(n, 256, 1216), 256, 0, st>>>(d, cur, ux, uy, vx, vy, n);
  return cudaGetLastError();
}

cudaError_t launch_fp64_to_fp32(const DevState &d, int cur, const double *ux, const double *uy,
                                const double *vx, const double *vy, int n, cudaStream_t st) {
  k_f64_to_f32<<<grid_for(n, 256, 1216), 256, 0, st>>>(d, cur, ux, uy, vx, vy, n);
  return cudaGetLastError();
}

}  // namespace cem
