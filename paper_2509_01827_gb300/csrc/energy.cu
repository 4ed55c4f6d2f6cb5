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

__device__ __forceinline__ void energy_pre(const DevState &d) {
  Counters *c = d.cnt;
  int rec = c->n_rec;
  if (rec >= d.rec_cap) {
    if (threadIdx.x == 0) atomicOr(&c->status, STAT_CAPACITY);
    return;
  }
  double wn = 0.0, wd = 0.0, ud = 0.0;
  for (int q = threadIdx.x; q < d.n_bc; q += TB) {
    int N = d.bc_nodes[q];
    wn += d.Wn[N];
    wd += d.Wd[N];
  }
  int nck = c->n_ck;
  for (int q = threadIdx.x; q < nck; q += TB) ud += d.ck_ud[q];
  wn = block_sum(wn);
  wd = block_sum(wd);
  ud = block_sum(ud);
  if (threadIdx.x == 0) {
    double *r = d.erec + (size_t)rec * 7;
    r[0] = (double)c->step;
    r[1] = (double)c->step * d.mat.dt;
    r[4] = wn;
    r[5] = wd;
    r[6] = ud;
  }
}

__device__ __forceinline__ void energy_post(const DevState &d, int nparts) {
  Counters *c = d.cnt;
  int rec = c->n_rec;
  if (rec >= d.rec_cap) return;
  double ke = 0.0, se = 0.0;
  for (int q = threadIdx.x; q < nparts; q += TB) {
    ke += d.e_part[2 * q];
    se += d.e_part[2 * q + 1];
  }
  ke = block_sum(ke);
  se = block_sum(se);
  if (threadIdx.x == 0) {
    double *r = d.erec + (size_t)rec * 7;
    r[2] = ke;
    r[3] = se;
    c->n_rec = rec + 1;
  }
}


__global__ void __launch_bounds__(TB) k_energy_pre(DevState d) { energy_pre(d); }

__global__ void __launch_bounds__(TB) k_energy_post(DevState d, int nparts) {
  energy_post(d, nparts);
}

// batched counterparts: one CTA per member
__global__ void __launch_bounds__(TB) k_energy_pre_batch(BatchDev b) {
  __shared__ DevState sd;
  int held = -1;
  const int n = *b.bstep;
  for (int s = blockIdx.x; s < b.n; s += gridDim.x) {
    stage_member(b.ds, s, sd, held);
    if (!member_active(sd, n)) continue;
    energy_pre(sd);
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

int grid_for(int n, int block, int maxb) {
  int b = (n + block - 1) / block;
  return b < 1 ? 1 : (b > maxb ? maxb : b);
}

}  // namespace

cudaError_t launch_energy_pre(const DevState &d, cudaStream_t st) {
  k_energy_pre<<<1, TB, 0, st>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_energy_post(const DevState &d, int nparts, cudaStream_t st) {
  k_energy_post<<<1, TB, 0, st>>>(d, nparts);
  return cudaGetLastError();
}


cudaError_t launch_energy_pre_batch(const BatchDev &b, cudaStream_t st) {
  k_energy_pre_batch<<<b.n < 1216 ? b.n : 1216, TB, 0, st>>>(b);
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
