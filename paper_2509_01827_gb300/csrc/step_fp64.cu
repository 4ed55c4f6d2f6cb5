// step_fp64.cu -- FP64 explicit step kernels (compiled with -fmad=false).
//
// One step of the explicit MCT-2D-CEM (see include/cem.h):
//   k_pieces64   internal force of every split-element piece (Eq. 6 with the
//                piece area), own strain at each edge point (smoothing off);
//   k_main64     one CTA per 32x8 tile of real nodes: ES-FEM edge strains
//                (Eqs. 1, 2, 4) of the intact elements around the tile,
//                stresses, the node gather of intact and piece forces in
//                increasing element id, and the central-difference update
//                with lumped mass, Neumann and Dirichlet loads;
//   k_phantom64  the same gather and update for phantom nodes;
//   k_eval64     energy release rate of the candidate paths of every
//                free-surface point (Sec. 2.2) and the Q4 cracking rule; the
//                proposals are appended with a warp ballot.
#include <cuda_runtime.h>

#include <cfloat>

#include "cem_internal.h"
#include "q4_fp64.cuh"
#include "eval_common.cuh"

namespace cem {

namespace {

constexpr int TX = 32, TY = 8, NT = TX * TY;
constexpr int UXn = TX + 4, UYn = TY + 4;  // nodes [i0-2, i0+TX+1] x [j0-2, j0+TY+1]
constexpr int EXn = TX + 3, EYn = TY + 3;  // elements [i0-2, i0+TX] x [j0-2, j0+TY]
constexpr int HXn = TX + 1, HYn = TY + 2;  // horizontal edges [i0-1, i0+TX) x [j0-1, j0+TY]
constexpr int VXn = TX + 2, VYn = TY + 1;  // vertical edges [i0-1, i0+TX] x [j0-1, j0+TY)

__device__ __forceinline__ double dot3(const double e[3], const double s[3]) {
  return e[0] * s[0] + e[1] * s[1] + e[2] * s[2];
}

// Block-wide sum of two values into e_part[blockIdx * 2 + {0,1}] (fixed tree).
__device__ void block_sum2(double a, double b, double *out) {
  __shared__ double wa[32], wb[32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0) { wa[w] = a; wb[w] = b; }
  __syncthreads();
  if (w == 0) {
    a = lane < nw ? wa[lane] : 0.0;
    b = lane < nw ? wb[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (lane == 0) { out[0] = a; out[1] = b; }
  }
}

// Central-difference update of one node (real or phantom); mirrors the
// oracle's expression order exactly.
struct NodeOut {
  double ke;
};

__device__ __forceinline__ double update_node(const DevState &d, int N, int cur, bool first,
                                              double fintx, double finty, uint8_t nf,
                                              double lamN, double lamD) {
  const double dt = d.mat.dt;
  const double dtv = first ? 0.5 * dt : dt;
  bool loaded = (nf & NF_LOADED) != 0;
  double fex = loaded ? lamN * d.Fx[N] : 0.0;
  double fey = loaded ? lamN * d.Fy[N] : 0.0;
  double minv = d.minv[N];
  double ax = (fex - fintx) * minv;
  double ay = (fey - finty) * minv;
  double vxo = d.vx[N], vyo = d.vy[N];
  double vxn = vxo + dtv * ax;
  double vyn = vyo + dtv * ay;
  if (nf & NF_DIRX) vxn = lamD * d.Vx[N];
  if (nf & NF_DIRY) vyn = lamD * d.Vy[N];
  double vbx = first ? vxo : 0.5 * (vxo + vxn);
  double vby = first ? vyo : 0.5 * (vyo + vyn);
  if (loaded) d.Wn[N] = d.Wn[N] + dt * (fex * vbx + fey * vby);
  if (nf & (NF_DIRX | NF_DIRY)) {
    double m = d.m[N];
    double Rx = m * ((vxn - vxo) / dtv) - (fex - fintx);
    double Ry = m * ((vyn - vyo) / dtv) - (fey - finty);
    double w = 0.0;
    if (nf & NF_DIRX) w = w + Rx * vbx;
    if (nf & NF_DIRY) w = w + Ry * vby;
    d.Wd[N] = d.Wd[N] + dt * w;
  }
  d.vx[N] = vxn;
  d.vy[N] = vyn;
  // a non-finite velocity (NaN or Inf) is reported through the status word
  if (!(fabs(vxn) <= DBL_MAX) || !(fabs(vyn) <= DBL_MAX)) atomicOr(&d.cnt->status, STAT_NONFINITE);
  d.ux[cur ^ 1][N] = d.ux[cur][N] + dt * vxn;
  d.uy[cur ^ 1][N] = d.uy[cur][N] + dt * vyn;
  return 0.5 * (d.m[N] * (vbx * vbx + vby * vby));
}

__device__ __forceinline__ void load_factors(const DevState &d, double &lamN, double &lamD) {
  int idx = d.cnt->step - d.cnt->lam_base;
  lamN = d.lamN[idx];
  lamD = d.lamD[idx];
}

// ------------------------------------------------------------------ pieces
__device__ __forceinline__ void pieces64(const DevState &d, VBlk vb, int cur, int energy,
                                         int part_off) {
  const int n = 2 * d.cnt->n_ck;
  double se = 0.0;
  for (int t = vb.x * blockDim.x + threadIdx.x; t < n; t += vb.gx * blockDim.x) {
    int c = t >> 1, p = t & 1;
    double u[4], v[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      int N = d.ck_node[c * 8 + p * 4 + a];
      u[a] = d.ux[cur][N];
      v[a] = d.uy[cur][N];
    }
    double s[4][3], e[4][3];
    strain64<0>(d.g, u, v, e[0]);
    strain64<1>(d.g, u, v, e[1]);
    strain64<2>(d.g, u, v, e[2]);
    strain64<3>(d.g, u, v, e[3]);
#pragma unroll
    for (int k = 0; k < 4; ++k) stress64(d.mat, e[k], s[k]);
    double qA = d.ck_Ap[c * 2 + p] * 0.25;
    double *f = d.pf + c * 16 + p * 8;
    node_force64<0>(d.g, s, qA, f[0], f[1]);
    node_force64<1>(d.g, s, qA, f[2], f[3]);
    node_force64<2>(d.g, s, qA, f[4], f[5]);
    node_force64<3>(d.g, s, qA, f[6], f[7]);
    if (energy) {
      double acc = 0.0;
#pragma unroll
      for (int k = 0; k < 4; ++k) acc = acc + 0.5 * (qA * dot3(e[k], s[k]));
      se += acc;
    }
  }
  if (energy) block_sum2(0.0, se, d.e_part + 2 * (part_off + vb.x));
}

__global__ void k_pieces64(DevState d, int cur, int energy, int part_off) {
  pieces64(d, hw_vblk(), cur, energy, part_off);
}

// -------------------------------------------------------------- main tile
__device__ __forceinline__ void main64_tile(const DevState &d, VBlk vb, int cur, int first,
                                            int energy) {
  __shared__ double sux[UYn][UXn], suy[UYn][UXn];
  __shared__ uint8_t sst[EYn][EXn];
  // stress (3) and eps.sigma (1) used by the element below/left (lo) and
  // above/right (hi) of each edge
  __shared__ double hlo[HYn][HXn][4], hhi[HYn][HXn][4];
  __shared__ double vlo[VYn][VXn][4], vhi[VYn][VXn][4];

  const Geo &g = d.g;
  const int i0 = vb.x * TX, j0 = vb.y * TY;
  const int tid = threadIdx.x;
  const double *uxc = d.ux[cur], *uyc = d.uy[cur];

  for (int q = tid; q < UXn * UYn; q += NT) {
    int li = q % UXn, lj = q / UXn, i = i0 - 2 + li, j = j0 - 2 + lj;
    double a = 0.0, b = 0.0;
    if (i >= 0 && j >= 0 && i <= g.nx && j <= g.ny) {
      int N = j * (g.nx + 1) + i;
      a = uxc[N];
      b = uyc[N];
    }
    sux[lj][li] = a;
    suy[lj][li] = b;
  }
  for (int q = tid; q < EXn * EYn; q += NT) {
    int li = q % EXn, lj = q / EXn, i = i0 - 2 + li, j = j0 - 2 + lj;
    uint8_t s = ST_OUT;
    if (i >= 0 && j >= 0 && i < g.nx && j < g.ny) s = d.estate[j * g.nx + i];
    sst[lj][li] = s;
  }
  __syncthreads();

  // element (ei, ej) -> its four nodes' displacements from shared memory
  auto gather = [&](int ei, int ej, double u[4], double v[4]) {
    int li = ei - (i0 - 2), lj = ej - (j0 - 2);
    u[0] = sux[lj][li];         v[0] = suy[lj][li];
    u[1] = sux[lj][li + 1];     v[1] = suy[lj][li + 1];
    u[2] = sux[lj + 1][li + 1]; v[2] = suy[lj + 1][li + 1];
    u[3] = sux[lj + 1][li];     v[3] = suy[lj + 1][li];
  };
  auto est = [&](int ei, int ej) -> int { return sst[ej - (j0 - 2)][ei - (i0 - 2)]; };

  // horizontal edges: below element (i, j-1) at its edge 2, above (i, j) at edge 0
  for (int q = tid; q < HXn * HYn; q += NT) {
    int li = q % HXn, lj = q / HXn, i = i0 - 1 + li, j = j0 - 1 + lj;
    int sb = est(i, j - 1), sa = est(i, j);
    double eb[3], ea[3], u[4], v[4];
    if (sb == ST_INTACT) { gather(i, j - 1, u, v); strain64<2>(g, u, v, eb); }
    if (sa == ST_INTACT) { gather(i, j, u, v); strain64<0>(g, u, v, ea); }
    if (sb == ST_INTACT && sa == ST_INTACT) {
      double e[3], s[3];
      for (int c = 0; c < 3; ++c) e[c] = 0.5 * eb[c] + 0.5 * ea[c];
      stress64(d.mat, e, s);
      double dd = dot3(e, s);
      for (int c = 0; c < 3; ++c) { hlo[lj][li][c] = s[c]; hhi[lj][li][c] = s[c]; }
      hlo[lj][li][3] = dd;
      hhi[lj][li][3] = dd;
    } else {
      if (sb == ST_INTACT) {
        double s[3];
        stress64(d.mat, eb, s);
        for (int c = 0; c < 3; ++c) hlo[lj][li][c] = s[c];
        hlo[lj][li][3] = dot3(eb, s);
      }
      if (sa == ST_INTACT) {
        double s[3];
        stress64(d.mat, ea, s);
        for (int c = 0; c < 3; ++c) hhi[lj][li][c] = s[c];
        hhi[lj][li][3] = dot3(ea, s);
      }
    }
  }
  // vertical edges: left element (i-1, j) at its edge 1, right (i, j) at edge 3
  for (int q = tid; q < VXn * VYn; q += NT) {
    int li = q % VXn, lj = q / VXn, i = i0 - 1 + li, j = j0 - 1 + lj;
    int sl = est(i - 1, j), sr = est(i, j);
    double el[3], er[3], u[4], v[4];
    if (sl == ST_INTACT) { gather(i - 1, j, u, v); strain64<1>(g, u, v, el); }
    if (sr == ST_INTACT) { gather(i, j, u, v); strain64<3>(g, u, v, er); }
    if (sl == ST_INTACT && sr == ST_INTACT) {
      double e[3], s[3];
      for (int c = 0; c < 3; ++c) e[c] = 0.5 * el[c] + 0.5 * er[c];
      stress64(d.mat, e, s);
      double dd = dot3(e, s);
      for (int c = 0; c < 3; ++c) { vlo[lj][li][c] = s[c]; vhi[lj][li][c] = s[c]; }
      vlo[lj][li][3] = dd;
      vhi[lj][li][3] = dd;
    } else {
      if (sl == ST_INTACT) {
        double s[3];
        stress64(d.mat, el, s);
        for (int c = 0; c < 3; ++c) vlo[lj][li][c] = s[c];
        vlo[lj][li][3] = dot3(el, s);
      }
      if (sr == ST_INTACT) {
        double s[3];
        stress64(d.mat, er, s);
        for (int c = 0; c < 3; ++c) vhi[lj][li][c] = s[c];
        vhi[lj][li][3] = dot3(er, s);
      }
    }
  }
  __syncthreads();

  // stresses used by intact element (ei, ej) at its edges 0..3
  auto elem_sig = [&](int ei, int ej, double s[4][3]) {
    int hi_ = ei - (i0 - 1), hj = ej - (j0 - 1);
    for (int c = 0; c < 3; ++c) {
      s[0][c] = hhi[hj][hi_][c];      // bottom edge h(ei, ej): element above it
      s[1][c] = vlo[hj][hi_ + 1][c];  // right edge v(ei+1, ej): element left of it
      s[2][c] = hlo[hj + 1][hi_][c];  // top edge h(ei, ej+1): element below it
      s[3][c] = vhi[hj][hi_][c];      // left edge v(ei, ej): element right of it
    }
  };

  const int tx = tid % TX, ty = tid / TX;
  const int i = i0 + tx, j = j0 + ty;
  double ke = 0.0, se = 0.0;
  if (i <= g.nx && j <= g.ny) {
    const int N = j * (g.nx + 1) + i;
    const double qA = g.A * 0.25;
    double fx = 0.0, fy = 0.0;
    // adjacent elements in increasing id: (i-1,j-1) a=2, (i,j-1) a=3, (i-1,j) a=1, (i,j) a=0
    const int ei[4] = {i - 1, i, i - 1, i}, ej[4] = {j - 1, j - 1, j, j}, la[4] = {2, 3, 1, 0};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int s = est(ei[q], ej[q]);
      if (s == ST_INTACT) {
        double sg[4][3], ax, ay;
        elem_sig(ei[q], ej[q], sg);
        node_force64_rt(g, la[q], sg, qA, ax, ay);
        fx = fx + ax;
        fy = fy + ay;
      } else if (s == ST_CRACKED) {
        int e = ej[q] * g.nx + ei[q];
        int c = d.crack_of[e];
        int side = (d.ck_info[c] >> (4 + la[q])) & 1;
        fx = fx + d.pf[c * 16 + side * 8 + 2 * la[q]];
        fy = fy + d.pf[c * 16 + side * 8 + 2 * la[q] + 1];
      }
    }
    double lamN, lamD;
    load_factors(d, lamN, lamD);
    ke = update_node(d, N, cur, first != 0, fx, fy, d.nflag[N], lamN, lamD);
    if (energy && i < g.nx && j < g.ny && est(i, j) == ST_INTACT) {
      int hi_ = i - (i0 - 1), hj = j - (j0 - 1);
      double dk[4] = {hhi[hj][hi_][3], vlo[hj][hi_ + 1][3], hlo[hj + 1][hi_][3], vhi[hj][hi_][3]};
      double acc = 0.0;
#pragma unroll
      for (int k = 0; k < 4; ++k) acc = acc + 0.5 * (qA * dk[k]);
      se = acc;
    }
  }
  if (energy) {
    int b = vb.y * vb.gx + vb.x;
    block_sum2(ke, se, d.e_part + 2 * b);
  }
}

__global__ void __launch_bounds__(NT) k_main64(DevState d, int cur, int first, int energy) {
  main64_tile(d, hw_vblk(), cur, first, energy);
}

// ---------------------------------------------------------------- phantoms
__device__ __forceinline__ void phantom64(const DevState &d, VBlk vb, int cur, int first,
                                          int energy, int part_off) {
  const int n = d.cnt->n_ph;
  double ke = 0.0;
  double lamN, lamD;
  load_factors(d, lamN, lamD);
  for (int t = vb.x * blockDim.x + threadIdx.x; t < n; t += vb.gx * blockDim.x) {
    int N = d.g.nn + t;
    // users' piece-force indices in increasing element id, -1 unused
    const int4 uf = reinterpret_cast<const int4 *>(d.ph_upf)[t];
    const int us[4] = {uf.x, uf.y, uf.z, uf.w};
    double fx = 0.0, fy = 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (us[q] < 0) break;
      fx = fx + d.pf[us[q]];
      fy = fy + d.pf[us[q] + 1];
    }
    ke += update_node(d, N, cur, first != 0, fx, fy, 0, lamN, lamD);
  }
  if (energy) block_sum2(ke, 0.0, d.e_part + 2 * (part_off + vb.x));
}

__global__ void k_phantom64(DevState d, int cur, int first, int energy, int part_off) {
  phantom64(d, hw_vblk(), cur, first, energy, part_off);
}

__device__ __forceinline__ void eval64(const DevState &d, VBlk vb, int cur) {
  const int n = d.cnt->n_S;
  const U64 U{d.ux[cur], d.uy[cur]};
  // whole warps iterate together so that the ballot sees every lane
  for (int base = vb.x * blockDim.x; base < n; base += vb.gx * blockDim.x) {
    int i = base + threadIdx.x;
    bool has = false;
    int key = 0, edge = 0, kk = -1;
    double Gk = 0.0;
    if (i < n) {
      edge = d.S[i];
      if (edge >= 0) {
        key = d.S_info[i];
        int e = key >> 2, k0 = key & 3;
        if (d.mat.scope != 2 || is_tip_edge(d, e, k0)) {
          double G[4];
          eval_G64(d, U, e, k0, G);
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

__global__ void k_eval64(DevState d, int cur) { eval64(d, hw_vblk(), cur); }

// ---------------------------------------------------------------- batched
// One launch per kernel kind for every member of a batch (persistent grids
// walking the work lists; 1-D items are (member, block, energy-partial
// offset, member's grid size)).
__global__ void __launch_bounds__(NT) k_main64_batch(BatchDev b, int first, int energy) {
  __shared__ DevState sd;
  int held = -1, w0, w1;
  const int n = *b.bstep;
  block_range(b.n_main, w0, w1);
  for (int w = w0; w < w1; ++w) {
    const int4 it = b.w_main[w];
    stage_member(b.ds, it.x, sd, held);
    if (!member_active(sd, n)) continue;
    main64_tile(sd, item_vblk(it), member_cur(sd, n), first, energy);
    __syncthreads();
  }
}

__global__ void k_pieces64_batch(BatchDev b, int energy) {
  __shared__ DevState sd;
  int held = -1, w0, w1;
  const int n = *b.bstep;
  block_range(b.n_pieces, w0, w1);
  for (int w = w0; w < w1; ++w) {
    const int4 it = b.w_pieces[w];
    stage_member(b.ds, it.x, sd, held);
    if (!member_active(sd, n)) continue;
    pieces64(sd, VBlk{it.y, 0, it.w, 1}, member_cur(sd, n), energy, it.z);
    __syncthreads();
  }
}

__global__ void k_phantom64_batch(BatchDev b, int first, int energy) {
  __shared__ DevState sd;
  int held = -1, w0, w1;
  const int n = *b.bstep;
  block_range(b.n_ph, w0, w1);
  for (int w = w0; w < w1; ++w) {
    const int4 it = b.w_ph[w];
    stage_member(b.ds, it.x, sd, held);
    if (!member_active(sd, n)) continue;
    phantom64(sd, VBlk{it.y, 0, it.w, 1}, member_cur(sd, n), first, energy, it.z);
    __syncthreads();
  }
}

__global__ void k_eval64_batch(BatchDev b) {
  __shared__ DevState sd;
  int held = -1, w0, w1;
  const int n = *b.bstep;
  block_range(b.n_eval, w0, w1);
  for (int w = w0; w < w1; ++w) {
    const int4 it = b.w_eval[w];
    stage_member(b.ds, it.x, sd, held);
    if (!member_active(sd, n)) continue;
    eval64(sd, VBlk{it.y, 0, it.w, 1}, member_cur(sd, n));
    __syncthreads();
  }
}

// ------------------------------------------------------------- init masses
__global__ void k_init_masses(DevState d) {
  const Geo &g = d.g;
  for (int N = blockIdx.x * blockDim.x + threadIdx.x; N < g.nn; N += gridDim.x * blockDim.x) {
    int r = g.nx + 1, i = N % r, j = N / r;
    const int di[4] = {-1, 0, -1, 0}, dj[4] = {-1, -1, 0, 0};
    double acc = 0.0;
    for (int q = 0; q < 4; ++q) {
      int ei = i + di[q], ej = j + dj[q];
      if (ei < 0 || ej < 0 || ei >= g.nx || ej >= g.ny) continue;
      if (d.estate[ej * g.nx + ei] == ST_INTACT) acc = acc + d.mat.rho * g.A * 0.25;
    }
    d.m[N] = acc;
    d.minv[N] = acc > 0.0 ? 1.0 / acc : 0.0;
  }
}

int grid_for(int n, int block, int maxb) {
  int b = (n + block - 1) / block;
  return b < 1 ? 1 : (b > maxb ? maxb : b);
}

}  // namespace

int energy_parts_fp32(const DevState &d);

int tiles_fp64(const DevState &d) {
  return ((d.g.nx + 1 + TX - 1) / TX) * ((d.g.ny + 1 + TY - 1) / TY);
}

int energy_parts_needed(const DevState &d) {
  if (d.precision == 1) return energy_parts_fp32(d);
  return tiles_fp64(d) + 2 * 1216 + 8;
}

int energy_parts_step_fp32(const DevState &d, int tile_rows);
int march_rows_solo(const DevState &d);

int energy_parts_step(const DevState &d) {
  if (d.precision == 1) return energy_parts_step_fp32(d, march_rows_solo(d));
  return tiles_fp64(d) + grid_pieces(d) + grid_phantoms(d);
}

cudaError_t launch_init_masses(const DevState &d, cudaStream_t st) {
  k_init_masses<<<grid_for(d.g.nn, 256, 4096), 256, 0, st>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_step_fp64(const DevState &d, int cur, bool first, bool energy,
                             const StepStreams &ss, cudaEvent_t *marks) {
  dim3 grid((d.g.nx + 1 + TX - 1) / TX, (d.g.ny + 1 + TY - 1) / TY);
  int tiles = grid.x * grid.y;
  int gp = grid_pieces(d);
  int gph = grid_phantoms(d);
  const int ge = grid_eval(d);
  cudaStream_t st = ss.main;
  if (marks) {
    k_pieces64<<<gp, 256, 0, st>>>(d, cur, energy ? 1 : 0, tiles);
    cudaEventRecord(marks[0], st);
    k_main64<<<grid, NT, 0, st>>>(d, cur, first ? 1 : 0, energy ? 1 : 0);
    cudaEventRecord(marks[1], st);
    k_phantom64<<<gph, 256, 0, st>>>(d, cur, first ? 1 : 0, energy ? 1 : 0, tiles + gp);
    cudaEventRecord(marks[2], st);
    k_eval64<<<ge, 256, 0, st>>>(d, cur);
    return cudaGetLastError();
  }
  cudaEventRecord(ss.fork, st);
  cudaStreamWaitEvent(ss.aux2, ss.fork, 0);
  k_eval64<<<ge, 256, 0, ss.aux2>>>(d, cur);
  launch_select(d, TRACK_STEP, ss.aux2);
  k_pieces64<<<gp, 256, 0, st>>>(d, cur, energy ? 1 : 0, tiles);
  cudaEventRecord(ss.fork, st);
  cudaStreamWaitEvent(ss.aux1, ss.fork, 0);
  k_phantom64<<<gph, 256, 0, ss.aux1>>>(d, cur, first ? 1 : 0, energy ? 1 : 0, tiles + gp);
  k_main64<<<grid, NT, 0, st>>>(d, cur, first ? 1 : 0, energy ? 1 : 0);
  cudaEventRecord(ss.join1, ss.aux1);
  cudaEventRecord(ss.join2, ss.aux2);
  cudaStreamWaitEvent(st, ss.join1, 0);
  cudaStreamWaitEvent(st, ss.join2, 0);
  return cudaGetLastError();
}

// The same fork/join as launch_step_fp64, one launch per kernel kind for all
// members of the batch.
cudaError_t launch_step_fp64_batch(const BatchDev &b, bool first, bool energy, int grid_main,
                                   const StepStreams &ss) {
  const int gm = grid_main < 1 ? 1 : grid_main;
  const int gp = grid_for(b.n_pieces, 1, 1216), gph = grid_for(b.n_ph, 1, 1216);
  const int ge = grid_for(b.n_eval, 1, 1216);
  cudaStream_t st = ss.main;
  cudaEventRecord(ss.fork, st);
  cudaStreamWaitEvent(ss.aux2, ss.fork, 0);
  k_eval64_batch<<<ge, 256, 0, ss.aux2>>>(b);
  cudaError_t e = launch_select_batch(b, ss.aux2);
  if (e != cudaSuccess) return e;
  k_pieces64_batch<<<gp, 256, 0, st>>>(b, energy ? 1 : 0);
  cudaEventRecord(ss.fork, st);
  cudaStreamWaitEvent(ss.aux1, ss.fork, 0);
  k_phantom64_batch<<<gph, 256, 0, ss.aux1>>>(b, first ? 1 : 0, energy ? 1 : 0);
  k_main64_batch<<<gm, NT, 0, st>>>(b, first ? 1 : 0, energy ? 1 : 0);
  cudaEventRecord(ss.join1, ss.aux1);
  cudaEventRecord(ss.join2, ss.aux2);
  cudaStreamWaitEvent(st, ss.join1, 0);
  cudaStreamWaitEvent(st, ss.join2, 0);
  return cudaGetLastError();
}

const void *phantom64_kernel() { return reinterpret_cast<const void *>(&k_phantom64); }

}  // namespace cem
