// step_fp32.cu -- FP32-mixed explicit step: FP32 element arithmetic,
// displacement kept as a compensated pair of floats (hi + lo, ~48-bit
// mantissa) and advanced with an error-free two-sum, FP64 energy sums.
//
// k_main32 is the kernel that touches every real node each step (its HBM
// floor is 54 bytes per node; the shared-memory stencil traffic bounds it in
// practice).  For each node it forms the strains at the midpoints of
// the 12 edges around it from node differences (Eq. 4 at the edge points):
// along an edge the tangential derivative is the difference of its two
// nodes, across it the normal derivative of each side is the sum of that
// side's two across-edge differences; with two intact neighbours the two
// sides are averaged (Eqs. 1-2 with equal areas), otherwise each intact side
// keeps its own strain; sigma = D eps per side (zero for split or missing
// sides); the node force is B^T sigma A/4 (Eq. 6) summed over those edges
// and sides, plus the forces of split-element pieces (evaluated in the tile
// from the pieces' nodes); then the central-difference update.  k_phantom32
// updates the phantom nodes, evaluating each user piece at the phantom; the
// two run side by side with the surface evaluation and the selection.
#include <cuda_runtime.h>

#include <cfloat>

#include "cem_internal.h"
#include "q4_fp64.cuh"

namespace cem {

namespace {


// Per-warp sums of the phantom update's kinetic energy, written to
// out[2w], out[2w + 1] for warp w of the block (fixed order, no shared
// memory: a kernel with static shared memory gets its own L1 / shared split
// and could not share SMs with the tile update).
__device__ __forceinline__ void warp_sum_parts(double a, double *out) {
  for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) {
    out[2 * (threadIdx.x >> 5)] = a;
    out[2 * (threadIdx.x >> 5) + 1] = 0.0;
  }
}

__device__ __forceinline__ void block_sum2(double a, double b, double *out) {
  __shared__ double wa[32], wb[32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int t = threadIdx.x + threadIdx.y * blockDim.x;  // 1-D or 2-D blocks
  int lane = t & 31, w = t >> 5, nw = (blockDim.x * blockDim.y + 31) >> 5;
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

// (hi, lo) += x with an error-free transformation (Knuth two-sum) and
// renormalisation, so the pair keeps about 48 significant bits.
__device__ __forceinline__ void df_add(float &hi, float &lo, float x) {
  float s = __fadd_rn(hi, x);
  float bb = __fsub_rn(s, hi);
  float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
  float l = __fadd_rn(lo, err);
  float h = __fadd_rn(s, l);
  lo = __fsub_rn(l, __fsub_rn(h, s));
  hi = h;
}

__device__ __forceinline__ float df_diff(float ah, float al, float bh, float bl) {
  return (bh - ah) + (bl - al);  // (b - a)
}

struct Stress3 {
  float xx, yy, xy;
};

__device__ __forceinline__ Stress3 stress32(const Mat &m, float exx, float eyy, float gxy) {
  Stress3 s;
  s.xx = fmaf(m.D11f, exx, m.D12f * eyy);
  s.yy = fmaf(m.D12f, exx, m.D11f * eyy);
  s.xy = m.D33f * gxy;
  return s;
}


// Central-difference update of a node that carries a load, a prescribed
// velocity, or whose kinetic energy is recorded this step.  Kept out of line:
// if it were inlined, the compiler could predicate its FP64 instructions into
// the update of every node, and on this GPU the FP64 pipe is 1/64 of FP32.
__device__ __noinline__ double update_special(const DevState &d, int N, int cur, int first,
                                              float fx, float fy, float4 U, float2 vo, float minv,
                                              int nf, int energy) {
  const int idx = d.cnt->step - d.cnt->lam_base;
  const double lamN = d.lamN[idx], lamD = d.lamD[idx];
  const float dt = d.mat.dtf;
  const float dtv = first ? 0.5f * dt : dt;
  float fex = 0.f, fey = 0.f;
  if (nf & NF_LOADED) {
    fex = (float)(lamN * d.Fx[N]);
    fey = (float)(lamN * d.Fy[N]);
  }
  const float vxo = vo.x, vyo = vo.y;
  float vxn = fmaf(dtv, (fex - fx) * minv, vxo);
  float vyn = fmaf(dtv, (fey - fy) * minv, vyo);
  if (nf & NF_DIRX) vxn = (float)(lamD * d.Vx[N]);
  if (nf & NF_DIRY) vyn = (float)(lamD * d.Vy[N]);
  const double vbx = first ? (double)vxo : 0.5 * ((double)vxo + (double)vxn);
  const double vby = first ? (double)vyo : 0.5 * ((double)vyo + (double)vyn);
  const double dtd = d.mat.dt;
  if (nf & NF_LOADED) d.Wn[N] += dtd * ((double)fex * vbx + (double)fey * vby);
  if (nf & (NF_DIRX | NF_DIRY)) {
    const double m = d.m[N];
    const double dv = first ? 0.5 * dtd : dtd;
    const double Rx = m * (((double)vxn - (double)vxo) / dv) - ((double)fex - (double)fx);
    const double Ry = m * (((double)vyn - (double)vyo) / dv) - ((double)fey - (double)fy);
    double w = 0.0;
    if (nf & NF_DIRX) w += Rx * vbx;
    if (nf & NF_DIRY) w += Ry * vby;
    d.Wd[N] += dtd * w;
  }
  d.v2[N] = make_float2(vxn, vyn);
  if (!(fabsf(vxn) <= FLT_MAX) || !(fabsf(vyn) <= FLT_MAX)) atomicOr(&d.cnt->status, STAT_NONFINITE);
  df_add(U.x, U.y, dt * vxn);
  df_add(U.z, U.w, dt * vyn);
  d.u4[cur ^ 1][N] = U;
  return energy ? 0.5 * (d.m[N] * (vbx * vbx + vby * vby)) : 0.0;
}

// Update of a node without loads: FP32 only.
__device__ __forceinline__ float2 update_plain(const DevState &d, int N, int cur, float dtv,
                                               float dt, float fx, float fy, float4 U, float2 vo,
                                               float minv) {
  const float vxn = fmaf(dtv, -fx * minv, vo.x);
  const float vyn = fmaf(dtv, -fy * minv, vo.y);
  d.v2[N] = make_float2(vxn, vyn);
  // a non-finite velocity (NaN or Inf) is reported through the status word
  if (!(fabsf(vxn) <= FLT_MAX) || !(fabsf(vyn) <= FLT_MAX)) atomicOr(&d.cnt->status, STAT_NONFINITE);
  df_add(U.x, U.y, dt * vxn);
  df_add(U.z, U.w, dt * vyn);
  d.u4[cur ^ 1][N] = U;
  return make_float2(vxn, vyn);
}

// ------------------------------------------------------------------ pieces
// One piece of split element c (side p): strains and stresses at its four
// edge points (Eq. 4 at the edge midpoints, from the displacements of the
// piece's own nodes) and its nodal forces f[2a], f[2a+1] at local nodes
// a = 0..3, FP32.  The tile kernel (forces at real nodes), the phantom
// update (forces at phantom nodes) and the piece kernel (every force; the
// profiling path) all evaluate pieces here, so a force is the same wherever
// it is used.
struct Piece32 {
  float ex[4], ey[4], gx[4];
  Stress3 s[4];
  float qA;
  float f[8];
};

__device__ __forceinline__ void piece32_state(const DevState &d, int c, int p, int cur,
                                              Piece32 &P) {
  const Geo &g = d.g;
  const float rx = g.rxf, ry = g.ryf;
  const float hx2 = 0.5f * rx, hy2 = 0.5f * ry;
  const int4 nd = reinterpret_cast<const int4 *>(d.ck_node)[c * 2 + p];
  const int nds[4] = {nd.x, nd.y, nd.z, nd.w};
  float xh[4], xl[4], yh[4], yl[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const float4 U = d.u4[cur][nds[a]];
    xh[a] = U.x; xl[a] = U.y; yh[a] = U.z; yl[a] = U.w;
  }
  // edge differences: a = u1-u0 (bottom), b = u2-u3 (top), c = u3-u0 (left), e = u2-u1 (right)
  float au = df_diff(xh[0], xl[0], xh[1], xl[1]), bu = df_diff(xh[3], xl[3], xh[2], xl[2]);
  float cu = df_diff(xh[0], xl[0], xh[3], xl[3]), eu = df_diff(xh[1], xl[1], xh[2], xl[2]);
  float av = df_diff(yh[0], yl[0], yh[1], yl[1]), bv = df_diff(yh[3], yl[3], yh[2], yl[2]);
  float cv = df_diff(yh[0], yl[0], yh[3], yl[3]), ev = df_diff(yh[1], yl[1], yh[2], yl[2]);
  P.ex[0] = rx * au;          P.ey[0] = hy2 * (cv + ev); P.gx[0] = fmaf(hy2, cu + eu, rx * av);
  P.ex[1] = hx2 * (au + bu);  P.ey[1] = ry * ev;         P.gx[1] = fmaf(ry, eu, hx2 * (av + bv));
  P.ex[2] = rx * bu;          P.ey[2] = hy2 * (cv + ev); P.gx[2] = fmaf(hy2, cu + eu, rx * bv);
  P.ex[3] = hx2 * (au + bu);  P.ey[3] = ry * cv;         P.gx[3] = fmaf(ry, cu, hx2 * (av + bv));
#pragma unroll
  for (int k = 0; k < 4; ++k) P.s[k] = stress32(d.mat, P.ex[k], P.ey[k], P.gx[k]);
  P.qA = (float)(d.ck_Ap[c * 2 + p] * 0.25);
}

// the piece's force at its local node a
__device__ __forceinline__ float2 piece32_force(const Geo &g, const Piece32 &P, int a) {
  const float hx2 = 0.5f * g.rxf, hy2 = 0.5f * g.ryf;
  float sx = 0.f, sy = 0.f;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float cx = dxn(k, a) * hx2, cy = dyn(k, a) * hy2;
    sx = fmaf(cx, P.s[k].xx, fmaf(cy, P.s[k].xy, sx));
    sy = fmaf(cy, P.s[k].yy, fmaf(cx, P.s[k].xy, sy));
  }
  // rounded products (never fused into the caller's sums), so that a force
  // is the same in every kernel that adds it
  return make_float2(__fmul_rn(sx, P.qA), __fmul_rn(sy, P.qA));
}

__device__ __forceinline__ void piece32(const DevState &d, int c, int p, int cur, Piece32 &P) {
  piece32_state(d, c, p, cur, P);
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const float2 F = piece32_force(d.g, P, a);
    P.f[2 * a] = F.x;
    P.f[2 * a + 1] = F.y;
  }
}

// strain energy of a piece, FP64 sums of its four edge points' shares
__device__ __forceinline__ double piece32_energy(const Piece32 &P) {
  double acc = 0.0;
#pragma unroll
  for (int k = 0; k < 4; ++k)
    acc += 0.5 * (double)P.qA *
           ((double)P.ex[k] * P.s[k].xx + (double)P.ey[k] * P.s[k].yy + (double)P.gx[k] * P.s[k].xy);
  return acc;
}

// Piece forces of split elements (the profiling path times the pieces'
// evaluation on its own; the step itself has the tile and phantom kernels
// evaluate them).
__device__ __forceinline__ void pieces32(const DevState &d, VBlk vb, int cur, int energy,
                                         int part_off) {
  const int n = 2 * d.cnt->n_ck;
  double se = 0.0;
  for (int t = vb.x * blockDim.x + threadIdx.x; t < n; t += vb.gx * blockDim.x) {
    const int c = t >> 1, p = t & 1;
    Piece32 P;
    piece32(d, c, p, cur, P);
    float *o = d.pff + c * 16 + p * 8;
#pragma unroll
    for (int q = 0; q < 8; ++q) o[q] = P.f[q];
    if (energy) se += piece32_energy(P);
  }
  if (energy) block_sum2(0.0, se, d.e_part + 2 * (part_off + vb.x));
}

__global__ void k_pieces32(DevState d, int cur, int energy, int part_off) {
  pieces32(d, hw_vblk(), cur, energy, part_off);
}

// -------------------------------------------------------------- main tile
// One CTA of 32 x 8 threads owns a tile of TX x TY real nodes, TX = 32 and
// TY = 8 or 16 (TY / 8 rows per thread).  Shared memory holds, with a
// two-node halo:
//   sU  displacement pairs (x.hi, x.lo, y.hi, y.lo) of nodes [i0-2, i0+TX+1] x [j0-2, j0+TY+1]
//   sD  node differences D(i,j) = (ux(i+1,j)-ux(i,j), uy(i+1,j)-uy(i,j),
//       ux(i,j+1)-ux(i,j), uy(i,j+1)-uy(i,j)) of nodes [i0-2, i0+TX] x [j0-2, j0+TY],
//       formed from the pairs as (hi_b - hi_a) + (lo_b - lo_a)
//   sH  horizontal edges h(i,j), i in [i0-1, i0+TX), j in [j0-1, j0+TY]:
//       with A the stress (xx, yy, xy) used by the element above and B the
//       one used by the element below (zero where that element is not
//       intact), AB = (A.yy, A.xy, B.yy, B.xy) and P = (A.xx + B.xx,
//       A.xy + B.xy)
//   sV  vertical edges v(i,j), i in [i0-1, i0+TX], j in [j0-1, j0+TY): with
//       R the stress used by the element right and L by the element left,
//       AB = (R.xx, R.xy, L.xx, L.xy) and P = (R.xy + L.xy, R.yy + L.yy)
// Tiles whose halo holds only intact elements keep one stress per edge
// instead.  sU is dead once sD is formed and shares its storage with sH;
// sD is dead once the edge stresses are formed and then holds the forces
// at real nodes of the split elements that touch the tile's nodes (the
// window of elements [i0-1, i0+TX-1] x [j0-1, j0+TY-1]), KSLOT elements at
// a time, with the window's split elements listed in increasing id.
constexpr int TX = 32, BX = 32, BY = 8;

// Rank of this thread's flag among the set flags of the block, in thread
// order, and their total.  Every thread of the block calls it.
__device__ __forceinline__ int block_rank(bool flag, int &total) {
  constexpr int NWARP = BX * BY / 32;
  __shared__ int s_cnt[NWARP];
  const int tid = threadIdx.x + threadIdx.y * BX, lane = tid & 31, w = tid >> 5;
  const unsigned b = __ballot_sync(0xffffffffu, flag);
  if (lane == 0) s_cnt[w] = __popc(b);
  __syncthreads();
  int off = 0, tot = 0;
#pragma unroll
  for (int q = 0; q < NWARP; ++q) {
    const int n = s_cnt[q];
    off += q < w ? n : 0;
    tot += n;
  }
  __syncthreads();
  total = tot;
  return off + __popc(b & ((1u << lane) - 1u));
}

// the low / high half of a float4 in shared memory (one 8-byte load)
__device__ __forceinline__ float2 lo2(const float4 &v) {
  return reinterpret_cast<const float2 *>(&v)[0];
}
__device__ __forceinline__ float2 hi2(const float4 &v) {
  return reinterpret_cast<const float2 *>(&v)[1];
}

template <int TY>
struct Tile {
  static constexpr int RY = TY / BY;  // node rows per thread
  static constexpr int UXn = TX + 4, UYn = TY + 4;
  static constexpr int DXn = TX + 3, DYn = TY + 3;
  static constexpr int EXn = TX + 3, EYn = TY + 3;
  static constexpr int HXn = TX + 1, HYn = TY + 2;
  static constexpr int VXn = TX + 2, VYn = TY + 1;
  struct SmemA {
    float4 U[UYn][UXn];
  };
  struct SmemB {
    float4 AB[HYn][HXn];
    float2 P[HYn][HXn];
  };
  union SmemMain {
    SmemA a;
    SmemB b;
  };
  struct SmemFastH {  // intact tiles: one stress per edge, as (xx, xy) and (yy, xy)
    float2 P[HYn][HXn], Q[HYn][HXn];
  };
  struct SmemFastV {
    float2 P[VYn][VXn], Q[VYn][VXn];
  };
  union SmemV {
    struct {
      float4 AB[VYn][VXn];
      float2 P[VYn][VXn];
    } gen;
    SmemFastV fast;
  };
  static constexpr int WXn = TX + 1, WYn = TY + 1, NWIN = WXn * WYn;
  static constexpr int KSLOT = (2 * DYn * DXn * (int)sizeof(float2) - 4 * NWIN) / 32;
  struct SmemD {
    float2 Dx[DYn][DXn], Dy[DYn][DXn];  // (dux, duy) along x and along y
  };
  struct SmemPieces {
    float2 slot[KSLOT][4];  // force at local node a of split element slot
    uint16_t list[NWIN];    // window index of the n-th split element
    uint16_t map[NWIN];     // rank of a split element in the list
  };
  static_assert(sizeof(SmemPieces) <= sizeof(SmemD), "piece slots fit in sD");
  struct Smem {  // > 48 KB for TY = 16: dynamic shared memory
    union {
      SmemMain ab;
      SmemFastH fh;
    } u1;
    union {
      SmemD d;
      SmemPieces pc;
    } u2;
    SmemV v;
    uint8_t st[EYn][EXn];
  };
};

template <bool ENERGY, int TY>
__device__ __forceinline__ void main32_tile(const DevState &d, VBlk vb, int cur, int first,
                                            typename Tile<TY>::Smem &T) {
  using C = Tile<TY>;
  constexpr int RY = C::RY, UXn = C::UXn, UYn = C::UYn, DXn = C::DXn, DYn = C::DYn;
  constexpr int EXn = C::EXn, EYn = C::EYn, HXn = C::HXn, HYn = C::HYn, VXn = C::VXn,
                VYn = C::VYn;
  float4 (*sU)[UXn] = T.u1.ab.a.U;
  float4 (*sHAB)[HXn] = T.u1.ab.b.AB;
  float2 (*sHP)[HXn] = T.u1.ab.b.P;
  float2 (*fHP)[HXn] = T.u1.fh.P, (*fHQ)[HXn] = T.u1.fh.Q;
  float2 (*sDx)[DXn] = T.u2.d.Dx, (*sDy)[DXn] = T.u2.d.Dy;
  float4 (*sVAB)[VXn] = T.v.gen.AB;
  float2 (*sVP)[VXn] = T.v.gen.P;
  float2 (*fVP)[VXn] = T.v.fast.P, (*fVQ)[VXn] = T.v.fast.Q;
  uint8_t (*sst)[EXn] = T.st;

  const Geo &g = d.g;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i0 = vb.x * TX, j0 = vb.y * TY;
  const int stride = g.nx + 1;
  const float4 *__restrict__ u4 = d.u4[cur];

  // own nodes (i, j0+ty+8r): issue their loads first
  const int i = i0 + tx;
  float2 own_v[RY];
  float own_mi[RY];
  int own_nf[RY];
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    const int j = j0 + ty + r * BY;
    if (i <= g.nx && j <= g.ny) {
      const int N = j * stride + i;
      own_v[r] = d.v2[N];
      own_mi[r] = d.minvf[N];
      own_nf[r] = d.nflag[N];
    } else {
      own_v[r] = make_float2(0.f, 0.f);
      own_mi[r] = 0.f;
      own_nf[r] = 0;
    }
  }
  // stage displacements and element states: every load is issued before
  // any shared store, so the block waits for one memory latency, not six
  const int tid0 = tx + ty * BX;
  constexpr int NU = (UXn * UYn + BX * BY - 1) / (BX * BY);
  constexpr int NE = (EXn * EYn + BX * BY - 1) / (BX * BY);
  float4 ureg[NU];
  int sreg[NE];
#pragma unroll
  for (int k = 0; k < NU; ++k) {
    const int q = tid0 + k * BX * BY;
    const int ly = q / UXn, lx = q - ly * UXn;
    const int jj = j0 - 2 + ly, ii = i0 - 2 + lx;
    ureg[k] = (q < UXn * UYn && jj >= 0 && jj <= g.ny && ii >= 0 && ii <= g.nx)
                  ? u4[jj * stride + ii] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int k = 0; k < NE; ++k) {
    const int q = tid0 + k * BX * BY;
    const int ly = q / EXn, lx = q - ly * EXn;
    const int jj = j0 - 2 + ly, ii = i0 - 2 + lx;
    sreg[k] = (q < EXn * EYn && jj >= 0 && jj < g.ny && ii >= 0 && ii < g.nx)
                  ? (int)d.estate[jj * g.nx + ii] : (int)ST_OUT;
  }
  int any_open = 0;  // some element of the halo is not intact
#pragma unroll
  for (int k = 0; k < NU; ++k) {
    const int q = tid0 + k * BX * BY;
    if (q < UXn * UYn) sU[q / UXn][q % UXn] = ureg[k];
  }
#pragma unroll
  for (int k = 0; k < NE; ++k) {
    const int q = tid0 + k * BX * BY;
    if (q < EXn * EYn) {
      sst[q / EXn][q % EXn] = (uint8_t)sreg[k];
      any_open |= sreg[k] != ST_INTACT;
    }
  }
  const bool general = __syncthreads_or(any_open) != 0;
  // own displacement pairs, needed by the update after sU is overwritten
  float4 own_u[RY];
#pragma unroll
  for (int r = 0; r < RY; ++r) own_u[r] = sU[ty + r * BY + 2][tx + 2];
  const int tid = tx + ty * BX;
  constexpr int NTH = BX * BY;
  for (int q = tid; q < DXn * DYn; q += NTH) {
    const int ly = q / DXn, lx = q - ly * DXn;
    const float4 U0 = sU[ly][lx], Ux = sU[ly][lx + 1], Uy = sU[ly + 1][lx];
    sDx[ly][lx] = make_float2((Ux.x - U0.x) + (Ux.y - U0.y), (Ux.z - U0.z) + (Ux.w - U0.w));
    sDy[ly][lx] = make_float2((Uy.x - U0.x) + (Uy.y - U0.y), (Uy.z - U0.z) + (Uy.w - U0.w));
  }
  __syncthreads();

  const Mat &m = d.mat;
  const float rx = g.rxf, ry = g.ryf;
  const float hx2 = 0.5f * rx, hy2 = 0.5f * ry, hx4 = 0.25f * rx, hy4 = 0.25f * ry;
  const float qA = g.qAf;
  float se = 0.f;    // strain energy of this thread's edges / qA (energy steps)
  double sep = 0.0;  // strain energy of the pieces of the split elements it owns

  if (!general) {
    // every element around the tile is intact: smoothed strain on every
    // edge, one stress per edge (stored in the .a arrays)
    for (int q = tid; q < HXn * HYn; q += NTH) {
      {
        const int ly = q / HXn, lx = q - ly * HXn;
        const float2 X0 = sDx[ly + 1][lx + 1];
        const float2 Y0 = sDy[ly + 1][lx + 1], Y1 = sDy[ly + 1][lx + 2];
        const float2 Z0 = sDy[ly][lx + 1], Z1 = sDy[ly][lx + 2];
        const float exx = rx * X0.x;
        const float eyy = hy4 * ((Y0.y + Y1.y) + (Z0.y + Z1.y));
        const float gxy = fmaf(hy4, (Y0.x + Y1.x) + (Z0.x + Z1.x), rx * X0.y);
        const Stress3 st = stress32(m, exx, eyy, gxy);
        fHP[ly][lx] = make_float2(st.xx, st.xy);
        fHQ[ly][lx] = make_float2(st.yy, st.xy);
        if (ENERGY && lx >= 1 && ly >= 1 && ly <= TY)
          se += exx * st.xx + eyy * st.yy + gxy * st.xy;
      }
    }
    for (int q = tid; q < VXn * VYn; q += NTH) {
      {
        const int ly = q / VXn, lx = q - ly * VXn;
        const float2 Y0 = sDy[ly + 1][lx + 1];
        const float2 X0 = sDx[ly + 1][lx + 1], X1 = sDx[ly + 2][lx + 1];
        const float2 W0 = sDx[ly + 1][lx], W1 = sDx[ly + 2][lx];
        const float exx = hx4 * ((X0.x + X1.x) + (W0.x + W1.x));
        const float eyy = ry * Y0.y;
        const float gxy = fmaf(hx4, (X0.y + X1.y) + (W0.y + W1.y), ry * Y0.x);
        const Stress3 st = stress32(m, exx, eyy, gxy);
        fVP[ly][lx] = make_float2(st.xx, st.xy);
        fVQ[ly][lx] = make_float2(st.yy, st.xy);
        if (ENERGY && lx >= 1 && lx <= TX && ly >= 1)
          se += exx * st.xx + eyy * st.yy + gxy * st.xy;
      }
    }
  } else {
    // horizontal edges h(ii,jj), ii = i0-1+lx, jj = j0-1+ly:
    // below element (ii, jj-1) = sst[ly][lx+1], above (ii, jj) = sst[ly+1][lx+1]
    for (int q = tid; q < HXn * HYn; q += NTH) {
      {
        const int ly = q / HXn, lx = q - ly * HXn;
        const int sb = sst[ly][lx + 1], sa = sst[ly + 1][lx + 1];
        float4 Ta = make_float4(0.f, 0.f, 0.f, 0.f), Tb = Ta;
        if (sa == ST_INTACT || sb == ST_INTACT) {
          const float2 X0 = sDx[ly + 1][lx + 1];                        // (ii,jj)
          const float2 Y0 = sDy[ly + 1][lx + 1], Y1 = sDy[ly + 1][lx + 2];  // (ii,jj), (ii+1,jj)
          const float exx = rx * X0.x, cdv = rx * X0.y;
          float eyy, gxy, w;
          if (sa == ST_INTACT && sb == ST_INTACT) {
            const float2 Z0 = sDy[ly][lx + 1], Z1 = sDy[ly][lx + 2];      // (ii,jj-1), (ii+1,jj-1)
            eyy = hy4 * ((Y0.y + Y1.y) + (Z0.y + Z1.y));
            gxy = fmaf(hy4, (Y0.x + Y1.x) + (Z0.x + Z1.x), cdv);
            w = 1.f;
          } else if (sa == ST_INTACT) {
            eyy = hy2 * (Y0.y + Y1.y);
            gxy = fmaf(hy2, Y0.x + Y1.x, cdv);
            w = 0.5f;
          } else {
            const float2 Z0 = sDy[ly][lx + 1], Z1 = sDy[ly][lx + 2];
            eyy = hy2 * (Z0.y + Z1.y);
            gxy = fmaf(hy2, Z0.x + Z1.x, cdv);
            w = 0.5f;
          }
          const Stress3 s = stress32(m, exx, eyy, gxy);
          const float4 S = make_float4(s.xx, s.yy, s.xy, 0.f);
          if (sa == ST_INTACT) Ta = S;
          if (sb == ST_INTACT) Tb = S;
          if (ENERGY && lx >= 1 && ly >= 1 && ly <= TY)
            se += w * (exx * s.xx + eyy * s.yy + gxy * s.xy);
        }
        sHAB[ly][lx] = make_float4(Ta.y, Ta.z, Tb.y, Tb.z);
        sHP[ly][lx] = make_float2(Ta.x + Tb.x, Ta.z + Tb.z);
      }
    }
    // vertical edges v(ii,jj), ii = i0-1+lx, jj = j0-1+ly:
    // left element (ii-1, jj) = sst[ly+1][lx], right (ii, jj) = sst[ly+1][lx+1]
    for (int q = tid; q < VXn * VYn; q += NTH) {
      {
        const int ly = q / VXn, lx = q - ly * VXn;
        const int sl = sst[ly + 1][lx], sr = sst[ly + 1][lx + 1];
        float4 Ta = make_float4(0.f, 0.f, 0.f, 0.f), Tb = Ta;
        if (sl == ST_INTACT || sr == ST_INTACT) {
          const float2 Y0 = sDy[ly + 1][lx + 1];                        // (ii,jj)
          const float2 X0 = sDx[ly + 1][lx + 1], X1 = sDx[ly + 2][lx + 1];  // (ii,jj), (ii,jj+1)
          const float eyy = ry * Y0.y, cdu = ry * Y0.x;
          float exx, gxy, w;
          if (sl == ST_INTACT && sr == ST_INTACT) {
            const float2 W0 = sDx[ly + 1][lx], W1 = sDx[ly + 2][lx];      // (ii-1,jj), (ii-1,jj+1)
            exx = hx4 * ((X0.x + X1.x) + (W0.x + W1.x));
            gxy = fmaf(hx4, (X0.y + X1.y) + (W0.y + W1.y), cdu);
            w = 1.f;
          } else if (sr == ST_INTACT) {
            exx = hx2 * (X0.x + X1.x);
            gxy = fmaf(hx2, X0.y + X1.y, cdu);
            w = 0.5f;
          } else {
            const float2 W0 = sDx[ly + 1][lx], W1 = sDx[ly + 2][lx];
            exx = hx2 * (W0.x + W1.x);
            gxy = fmaf(hx2, W0.y + W1.y, cdu);
            w = 0.5f;
          }
          const Stress3 s = stress32(m, exx, eyy, gxy);
          const float4 S = make_float4(s.xx, s.yy, s.xy, 0.f);
          if (sr == ST_INTACT) Ta = S;
          if (sl == ST_INTACT) Tb = S;
          if (ENERGY && lx >= 1 && lx <= TX && ly >= 1)
            se += w * (exx * s.xx + eyy * s.yy + gxy * s.xy);
        }
        sVAB[ly][lx] = make_float4(Ta.x, Ta.z, Tb.x, Tb.z);
        sVP[ly][lx] = make_float2(Ta.z + Tb.z, Ta.y + Tb.y);
      }
    }
    __syncthreads();
  }
  __syncthreads();

  // element forces of the own nodes
  float fxr[RY], fyr[RY];
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    // edge arrays: edge (i', j') at [j' - (j0-1)][i' - (i0-1)]
    const int ci = tx + 1, cj = ty + r * BY + 1;
    float fx, fy;
    if (!general) {
      // one stress per edge: the two sides of every edge carry the same sigma
      // (xx, xy) of h(i-1,j), h(i,j); (yy, xy) of the rows above / below
      const float2 H1 = fHP[cj][ci - 1], H2 = fHP[cj][ci];
      const float2 Hu0 = fHQ[cj + 1][ci - 1], Hu1 = fHQ[cj + 1][ci];
      const float2 Hd0 = fHQ[cj - 1][ci - 1], Hd1 = fHQ[cj - 1][ci];
      // (yy, xy) of v(i,j-1), v(i,j); (xx, xy) of the columns left / right
      const float2 V1 = fVQ[cj - 1][ci], V2 = fVQ[cj][ci];
      const float2 Vl0 = fVP[cj - 1][ci - 1], Vl1 = fVP[cj][ci - 1];
      const float2 Vr0 = fVP[cj - 1][ci + 1], Vr1 = fVP[cj][ci + 1];
      fx = (2.f * rx) * (H1.x - H2.x) + hy2 * ((Hd0.y + Hd1.y) - (Hu0.y + Hu1.y)) +
           (2.f * ry) * (V1.y - V2.y) + hx2 * ((Vl0.x + Vl1.x) - (Vr0.x + Vr1.x));
      fy = (2.f * rx) * (H1.y - H2.y) + hy2 * ((Hd0.x + Hd1.x) - (Hu0.x + Hu1.x)) +
           (2.f * ry) * (V1.x - V2.x) + hx2 * ((Vl0.y + Vl1.y) - (Vr0.y + Vr1.y));
    } else {
      // the across-edge differences (B - A, L - R) of the node's own four
      // edges are zero when the four elements around it are all intact or
      // all not: those nodes skip the per-side loads of these edges
      const int ey = ty + r * BY + 1, ex = tx + 1;
      const bool i00 = sst[ey][ex] == ST_INTACT, i01 = sst[ey][ex + 1] == ST_INTACT;
      const bool i10 = sst[ey + 1][ex] == ST_INTACT, i11 = sst[ey + 1][ex + 1] == ST_INTACT;
      const bool mixed = !((i00 && i01 && i10 && i11) || !(i00 || i01 || i10 || i11));
      // h(i-1, j), h(i, j): N is the right / left node of both elements
      const float2 P1 = sHP[cj][ci - 1], P2 = sHP[cj][ci];
      if (mixed) {
        const float4 Q1 = sHAB[cj][ci - 1], Q2 = sHAB[cj][ci];
        fx = rx * (P1.x - P2.x) + hy2 * ((Q1.w - Q1.y) + (Q2.w - Q2.y));
        fy = rx * (P1.y - P2.y) + hy2 * ((Q1.z - Q1.x) + (Q2.z - Q2.x));
      } else {
        fx = rx * (P1.x - P2.x);
        fy = rx * (P1.y - P2.y);
      }
      // h(i-1, j+1), h(i, j+1): N is a lower node of their below element (B);
      // h(i-1, j-1), h(i, j-1): N is an upper node of their above element (A)
      const float2 Bu0 = hi2(sHAB[cj + 1][ci - 1]), Bu1 = hi2(sHAB[cj + 1][ci]);
      const float2 Ad0 = lo2(sHAB[cj - 1][ci - 1]), Ad1 = lo2(sHAB[cj - 1][ci]);
      fx += hy2 * ((Ad0.y + Ad1.y) - (Bu0.y + Bu1.y));
      fy += hy2 * ((Ad0.x + Ad1.x) - (Bu0.x + Bu1.x));
      // v(i, j-1): N top node; v(i, j): N bottom node of both elements
      const float2 S1 = sVP[cj - 1][ci], S2 = sVP[cj][ci];
      if (mixed) {
        const float4 W1 = sVAB[cj - 1][ci], W2 = sVAB[cj][ci];
        fx += ry * (S1.x - S2.x) + hx2 * ((W1.z - W1.x) + (W2.z - W2.x));
        fy += ry * (S1.y - S2.y) + hx2 * ((W1.w - W1.y) + (W2.w - W2.y));
      } else {
        fx += ry * (S1.x - S2.x);
        fy += ry * (S1.y - S2.y);
      }
      // v(i-1, j-1), v(i-1, j): N is a right node of their right element (R);
      // v(i+1, j-1), v(i+1, j): N is a left node of their left element (L)
      const float2 Rl0 = lo2(sVAB[cj - 1][ci - 1]), Rl1 = lo2(sVAB[cj][ci - 1]);
      const float2 Lr0 = hi2(sVAB[cj - 1][ci + 1]), Lr1 = hi2(sVAB[cj][ci + 1]);
      fx += hx2 * ((Rl0.x + Rl1.x) - (Lr0.x + Lr1.x));
      fy += hx2 * ((Rl0.y + Rl1.y) - (Lr0.y + Lr1.y));
    }
    fxr[r] = fx * qA;
    fyr[r] = fy * qA;
  }

  if (general) {
    // forces of the pieces of split elements at the own nodes, added in
    // increasing element id.  Window element (wx, wy) is (i0-1+wx, j0-1+wy),
    // its state sst[wy+1][wx+1].  The pieces are evaluated here from their
    // nodes' displacements, so the update does not wait for the piece kernel.
    __syncthreads();  // sD is dead: its storage now holds the piece forces
    constexpr int WXn = C::WXn, NWIN = C::NWIN, KSLOT = C::KSLOT;
    uint16_t *wlist = T.u2.pc.list, *wmap = T.u2.pc.map;
    float2 (*slot)[4] = T.u2.pc.slot;
    int nl = 0;
    for (int q0 = 0; q0 < NWIN; q0 += NTH) {
      const int q = q0 + tid;
      bool cr = false;
      if (q < NWIN) {
        const int wy = q / WXn, wx = q - wy * WXn;
        cr = sst[wy + 1][wx + 1] == ST_CRACKED;
      }
      int tot;
      const int rk = nl + block_rank(cr, tot);
      if (q < NWIN) wmap[q] = cr ? (uint16_t)rk : (uint16_t)0xffff;
      if (cr) wlist[rk] = (uint16_t)q;
      nl += tot;
    }
    __syncthreads();
    for (int base = 0; base < nl; base += KSLOT) {
      const int nb = nl - base < KSLOT ? nl - base : KSLOT;
      for (int t = tid; t < 2 * nb; t += NTH) {
        const int li = base + (t >> 1), p = t & 1;
        const int q = wlist[li];
        const int wy = q / WXn, wx = q - wy * WXn;
        const int c = d.crack_of[(j0 - 1 + wy) * g.nx + i0 - 1 + wx];
        const int info = d.ck_info[c];
        Piece32 P;
        piece32(d, c, p, cur, P);
#pragma unroll
        for (int a = 0; a < 4; ++a)  // piece p holds the real nodes of side p
          if (((info >> (4 + a)) & 1) == p)
            slot[li - base][a] = make_float2(P.f[2 * a], P.f[2 * a + 1]);
        // the tile owns elements [i0, i0+TX) x [j0, j0+TY)
        if (ENERGY && wx >= 1 && wx <= TX && wy >= 1 && wy <= TY) sep += piece32_energy(P);
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        // elements (i-1, j-1), (i, j-1), (i-1, j), (i, j) of node (i, j) and
        // the node's local index in each
        const int wy0 = ty + r * BY, wx0 = tx;
        const int dwx[4] = {0, 1, 0, 1}, dwy[4] = {0, 0, 1, 1}, la[4] = {2, 3, 1, 0};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int q = (wy0 + dwy[k]) * WXn + wx0 + dwx[k];
          if (sst[wy0 + dwy[k] + 1][wx0 + dwx[k] + 1] == ST_CRACKED) {
            const int li = wmap[q];
            if (li >= base && li < base + nb) {
              const float2 F = slot[li - base][la[k]];
              fxr[r] += F.x;
              fyr[r] += F.y;
            }
          }
        }
      }
      __syncthreads();
    }
  }

  double ke = 0.0;  // nodes with loads or prescribed velocities (FP64 path)
  float ke2 = 0.f;  // 2 KE of the other nodes
  const float dt = m.dtf;
  const float dtv = first ? 0.5f * dt : dt;
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    const int j = j0 + ty + r * BY;
    if (i > g.nx || j > g.ny) continue;
    const float fx = fxr[r], fy = fyr[r];
    const int N = j * stride + i;
    if (own_nf[r]) {
      ke += update_special(d, N, cur, first, fx, fy, own_u[r], own_v[r], own_mi[r], own_nf[r],
                           ENERGY ? 1 : 0);
    } else {
      const float2 vn = update_plain(d, N, cur, dtv, dt, fx, fy, own_u[r], own_v[r], own_mi[r]);
      if (ENERGY && own_mi[r] > 0.f) {
        // KE of the mid-step velocity, FP32 like the velocities themselves
        const float bx = first ? own_v[r].x : 0.5f * (own_v[r].x + vn.x);
        const float by = first ? own_v[r].y : 0.5f * (own_v[r].y + vn.y);
        ke2 += __fdividef(fmaf(bx, bx, by * by), own_mi[r]);
      }
    }
  }
  if (ENERGY)
    block_sum2(ke + 0.5 * (double)ke2, (double)qA * (double)se + sep,
               d.e_part + 2 * (vb.y * vb.gx + vb.x));
}

template <bool ENERGY, int TY>
__global__ void __launch_bounds__(BX * BY, 4) k_main32(DevState d, int cur,
                                                                      int first) {
  // launched as a programmatic dependent of the kernel before it (the
  // previous step's split writes): wait until that kernel has completed and
  // its writes are visible; then let the split writes that follow be placed
  // once every tile CTA has started (they wait for this kernel themselves)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;");
  extern __shared__ float4 smem_dyn[];
  main32_tile<ENERGY, TY>(d, hw_vblk(), cur, first,
                          *reinterpret_cast<typename Tile<TY>::Smem *>(smem_dyn));
}

// ---------------------------------------------------------------- phantoms
__device__ __forceinline__ void phantom32(const DevState &d, VBlk vb, int cur, int first,
                                          int energy, int part_off) {
  const int n = d.cnt->n_ph;
  double ke = 0.0;
  const float dt = d.mat.dtf;
  const float dtv = first ? 0.5f * dt : dt;
  for (int t = vb.x * blockDim.x + threadIdx.x; t < n; t += vb.gx * blockDim.x) {
    int N = d.g.nn + t;
    // users' piece-force indices c*16 + p*8 + 2a in increasing element id,
    // -1 unused: the phantom is local node a of piece p of split c, whose
    // force there is evaluated here
    const int4 uf = reinterpret_cast<const int4 *>(d.ph_upf)[t];
    const int ufs[4] = {uf.x, uf.y, uf.z, uf.w};
    float fx = 0.f, fy = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (ufs[q] >= 0) {
        Piece32 P;
        piece32_state(d, ufs[q] >> 4, (ufs[q] >> 3) & 1, cur, P);
        const float2 F = piece32_force(d.g, P, (ufs[q] >> 1) & 3);
        fx += F.x;
        fy += F.y;
      }
    }
    if (energy)
      ke += update_special(d, N, cur, first, fx, fy, d.u4[cur][N], d.v2[N], d.minvf[N], 0, 1);
    else
      update_plain(d, N, cur, dtv, dt, fx, fy, d.u4[cur][N], d.v2[N], d.minvf[N]);
  }
  if (energy) warp_sum_parts(ke, d.e_part + 2 * (part_off + vb.x * kPhWarps));
}

__global__ void k_phantom32(DevState d, int cur, int first, int energy, int part_off) {
  phantom32(d, hw_vblk(), cur, first, energy, part_off);
}

// ---------------------------------------------------------------- batched
// One launch per kernel kind for every member of a batch.  The grids are
// persistent: blocks walk the work list with a stride of the grid size.
// 1-D items are (member, block, energy-partial offset, member's grid size).
template <bool ENERGY, int TY>
__global__ void __launch_bounds__(BX * BY, 4) k_main32_batch(BatchDev b,
                                                                            int first) {
  extern __shared__ float4 smem_dyn[];
  auto &T = *reinterpret_cast<typename Tile<TY>::Smem *>(smem_dyn);
  __shared__ DevState sd;
  int held = -1, w0, w1;
  const int n = *b.bstep;
  block_range(b.n_main, w0, w1);
  for (int w = w0; w < w1; ++w) {
    const int4 it = b.w_main[w];
    stage_member(b.ds, it.x, sd, held);
    if (!member_active(sd, n)) continue;
    main32_tile<ENERGY, TY>(sd, item_vblk(it), member_cur(sd, n), first, T);
    __syncthreads();
  }
}

__global__ void k_phantom32_batch(BatchDev b, int first, int energy) {
  __shared__ DevState sd;
  int held = -1, w0, w1;
  const int n = *b.bstep;
  block_range(b.n_ph, w0, w1);
  for (int w = w0; w < w1; ++w) {
    const int4 it = b.w_ph[w];
    stage_member(b.ds, it.x, sd, held);
    if (!member_active(sd, n)) continue;
    phantom32(sd, VBlk{it.y, 0, it.w, 1}, member_cur(sd, n), first, energy, it.z);
    __syncthreads();
  }
}

int grid_for(int n, int block, int maxb) {
  int b = (n + block - 1) / block;
  return b < 1 ? 1 : (b > maxb ? maxb : b);
}

template <bool ENERGY, int TY>
cudaError_t set_smem_attr() {
  static bool done = false;
  if (!done) {
    cudaError_t e = cudaFuncSetAttribute(k_main32<ENERGY, TY>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(typename Tile<TY>::Smem));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_main32_batch<ENERGY, TY>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(typename Tile<TY>::Smem));
    if (e != cudaSuccess) return e;
    done = true;
  }
  return cudaSuccess;
}

cudaError_t set_all_smem_attrs() {
  static bool side = false;
  if (!side) {
    cudaError_t e = match_tile_carveout(k_phantom32);
    if (e == cudaSuccess) e = match_tile_carveout(k_phantom32_batch);
    if (e != cudaSuccess) return e;
    side = true;
  }
  cudaError_t e;
  if ((e = set_smem_attr<true, 16>()) != cudaSuccess) return e;
  if ((e = set_smem_attr<false, 16>()) != cudaSuccess) return e;
  if ((e = set_smem_attr<true, 8>()) != cudaSuccess) return e;
  return set_smem_attr<false, 8>();
}

}  // namespace

cudaError_t launch_eval32(const DevState &d, int cur, cudaStream_t st);
cudaError_t launch_eval32_batch(const BatchDev &b, cudaStream_t st);

int tiles_fp32(const DevState &d, int tile_rows) {
  return ((d.g.nx + 1 + TX - 1) / TX) * ((d.g.ny + 1 + tile_rows - 1) / tile_rows);
}

// energy partials: tiles of the smallest tile height first, then the
// phantom update's warps (at most 1216 blocks of kPhWarps)
int energy_parts_fp32(const DevState &d) { return tiles_fp32(d, 8) + kPhWarps * 1216 + 8; }

int grid_pieces(const DevState &d) { return grid_for(2 * d.ck_cap, 256, 1216); }
// side-branch grids: two phantom blocks and one evaluation block per SM, so that
// they start together with the tile update and share the SMs with it
int grid_phantoms(const DevState &d) { return grid_for(d.ph_cap, 256, 304); }

// energy partials one FP32 step writes with the given tile height
int energy_parts_step_fp32(const DevState &d, int tile_rows) {
  return tiles_fp32(d, tile_rows) + kPhWarps * grid_phantoms(d);
}

cudaError_t launch_step_fp32(const DevState &d, int cur, bool first, bool energy,
                             const StepStreams &ss, cudaEvent_t *marks) {
  constexpr int TYs = 16;  // tile height of a mesh stepped alone
  const dim3 grid((d.g.nx + 1 + TX - 1) / TX, (d.g.ny + 1 + TYs - 1) / TYs);
  const dim3 block(BX, BY);
  const int tiles = grid.x * grid.y;  // energy partials of the tiles come first
  const int gp = grid_pieces(d);
  const int gph = grid_phantoms(d);
  cudaError_t e = set_all_smem_attrs();
  if (e != cudaSuccess) return e;
  constexpr size_t smem = sizeof(Tile<TYs>::Smem);
  cudaStream_t st = ss.main;
  auto main_kernel = [&](cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const int f = first ? 1 : 0;
    if (energy) cudaLaunchKernelEx(&cfg, k_main32<true, TYs>, d, cur, f);
    else cudaLaunchKernelEx(&cfg, k_main32<false, TYs>, d, cur, f);
  };
  if (marks) {
    // the pieces' evaluation alone (its energy partials land past the
    // phantom update's and are not summed), then the step's own kernels
    k_pieces32<<<gp, 256, 0, st>>>(d, cur, 0, tiles + gph);
    cudaEventRecord(marks[0], st);
    main_kernel(st);
    cudaEventRecord(marks[1], st);
    k_phantom32<<<gph, 32 * kPhWarps, 0, st>>>(d, cur, first ? 1 : 0, energy ? 1 : 0, tiles);
    cudaEventRecord(marks[2], st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_eval32(d, cur, st);
  }
  // the tile update and the phantom update evaluate the pieces they need
  // themselves, so the three branches start together
  cudaEventRecord(ss.fork, st);
  cudaStreamWaitEvent(ss.aux2, ss.fork, 0);
  cudaStreamWaitEvent(ss.aux1, ss.fork, 0);
  e = launch_eval32(d, cur, ss.aux2);
  if (e != cudaSuccess) return e;
  e = launch_select(d, TRACK_STEP, ss.aux2);
  if (e != cudaSuccess) return e;
  k_phantom32<<<gph, 32 * kPhWarps, 0, ss.aux1>>>(d, cur, first ? 1 : 0, energy ? 1 : 0, tiles);
  main_kernel(st);
  cudaEventRecord(ss.join1, ss.aux1);
  cudaEventRecord(ss.join2, ss.aux2);
  cudaStreamWaitEvent(st, ss.join1, 0);
  cudaStreamWaitEvent(st, ss.join2, 0);
  return cudaGetLastError();
}

// The same fork/join as launch_step_fp32, one launch per kernel kind for all
// members of the batch.
cudaError_t launch_step_fp32_batch(const BatchDev &b, bool first, bool energy, int tile_rows,
                                   int grid_main, const StepStreams &ss) {
  cudaError_t e = set_all_smem_attrs();
  if (e != cudaSuccess) return e;
  const dim3 block(BX, BY);
  const int gm = grid_main < 1 ? 1 : grid_main;
  const int gph = grid_for(b.n_ph, 1, 1216);
  cudaStream_t st = ss.main;
  cudaEventRecord(ss.fork, st);
  cudaStreamWaitEvent(ss.aux2, ss.fork, 0);
  cudaStreamWaitEvent(ss.aux1, ss.fork, 0);
  e = launch_eval32_batch(b, ss.aux2);
  if (e != cudaSuccess) return e;
  e = launch_select_batch(b, ss.aux2);
  if (e != cudaSuccess) return e;
  k_phantom32_batch<<<gph, 32 * kPhWarps, 0, ss.aux1>>>(b, first ? 1 : 0, energy ? 1 : 0);
  const int f = first ? 1 : 0;
  if (tile_rows == 8) {
    constexpr size_t sm = sizeof(Tile<8>::Smem);
    if (energy) k_main32_batch<true, 8><<<gm, block, sm, st>>>(b, f);
    else k_main32_batch<false, 8><<<gm, block, sm, st>>>(b, f);
  } else {
    constexpr size_t sm = sizeof(Tile<16>::Smem);
    if (energy) k_main32_batch<true, 16><<<gm, block, sm, st>>>(b, f);
    else k_main32_batch<false, 16><<<gm, block, sm, st>>>(b, f);
  }
  cudaEventRecord(ss.join1, ss.aux1);
  cudaEventRecord(ss.join2, ss.aux2);
  cudaStreamWaitEvent(st, ss.join1, 0);
  cudaStreamWaitEvent(st, ss.join2, 0);
  return cudaGetLastError();
}

}  // namespace cem
