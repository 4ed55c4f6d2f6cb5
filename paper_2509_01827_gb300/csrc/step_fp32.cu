// step_fp32.cu -- FP32-mixed explicit step: FP32 element arithmetic,
// displacement kept as a compensated pair of floats (hi + lo, ~48-bit
// mantissa) and advanced with an error-free two-sum, FP64 energy sums.
//
// One step is four kernels: k_pieces32 evaluates the pieces of every split
// element (their forces at all eight nodes for the phantom update, and at
// each element's real nodes for the node update); k_march32 updates every
// real node (its HBM floor is 53 bytes per active element: u read and
// written as 16-byte compensated pairs, v read and written as float2, 1/m
// read, one element-state byte); k_phantom32 updates the phantom nodes from
// the piece forces; the surface evaluation and the selection run beside them.
// k_march32 forms, for each node, the strains at the midpoints of the edges
// around it from node differences (Eq. 4 at the edge points): along an edge
// the tangential derivative is the difference of its two nodes, across it the
// normal derivative of each side is the sum of that side's two across-edge
// differences; with two intact neighbours the two sides are averaged (Eqs.
// 1-2 with equal areas), otherwise each intact side keeps its own strain;
// sigma = D eps per side (zero for split or missing sides); the node force is
// B^T sigma A/4 (Eq. 6) summed over those edges and sides, plus the piece
// forces of the split elements it belongs to; then the central-difference
// update.
#include <cuda_runtime.h>

#include <algorithm>
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

// Piece forces of every split element, evaluated once per step before the
// node updates, one thread per split element: all eight nodal forces of each
// piece into pff (the phantom update gathers them), and each real node's
// force (from the piece on its side) into the element's pfe record (the node
// update adds them).
__device__ __forceinline__ void pieces32(const DevState &d, VBlk vb, int cur, int energy,
                                         int part_off) {
  const int n = d.cnt->n_ck;
  double se = 0.0;
  for (int c = vb.x * blockDim.x + threadIdx.x; c < n; c += vb.gx * blockDim.x) {
    const int info = d.ck_info[c];
    const int e = d.ck_elem[c];
    float2 fr[4];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      Piece32 P;
      piece32(d, c, p, cur, P);
      float4 *o = reinterpret_cast<float4 *>(d.pff + c * 16 + p * 8);
      o[0] = make_float4(P.f[0], P.f[1], P.f[2], P.f[3]);
      o[1] = make_float4(P.f[4], P.f[5], P.f[6], P.f[7]);
#pragma unroll
      for (int a = 0; a < 4; ++a)  // piece p holds the real nodes of side p
        if (((info >> (4 + a)) & 1) == p) fr[a] = make_float2(P.f[2 * a], P.f[2 * a + 1]);
      if (energy) se += piece32_energy(P);
    }
    float4 *r = reinterpret_cast<float4 *>(d.pfe) + (size_t)e * 2;
    r[0] = make_float4(fr[0].x, fr[0].y, fr[1].x, fr[1].y);
    r[1] = make_float4(fr[2].x, fr[2].y, fr[3].x, fr[3].y);
  }
  if (energy) block_sum2(0.0, se, d.e_part + 2 * (part_off + vb.x));
}

__global__ void k_pieces32(DevState d, int cur, int energy, int part_off) {
  // a programmatic dependent of the previous step's split writes (see k_march32)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;");
  pieces32(d, hw_vblk(), cur, energy, part_off);
}

// -------------------------------------------------------------- warp march
// One warp updates a tile of WX x TY real nodes by marching up its node
// rows.  Lane l holds the two node columns c_k = i0 - 2 + 2 l + k (columns
// i0-2 .. i0+61); lanes 1..30 own the tile's WX = 60 columns, lanes 0 and 31
// only supply the values the owned columns need from their neighbours.
// Vertical neighbours are the lane's own registers from earlier rows;
// horizontal ones are the lane's other column or come from the adjacent lanes
// by warp shuffles (shared memory only stages the rows in flight).  Iteration
// t loads node row t and forms
//   Dx(c,t)   = u(c+1,t) - u(c,t)    tangential difference of edge h(c,t)
//   Dy(c,t-1) = u(c,t) - u(c,t-1)    tangential difference of edge v(c,t-1)
// (compensated pairs: (hi_b - hi_a) + (lo_b - lo_a)), then the strain and
// the stress used on each side of edges h(c,t-1) and v(c,t-1) (Eq. 4 at the
// edge midpoints: the tangential derivative is the edge's own difference,
// the normal derivative of a side the sum of that side's two across-edge
// differences; with both sides intact they are averaged, Eqs. 1-2 with equal
// areas; a side that is not intact uses nothing and gets nothing), and adds
// each side's B^T sigma A/4 (Eq. 6) to the forces of the nodes it touches
// (rows t-2 .. t of columns c-1, c, c+1), as well as the forces of the
// pieces of split element (c,t-1) at its real nodes.  Node row t-2 then has
// every contribution: its force is summed across the lanes and the node
// takes its central-difference update.
__device__ __forceinline__ Stress3 masked(const Stress3 &s, bool on) {
  Stress3 r;
  r.xx = on ? s.xx : 0.f;
  r.yy = on ? s.yy : 0.f;
  r.xy = on ? s.xy : 0.f;
  return r;
}

// Packed FP32 pairs (add/sub/mul .rn.f32x2): one instruction works on both
// lanes of a float2, each lane rounded as the scalar operation would be and
// never contracted with a neighbouring multiply, so every force sum below is
// the same in the all-intact branch and the general one.
__device__ __forceinline__ unsigned long long pk2(float2 a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ float2 upk2(unsigned long long r) {
  float2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
__device__ __forceinline__ float2 padd(float2 a, float2 b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk2(a)), "l"(pk2(b)));
  return upk2(r);
}
__device__ __forceinline__ float2 psub(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk2(a)), "l"(pk2(b)));
  return upk2(r);
}
__device__ __forceinline__ float2 pmul(float2 a, float2 b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk2(a)), "l"(pk2(b)));
  return upk2(r);
}
// (b - a) of two compensated pairs per component: (b.hi - a.hi) + (b.lo - a.lo)
__device__ __forceinline__ float2 pdiff(const float4 &a, const float4 &b) {
  const float2 tx = psub(make_float2(b.x, b.y), make_float2(a.x, a.y));
  const float2 ty = psub(make_float2(b.z, b.w), make_float2(a.z, a.w));
  return make_float2(tx.x + tx.y, ty.x + ty.y);
}

// Node data in flight per warp: u, v and 1/m of node rows t-2 .. t+kAhead-1
// sit in a shared-memory ring filled by asynchronous copies (cp.async),
// issued kAhead rows ahead of their use, so that the march holds no
// prefetch registers for them.
constexpr int kRing = 4, kAhead = kRing - 2;
// Node columns per lane: lane l holds columns c_k = i0 - kHalo*kCols +
// kCols*l + k, k < kCols; the kHalo lanes on each side only supply the
// values the owned columns need (two columns of neighbours on each side).
constexpr int kCols = 2;
constexpr int kHalo = (2 + kCols - 1) / kCols;
constexpr int WX = (32 - 2 * kHalo) * kCols;  // owned columns of a tile
static_assert(WX == kMarchWX && kHalo * kCols == kMarchLeft && 32 * kCols == kMarchSpan,
              "the row flags describe these tiles");
struct MarchRing {
  float4 u[kRing][kCols][32];
  float2 v[kRing][kCols][32];
  float mi[kRing][kCols][32];
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(valid)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem, int valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(s), "l"(gmem), "r"(valid)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem, int valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(s), "l"(gmem), "r"(valid)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void prefetch_l1(const void *p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// The tile height TY (node rows) is chosen at launch, at most 64.  CLEAN:
// every element the tile reads is intact and no node it updates has a load
// or a prescribed velocity (the general branch, the pieces and the special
// updates drop out at compile time).
template <bool ENERGY, bool CLEAN>
__device__ __forceinline__ void march32_tile(const DevState &d, int tile_x, int tile_y, int TY,
                                             int cur, int first, double *part, MarchRing &ring) {
  constexpr int K = kCols;
  const Geo &g = d.g;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int i0 = tile_x * WX, j0 = tile_y * TY;
  const int c0 = i0 - kHalo * K + K * lane;  // column of k = 0
  const int stride = g.nx + 1;
  const bool own_lane = lane >= kHalo && lane < 32 - kHalo;
  const float4 *__restrict__ u4 = d.u4[cur];
  const float rx = g.rxf, ry = g.ryf;
  const float hx2 = 0.5f * rx, hy2 = 0.5f * ry;
  const float2 RX = make_float2(rx, rx), RY = make_float2(ry, ry);
  const float2 HX2 = make_float2(hx2, hx2), HY2 = make_float2(hy2, hy2);
  // D scaled by A/4: the stresses below are A/4 sigma, so that every edge
  // term is a force and a piece force adds to it directly
  Mat mq = d.mat;
  mq.D11f *= g.qAf;
  mq.D12f *= g.qAf;
  mq.D33f *= g.qAf;
  const float dt = d.mat.dtf;
  const float dtv = first ? 0.5f * dt : dt;

  // stage node row r into ring slot r mod kRing (zeros outside the mesh; v
  // and 1/m only for the owned nodes), one commit group per row
  auto stage = [&](int r) {
    const int q = (r + 4 * kRing) & (kRing - 1);
    const bool rin = r >= 0 && r <= g.ny;
    const bool rown = own_lane && r >= j0 && r < j0 + TY;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int c = c0 + k;
      const bool in = rin && c >= 0 && c <= g.nx;
      const int N = in ? r * stride + c : 0;
      cp_async16(&ring.u[q][k][lane], u4 + N, in ? 16 : 0);
      const bool mine = in && rown;
      cp_async8(&ring.v[q][k][lane], d.v2 + N, mine ? 8 : 0);
      cp_async4(&ring.mi[q][k][lane], d.minvf + N, mine ? 4 : 0);
    }
    cp_async_commit();
  };
  // a clean tile reads no element state and no node flag: they are known
  auto load_es = [&](int r, int k) -> int {  // state of element (c_k, r)
    if (CLEAN) return (int)ST_INTACT;
    const int c = c0 + k;
    return (c >= 0 && c < g.nx && r >= 0 && r < g.ny) ? (int)d.estate[r * g.nx + c] : (int)ST_OUT;
  };
  auto load_nf = [&](int r, int k) -> int {
    if (CLEAN) return 0;
    const int c = c0 + k;
    return (own_lane && c <= g.nx && r >= j0 && r < j0 + TY && r <= g.ny)
               ? (int)d.nflag[r * stride + c] : 0;
  };

#pragma unroll
  for (int q = 0; q <= kAhead; ++q) stage(j0 - 2 + q);  // rows j0-2 .. j0+kAhead-2
  cp_async_wait<kAhead>();  // row j0 - 2 is in
  const float2 z2 = make_float2(0.f, 0.f);
  float4 U1[K];         // u(c_k, t-1)
  int es1[K], esn[K];   // elements (c_k, t-2) and (c_k, t-1), the latter loaded a row ahead
  int nf1[K], nf2[K];   // node flags of rows t-1, t-2
  float2 Dx1[K], Dy2[K];  // Dx(c_k, t-1), Dy(c_k, t-2)
  // force sums of nodes (c_k, t-2+q), q = 0..2
  float2 own0[K], own1[K];
  unsigned long long spmask[K];  // owned rows whose node has a load or prescribed velocity
#pragma unroll
  for (int k = 0; k < K; ++k) {
    U1[k] = ring.u[(j0 - 2 + 4 * kRing) & (kRing - 1)][k][lane];
    es1[k] = load_es(j0 - 3, k);
    esn[k] = load_es(j0 - 2, k);
    nf1[k] = nf2[k] = 0;
    Dx1[k] = Dy2[k] = own0[k] = own1[k] = z2;
    spmask[k] = 0;
  }
  float2 DxL1 = z2, DyR2 = z2;  // Dx(c_0 - 1, t-1), Dy(c_{K-1} + 1, t-2)
  // terms this lane adds for the column right of its last (ua) and left of
  // its first (da), rows t-2 and t-1
  float2 ua0 = z2, ua1 = z2, da0 = z2, da1 = z2;
  unsigned pk_on = 0;  // bit k: element (c_k, t-2) is split; its piece forces come this row
  bool bad = false;    // some updated velocity is not finite
  float se = 0.f;      // A/4 eps.sigma of owned edges
  double ke = 0.0;     // kinetic energy of special nodes
  float ke2 = 0.f;     // 2 KE of the other nodes

#pragma unroll 1
  for (int t = j0 - 1; t <= j0 + TY + 1; ++t) {
    cp_async_wait<kAhead - 1>();  // rows up to t are in
    const int sl = (t + 4 * kRing) & (kRing - 1);
    float4 U0[K];
    int es0[K], nf0[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      U0[k] = ring.u[sl][k][lane];
      es0[k] = esn[k];  // element (c_k, t-1)
      esn[k] = load_es(t, k);
      nf0[k] = load_nf(t, k);
    }
    const bool owned_row = ENERGY && t - 1 >= j0 && t - 1 < j0 + TY;
    // ---- differences: Dx(c_k, t), Dy(c_k, t-1), and the lane's neighbours
    float2 Dx0[K], Dy1[K];
    {
      float4 Ur;  // u(c_{K-1} + 1, t) from the next lane
      Ur.x = __shfl_down_sync(FULL, U0[0].x, 1);
      Ur.y = __shfl_down_sync(FULL, U0[0].y, 1);
      Ur.z = __shfl_down_sync(FULL, U0[0].z, 1);
      Ur.w = __shfl_down_sync(FULL, U0[0].w, 1);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float4 R = k < K - 1 ? U0[k < K - 1 ? k + 1 : k] : Ur;
        Dx0[k] = pdiff(U0[k], R);
        Dy1[k] = pdiff(U1[k], U0[k]);
      }
    }
    float2 DyRl, DxLf;  // Dy(c_{K-1} + 1, t-1), Dx(c_0 - 1, t)
    DyRl.x = __shfl_down_sync(FULL, Dy1[0].x, 1);
    DyRl.y = __shfl_down_sync(FULL, Dy1[0].y, 1);
    DxLf.x = __shfl_up_sync(FULL, Dx0[K - 1].x, 1);
    DxLf.y = __shfl_up_sync(FULL, Dx0[K - 1].y, 1);
    const int esLf = __shfl_up_sync(FULL, es0[K - 1], 1);  // element (c_0 - 1, t-1)
    float2 own2[K], ua2 = z2, da2 = z2;  // row t
#pragma unroll
    for (int k = 0; k < K; ++k) own2[k] = z2;
    bool intact = true;
#pragma unroll
    for (int k = 0; k < K; ++k) intact = intact && es0[k] == ST_INTACT && es1[k] == ST_INTACT;
    intact = CLEAN || __all_sync(FULL, intact && esLf == ST_INTACT);
    // the edges of row j0 - 2 only touch node rows below the tile: the first
    // row marched only forms its differences
    if (t >= j0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float2 DyR1 = k < K - 1 ? Dy1[k < K - 1 ? k + 1 : k] : DyRl;
      const float2 DyR2k = k < K - 1 ? Dy2[k < K - 1 ? k + 1 : k] : DyR2;
      const float2 DxL0 = k > 0 ? Dx0[k > 0 ? k - 1 : k] : DxLf;
      const float2 DxL1k = k > 0 ? Dx1[k > 0 ? k - 1 : k] : DxL1;
      const int esL0 = k > 0 ? es0[k > 0 ? k - 1 : k] : esLf;
      const bool owned_edge = owned_row && own_lane && c0 + k <= g.nx;
      // right neighbour column's sums (this lane's next column, or ua)
      float2 &nr0 = k < K - 1 ? own0[k < K - 1 ? k + 1 : k] : ua0;
      float2 &nr1 = k < K - 1 ? own1[k < K - 1 ? k + 1 : k] : ua1;
      float2 &nr2 = k < K - 1 ? own2[k < K - 1 ? k + 1 : k] : ua2;
      float2 &nl1 = k > 0 ? own1[k > 0 ? k - 1 : k] : da1;
      float2 &nl2 = k > 0 ? own2[k > 0 ? k - 1 : k] : da2;
      if (intact) {
        // every element around the row's edges is intact: one averaged
        // stress per edge (the general branch with both sides intact, term
        // for term: its zero differences drop out exactly)
        {  // h(c_k, t-1)
          const float2 sY = padd(padd(Dy1[k], DyR1), padd(Dy2[k], DyR2k));
          const float q = 0.5f * hy2;
          const float2 mD = pmul(RX, Dx1[k]);
          const float exx = mD.x, eyy = q * sY.y, gxy = fmaf(q, sY.x, mD.y);
          const Stress3 s = stress32(mq, exx, eyy, gxy);
          const float2 sxp = make_float2(s.xx, s.xy);
          const float2 P = pmul(RX, padd(sxp, sxp));
          own1[k] = psub(own1[k], P);
          nr1 = padd(nr1, P);
          const float2 Bv = make_float2(hy2 * s.xy, hy2 * s.yy);
          own0[k] = psub(own0[k], Bv);
          nr0 = psub(nr0, Bv);
          own2[k] = padd(own2[k], Bv);
          nr2 = padd(nr2, Bv);
          if (owned_edge) se += exx * s.xx + eyy * s.yy + gxy * s.xy;
        }
        {  // v(c_k, t-1)
          const float2 sX = padd(padd(Dx1[k], Dx0[k]), padd(DxL1k, DxL0));
          const float q = 0.5f * hx2;
          const float2 mD = pmul(RY, Dy1[k]);
          const float exx = q * sX.x, eyy = mD.y, gxy = fmaf(q, sX.y, mD.x);
          const Stress3 s = stress32(mq, exx, eyy, gxy);
          const float2 syp = make_float2(s.xy, s.yy);
          const float2 S = pmul(RY, padd(syp, syp));
          own1[k] = psub(own1[k], S);
          own2[k] = padd(own2[k], S);
          const float2 Rv = make_float2(hx2 * s.xx, hx2 * s.xy);
          nr1 = padd(nr1, Rv);
          nr2 = padd(nr2, Rv);
          nl1 = psub(nl1, Rv);
          nl2 = psub(nl2, Rv);
          if (owned_edge) se += exx * s.xx + eyy * s.yy + gxy * s.xy;
        }
      } else {
        {  // h(c_k, t-1): above element (c_k, t-1), below (c_k, t-2)
          const bool ia = es0[k] == ST_INTACT, ib = es1[k] == ST_INTACT, both = ia && ib;
          const float2 upv = padd(Dy1[k], DyR1), dnv = padd(Dy2[k], DyR2k);
          const float2 sY = both ? padd(upv, dnv) : (ia ? upv : dnv);
          const float fy = both ? 0.5f * hy2 : hy2;
          const float2 mD = pmul(RX, Dx1[k]);
          const float exx = mD.x, eyy = fy * sY.y, gxy = fmaf(fy, sY.x, mD.y);
          const Stress3 s = stress32(mq, exx, eyy, gxy);
          const Stress3 A = masked(s, ia), B = masked(s, ib);
          // node (c_k, t-1) is the left node of h, its right neighbour the right node
          const float2 T = pmul(HY2, psub(make_float2(B.xy, B.yy), make_float2(A.xy, A.yy)));
          const float2 P = pmul(RX, padd(make_float2(A.xx, A.xy), make_float2(B.xx, B.xy)));
          own1[k] = padd(own1[k], psub(T, P));
          nr1 = padd(nr1, padd(T, P));
          // upper nodes of the element below, lower nodes of the element above
          const float2 Bv = make_float2(hy2 * B.xy, hy2 * B.yy);
          const float2 Av = make_float2(hy2 * A.xy, hy2 * A.yy);
          own0[k] = psub(own0[k], Bv);
          nr0 = psub(nr0, Bv);
          own2[k] = padd(own2[k], Av);
          nr2 = padd(nr2, Av);
          if (owned_edge) {
            const float w = both ? 1.f : ((ia || ib) ? 0.5f : 0.f);
            se += w * (exx * s.xx + eyy * s.yy + gxy * s.xy);
          }
        }
        {  // v(c_k, t-1): right element (c_k, t-1), left (c_k - 1, t-1)
          const bool ir = es0[k] == ST_INTACT, il = esL0 == ST_INTACT, both = ir && il;
          const float2 rt = padd(Dx1[k], Dx0[k]), lt = padd(DxL1k, DxL0);
          const float2 sX = both ? padd(rt, lt) : (ir ? rt : lt);
          const float fx = both ? 0.5f * hx2 : hx2;
          const float2 mD = pmul(RY, Dy1[k]);
          const float exx = fx * sX.x, eyy = mD.y, gxy = fmaf(fx, sX.y, mD.x);
          const Stress3 s = stress32(mq, exx, eyy, gxy);
          const Stress3 R = masked(s, ir), L = masked(s, il);
          // node (c_k, t-1) is the lower node of v, node (c_k, t) its upper node
          const float2 S = pmul(RY, padd(make_float2(R.xy, R.yy), make_float2(L.xy, L.yy)));
          const float2 W = pmul(HX2, psub(make_float2(L.xx, L.xy), make_float2(R.xx, R.xy)));
          own1[k] = padd(own1[k], psub(W, S));
          own2[k] = padd(own2[k], padd(W, S));
          // left nodes of the element right, right nodes of the element left
          const float2 Rv = make_float2(hx2 * R.xx, hx2 * R.xy);
          const float2 Lv = make_float2(hx2 * L.xx, hx2 * L.xy);
          nr1 = padd(nr1, Rv);
          nr2 = padd(nr2, Rv);
          nl1 = psub(nl1, Lv);
          nl2 = psub(nl2, Lv);
          if (owned_edge) {
            const float w = both ? 1.f : ((ir || il) ? 0.5f : 0.f);
            se += w * (exx * s.xx + eyy * s.yy + gxy * s.xy);
          }
        }
      }
    }
    }
    // ---- pieces of split elements (c_k, t-2), prefetched into L1 one row ago:
    // local nodes 0 (c_k, t-2), 1 (c_k+1, t-2), 2 (c_k+1, t-1), 3 (c_k, t-1)
    if (!CLEAN && __any_sync(FULL, pk_on != 0)) {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if ((pk_on >> k) & 1) {
          const float4 *q = reinterpret_cast<const float4 *>(d.pfe) + (size_t)((t - 2) * g.nx + c0 + k) * 2;
          const float4 p0 = q[0], p1 = q[1];
          float2 &nr0 = k < K - 1 ? own0[k < K - 1 ? k + 1 : k] : ua0;
          float2 &nr1 = k < K - 1 ? own1[k < K - 1 ? k + 1 : k] : ua1;
          own0[k] = padd(own0[k], make_float2(p0.x, p0.y));
          nr0 = padd(nr0, make_float2(p0.z, p0.w));
          nr1 = padd(nr1, make_float2(p1.x, p1.y));
          own1[k] = padd(own1[k], make_float2(p1.z, p1.w));
        }
      }
    }
    pk_on = 0;
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (es0[k] == ST_CRACKED) {
        pk_on |= 1u << k;
        prefetch_l1(d.pfe + (size_t)((t - 1) * g.nx + c0 + k) * 8);
      }
    // ---- nodes (c_k, t-2): every edge and piece touching them is in
    {
      const float ux = __shfl_up_sync(FULL, ua0.x, 1), uy = __shfl_up_sync(FULL, ua0.y, 1);
      const float dx = __shfl_down_sync(FULL, da0.x, 1), dy = __shfl_down_sync(FULL, da0.y, 1);
      own0[0] = padd(own0[0], make_float2(ux, uy));
      own0[K - 1] = padd(own0[K - 1], make_float2(dx, dy));
    }
    const int r = t - 2;
    if (own_lane && r >= j0 && r <= g.ny) {
      const int s2 = (r + 4 * kRing) & (kRing - 1);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int c = c0 + k;
        if (c > g.nx) continue;
        const int N = r * stride + c;
        const float fx = own0[k].x, fy = own0[k].y;
        if (nf2[k]) {
          // nodes with loads or prescribed velocities are updated after the
          // march (FP64 work, out of the loop's registers)
          d.fsp[N] = make_float2(fx, fy);
          spmask[k] |= 1ull << (r - j0);
        } else {
          const float4 Uo = ring.u[s2][k][lane];
          const float2 vo = ring.v[s2][k][lane];
          const float mio = ring.mi[s2][k][lane];
          const float vxn = fmaf(dtv, -fx * mio, vo.x);
          const float vyn = fmaf(dtv, -fy * mio, vo.y);
          d.v2[N] = make_float2(vxn, vyn);
          bad |= !(fabsf(vxn + vyn) <= FLT_MAX);  // NaN or Inf in either
          float4 U = Uo;
          df_add(U.x, U.y, dt * vxn);
          df_add(U.z, U.w, dt * vyn);
          d.u4[cur ^ 1][N] = U;
          if (ENERGY && mio > 0.f) {
            const float bx = first ? vo.x : 0.5f * (vo.x + vxn);
            const float by = first ? vo.y : 0.5f * (vo.y + vyn);
            ke2 += __fdividef(fmaf(bx, bx, by * by), mio);
          }
        }
      }
    }
    // ---- the next row in flight, then advance the pipeline by one row
    stage(t + kAhead);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      U1[k] = U0[k];
      es1[k] = es0[k];
      nf2[k] = nf1[k]; nf1[k] = nf0[k];
      Dx1[k] = Dx0[k];
      Dy2[k] = Dy1[k];
      own0[k] = own1[k]; own1[k] = own2[k];
    }
    DxL1 = DxLf;
    DyR2 = DyRl;
    ua0 = ua1; ua1 = ua2;
    da0 = da1; da1 = da2;
  }
  cp_async_wait<0>();  // no copy into the ring outlives the tile
#pragma unroll
  for (int k = 0; k < K; ++k) {
    while (spmask[k]) {
      const int r = j0 + __ffsll((long long)spmask[k]) - 1;
      spmask[k] &= spmask[k] - 1;
      const int N = r * stride + c0 + k;
      const float2 F = d.fsp[N];
      ke += update_special(d, N, cur, first, F.x, F.y, u4[N], d.v2[N], d.minvf[N],
                           (int)d.nflag[N], ENERGY ? 1 : 0);
    }
  }
  // a non-finite velocity (NaN or Inf) is reported through the status word
  if (__any_sync(FULL, bad) && lane == 0) atomicOr(&d.cnt->status, STAT_NONFINITE);
  if (ENERGY) {
    double a = ke + 0.5 * (double)ke2, b = (double)se;
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(FULL, a, o);
      b += __shfl_down_sync(FULL, b, o);
    }
    if (lane == 0) {
      part[0] = a;
      part[1] = b;
    }
  }
}

// A CTA of four warps takes a group of four consecutive tiles (tile index
// = tile row * tiles per row + tile column); warp w marches tile 4 g + w.
// Neighbouring warps share their halo columns through L1.  Each tile writes
// its own energy partial pair, tiles past the last write zeros.
constexpr int kMarchWarps = 4;
// tile heights: at least 8 node rows (the energy partials are sized for
// that), at most 64 (one bit per owned row; cem_batch_set_config checks it)
constexpr int kMarchRowsMin = 8;

__host__ __device__ inline int march_tiles_x(int nx) { return (nx + 1 + WX - 1) / WX; }
__host__ __device__ inline int march_tiles_y(int ny, int ty) { return (ny + 1 + ty - 1) / ty; }
__host__ __device__ inline int march_groups(int nx, int ny, int ty) {
  return (march_tiles_x(nx) * march_tiles_y(ny, ty) + kMarchWarps - 1) / kMarchWarps;
}

// Warp-uniform: every element of rows j0-2 .. j0+TY that the tile's lanes
// read is intact, and no owned node of rows j0 .. j0+TY-1 has a load or a
// prescribed velocity (from the row flags; tiles at the mesh edge are never
// clean).
__device__ __forceinline__ bool tile_clean(const DevState &d, int tile_x, int j0, int TY) {
  const int ntx = march_tiles_x_of(d.g.nx), lane = threadIdx.x & 31;
  bool ok = true;
  for (int q = lane; q < TY + 3; q += 32) {
    const int r = j0 - 2 + q;
    const int f = (r >= 0 && r <= d.g.ny) ? (int)__ldcg(d.mrow + (size_t)r * ntx + tile_x) : 0;
    ok = ok && (f & 0x100) && (r < j0 || r >= j0 + TY || (f & 1));
  }
  return __all_sync(0xffffffffu, ok);
}

template <bool ENERGY>
__device__ __forceinline__ void march32_group(const DevState &d, int group, int ty, int cur,
                                              int first, MarchRing *rings) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tix = group * kMarchWarps + w;
  const int ntx = march_tiles_x(d.g.nx), nty = march_tiles_y(d.g.ny, ty);
  double *part = d.e_part + 2 * tix;
  if (tix < ntx * nty) {
    const int tile_x = tix % ntx, tile_y = tix / ntx;
    if (tile_clean(d, tile_x, tile_y * ty, ty)) {
      march32_tile<ENERGY, true>(d, tile_x, tile_y, ty, cur, first, part, rings[w]);
    } else {
      // the other tiles read the piece forces of the kernel before this one
      // (when launched as its programmatic dependent): wait until it has
      // completed and its writes are visible
      asm volatile("griddepcontrol.wait;" ::: "memory");
      march32_tile<ENERGY, false>(d, tile_x, tile_y, ty, cur, first, part, rings[w]);
    }
  } else if (ENERGY && lane == 0) {
    part[0] = 0.0;
    part[1] = 0.0;
  }
}

template <bool ENERGY>
__global__ void __launch_bounds__(32 * kMarchWarps, 4) k_march32(DevState d, int cur, int first,
                                                                  int ty) {
  // launched as a programmatic dependent of the kernel before it (the piece
  // forces), which writes only the piece forces and its energy partials: a
  // clean tile reads neither and starts at once, the others wait for that
  // kernel (march32_group).  Everything else the tiles read was written by
  // kernels that completed before the piece forces started.  The kernels
  // that follow may be placed once every CTA of this kernel has started
  // (they wait for it themselves).
  asm volatile("griddepcontrol.launch_dependents;");
  __shared__ MarchRing rings[kMarchWarps];
  march32_group<ENERGY>(d, blockIdx.x, ty, cur, first, rings);
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
    // -1 unused: the phantom is local node a of piece p of split c
    const int4 uf = reinterpret_cast<const int4 *>(d.ph_upf)[t];
    const int ufs[4] = {uf.x, uf.y, uf.z, uf.w};
    float fx = 0.f, fy = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (ufs[q] >= 0) {
        const float2 F = *reinterpret_cast<const float2 *>(d.pff + ufs[q]);
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
// 1-D items are (member, block, energy-partial offset, member's grid size);
// the node update's items are (member, tile group, 0, groups).
template <bool ENERGY>
__global__ void __launch_bounds__(32 * kMarchWarps, 4) k_march32_batch(BatchDev b, int first,
                                                                        int ty) {
  __shared__ DevState sd;
  __shared__ MarchRing rings[kMarchWarps];
  int held = -1, w0, w1;
  const int n = *b.bstep;
  block_range(b.n_main, w0, w1);
  for (int w = w0; w < w1; ++w) {
    const int4 it = b.w_main[w];
    stage_member(b.ds, it.x, sd, held);
    if (!member_active(sd, n)) continue;
    march32_group<ENERGY>(sd, it.y, ty, member_cur(sd, n), first, rings);
  }
}


__global__ void k_pieces32_batch(BatchDev b, int energy) {
  __shared__ DevState sd;
  int held = -1, w0, w1;
  const int n = *b.bstep;
  block_range(b.n_pieces, w0, w1);
  for (int w = w0; w < w1; ++w) {
    const int4 it = b.w_pieces[w];
    stage_member(b.ds, it.x, sd, held);
    if (!member_active(sd, n)) continue;
    pieces32(sd, VBlk{it.y, 0, it.w, 1}, member_cur(sd, n), energy, it.z);
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

cudaError_t set_all_smem_attrs() {
  static bool done = false;
  if (!done) {
    // every kernel of the step asks for one shared-memory split, so that the
    // side branches can share SMs with the node update
    cudaError_t e = match_tile_carveout(k_phantom32);
    if (e == cudaSuccess) e = match_tile_carveout(k_phantom32_batch);
    if (e == cudaSuccess) e = match_tile_carveout(k_pieces32);
    if (e == cudaSuccess) e = match_tile_carveout(k_pieces32_batch);
    if (e == cudaSuccess) e = match_tile_carveout(k_march32<true>);
    if (e == cudaSuccess) e = match_tile_carveout(k_march32<false>);
    if (e == cudaSuccess) e = match_tile_carveout(k_march32_batch<true>);
    if (e == cudaSuccess) e = match_tile_carveout(k_march32_batch<false>);
    if (e != cudaSuccess) return e;
    done = true;
  }
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_eval32(const DevState &d, int cur, cudaStream_t st);
cudaError_t launch_eval32_batch(const BatchDev &b, cudaStream_t st);

// Tile height of a mesh stepped alone: 8 node rows.  Many short tiles (3-4
// waves of resident warps on the 2048 x 2048 plate) measured faster than
// one wave of tall ones (2048^2 step: 65 us at 8 rows, 73 at 16, 96 at 32).
int march_rows_solo(const DevState &) { return kMarchRowsMin; }

namespace {
// one thread per (node row, tile column) entry of the row flags
__global__ void k_march_rows(DevState d) {
  const Geo &g = d.g;
  const int ntx = march_tiles_x_of(g.nx), stride = g.nx + 1;
  const long n = (long)(g.ny + 1) * ntx;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    const int r = (int)(q / ntx), tx = (int)(q % ntx);
    bool quiet = true;
    for (int c = tx * kMarchWX; c < tx * kMarchWX + kMarchWX && c <= g.nx; ++c)
      quiet = quiet && d.nflag[r * stride + c] == 0;
    bool intact = r < g.ny;
    for (int c = tx * kMarchWX - kMarchLeft; intact && c < tx * kMarchWX - kMarchLeft + kMarchSpan; ++c)
      intact = c >= 0 && c < g.nx && d.estate[r * g.nx + c] == ST_INTACT;
    d.mrow[q] = (uint16_t)((quiet ? 1 : 0) | (intact ? 0x100 : 0));
  }
}
}  // namespace

cudaError_t launch_march_rows(const DevState &d, cudaStream_t st) {
  const long n = (long)(d.g.ny + 1) * march_tiles_x_of(d.g.nx);
  const int grid = (int)std::min<long>((n + 255) / 256, 4096);
  k_march_rows<<<grid, 256, 0, st>>>(d);
  return cudaGetLastError();
}

// energy partials of the node update: one per tile, in groups of four
int tiles_fp32(const DevState &d, int tile_rows) {
  return march_groups(d.g.nx, d.g.ny, tile_rows) * kMarchWarps;
}
int groups_fp32(const DevState &d, int tile_rows) {
  return march_groups(d.g.nx, d.g.ny, tile_rows);
}

// energy partials: tiles of the smallest tile height first, then the piece
// blocks (at most 1216), then the phantom update's warps (at most 1216
// blocks of kPhWarps)
int energy_parts_fp32(const DevState &d) { return tiles_fp32(d, 8) + kPhWarps * 1216 + 1216 + 8; }

// piece-force blocks: one thread per split element in FP32, per piece in FP64
int grid_pieces(const DevState &d) {
  return grid_for(d.precision == 1 ? d.ck_cap : 2 * d.ck_cap, 256, 1216);
}
// side-branch grids: two phantom blocks and one evaluation block per SM, so that
// they start together with the node update and share the SMs with it
int grid_phantoms(const DevState &d) { return grid_for(d.ph_cap, 256, 304); }

// energy partials one FP32 step writes with the given tile height
int energy_parts_step_fp32(const DevState &d, int tile_rows) {
  return tiles_fp32(d, tile_rows) + grid_pieces(d) + kPhWarps * grid_phantoms(d);
}

cudaError_t launch_step_fp32(const DevState &d, int cur, bool first, bool energy,
                             const StepStreams &ss, cudaEvent_t *marks) {
  const int ty = march_rows_solo(d);
  const int groups = groups_fp32(d, ty);
  const int tiles = groups * kMarchWarps;  // energy partials: tiles, piece blocks, phantom warps
  const int gp = grid_pieces(d);
  const int gph = grid_phantoms(d);
  const int en = energy ? 1 : 0, f = first ? 1 : 0;
  cudaError_t e = set_all_smem_attrs();
  if (e != cudaSuccess) return e;
  cudaStream_t st = ss.main;
  auto node_update = [&]() {
    // a programmatic dependent of the piece forces before it on the main stream
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(groups);
    cfg.blockDim = dim3(32 * kMarchWarps);
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (energy) cudaLaunchKernelEx(&cfg, k_march32<true>, d, cur, f, ty);
    else cudaLaunchKernelEx(&cfg, k_march32<false>, d, cur, f, ty);
  };
  if (marks) {
    // the step's kernels one after another
    k_pieces32<<<gp, 256, 0, st>>>(d, cur, en, tiles);
    cudaEventRecord(marks[0], st);
    node_update();
    cudaEventRecord(marks[1], st);
    k_phantom32<<<gph, 32 * kPhWarps, 0, st>>>(d, cur, f, en, tiles + gp);
    cudaEventRecord(marks[2], st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_eval32(d, cur, st);
  }
  // the surface evaluation and selection read only the state before the
  // step (aux2); the piece forces come first on main, then the node update
  // there and the phantom update (aux1) side by side
  cudaEventRecord(ss.fork, st);
  cudaStreamWaitEvent(ss.aux2, ss.fork, 0);
  e = launch_eval32(d, cur, ss.aux2);
  if (e != cudaSuccess) return e;
  e = launch_select(d, TRACK_STEP, ss.aux2);
  if (e != cudaSuccess) return e;
  k_pieces32<<<gp, 256, 0, st>>>(d, cur, en, tiles);
  cudaEventRecord(ss.join1, st);
  cudaStreamWaitEvent(ss.aux1, ss.join1, 0);
  k_phantom32<<<gph, 32 * kPhWarps, 0, ss.aux1>>>(d, cur, f, en, tiles + gp);
  node_update();
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
  const int gm = grid_main < 1 ? 1 : grid_main;
  const int gp = grid_for(b.n_pieces, 1, 1216), gph = grid_for(b.n_ph, 1, 1216);
  const int f = first ? 1 : 0, en = energy ? 1 : 0;
  cudaStream_t st = ss.main;
  cudaEventRecord(ss.fork, st);
  cudaStreamWaitEvent(ss.aux2, ss.fork, 0);
  e = launch_eval32_batch(b, ss.aux2);
  if (e != cudaSuccess) return e;
  e = launch_select_batch(b, ss.aux2);
  if (e != cudaSuccess) return e;
  k_pieces32_batch<<<gp, 256, 0, st>>>(b, en);
  cudaEventRecord(ss.join1, st);
  cudaStreamWaitEvent(ss.aux1, ss.join1, 0);
  k_phantom32_batch<<<gph, 32 * kPhWarps, 0, ss.aux1>>>(b, f, en);
  const dim3 block(32 * kMarchWarps);
  if (energy) k_march32_batch<true><<<gm, block, 0, st>>>(b, f, tile_rows);
  else k_march32_batch<false><<<gm, block, 0, st>>>(b, f, tile_rows);
  cudaEventRecord(ss.join1, ss.aux1);
  cudaEventRecord(ss.join2, ss.aux2);
  cudaStreamWaitEvent(st, ss.join1, 0);
  cudaStreamWaitEvent(st, ss.join2, 0);
  return cudaGetLastError();
}

const void *phantom32_kernel() { return reinterpret_cast<const void *>(&k_phantom32); }

}  // namespace cem
