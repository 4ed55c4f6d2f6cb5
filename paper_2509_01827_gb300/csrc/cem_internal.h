// cem_internal.h -- device state and kernel entry points of libcem (not part
// of the public ABI; see include/cem.h for that).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cem {

enum : int { ST_INTACT = 0, ST_CRACKED = 1, ST_OUT = 2 };

// node flags
enum : uint8_t { NF_LOADED = 1, NF_DIRX = 2, NF_DIRY = 4 };

// device status bits
enum : int { STAT_CAPACITY = 1, STAT_NONFINITE = 2, STAT_TIMEOUT = 4 };

// FP32 node-update tiles: tile column tx owns node columns
// [tx * kMarchWX, tx * kMarchWX + kMarchWX) and its lanes read element
// columns [tx * kMarchWX - kMarchLeft, tx * kMarchWX - kMarchLeft + kMarchSpan).
constexpr int kMarchWX = 60, kMarchLeft = 2, kMarchSpan = 64;
__host__ __device__ inline int march_tiles_x_of(int nx) { return (nx + kMarchWX) / kMarchWX; }

// Counters live in device memory so that captured graphs can be replayed.
struct Counters {
  int n_ph;       // phantom nodes in use
  int n_ck;       // split elements in use
  int n_S;        // surface-list length (including tombstones)
  int n_dead;     // tombstones in the surface list
  int n_prop;     // proposals of the current step
  int status;     // STAT_* bits
  int step;       // steps taken
  int lam_base;   // first step of the uploaded load-factor table
  int n_rec;      // energy records written
  int n_win_last; // winners of the last step (diagnostic)
  int n_prop_last; // proposals of the last step (diagnostic)
  // planned by the selection kernel, committed by the apply kernel
  int pend_nwin, pend_nph, pend_nck, pend_nS, pend_dead;
  int pend_step;  // step of the planned splits (read by the apply kernel)
  int pad[1];
  int apply_done;  // blocks of the split writes finished this step (status ring)
};

struct Geo {
  int nx, ny, nn, ne, nh, ned;
  double hx, hy, A;
  double rx, rxh, ry, ryh; // 1/hx, 0.5/hx, 1/hy, 0.5/hy
  // FP32 copies for the FP32-mixed kernels (no FP64 work on the hot path)
  float rxf, ryf, qAf;     // 1/hx, 1/hy, A/4
  float DXf[4], DYf[4];    // reference vector X_N2 - X_N1 of local edge k
  float nxf[4][4], nyf[4][4];  // unit normal of candidate path k0 -> k
};

struct Mat {
  double D11, D12, D33, rho, gamma, dt;
  int gamma_mode, scope;
  float D11f, D12f, D33f, dtf;
};

// Surface-list entry payload: packed (ahead element * 4 + local edge k0).
struct DevState {
  Geo g;
  Mat mat;
  int precision;
  int ph_cap, ck_cap, list_cap, prop_cap, ncap;
  int lam_cap;
  // batched stepping (cem_batch_create): the member takes no step at or
  // after step_end (INT_MAX when stepped alone), and its current
  // displacement buffer at batch step n is (n & 1) ^ cur_xor
  int step_end, cur_xor;

  // node arrays over ncap = nn + ph_cap; FP64 mode
  double *ux[2], *uy[2];
  double *vx, *vy;
  // FP32-mixed mode, one record per node: displacement as compensated
  // float pairs (x.hi, x.lo, y.hi, y.lo) and velocity (x, y)
  float4 *u4[2];
  float2 *v2;
  float *minvf;
  double *m, *minv;
  double *Wn, *Wd;
  uint8_t *nflag;        // [nn]
  double *Fx, *Fy;       // [nn] Neumann load at unit load factor
  double *Vx, *Vy;       // [nn] prescribed velocity at unit load factor
  int *bc_nodes;         // nodes with a load or a prescribed velocity
  int n_bc;

  // elements
  uint8_t *estate;       // [ne]
  int *crack_of;         // [ne]
  float *gc;             // [ne]

  // split-element table [ck_cap]
  int *ck_elem;
  int *ck_info;          // ka | kb << 2 | side(a) << (4 + a)
  int *ck_node;          // [ck_cap * 8], piece p local a at p*4+a
  double *ck_Ap;         // [ck_cap * 2]
  double *ck_ud;
  int *ck_step;
  double *pf;            // [ck_cap * 16] piece nodal forces (FP64 mode)
  float *pff;            // [ck_cap * 16] piece nodal forces (FP32 mode)
  float *pfe;            // [ne * 8] FP32 mode: forces of a split element's pieces at its
                         // four real nodes (local node a: the piece on its side)
  float2 *fsp;           // [nn] FP32 mode: internal force of a node with a load or a
                         // prescribed velocity, handed from the march to its update
  // [(ny + 1) * march_tiles_x_of(nx)] row flags of the FP32 node update, per
  // node row r and tile column: low byte 1 when no owned node of the tile in
  // row r has a load or a prescribed velocity, high byte 1 when every
  // element of row r that the tile's lanes read is intact (cleared by the
  // apply kernel when it splits one of them)
  uint16_t *mrow;

  // phantoms [ph_cap]
  int *ph_owner;
  int *ph_creator;       // e * 4 + a
  int *ph_nuser;
  int *ph_users;         // [ph_cap * 4], (e << 3) | (p << 2) | a, sorted by e
  int *ph_upf;           // [ph_cap * 4], piece-force index c*16 + p*8 + 2a of each user, -1 unused
  double *ph_uap;        // [ph_cap * 4], area of each user's piece

  // surface list [list_cap]
  int *S;                // edge id or -1 (tombstone)
  int *S_info;           // ahead * 4 + k0
  double *S_G;           // largest candidate G at the last evaluation
  int *spos;             // [ned] position in S or -1

  // proposals of the current step [prop_cap]
  int *pr_key;           // ahead * 4 + k0
  int *pr_edge;
  int *pr_k;
  double *pr_G;

  // split plans of the current step [prop_cap], in increasing element id
  int *pl_e;
  int *pl_info;          // ka | kb << 2 | side(a) << (4+a) | append(k) << (8+k)
  int *pl_reuse;         // [4] phantom reused for local node a, or -1
  int *pl_tomb;          // [4] surface-list position to tombstone for edge k, or -1
  int *pl_c;             // split-table slot
  int *pl_ph0;           // first new phantom id
  int *pl_app0;          // first surface-list position of its appended edges
  double *pl_alpha;      // [2] piece area fractions
  // per local node a of each plan, computed by the selection kernel so that
  // the split writes need no dependent loads: the real node's mass after the
  // split, its phantom's mass after it, the phantom's mass before (-1: new),
  // the mass the phantom gains, and the phantom's complete user list
  double *pl_mreal, *pl_mph, *pl_mold, *pl_dm;  // [4]
  double *pl_mireal, *pl_miph;  // [4] inverses of pl_mreal and pl_mph (0 for no mass)
  int *pl_users, *pl_upf;  // [16]: 4 users of the phantom of each local node
  double *pl_uap;          // [16]: their piece areas
  int *pl_nu;              // [4]

  // selection scratch for steps with more proposals than its shared memory
  // holds [prop_cap]: sorted keys, winners, G, edge and exit edge
  unsigned long long *sel_sk;
  int *sel_win;
  double *sel_G;
  int *sel_E;
  uint8_t *sel_K;

  Counters *cnt;
  double *lamN, *lamD;   // [lam_cap] load factors of steps lam_base + i

  // energy
  double *e_part;        // per-block partial sums
  int e_part_cap;
  double *e_pre;         // [EPRE * 3] partial sums of the energy prologue
  double *erec;          // [rec_cap * 7]
  int rec_cap;
};

// A virtual thread block.  Kernels stepped alone use the hardware block;
// batched kernels take (member, block) items from a work list, so that every
// member sees the same block decomposition (and the same fixed-order energy
// partial sums) as when it is stepped alone.
// The energy prologue sums the boundary work and the dissipated energy in
// EPRE fixed chunks (one block of EPRE_TB threads each), added in order by
// the epilogue.
constexpr int EPRE = 128, EPRE_TB = 256;
// warps of an FP32 phantom-update block; each writes its own energy partial
constexpr int kPhWarps = 8;

struct VBlk {
  int x, y, gx, gy;
};
#ifdef __CUDACC__
__device__ __forceinline__ VBlk hw_vblk() {
  return VBlk{(int)blockIdx.x, (int)blockIdx.y, (int)gridDim.x, (int)gridDim.y};
}
#endif

// Device view of a batch of independent meshes stepped in lock-step by one
// launch per kernel kind.  Work items are int4 (member, x, y, gx | gy << 16).
struct BatchDev {
  const DevState *ds;   // [n] device copies of the members' states
  int n;
  int *bstep;           // batch step; advanced by the last block of the apply kernel
  int *arrive;          // arrival counter of that kernel (returns to 0)
  const int4 *w_main; int n_main;      // tile update
  const int4 *w_pieces; int n_pieces;  // piece forces
  const int4 *w_ph; int n_ph;          // phantom update
  const int4 *w_eval; int n_eval;      // surface evaluation
  const int *nparts;    // [n] energy partial sums of each member
};

#ifdef __CUDACC__
__device__ __forceinline__ VBlk item_vblk(int4 it) {
  return VBlk{it.y, it.z, it.w & 0xffff, it.w >> 16};
}
// member is stepped at batch step n
__device__ __forceinline__ bool member_active(const DevState &d, int n) { return n < d.step_end; }
__device__ __forceinline__ int member_cur(const DevState &d, int n) { return (n & 1) ^ d.cur_xor; }

// A block's share of a work list: a contiguous range, so that consecutive
// items mostly belong to one member.
__device__ __forceinline__ void block_range(int n, int &begin, int &end) {
  begin = (int)(((long long)n * blockIdx.x) / gridDim.x);
  end = (int)(((long long)n * (blockIdx.x + 1)) / gridDim.x);
}

// Copies member s's state into the block's shared copy `sh` when it is not
// already there (block-uniform; `held` is the member held, -1 at first).
// Kernels then read the state from shared memory instead of re-loading its
// fields from global memory after every store.
__device__ __forceinline__ void stage_member(const DevState *ds, int s, DevState &sh, int &held) {
  if (s == held) return;
  __syncthreads();  // every thread is done with the previous member
  const int nt = blockDim.x * blockDim.y;
  const int t = threadIdx.x + threadIdx.y * blockDim.x;
  const int *src = reinterpret_cast<const int *>(ds + s);
  int *dst = reinterpret_cast<int *>(&sh);
  for (int i = t; i < (int)(sizeof(DevState) / 4); i += nt) dst[i] = src[i];
  __syncthreads();
  held = s;
}
#endif

// ------------------------------------------------------------------ launch
// The kernels that run beside the FP32 tile update ask for the shared-memory
// split the tile update itself runs in (164 KB of shared memory for its
// four 40 KB CTAs, the rest L1).  An SM changes its L1 / shared split only
// when it is empty, so a side kernel left at its own small split would keep
// the tile update off every SM it occupies until it drains.  71% of the 228
// KB maximum is the smallest request that maps to the 164 KB split.
constexpr int kSideCarveoutPct = 71;
template <class K>
inline cudaError_t match_tile_carveout(K *kernel) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                              kSideCarveoutPct);
}

// All launchers enqueue on `st` and return cudaGetLastError().
cudaError_t launch_init_masses(const DevState &d, cudaStream_t st);
// Streams of one step.  The tile update of real nodes (main), the phantom
// update (aux1) and the surface evaluation followed by the tracking
// selection (aux2, read only the previous state) run concurrently and join
// back into `main`, where the split writes follow; the side branches' streams
// have the highest priority.  In FP32 the tile and phantom updates evaluate
// the split pieces they need themselves; in FP64 the piece forces run on
// `main` before the tile and phantom updates.  With marks (profiling) the four step kernels
// (the FP32 piece evaluation timed on its own) run one after the other on
// `main`, marks[0..2] are recorded after the first three, and the caller
// launches selection and writes.
struct StepStreams {
  cudaStream_t main, aux1, aux2;
  cudaEvent_t fork, join1, join2;
};
// Kernel functions the step graphs' edges are checked against
// (ordinary_side_edges in api.cpp).
const void *apply_kernel();
const void *select_kernel();
const void *phantom32_kernel();
const void *phantom64_kernel();
constexpr int kStepKernels = 4;
cudaError_t launch_step_fp64(const DevState &d, int cur, bool first, bool energy,
                             const StepStreams &ss, cudaEvent_t *marks = nullptr);
cudaError_t launch_step_fp32(const DevState &d, int cur, bool first, bool energy,
                             const StepStreams &ss, cudaEvent_t *marks = nullptr);
// Tracking: selection and planning (one CTA; may run concurrently with the
// node updates) then the split writes (many CTAs; after the node updates).
cudaError_t launch_select(const DevState &d, int mode, cudaStream_t st);
// programmatic: launched as a programmatic dependent of the kernel before it
// (used in captured step graphs, whose edges ordinary_side_edges fixes);
// ring: when given, the last block to finish copies the counters into
// ring[steps taken % kStatusRing] (mapped pinned memory)
cudaError_t launch_apply(const DevState &d, int cur_next, int mode, cudaStream_t st,
                         bool programmatic = false, Counters *ring = nullptr);
cudaError_t launch_build_surface(const DevState &d, cudaStream_t st);
// copies the counters into host_mapped (a device alias of mapped pinned memory)
cudaError_t launch_status_copy(const Counters *cnt, Counters *host_mapped, cudaStream_t st);
// slots of the per-step status ring of pipelined step calls; a call of at
// most kStatusRing / 2 steps has every step's status word read back
constexpr int kStatusRing = 64;
// proposals one step can hold: the selection sorts (a power of two) that many
// at most, in shared memory or in its global scratch of that size
int track_sort_capacity();
cudaError_t launch_surface_info(const DevState &d, int *out3, cudaStream_t st);
cudaError_t launch_debug_filter(const DevState &d, int n, cudaStream_t st);
cudaError_t launch_energy_pre(const DevState &d, cudaStream_t st);
// element mean stress (sxx, syy, sxy) and largest principal stress into
// out4[0..ne), [ne..2ne), [2ne..3ne), [3ne..4ne)
// rebuilds the node update's row flags from nflag and estate
cudaError_t launch_march_rows(const DevState &d, cudaStream_t st);
cudaError_t launch_element_stress(const DevState &d, int cur, double *out4, cudaStream_t st);
// fragments: labels[2 e + p] of every piece (-1: none), *count fragments;
// device scratch of fragments_scratch_bytes
size_t fragments_scratch_bytes(const DevState &d, int n_nodes);
cudaError_t launch_fragments(const DevState &d, int n_nodes, void *scratch, int *labels,
                             int *count, cudaStream_t st);
cudaError_t launch_energy_post(const DevState &d, int nparts, cudaStream_t st);
cudaError_t launch_fp32_to_fp64(const DevState &d, int cur, double *ux, double *uy,
                                double *vx, double *vy, int n, cudaStream_t st);
cudaError_t launch_fp64_to_fp32(const DevState &d, int cur, const double *ux,
                                const double *uy, const double *vx, const double *vy,
                                int n, cudaStream_t st);
int energy_parts_needed(const DevState &d);  // capacity of e_part
int energy_parts_step(const DevState &d);    // partials one step writes (alone)

// batched counterparts (see BatchDev); tile_rows selects the FP32 tile
// update's tile height (8 or 16 node rows), grid_main its persistent grid
int tiles_fp32(const DevState &d, int tile_rows);   // energy partials of the node update
int groups_fp32(const DevState &d, int tile_rows);  // its CTAs (four warp tiles each)
int tiles_fp64(const DevState &d);
int grid_pieces(const DevState &d);
int grid_phantoms(const DevState &d);
int grid_eval(const DevState &d);
cudaError_t launch_step_fp32_batch(const BatchDev &b, bool first, bool energy, int tile_rows,
                                   int grid_main, const StepStreams &ss);
cudaError_t launch_step_fp64_batch(const BatchDev &b, bool first, bool energy, int grid_main,
                                   const StepStreams &ss);
cudaError_t launch_select_batch(const BatchDev &b, cudaStream_t st);
cudaError_t launch_apply_batch(const BatchDev &b, cudaStream_t st);
cudaError_t launch_energy_pre_batch(const BatchDev &b, cudaStream_t st);
cudaError_t launch_energy_post_batch(const BatchDev &b, cudaStream_t st);
cudaError_t launch_gather_counters(const BatchDev &b, Counters *out, cudaStream_t st);

// track modes
enum : int { TRACK_STEP = 0, TRACK_PRECRACK = 1, TRACK_DEBUG = 2 };

}  // namespace cem
