// track.cu -- multi-tip crack tracking: selection, split and surface list
// (compiled with -fmad=false: the split's masses, momentum merge and
// dissipated energy follow the FP64 expression order of the definition).
//
// Each step's tracking is two kernels.  k_select (one CTA) runs on the
// evaluation stream, concurrently with the node updates, and
//   1. compacts the surface list with warp ballots when half of it is dead;
//   2. sorts the step's proposals by (ahead element, local edge) with a
//      bitonic sort in shared memory (the warp-ballot append of the
//      evaluation is unordered; the sort makes everything after it
//      deterministic);
//   3. selects winners (Sec. 3): a proposal wins if its key (G, -edge id) is
//      the strict maximum among proposals whose ahead elements share a node
//      with its own (binary searches over the three neighbouring rows), or
//      the single global maximum, or -- pre-cracks -- unconditionally;
//   4. plans each winner's split (eight threads per winner): sides of the
//      segment between the entry and exit edge midpoints (crack patterns I
//      and II, Fig. 2-3), phantoms shared with a cracked neighbour across a
//      cut edge, area fractions, split-table slot, phantom ids and
//      surface-list positions by prefix sums in increasing element id, and
//      the lumped masses and phantom user lists the split will produce (no
//      other winner touches the same nodes), so that the writes below need
//      no dependent reads.
// k_apply (many CTAs, eight threads per winner) runs after the node updates
// and only writes the plan: split records, phantoms (copies of u^{n+1},
// v^{n+1/2}), masses, the momentum-conserving merge into shared phantoms,
// U_d = G_c * segment length, surface-list tombstones and appends, and the
// counters.
#include <cuda_runtime.h>
#include <stdint.h>

#include "cem_internal.h"
#include "q4_fp64.cuh"

namespace cem {

namespace {

// Element e is split: the tiles of the FP32 node update whose lanes read its
// column lose the all-intact flag of its row (every tile column tx with
// tx * W - L <= i < tx * W - L + S).
__device__ __forceinline__ void march_rows_split(const DevState &d, int e) {
  if (!d.mrow) return;
  const int i = e % d.g.nx, j = e / d.g.nx, ntx = march_tiles_x_of(d.g.nx);
  const int a = i + kMarchLeft - kMarchSpan;
  const int lo = a < 0 ? 0 : a / kMarchWX + 1;
  const int hi = min((i + kMarchLeft) / kMarchWX, ntx - 1);
  for (int tx = lo; tx <= hi; ++tx)
    reinterpret_cast<uint8_t *>(d.mrow + (size_t)j * ntx + tx)[1] = 0;
}

// The selection CTA is sized to fit in the SM resources one tile-update CTA
// frees (256 threads x 64 registers, under 48 KB of shared memory), so that
// it runs beside the tile update.
constexpr int TB = 256;            // threads of the tracking CTA
constexpr int SORT_CAP = 8192;     // proposals per step (power of two)
constexpr int SEL_SMEM_CAP = 1024; // proposals staged in shared memory (power of two)
constexpr int WB = TB / 8;         // winners split per batch (eight threads each)

// dynamic shared memory of the selection CTA: sorted keys, winners and the
// proposals' G, edge and exit edge, for up to SEL_SMEM_CAP proposals (steps
// with more use the global scratch of the same layout)
constexpr size_t select_smem_bytes() {
  return SEL_SMEM_CAP *
         (sizeof(unsigned long long) + sizeof(int) + sizeof(double) + sizeof(int) + 1);
}

// ------------------------------------------------------------ block scan
// Exclusive scan of v over the block; returns the prefix, *total = sum.
__device__ int block_exscan(int v, int *total) {
  __shared__ int ws[32];
  __shared__ int tot;
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    ws[lane] = s;
    if (lane == 31) tot = s;
  }
  __syncthreads();
  int pre = (w > 0 ? ws[w - 1] : 0) + x - v;
  int t = tot;
  __syncthreads();
  *total = t;
  return pre;
}

__device__ __forceinline__ double inverse_mass(double m) { return m > 0.0 ? 1.0 / m : 0.0; }

// a node's lumped mass and its inverse (planned by the selection, which runs
// beside the node updates, so the split writes do no FP64 division for it)
__device__ void set_mass(const DevState &d, int N, double m, double mi) {
  d.m[N] = m;
  d.minv[N] = mi;
  if (d.precision == 1) d.minvf[N] = (float)mi;
}

// Area fractions of the two pieces by the shoelace formula in natural
// coordinates (the reference square has area 4).  A piece's polygon visits
// the element's nodes and edge points in counter-clockwise order, keeping
// the nodes on its side and the two edge points of the segment; the terms
// are added in that order with the closing term last.
__device__ __forceinline__ void area_fractions(int ka, int kb, const int side[4], double alpha[2]) {
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    double x0 = 0.0, y0 = 0.0, xp = 0.0, yp = 0.0, twice = 0.0;
    bool have = false;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      const int q = w >> 1;
      const bool in = (w & 1) == 0 ? side[q] == p : (q == ka || q == kb);
      if (!in) continue;
      const double x = (w & 1) == 0 ? xi_n(q) : xi_g(q);
      const double y = (w & 1) == 0 ? eta_n(q) : eta_g(q);
      if (!have) {
        x0 = x;
        y0 = y;
        have = true;
      } else {
        twice = twice + (xp * y - x * yp);
      }
      xp = x;
      yp = y;
    }
    twice = twice + (xp * y0 - x0 * yp);
    alpha[p] = fabs(twice) * 0.5 / 4.0;
  }
}

// Sorted proposals live in shared memory as (key << 32 | index).
__device__ __forceinline__ int lower_bound_key(const unsigned long long *sk, int n, int key) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if ((int)(sk[mid] >> 32) < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ bool key_greater(double Ga, int ea, double Gb, int eb) {
  return Ga > Gb || (Ga == Gb && ea < eb);
}

__device__ bool tip_of(const DevState &d, int e, int k0) {
  int f = elem_neighbor(d.g, e, k0);
  if (estatus(d, f) != ST_CRACKED) return false;
  int info = d.ck_info[d.crack_of[f]];
  int kf = (k0 + 2) & 3;
  return (info & 3) == kf || ((info >> 2) & 3) == kf;
}

// Stable compaction of the surface list (warp ballots + block scan).
__device__ void compact_surface(const DevState &d) {
  Counters *cnt = d.cnt;
  int n = cnt->n_S, out = 0;
  for (int base = 0; base < n; base += TB) {
    int i = base + threadIdx.x;
    int e = -1, inf = 0;
    double gl = 0.0;
    if (i < n) { e = d.S[i]; inf = d.S_info[i]; gl = d.S_G[i]; }
    int live = (i < n && e >= 0) ? 1 : 0;
    int tot;
    int pos = block_exscan(live, &tot);
    __syncthreads();  // every read of this chunk precedes the writes
    if (live) {
      int dst = out + pos;
      d.S[dst] = e;
      d.S_info[dst] = inf;
      d.S_G[dst] = gl;
      d.spos[e] = dst;
    }
    out += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    cnt->n_S = out;
    cnt->n_dead = 0;
  }
}

// What the split of element e needs about its local node a (real node N),
// read in two levels of independent loads: the phantom the split reuses and,
// for N's lumped mass after the split, the states of the elements around N
// and the areas of their pieces that hold N.
struct NodePlan {
  int P;          // phantom to reuse, or -1
  int qe;         // position of e among the four elements around N
  int st[4];      // their states (e counted as split, ST_OUT outside)
  double Ap[4];   // area of the piece of each holding N (e's filled in later)
};

__device__ __forceinline__ void node_plan(const DevState &d, int e, int ka, int kb, int a,
                                          NodePlan &np) {
  const Geo &g = d.g;
  const int N = elem_node(g, e, a);
  const int r = g.nx + 1, i = N % r, j = N / r;
  const int di[4] = {-1, 0, -1, 0}, dj[4] = {-1, -1, 0, 0}, la[4] = {2, 3, 1, 0};
  int eq[4], st[4], cq[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int ei = i + di[q], ej = j + dj[q];
    eq[q] = (ei < 0 || ej < 0 || ei >= g.nx || ej >= g.ny) ? -1 : ej * g.nx + ei;
  }
  // level 1: states and split-table slots of the four elements
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    st[q] = eq[q] < 0 ? ST_OUT : (int)d.estate[eq[q]];
    cq[q] = eq[q] < 0 ? -1 : d.crack_of[eq[q]];
  }
  // level 2: split records of the split ones
  int inf[4], nd[4][2];
  double A2[4][2];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    inf[q] = 0;
    nd[q][0] = nd[q][1] = -1;
    A2[q][0] = A2[q][1] = 0.0;
    if (st[q] == ST_CRACKED && eq[q] != e && cq[q] >= 0) {
      const int c = cq[q];
      inf[q] = d.ck_info[c];
      A2[q][0] = d.ck_Ap[c * 2];
      A2[q][1] = d.ck_Ap[c * 2 + 1];
      nd[q][0] = d.ck_node[c * 8 + la[q]];
      nd[q][1] = d.ck_node[c * 8 + 4 + la[q]];
    }
  }
  np.qe = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (eq[q] == e) np.qe = q;
    np.st[q] = eq[q] < 0 ? ST_OUT : (eq[q] == e ? ST_CRACKED : st[q]);
    np.Ap[q] = g.A;
    if (st[q] == ST_CRACKED && eq[q] != e && cq[q] >= 0)
      np.Ap[q] = ((inf[q] >> (4 + la[q])) & 1) ? A2[q][1] : A2[q][0];
  }
  // the phantom to reuse: across the cut edges of e that contain N (first
  // in increasing local edge index), held by a split neighbour whose own
  // segment also cuts that edge
  np.P = -1;
  const int k1 = (a + 3) & 3, k2 = a;
  const int kk[2] = {k1 < k2 ? k1 : k2, k1 < k2 ? k2 : k1};
#pragma unroll
  for (int t = 1; t >= 0; --t) {
    const int k = kk[t];
    if (k != ka && k != kb) continue;
    const int f = elem_neighbor(g, e, k), kf = (k + 2) & 3;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (f >= 0 && eq[q] == f && st[q] == ST_CRACKED && cq[q] >= 0 &&
          ((inf[q] & 3) == kf || ((inf[q] >> 2) & 3) == kf))
        np.P = ((inf[q] >> (4 + la[q])) & 1) ? nd[q][0] : nd[q][1];
    }
  }
}

// Selection and planning (one CTA).  Reads the step's proposals and the
// current crack state, never writes it: the node-update kernels may run
// concurrently.  Produces, for each winner in increasing element id, its
// split plan (sides, phantoms to reuse, area fractions, split-table slot,
// first new phantom id, surface-list appends and tombstones) and the
// counters the apply kernel commits.  Global loads are issued in few
// dependent levels (the proposals' fields are staged in shared memory with
// the keys), since this single CTA runs beside the node updates.
__device__ __forceinline__ void select_plan(const DevState &d, int mode,
                                            unsigned long long *smem) {
  __shared__ int s_n, s_nwin, s_stop, s_nph, s_nck, s_nS, s_dead, s_done, s_compact;
  __shared__ int b_e[WB], b_ka[WB], b_kb[WB], b_side[WB][4], b_reuse[WB][4], b_app[WB],
      b_tomb[WB][4], b_c[WB];
  __shared__ double b_alpha[WB][2];
  // sides of the four nodes (bit a) and area fractions of a split entering
  // at edge point ka and leaving at kb, for the 12 pairs ka != kb
  __shared__ int s_sides[16];
  __shared__ double s_alpha[16][2];
  Counters *cnt = d.cnt;
  const Geo &g = d.g;
  const int tid = threadIdx.x;
  if (tid >= 32 && tid < 48) {
    const int ka = (tid - 32) >> 2, kb = (tid - 32) & 3;
    int side[4] = {0, 0, 0, 0}, bits = 0;
    double alpha[2] = {0.0, 0.0};
    if (ka != kb) {
      const double pax = xi_g(ka), pay = eta_g(ka), pbx = xi_g(kb), pby = eta_g(kb);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const double cross = (pbx - pax) * (eta_n(a) - pay) - (pby - pay) * (xi_n(a) - pax);
        side[a] = cross > 0.0 ? 0 : 1;
        bits |= side[a] << a;
      }
      area_fractions(ka, kb, side, alpha);
    }
    s_sides[tid - 32] = bits;
    s_alpha[tid - 32][0] = alpha[0];
    s_alpha[tid - 32][1] = alpha[1];
  }
  if (tid == 0) {
    const int n_dead = cnt->n_dead, nS = cnt->n_S;
    int n = cnt->n_prop;
    if (n > d.prop_cap) n = d.prop_cap;
    s_n = n;
    s_nph = cnt->n_ph;
    s_nck = cnt->n_ck;
    s_nS = nS;
    // stable compaction of the surface list when half of it is dead (the
    // evaluation of this step has finished; nothing else reads the list now)
    s_compact = mode == TRACK_STEP && n_dead > 1024 && 2 * n_dead > nS;
    s_nwin = 0;
    s_stop = 0;
    s_dead = 0;
    s_done = 0;
  }
  __syncthreads();
  if (s_compact) {
    compact_surface(d);
    __syncthreads();
    if (tid == 0) s_nS = cnt->n_S;
    __syncthreads();
  }
  const int n = s_n;
  // sorted (key << 32 | index), winners (sorted positions), and G, edge and
  // exit edge of proposal i
  const bool staged = n <= SEL_SMEM_CAP;
  unsigned long long *sk = staged ? smem : d.sel_sk;
  int *swin = staged ? (int *)(smem + SEL_SMEM_CAP) : d.sel_win;
  double *oG = staged ? (double *)(smem + SEL_SMEM_CAP) + SEL_SMEM_CAP / 2 : d.sel_G;
  int *oE = staged ? (int *)(oG + SEL_SMEM_CAP) : d.sel_E;
  uint8_t *oK = staged ? (uint8_t *)(oE + SEL_SMEM_CAP) : d.sel_K;
  if (n > 0) {
    // ---- load keys and fields; debug proposals that are not surface points
    //      (or not tips under the tips-only scope) sort to the end
    int P2 = 1;
    while (P2 < n) P2 <<= 1;
    for (int i = tid; i < P2; i += TB) {
      unsigned long long v = ~0ull;
      if (i < n) {
        const int key = d.pr_key[i], ed = d.pr_edge[i], kx = d.pr_k[i];
        oG[i] = d.pr_G[i];
        oE[i] = ed;
        oK[i] = (uint8_t)kx;
        bool valid = true;
        if (mode == TRACK_DEBUG) {
          int pos = d.spos[ed];
          valid = pos >= 0 && d.S_info[pos] == key && kx != (key & 3);
          if (!valid) atomicOr(&cnt->pad[0], 1);
          if (valid && d.mat.scope == 2) valid = tip_of(d, key >> 2, key & 3);
        }
        if (valid) v = ((unsigned long long)(unsigned)key << 32) | (unsigned)i;
      }
      sk[i] = v;
    }
    __syncthreads();
    if (P2 <= 32) {
      // one warp sorts up to 32 keys (no block-wide barriers)
      if (tid < 32) {
        for (int k = 2; k <= P2; k <<= 1) {
          for (int j = k >> 1; j > 0; j >>= 1) {
            const int i = tid, l = i ^ j;
            if (i < P2 && l > i) {
              unsigned long long a = sk[i], b = sk[l];
              bool up = (i & k) == 0;
              if ((a > b) == up) { sk[i] = b; sk[l] = a; }
            }
            __syncwarp();
          }
        }
      }
      __syncthreads();
    } else {
      for (int k = 2; k <= P2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
          for (int i = tid; i < P2; i += TB) {
            int l = i ^ j;
            if (l > i) {
              unsigned long long a = sk[i], b = sk[l];
              bool up = (i & k) == 0;
              if ((a > b) == up) { sk[i] = b; sk[l] = a; }
            }
          }
          __syncthreads();
        }
      }
    }
    __shared__ int s_valid;
    if (tid == 0) s_valid = 0;
    __syncthreads();
    for (int i = tid; i < n; i += TB)
      if (sk[i] != ~0ull && (i + 1 == n || sk[i + 1] == ~0ull)) s_valid = i + 1;
    __syncthreads();
    const int nv = s_valid;

    // ---- winners
    if (mode != TRACK_PRECRACK && d.mat.scope == 1) {
      if (tid == 0) {
        int best = -1;
        for (int i = 0; i < nv; ++i) {
          int idx = (int)(sk[i] & 0xffffffffu);
          if (best < 0 || key_greater(oG[idx], oE[idx], oG[best], oE[best])) best = idx;
        }
        int wi = -1;
        for (int i = 0; i < nv; ++i)
          if ((int)(sk[i] & 0xffffffffu) == best) wi = i;
        if (wi >= 0) { swin[0] = wi; s_nwin = 1; }
      }
      __syncthreads();
    } else {
      for (int base = 0; base < nv; base += TB) {
        int i = base + tid;
        int win = 0;
        if (i < nv) {
          win = 1;
          if (mode != TRACK_PRECRACK) {
            int idx = (int)(sk[i] & 0xffffffffu);
            int key = (int)(sk[i] >> 32), e = key >> 2;
            double G = oG[idx];
            int ed = oE[idx];
            int ei = e % g.nx, ej = e / g.nx;
            for (int dj = -1; dj <= 1 && win; ++dj) {
              int row = ej + dj;
              if (row < 0 || row >= g.ny) continue;
              int lo_e = row * g.nx + (ei > 0 ? ei - 1 : 0);
              int hi_e = row * g.nx + (ei < g.nx - 1 ? ei + 1 : g.nx - 1);
              int q = lower_bound_key(sk, nv, lo_e * 4);
              for (; q < nv && (int)(sk[q] >> 32) <= hi_e * 4 + 3; ++q) {
                if (q == i) continue;
                int qi = (int)(sk[q] & 0xffffffffu);
                if (!key_greater(G, ed, oG[qi], oE[qi])) { win = 0; break; }
              }
            }
          }
        }
        int tot;
        int pos = block_exscan(win, &tot);
        if (win) swin[s_nwin + pos] = i;
        __syncthreads();
        if (tid == 0) s_nwin += tot;
        __syncthreads();
      }
    }
    const int nwin = s_nwin;

    // ---- plan the splits, WB winners at a time, eight threads each
    const int lane = tid & 7, wl = tid >> 3;
    for (int base = 0; base < nwin; base += WB) {
      const int nb = nwin - base < WB ? nwin - base : WB;
      const bool act = wl < nb && !s_stop;
      if (act && lane == 0) {
        const int i = swin[base + wl];
        const int idx = (int)(sk[i] & 0xffffffffu);
        const int key = (int)(sk[i] >> 32);
        b_e[wl] = key >> 2;
        b_ka[wl] = key & 3;
        b_kb[wl] = oK[idx];
        b_app[wl] = 0;
      }
      __syncthreads();
      NodePlan np;
      int nu = 0;
      int4 u4 = make_int4(0, 0, 0, 0), f4 = u4;
      double2 A01 = make_double2(0.0, 0.0), A23 = A01;
      double mold = -1.0;
      if (act && lane < 4) {
        // local node a: side, the phantom to reuse and the mass inputs, then
        // (consumed only after the scans below) the reused phantom's user
        // list with its users' piece areas
        const int e = b_e[wl], ka = b_ka[wl], kb = b_kb[wl], a = lane;
        b_side[wl][a] = (s_sides[ka * 4 + kb] >> a) & 1;
        node_plan(d, e, ka, kb, a, np);
        b_reuse[wl][a] = np.P;
        if (np.P >= 0) {
          const int t = np.P - g.nn;
          nu = d.ph_nuser[t];
          u4 = reinterpret_cast<const int4 *>(d.ph_users)[t];
          f4 = reinterpret_cast<const int4 *>(d.ph_upf)[t];
          A01 = reinterpret_cast<const double2 *>(d.ph_uap)[2 * t];
          A23 = reinterpret_cast<const double2 *>(d.ph_uap)[2 * t + 1];
          mold = d.m[np.P];
        }
      } else if (act) {
        // local edge k: appended to the surface list if the element across
        // it is intact, else its current entry (if any) becomes a tombstone
        const int e = b_e[wl], k = lane - 4;
        const int f = elem_neighbor(g, e, k);
        const int ed = elem_edge(g, e, k);
        const int sf = estatus(d, f), pos = d.spos[ed];
        b_tomb[wl][k] = -1;
        if (sf == ST_INTACT) {
          atomicOr(&b_app[wl], 1 << k);
        } else {
          b_tomb[wl][k] = pos;
        }
      }
      __syncthreads();
      int nnew = 0, napp = 0, ndead = 0;
      if (act && lane == 0) {
        for (int a = 0; a < 4; ++a) {
          nnew += b_reuse[wl][a] < 0;
          ndead += b_tomb[wl][a] >= 0;
        }
        napp = __popc(b_app[wl]);
      }
      int tot_new, tot_app;
      const int pre_new = block_exscan(nnew, &tot_new);
      const int pre_app = block_exscan(napp, &tot_app);
      if (tid == 0) {
        const bool fits = !s_stop && s_nph + tot_new <= d.ph_cap && s_nck + nb <= d.ck_cap &&
                          s_nS + tot_app <= d.list_cap;
        if (!fits) {
          s_stop = 1;
          atomicOr(&cnt->status, STAT_CAPACITY);
        }
      }
      __syncthreads();
      if (act && lane == 0 && !s_stop) {
        const int w = base + wl, pk = b_ka[wl] * 4 + b_kb[wl];
        const double alpha[2] = {s_alpha[pk][0], s_alpha[pk][1]};
        const int info = b_ka[wl] | (b_kb[wl] << 2) | (b_app[wl] << 8) | (s_sides[pk] << 4);
        d.pl_e[w] = b_e[wl];
        d.pl_info[w] = info;
        for (int a = 0; a < 4; ++a) {
          d.pl_reuse[w * 4 + a] = b_reuse[wl][a];
          d.pl_tomb[w * 4 + a] = b_tomb[wl][a];
        }
        d.pl_alpha[w * 2] = alpha[0];
        d.pl_alpha[w * 2 + 1] = alpha[1];
        d.pl_c[w] = s_nck + wl;
        d.pl_ph0[w] = g.nn + s_nph + pre_new;
        d.pl_app0[w] = s_nS + pre_app;
        b_alpha[wl][0] = alpha[0];
        b_alpha[wl][1] = alpha[1];
        b_c[wl] = s_nck + wl;
      }
      if (act && lane == 0 && !s_stop) atomicAdd(&s_dead, ndead);
      __syncthreads();
      if (act && lane < 4 && !s_stop) {
        // local node a: masses after the split and the phantom's user list
        const int w = base + wl, e = b_e[wl], a = lane;
        const int sa = b_side[wl][a];
        const double alpha[2] = {b_alpha[wl][0], b_alpha[wl][1]};
        // the real node: rho A_p / 4 of every piece around it that uses it,
        // in increasing element id (the planned piece in place of e)
        double mreal = 0.0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const double Ap = q == np.qe ? alpha[sa] * g.A : np.Ap[q];
          if (np.st[q] != ST_OUT) mreal = mreal + d.mat.rho * Ap * 0.25;
        }
        d.pl_mreal[w * 4 + a] = mreal;
        d.pl_mireal[w * 4 + a] = inverse_mass(mreal);
        // the reused phantom's users (sorted by element) and their areas
        int us[4] = {u4.x, u4.y, u4.z, u4.w}, uf[4] = {f4.x, f4.y, f4.z, f4.w};
        double Au[4] = {A01.x, A01.y, A23.x, A23.y};
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (q >= nu) { us[q] = 0x7fffffff; uf[q] = -1; Au[q] = 0.0; }
        const int p = 1 - sa;  // the piece that uses the phantom of a
        const int code = (e << 3) | (p << 2) | a, cf = b_c[wl] * 16 + p * 8 + 2 * a;
        const double Anew = alpha[p] * g.A;
        // insert the new user in increasing element id (as the split writes
        // did): before the first user of a larger element; a full list of
        // four keeps its first four entries
        int pos = 4;
#pragma unroll
        for (int q = 3; q >= 0; --q)
          if (q >= nu || (us[q] >> 3) > e) pos = q;
        int out[4], outf[4];
        double outA[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          if (t < pos) {
            out[t] = us[t]; outf[t] = uf[t]; outA[t] = Au[t];
          } else if (t == pos) {
            out[t] = code; outf[t] = cf; outA[t] = Anew;
          } else if (t - 1 < nu) {
            out[t] = us[t - 1]; outf[t] = uf[t - 1]; outA[t] = Au[t - 1];
          } else {
            out[t] = -1; outf[t] = -1; outA[t] = 0.0;
          }
        }
        // the phantom's mass: rho A_p / 4 of each user piece, in list order
        double acc = 0.0;
        const int nun = nu < 4 ? nu + 1 : 4;
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (q < nun) acc = acc + d.mat.rho * outA[q] * 0.25;
        d.pl_mph[w * 4 + a] = acc;
        d.pl_miph[w * 4 + a] = inverse_mass(acc);
        d.pl_mold[w * 4 + a] = mold;
        d.pl_dm[w * 4 + a] = d.mat.rho * Anew * 0.25;
        d.pl_nu[w * 4 + a] = nu;  // users before the insertion (4: list full)
        for (int q = 0; q < 4; ++q) {
          d.pl_users[w * 16 + a * 4 + q] = out[q];
          d.pl_upf[w * 16 + a * 4 + q] = outf[q];
          d.pl_uap[w * 16 + a * 4 + q] = outA[q];
        }
      }
      __syncthreads();
      if (tid == 0 && !s_stop) {
        s_nph += tot_new;
        s_nck += nb;
        s_nS += tot_app;
        s_done = base + nb;
      }
      __syncthreads();
    }
  }
  __syncthreads();
  if (tid == 0) {
    cnt->pend_nwin = s_done;
    cnt->pend_nph = s_nph;
    cnt->pend_nck = s_nck;
    cnt->pend_nS = s_nS;
    cnt->pend_dead = s_dead;
    cnt->pend_step = cnt->step;
    cnt->n_prop_last = cnt->n_prop;
    cnt->n_prop = 0;
  }
}

__global__ void __launch_bounds__(TB, 4) k_select(DevState d, int mode) {
  extern __shared__ unsigned long long smem[];
  select_plan(d, mode, smem);
}

// one CTA per member of a batch
__global__ void __launch_bounds__(TB, 4) k_select_batch(BatchDev b) {
  extern __shared__ unsigned long long smem[];
  __shared__ DevState sd;
  int held = -1;
  const int n = *b.bstep;
  for (int s = blockIdx.x; s < b.n; s += gridDim.x) {
    stage_member(b.ds, s, sd, held);
    if (!member_active(sd, n)) continue;
    select_plan(sd, TRACK_STEP, smem);
    __syncthreads();
  }
}

// Split writes: eight threads per planned winner (lanes 0-3: local nodes,
// 4-7: their phantoms / the split record), winners in parallel, in two
// phases.  Phase 1 writes what no kernel of the step reads or writes: the
// split record, the node lists, new phantoms' tables and work accumulators,
// the phantom user lists and the surface list (the piece, phantom,
// evaluation and selection kernels have finished).  Phase 2 writes what the
// node update reads or produces: new phantoms copy u^{n+1} and v^{n+1/2} of
// their real node, shared phantoms take the momentum-conserving merge, the
// masses, the element state and the node update's row flags, and the counter
// commit.  k_apply runs phase 1 before its grid-dependency wait, beside the
// node update's last wave.
__device__ __forceinline__ int apply_phantom(const DevState &d, int w, int a) {
  int P = d.pl_reuse[w * 4 + a];
  if (P < 0) {
    int rank = 0;
    for (int q = 0; q < a; ++q) rank += d.pl_reuse[w * 4 + q] < 0;
    P = d.pl_ph0[w] + rank;
  }
  return P;
}

__device__ __forceinline__ void apply_tables(const DevState &d, VBlk vb, int mode) {
  Counters *cnt = d.cnt;
  const Geo &g = d.g;
  const int nw = cnt->pend_nwin;
  const int step = cnt->pend_step;
  const int lane32 = threadIdx.x & 31, lane = lane32 & 7, grp = lane32 >> 3;
  const int warp = (vb.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (vb.gx * blockDim.x) >> 5;
  for (int wb = warp * 4; wb < nw; wb += nwarps * 4) {
    const int w = wb + grp;
    const bool act = w < nw;
    const int a = lane & 3;
    if (act && lane < 4) {
      // local node a: its phantom (new or shared), node lists, user list
      const int e = d.pl_e[w], info = d.pl_info[w], c = d.pl_c[w];
      const int sd = (info >> (4 + a)) & 1;
      const int N = elem_node(g, e, a);
      const int P = apply_phantom(d, w, a);
      const int t = P - g.nn;
      if (d.pl_reuse[w * 4 + a] < 0) {
        d.ph_owner[t] = N;
        d.ph_creator[t] = e * 4 + a;
        d.Wn[P] = 0.0;
        d.Wd[P] = 0.0;
      }
      d.ck_node[c * 8 + sd * 4 + a] = N;
      d.ck_node[c * 8 + (1 - sd) * 4 + a] = P;
      const int nu = d.pl_nu[w * 4 + a];
      if (nu >= 4) {
        atomicOr(&cnt->status, STAT_CAPACITY);
      } else {
        reinterpret_cast<int4 *>(d.ph_users)[t] = reinterpret_cast<const int4 *>(d.pl_users)[w * 4 + a];
        reinterpret_cast<int4 *>(d.ph_upf)[t] = reinterpret_cast<const int4 *>(d.pl_upf)[w * 4 + a];
        const double2 *ua = reinterpret_cast<const double2 *>(d.pl_uap + w * 16 + a * 4);
        reinterpret_cast<double2 *>(d.ph_uap)[2 * t] = ua[0];
        reinterpret_cast<double2 *>(d.ph_uap)[2 * t + 1] = ua[1];
        d.ph_nuser[t] = nu + 1;
      }
    } else if (act) {
      // lanes 4-7: surface list at local edge k = lane - 4; lane 4 also
      // writes the split record
      const int e = d.pl_e[w], info = d.pl_info[w];
      const int k = lane - 4;
      const int ed = elem_edge(g, e, k);
      const int app = (info >> 8) & 15;
      if ((app >> k) & 1) {
        const int dst = d.pl_app0[w] + __popc(app & ((1 << k) - 1));
        const int f = elem_neighbor(g, e, k);
        d.S[dst] = ed;
        d.S_info[dst] = f * 4 + ((k + 2) & 3);
        d.S_G[dst] = 0.0;
        d.spos[ed] = dst;
      } else {
        const int pos = d.pl_tomb[w * 4 + k];
        if (pos >= 0) {
          d.S[pos] = -1;
          d.spos[ed] = -1;
        }
      }
      if (lane == 4) {
        const int c = d.pl_c[w];
        const int ka = info & 3, kb = (info >> 2) & 3;
        d.ck_elem[c] = e;
        d.ck_info[c] = info & 0xff;
        d.ck_Ap[c * 2] = d.pl_alpha[w * 2] * g.A;
        d.ck_Ap[c * 2 + 1] = d.pl_alpha[w * 2 + 1] * g.A;
        d.ck_step[c] = mode == TRACK_PRECRACK ? -1 : step;
        if (mode == TRACK_PRECRACK) {
          d.ck_ud[c] = 0.0;
        } else {
          const double xa = (xi_g(ka) + 1.0) * (0.5 * g.hx), ya = (eta_g(ka) + 1.0) * (0.5 * g.hy);
          const double xb = (xi_g(kb) + 1.0) * (0.5 * g.hx), yb = (eta_g(kb) + 1.0) * (0.5 * g.hy);
          const double sx = xb - xa, sy = yb - ya;
          const double L = sqrt(sx * sx + sy * sy);
          d.ck_ud[c] = (double)d.gc[e] * L;
        }
        d.crack_of[e] = c;
      }
    }
  }
}

// What the node writes need of winner w's local node a: the real node N,
// its phantom P (new when reuse < 0, else shared), the masses before and
// after the split and the mass moved.
struct SplitNode {
  int N, P, reuse;
  double mold, mnew, mreal, dm, mireal, miph;
};

__device__ __forceinline__ SplitNode split_node(const DevState &d, int w, int a) {
  SplitNode q;
  q.N = elem_node(d.g, d.pl_e[w], a);
  q.P = apply_phantom(d, w, a);
  q.reuse = d.pl_reuse[w * 4 + a];
  q.mold = d.pl_mold[w * 4 + a];
  q.mnew = d.pl_mph[w * 4 + a];
  q.mreal = d.pl_mreal[w * 4 + a];
  q.dm = d.pl_dm[w * 4 + a];
  q.mireal = d.pl_mireal[w * 4 + a];
  q.miph = d.pl_miph[w * 4 + a];
  return q;
}

// local node a: the new phantom's state, or the momentum-conserving merge
// into a shared phantom; the masses after the split
__device__ __forceinline__ void node_apply(const DevState &d, const SplitNode &q, int cur_next) {
  const int N = q.N, P = q.P;
  if (q.reuse < 0) {
    if (d.precision == 1) {
      d.u4[cur_next][P] = d.u4[cur_next][N];
      d.v2[P] = d.v2[N];
    } else {
      d.ux[cur_next][P] = d.ux[cur_next][N]; d.uy[cur_next][P] = d.uy[cur_next][N];
      d.vx[P] = d.vx[N]; d.vy[P] = d.vy[N];
    }
  } else if (q.mold >= 0.0) {
    // merge: the phantom gains mass dm moving with its real node
    if (d.precision == 1) {
      const float2 vp = d.v2[P], vn = d.v2[N];
      const double vx = ((q.mold * (double)vp.x) + q.dm * (double)vn.x) / q.mnew;
      const double vy = ((q.mold * (double)vp.y) + q.dm * (double)vn.y) / q.mnew;
      d.v2[P] = make_float2((float)vx, (float)vy);
    } else {
      d.vx[P] = (q.mold * d.vx[P] + q.dm * d.vx[N]) / q.mnew;
      d.vy[P] = (q.mold * d.vy[P] + q.dm * d.vy[N]) / q.mnew;
    }
  }
  set_mass(d, N, q.mreal, q.mireal);
  set_mass(d, P, q.mnew, q.miph);
}

__device__ __forceinline__ void elem_split(const DevState &d, int e) {
  d.estate[e] = ST_CRACKED;
  march_rows_split(d, e);
}

// the commit changes no value that another block of this kernel reads
__device__ __forceinline__ void apply_commit(const DevState &d, VBlk vb, int mode) {
  Counters *cnt = d.cnt;
  if (vb.x == 0 && threadIdx.x == 0) {
    const int step = cnt->pend_step;
    cnt->n_ph = cnt->pend_nph;
    cnt->n_ck = cnt->pend_nck;
    cnt->n_S = cnt->pend_nS;
    cnt->n_dead += cnt->pend_dead;
    cnt->n_win_last = cnt->pend_nwin;
    if (mode == TRACK_STEP) cnt->step = step + 1;
  }
}

__device__ __forceinline__ void apply_nodes(const DevState &d, VBlk vb, int cur_next, int mode) {
  const int nw = d.cnt->pend_nwin;
  const int lane32 = threadIdx.x & 31, lane = lane32 & 7, grp = lane32 >> 3;
  const int warp = (vb.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (vb.gx * blockDim.x) >> 5;
  for (int wb = warp * 4; wb < nw; wb += nwarps * 4) {
    const int w = wb + grp;
    const bool act = w < nw;
    if (act && lane < 4) node_apply(d, split_node(d, w, lane & 3), cur_next);
    else if (act && lane == 4) elem_split(d, d.pl_e[w]);
  }
  apply_commit(d, vb, mode);
}

__device__ __forceinline__ void apply_plan(const DevState &d, VBlk vb, int cur_next, int mode) {
  apply_tables(d, vb, mode);
  apply_nodes(d, vb, cur_next, mode);
}

// With a status ring, the last block of the split writes to finish copies
// the counters (committed by block 0) into ring[steps taken % kStatusRing].
__device__ __forceinline__ void ring_status(const DevState &d, Counters *ring) {
  __shared__ bool last;
  __syncthreads();  // every write of this block is issued
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&d.cnt->apply_done, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  constexpr int n = (int)(sizeof(Counters) / sizeof(int));
  volatile int *c = reinterpret_cast<volatile int *>(d.cnt);
  if (threadIdx.x == 0) c[offsetof(Counters, apply_done) / sizeof(int)] = 0;
  __syncthreads();
  const int slot = c[offsetof(Counters, step) / sizeof(int)] % kStatusRing;
  if (threadIdx.x < n) reinterpret_cast<volatile int *>(ring + slot)[threadIdx.x] = c[threadIdx.x];
}

// In a step graph, launched as a programmatic dependent of the node update
// (the selection and the phantom update before it have completed): its CTAs
// may be placed while the node update's last wave still runs, write phase 1
// and read their plan, none of which the node update touches, and wait here
// until the node update has completed and its writes are visible.
__global__ void __launch_bounds__(256) k_apply(DevState d, int cur_next, int mode, Counters *ring) {
  const VBlk vb = hw_vblk();
  apply_tables(d, vb, mode);
  // with at most four winners per warp each thread has at most one node
  // write (or the element's): its plan is read before the wait, so that
  // only the node update's own outputs are read after it
  const int nw = d.cnt->pend_nwin;
  const int lane32 = threadIdx.x & 31, lane = lane32 & 7;
  const int w = ((vb.x * blockDim.x + threadIdx.x) >> 5) * 4 + (lane32 >> 3);
  const bool one_pass = nw <= ((vb.gx * blockDim.x) >> 5) * 4;
  SplitNode q;
  int es = -1;
  if (one_pass && w < nw) {
    if (lane < 4) q = split_node(d, w, lane);
    else if (lane == 4) es = d.pl_e[w];
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;");
  if (!one_pass) {
    apply_nodes(d, vb, cur_next, mode);
  } else {
    if (w < nw && lane < 4) node_apply(d, q, cur_next);
    if (es >= 0) elem_split(d, es);
    apply_commit(d, vb, mode);
  }
  if (ring) ring_status(d, ring);
}

// APPLY_VB virtual CTAs per member of a batch; the last CTA to finish
// advances the batch step (every CTA has read it before it arrives).
constexpr int APPLY_VB = 8;

__global__ void __launch_bounds__(256) k_apply_batch(BatchDev b) {
  __shared__ DevState sd;
  int held = -1, w0, w1;
  const int n = *b.bstep;
  block_range(b.n * APPLY_VB, w0, w1);
  for (int w = w0; w < w1; ++w) {
    stage_member(b.ds, w / APPLY_VB, sd, held);
    if (!member_active(sd, n)) continue;
    apply_plan(sd, VBlk{w % APPLY_VB, 0, APPLY_VB, 1}, member_cur(sd, n) ^ 1, TRACK_STEP);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(b.arrive, 1) == (int)gridDim.x - 1) {
      *b.arrive = 0;
      *b.bstep = n + 1;
    }
  }
}

// Builds the surface list from scratch in edge-id order, in two passes over
// fixed contiguous edge ranges (one per block): the live surface points of
// each range are counted, then each block writes its range's points in
// order after the points of the ranges before it.  The selection's winner
// scratch holds the per-range counts (it is idle at set-up).
constexpr int kSurfBlocks = 1216;

__device__ __forceinline__ bool surface_point(const DevState &d, int gid, int &info) {
  int lo, klo, hi, khi;
  edge_sides(d.g, gid, lo, klo, hi, khi);
  const bool ilo = estatus(d, lo) == ST_INTACT, ihi = estatus(d, hi) == ST_INTACT;
  info = ilo ? lo * 4 + klo : hi * 4 + khi;
  return ilo != ihi;
}

__global__ void __launch_bounds__(TB) k_surface_count(DevState d, int chunk) {
  const int e0 = blockIdx.x * chunk, e1 = min(d.g.ned, e0 + chunk);
  int live = 0;
  for (int gid = e0 + threadIdx.x; gid < e1; gid += TB) {
    int info;
    live += surface_point(d, gid, info) ? 1 : 0;
    d.spos[gid] = -1;
  }
  int tot;
  block_exscan(live, &tot);
  if (threadIdx.x == 0) d.sel_win[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(TB) k_surface_write(DevState d, int chunk) {
  __shared__ int s_out;
  if (threadIdx.x == 0) {
    int o = 0;
    for (int q = 0; q < (int)blockIdx.x; ++q) o += d.sel_win[q];
    s_out = o;
  }
  __syncthreads();
  int out = s_out;
  const int e0 = blockIdx.x * chunk, e1 = min(d.g.ned, e0 + chunk);
  for (int base = e0; base < e1; base += TB) {
    const int gid = base + threadIdx.x;
    int info = 0;
    const int live = gid < e1 && surface_point(d, gid, info) ? 1 : 0;
    int tot;
    const int pos = block_exscan(live, &tot);
    if (live) {
      const int dst = out + pos;
      if (dst < d.list_cap) {
        d.S[dst] = gid;
        d.S_info[dst] = info;
        d.S_G[dst] = 0.0;
        d.spos[gid] = dst;
      }
    }
    out += tot;
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
    if (out > d.list_cap) {
      atomicOr(&d.cnt->status, STAT_CAPACITY);
      out = d.list_cap;
    }
    d.cnt->n_S = out;
    d.cnt->n_dead = 0;
  }
}

__global__ void k_surface_info(DevState d, int *out3) {
  int n = d.cnt->n_S;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int ed = d.S[i];
    int inf = d.S_info[i];
    out3[3 * i] = ed;
    out3[3 * i + 1] = ed >= 0 ? inf : -1;
    out3[3 * i + 2] = ed >= 0 ? (tip_of(d, inf >> 2, inf & 3) ? 1 : 0) : 0;
  }
}

// The status word of a pipelined step call, copied by a kernel into mapped
// pinned host memory: no copy-engine operation between the calls' graphs.
__global__ void k_status_copy(const Counters *cnt, Counters *out) {
  constexpr int n = (int)(sizeof(Counters) / sizeof(int));
  const int i = threadIdx.x;
  if (i < n) reinterpret_cast<volatile int *>(out)[i] = reinterpret_cast<const int *>(cnt)[i];
}

}  // namespace

cudaError_t launch_select(const DevState &d, int mode, cudaStream_t st) {
  size_t sm = select_smem_bytes();
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_select, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e == cudaSuccess) e = match_tile_carveout(k_select);
    if (e == cudaSuccess) e = match_tile_carveout(k_apply);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_select<<<1, TB, sm, st>>>(d, mode);
  return cudaGetLastError();
}

cudaError_t launch_apply(const DevState &d, int cur_next, int mode, cudaStream_t st,
                         bool programmatic, Counters *ring) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(64);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = programmatic ? 1 : 0;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_apply, d, cur_next, mode, ring);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_status_copy(const Counters *cnt, Counters *host_mapped, cudaStream_t st) {
  k_status_copy<<<1, 32, 0, st>>>(cnt, host_mapped);
  return cudaGetLastError();
}

cudaError_t launch_build_surface(const DevState &d, cudaStream_t st) {
  const int chunk = (d.g.ned + kSurfBlocks - 1) / kSurfBlocks;
  const int blocks = (d.g.ned + chunk - 1) / chunk;
  k_surface_count<<<blocks, TB, 0, st>>>(d, chunk);
  k_surface_write<<<blocks, TB, 0, st>>>(d, chunk);
  return cudaGetLastError();
}

cudaError_t launch_surface_info(const DevState &d, int *out3, cudaStream_t st) {
  k_surface_info<<<256, 256, 0, st>>>(d, out3);
  return cudaGetLastError();
}

cudaError_t launch_select_batch(const BatchDev &b, cudaStream_t st) {
  size_t sm = select_smem_bytes();
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_select_batch,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess) e = match_tile_carveout(k_select_batch);
    if (e == cudaSuccess) e = match_tile_carveout(k_apply_batch);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_select_batch<<<b.n < 304 ? b.n : 304, TB, sm, st>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_apply_batch(const BatchDev &b, cudaStream_t st) {
  const int nb = b.n * APPLY_VB;
  k_apply_batch<<<nb < 2432 ? nb : 2432, 256, 0, st>>>(b);
  return cudaGetLastError();
}

int track_sort_capacity() { return SORT_CAP; }

const void *apply_kernel() { return reinterpret_cast<const void *>(&k_apply); }
const void *select_kernel() { return reinterpret_cast<const void *>(&k_select); }

}  // namespace cem
