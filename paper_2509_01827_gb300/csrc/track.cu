// track.cu -- multi-tip crack tracking: selection, split and surface list
// (compiled with -fmad=false: the split's masses, momentum merge and
// dissipated energy follow the FP64 expression order of the definition).
//
// k_track runs as ONE cooperative CTA per step.  It
//   1. sorts the step's proposals by (ahead element, local edge) with a
//      bitonic sort in shared memory (the warp-ballot append of k_eval is
//      unordered; the sort makes everything after it deterministic);
//   2. selects winners (Sec. 3): a proposal wins if its key (G, -edge id)
//      is the strict maximum among proposals whose ahead elements share a
//      node with its own (binary searches over the three neighbouring rows),
//      or the single global maximum, or -- pre-cracks -- unconditionally;
//   3. splits each winner (in increasing element id) along the segment
//      between the midpoints of its entry and exit edges into two
//      phantom-node pieces (crack patterns I and II, Fig. 2-3), sharing a
//      phantom with the cracked neighbour across a cut edge, recomputes the
//      lumped masses it touches, merges momentum into shared phantoms and
//      records U_d = G_c * segment length;
//   4. updates the device-side surface list: tombstones edges that lost their
//      intact element, appends edges that gained one, and compacts the list
//      with warp ballots when half of it is dead.
#include <cuda_runtime.h>
#include <stdint.h>

#include "cem_internal.h"
#include "q4_fp64.cuh"

namespace cem {

namespace {

constexpr int TB = 1024;           // threads of the tracking CTA
constexpr int SORT_CAP = 8192;     // proposals per step (power of two)
constexpr int WB = TB / 8;         // winners split per batch (eight threads each)

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

__device__ double mass_real(const DevState &d, int N) {
  const Geo &g = d.g;
  int r = g.nx + 1, i = N % r, j = N / r;
  const int di[4] = {-1, 0, -1, 0}, dj[4] = {-1, -1, 0, 0}, la[4] = {2, 3, 1, 0};
  double acc = 0.0;
  for (int q = 0; q < 4; ++q) {
    int ei = i + di[q], ej = j + dj[q];
    if (ei < 0 || ej < 0 || ei >= g.nx || ej >= g.ny) continue;
    int e = ej * g.nx + ei, st = d.estate[e];
    if (st == ST_INTACT) {
      acc = acc + d.mat.rho * g.A * 0.25;
    } else if (st == ST_CRACKED) {
      int c = d.crack_of[e];
      int side = (d.ck_info[c] >> (4 + la[q])) & 1;
      acc = acc + d.mat.rho * d.ck_Ap[c * 2 + side] * 0.25;
    }
  }
  return acc;
}

__device__ double mass_phantom(const DevState &d, int P) {
  int t = P - d.g.nn;
  double acc = 0.0;
  for (int q = 0; q < d.ph_nuser[t]; ++q) {
    int u = d.ph_users[t * 4 + q];
    int c = d.crack_of[u >> 3];
    acc = acc + d.mat.rho * d.ck_Ap[c * 2 + ((u >> 2) & 1)] * 0.25;
  }
  return acc;
}

__device__ void set_mass(const DevState &d, int N, double m) {
  d.m[N] = m;
  double mi = m > 0.0 ? 1.0 / m : 0.0;
  d.minv[N] = mi;
  if (d.precision == 1) d.minvf[N] = (float)mi;
}

// Phantom of local node a of element e that the split (entry ka, exit kb)
// reuses: the one held by the cracked neighbour across a cut edge of e that
// contains the node, if that edge is cut in the neighbour too (first such
// edge in increasing local edge index); -1 when a new phantom is needed.
__device__ int reuse_lookup(const DevState &d, int e, int ka, int kb, int a) {
  const Geo &g = d.g;
  const int k1 = (a + 3) & 3, k2 = a;
  const int kk[2] = {k1 < k2 ? k1 : k2, k1 < k2 ? k2 : k1};
  const int N = elem_node(g, e, a);
  for (int q = 0; q < 2; ++q) {
    const int k = kk[q];
    if (k != ka && k != kb) continue;
    const int f = elem_neighbor(g, e, k);
    if (estatus(d, f) != ST_CRACKED) continue;
    const int cf = d.crack_of[f];
    const int inf = d.ck_info[cf];
    const int kf = (k + 2) & 3;
    if ((inf & 3) != kf && ((inf >> 2) & 3) != kf) continue;
    int af = -1;
    for (int b = 0; b < 4; ++b)
      if (elem_node(g, f, b) == N) af = b;
    const int sf = (inf >> (4 + af)) & 1;
    return d.ck_node[cf * 8 + (1 - sf) * 4 + af];
  }
  return -1;
}

// Area fractions of the two pieces by the shoelace formula in natural
// coordinates (the reference square has area 4).
__device__ void area_fractions(int ka, int kb, const int side[4], double alpha[2]) {
  for (int p = 0; p < 2; ++p) {
    double px[6], py[6];
    int nv = 0;
    for (int w = 0; w < 8; ++w) {
      if ((w & 1) == 0) {
        const int a = w >> 1;
        if (side[a] == p) { px[nv] = xi_n(a); py[nv] = eta_n(a); ++nv; }
      } else {
        const int k = w >> 1;
        if (k == ka || k == kb) { px[nv] = xi_g(k); py[nv] = eta_g(k); ++nv; }
      }
    }
    double twice = 0.0;
    for (int v = 0; v < nv; ++v) {
      const int w = (v + 1) % nv;
      twice = twice + (px[v] * py[w] - px[w] * py[v]);
    }
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

__global__ void __launch_bounds__(TB) k_track(DevState d, int cur_next, int mode) {
  extern __shared__ unsigned long long smem[];
  unsigned long long *sk = smem;                    // [SORT_CAP]
  int *swin = (int *)(smem + SORT_CAP);             // [SORT_CAP]
  __shared__ int s_n, s_nwin, s_stop, s_nph, s_nck, s_nS, s_dead;
  Counters *cnt = d.cnt;
  const Geo &g = d.g;
  const int tid = threadIdx.x;
  if (tid == 0) {
    int n = cnt->n_prop;
    if (n > d.prop_cap) n = d.prop_cap;
    s_n = n;
    s_nwin = 0;
    s_stop = 0;
    s_nph = cnt->n_ph;
    s_nck = cnt->n_ck;
    s_nS = cnt->n_S;
    s_dead = 0;
  }
  __syncthreads();
  const int n = s_n;
  if (n > 0) {
    // ---- load keys; debug proposals that are not surface points (or not
    //      tips under the tips-only scope) sort to the end
    int P2 = 1;
    while (P2 < n) P2 <<= 1;
    for (int i = tid; i < P2; i += TB) {
      unsigned long long v = ~0ull;
      if (i < n) {
        int key = d.pr_key[i];
        bool valid = true;
        if (mode == TRACK_DEBUG) {
          int ed = d.pr_edge[i];
          int pos = d.spos[ed];
          valid = pos >= 0 && d.S_info[pos] == key && d.pr_k[i] != (key & 3);
          if (!valid) atomicOr(&cnt->pad[0], 1);
          if (valid && d.mat.scope == 2) valid = tip_of(d, key >> 2, key & 3);
        }
        if (valid) v = ((unsigned long long)(unsigned)key << 32) | (unsigned)i;
      }
      sk[i] = v;
    }
    __syncthreads();
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
    // number of valid sorted entries
    __shared__ int s_valid;
    if (tid == 0) s_valid = 0;
    __syncthreads();
    for (int i = tid; i < n; i += TB)
      if (sk[i] != ~0ull && (i + 1 == n || sk[i + 1] == ~0ull)) s_valid = i + 1;
    __syncthreads();
    const int nv = s_valid;

    // ---- winners
    if (mode != TRACK_PRECRACK && d.mat.scope == 1) {
      // global: the single largest (G, -edge)
      if (tid == 0) {
        int best = -1;
        for (int i = 0; i < nv; ++i) {
          int idx = (int)(sk[i] & 0xffffffffu);
          if (best < 0 || key_greater(d.pr_G[idx], d.pr_edge[idx], d.pr_G[best], d.pr_edge[best]))
            best = idx;
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
            double G = d.pr_G[idx];
            int ed = d.pr_edge[idx];
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
                if (!key_greater(G, ed, d.pr_G[qi], d.pr_edge[qi])) { win = 0; break; }
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
    const int step = cnt->step;

    // ---- split winners in increasing element id, WB at a time with eight
    //      threads per winner (lanes 0-3: local nodes, 4-7: their phantoms),
    //      so that each phase's chain of dependent loads stays short
    __shared__ int b_e[WB], b_ka[WB], b_kb[WB], b_side[WB][4], b_n4[WB][4], b_reuse[WB][4];
    __shared__ int b_node[WB][2][4], b_c[WB], b_ph0[WB];
    __shared__ double b_alpha[WB][2], b_mold[WB][4];
    __shared__ int s_fits;
    const int lane = tid & 7, wl = tid >> 3;  // winner slot in the batch
    for (int base = 0; base < nwin; base += WB) {
      const int nb = nwin - base < WB ? nwin - base : WB;
      const bool act = wl < nb && !s_stop;
      // phase 1: plan
      if (act && lane == 0) {
        const int i = swin[base + wl];
        const int idx = (int)(sk[i] & 0xffffffffu);
        const int key = (int)(sk[i] >> 32);
        b_e[wl] = key >> 2;
        b_ka[wl] = key & 3;
        b_kb[wl] = d.pr_k[idx];
      }
      __syncthreads();
      if (act && lane < 4) {
        const int e = b_e[wl], ka = b_ka[wl], kb = b_kb[wl], a = lane;
        const double pax = xi_g(ka), pay = eta_g(ka), pbx = xi_g(kb), pby = eta_g(kb);
        const double cross = (pbx - pax) * (eta_n(a) - pay) - (pby - pay) * (xi_n(a) - pax);
        b_side[wl][a] = cross > 0.0 ? 0 : 1;
        b_n4[wl][a] = elem_node(g, e, a);
        b_reuse[wl][a] = reuse_lookup(d, e, ka, kb, a);
      }
      __syncthreads();
      if (act && lane == 4) {
        int side[4];
        for (int a = 0; a < 4; ++a) side[a] = b_side[wl][a];
        area_fractions(b_ka[wl], b_kb[wl], side, b_alpha[wl]);
      }
      // phase 2: crack slots and phantom ids in winner order
      int nnew = 0;
      if (act && lane == 0)
        for (int a = 0; a < 4; ++a) nnew += b_reuse[wl][a] < 0;
      int tot_new;
      const int pre_new = block_exscan(nnew, &tot_new);
      if (tid == 0)
        s_fits = !s_stop && s_nph + tot_new <= d.ph_cap && s_nck + nb <= d.ck_cap;
      if (act && lane == 0) {
        b_c[wl] = s_nck + wl;
        b_ph0[wl] = g.nn + s_nph + pre_new;
      }
      __syncthreads();
      const bool go = act && s_fits;
      // phase 3: phantoms (new ones copy the real node's state) and the record
      if (go && lane < 4) {
        const int a = lane, sd = b_side[wl][a], N = b_n4[wl][a];
        b_node[wl][sd][a] = N;
        int P = b_reuse[wl][a];
        if (P < 0) {
          int rank = 0;
          for (int q = 0; q < a; ++q) rank += b_reuse[wl][q] < 0;
          P = b_ph0[wl] + rank;
          const int t = P - g.nn;
          d.ph_owner[t] = N;
          d.ph_creator[t] = b_e[wl] * 4 + a;
          d.ph_nuser[t] = 0;
          d.Wn[P] = 0.0;
          d.Wd[P] = 0.0;
          if (d.precision == 1) {
            d.u4[cur_next][P] = d.u4[cur_next][N];
            d.v2[P] = d.v2[N];
          } else {
            d.ux[cur_next][P] = d.ux[cur_next][N]; d.uy[cur_next][P] = d.uy[cur_next][N];
            d.vx[P] = d.vx[N]; d.vy[P] = d.vy[N];
          }
          b_mold[wl][a] = -1.0;
        } else {
          b_mold[wl][a] = d.m[P];
        }
        b_node[wl][1 - sd][a] = P;
      }
      if (go && lane == 4) {
        const int e = b_e[wl], c = b_c[wl], ka = b_ka[wl], kb = b_kb[wl];
        int info = ka | (kb << 2);
        for (int a = 0; a < 4; ++a) info |= b_side[wl][a] << (4 + a);
        d.ck_elem[c] = e;
        d.ck_info[c] = info;
        d.ck_Ap[c * 2] = b_alpha[wl][0] * g.A;
        d.ck_Ap[c * 2 + 1] = b_alpha[wl][1] * g.A;
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
        d.estate[e] = ST_CRACKED;
      }
      __syncthreads();
      // phase 4: node lists of the pieces and the phantoms' users
      if (go && lane < 4) {
        const int a = lane, c = b_c[wl], e = b_e[wl];
        d.ck_node[c * 8 + a] = b_node[wl][0][a];
        d.ck_node[c * 8 + 4 + a] = b_node[wl][1][a];
        const int p = 1 - b_side[wl][a];
        const int t = b_node[wl][p][a] - g.nn;
        const int nu = d.ph_nuser[t];
        if (nu >= 4) {
          atomicOr(&cnt->status, STAT_CAPACITY);
        } else {
          int q = nu;
          while (q > 0 && (d.ph_users[t * 4 + q - 1] >> 3) > e) {
            d.ph_users[t * 4 + q] = d.ph_users[t * 4 + q - 1];
            --q;
          }
          d.ph_users[t * 4 + q] = (e << 3) | (p << 2) | a;
          d.ph_nuser[t] = nu + 1;
        }
      }
      __syncthreads();
      // phase 5: masses of the four real nodes (lanes 0-3) and of their
      // phantoms (lanes 4-7, momentum-conserving merge into shared ones)
      if (go && lane < 4) {
        const int N = b_n4[wl][lane];
        set_mass(d, N, mass_real(d, N));
      } else if (go) {
        const int a = lane - 4, p = 1 - b_side[wl][a];
        const int P = b_node[wl][p][a];
        const double mnew = mass_phantom(d, P);
        const double mold = b_mold[wl][a];
        if (mold >= 0.0) {
          const double dm = d.mat.rho * (b_alpha[wl][p] * g.A) * 0.25;
          const int N = b_n4[wl][a];
          if (d.precision == 1) {
            const float2 vp = d.v2[P], vn = d.v2[N];
            const double vx = ((mold * (double)vp.x) + dm * (double)vn.x) / mnew;
            const double vy = ((mold * (double)vp.y) + dm * (double)vn.y) / mnew;
            d.v2[P] = make_float2((float)vx, (float)vy);
          } else {
            d.vx[P] = (mold * d.vx[P] + dm * d.vx[N]) / mnew;
            d.vy[P] = (mold * d.vy[P] + dm * d.vy[N]) / mnew;
          }
        }
        set_mass(d, P, mnew);
      }
      // phase 6: surface list -- lanes 0-3 look at edge k = lane
      int app = 0, app_edge = 0, app_info = 0;
      if (go && lane < 4) {
        const int e = b_e[wl], k = lane;
        const int ed = elem_edge(g, e, k);
        const int f = elem_neighbor(g, e, k);
        if (estatus(d, f) == ST_INTACT) {
          app = 1;
          app_edge = ed;
          app_info = f * 4 + ((k + 2) & 3);
        } else {
          const int pos = d.spos[ed];
          if (pos >= 0) {
            d.S[pos] = -1;
            d.spos[ed] = -1;
            atomicAdd(&s_dead, 1);
          }
        }
      }
      int tot_app;
      const int pre_app = block_exscan(app, &tot_app);
      const bool lfits = s_nS + tot_app <= d.list_cap;
      if (app && lfits) {
        const int dst = s_nS + pre_app;
        d.S[dst] = app_edge;
        d.S_info[dst] = app_info;
        d.S_G[dst] = 0.0;
        d.spos[app_edge] = dst;
      }
      __syncthreads();
      if (tid == 0) {
        if (!s_fits || !lfits) {
          s_stop = 1;
          atomicOr(&cnt->status, STAT_CAPACITY);
        } else {
          s_nph += tot_new;
          s_nck += nb;
          s_nS += tot_app;
        }
      }
      __syncthreads();
    }
    if (tid == 0) {
      cnt->n_ph = s_nph;
      cnt->n_ck = s_nck;
      cnt->n_S = s_nS;
      cnt->n_dead += s_dead;
      cnt->n_win_last = nwin;
    }
    __syncthreads();
    if (cnt->n_dead > 1024 && 2 * cnt->n_dead > cnt->n_S) {
      __syncthreads();
      compact_surface(d);
    }
  } else if (tid == 0) {
    cnt->n_win_last = 0;
  }
  __syncthreads();
  if (tid == 0) {
    cnt->n_prop_last = cnt->n_prop;
    cnt->n_prop = 0;
    if (mode == TRACK_STEP) cnt->step = cnt->step + 1;
  }
}

// Builds the surface list from scratch in edge-id order (one CTA).
__global__ void __launch_bounds__(TB) k_build_surface(DevState d) {
  const Geo &g = d.g;
  int out = 0;
  for (int base = 0; base < g.ned; base += TB) {
    int gid = base + threadIdx.x;
    int live = 0, info = 0;
    if (gid < g.ned) {
      int lo, klo, hi, khi;
      edge_sides(g, gid, lo, klo, hi, khi);
      bool ilo = estatus(d, lo) == ST_INTACT, ihi = estatus(d, hi) == ST_INTACT;
      if (ilo != ihi) {
        live = 1;
        info = ilo ? lo * 4 + klo : hi * 4 + khi;
      }
      d.spos[gid] = -1;
    }
    int tot;
    int pos = block_exscan(live, &tot);
    if (live) {
      int dst = out + pos;
      if (dst < d.list_cap) {
        d.S[dst] = gid;
        d.S_info[dst] = info;
        d.S_G[dst] = 0.0;
        d.spos[gid] = dst;
      }
    }
    out += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
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

}  // namespace

cudaError_t launch_track(const DevState &d, int cur_next, int mode, cudaStream_t st) {
  size_t sm = SORT_CAP * sizeof(unsigned long long) + SORT_CAP * sizeof(int);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_track, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_track<<<1, TB, sm, st>>>(d, cur_next, mode);
  return cudaGetLastError();
}

cudaError_t launch_build_surface(const DevState &d, cudaStream_t st) {
  k_build_surface<<<1, TB, 0, st>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_surface_info(const DevState &d, int *out3, cudaStream_t st) {
  k_surface_info<<<256, 256, 0, st>>>(d, out3);
  return cudaGetLastError();
}

int track_sort_capacity() { return SORT_CAP; }

}  // namespace cem
