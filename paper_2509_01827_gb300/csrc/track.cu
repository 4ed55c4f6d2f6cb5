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

struct SplitPlan {
  int e, ka, kb;
  int side[4];
  int n4[4];
  int reuse[4];  // phantom reused for local node a, or -1
  double alpha[2];
};

__device__ void plan_split(const DevState &d, int e, int ka, int kb, SplitPlan &sp) {
  const Geo &g = d.g;
  sp.e = e; sp.ka = ka; sp.kb = kb;
  double pax = xi_g(ka), pay = eta_g(ka), pbx = xi_g(kb), pby = eta_g(kb);
  for (int a = 0; a < 4; ++a) {
    double cross = (pbx - pax) * (eta_n(a) - pay) - (pby - pay) * (xi_n(a) - pax);
    sp.side[a] = cross > 0.0 ? 0 : 1;
    sp.n4[a] = elem_node(g, e, a);
  }
  // shoelace area fractions in natural coordinates (reference square area 4)
  for (int p = 0; p < 2; ++p) {
    double px[6], py[6];
    int nv = 0;
    for (int w = 0; w < 8; ++w) {
      if ((w & 1) == 0) {
        int a = w >> 1;
        if (sp.side[a] == p) { px[nv] = xi_n(a); py[nv] = eta_n(a); ++nv; }
      } else {
        int k = w >> 1;
        if (k == ka || k == kb) { px[nv] = xi_g(k); py[nv] = eta_g(k); ++nv; }
      }
    }
    double twice = 0.0;
    for (int v = 0; v < nv; ++v) {
      int w = (v + 1) % nv;
      twice = twice + (px[v] * py[w] - px[w] * py[v]);
    }
    sp.alpha[p] = fabs(twice) * 0.5 / 4.0;
  }
  // phantoms to reuse from a cracked neighbour across a shared cut edge
  for (int a = 0; a < 4; ++a) {
    sp.reuse[a] = -1;
    int k1 = (a + 3) & 3, k2 = a;
    int kk[2] = {k1 < k2 ? k1 : k2, k1 < k2 ? k2 : k1};
    for (int q = 0; q < 2 && sp.reuse[a] < 0; ++q) {
      int k = kk[q];
      if (k != ka && k != kb) continue;
      int f = elem_neighbor(g, e, k);
      if (estatus(d, f) != ST_CRACKED) continue;
      int cf = d.crack_of[f];
      int inf = d.ck_info[cf];
      int kf = (k + 2) & 3;
      if ((inf & 3) != kf && ((inf >> 2) & 3) != kf) continue;
      int af = -1;
      for (int b = 0; b < 4; ++b)
        if (elem_node(g, f, b) == sp.n4[a]) af = b;
      int sf = (inf >> (4 + af)) & 1;
      sp.reuse[a] = d.ck_node[cf * 8 + (1 - sf) * 4 + af];
    }
  }
}

__device__ int count_new(const SplitPlan &sp) {
  int c = 0;
  for (int a = 0; a < 4; ++a) c += sp.reuse[a] < 0;
  return c;
}

// Writes the split of one winner (crack slot c, first new phantom id ph0).
__device__ bool apply_split(const DevState &d, const SplitPlan &sp, int c, int ph0, int cur_next,
                            int step, bool precrack) {
  const Geo &g = d.g;
  const int e = sp.e;
  int node[2][4];
  double mold[4];
  int nextp = ph0;
  for (int a = 0; a < 4; ++a) {
    node[sp.side[a]][a] = sp.n4[a];
    int p = 1 - sp.side[a];
    int P = sp.reuse[a];
    if (P < 0) {
      P = nextp++;
      int t = P - g.nn, N = sp.n4[a];
      d.ph_owner[t] = N;
      d.ph_creator[t] = e * 4 + a;
      d.ph_nuser[t] = 0;
      d.Wn[P] = 0.0;
      d.Wd[P] = 0.0;
      if (d.precision == 1) {
        d.uxh[cur_next][P] = d.uxh[cur_next][N]; d.uxl[cur_next][P] = d.uxl[cur_next][N];
        d.uyh[cur_next][P] = d.uyh[cur_next][N]; d.uyl[cur_next][P] = d.uyl[cur_next][N];
        d.vxf[P] = d.vxf[N]; d.vyf[P] = d.vyf[N];
      } else {
        d.ux[cur_next][P] = d.ux[cur_next][N]; d.uy[cur_next][P] = d.uy[cur_next][N];
        d.vx[P] = d.vx[N]; d.vy[P] = d.vy[N];
      }
      mold[a] = -1.0;
    } else {
      mold[a] = d.m[P];
    }
    node[p][a] = P;
  }
  int info = sp.ka | (sp.kb << 2);
  for (int a = 0; a < 4; ++a) info |= sp.side[a] << (4 + a);
  d.ck_elem[c] = e;
  d.ck_info[c] = info;
  for (int p = 0; p < 2; ++p)
    for (int a = 0; a < 4; ++a) d.ck_node[c * 8 + p * 4 + a] = node[p][a];
  d.ck_Ap[c * 2] = sp.alpha[0] * g.A;
  d.ck_Ap[c * 2 + 1] = sp.alpha[1] * g.A;
  d.ck_step[c] = precrack ? -1 : step;
  if (precrack) {
    d.ck_ud[c] = 0.0;
  } else {
    double xa = (xi_g(sp.ka) + 1.0) * (0.5 * g.hx), ya = (eta_g(sp.ka) + 1.0) * (0.5 * g.hy);
    double xb = (xi_g(sp.kb) + 1.0) * (0.5 * g.hx), yb = (eta_g(sp.kb) + 1.0) * (0.5 * g.hy);
    double sx = xb - xa, sy = yb - ya;
    double L = sqrt(sx * sx + sy * sy);
    d.ck_ud[c] = (double)d.gc[e] * L;
  }
  d.crack_of[e] = c;
  d.estate[e] = ST_CRACKED;
  // users of the phantoms, kept sorted by element id
  bool ok = true;
  for (int a = 0; a < 4; ++a) {
    int p = 1 - sp.side[a];
    int t = node[p][a] - g.nn;
    int nu = d.ph_nuser[t];
    if (nu >= 4) { ok = false; continue; }
    int q = nu;
    int code = (e << 3) | (p << 2) | a;
    while (q > 0 && (d.ph_users[t * 4 + q - 1] >> 3) > e) {
      d.ph_users[t * 4 + q] = d.ph_users[t * 4 + q - 1];
      --q;
    }
    d.ph_users[t * 4 + q] = code;
    d.ph_nuser[t] = nu + 1;
  }
  // masses touched by the split
  for (int a = 0; a < 4; ++a) set_mass(d, sp.n4[a], mass_real(d, sp.n4[a]));
  for (int a = 0; a < 4; ++a) {
    int p = 1 - sp.side[a];
    int P = node[p][a];
    double mnew = mass_phantom(d, P);
    if (mold[a] >= 0.0) {
      // momentum-conserving merge of the mass moved from the real node
      double dm = d.mat.rho * (sp.alpha[p] * g.A) * 0.25;
      int N = sp.n4[a];
      if (d.precision == 1) {
        double vx = ((mold[a] * (double)d.vxf[P]) + dm * (double)d.vxf[N]) / mnew;
        double vy = ((mold[a] * (double)d.vyf[P]) + dm * (double)d.vyf[N]) / mnew;
        d.vxf[P] = (float)vx;
        d.vyf[P] = (float)vy;
      } else {
        d.vx[P] = (mold[a] * d.vx[P] + dm * d.vx[N]) / mnew;
        d.vy[P] = (mold[a] * d.vy[P] + dm * d.vy[N]) / mnew;
      }
    }
    set_mass(d, P, mnew);
  }
  return ok;
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

    // ---- split winners in increasing element id, 1024 at a time
    for (int base = 0; base < nwin; base += TB) {
      int w = base + tid;
      bool act = w < nwin && !s_stop;
      SplitPlan sp;
      int nnew = 0;
      if (act) {
        int i = swin[w];
        int idx = (int)(sk[i] & 0xffffffffu);
        int key = (int)(sk[i] >> 32);
        plan_split(d, key >> 2, key & 3, d.pr_k[idx], sp);
        nnew = count_new(sp);
      }
      int tot_new;
      int pre_new = block_exscan(act ? nnew : 0, &tot_new);
      int nact = nwin - base < TB ? nwin - base : TB;
      bool fits = !s_stop && s_nph + tot_new <= d.ph_cap && s_nck + nact <= d.ck_cap;
      bool ok = true;
      if (act && fits)
        ok = apply_split(d, sp, s_nck + (w - base), g.nn + s_nph + pre_new, cur_next, step,
                         mode == TRACK_PRECRACK);
      if (act && !ok) atomicOr(&cnt->status, STAT_CAPACITY);
      // surface list: appends and tombstones
      int napp = 0;
      int app_edge[4], app_info[4];
      if (act && fits) {
        for (int k = 0; k < 4; ++k) {
          int ed = elem_edge(g, sp.e, k);
          int f = elem_neighbor(g, sp.e, k);
          if (estatus(d, f) == ST_INTACT) {
            app_edge[napp] = ed;
            app_info[napp] = f * 4 + ((k + 2) & 3);
            ++napp;
          } else {
            int pos = d.spos[ed];
            if (pos >= 0) {
              d.S[pos] = -1;
              d.spos[ed] = -1;
              atomicAdd(&s_dead, 1);
            }
          }
        }
      }
      int tot_app;
      int pre_app = block_exscan(napp, &tot_app);
      bool lfits = s_nS + tot_app <= d.list_cap;
      if (act && fits && lfits) {
        for (int q = 0; q < napp; ++q) {
          int dst = s_nS + pre_app + q;
          d.S[dst] = app_edge[q];
          d.S_info[dst] = app_info[q];
          d.S_G[dst] = 0.0;
          d.spos[app_edge[q]] = dst;
        }
      }
      __syncthreads();
      if (tid == 0) {
        if (!fits || !lfits) {
          s_stop = 1;
          atomicOr(&cnt->status, STAT_CAPACITY);
        } else {
          s_nph += tot_new;
          s_nck += nact;
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
