// fragments.cu -- fragments of the cracked body (Sec. 4.4 counts them for
// the pressurised cylinder, Table 1).
//
// A piece is an intact active element (its four real nodes) or one side of a
// split element (its node list: the real nodes on that side and phantom
// copies of the others).  Pieces that share a node, real or phantom, share its
// degrees of freedom and move together; a fragment is a connected set of
// pieces under that relation.  The nodes are joined by a lock-free
// union-find (each piece links its nodes; links go from the larger root to
// the smaller, by compare-and-swap on the root), then every node is pointed
// at its root and every piece takes its first node's root.  Fragments are numbered in increasing order of their
// lowest piece index 2 e + p, so the labels do not depend on the order in
// which the threads linked.
#include <cuda_runtime.h>

#include <climits>

#include "cem_internal.h"

namespace cem {

namespace {

// Reads go to L2 (ld.global.cg), where the links are made: an SM's L1 could
// still hold a link target as a root after another SM linked it.  While
// links are being made the walk only reads; once they are all made, a second
// pass compresses every path (uf_flatten_find).
__device__ __forceinline__ int uf_root(const int *parent, int x) {
  int p = __ldcg(parent + x);
  while (p != x) {
    x = p;
    p = __ldcg(parent + x);
  }
  return x;
}

__device__ __forceinline__ void uf_unite(int *parent, int a, int b) {
  for (;;) {
    a = uf_root(parent, a);
    b = uf_root(parent, b);
    if (a == b) return;
    if (a > b) {
      const int t = a;
      a = b;
      b = t;
    }
    // link the larger root under the smaller, unless another thread linked
    // it meanwhile (then retry from what it points to now)
    const int old = atomicCAS(&parent[b], b, a);
    if (old == b) return;
    b = old;
  }
}

// the node list of piece q = 2 e + p (false: no such piece)
__device__ __forceinline__ bool piece_nodes(const DevState &d, int q, int n[4]) {
  const int e = q >> 1, p = q & 1;
  const int st = d.estate[e];
  if (st == ST_INTACT) {
    if (p) return false;
    const int i = e % d.g.nx, j = e / d.g.nx, r = d.g.nx + 1;
    n[0] = j * r + i;
    n[1] = j * r + i + 1;
    n[2] = (j + 1) * r + i + 1;
    n[3] = (j + 1) * r + i;
    return true;
  }
  if (st != ST_CRACKED) return false;
  const int4 v = reinterpret_cast<const int4 *>(d.ck_node)[d.crack_of[e] * 2 + p];
  n[0] = v.x;
  n[1] = v.y;
  n[2] = v.z;
  n[3] = v.w;
  return true;
}

__global__ void k_frag_init(int *parent, int *minp, int n) {
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
    parent[x] = x;
    minp[x] = INT_MAX;
  }
}

__global__ void k_frag_link(DevState d, int *parent, int nq) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
    int n[4];
    if (!piece_nodes(d, q, n)) continue;
    uf_unite(parent, n[0], n[1]);
    uf_unite(parent, n[0], n[2]);
    uf_unite(parent, n[0], n[3]);
  }
}

// every node points at its root (no links are made any more)
__global__ void k_frag_flatten(int *parent, int n) {
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x)
    parent[x] = uf_root(parent, x);
}

__global__ void k_frag_minpiece(DevState d, const int *parent, int *minp, int nq) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
    int n[4];
    if (piece_nodes(d, q, n)) atomicMin(&minp[__ldcg(parent + n[0])], q);
  }
}

// rep[q] = 1 where piece q is the lowest piece of its fragment
__global__ void k_frag_rep(DevState d, const int *parent, const int *minp, int *rep, int nq) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
    int n[4];
    rep[q] = piece_nodes(d, q, n) && minp[parent[n[0]]] == q ? 1 : 0;
  }
}

// exclusive scan of rep in blocks of 2 x 1024 entries; block totals to tot
constexpr int SB = 1024;
__global__ void k_scan_blocks(int *a, int n, int *tot) {
  __shared__ int s[2 * SB];
  const int base = blockIdx.x * 2 * SB, t = threadIdx.x;
  s[t] = base + t < n ? a[base + t] : 0;
  s[t + SB] = base + t + SB < n ? a[base + t + SB] : 0;
  // up-sweep
  for (int d = 1, off = 1; d <= SB; d <<= 1, off <<= 1) {
    __syncthreads();
    const int i = (2 * t + 2) * off - 1;
    if (t < SB / d) s[i] += s[i - off];
  }
  __syncthreads();
  if (t == 0) {
    tot[blockIdx.x] = s[2 * SB - 1];
    s[2 * SB - 1] = 0;
  }
  // down-sweep
  for (int d = SB, off = SB; d >= 1; d >>= 1, off >>= 1) {
    __syncthreads();
    const int i = (2 * t + 2) * off - 1;
    if (t < SB / d) {
      const int x = s[i - off];
      s[i - off] = s[i];
      s[i] += x;
    }
  }
  __syncthreads();
  if (base + t < n) a[base + t] = s[t];
  if (base + t + SB < n) a[base + t + SB] = s[t + SB];
}

// exclusive scan of the block totals by one block (serial in chunks)
__global__ void k_scan_totals(int *tot, int nb, int *count) {
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int c0 = 0; c0 < nb; c0 += blockDim.x) {
    const int i = c0 + threadIdx.x;
    const int v = i < nb ? tot[i] : 0;
    // inclusive warp-by-warp scan of this chunk
    __shared__ int ws[32];
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if ((threadIdx.x & 31) >= o) x += y;
    }
    if ((threadIdx.x & 31) == 31) ws[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
      int w = threadIdx.x < (int)(blockDim.x >> 5) ? ws[threadIdx.x] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, w, o);
        if (threadIdx.x >= o) w += y;
      }
      ws[threadIdx.x] = w;
    }
    __syncthreads();
    const int warp_off = (threadIdx.x >> 5) ? ws[(threadIdx.x >> 5) - 1] : 0;
    if (i < nb) tot[i] = carry + warp_off + x - v;  // exclusive
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += warp_off + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = carry;
}

__global__ void k_scan_add(int *a, int n, const int *tot) {
  const int base = blockIdx.x * 2 * SB;
  const int add = tot[blockIdx.x];
  for (int t = threadIdx.x; t < 2 * SB; t += blockDim.x)
    if (base + t < n) a[base + t] += add;
}

// label of piece q: the rank of its fragment's lowest piece (-1: no piece)
__global__ void k_frag_label(DevState d, const int *parent, const int *minp, const int *rank,
                             int *label, int nq) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
    int n[4];
    label[q] = piece_nodes(d, q, n) ? rank[minp[parent[n[0]]]] : -1;
  }
}

int grid_of(long n) {
  long b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 8 * 1216 ? 8 * 1216 : b));
}

}  // namespace

size_t fragments_scratch_bytes(const DevState &d, int n_nodes) {
  const size_t nq = 2 * (size_t)d.g.ne;
  const size_t nb = (nq + 2 * SB - 1) / (2 * SB);
  return 4 * ((size_t)n_nodes * 2 + nq + nb + 1);
}

cudaError_t launch_fragments(const DevState &d, int n_nodes, void *scratch, int *labels,
                             int *count, cudaStream_t st) {
  const int nq = 2 * d.g.ne;
  const int nb = (nq + 2 * SB - 1) / (2 * SB);
  int *parent = static_cast<int *>(scratch);
  int *minp = parent + n_nodes;  // indexed by root node id
  int *rank = minp + n_nodes;    // [nq]
  int *tot = rank + nq;          // [nb]
  const int g = grid_of(nq > n_nodes ? nq : n_nodes);
  k_frag_init<<<g, 256, 0, st>>>(parent, minp, n_nodes);
  k_frag_link<<<g, 256, 0, st>>>(d, parent, nq);
  k_frag_flatten<<<g, 256, 0, st>>>(parent, n_nodes);
  k_frag_minpiece<<<g, 256, 0, st>>>(d, parent, minp, nq);
  k_frag_rep<<<g, 256, 0, st>>>(d, parent, minp, rank, nq);
  k_scan_blocks<<<nb, SB, 0, st>>>(rank, nq, tot);
  k_scan_totals<<<1, 1024, 0, st>>>(tot, nb, count);
  k_scan_add<<<nb, 256, 0, st>>>(rank, nq, tot);
  k_frag_label<<<g, 256, 0, st>>>(d, parent, minp, rank, labels, nq);
  return cudaGetLastError();
}

}  // namespace cem
