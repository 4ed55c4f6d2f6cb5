// api.cpp -- host runtime behind the C ABI of include/cem.h.
//
// Owns the device state of one structured mesh, builds the problem on the
// host (loads, masses via a kernel, pre-cracks via the tracking kernel),
// captures one CUDA graph per (displacement buffer, energy-record) variant of
// the explicit step, and replays them.  Host arithmetic that must agree with
// the definition bit for bit (D matrix, time step, equivalent nodal forces,
// load factors) is compiled with -ffp-contract=off.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/cem.h"
#include "cem_internal.h"
#include "tri_internal.h"

using namespace cem;

struct BatchPlan;

struct cem_handle {
  DevState d{};
  int device = 0;
  cudaStream_t st = nullptr;
  cem_alloc_fn alloc = nullptr;
  cem_free_fn free_fn = nullptr;
  void *ctx = nullptr;
  std::vector<void *> blocks;
  int nx = 0, ny = 0;
  double hx = 0, hy = 0;
  std::vector<uint8_t> active;
  std::vector<int> precracks;
  double dt_factor = 0.5, dt_explicit = 0.0;
  bool material = false;
  // loads (host mirrors, uploaded on change)
  std::vector<double> Fx, Fy, Vx, Vy;
  std::vector<uint8_t> nflag;
  bool neu_set = false, dir_set = false;
  int neu_law = 0, dir_law = 0;
  double neu_t0 = 0, neu_tau = 0, dir_t0 = 0, dir_tau = 0;
  int cur = 0;
  bool mrow_stale = true;  // the FP32 node update's row flags need a rebuild
  long step = 0;
  int energy_every = 0;
  cudaGraphExec_t graphs[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [cur][energy]
  // graphs of kGraphSteps consecutive steps, keyed by cur | energy mask << 1
  std::map<unsigned, cudaGraphExec_t> multi;
  Counters *h_cnt = nullptr;  // pinned
  double *h_lam = nullptr;    // pinned staging of the load-factor table
  bool own_stream = false;
  StepStreams ss{};           // fork/join streams and events of one step
  long launches = 0;           // kernels enqueued (graph replays count their nodes)
  long lam_lo = 0, lam_n = 0;  // steps [lam_lo, lam_lo + lam_n) have device load factors
  void *scratch = nullptr;     // reusable device scratch for getters
  size_t scratch_bytes = 0;
  std::string err;
  BatchPlan *batch = nullptr;   // set on a batch handle (cem_batch_create)
  cem_handle *in_batch = nullptr;  // set on a member of a batch
  TriMesh *tri = nullptr;          // set on an unstructured triangle mesh (tri.cu)
  // cem_step_async: two pinned status slots, their events, which are pending
  Counters *h_async = nullptr;  // two status slots, mapped pinned memory
  Counters *d_async = nullptr;  // their device alias
  cudaEvent_t async_ev[2] = {nullptr, nullptr};
  int async_next = 0;
  unsigned async_pending = 0;
  long async_from[2] = {0, 0};  // steps taken before the call held by each slot
  int async_steps[2] = {0, 0};  // and its step count (0: no per-step words)
  // per-step status words of pipelined calls: kStatusRing slots of mapped
  // pinned memory, each step's written by the last block of its split writes
  Counters *h_ring = nullptr, *d_ring = nullptr;
  bool ring_on = false;          // the steps being enqueued write their word
  cudaGraphExec_t rgraphs[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // with the words
  std::map<unsigned, cudaGraphExec_t> rmulti;
};

namespace {

std::string g_create_error;

cem_status fail(cem_handle *h, cem_status code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (h) h->err = buf; else g_create_error = buf;
  return code;
}

// a triangle-mesh call's status, its message kept on the handle
cem_status tri_rc(cem_handle *h, cem_status rc, const std::string &e) {
  if (rc != CEM_OK) h->err = e;
  return rc;
}

#define TRI_NOT_AVAILABLE(h)                                                          \
  do {                                                                                \
    if ((h)->tri) return fail((h), CEM_ERR_STATE, "not available on a triangle mesh"); \
  } while (0)

#define CUDA_TRY(h, expr)                                                               \
  do {                                                                                  \
    cudaError_t _e = (expr);                                                            \
    if (_e != cudaSuccess)                                                              \
      return fail((h), CEM_ERR_CUDA, "%s failed: %s", #expr, cudaGetErrorString(_e)); \
  } while (0)

void *dalloc(cem_handle *h, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~(size_t)255;
  void *p = nullptr;
  if (h->alloc) {
    p = h->alloc(bytes, h->ctx);
  } else if (cudaMallocAsync(&p, bytes, h->st) != cudaSuccess) {
    p = nullptr;
  }
  if (p) {
    h->blocks.push_back(p);
    if (cudaMemsetAsync(p, 0, bytes, h->st) != cudaSuccess) return nullptr;
  }
  return p;
}

// Device scratch reused by getters; grows geometrically.
void *scratch(cem_handle *h, size_t bytes) {
  if (bytes <= h->scratch_bytes) return h->scratch;
  size_t want = std::max(bytes, 2 * h->scratch_bytes);
  void *p = dalloc(h, want);
  if (!p) return nullptr;
  h->scratch = p;
  h->scratch_bytes = want;
  return p;
}

template <class T>
bool dalloc_n(cem_handle *h, T *&p, size_t n) {
  p = (T *)dalloc(h, n * sizeof(T));
  return p != nullptr;
}

double law_eval(int law, double t, double t0, double tau) {
  if (law == CEM_LAW_CONST) return 1.0;
  if (t <= t0) return t / t0;
  if (law == CEM_LAW_RAMP) return 1.0;
  return exp(-(t - t0) / tau);
}

void edge_sides_host(const cem_handle *h, int g, int &lo, int &hi) {
  int nx = h->nx, ny = h->ny, nh = nx * (ny + 1);
  if (g < nh) {
    int j = g / nx, i = g % nx;
    lo = j > 0 ? (j - 1) * nx + i : -1;
    hi = j < ny ? j * nx + i : -1;
  } else {
    int gg = g - nh, j = gg / (nx + 1), i = gg % (nx + 1);
    lo = i > 0 ? j * nx + i - 1 : -1;
    hi = i < nx ? j * nx + i : -1;
  }
}

void edge_nodes_host(const cem_handle *h, int g, int &n1, int &n2) {
  int nx = h->nx, ny = h->ny, nh = nx * (ny + 1), r = nx + 1;
  if (g < nh) {
    int j = g / nx, i = g % nx;
    n1 = j * r + i; n2 = j * r + i + 1;
  } else {
    int gg = g - nh, j = gg / r, i = gg % r;
    n1 = j * r + i; n2 = (j + 1) * r + i;
  }
}

int local_edge_host(const cem_handle *h, int e, int g) {
  int nx = h->nx, ny = h->ny, nh = nx * (ny + 1);
  int i = e % nx, j = e / nx;
  if (g == j * nx + i) return 0;
  if (g == nh + j * (nx + 1) + i + 1) return 1;
  if (g == (j + 1) * nx + i) return 2;
  if (g == nh + j * (nx + 1) + i) return 3;
  return -1;
}

// Status word of the counters mirrored in h->h_cnt.
cem_status check_counters(cem_handle *h, const Counters &c) {
  int s = c.status;
  if (s & STAT_CAPACITY)
    return fail(h, CEM_ERR_CAPACITY,
                "capacity exceeded (phantoms %d/%d, cracks %d/%d, list %d/%d, proposals cap %d)",
                c.n_ph, h->d.ph_cap, c.n_ck, h->d.ck_cap, c.n_S, h->d.list_cap, h->d.prop_cap);
  if (s & STAT_NONFINITE) return fail(h, CEM_ERR_NONFINITE, "non-finite displacement or velocity");
  if (s & STAT_TIMEOUT) return fail(h, CEM_ERR_TIMEOUT, "device wait timed out");
  return CEM_OK;
}

cem_status check_status(cem_handle *h) { return check_counters(h, *h->h_cnt); }

cem_status sync_status(cem_handle *h) {
  CUDA_TRY(h, cudaMemcpyAsync(h->h_cnt, h->d.cnt, sizeof(Counters), cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  return check_status(h);
}

cem_status upload_loads(cem_handle *h) {
  size_t nn = (size_t)h->d.g.nn;
  CUDA_TRY(h, cudaMemcpyAsync(h->d.Fx, h->Fx.data(), nn * 8, cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(h->d.Fy, h->Fy.data(), nn * 8, cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(h->d.Vx, h->Vx.data(), nn * 8, cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(h->d.Vy, h->Vy.data(), nn * 8, cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(h->d.nflag, h->nflag.data(), nn, cudaMemcpyHostToDevice, h->st));
  std::vector<int> bc;
  for (size_t N = 0; N < nn; ++N)
    if (h->nflag[N]) bc.push_back((int)N);
  if (!bc.empty())
    CUDA_TRY(h, cudaMemcpyAsync(h->d.bc_nodes, bc.data(), bc.size() * 4, cudaMemcpyHostToDevice, h->st));
  h->d.n_bc = (int)bc.size();
  h->mrow_stale = true;
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  return CEM_OK;
}

// Row flags of the FP32 node update, rebuilt before a step whenever the
// node flags or element states were written from the host (the apply kernel
// keeps them current as elements split).
cem_status ensure_march_rows(cem_handle *h) {
  if (!h->mrow_stale || h->d.precision != CEM_FP32_MIXED) return CEM_OK;
  CUDA_TRY(h, launch_march_rows(h->d, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));  // a batch steps its members on its own stream
  h->mrow_stale = false;
  return CEM_OK;
}

void drop_graphs(cem_handle *h) {
  for (auto *set : {&h->graphs, &h->rgraphs})
    for (auto &row : *set)
      for (auto &g : row)
        if (g) { cudaGraphExecDestroy(g); g = nullptr; }
  for (auto *m : {&h->multi, &h->rmulti}) {
    for (auto &kv : *m) cudaGraphExecDestroy(kv.second);
    m->clear();
  }
}

// kernels one step launches: the step kernels, selection and split writes,
// the energy prologue and epilogue on record steps
int kernels_in_step(const cem_handle *, bool energy) { return kStepKernels + 2 + (energy ? 2 : 0); }

// Enqueues one explicit step (buffers cur -> cur^1) on the stream.  With
// marks (profiling) events are recorded after the energy prologue, after
// each step kernel, after the energy epilogue, after the tracking selection
// and after the split writes: marks[0..7].
cudaError_t enqueue_step(cem_handle *h, int cur, bool first, bool energy,
                         cudaEvent_t *marks = nullptr) {
  const DevState &d = h->d;
  cudaError_t e;
  if (energy && (e = launch_energy_pre(d, h->st)) != cudaSuccess) return e;
  if (marks) cudaEventRecord(marks[0], h->st);
  if (d.precision == CEM_FP32_MIXED) e = launch_step_fp32(d, cur, first, energy, h->ss, marks ? marks + 1 : nullptr);
  else e = launch_step_fp64(d, cur, first, energy, h->ss, marks ? marks + 1 : nullptr);
  if (e != cudaSuccess) return e;
  if (marks) cudaEventRecord(marks[4], h->st);
  if (energy && (e = launch_energy_post(d, energy_parts_step(d), h->st)) != cudaSuccess) return e;
  if (marks) {
    cudaEventRecord(marks[5], h->st);
    e = launch_select(d, TRACK_STEP, h->st);
    if (e != cudaSuccess) return e;
    cudaEventRecord(marks[6], h->st);
  }
  // a programmatic dependent of the node update only in a captured graph
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const bool captured = !marks && cudaStreamIsCapturing(h->st, &cs) == cudaSuccess &&
                        cs == cudaStreamCaptureStatusActive;
  e = launch_apply(d, cur ^ 1, TRACK_STEP, h->st, captured,
                   h->ring_on && !marks ? h->d_ring : nullptr);
  if (marks) cudaEventRecord(marks[7], h->st);
  return e;
}

// Load factors of steps [h->step, h->step + chunk) into the device table,
// enqueued on stream st (the handle's own stream by default).
cem_status upload_load_factors(cem_handle *h, int chunk, cudaStream_t st = nullptr) {
  if (!st) st = h->st;
  const DevState &d = h->d;
  const double dt = d.mat.dt;
  double *lamN = h->h_lam, *lamD = h->h_lam + d.lam_cap;
  for (int q = 0; q < chunk; ++q) {
    long s = h->step + q;
    lamN[q] = h->neu_set ? law_eval(h->neu_law, (double)s * dt, h->neu_t0, h->neu_tau) : 0.0;
    lamD[q] = h->dir_set ? law_eval(h->dir_law, ((double)s + 0.5) * dt, h->dir_t0, h->dir_tau) : 0.0;
  }
  int base = (int)h->step;
  h->h_cnt->lam_base = base;
  h->lam_lo = h->step;
  h->lam_n = chunk;
  CUDA_TRY(h, cudaMemcpyAsync(d.lamN, lamN, chunk * 8, cudaMemcpyHostToDevice, st));
  CUDA_TRY(h, cudaMemcpyAsync(d.lamD, lamD, chunk * 8, cudaMemcpyHostToDevice, st));
  CUDA_TRY(h, cudaMemcpyAsync(&d.cnt->lam_base, &h->h_cnt->lam_base, 4, cudaMemcpyHostToDevice, st));
  // the pinned staging is reused only after the stream has been synchronised
  return CEM_OK;
}

// The streams of a step's side branches (evaluation + selection, piece
// forces + phantom update) get the highest priority: their short kernels
// then take SM slots as the tile update's CTAs retire instead of queueing
// behind its remaining waves.  Step graphs are instantiated so that kernel
// nodes keep the priority of the stream they were captured from.
cudaError_t create_aux_streams(StepStreams &ss) {
  int least = 0, greatest = 0;
  cudaError_t ce = cudaDeviceGetStreamPriorityRange(&least, &greatest);
  if (ce == cudaSuccess) ce = cudaStreamCreateWithPriority(&ss.aux1, cudaStreamNonBlocking, greatest);
  if (ce == cudaSuccess) ce = cudaStreamCreateWithPriority(&ss.aux2, cudaStreamNonBlocking, greatest);
  return ce;
}

// A kernel launched as a programmatic dependent right after cross-stream
// joins is captured with programmatic edges from every joined kernel, not
// only from the kernel before it in its stream.  The split writes read the
// selection's plan before their grid-dependency wait, so their edges from the
// side branches' last kernels (the selection, the phantom update) are made
// ordinary here: the split writes then start after those have completed,
// while only the node update (or the energy epilogue) may still be running.
cudaError_t ordinary_side_edges(cudaGraph_t g) {
  auto func_of = [](cudaGraphNode_t nd) -> const void * {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) != cudaSuccess || t != cudaGraphNodeTypeKernel) return nullptr;
    cudaKernelNodeParams p;
    return cudaGraphKernelNodeGetParams(nd, &p) == cudaSuccess ? p.func : nullptr;
  };
  const void *side[3] = {select_kernel(), phantom32_kernel(), phantom64_kernel()};
  size_t n = 0;
  cudaError_t e = cudaGraphGetNodes(g, nullptr, &n);
  std::vector<cudaGraphNode_t> nodes(n);
  if (e == cudaSuccess && n) e = cudaGraphGetNodes(g, nodes.data(), &n);
  for (size_t i = 0; i < n && e == cudaSuccess; ++i) {
    if (func_of(nodes[i]) != apply_kernel()) continue;
    size_t m = 0;
    e = cudaGraphNodeGetDependencies(nodes[i], nullptr, nullptr, &m);
    std::vector<cudaGraphNode_t> from(m);
    std::vector<cudaGraphEdgeData> ed(m);
    if (e == cudaSuccess && m) e = cudaGraphNodeGetDependencies(nodes[i], from.data(), ed.data(), &m);
    for (size_t k = 0; k < m && e == cudaSuccess; ++k) {
      if (ed[k].type != cudaGraphDependencyTypeProgrammatic) continue;
      const void *f = func_of(from[k]);
      if (f != side[0] && f != side[1] && f != side[2]) continue;
      e = cudaGraphRemoveDependencies(g, &from[k], &nodes[i], &ed[k], 1);
      if (e == cudaSuccess) e = cudaGraphAddDependencies(g, &from[k], &nodes[i], nullptr, 1);
    }
  }
  return e;
}

cem_status graph_for(cem_handle *h, int cur, int energy, cudaGraphExec_t *out) {
  cudaGraphExec_t &slot = h->ring_on ? h->rgraphs[cur][energy] : h->graphs[cur][energy];
  if (!slot) {
    cudaGraph_t g;
    CUDA_TRY(h, cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue_step(h, cur, false, energy != 0);
    cudaError_t e2 = cudaStreamEndCapture(h->st, &g);
    if (e != cudaSuccess) return fail(h, CEM_ERR_CUDA, "capture: %s", cudaGetErrorString(e));
    if (e2 != cudaSuccess) return fail(h, CEM_ERR_CUDA, "end capture: %s", cudaGetErrorString(e2));
    cudaError_t e3 = ordinary_side_edges(g);
    if (e3 == cudaSuccess) e3 = cudaGraphInstantiate(&slot, g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) return fail(h, CEM_ERR_CUDA, "instantiate: %s", cudaGetErrorString(e3));
  }
  *out = slot;
  return CEM_OK;
}

// Consecutive steps replayed as one graph: the launch of a graph costs a few
// microseconds of idle GPU between graphs, which a dependency inside one
// graph does not.  kGraphSteps is even, so the displacement buffer index is
// the same after the group as before it.  A group holds an energy record only
// in its first step (single steps realign the groups), so there are two
// group graphs per buffer index, built once.
constexpr int kGraphSteps = 8;

// Energy-record mask of the kGraphSteps steps from `step`, or -1 when a
// record falls after the first of them (the caller takes a single step).
int group_mask(long step, int energy_every) {
  if (energy_every <= 0) return 0;
  for (int r = 1; r < kGraphSteps; ++r)
    if ((step + r) % energy_every == 0) return -1;
  return step % energy_every == 0 ? 1 : 0;
}

cem_status multi_graph_for(cem_handle *h, int cur, unsigned mask, cudaGraphExec_t *out) {
  const unsigned key = (unsigned)cur | (mask << 1);
  auto &cache = h->ring_on ? h->rmulti : h->multi;
  auto it = cache.find(key);
  if (it == cache.end()) {
    cudaGraph_t g;
    CUDA_TRY(h, cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < kGraphSteps && e == cudaSuccess; ++q)
      e = enqueue_step(h, cur ^ (q & 1), false, ((mask >> q) & 1) != 0);
    cudaError_t e2 = cudaStreamEndCapture(h->st, &g);
    if (e != cudaSuccess) return fail(h, CEM_ERR_CUDA, "capture: %s", cudaGetErrorString(e));
    if (e2 != cudaSuccess) return fail(h, CEM_ERR_CUDA, "end capture: %s", cudaGetErrorString(e2));
    cudaGraphExec_t x = nullptr;
    cudaError_t e3 = ordinary_side_edges(g);
    if (e3 == cudaSuccess) e3 = cudaGraphInstantiate(&x, g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) return fail(h, CEM_ERR_CUDA, "instantiate: %s", cudaGetErrorString(e3));
    it = cache.emplace(key, x).first;
  }
  *out = it->second;
  return CEM_OK;
}

cem_status batch_step(cem_handle *b, int n);
cem_status batch_counts(cem_handle *b, cem_counts *out);
void batch_release(cem_handle *b);
void batch_detach(cem_handle *member);

}  // namespace

extern "C" {

const char *cem_last_error(const cem_handle *h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

cem_status cem_tri_mesh_create(const cem_tri_mesh_desc *desc, cem_handle **out) {
  if (!desc || !out) return fail(nullptr, CEM_ERR_ARG, "null argument");
  *out = nullptr;
  std::string e;
  TriMesh *t = tri_create(desc, e);
  if (!t) return fail(nullptr, e.rfind("CUDA", 0) == 0 || e.rfind("device", 0) == 0 ? CEM_ERR_CUDA : CEM_ERR_ARG,
                      "%s", e.c_str());
  cem_handle *h = new cem_handle();
  h->tri = t;
  h->device = desc->device;
  *out = h;
  return CEM_OK;
}

cem_status cem_tri_eval_surface(cem_handle *h, int n, const int *edge, const int *elem, double *G,
                                int *choice) {
  if (!h) return CEM_ERR_ARG;
  if (!h->tri) return fail(h, CEM_ERR_STATE, "not a triangle mesh");
  std::string e;
  return tri_rc(h, tri_eval_surface(h->tri, n, edge, elem, G, choice, e), e);
}

cem_status cem_mesh_create(const cem_mesh_desc *desc, cem_handle **out) {
  if (!desc || !out) return fail(nullptr, CEM_ERR_ARG, "null argument");
  *out = nullptr;
  if (desc->nx < 1 || desc->ny < 1 || !(desc->hx > 0) || !(desc->hy > 0))
    return fail(nullptr, CEM_ERR_ARG, "bad mesh size");
  long ne = (long)desc->nx * desc->ny, nn = (long)(desc->nx + 1) * (desc->ny + 1);
  if (ne > (1L << 27)) return fail(nullptr, CEM_ERR_ARG, "mesh too large (max 2^27 elements)");
  if (desc->precision != CEM_FP64 && desc->precision != CEM_FP32_MIXED)
    return fail(nullptr, CEM_ERR_ARG, "bad precision");
  if (desc->alloc && !desc->free) return fail(nullptr, CEM_ERR_ARG, "alloc without free");
  if (desc->n_precracks < 0 || (desc->n_precracks > 0 && !desc->precrack))
    return fail(nullptr, CEM_ERR_ARG, "bad pre-crack list");
  cem_handle *h = new (std::nothrow) cem_handle();
  if (!h) return fail(nullptr, CEM_ERR_ARG, "out of host memory");
  h->device = desc->device;
  h->st = (cudaStream_t)desc->cuda_stream;
  h->alloc = desc->alloc;
  h->free_fn = desc->free;
  h->ctx = desc->alloc_ctx;
  h->nx = desc->nx; h->ny = desc->ny; h->hx = desc->hx; h->hy = desc->hy;
  h->dt_factor = desc->dt_factor > 0 ? desc->dt_factor : 0.5;
  h->dt_explicit = desc->dt;
  h->energy_every = desc->energy_every > 0 ? desc->energy_every : 0;
  h->active.assign((size_t)ne, 1);
  if (desc->elem_active)
    for (long e = 0; e < ne; ++e) h->active[e] = desc->elem_active[e] != 0;
  for (int q = 0; q < desc->n_precracks; ++q) {
    int e = desc->precrack[3 * q], ka = desc->precrack[3 * q + 1], kb = desc->precrack[3 * q + 2];
    if (e < 0 || e >= ne || !h->active[e] || ka < 0 || ka > 3 || kb < 0 || kb > 3 || ka == kb) {
      delete h;
      return fail(nullptr, CEM_ERR_ARG, "bad pre-crack triple %d", q);
    }
    for (int r = 0; r < q; ++r)
      if (desc->precrack[3 * r] == e) {
        delete h;
        return fail(nullptr, CEM_ERR_ARG, "element %d pre-cracked twice", e);
      }
    h->precracks.insert(h->precracks.end(), {e, ka, kb});
  }
  cudaError_t ce = cudaSetDevice(h->device);
  if (ce == cudaSuccess && !h->st) {
    // graphs cannot be captured on the legacy default stream: use our own
    ce = cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking);
    h->own_stream = ce == cudaSuccess;
  }
  if (ce == cudaSuccess) ce = create_aux_streams(h->ss);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&h->ss.fork, cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&h->ss.join1, cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&h->ss.join2, cudaEventDisableTiming);
  h->ss.main = h->st;
  if (ce != cudaSuccess) {
    delete h;
    return fail(nullptr, CEM_ERR_CUDA, "device set-up: %s", cudaGetErrorString(ce));
  }
  DevState &d = h->d;
  d.step_end = INT_MAX;
  d.cur_xor = 0;
  d.g.nx = desc->nx; d.g.ny = desc->ny; d.g.nn = (int)nn; d.g.ne = (int)ne;
  d.g.nh = desc->nx * (desc->ny + 1);
  d.g.ned = d.g.nh + (desc->nx + 1) * desc->ny;
  d.g.hx = desc->hx; d.g.hy = desc->hy; d.g.A = desc->hx * desc->hy;
  d.g.rx = 1.0 / desc->hx; d.g.rxh = d.g.rx * 0.5;
  d.g.ry = 1.0 / desc->hy; d.g.ryh = d.g.ry * 0.5;
  d.g.rxf = (float)d.g.rx; d.g.ryf = (float)d.g.ry; d.g.qAf = (float)(d.g.A * 0.25);
  {
    // reference edge vectors and candidate-path normals for the FP32 mode
    const double XN[4] = {-1, 1, 1, -1}, EN[4] = {-1, -1, 1, 1};
    const double XG[4] = {0, 1, 0, -1}, EG[4] = {-1, 0, 1, 0};
    for (int k0 = 0; k0 < 4; ++k0) {
      double DX = (XN[(k0 + 1) % 4] - XN[k0]) * (0.5 * desc->hx);
      double DY = (EN[(k0 + 1) % 4] - EN[k0]) * (0.5 * desc->hy);
      d.g.DXf[k0] = (float)DX;
      d.g.DYf[k0] = (float)DY;
      for (int k = 0; k < 4; ++k) {
        if (k == k0) { d.g.nxf[k0][k] = d.g.nyf[k0][k] = 0.f; continue; }
        double sx = (XG[k] - XG[k0]) * (0.5 * desc->hx), sy = (EG[k] - EG[k0]) * (0.5 * desc->hy);
        double rx = -sy, ry = sx;
        if (rx * DX + ry * DY < 0.0) { rx = -rx; ry = -ry; }
        double len = sqrt(sx * sx + sy * sy);
        d.g.nxf[k0][k] = (float)(rx / len);
        d.g.nyf[k0][k] = (float)(ry / len);
      }
    }
  }
  d.precision = desc->precision;
  d.ph_cap = desc->phantom_capacity > 0 ? desc->phantom_capacity : (int)(ne / 4 + 4096);
  d.ck_cap = desc->crack_capacity > 0 ? desc->crack_capacity : (int)(ne / 4 + 4096);
  long rim = 0;
  for (int g = 0; g < d.g.ned; ++g) {
    int lo, hi;
    edge_sides_host(h, g, lo, hi);
    bool alo = lo >= 0 && h->active[lo], ahi = hi >= 0 && h->active[hi];
    rim += alo != ahi;
  }
  long lc = desc->list_capacity > 0 ? desc->list_capacity
                                    : 2 * (rim + 4L * d.ck_cap) + 8192;
  if (lc > (1L << 30)) lc = 1L << 30;
  d.list_cap = (int)lc;
  d.prop_cap = track_sort_capacity();
  d.ncap = d.g.nn + d.ph_cap;
  d.lam_cap = 4096;
  d.rec_cap = 65536;
  size_t nc = (size_t)d.ncap, nec = (size_t)ne;
  bool ok = true;
  if (d.precision == CEM_FP64) {
    for (int b = 0; b < 2; ++b) ok = ok && dalloc_n(h, d.ux[b], nc) && dalloc_n(h, d.uy[b], nc);
    ok = ok && dalloc_n(h, d.vx, nc) && dalloc_n(h, d.vy, nc) && dalloc_n(h, d.pf, (size_t)d.ck_cap * 16);
  } else {
    for (int b = 0; b < 2; ++b) ok = ok && dalloc_n(h, d.u4[b], nc);
    ok = ok && dalloc_n(h, d.v2, nc) && dalloc_n(h, d.minvf, nc) &&
         dalloc_n(h, d.pff, (size_t)d.ck_cap * 16) && dalloc_n(h, d.pfe, nec * 8) &&
         dalloc_n(h, d.fsp, (size_t)nn);
  }
  ok = ok && dalloc_n(h, d.m, nc) && dalloc_n(h, d.minv, nc) && dalloc_n(h, d.Wn, nc) &&
       dalloc_n(h, d.Wd, nc) && dalloc_n(h, d.nflag, (size_t)nn) && dalloc_n(h, d.Fx, (size_t)nn) &&
       dalloc_n(h, d.Fy, (size_t)nn) && dalloc_n(h, d.Vx, (size_t)nn) && dalloc_n(h, d.Vy, (size_t)nn) &&
       dalloc_n(h, d.bc_nodes, (size_t)nn) && dalloc_n(h, d.estate, nec) &&
       dalloc_n(h, d.mrow, (size_t)(d.g.ny + 1) * march_tiles_x_of(d.g.nx)) &&
       dalloc_n(h, d.crack_of, nec) && dalloc_n(h, d.gc, nec) &&
       dalloc_n(h, d.ck_elem, (size_t)d.ck_cap) && dalloc_n(h, d.ck_info, (size_t)d.ck_cap) &&
       dalloc_n(h, d.ck_node, (size_t)d.ck_cap * 8) && dalloc_n(h, d.ck_Ap, (size_t)d.ck_cap * 2) &&
       dalloc_n(h, d.ck_ud, (size_t)d.ck_cap) && dalloc_n(h, d.ck_step, (size_t)d.ck_cap) &&
       dalloc_n(h, d.ph_owner, (size_t)d.ph_cap) && dalloc_n(h, d.ph_creator, (size_t)d.ph_cap) &&
       dalloc_n(h, d.ph_nuser, (size_t)d.ph_cap) && dalloc_n(h, d.ph_users, (size_t)d.ph_cap * 4) &&
       dalloc_n(h, d.ph_upf, (size_t)d.ph_cap * 4) && dalloc_n(h, d.ph_uap, (size_t)d.ph_cap * 4) &&
       dalloc_n(h, d.S, (size_t)d.list_cap) && dalloc_n(h, d.S_info, (size_t)d.list_cap) &&
       dalloc_n(h, d.S_G, (size_t)d.list_cap) && dalloc_n(h, d.spos, (size_t)d.g.ned) &&
       dalloc_n(h, d.pr_key, (size_t)d.prop_cap) && dalloc_n(h, d.pr_edge, (size_t)d.prop_cap) &&
       dalloc_n(h, d.pr_k, (size_t)d.prop_cap) && dalloc_n(h, d.pr_G, (size_t)d.prop_cap) &&
       dalloc_n(h, d.pl_e, (size_t)d.prop_cap) && dalloc_n(h, d.pl_info, (size_t)d.prop_cap) &&
       dalloc_n(h, d.pl_reuse, (size_t)d.prop_cap * 4) && dalloc_n(h, d.pl_tomb, (size_t)d.prop_cap * 4) &&
       dalloc_n(h, d.pl_c, (size_t)d.prop_cap) && dalloc_n(h, d.pl_ph0, (size_t)d.prop_cap) &&
       dalloc_n(h, d.pl_app0, (size_t)d.prop_cap) && dalloc_n(h, d.pl_alpha, (size_t)d.prop_cap * 2) &&
       dalloc_n(h, d.pl_mreal, (size_t)d.prop_cap * 4) && dalloc_n(h, d.pl_mph, (size_t)d.prop_cap * 4) &&
       dalloc_n(h, d.pl_mold, (size_t)d.prop_cap * 4) && dalloc_n(h, d.pl_dm, (size_t)d.prop_cap * 4) &&
       dalloc_n(h, d.pl_mireal, (size_t)d.prop_cap * 4) && dalloc_n(h, d.pl_miph, (size_t)d.prop_cap * 4) &&
       dalloc_n(h, d.pl_users, (size_t)d.prop_cap * 16) && dalloc_n(h, d.pl_upf, (size_t)d.prop_cap * 16) &&
       dalloc_n(h, d.pl_uap, (size_t)d.prop_cap * 16) &&
       dalloc_n(h, d.pl_nu, (size_t)d.prop_cap * 4) &&
       dalloc_n(h, d.sel_sk, (size_t)d.prop_cap) && dalloc_n(h, d.sel_win, (size_t)d.prop_cap) &&
       dalloc_n(h, d.sel_G, (size_t)d.prop_cap) && dalloc_n(h, d.sel_E, (size_t)d.prop_cap) &&
       dalloc_n(h, d.sel_K, (size_t)d.prop_cap) &&
       dalloc_n(h, d.cnt, 1) && dalloc_n(h, d.lamN, (size_t)d.lam_cap) &&
       dalloc_n(h, d.lamD, (size_t)d.lam_cap) && dalloc_n(h, d.erec, (size_t)d.rec_cap * 7);
  d.e_part_cap = energy_parts_needed(d);
  ok = ok && dalloc_n(h, d.e_part, (size_t)d.e_part_cap * 2) && dalloc_n(h, d.e_pre, (size_t)EPRE * 3);
  if (!ok || cudaHostAlloc((void **)&h->h_cnt, sizeof(Counters), cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc((void **)&h->h_lam, 2 * sizeof(double) * d.lam_cap, cudaHostAllocDefault) != cudaSuccess) {
    g_create_error = "device allocation failed";
    cem_mesh_destroy(h);
    return CEM_ERR_CUDA;
  }
  // element states and crack map
  std::vector<uint8_t> st((size_t)ne);
  for (long e = 0; e < ne; ++e) st[e] = h->active[e] ? ST_INTACT : ST_OUT;
  std::vector<int> minus1(std::max((size_t)ne, (size_t)d.g.ned), -1);
  if (cudaMemcpyAsync(d.estate, st.data(), nec, cudaMemcpyHostToDevice, h->st) != cudaSuccess ||
      cudaMemcpyAsync(d.crack_of, minus1.data(), nec * 4, cudaMemcpyHostToDevice, h->st) != cudaSuccess ||
      cudaMemcpyAsync(d.spos, minus1.data(), (size_t)d.g.ned * 4, cudaMemcpyHostToDevice, h->st) != cudaSuccess ||
      cudaStreamSynchronize(h->st) != cudaSuccess) {
    g_create_error = "initial upload failed";
    cem_mesh_destroy(h);
    return CEM_ERR_CUDA;
  }
  h->Fx.assign((size_t)nn, 0.0); h->Fy.assign((size_t)nn, 0.0);
  h->Vx.assign((size_t)nn, 0.0); h->Vy.assign((size_t)nn, 0.0);
  h->nflag.assign((size_t)nn, 0);
  *out = h;
  return CEM_OK;
}

void cem_mesh_destroy(cem_handle *h) {
  if (!h) return;
  if (h->tri) {
    tri_destroy(h->tri);
    delete h;
    return;
  }
  cudaSetDevice(h->device);
  if (h->batch) batch_release(h);
  if (h->in_batch) batch_detach(h);
  drop_graphs(h);
  if (h->st) cudaStreamSynchronize(h->st); else cudaDeviceSynchronize();
  for (void *p : h->blocks) {
    if (h->free_fn) h->free_fn(p, h->ctx);
    else cudaFreeAsync(p, h->st);
  }
  if (h->st) cudaStreamSynchronize(h->st); else cudaDeviceSynchronize();
  if (h->h_cnt) cudaFreeHost(h->h_cnt);
  if (h->h_lam) cudaFreeHost(h->h_lam);
  if (h->h_async) cudaFreeHost(h->h_async);
  if (h->h_ring) cudaFreeHost(h->h_ring);
  for (cudaEvent_t ev : h->async_ev)
    if (ev) cudaEventDestroy(ev);
  if (h->ss.aux1) cudaStreamDestroy(h->ss.aux1);
  if (h->ss.aux2) cudaStreamDestroy(h->ss.aux2);
  if (h->ss.fork) cudaEventDestroy(h->ss.fork);
  if (h->ss.join1) cudaEventDestroy(h->ss.join1);
  if (h->ss.join2) cudaEventDestroy(h->ss.join2);
  if (h->own_stream) cudaStreamDestroy(h->st);
  delete h;
}

cem_status cem_set_material(cem_handle *h, double E, double nu, double rho,
                            const float *gc_per_elem, double gc_uniform, int plane_strain,
                            double gamma, int gamma_mode, int mct_scope) {
  if (!h) return CEM_ERR_ARG;
  if (h->tri) {
    std::string e;
    return tri_rc(h, tri_set_material(h->tri, E, nu, rho, plane_strain, gc_per_elem, gc_uniform,
                                      gamma, gamma_mode, e), e);
  }
  if (h->batch) return fail(h, CEM_ERR_STATE, "not valid on a batch handle");
  if (h->material) return fail(h, CEM_ERR_STATE, "material already set");
  if (!(E > 0) || !(nu > -1.0 && nu < 0.5) || !(rho > 0)) return fail(h, CEM_ERR_ARG, "bad material");
  if (mct_scope < 0 || mct_scope > 2 || gamma_mode < 0 || gamma_mode > 1)
    return fail(h, CEM_ERR_ARG, "bad scope or gamma mode");
  CUDA_TRY(h, cudaSetDevice(h->device));
  Mat &m = h->d.mat;
  if (plane_strain) {
    double c = E / ((1.0 + nu) * (1.0 - 2.0 * nu));
    m.D11 = c * (1.0 - nu);
    m.D12 = c * nu;
    m.D33 = c * (1.0 - 2.0 * nu) * 0.5;
  } else {
    double c = E / (1.0 - nu * nu);
    m.D11 = c;
    m.D12 = c * nu;
    m.D33 = c * (1.0 - nu) * 0.5;
  }
  m.D11f = (float)m.D11; m.D12f = (float)m.D12; m.D33f = (float)m.D33;
  m.rho = rho; m.gamma = gamma; m.gamma_mode = gamma_mode; m.scope = mct_scope;
  if (h->dt_explicit > 0) {
    m.dt = h->dt_explicit;
  } else {
    double cd;
    if (plane_strain) cd = sqrt((E * (1.0 - nu)) / (rho * ((1.0 + nu) * (1.0 - 2.0 * nu))));
    else cd = sqrt(E / (rho * (1.0 - nu * nu)));
    double hmin = h->hx < h->hy ? h->hx : h->hy;
    m.dt = h->dt_factor * hmin / cd;
  }
  m.dtf = (float)m.dt;
  const DevState &d = h->d;
  std::vector<float> gc((size_t)d.g.ne);
  for (int e = 0; e < d.g.ne; ++e) gc[e] = gc_per_elem ? gc_per_elem[e] : (float)gc_uniform;
  CUDA_TRY(h, cudaMemcpyAsync(d.gc, gc.data(), gc.size() * 4, cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(h, launch_init_masses(d, h->st));
  if (d.precision == CEM_FP32_MIXED) {
    // minvf follows minv
    std::vector<double> mi((size_t)d.g.nn);
    CUDA_TRY(h, cudaMemcpyAsync(mi.data(), d.minv, mi.size() * 8, cudaMemcpyDeviceToHost, h->st));
    CUDA_TRY(h, cudaStreamSynchronize(h->st));
    std::vector<float> mf(mi.size());
    for (size_t q = 0; q < mi.size(); ++q) mf[q] = (float)mi[q];
    CUDA_TRY(h, cudaMemcpyAsync(d.minvf, mf.data(), mf.size() * 4, cudaMemcpyHostToDevice, h->st));
  }
  // pre-cracks, one at a time in the given order (the same split routine)
  for (size_t q = 0; q < h->precracks.size(); q += 3) {
    int e = h->precracks[q], ka = h->precracks[q + 1], kb = h->precracks[q + 2];
    int i = e % h->nx, j = e / h->nx, nh = h->nx * (h->ny + 1);
    int edge = ka == 0 ? j * h->nx + i : ka == 1 ? nh + j * (h->nx + 1) + i + 1
             : ka == 2 ? (j + 1) * h->nx + i : nh + j * (h->nx + 1) + i;
    int key = e * 4 + ka;
    double G = 0.0;
    int one = 1;
    CUDA_TRY(h, cudaMemcpyAsync(d.pr_key, &key, 4, cudaMemcpyHostToDevice, h->st));
    CUDA_TRY(h, cudaMemcpyAsync(d.pr_edge, &edge, 4, cudaMemcpyHostToDevice, h->st));
    CUDA_TRY(h, cudaMemcpyAsync(d.pr_k, &kb, 4, cudaMemcpyHostToDevice, h->st));
    CUDA_TRY(h, cudaMemcpyAsync(d.pr_G, &G, 8, cudaMemcpyHostToDevice, h->st));
    CUDA_TRY(h, cudaMemcpyAsync(&d.cnt->n_prop, &one, 4, cudaMemcpyHostToDevice, h->st));
    CUDA_TRY(h, launch_select(d, TRACK_PRECRACK, h->st));
    CUDA_TRY(h, launch_apply(d, h->cur, TRACK_PRECRACK, h->st));
    CUDA_TRY(h, cudaStreamSynchronize(h->st));
  }
  CUDA_TRY(h, launch_build_surface(d, h->st));
  h->material = true;
  h->mrow_stale = true;
  return sync_status(h);
}

cem_status cem_set_bc(cem_handle *h, int kind, int n_items, const int *items, int comp_mask,
                      int law, double a0, double t0, double tau) {
  if (!h) return CEM_ERR_ARG;
  if (h->tri) {
    std::string e;
    return tri_rc(h, tri_set_bc(h->tri, kind, n_items, items, comp_mask, law, a0, t0, tau, e), e);
  }
  if (h->batch || h->in_batch) return fail(h, CEM_ERR_STATE, "not valid on a batch or its members");
  if (h->step != 0) return fail(h, CEM_ERR_STATE, "loads must be set before the first step");
  if (n_items < 0 || (n_items > 0 && !items)) return fail(h, CEM_ERR_ARG, "bad items");
  if (law < 0 || law > 2) return fail(h, CEM_ERR_ARG, "bad law");
  if (law != CEM_LAW_CONST && !(t0 > 0)) return fail(h, CEM_ERR_ARG, "t0 must be > 0");
  if (law == CEM_LAW_RAMP_EXP && !(tau > 0)) return fail(h, CEM_ERR_ARG, "tau must be > 0");
  const int nh = h->nx * (h->ny + 1), ned = nh + (h->nx + 1) * h->ny;
  const int nn = (h->nx + 1) * (h->ny + 1);
  if (kind == CEM_TRACTION || kind == CEM_PRESSURE) {
    if (h->neu_set && (h->neu_law != law || h->neu_t0 != t0 || h->neu_tau != tau))
      return fail(h, CEM_ERR_ARG, "all Neumann loads share one time law");
    for (int q = 0; q < n_items; ++q) {
      int g = items[q], lo, hi;
      if (g < 0 || g >= ned) return fail(h, CEM_ERR_ARG, "edge %d is not a boundary edge", g);
      edge_sides_host(h, g, lo, hi);
      bool alo = lo >= 0 && h->active[lo], ahi = hi >= 0 && h->active[hi];
      if (alo == ahi) return fail(h, CEM_ERR_ARG, "edge %d is not a boundary edge", g);
    }
    std::vector<int> sorted(items, items + n_items);
    std::sort(sorted.begin(), sorted.end());
    for (int g : sorted) {
      int lo, hi, n1, n2;
      edge_sides_host(h, g, lo, hi);
      bool alo = lo >= 0 && h->active[lo];
      bool horiz = g < nh;
      double sgn = alo ? 1.0 : -1.0;  // outward normal of the material side
      double ox = horiz ? 0.0 : sgn, oy = horiz ? sgn : 0.0;
      double L = horiz ? h->hx : h->hy;
      double tx, ty;
      if (kind == CEM_TRACTION) {
        tx = (comp_mask & 1) ? a0 : 0.0;
        ty = (comp_mask & 2) ? a0 : 0.0;
      } else {
        tx = -a0 * ox;
        ty = -a0 * oy;
      }
      double half = 0.5 * L;
      edge_nodes_host(h, g, n1, n2);
      h->Fx[n1] = h->Fx[n1] + half * tx; h->Fy[n1] = h->Fy[n1] + half * ty;
      h->Fx[n2] = h->Fx[n2] + half * tx; h->Fy[n2] = h->Fy[n2] + half * ty;
      h->nflag[n1] |= NF_LOADED;
      h->nflag[n2] |= NF_LOADED;
    }
    h->neu_set = true; h->neu_law = law; h->neu_t0 = t0; h->neu_tau = tau;
  } else if (kind == CEM_VELOCITY) {
    if (h->dir_set && (h->dir_law != law || h->dir_t0 != t0 || h->dir_tau != tau))
      return fail(h, CEM_ERR_ARG, "all Dirichlet loads share one time law");
    if ((comp_mask & 3) == 0) return fail(h, CEM_ERR_ARG, "empty component mask");
    for (int q = 0; q < n_items; ++q)
      if (items[q] < 0 || items[q] >= nn) return fail(h, CEM_ERR_ARG, "bad node %d", items[q]);
    for (int q = 0; q < n_items; ++q) {
      int N = items[q];
      if (comp_mask & 1) { h->nflag[N] |= NF_DIRX; h->Vx[N] = a0; }
      if (comp_mask & 2) { h->nflag[N] |= NF_DIRY; h->Vy[N] = a0; }
    }
    h->dir_set = true; h->dir_law = law; h->dir_t0 = t0; h->dir_tau = tau;
  } else {
    return fail(h, CEM_ERR_ARG, "bad load kind");
  }
  CUDA_TRY(h, cudaSetDevice(h->device));
  return upload_loads(h);
}

cem_status cem_set_fields(cem_handle *h, int which, const void *data, long n_bytes, int on_device) {
  if (!h || !data) return CEM_ERR_ARG;
  if (h->tri) {
    std::string e;
    return tri_rc(h, tri_set_fields(h->tri, which, data, n_bytes, on_device, e), e);
  }
  if (h->batch || h->in_batch) return fail(h, CEM_ERR_STATE, "not valid on a batch or its members");
  if (h->step != 0) return fail(h, CEM_ERR_STATE, "fields can only be set before the first step");
  if (which != CEM_FIELD_U && which != CEM_FIELD_V) return fail(h, CEM_ERR_ARG, "field not settable");
  CUDA_TRY(h, cudaSetDevice(h->device));
  CUDA_TRY(h, cudaMemcpyAsync(h->h_cnt, h->d.cnt, sizeof(Counters), cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  long n = h->d.g.nn + h->h_cnt->n_ph;
  if (n_bytes != 16 * n) return fail(h, CEM_ERR_ARG, "expected %ld bytes", 16 * n);
  cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const DevState &d = h->d;
  if (d.precision == CEM_FP64) {
    double *dx = which == CEM_FIELD_U ? d.ux[h->cur] : d.vx;
    double *dy = which == CEM_FIELD_U ? d.uy[h->cur] : d.vy;
    CUDA_TRY(h, cudaMemcpyAsync(dx, data, n * 8, kind, h->st));
    CUDA_TRY(h, cudaMemcpyAsync(dy, (const char *)data + n * 8, n * 8, kind, h->st));
  } else {
    double *tmp = (double *)scratch(h, (size_t)n * 16);
    if (!tmp) return fail(h, CEM_ERR_CUDA, "temporary allocation failed");
    CUDA_TRY(h, cudaMemcpyAsync(tmp, data, n * 16, kind, h->st));
    if (which == CEM_FIELD_U)
      CUDA_TRY(h, launch_fp64_to_fp32(d, h->cur, tmp, tmp + n, nullptr, nullptr, (int)n, h->st));
    else
      CUDA_TRY(h, launch_fp64_to_fp32(d, h->cur, nullptr, nullptr, tmp, tmp + n, (int)n, h->st));
  }
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  return CEM_OK;
}

// Enqueues n steps of a mesh handle on its stream (graph replays) without
// waiting for them; the load-factor staging is rewritten only after the
// copies that read it have finished.
cem_status enqueue_steps(cem_handle *h, int n) {
  CUDA_TRY(h, cudaSetDevice(h->device));
  cem_status rs = ensure_march_rows(h);
  if (rs != CEM_OK) return rs;
  const DevState &d = h->d;
  int done = 0;
  while (done < n) {
    cem_status rc;
    if (h->step < h->lam_lo || h->step >= h->lam_lo + h->lam_n) {
      // a fresh table of load factors (the pinned staging is rewritten only
      // after the copies that read it have finished)
      CUDA_TRY(h, cudaStreamSynchronize(h->st));
      rc = upload_load_factors(h, d.lam_cap);
      if (rc != CEM_OK) return rc;
    }
    const int chunk = (int)std::min((long)(n - done), h->lam_lo + h->lam_n - h->step);
    for (int q = 0; q < chunk;) {
      const int gm = group_mask(h->step, h->energy_every);
      if (h->step > 0 && chunk - q >= kGraphSteps && gm >= 0) {
        const unsigned mask = (unsigned)gm;
        const long kernels = kGraphSteps * kernels_in_step(h, false) +
                             (mask ? kernels_in_step(h, true) - kernels_in_step(h, false) : 0);
        cudaGraphExec_t gx;
        rc = multi_graph_for(h, h->cur, mask, &gx);
        if (rc != CEM_OK) return rc;
        CUDA_TRY(h, cudaGraphLaunch(gx, h->st));
        h->launches += kernels;
        h->step += kGraphSteps;
        q += kGraphSteps;
        continue;
      }
      bool energy = h->energy_every > 0 && (h->step % h->energy_every) == 0;
      if (h->step == 0) {
        CUDA_TRY(h, enqueue_step(h, h->cur, true, energy));
      } else {
        cudaGraphExec_t gx;
        rc = graph_for(h, h->cur, energy ? 1 : 0, &gx);
        if (rc != CEM_OK) return rc;
        CUDA_TRY(h, cudaGraphLaunch(gx, h->st));
      }
      h->launches += kernels_in_step(h, energy);
      h->cur ^= 1;
      h->step += 1;
      ++q;
    }
    done += chunk;
  }
  return CEM_OK;
}

// The status of the oldest pending cem_step_async call, after waiting for it:
// every step's status word in the ring (a call of 1 .. kStatusRing / 2
// steps; the last one is the call's status), else the word copied after
// the call.
cem_status async_collect(cem_handle *h) {
  const int slot = h->async_next ^ 1;
  int first = (h->async_pending & (1u << h->async_next)) ? h->async_next : slot;
  if (!(h->async_pending & (1u << first))) return CEM_OK;
  CUDA_TRY(h, cudaEventSynchronize(h->async_ev[first]));
  h->async_pending &= ~(1u << first);
  for (int q = 0; q < h->async_steps[first]; ++q) {
    const long taken = h->async_from[first] + q + 1;  // steps taken after step q of the call
    const Counters c = h->h_ring[taken % kStatusRing];
    if (c.step != (int)taken)
      return fail(h, CEM_ERR_CUDA, "status word of step %ld missing from the ring", taken - 1);
    cem_status rc = check_counters(h, c);
    if (rc != CEM_OK) return rc;
  }
  return h->async_steps[first] > 0 ? CEM_OK : check_counters(h, h->h_async[first]);
}

// waits for every pending cem_step_async call; the first error
cem_status async_drain(cem_handle *h) {
  cem_status rc = CEM_OK;
  while (h->async_pending) {
    cem_status r = async_collect(h);
    if (rc == CEM_OK) rc = r;
  }
  return rc;
}

cem_status step_checks(cem_handle *h, int n) {
  if (h->in_batch) return fail(h, CEM_ERR_STATE, "a member of a batch is stepped by the batch");
  if (!h->material) return fail(h, CEM_ERR_STATE, "cem_set_material must come first");
  if (n < 0) return fail(h, CEM_ERR_ARG, "negative step count");
  return CEM_OK;
}

cem_status cem_step(cem_handle *h, int n) {
  if (!h) return CEM_ERR_ARG;
  if (h->tri) {
    std::string e;
    return tri_rc(h, tri_step(h->tri, n, e), e);
  }
  if (h->batch) return batch_step(h, n);
  cem_status rc = step_checks(h, n);
  if (rc != CEM_OK) return rc;
  rc = async_drain(h);
  if (rc != CEM_OK) return rc;
  if (n == 0) return CEM_OK;
  rc = enqueue_steps(h, n);
  if (rc != CEM_OK) return rc;
  // one read-back of the status word (non-finite velocities and capacity
  // overflows are flagged by the kernels themselves)
  return sync_status(h);
}

cem_status cem_step_async(cem_handle *h, int n) {
  if (!h) return CEM_ERR_ARG;
  if (h->tri || h->batch) return fail(h, CEM_ERR_STATE, "cem_step_async steps a structured mesh handle");
  cem_status rc = step_checks(h, n);
  if (rc != CEM_OK) return rc;
  CUDA_TRY(h, cudaSetDevice(h->device));
  if (!h->h_async) {
    CUDA_TRY(h, cudaHostAlloc((void **)&h->h_async, 2 * sizeof(Counters), cudaHostAllocMapped));
    CUDA_TRY(h, cudaHostGetDevicePointer((void **)&h->d_async, h->h_async, 0));
    CUDA_TRY(h, cudaHostAlloc((void **)&h->h_ring, kStatusRing * sizeof(Counters),
                              cudaHostAllocMapped));
    CUDA_TRY(h, cudaHostGetDevicePointer((void **)&h->d_ring, h->h_ring, 0));
    for (auto &ev : h->async_ev) CUDA_TRY(h, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  }
  // a slot still pending from two calls ago is collected first
  if (h->async_pending & (1u << h->async_next)) {
    rc = async_collect(h);
    if (rc != CEM_OK) return rc;
  }
  const int slot = h->async_next;
  // every step writes its status word when the call is short enough that
  // the next call cannot overwrite them before they are read
  h->async_from[slot] = h->step;
  h->async_steps[slot] = n <= kStatusRing / 2 ? n : 0;
  if (n > 0) {
    h->ring_on = n <= kStatusRing / 2;
    rc = enqueue_steps(h, n);
    h->ring_on = false;
    if (rc != CEM_OK) return rc;
  }
  if (h->async_steps[slot] == 0) {
    // no per-step words: the status word after the call
    CUDA_TRY(h, launch_status_copy(h->d.cnt, h->d_async + slot, h->st));
    h->launches += 1;
  }
  CUDA_TRY(h, cudaEventRecord(h->async_ev[slot], h->st));
  h->async_pending |= 1u << slot;
  h->async_next ^= 1;
  // the previous call's status, while this call's steps run
  if (h->async_pending & (1u << h->async_next)) return async_collect(h);
  return CEM_OK;
}

cem_status cem_sync(cem_handle *h) {
  if (!h) return CEM_ERR_ARG;
  if (h->tri || h->batch) return CEM_OK;
  CUDA_TRY(h, cudaSetDevice(h->device));
  return async_drain(h);
}

cem_status cem_profile_steps(cem_handle *h, int n, double *ms) {
  if (!h || !ms) return CEM_ERR_ARG;
  TRI_NOT_AVAILABLE(h);
  if (h->batch || h->in_batch) return fail(h, CEM_ERR_STATE, "not valid on a batch or its members");
  if (!h->material) return fail(h, CEM_ERR_STATE, "cem_set_material must come first");
  if (n < 1 || n > h->d.lam_cap) return fail(h, CEM_ERR_ARG, "1 <= n <= %d", h->d.lam_cap);
  CUDA_TRY(h, cudaSetDevice(h->device));
  for (int q = 0; q < 9; ++q) ms[q] = 0.0;
  cem_status rc = ensure_march_rows(h);
  if (rc != CEM_OK) return rc;
  rc = upload_load_factors(h, n);
  if (rc != CEM_OK) return rc;
  const int M = 9;  // events per step: start + 8 marks
  std::vector<cudaEvent_t> ev((size_t)n * M);
  for (auto &e : ev) CUDA_TRY(h, cudaEventCreate(&e));
  long kernels = 0;
  cudaError_t err = cudaSuccess;
  for (int q = 0; q < n && err == cudaSuccess; ++q) {
    bool energy = h->energy_every > 0 && (h->step % h->energy_every) == 0;
    cudaEventRecord(ev[(size_t)q * M], h->st);
    err = enqueue_step(h, h->cur, h->step == 0, energy, &ev[(size_t)q * M + 1]);
    kernels += kernels_in_step(h, energy);
    h->cur ^= 1;
    h->step += 1;
  }
  cudaError_t es = cudaStreamSynchronize(h->st);
  if (err == cudaSuccess && es == cudaSuccess) {
    float t;
    cudaEventElapsedTime(&t, ev[0], ev[(size_t)(n - 1) * M + 8]);
    ms[0] = t;
    for (int q = 0; q < n; ++q) {
      cudaEvent_t *e = &ev[(size_t)q * M];
      float a, b, c, dd, f, g, k, w;
      cudaEventElapsedTime(&a, e[0], e[1]);  // energy prologue
      cudaEventElapsedTime(&b, e[1], e[2]);  // pieces
      cudaEventElapsedTime(&c, e[2], e[3]);  // tile update
      cudaEventElapsedTime(&dd, e[3], e[4]); // phantoms
      cudaEventElapsedTime(&f, e[4], e[5]);  // evaluation
      cudaEventElapsedTime(&g, e[5], e[6]);  // energy epilogue
      cudaEventElapsedTime(&k, e[6], e[7]);  // tracking selection
      cudaEventElapsedTime(&w, e[7], e[8]);  // split writes
      ms[1] += b; ms[2] += c; ms[3] += dd; ms[4] += f; ms[5] += k; ms[6] += a + g; ms[8] += w;
    }
  }
  for (auto &e : ev) cudaEventDestroy(e);
  if (err != cudaSuccess) return fail(h, CEM_ERR_CUDA, "profiled step: %s", cudaGetErrorString(err));
  if (es != cudaSuccess) return fail(h, CEM_ERR_CUDA, "profiled step sync: %s", cudaGetErrorString(es));
  ms[7] = (double)kernels;
  h->launches += kernels;
  return sync_status(h);
}

cem_status cem_get_counts(cem_handle *h, cem_counts *out) {
  if (!h || !out) return CEM_ERR_ARG;
  if (h->tri) {
    tri_counts(h->tri, out);
    return CEM_OK;
  }
  if (h->batch) return batch_counts(h, out);
  CUDA_TRY(h, cudaSetDevice(h->device));
  CUDA_TRY(h, cudaMemcpyAsync(h->h_cnt, h->d.cnt, sizeof(Counters), cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  const Counters c = *h->h_cnt;
  out->n_nodes = h->d.g.nn;
  out->n_phantoms = c.n_ph;
  out->n_elems = h->d.g.ne;
  long act = 0;
  for (uint8_t a : h->active) act += a;
  out->n_active = act;
  out->n_cracked = c.n_ck;
  out->n_energy = c.n_rec;
  out->step = c.step;
  out->dt = h->d.mat.dt;
  out->t = (double)c.step * h->d.mat.dt;
  out->kernel_launches = h->launches;
  out->last_proposals = c.n_prop_last;
  out->last_winners = c.n_win_last;
  out->n_surface = 0;
  out->n_tips = 0;
  if (c.n_S > 0) {
    int *tmp = (int *)scratch(h, (size_t)c.n_S * 12);
    if (!tmp) return fail(h, CEM_ERR_CUDA, "temporary allocation failed");
    CUDA_TRY(h, launch_surface_info(h->d, tmp, h->st));
    std::vector<int> v((size_t)c.n_S * 3);
    CUDA_TRY(h, cudaMemcpyAsync(v.data(), tmp, v.size() * 4, cudaMemcpyDeviceToHost, h->st));
    CUDA_TRY(h, cudaStreamSynchronize(h->st));
    for (int i = 0; i < c.n_S; ++i)
      if (v[3 * i] >= 0) { out->n_surface++; out->n_tips += v[3 * i + 2]; }
  }
  return CEM_OK;
}

cem_status cem_get_fields(cem_handle *h, int which, void *out, long n_bytes, int on_device) {
  if (!h || !out) return CEM_ERR_ARG;
  if (h->tri) {
    std::string e;
    return tri_rc(h, tri_get_fields(h->tri, which, out, n_bytes, on_device, e), e);
  }
  if (h->batch) return fail(h, CEM_ERR_STATE, "batch handle: query its members");
  CUDA_TRY(h, cudaSetDevice(h->device));
  CUDA_TRY(h, cudaMemcpyAsync(h->h_cnt, h->d.cnt, sizeof(Counters), cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  const DevState &d = h->d;
  long n = d.g.nn + h->h_cnt->n_ph;
  cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  long need;
  switch (which) {
    case CEM_FIELD_U:
    case CEM_FIELD_V: need = 16 * n; break;
    case CEM_FIELD_MASS: need = 8 * n; break;
    case CEM_FIELD_STATE: need = d.g.ne; break;
    case CEM_FIELD_ENERGY: need = 56L * h->h_cnt->n_rec; break;
    case CEM_FIELD_GC: need = 4L * d.g.ne; break;
    case CEM_FIELD_SIGMA: need = 24L * d.g.ne; break;
    case CEM_FIELD_SIGMA1: need = 8L * d.g.ne; break;
    default: return fail(h, CEM_ERR_ARG, "unknown field %d", which);
  }
  if (n_bytes < need) return fail(h, CEM_ERR_ARG, "buffer too small: need %ld bytes", need);
  char *o = (char *)out;
  if (which == CEM_FIELD_U || which == CEM_FIELD_V) {
    if (d.precision == CEM_FP64) {
      const double *sx = which == CEM_FIELD_U ? d.ux[h->cur] : d.vx;
      const double *sy = which == CEM_FIELD_U ? d.uy[h->cur] : d.vy;
      CUDA_TRY(h, cudaMemcpyAsync(o, sx, n * 8, kind, h->st));
      CUDA_TRY(h, cudaMemcpyAsync(o + n * 8, sy, n * 8, kind, h->st));
    } else {
      double *tmp = (double *)scratch(h, (size_t)n * 16);
      if (!tmp) return fail(h, CEM_ERR_CUDA, "temporary allocation failed");
      if (which == CEM_FIELD_U)
        CUDA_TRY(h, launch_fp32_to_fp64(d, h->cur, tmp, tmp + n, nullptr, nullptr, (int)n, h->st));
      else
        CUDA_TRY(h, launch_fp32_to_fp64(d, h->cur, nullptr, nullptr, tmp, tmp + n, (int)n, h->st));
      CUDA_TRY(h, cudaMemcpyAsync(o, tmp, n * 16, kind, h->st));
    }
  } else if (which == CEM_FIELD_MASS) {
    CUDA_TRY(h, cudaMemcpyAsync(o, d.m, n * 8, kind, h->st));
  } else if (which == CEM_FIELD_STATE) {
    CUDA_TRY(h, cudaMemcpyAsync(o, d.estate, d.g.ne, kind, h->st));
  } else if (which == CEM_FIELD_ENERGY) {
    if (need) CUDA_TRY(h, cudaMemcpyAsync(o, d.erec, need, kind, h->st));
  } else if (which == CEM_FIELD_SIGMA || which == CEM_FIELD_SIGMA1) {
    double *tmp = (double *)scratch(h, (size_t)d.g.ne * 32);
    if (!tmp) return fail(h, CEM_ERR_CUDA, "temporary allocation failed");
    CUDA_TRY(h, launch_element_stress(d, h->cur, tmp, h->st));
    const double *src = which == CEM_FIELD_SIGMA ? tmp : tmp + 3 * (size_t)d.g.ne;
    CUDA_TRY(h, cudaMemcpyAsync(o, src, need, kind, h->st));
  } else {
    CUDA_TRY(h, cudaMemcpyAsync(o, d.gc, need, kind, h->st));
  }
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  return CEM_OK;
}

// ------------------------------------------------------------- checkpoint
// The state blob: a header, the counters, then every array that evolves from
// step to step, each cut to the entries in use, in a fixed order.  Arrays
// that a step recomputes before it reads them (piece forces, proposals,
// plans, energy partials) are not saved.
namespace {

constexpr unsigned kBlobMagic = 0x53454d43u;  // "CEMS"
constexpr int kBlobVersion = 1;

struct BlobHeader {
  unsigned magic;
  int version, precision, nx, ny, nn, ne, ned;
  int n_ph, n_ck, n_S, n_rec;
  long step;
  double dt;
  int pad[6];
};

struct BlobPart {
  void *dev;
  size_t bytes;
};

// the arrays of the blob, in order, sized by the counts c
std::vector<BlobPart> blob_parts(const cem_handle *h, const Counters &c) {
  const DevState &d = h->d;
  const size_t N = (size_t)d.g.nn + c.n_ph, ne = d.g.ne, nck = c.n_ck, nph = c.n_ph;
  std::vector<BlobPart> p;
  if (d.precision == CEM_FP64) {
    p.push_back({d.ux[h->cur], N * 8});
    p.push_back({d.uy[h->cur], N * 8});
    p.push_back({d.vx, N * 8});
    p.push_back({d.vy, N * 8});
  } else {
    p.push_back({d.u4[h->cur], N * 16});
    p.push_back({d.v2, N * 8});
    p.push_back({d.minvf, N * 4});
  }
  p.push_back({d.m, N * 8});
  p.push_back({d.minv, N * 8});
  p.push_back({d.Wn, N * 8});
  p.push_back({d.Wd, N * 8});
  p.push_back({d.estate, ne});
  p.push_back({d.crack_of, ne * 4});
  p.push_back({d.ck_elem, nck * 4});
  p.push_back({d.ck_info, nck * 4});
  p.push_back({d.ck_node, nck * 32});
  p.push_back({d.ck_Ap, nck * 16});
  p.push_back({d.ck_ud, nck * 8});
  p.push_back({d.ck_step, nck * 4});
  p.push_back({d.ph_owner, nph * 4});
  p.push_back({d.ph_creator, nph * 4});
  p.push_back({d.ph_nuser, nph * 4});
  p.push_back({d.ph_users, nph * 16});
  p.push_back({d.ph_upf, nph * 16});
  p.push_back({d.ph_uap, nph * 32});
  p.push_back({d.S, (size_t)c.n_S * 4});
  p.push_back({d.S_info, (size_t)c.n_S * 4});
  p.push_back({d.S_G, (size_t)c.n_S * 8});
  p.push_back({d.spos, (size_t)d.g.ned * 4});
  p.push_back({d.erec, (size_t)c.n_rec * 56});
  return p;
}

size_t blob_bytes(const std::vector<BlobPart> &parts) {
  size_t b = sizeof(BlobHeader) + sizeof(Counters);
  for (const auto &q : parts) b += q.bytes;
  return b;
}

cem_status blob_usable(cem_handle *h) {
  if (h->batch || h->in_batch) return fail(h, CEM_ERR_STATE, "not valid on a batch or its members");
  if (!h->material) return fail(h, CEM_ERR_STATE, "cem_set_material must come first");
  return CEM_OK;
}

}  // namespace

cem_status cem_state_size(cem_handle *h, long *n_bytes) {
  if (!h || !n_bytes) return CEM_ERR_ARG;
  TRI_NOT_AVAILABLE(h);
  cem_status rc = blob_usable(h);
  if (rc != CEM_OK) return rc;
  CUDA_TRY(h, cudaSetDevice(h->device));
  rc = sync_status(h);
  if (rc != CEM_OK) return rc;
  *n_bytes = (long)blob_bytes(blob_parts(h, *h->h_cnt));
  return CEM_OK;
}

cem_status cem_save_state(cem_handle *h, void *blob, long n_bytes) {
  if (!h || !blob) return CEM_ERR_ARG;
  TRI_NOT_AVAILABLE(h);
  cem_status rc = blob_usable(h);
  if (rc != CEM_OK) return rc;
  CUDA_TRY(h, cudaSetDevice(h->device));
  rc = sync_status(h);
  if (rc != CEM_OK) return rc;
  const Counters c = *h->h_cnt;
  const auto parts = blob_parts(h, c);
  const size_t need = blob_bytes(parts);
  if ((size_t)n_bytes < need) return fail(h, CEM_ERR_ARG, "blob needs %zu bytes", need);
  BlobHeader hd{};
  hd.magic = kBlobMagic;
  hd.version = kBlobVersion;
  hd.precision = h->d.precision;
  hd.nx = h->d.g.nx;
  hd.ny = h->d.g.ny;
  hd.nn = h->d.g.nn;
  hd.ne = h->d.g.ne;
  hd.ned = h->d.g.ned;
  hd.n_ph = c.n_ph;
  hd.n_ck = c.n_ck;
  hd.n_S = c.n_S;
  hd.n_rec = c.n_rec;
  hd.step = h->step;
  hd.dt = h->d.mat.dt;
  char *o = static_cast<char *>(blob);
  memcpy(o, &hd, sizeof hd);
  memcpy(o + sizeof hd, &c, sizeof c);
  size_t off = sizeof hd + sizeof c;
  for (const auto &q : parts) {
    if (q.bytes) CUDA_TRY(h, cudaMemcpyAsync(o + off, q.dev, q.bytes, cudaMemcpyDeviceToHost, h->st));
    off += q.bytes;
  }
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  return CEM_OK;
}

cem_status cem_load_state(cem_handle *h, const void *blob, long n_bytes) {
  if (!h || !blob) return CEM_ERR_ARG;
  TRI_NOT_AVAILABLE(h);
  cem_status rc = blob_usable(h);
  if (rc != CEM_OK) return rc;
  if ((size_t)n_bytes < sizeof(BlobHeader) + sizeof(Counters))
    return fail(h, CEM_ERR_ARG, "blob too short");
  BlobHeader hd;
  Counters c;
  const char *in = static_cast<const char *>(blob);
  memcpy(&hd, in, sizeof hd);
  memcpy(&c, in + sizeof hd, sizeof c);
  const DevState &d = h->d;
  if (hd.magic != kBlobMagic || hd.version != kBlobVersion)
    return fail(h, CEM_ERR_ARG, "not a state blob of this library version");
  if (hd.precision != d.precision || hd.nx != d.g.nx || hd.ny != d.g.ny || hd.nn != d.g.nn ||
      hd.ne != d.g.ne || hd.ned != d.g.ned)
    return fail(h, CEM_ERR_ARG, "blob of another mesh or precision");
  if (hd.dt != d.mat.dt) return fail(h, CEM_ERR_ARG, "blob of another time step (material)");
  if (c.n_ph > d.ph_cap || c.n_ck > d.ck_cap || c.n_S > d.list_cap || c.n_rec > d.rec_cap ||
      c.n_ph < 0 || c.n_ck < 0 || c.n_S < 0 || c.n_rec < 0 || hd.step < 0)
    return fail(h, CEM_ERR_CAPACITY, "the blob's phantoms, splits, list or records exceed "
                                     "this handle's capacities");
  const auto parts = blob_parts(h, c);
  if ((size_t)n_bytes < blob_bytes(parts)) return fail(h, CEM_ERR_ARG, "blob truncated");
  CUDA_TRY(h, cudaSetDevice(h->device));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  size_t off = sizeof hd + sizeof c;
  for (const auto &q : parts) {
    if (q.bytes) CUDA_TRY(h, cudaMemcpyAsync(q.dev, in + off, q.bytes, cudaMemcpyHostToDevice, h->st));
    off += q.bytes;
  }
  // counters of the saved step; the transient ones (plans of a step in
  // flight) start clear, and the load-factor table is rebuilt at the next step
  Counters k = c;
  k.n_prop = 0;
  k.pend_nwin = 0;
  k.lam_base = (int)hd.step;
  *h->h_cnt = k;
  CUDA_TRY(h, cudaMemcpyAsync(d.cnt, h->h_cnt, sizeof(Counters), cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  h->step = hd.step;
  h->lam_lo = 0;
  h->lam_n = 0;
  h->mrow_stale = true;
  return check_status(h);
}

cem_status cem_get_fragments(cem_handle *h, int *n_fragments, int *piece_fragment, long cap) {
  if (!h || !n_fragments) return CEM_ERR_ARG;
  TRI_NOT_AVAILABLE(h);
  if (h->batch) return fail(h, CEM_ERR_STATE, "batch handle: query its members");
  CUDA_TRY(h, cudaSetDevice(h->device));
  cem_status rc = sync_status(h);
  if (rc != CEM_OK) return rc;
  const DevState &d = h->d;
  const long nq = 2L * d.g.ne;
  if (piece_fragment && cap < nq) return fail(h, CEM_ERR_ARG, "need room for %ld pieces", nq);
  const int n_nodes = d.g.nn + h->h_cnt->n_ph;
  const size_t sb = fragments_scratch_bytes(d, n_nodes);
  char *tmp = (char *)scratch(h, sb + (size_t)nq * 4 + 256);
  if (!tmp) return fail(h, CEM_ERR_CUDA, "temporary allocation failed");
  int *labels = reinterpret_cast<int *>(tmp + ((sb + 255) & ~(size_t)255));
  int *count = reinterpret_cast<int *>(tmp) + sb / 4 - 1;
  CUDA_TRY(h, launch_fragments(d, n_nodes, tmp, labels, count, h->st));
  int c = 0;
  CUDA_TRY(h, cudaMemcpyAsync(&c, count, 4, cudaMemcpyDeviceToHost, h->st));
  if (piece_fragment)
    CUDA_TRY(h, cudaMemcpyAsync(piece_fragment, labels, (size_t)nq * 4, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  *n_fragments = c;
  return CEM_OK;
}

cem_status cem_get_cracks(cem_handle *h, cem_crack *out, int cap, int *n_out) {
  if (!h || !n_out) return CEM_ERR_ARG;
  TRI_NOT_AVAILABLE(h);
  if (h->batch) return fail(h, CEM_ERR_STATE, "batch handle: query its members");
  CUDA_TRY(h, cudaSetDevice(h->device));
  CUDA_TRY(h, cudaMemcpyAsync(h->h_cnt, h->d.cnt, sizeof(Counters), cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  int n = h->h_cnt->n_ck;
  *n_out = n;
  if (!out || n == 0) return CEM_OK;
  if (cap < n) return fail(h, CEM_ERR_ARG, "need room for %d cracks", n);
  const DevState &d = h->d;
  std::vector<int> el(n), info(n), nodes((size_t)n * 8), stp(n);
  std::vector<double> Ap((size_t)n * 2), ud(n);
  CUDA_TRY(h, cudaMemcpyAsync(el.data(), d.ck_elem, n * 4, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(info.data(), d.ck_info, n * 4, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(nodes.data(), d.ck_node, n * 32, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(stp.data(), d.ck_step, n * 4, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(Ap.data(), d.ck_Ap, n * 16, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(ud.data(), d.ck_ud, n * 8, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  std::vector<int> order(n);
  for (int q = 0; q < n; ++q) order[q] = q;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return el[a] < el[b]; });
  for (int r = 0; r < n; ++r) {
    int q = order[r];
    cem_crack &c = out[r];
    c.elem = el[q];
    c.ka = info[q] & 3;
    c.kb = (info[q] >> 2) & 3;
    c.step = stp[q];
    for (int p = 0; p < 2; ++p)
      for (int a = 0; a < 4; ++a) c.node[p][a] = nodes[(size_t)q * 8 + p * 4 + a];
    c.Ap[0] = Ap[2 * q];
    c.Ap[1] = Ap[2 * q + 1];
    c.ud = ud[q];
  }
  return CEM_OK;
}

cem_status cem_get_phantoms(cem_handle *h, cem_phantom *out, int cap, int *n_out) {
  if (!h || !n_out) return CEM_ERR_ARG;
  TRI_NOT_AVAILABLE(h);
  if (h->batch) return fail(h, CEM_ERR_STATE, "batch handle: query its members");
  CUDA_TRY(h, cudaSetDevice(h->device));
  CUDA_TRY(h, cudaMemcpyAsync(h->h_cnt, h->d.cnt, sizeof(Counters), cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  int n = h->h_cnt->n_ph;
  *n_out = n;
  if (!out || n == 0) return CEM_OK;
  if (cap < n) return fail(h, CEM_ERR_ARG, "need room for %d phantoms", n);
  const DevState &d = h->d;
  std::vector<int> own(n), cr(n), nu(n), us((size_t)n * 4);
  CUDA_TRY(h, cudaMemcpyAsync(own.data(), d.ph_owner, n * 4, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(cr.data(), d.ph_creator, n * 4, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(nu.data(), d.ph_nuser, n * 4, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(us.data(), d.ph_users, n * 16, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  for (int q = 0; q < n; ++q) {
    cem_phantom &p = out[q];
    p.id = d.g.nn + q;
    p.owner = own[q];
    p.creator_elem = cr[q] >> 2;
    p.creator_local = cr[q] & 3;
    p.n_users = nu[q];
    for (int u = 0; u < 4; ++u) {
      int code = us[(size_t)q * 4 + u];
      bool used = u < nu[q];
      p.users[u][0] = used ? code >> 3 : -1;
      p.users[u][1] = used ? (code >> 2) & 1 : -1;
      p.users[u][2] = used ? code & 3 : -1;
    }
  }
  return CEM_OK;
}

static cem_status surface_rows(cem_handle *h, std::vector<int> &rows) {
  CUDA_TRY(h, cudaSetDevice(h->device));
  CUDA_TRY(h, cudaMemcpyAsync(h->h_cnt, h->d.cnt, sizeof(Counters), cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  int n = h->h_cnt->n_S;
  rows.clear();
  if (n == 0) return CEM_OK;
  int *tmp = (int *)scratch(h, (size_t)n * 12);
  if (!tmp) return fail(h, CEM_ERR_CUDA, "temporary allocation failed");
  CUDA_TRY(h, launch_surface_info(h->d, tmp, h->st));
  std::vector<int> v((size_t)n * 3);
  CUDA_TRY(h, cudaMemcpyAsync(v.data(), tmp, v.size() * 4, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  std::vector<int> idx;
  for (int i = 0; i < n; ++i)
    if (v[3 * i] >= 0) idx.push_back(i);
  std::sort(idx.begin(), idx.end(), [&](int a, int b) { return v[3 * a] < v[3 * b]; });
  for (int i : idx) rows.insert(rows.end(), {v[3 * i], v[3 * i + 1], v[3 * i + 2], i});
  return CEM_OK;
}

cem_status cem_get_surface(cem_handle *h, int *edge, int *ahead, int *is_tip, int cap, int *n_out) {
  if (!h || !n_out) return CEM_ERR_ARG;
  TRI_NOT_AVAILABLE(h);
  if (h->batch) return fail(h, CEM_ERR_STATE, "batch handle: query its members");
  std::vector<int> rows;
  cem_status rc = surface_rows(h, rows);
  if (rc != CEM_OK) return rc;
  int n = (int)(rows.size() / 4);
  *n_out = n;
  if (n > cap && (edge || ahead || is_tip)) return fail(h, CEM_ERR_ARG, "need room for %d points", n);
  for (int q = 0; q < n && q < cap; ++q) {
    if (edge) edge[q] = rows[4 * q];
    if (ahead) ahead[q] = rows[4 * q + 1] >> 2;
    if (is_tip) is_tip[q] = rows[4 * q + 2];
  }
  return CEM_OK;
}

cem_status cem_get_crack_tips(cem_handle *h, cem_tip *out, int cap, int *n_out) {
  if (!h || !n_out) return CEM_ERR_ARG;
  TRI_NOT_AVAILABLE(h);
  if (h->batch) return fail(h, CEM_ERR_STATE, "batch handle: query its members");
  std::vector<int> rows;
  cem_status rc = surface_rows(h, rows);
  if (rc != CEM_OK) return rc;
  const DevState &d = h->d;
  int nS = h->h_cnt->n_S, nck = h->h_cnt->n_ck;
  std::vector<double> SG(nS > 0 ? nS : 1);
  std::vector<int> crack_of((size_t)d.g.ne), stp(nck > 0 ? nck : 1);
  if (nS) CUDA_TRY(h, cudaMemcpyAsync(SG.data(), d.S_G, (size_t)nS * 8, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(crack_of.data(), d.crack_of, crack_of.size() * 4, cudaMemcpyDeviceToHost, h->st));
  if (nck) CUDA_TRY(h, cudaMemcpyAsync(stp.data(), d.ck_step, (size_t)nck * 4, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  int n = 0;
  for (size_t q = 0; q < rows.size(); q += 4) {
    if (!rows[q + 2]) continue;
    if (out && n < cap) {
      int g = rows[q], info = rows[q + 1], e = info >> 2, k0 = info & 3;
      int nh = h->nx * (h->ny + 1), i = e % h->nx, j = e / h->nx;
      int f = k0 == 0 ? e - h->nx : k0 == 1 ? e + 1 : k0 == 2 ? e + h->nx : e - 1;
      cem_tip &t = out[n];
      t.edge_id = g;
      t.ahead_elem = e;
      if (g < nh) {
        int jj = g / h->nx, ii = g % h->nx;
        t.x = (ii + 0.5) * h->hx; t.y = jj * h->hy;
      } else {
        int gg = g - nh, jj = gg / (h->nx + 1), ii = gg % (h->nx + 1);
        t.x = ii * h->hx; t.y = (jj + 0.5) * h->hy;
      }
      (void)i; (void)j;
      t.G_last = SG[rows[q + 3]];
      t.parent = f;
      int c = crack_of[f];
      t.birth_step = c >= 0 ? stp[c] : -1;
    }
    ++n;
  }
  *n_out = n;
  if (out && n > cap) return fail(h, CEM_ERR_ARG, "need room for %d tips", n);
  return CEM_OK;
}

cem_status cem_debug_apply_proposals(cem_handle *h, int n, const int *edge, const int *elem,
                                     const int *k, const double *G) {
  if (!h) return CEM_ERR_ARG;
  TRI_NOT_AVAILABLE(h);
  if (h->batch || h->in_batch) return fail(h, CEM_ERR_STATE, "not valid on a batch or its members");
  if (!h->material) return fail(h, CEM_ERR_STATE, "material first");
  if (n < 0 || n > h->d.prop_cap) return fail(h, CEM_ERR_ARG, "bad proposal count");
  if (n == 0) return CEM_OK;
  std::vector<int> key(n);
  for (int q = 0; q < n; ++q) {
    if (elem[q] < 0 || elem[q] >= h->d.g.ne || k[q] < 0 || k[q] > 3)
      return fail(h, CEM_ERR_ARG, "proposal %d is not a surface point of its element", q);
    int k0 = local_edge_host(h, elem[q], edge[q]);
    if (k0 < 0 || k0 == k[q]) return fail(h, CEM_ERR_ARG, "proposal %d is not a surface point of its element", q);
    key[q] = elem[q] * 4 + k0;
  }
  CUDA_TRY(h, cudaSetDevice(h->device));
  const DevState &d = h->d;
  CUDA_TRY(h, cudaMemcpyAsync(d.pr_key, key.data(), n * 4, cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(d.pr_edge, edge, n * 4, cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(d.pr_k, k, n * 4, cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(d.pr_G, G, n * 8, cudaMemcpyHostToDevice, h->st));
  int zero = 0;
  CUDA_TRY(h, cudaMemcpyAsync(&d.cnt->n_prop, &n, 4, cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(&d.cnt->pad[0], &zero, 4, cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  CUDA_TRY(h, launch_select(d, TRACK_DEBUG, h->st));
  CUDA_TRY(h, launch_apply(d, h->cur, TRACK_DEBUG, h->st));
  cem_status rc = sync_status(h);
  if (rc != CEM_OK) return rc;
  if (h->h_cnt->pad[0]) return fail(h, CEM_ERR_ARG, "a proposal is not a surface point of its element");
  return CEM_OK;
}

}  // extern "C"

// ===================================================================== batch
// A batch steps many independent meshes in lock-step: one launch per kernel
// kind covers every member (work lists of (member, block) items walked by
// persistent grids), one CUDA graph per step.  Members keep their own device
// state and stay queryable; each stops at its own step limit.
struct BatchPlan {
  std::vector<cem_handle *> members;
  std::vector<long> step_end;
  int precision = 0;
  int energy_every = 0;
  long step = 0;           // batch step (equals every active member's step)
  int tile_rows = 16;      // FP32 tile height (8 .. 64 node rows)
  int grid_main = 0;       // persistent grid of the tile update
  int sms = 0;
  BatchDev bd{};
  char *dev = nullptr;     // device block: states, work lists, counters
  size_t dev_bytes = 0;
  cudaGraphExec_t graphs[2] = {nullptr, nullptr};  // [energy]
  std::vector<double> tune_ms;  // autotuner timings, candidate order
  Counters *d_cnts = nullptr;   // [n] gathered counters (device)
  Counters *h_cnts = nullptr;   // [n] pinned read-back
};

namespace {

void batch_drop_graphs(BatchPlan *p) {
  for (auto &g : p->graphs)
    if (g) { cudaGraphExecDestroy(g); g = nullptr; }
}

// Host copies of the members' states and the work lists for the current
// tile height, uploaded into the batch's device block.
cem_status batch_upload(cem_handle *b) {
  BatchPlan *p = b->batch;
  const int n = (int)p->members.size();
  std::vector<DevState> ds((size_t)n);
  std::vector<int4> wm, wp, wph, we;
  std::vector<int> nparts((size_t)n);
  for (int s = 0; s < n; ++s) {
    cem_handle *m = p->members[s];
    if (ensure_march_rows(m) != CEM_OK) return fail(b, CEM_ERR_CUDA, "member %d: row flags", s);
    DevState d = m->d;
    d.step_end = (int)std::min<long>(p->step_end[s], (long)INT_MAX);
    d.cur_xor = m->cur ^ (int)(m->step & 1);
    ds[s] = d;
    int tiles;
    if (p->precision == CEM_FP32_MIXED) {
      // FP32 node update: one item per group of four warp tiles
      const int ng = groups_fp32(d, p->tile_rows);
      for (int q = 0; q < ng; ++q) wm.push_back(make_int4(s, q, 0, ng));
      tiles = tiles_fp32(d, p->tile_rows);
    } else {
      const int gx = (d.g.nx + 1 + 31) / 32, gy = tiles_fp64(d) / gx;
      for (int y = 0; y < gy; ++y)
        for (int x = 0; x < gx; ++x) wm.push_back(make_int4(s, x, y, gx | (gy << 16)));
      tiles = gx * gy;
    }
    // a member's piece and phantom grids are sized for its capacities; in
    // FP32 eight virtual blocks per member walk the live splits and phantoms
    // (its counts, not its capacities, set the work: 78.9 against 102.1 us
    // per step of the 64-specimen batch).  FP64 keeps a solo run's grids, so
    // that its energy partials are grouped, and rounded, as when stepped alone.
    int gph = grid_phantoms(d), gp = grid_pieces(d);
    if (p->precision == CEM_FP32_MIXED) {
      gph = std::min(gph, 8);
      gp = std::min(gp, 8);
    }
    for (int q = 0; q < gp; ++q) wp.push_back(make_int4(s, q, tiles, gp));
    for (int q = 0; q < gph; ++q) wph.push_back(make_int4(s, q, tiles + gp, gph));
    // the evaluation has no energy partials: a few virtual blocks per member
    // walk its list (its length, not its capacity, sets the work)
    const int ge = std::min(grid_eval(d), 8);
    for (int q = 0; q < ge; ++q) we.push_back(make_int4(s, q, 0, ge));
    // FP32 phantom blocks write one energy partial per warp
    nparts[s] = tiles + gp + (p->precision == CEM_FP32_MIXED ? kPhWarps : 1) * gph;
  }
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t o_ds = 0, o_m = al(o_ds + ds.size() * sizeof(DevState));
  const size_t o_p = al(o_m + wm.size() * 16), o_ph = al(o_p + wp.size() * 16);
  const size_t o_e = al(o_ph + wph.size() * 16);
  const size_t o_np = al(o_e + we.size() * 16), o_ctr = al(o_np + nparts.size() * 4);
  const size_t bytes = o_ctr + 256;
  if (bytes > p->dev_bytes) {
    // grows only when a smaller tile height needs longer lists
    p->dev = (char *)dalloc(b, bytes);
    if (!p->dev) return fail(b, CEM_ERR_CUDA, "batch device allocation failed");
    p->dev_bytes = bytes;
  }
  std::vector<char> host(bytes, 0);
  memcpy(host.data() + o_ds, ds.data(), ds.size() * sizeof(DevState));
  memcpy(host.data() + o_m, wm.data(), wm.size() * 16);
  memcpy(host.data() + o_p, wp.data(), wp.size() * 16);
  memcpy(host.data() + o_ph, wph.data(), wph.size() * 16);
  memcpy(host.data() + o_e, we.data(), we.size() * 16);
  memcpy(host.data() + o_np, nparts.data(), nparts.size() * 4);
  int *ctr = (int *)(host.data() + o_ctr);
  ctr[0] = (int)p->step;  // batch step
  ctr[1] = 0;             // arrivals
  CUDA_TRY(b, cudaMemcpyAsync(p->dev, host.data(), bytes, cudaMemcpyHostToDevice, b->st));
  CUDA_TRY(b, cudaStreamSynchronize(b->st));
  BatchDev &bd = p->bd;
  bd.ds = (const DevState *)(p->dev + o_ds);
  bd.n = n;
  bd.bstep = (int *)(p->dev + o_ctr);
  bd.arrive = bd.bstep + 1;
  bd.w_main = (const int4 *)(p->dev + o_m); bd.n_main = (int)wm.size();
  bd.w_pieces = (const int4 *)(p->dev + o_p); bd.n_pieces = (int)wp.size();
  bd.w_ph = (const int4 *)(p->dev + o_ph); bd.n_ph = (int)wph.size();
  bd.w_eval = (const int4 *)(p->dev + o_e); bd.n_eval = (int)we.size();
  bd.nparts = (const int *)(p->dev + o_np);
  batch_drop_graphs(p);
  return CEM_OK;
}

int batch_kernels_in_step(bool energy) { return kStepKernels + 2 + (energy ? 2 : 0); }

cudaError_t batch_enqueue_step(cem_handle *b, bool first, bool energy) {
  BatchPlan *p = b->batch;
  cudaError_t e;
  if (energy && (e = launch_energy_pre_batch(p->bd, b->st)) != cudaSuccess) return e;
  if (p->precision == CEM_FP32_MIXED)
    e = launch_step_fp32_batch(p->bd, first, energy, p->tile_rows, p->grid_main, b->ss);
  else
    e = launch_step_fp64_batch(p->bd, first, energy, p->grid_main, b->ss);
  if (e != cudaSuccess) return e;
  if (energy && (e = launch_energy_post_batch(p->bd, b->st)) != cudaSuccess) return e;
  return launch_apply_batch(p->bd, b->st);
}

cem_status batch_graph(cem_handle *b, int energy, cudaGraphExec_t *out) {
  BatchPlan *p = b->batch;
  if (!p->graphs[energy]) {
    cudaGraph_t g;
    CUDA_TRY(b, cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = batch_enqueue_step(b, false, energy != 0);
    cudaError_t e2 = cudaStreamEndCapture(b->st, &g);
    if (e != cudaSuccess) return fail(b, CEM_ERR_CUDA, "batch capture: %s", cudaGetErrorString(e));
    if (e2 != cudaSuccess) return fail(b, CEM_ERR_CUDA, "batch end capture: %s", cudaGetErrorString(e2));
    cudaError_t e3 = cudaGraphInstantiate(&p->graphs[energy], g,
                                          cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) return fail(b, CEM_ERR_CUDA, "batch instantiate: %s", cudaGetErrorString(e3));
  }
  *out = p->graphs[energy];
  return CEM_OK;
}

// Advances every member that has not reached its limit by n steps (fewer at
// its limit).  ev_t0 / ev_t1, when given, bracket the steps on the stream.
cem_status batch_run(cem_handle *b, int n, cudaEvent_t ev_t0, cudaEvent_t ev_t1) {
  BatchPlan *p = b->batch;
  int lam_cap = INT_MAX;
  for (size_t s = 0; s < p->members.size(); ++s) {
    cem_handle *m = p->members[s];
    if (!m) return fail(b, CEM_ERR_STATE, "member %d was destroyed", (int)s);
    if (m->step != std::min(p->step, p->step_end[s]))
      return fail(b, CEM_ERR_STATE, "member %d is out of step with the batch", (int)s);
    lam_cap = std::min(lam_cap, m->d.lam_cap);
  }
  if (ev_t0) CUDA_TRY(b, cudaEventRecord(ev_t0, b->st));
  int done = 0;
  while (done < n) {
    const int chunk = std::min(n - done, lam_cap);
    // on the batch stream, ahead of the steps that read them, when a
    // member's resident table does not cover the chunk; each member's pinned
    // staging is reused only after the synchronisation below
    for (cem_handle *m : p->members) {
      if (m->step >= m->lam_lo && m->step + chunk <= m->lam_lo + m->lam_n) continue;
      cem_status rc = upload_load_factors(m, lam_cap, b->st);
      if (rc != CEM_OK) return fail(b, rc, "load factors: %s", m->err.c_str());
    }
    for (int q = 0; q < chunk;) {
      // one graph per step: grouping steps as for a single mesh measured
      // slower for the 64-specimen batch (113 us against 106 us per step)
      const bool energy = p->energy_every > 0 && (p->step % p->energy_every) == 0;
      if (p->step == 0) {
        CUDA_TRY(b, batch_enqueue_step(b, true, energy));
      } else {
        cudaGraphExec_t gx;
        cem_status rc = batch_graph(b, energy ? 1 : 0, &gx);
        if (rc != CEM_OK) return rc;
        CUDA_TRY(b, cudaGraphLaunch(gx, b->st));
      }
      b->launches += batch_kernels_in_step(energy);
      p->step += 1;
      ++q;
    }
    if (done + chunk == n && ev_t1) CUDA_TRY(b, cudaEventRecord(ev_t1, b->st));
    CUDA_TRY(b, cudaStreamSynchronize(b->st));
    for (size_t s = 0; s < p->members.size(); ++s) {
      cem_handle *m = p->members[s];
      const long adv = std::max(0L, std::min((long)chunk, p->step_end[s] - m->step));
      m->step += adv;
      m->cur ^= (int)(adv & 1);
    }
    done += chunk;
  }
  return CEM_OK;
}

// One read-back of all members' counters (the kernels flag non-finite
// velocities and capacity overflows in them).
cem_status batch_finish(cem_handle *b) {
  BatchPlan *p = b->batch;
  CUDA_TRY(b, launch_gather_counters(p->bd, p->d_cnts, b->st));
  b->launches += 1;
  const size_t n = p->members.size();
  CUDA_TRY(b, cudaMemcpyAsync(p->h_cnts, p->d_cnts, n * sizeof(Counters), cudaMemcpyDeviceToHost,
                              b->st));
  CUDA_TRY(b, cudaStreamSynchronize(b->st));
  for (size_t s = 0; s < n; ++s) {
    cem_handle *m = p->members[s];
    *m->h_cnt = p->h_cnts[s];
    cem_status rc = check_status(m);
    if (rc != CEM_OK) return fail(b, rc, "member %d: %s", (int)s, m->err.c_str());
  }
  return CEM_OK;
}

cem_status batch_step(cem_handle *b, int n) {
  if (n < 0) return fail(b, CEM_ERR_ARG, "negative step count");
  if (n == 0) return CEM_OK;
  CUDA_TRY(b, cudaSetDevice(b->device));
  cem_status rc = batch_run(b, n, nullptr, nullptr);
  if (rc != CEM_OK) return rc;
  return batch_finish(b);
}

cem_status batch_counts(cem_handle *b, cem_counts *out) {
  BatchPlan *p = b->batch;
  cem_counts sum{};
  for (size_t s = 0; s < p->members.size(); ++s) {
    cem_handle *m = p->members[s];
    if (!m) return fail(b, CEM_ERR_STATE, "member %d was destroyed", (int)s);
    cem_counts c;
    cem_status rc = cem_get_counts(m, &c);
    if (rc != CEM_OK) return fail(b, rc, "member %d: %s", (int)s, m->err.c_str());
    sum.n_nodes += c.n_nodes;
    sum.n_phantoms += c.n_phantoms;
    sum.n_elems += c.n_elems;
    sum.n_active += c.n_active;
    sum.n_cracked += c.n_cracked;
    sum.n_surface += c.n_surface;
    sum.n_tips += c.n_tips;
    sum.n_energy += c.n_energy;
    sum.last_proposals += c.last_proposals;
    sum.last_winners += c.last_winners;
  }
  sum.step = p->step;
  sum.dt = 0.0;
  sum.t = 0.0;
  sum.kernel_launches = b->launches;
  *out = sum;
  return CEM_OK;
}

void batch_release(cem_handle *b) {
  BatchPlan *p = b->batch;
  if (b->st) cudaStreamSynchronize(b->st);
  batch_drop_graphs(p);
  if (p->h_cnts) cudaFreeHost(p->h_cnts);
  for (cem_handle *m : p->members)
    if (m) m->in_batch = nullptr;
  delete p;
  b->batch = nullptr;
}

void batch_detach(cem_handle *member) {
  BatchPlan *p = member->in_batch->batch;
  if (p)
    for (auto &m : p->members)
      if (m == member) m = nullptr;
  member->in_batch = nullptr;
}

}  // namespace

cem_status cem_batch_create(cem_handle *const *members, int n, const long *step_end,
                            void *cuda_stream, cem_handle **out) {
  if (!out) return fail(nullptr, CEM_ERR_ARG, "null argument");
  *out = nullptr;
  if (!members || n < 1 || n > (1 << 16)) return fail(nullptr, CEM_ERR_ARG, "1 <= n <= 65536 members");
  for (int s = 0; s < n; ++s) {
    cem_handle *m = members[s];
    if (!m || m->batch) return fail(nullptr, CEM_ERR_ARG, "member %d is not a mesh handle", s);
    if (m->tri) return fail(nullptr, CEM_ERR_STATE, "member %d is a triangle mesh", s);
    if (m->in_batch) return fail(nullptr, CEM_ERR_STATE, "member %d is already in a batch", s);
    if (!m->material) return fail(nullptr, CEM_ERR_STATE, "member %d has no material", s);
    for (int r = 0; r < s; ++r)
      if (members[r] == m) return fail(nullptr, CEM_ERR_ARG, "member %d repeated", s);
    const cem_handle *m0 = members[0];
    if (m->device != m0->device || m->d.precision != m0->d.precision ||
        m->energy_every != m0->energy_every || m->step != m0->step)
      return fail(nullptr, CEM_ERR_ARG,
                  "member %d differs from member 0 in device, precision, energy_every or step", s);
    if (step_end && step_end[s] < m->step)
      return fail(nullptr, CEM_ERR_ARG, "member %d: step limit before its current step", s);
    if (m->d.g.nx + 1 >= (1 << 15) || m->d.g.ny + 1 >= (1 << 15))
      return fail(nullptr, CEM_ERR_ARG, "member %d: batched meshes are limited to 32766 x 32766", s);
  }
  cem_handle *m0 = members[0];
  cem_handle *b = new (std::nothrow) cem_handle();
  if (!b) return fail(nullptr, CEM_ERR_ARG, "out of host memory");
  b->device = m0->device;
  b->alloc = m0->alloc;
  b->free_fn = m0->free_fn;
  b->ctx = m0->ctx;
  b->material = true;
  b->st = (cudaStream_t)cuda_stream;
  cudaError_t ce = cudaSetDevice(b->device);
  if (ce == cudaSuccess && !b->st) {
    ce = cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking);
    b->own_stream = ce == cudaSuccess;
  }
  if (ce == cudaSuccess) ce = create_aux_streams(b->ss);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&b->ss.fork, cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&b->ss.join1, cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&b->ss.join2, cudaEventDisableTiming);
  b->ss.main = b->st;
  int sms = 0;
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  for (int s = 0; s < n && ce == cudaSuccess; ++s) ce = cudaStreamSynchronize(members[s]->st);
  if (ce != cudaSuccess) {
    cem_mesh_destroy(b);
    return fail(nullptr, CEM_ERR_CUDA, "batch set-up: %s", cudaGetErrorString(ce));
  }
  BatchPlan *p = new (std::nothrow) BatchPlan();
  if (!p) {
    cem_mesh_destroy(b);
    return fail(nullptr, CEM_ERR_ARG, "out of host memory");
  }
  b->batch = p;
  p->members.assign(members, members + n);
  p->step_end.resize((size_t)n);
  for (int s = 0; s < n; ++s) p->step_end[s] = step_end ? step_end[s] : (long)INT_MAX;
  p->precision = m0->d.precision;
  p->energy_every = m0->energy_every;
  p->step = m0->step;
  p->sms = sms;
  p->tile_rows = 16;
  p->grid_main = 3 * sms;
  cem_status rc = batch_upload(b);
  if (rc == CEM_OK) {
    p->d_cnts = (Counters *)dalloc(b, (size_t)n * sizeof(Counters));
    if (!p->d_cnts ||
        cudaHostAlloc((void **)&p->h_cnts, (size_t)n * sizeof(Counters), cudaHostAllocDefault) !=
            cudaSuccess)
      rc = fail(b, CEM_ERR_CUDA, "batch counter buffers");
  }
  if (rc != CEM_OK) {
    g_create_error = b->err;
    cem_mesh_destroy(b);
    return rc;
  }
  for (int s = 0; s < n; ++s) members[s]->in_batch = b;
  *out = b;
  return CEM_OK;
}

cem_status cem_batch_set_config(cem_handle *b, int tile_rows, int grid_main) {
  if (!b) return CEM_ERR_ARG;
  TRI_NOT_AVAILABLE(b);
  if (!b->batch) return fail(b, CEM_ERR_STATE, "not a batch handle");
  BatchPlan *p = b->batch;
  if (tile_rows < 8 || tile_rows > 64) return fail(b, CEM_ERR_ARG, "tile_rows must be in 8 .. 64");
  if (grid_main < 1 || grid_main > 64 * p->sms) return fail(b, CEM_ERR_ARG, "1 <= grid_main <= 64 * SMs");
  CUDA_TRY(b, cudaSetDevice(b->device));
  const bool relist = p->precision == CEM_FP32_MIXED && tile_rows != p->tile_rows;
  p->tile_rows = p->precision == CEM_FP32_MIXED ? tile_rows : 16;
  if (grid_main != p->grid_main) batch_drop_graphs(p);
  p->grid_main = grid_main;
  if (relist) return batch_upload(b);
  return CEM_OK;
}

cem_status cem_batch_autotune(cem_handle *b, int steps_per_candidate, int *tile_rows,
                              int *grid_main) {
  if (!b) return CEM_ERR_ARG;
  TRI_NOT_AVAILABLE(b);
  if (!b->batch) return fail(b, CEM_ERR_STATE, "not a batch handle");
  BatchPlan *p = b->batch;
  if (steps_per_candidate < 1) return fail(b, CEM_ERR_ARG, "steps_per_candidate >= 1");
  CUDA_TRY(b, cudaSetDevice(b->device));
  std::vector<std::pair<int, int>> cand;
  const int rows[4] = {16, 8, 32, 64};
  for (int r = 0; r < (p->precision == CEM_FP32_MIXED ? 4 : 1); ++r)
    for (int k = 1; k <= 4; ++k) cand.push_back({rows[r], k * p->sms});
  cudaEvent_t e0, e1;
  CUDA_TRY(b, cudaEventCreate(&e0));
  CUDA_TRY(b, cudaEventCreate(&e1));
  p->tune_ms.assign(cand.size(), 0.0);
  double best = 1e300;
  std::pair<int, int> pick = {p->tile_rows, p->grid_main};
  cem_status rc = CEM_OK;
  for (size_t c = 0; c < cand.size() && rc == CEM_OK; ++c) {
    rc = cem_batch_set_config(b, cand[c].first, cand[c].second);
    if (rc == CEM_OK) rc = batch_run(b, 1, nullptr, nullptr);  // capture, untimed
    if (rc == CEM_OK) rc = batch_run(b, steps_per_candidate, e0, e1);
    if (rc == CEM_OK) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      p->tune_ms[c] = ms;
      if (ms < best) { best = ms; pick = cand[c]; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != CEM_OK) return rc;
  rc = cem_batch_set_config(b, pick.first, pick.second);
  if (rc != CEM_OK) return rc;
  if (tile_rows) *tile_rows = p->tile_rows;
  if (grid_main) *grid_main = p->grid_main;
  return batch_finish(b);
}
