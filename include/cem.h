/*
 * cem.h -- C ABI of the GB300-native explicit MCT-2D-CEM time step.
 *
 * Method: the Multiple Crack-tips Tracking two-dimensional Crack Element Model
 * (arXiv 2509.01827).  One explicit step of a structured bilinear
 * quadrilateral (Q4) mesh is
 *   (1) ES-FEM strain at the edge midpoints, plane stress/strain sigma = D eps,
 *       internal force of intact elements and of split-element pieces
 *       (Sec. 2.1, Eqs. 1, 2, 4, 6);
 *   (2) a deterministic node gather, then the central-difference update with
 *       lumped mass and Neumann / Dirichlet loads (Sec. 2 "explicit
 *       formulation"; load laws of Secs. 4.1, 4.3, 4.4; equivalent nodal forces
 *       of tractions, Sec. 4.3);
 *   (3) multi-tip crack tracking: every free-surface edge point evaluates the
 *       energy release rate G of its candidate paths (Sec. 2.2), applies the
 *       Q4 cracking conditions, and the largest G in its neighbourhood splits
 *       its element (Sec. 3); the device-side surface/tip list grows and
 *       shrinks by stream compaction.
 * All of it runs in this library's own CUDA kernels for sm_103a.
 *
 * Numbering (structured nx * ny mesh, element size hx * hy, unit thickness):
 *   node (i,j), 0<=i<=nx, 0<=j<=ny         id = j*(nx+1) + i, X = (i*hx, j*hy)
 *   element (i,j), 0<=i<nx, 0<=j<ny        id = j*nx + i
 *   element local nodes (counter-clockwise) 0:(i,j) 1:(i+1,j) 2:(i+1,j+1) 3:(i,j+1)
 *   element local edges 0 bottom, 1 right, 2 top, 3 left; edge k joins local
 *   nodes k and (k+1)%4 and its quadrature point is its midpoint
 *   horizontal edge (i,j), nodes (i,j)-(i+1,j), 0<=j<=ny: id = j*nx + i
 *   vertical edge (i,j),   nodes (i,j)-(i,j+1), 0<=j<ny:  id = nx*(ny+1) + j*(nx+1) + i
 *   Real nodes are [0, (nx+1)(ny+1)); phantom nodes of split elements follow.
 *
 * Conventions:
 *   - Every input array is copied during the call; the caller keeps ownership.
 *   - The library owns its device state.  It allocates it with the caller's
 *     allocator callbacks when given (e.g. PyTorch's caching allocator), else
 *     with cudaMallocAsync on the handle's stream.
 *   - Functions return a cem_status; nothing throws across the ABI;
 *     cem_last_error() returns the message of the last failure on a handle.
 *   - A handle is used by one host thread at a time.  All device work goes to
 *     the stream given in the descriptor; with NULL the library creates its
 *     own non-blocking stream (graphs cannot be captured on the legacy
 *     default stream).
 *   - Floating-point state is SI: metres, seconds, pascals, kilograms.
 */
#ifndef CEM_H
#define CEM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cem_handle cem_handle; /* opaque, library-owned */

typedef enum {
  CEM_OK = 0,
  CEM_ERR_ARG = -1,       /* invalid argument (message says which) */
  CEM_ERR_CUDA = -2,      /* a CUDA runtime call failed */
  CEM_ERR_CAPACITY = -3,  /* a phantom/crack/list/winner capacity was exceeded */
  CEM_ERR_NONFINITE = -4, /* a displacement or velocity became NaN or Inf */
  CEM_ERR_TIMEOUT = -5,   /* a bounded device-side wait gave up; the solver has no
                             device-side waits and never returns it (the surrogate
                             kernels of cem_surrogate.h report theirs through
                             cem_sg_timeouts) */
  CEM_ERR_STATE = -6      /* call out of order (e.g. stepping before material) */
} cem_status;

typedef enum { CEM_FP64 = 0, CEM_FP32_MIXED = 1 } cem_precision;

typedef enum { CEM_TRACTION = 0, CEM_PRESSURE = 1, CEM_VELOCITY = 2 } cem_bc_kind;
typedef enum { CEM_LAW_CONST = 0, CEM_LAW_RAMP = 1, CEM_LAW_RAMP_EXP = 2 } cem_law;
typedef enum { CEM_SCOPE_NBHD = 0, CEM_SCOPE_GLOBAL = 1, CEM_SCOPE_TIPS = 2 } cem_scope;
typedef enum { CEM_GAMMA_LITERAL = 0, CEM_GAMMA_RATIO = 1 } cem_gamma_mode;

typedef void *(*cem_alloc_fn)(size_t bytes, void *ctx);
typedef void (*cem_free_fn)(void *ptr, void *ctx);

typedef struct {
  int nx, ny;                        /* elements along x and y, >= 1 */
  double hx, hy;                     /* element size (m), > 0 */
  const unsigned char *elem_active;  /* [nx*ny], 0 = hole; NULL = all active */
  int n_precracks;                   /* split at t = 0, in the given order, */
  const int *precrack;               /* [3*n]: (element, entry edge, exit edge) */
  int phantom_capacity;              /* max phantom nodes; 0 = nx*ny/4 + 4096 */
  int crack_capacity;                /* max split elements; 0 = nx*ny/4 + 4096 */
  int list_capacity;                 /* max surface-list entries; 0 = automatic */
  int precision;                     /* cem_precision */
  double dt_factor;                  /* dt = dt_factor * min(hx,hy) / c_d (0 -> 0.5) */
  double dt;                         /* > 0 overrides dt_factor */
  int energy_every;                  /* record energies every K steps (0 = never) */
  void *cuda_stream;                 /* cudaStream_t, NULL = a stream of the library's own */
  int device;                        /* CUDA device ordinal */
  cem_alloc_fn alloc;                /* optional device allocator */
  cem_free_fn free;                  /* required when alloc is given */
  void *alloc_ctx;
} cem_mesh_desc;

/* Builds the structured mesh and its device state (one bulk host-to-device
 * copy).  Pre-cracks are applied by cem_set_material, which fixes the masses.
 * Errors: CEM_ERR_ARG (sizes, capacities, pre-crack triples), CEM_ERR_CUDA. */
cem_status cem_mesh_create(const cem_mesh_desc *desc, cem_handle **out);

/* Unstructured mesh of constant-strain triangles, the paper's own element
 * (Sec. 2.1): ES-FEM edge strains, the area-weighted average of the two
 * triangles beside an edge (Eqs. 1, 3), and internal forces B_j^T sigma
 * A_j / 3 from every triangle j of every edge (Eq. 5); lumped masses
 * rho A / 3 per node; FP64 or FP32-mixed.  The triangles do not crack on
 * this path.
 * Edges are the distinct node pairs {a, b} of the triangles' sides,
 * numbered in increasing (min(a,b), max(a,b)): cem_set_bc's traction and
 * pressure items are these edge ids (boundary edges only, outward normal
 * from the counter-clockwise triangle), its velocity items node ids.
 * On such a handle cem_set_material (G_c and gamma serve cem_tri_eval_surface;
 * the scope is ignored),
 * cem_set_bc, cem_set_fields (U, V), cem_step, cem_get_fields (U, V, MASS,
 * ENERGY with U_d = 0), cem_get_counts, cem_last_error and cem_mesh_destroy
 * work; every other call returns CEM_ERR_STATE. */
typedef struct {
  int n_nodes, n_elems;              /* >= 3, >= 1 */
  const double *X;                   /* [2*n_nodes]: x, y of node N at X[2N], X[2N+1] (m); copied */
  const int *conn;                   /* [3*n_elems]: nodes of element e at conn[3e..3e+2],
                                        counter-clockwise; copied */
  int precision;                     /* cem_precision: CEM_FP64, or CEM_FP32_MIXED (FP32
                                        element arithmetic, displacement as compensated
                                        float pairs, FP64 energies) */
  double dt_factor;                  /* dt = dt_factor * h_min / c_d (0 -> 0.5), h_min the
                                        smallest altitude 2A / longest side */
  double dt;                         /* > 0 overrides dt_factor */
  int energy_every;                  /* record energies every K steps (0 = never) */
  void *cuda_stream;                 /* cudaStream_t, NULL = a stream of the library's own */
  int device;                        /* CUDA device ordinal */
  cem_alloc_fn alloc;                /* optional device allocator */
  cem_free_fn free;                  /* required when alloc is given */
  void *alloc_ctx;
} cem_tri_mesh_desc;

/* Builds the triangle mesh (geometry, edge list, per-node gather lists) and
 * its device state.  Errors: CEM_ERR_ARG (sizes, node ids, a clockwise or
 * degenerate triangle, an edge of more than two triangles), CEM_ERR_CUDA. */
cem_status cem_tri_mesh_create(const cem_tri_mesh_desc *desc, cem_handle **out);

/* Crack evaluation of constant-strain triangles at n surface points (Sec.
 * 2.2, the CST rules), FP64 from the current displacement (in FP32-mixed
 * mode the float pairs are summed first).  Point q is edge edge[q] of
 * element elem[q] (the element ahead), with nodes N1, N2 in the element's
 * counter-clockwise order.  delta_d = (u_N2 - u_N1) when the edge is
 * stretched (|x_N2 - x_N1|^2 > |X_N2 - X_N1|^2), else 0.  G[2q + j], j = 0,
 * 1, is the energy release rate delta_d . (sigma n) / 2 of the path from the
 * edge's midpoint to the midpoint of the element's local edge k0 + 1 + j
 * (mod 3), k0 the point's own local edge: n the segment's unit normal with
 * n . (X_N2 - X_N1) > 0, sigma that edge's smoothed stress.  choice[q] is
 * the local edge of the chosen path or -1: paths with G above the element's
 * G_c qualify; of two, path p wins if G_p > gamma (G_p - G_q) (ratio mode:
 * G_p > gamma G_q), the larger G when both pass (the lower local edge on a
 * tie); G_c, gamma and its mode come from cem_set_material.  Host arrays:
 * edge, elem [n]; G [2n]; choice [n].  Errors: CEM_ERR_ARG (an edge that is
 * not an edge of its element), CEM_ERR_STATE (not a triangle mesh, or before
 * cem_set_material). */
cem_status cem_tri_eval_surface(cem_handle *h, int n, const int *edge, const int *elem,
                                double *G, int *choice);

/* Linear elastic material (E > 0, -1 < nu < 0.5, rho > 0), per-element
 * critical energy release rate G_c (gc_per_elem[nx*ny], FP32, or NULL for
 * gc_uniform), plane strain (1) or plane stress (0), the split ratio gamma
 * of the Q4 cracking conditions (Sec. 2.2) with gamma_mode
 * CEM_GAMMA_LITERAL (G_p > gamma (G_p - G_q)) or CEM_GAMMA_RATIO
 * (G_p > gamma G_q), and the tracking scope (Sec. 3): CEM_SCOPE_NBHD (a
 * proposal wins if its (G, -edge id) is the largest among proposals whose
 * elements share a node with its own), CEM_SCOPE_GLOBAL (one winner per
 * step) or CEM_SCOPE_TIPS (only crack fronts propose).  Computes lumped
 * masses, the time step, then applies the descriptor's pre-cracks.  Call
 * once, before cem_set_bc / cem_step.  Errors: CEM_ERR_ARG, CEM_ERR_STATE
 * (called twice), CEM_ERR_CAPACITY (pre-cracks exceed capacities). */
cem_status cem_set_material(cem_handle *h, double E, double nu, double rho,
                            const float *gc_per_elem, double gc_uniform,
                            int plane_strain, double gamma, int gamma_mode,
                            int mct_scope);

/* Adds a load.  CEM_TRACTION: items are boundary edge ids; each node of an
 * edge of length L receives L/2 * a0 along x (comp_mask bit 0) and/or y
 * (bit 1).  CEM_PRESSURE: boundary edge ids; pressure a0 pushes into the
 * material along the inward normal.  CEM_VELOCITY: node ids; the masked
 * velocity components are prescribed as law(t) * a0.  Time law:
 * CEM_LAW_CONST 1; CEM_LAW_RAMP t/t0 then 1 (Secs. 4.1, 4.3);
 * CEM_LAW_RAMP_EXP t/t0 then exp(-(t-t0)/tau) (Sec. 4.4).  All Neumann loads
 * share one law, all Dirichlet loads share one law.  Loads act on real
 * nodes only.  Errors: CEM_ERR_ARG (not a boundary edge, bad node, law
 * mismatch), CEM_ERR_STATE (after the first step). */
cem_status cem_set_bc(cem_handle *h, int kind, int n_items, const int *items,
                      int comp_mask, int law, double a0, double t0, double tau);

/* Which field cem_set_fields / cem_get_fields move.  Node fields are FP64
 * arrays over all nodes (real then phantom): x block then y block. */
typedef enum {
  CEM_FIELD_U = 0,       /* double[2 * n_nodes_total] */
  CEM_FIELD_V = 1,       /* double[2 * n_nodes_total] */
  CEM_FIELD_MASS = 2,    /* double[n_nodes_total] (get only) */
  CEM_FIELD_STATE = 3,   /* uint8[nx*ny]: 0 intact, 1 split, 2 inactive (get only) */
  CEM_FIELD_ENERGY = 4,  /* double[7 * n_energy]: step, t, KE, SE, W_ext, W_dir, U_d */
  CEM_FIELD_GC = 5,      /* float[nx*ny] (get only) */
  CEM_FIELD_SIGMA = 6,   /* double[3 * nx*ny]: element mean stress sxx[ne], syy[ne],
                            sxy[ne] (Pa; get only): an intact element averages over its
                            four edge points the stress its internal force uses there
                            (Eqs. 1-2 smoothing applied); a split element weights its
                            pieces' means by their areas; inactive elements 0 */
  CEM_FIELD_SIGMA1 = 7   /* double[nx*ny]: largest principal value of that stress,
                            (sxx+syy)/2 + sqrt(((sxx-syy)/2)^2 + sxy^2) (the stress
                            contours of Sec. 4; get only) */
} cem_field;

/* Sets initial u or v of all current nodes before the first step.
 * data is host memory (on_device = 0) or a device pointer (1); n_bytes must
 * equal the field size.  Errors: CEM_ERR_ARG, CEM_ERR_STATE. */
cem_status cem_set_fields(cem_handle *h, int which, const void *data,
                          long n_bytes, int on_device);

/* Advances n explicit steps on the handle's stream (CUDA-graph replays) and
 * synchronises once at the end to read the device status word.  Returns the
 * first device error: CEM_ERR_CAPACITY, CEM_ERR_NONFINITE; or CEM_ERR_STATE
 * before cem_set_material. */
cem_status cem_step(cem_handle *h, int n);

/* Pipelined stepping of a structured mesh handle: enqueues n steps like
 * cem_step (eight-step graphs where they fit).  With 1 <= n <= 32 every step
 * writes its status word into a 64-slot ring in mapped pinned host memory
 * (the last block of its split writes does); otherwise a one-warp kernel
 * copies the status word there after the call (no copy-engine operation
 * between graphs either way).  Then waits for the previous cem_step_async
 * call's steps to finish and returns that call's status, checking each of
 * its steps' words (the first call returns CEM_OK).  The
 * host's wait overlaps the steps just enqueued, so back-to-back calls keep
 * the GPU busy; each call's errors (CEM_ERR_NONFINITE, CEM_ERR_CAPACITY)
 * are reported by the call after it, or by cem_sync.  cem_step drains
 * pending asynchronous calls first.  CEM_ERR_STATE on a batch or triangle
 * handle. */
cem_status cem_step_async(cem_handle *h, int n);

/* Waits for every pending cem_step_async call of the handle and returns the
 * first error among them (CEM_OK if none or nothing is pending). */
cem_status cem_sync(cem_handle *h);

/* Copies a field into out (host, or device pointer when on_device = 1).
 * n_bytes must be at least the field size (see cem_get_counts). */
cem_status cem_get_fields(cem_handle *h, int which, void *out, long n_bytes,
                          int on_device);

typedef struct {
  long n_nodes;      /* real nodes */
  long n_phantoms;   /* phantom nodes */
  long n_elems;
  long n_active;     /* active elements */
  long n_cracked;    /* split elements (pre-cracks included) */
  long n_surface;    /* free-surface edge points */
  long n_tips;       /* surface points on a cut edge (crack fronts) */
  long n_energy;     /* energy records */
  long step;         /* steps taken */
  double dt;         /* time step (s) */
  double t;          /* step * dt */
  long kernel_launches; /* kernels this handle has enqueued (graph nodes included) */
  long last_proposals;  /* proposals evaluated in the last step */
  long last_winners;    /* splits made in the last step */
} cem_counts;

cem_status cem_get_counts(cem_handle *h, cem_counts *out);

/* A crack front: a surface edge point on a cut edge whose other element is
 * intact (the element "ahead").  Sorted by edge id. */
typedef struct {
  int edge_id;       /* edge id of the tip point */
  int ahead_elem;    /* intact element ahead of it */
  double x, y;       /* reference coordinates of the edge midpoint (m) */
  double G_last;     /* largest candidate G at the last evaluation (J/m^2) */
  int birth_step;    /* step at which the cut reached this edge (-1: pre-crack) */
  int parent;        /* the split element behind the tip */
} cem_tip;

cem_status cem_get_crack_tips(cem_handle *h, cem_tip *out, int cap, int *n_out);

/* One split element.  node[p][a] is the node used by piece p at local node
 * a (a real node id or a phantom id); Ap are the piece areas; ud is the
 * energy dissipated by this split (G_c * segment length; 0 for pre-cracks). */
typedef struct {
  int elem, ka, kb, step;
  int node[2][4];
  double Ap[2];
  double ud;
} cem_crack;

/* Split elements sorted by element id. */
cem_status cem_get_cracks(cem_handle *h, cem_crack *out, int cap, int *n_out);

/* One phantom node: its id, the real node it duplicates, the element and
 * local node that created it, and its users (element, piece, local node),
 * sorted by element; unused slots are -1. */
typedef struct {
  int id, owner, creator_elem, creator_local, n_users;
  int users[4][3];
} cem_phantom;

/* Phantoms in id order. */
cem_status cem_get_phantoms(cem_handle *h, cem_phantom *out, int cap, int *n_out);

/* Free-surface edge points sorted by edge id: edge, ahead element, tip flag. */
cem_status cem_get_surface(cem_handle *h, int *edge, int *ahead, int *is_tip,
                           int cap, int *n_out);

/* Profiling: advances n steps like cem_step but with direct kernel launches,
 * one after the other, bracketed by CUDA events on the handle's stream, and
 * returns device milliseconds in ms[9]: [0] all n steps (first event to
 * last), [1] piece forces (FP32: the pieces' evaluation timed on its own;
 * the step itself evaluates them inside the tile and phantom updates),
 * [2] tile update of real nodes, [3] phantom update, [4] surface
 * evaluation, [5] tracking selection, [6] energy records, [7] number of
 * kernels, [8] split writes. */
cem_status cem_profile_steps(cem_handle *h, int n, double *ms);

/* Testing hook for the tracking bookkeeping: runs the selection and split
 * (Sec. 3) on caller-given proposals (surface edge id, its ahead element,
 * chosen exit edge, G) without a mechanics step.  Errors: CEM_ERR_ARG when a
 * proposal is not a surface point of its element. */
cem_status cem_debug_apply_proposals(cem_handle *h, int n, const int *edge,
                                     const int *elem, const int *k,
                                     const double *G);

/* Batched stepping of many independent meshes (specimen sweeps): every
 * member advances by exactly the step defined above (Secs. 2-3); the batch
 * only changes how the work is launched.  One launch per kernel kind covers
 * all members (persistent grids walking lists of (member, tile or block)
 * items, one CUDA graph per step), so small meshes no longer pay one set of
 * launches each.
 *
 * cem_batch_create: members[n] are mesh handles with their material (and
 * loads) set, on one device, with the same precision, energy_every and
 * current step.  step_end[n] (host, may be NULL = no limit) is the step
 * count at which each member stops; cem_step(batch, k) advances every member
 * by k steps or up to its limit.  cuda_stream as in cem_mesh_desc.  While
 * in the batch a member cannot be stepped, loaded or given fields on its
 * own; its getters work as usual and read its state.  Members must outlive
 * the batch (destroy the batch first); destroying a member detaches it and
 * the batch then refuses to step.  The batch's own device memory (states
 * and work lists, a few KB per member) comes from member 0's allocator.
 * On a batch handle cem_get_counts returns sums over the members (step =
 * batch step, dt = t = 0); the other getters return CEM_ERR_STATE.
 * Errors: CEM_ERR_ARG (mismatched members), CEM_ERR_STATE (member without
 * material or already in a batch), CEM_ERR_CUDA.  cem_step on a batch also
 * returns the first member error, naming the member in the message. */
cem_status cem_batch_create(cem_handle *const *members, int n, const long *step_end,
                            void *cuda_stream, cem_handle **out);

/* Launch configuration of a batch: tile_rows (8 .. 64) is the height of the
 * FP32 node update's tiles (28 nodes wide, one warp each; the FP64 tiles are
 * fixed at 32 x 8), grid_main the persistent grid of the node update
 * (1 .. 64 x SMs).  Nodal results do not depend on it; in FP32 the energy
 * records group their partial sums by tile (last-bit differences).
 * Default 16, 3 x SMs. */
cem_status cem_batch_set_config(cem_handle *batch, int tile_rows, int grid_main);

/* Autotuner: times steps_per_candidate real steps (after one untimed step)
 * for each candidate configuration -- tile heights {16, 8, 32, 64} (FP32
 * only) x grids {1, 2, 3, 4} x SMs -- keeps the fastest and returns it.  The timed
 * steps advance the simulation like cem_step. */
cem_status cem_batch_autotune(cem_handle *batch, int steps_per_candidate, int *tile_rows,
                              int *grid_main);

/* Allocation-free energy check.  The paper has no counterpart: this is a
 * library convenience for callers that cannot allocate device memory, such
 * as a host application whose device memory is all handed to its own
 * fixed-size arena, or a monitor that samples energies while other streams
 * are busy and must not call cudaMalloc / cudaFree (cudaFree synchronises the
 * device).  It allocates nothing: no cudaMalloc, no cudaFree, no allocating
 * library routine.
 *
 * Computes, for one state of an uncracked nx * ny mesh (holes allowed), the
 * kinetic energy 1/2 sum m_N |v_N|^2 with row-sum lumped masses and the
 * ES-FEM strain energy (each active element owns A/4 of each of its four
 * edge points; an edge point shared with an active element uses the mean of
 * the two elements' strains), the same quantities as KE and SE of an energy
 * record of cem_step for a mesh without splits.  Only the grouping of the
 * partial sums differs, so the two agree to rounding.
 *
 * Arguments (all pointers are device memory of the calling thread's current
 * device; the caller owns them): elem_active uint8[nx*ny] (0 = hole) or NULL;
 * u and v double[2*(nx+1)*(ny+1)] (x block then y block, node id
 * j*(nx+1)+i); out double[2] receives KE then SE.  E, nu, rho, plane_strain
 * as in cem_set_material.  cuda_stream is a cudaStream_t (NULL = the legacy
 * default stream); the call only enqueues work, so read out after the stream
 * is synchronised.  err (host, may be NULL) receives a message of at most
 * err_len bytes on failure.
 *
 * Scratch and its limit: one (KE, SE) pair per node row in a fixed device
 * array of 2 * (CEM_NOALLOC_MAX_NY + 1) doubles (256 KiB + 16 B), which every
 * device that loads the library holds until the process exits.  Meshes with
 * ny > CEM_NOALLOC_MAX_NY are rejected with CEM_ERR_ARG.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress, with
 * the device current); make that first call before any stream capture.  A
 * cudaDeviceReset unloads the array: the next call finds its cached address
 * stale and looks it up again (so make that call outside a capture too).  All
 * calls on a device share the array: calls whose work overlaps on the GPU
 * (different streams or host threads without an order between them) race
 * and corrupt each other's results, so order them.  Nothing in the array
 * has to start at zero: each call writes every slot it reads.
 *
 * Errors: CEM_ERR_ARG (sizes, material, a missing pointer or one that is not
 * device memory of the current device), CEM_ERR_CUDA (no device, symbol
 * lookup or launch failure). */
#define CEM_NOALLOC_MAX_NY 16384
cem_status cem_state_energy_noalloc(int nx, int ny, double hx, double hy,
                                    const unsigned char *elem_active, double E,
                                    double nu, double rho, int plane_strain,
                                    const double *u, const double *v, double *out,
                                    void *cuda_stream, char *err, int err_len);

/* Fragments of the cracked body (Sec. 4.4 reports fragment counts, Table
 * 1).  A piece is an intact active element, or one side of a split element
 * (its node list: real nodes on that side, phantom copies of the others);
 * pieces that share a node, real or phantom, move together, and a fragment
 * is a connected set of pieces under that relation.  *n_fragments = their
 * number; piece_fragment (host, may be NULL; cap >= 2 * nx * ny entries)
 * receives the fragment of piece 2 e + p (p = 0 for an intact element, p =
 * side for a split one; -1 where there is no such piece), fragments numbered
 * in increasing order of their lowest piece.  Computed on the device by a
 * union-find over the nodes.  Errors: CEM_ERR_ARG (cap too small),
 * CEM_ERR_STATE (batch handle), CEM_ERR_CUDA. */
cem_status cem_get_fragments(cem_handle *h, int *n_fragments, int *piece_fragment, long cap);

/* Checkpoint and restart of a run (the paper has none: a library service,
 * so that a long explicit run can be stopped and resumed).  The state blob
 * holds the step counter and every quantity that carries over from one step
 * to the next: displacements and velocities of real and phantom nodes (the
 * current buffer), lumped masses and their inverses, boundary-work
 * accumulators, element states, the split-element table, the phantom table,
 * the surface / tip list, and the energy records.  The mesh, material and
 * loads are not in it: load into a handle built with the same descriptor,
 * material and loads.  A run of 2N steps and a run of N steps, saved,
 * loaded into a fresh handle and run N more steps end bit-identical.
 *
 * cem_state_size: *n_bytes = the blob size at the current step (it grows
 * with the splits).  cem_save_state: writes the blob into the caller's host
 * buffer blob of n_bytes (>= the size).  cem_load_state: replaces the
 * handle's state by the blob's (copied; the caller keeps the buffer).
 * Errors: CEM_ERR_ARG (buffer too small, not a blob, another mesh, precision
 * or time step), CEM_ERR_CAPACITY (the blob's phantoms, splits, list entries
 * or records exceed the handle's capacities), CEM_ERR_STATE (no material,
 * or a batch / batch member), CEM_ERR_CUDA. */
cem_status cem_state_size(cem_handle *h, long *n_bytes);
cem_status cem_save_state(cem_handle *h, void *blob, long n_bytes);
cem_status cem_load_state(cem_handle *h, const void *blob, long n_bytes);

/* Message of the last failure on h (or of the last failed create when h is
 * NULL).  Valid until the next call on h. */
const char *cem_last_error(const cem_handle *h);

/* Frees the device state and the handle. */
void cem_mesh_destroy(cem_handle *h);

#ifdef __cplusplus
}
#endif
#endif
